/*
 * eik.h -- C ABI of the GB300 block-based restarted narrow-band fast marching
 * solver (libeik.so).
 *
 * Problem (Sec. 1, Eq. (1.1)): |grad psi(x)| F(x) = 1 in the grid, psi = 0 on
 * the point sources, F >= 0 (F = 0 marks a barrier node that is never solved,
 * Sec. 3.3).  Discretisation (Sec. 2.1, Eqs. (2.1)-(2.2)): first-order Godunov
 * upwind differences on a node-centred uniform grid of spacing h, node (i,j,k)
 * at physical (i*h, j*h, k*h).  Method (Sec. 2.3-2.6, Alg. 6): the grid is cut
 * into blocks; each restart raises a global bound by a stride, marches every
 * active block's narrow band up to that bound (Alg. 4 with Algs. 2-3), and
 * exchanges ghost layers between neighbouring blocks with a min-merge
 * (Alg. 5), until no block is active.
 *
 * Conventions shared by every entry point:
 *  - Arrays of grid values are nx*ny*nz elements, x fastest:
 *    idx = (k*ny + j)*nx + i.  Element type follows the context precision:
 *    float for EIK_FP32, double for EIK_FP64.
 *  - "on_device" flags say whether a pointer is device memory (non-zero) or
 *    host memory (zero).  The caller owns every buffer it passes; the library
 *    copies what it keeps and never frees caller memory.
 *  - The library owns all device memory it allocates; eik_destroy frees it.
 *  - Every call is validated.  Errors are return codes, never exceptions or
 *    aborts; eik_last_error() describes the most recent failure.
 *  - Work is issued on the stream given to eik_create (NULL = the legacy
 *    default stream).  eik_solve and eik_result return after that work has
 *    finished; eik_solve_async returns after queueing it.
 *  - One context is used by one host thread at a time.
 */
#ifndef EIK_H
#define EIK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eik_ctx eik_ctx;

typedef enum {
    EIK_OK = 0,
    EIK_EINVAL = 1,    /* invalid argument (dims, h, F, sources, parameters) */
    EIK_ENOMEM = 2,    /* a device or host allocation failed */
    EIK_ECUDA = 3,     /* a CUDA call failed (eik_last_error has the CUDA message) */
    EIK_ETIMEOUT = 4,  /* the restart cap was reached or a device wait ran out of iterations */
    EIK_ESTATE = 5,    /* call out of order: e.g. eik_solve before any source */
    EIK_ENOTSUP = 6    /* valid request this build does not support */
} eik_status;

typedef enum { EIK_FP32 = 0, EIK_FP64 = 1 } eik_precision;

/*
 * eik_create -- build a solver context for one grid and speed function.
 *   out          receives the context (set to NULL on failure).
 *   dims         nx, ny, nz >= 1 (grid nodes per axis); nx*ny*nz < 2^31.
 *   h            grid spacing, finite and > 0.
 *   F            nx*ny*nz speeds (float for EIK_FP32, double for EIK_FP64),
 *                each finite and >= 0.  Copied; the caller keeps its buffer.
 *   F_on_device  non-zero if F is device memory.
 *   precision    EIK_FP32: psi and F stored and updated in single precision
 *                (the upwind root falls back to double, Alg. 3, when its
 *                discriminant is small relative to k*(h/F)^2 or (h/F)^2
 *                underflows); EIK_FP64: everything in double.
 *   stream       a cudaStream_t, or NULL.
 * Errors: EIK_EINVAL (bad dims/h, F < 0, NaN or inf), EIK_ENOMEM, EIK_ECUDA.
 */
eik_status eik_create(eik_ctx **out, const int32_t dims[3], double h, const void *F,
                      int F_on_device, eik_precision precision, void *stream);

/*
 * eik_set_speed -- replace the speed function of an existing context (same
 * grid, h and precision); F as in eik_create.  Sources are kept.
 * Errors: EIK_EINVAL (NULL F, F < 0, NaN or inf; the old speeds are then
 * undefined until a successful call), EIK_ESTATE (a solve is in flight).
 */
eik_status eik_set_speed(eik_ctx *ctx, const void *F, int F_on_device);

/*
 * eik_set_speed_async -- eik_set_speed without waiting: the copy of F and its
 * re-layout are queued on the context's stream and the call returns.  F must
 * stay valid (and unchanged) until eik_sync or the next solve on ctx; host F
 * should be pinned, or the copy is not asynchronous.  The validation of F is
 * reported by the next eik_solve_async / eik_solve_ex / eik_solve (which then
 * do not run) or eik_sync, as EIK_EINVAL.  A later eik_set_speed(_async)
 * supersedes it.  Errors here: EIK_EINVAL (NULL F), EIK_ESTATE (solve in flight).
 */
eik_status eik_set_speed_async(eik_ctx *ctx, const void *F, int F_on_device);

/*
 * eik_source_nodes -- the fixed nodes (Alg. 1) a solve of this grid, speed
 * function and sources starts from, computed on the host with the same code
 * and the same rounding of h/F as eik_solve (no device needed).
 *   F, precision  as in eik_create; F must be host memory here.
 *   idx_out       linear indices (k*ny + j)*nx + i (nullable), ordered by brick
 *                 and node within the brick; psi0_out their psi0 (nullable).
 *   cap           capacity of the outputs; *n_out gets the count even when
 *                 it exceeds cap (then EIK_EINVAL and nothing is written).
 * Errors: EIK_EINVAL (bad dims, h, precision, F, or a source outside the grid).
 */
eik_status eik_source_nodes(const int32_t dims[3], double h, const void *F, eik_precision precision,
                            int32_t nsrc, const double *xyz, int64_t *idx_out, double *psi0_out, int64_t cap,
                            int64_t *n_out);

/*
 * eik_add_sources -- add point sources (Gamma of Eq. (1.1)).
 *   xyz  n*3 physical coordinates (x, y, z), origin at node 0, each within
 *        [0, (n_axis - 1)*h].  The nodes of the grid cell containing a source
 *        (one node if it lies on a node, 2/4 on an edge/face, 8 inside) become
 *        fixed with psi0 = distance / F there (Alg. 1, "on or adjacent to
 *        Gamma"); a node reached by several sources keeps the smallest psi0.
 * Errors: EIK_EINVAL (n < 0, a coordinate outside the grid box or not finite).
 */
eik_status eik_add_sources(eik_ctx *ctx, int32_t n, const double *xyz);

/* eik_clear_sources -- forget every source added so far. */
eik_status eik_clear_sources(eik_ctx *ctx);

/* Schedules of the restart bound (Alg. 6: bound <- min(bound + stride, width)). */
typedef enum {
    EIK_SCHED_FIXED = 0,   /* every restart advances the bound by `stride` with block edge `block_dim` */
    EIK_SCHED_LEARNED = 1, /* after restart k the schedule network (eik_set_schedule) picks the stride
                              and block edge of restart k+2 (one restart ahead, so that waiting warps can
                              start the next restart early); `stride` and `block_dim` set restarts 1-2 */
    EIK_SCHED_RANDOM = 2   /* each restart's stride and block edge drawn from the action table with
                              `seed` (to record training data), also one restart ahead */
} eik_schedule;

typedef struct {
    double stride;          /* bound increment in psi units (> 0; +inf = the naive block method); 0 selects
                               the learned schedule (as schedule = EIK_SCHED_LEARNED, with 2h for restarts
                               1-2) */
    int32_t block_dim;      /* block edge in nodes: 8 (one warp per block), 16 (one CTA per block of
                               2x2x2 bricks) or 32 (one CTA of 1024 threads per 32^3 block, its tile in
                               shared memory; FP32 and the fixed schedule only, no restart log: else
                               EIK_ENOTSUP; the context allocates the 32^3 layout on its first such solve:
                               two copies of psi and h/F, about 3.1x the grid's FP32 bytes); 0 = picked: by the
                               network under the learned schedule (8 for restarts 1-2), else the edge
                               eik_autotune chose for the context, else 8 */
    int32_t schedule;       /* eik_schedule */
    double window;          /* acceptance window factor omega: each march round accepts every band
                               point within omega * h / F_max(block) of the band minimum
                               (0 = default 2; 1/sqrt(3) is the smallest increment of Alg. 3) */
    double fallback_tau;    /* FP32 mode: fall back to double when D < tau * k * (h/F)^2 (0 = default 1/8) */
    int64_t max_restarts;   /* restart cap (0 = default 1 << 24); reaching it returns EIK_ETIMEOUT */
    int32_t log_restarts;   /* non-zero: record per-restart statistics (eik_restart_log) */
    int32_t seed;           /* EIK_SCHED_RANDOM seed */
    void *loop_events[2];   /* optional cudaEvent_t pair the library records on its stream right
                               before and right after the restart-loop kernel (NULL: none) */
    double switch_margin;   /* EIK_SCHED_LEARNED: keep the current action unless another one's predicted
                               log cost rate is lower by more than this (default 0.02) */
    double width;           /* width_band of Alg. 6 (0 = +inf: the full solve).  A finite width caps the
                               bound: psi is exact at every node with psi <= width; a node above it keeps a
                               tentative value >= its exact one, or +inf */
    int64_t wait_polls;     /* polls (of 32 ns - 4 us naps) before a device-side wait gives up and the solve
                               ends with EIK_ETIMEOUT (0 = default 2^22, seconds).  Small values let a
                               test make the waits run out; the context stays usable */
} eik_params;

/* Per-solve statistics, filled by eik_solve / eik_wait. */
typedef struct {
    int64_t restarts;       /* nr: iterations of the restart loop of Alg. 6 */
    int64_t marches;        /* block marches (active or flagged blocks, summed over restarts), in 8^3
                               bricks: a 16^3 block counts 8, a 32^3 block 64 */
    int64_t accepted;       /* band points accepted (heap pops in Alg. 4), refreshes included */
    int64_t solves;         /* upwind solves (Alg. 3 calls) */
    int64_t updates;        /* solves that lowered psi (Alg. 2 accepted updates) */
    int64_t fallbacks;      /* FP32 roots recomputed in double */
    int64_t rounds;         /* acceptance rounds over all marches */
    double device_ms;       /* device time of the restart loop (%globaltimer) */
    double final_bound;     /* bound of the last restart */
    int32_t status;         /* eik_status of the device run */
    int32_t block_dim;      /* block edge used */
} eik_stats;

/* One record per restart when eik_params.log_restarts is set. */
typedef struct {
    int32_t k;              /* restart index, 1-based */
    int32_t active;         /* 8^3 bricks marched in this restart */
    int64_t band;           /* band points left (pending) at the end of the restart */
    int64_t accepted;       /* points accepted in this restart */
    int64_t solves;         /* upwind solves in this restart */
    double bound;           /* bound_band of this restart */
    double stride;          /* stride that produced this bound */
    double rmin;            /* min h/F over the marched blocks */
    double rmax;            /* max h/F over the marched blocks */
    double ms;              /* device time of the restart */
    int32_t block_dim;      /* block edge of this restart */
    int32_t next_action;    /* action chosen after this restart, for the restart after the next one
                               (-1: fixed schedule) */
    float features[10];     /* the schedule network's input after this restart */
} eik_restart_rec;

/* eik_params_default -- fill *p with the defaults above and stride = 2h-equivalent 0 (caller sets stride). */
void eik_params_default(eik_params *p);

/*
 * eik_solve -- run the method (Alg. 6: restarts that raise bound_band by the
 * stride, march every active block up to it with Algs. 2-4 and exchange ghost
 * layers with Alg. 5, until no block is active) and wait for it.
 *   stride     > 0 (may be +inf: the naive block method of Sec. 3.4): every
 *              restart raises the bound by it.  0: the learned schedule picks
 *              the stride (and, with block_dim 0, the block edge) of every
 *              restart from restart 3 on; restarts 1-2 take 2h.  The
 *              context's network weights are used (every context starts
 *              with the shipped ones; eik_set_schedule replaces them).
 *   block_dim  8, 16 or 32 (see eik_params.block_dim); 0 = picked (the
 *              network under the learned schedule, else the edge
 *              eik_autotune chose for the context, else 8).
 *   stats      nullable.
 * The result does not depend on the stride, the schedule or the block edge,
 * bit for bit (the root of Alg. 3 is evaluated as a monotone function of the
 * neighbour values, so every order of work reaches the same fixed point).
 * Returns EIK_ESTATE if no source was added or stride 0 is asked for after
 * the weights were unloaded, EIK_EINVAL for a negative or NaN stride or
 * another block edge, EIK_ETIMEOUT if the restart cap or a device wait limit
 * was hit.
 */
eik_status eik_solve(eik_ctx *ctx, double stride, int32_t block_dim, eik_stats *stats);

/* eik_solve_ex -- eik_solve with every parameter; waits for completion. */
eik_status eik_solve_ex(eik_ctx *ctx, const eik_params *params, eik_stats *stats);

/* eik_solve_async -- queue the solve on the context's stream and return;
 * eik_wait then synchronises and reports. */
eik_status eik_solve_async(eik_ctx *ctx, const eik_params *params);
eik_status eik_wait(eik_ctx *ctx, eik_stats *stats);

/*
 * eik_autotune -- pick the fixed stride and block edge of this context's
 * grid by timing solves on the device (the paper's Secs. 3.4-3.6 study the
 * same two parameters).  Candidates: stride c*h with c in {1, 1.5, 2, 2.5, 3,
 * 4} and block edge 8 or 16.  Successive halving: time every candidate once,
 * keep the best third, time the survivors twice as often, until one is left
 * (at most `rounds` rounds; 0 = no limit).  Later solves with block_dim 0 and
 * a fixed stride use the chosen edge.  stride_out, block_out, best_ms (its
 * median device time) are nullable.  The context's psi afterwards is that of
 * the last timed solve.  Errors: EIK_ESTATE (no source, or a solve in flight).
 */
eik_status eik_autotune(eik_ctx *ctx, int32_t rounds, double *stride_out, int32_t *block_out, double *best_ms);

/*
 * eik_restart_log -- copy up to cap per-restart records of the last solve
 * (made with log_restarts set) into out (host memory); *n gets the count.
 */
eik_status eik_restart_log(eik_ctx *ctx, eik_restart_rec *out, int64_t cap, int64_t *n);

/*
 * eik_result -- copy psi of the last solve into psi_out (nx*ny*nz, context
 * precision, x fastest).  This is psi_i,j,k of Sec. 2.1 on every node of the
 * grid at the end of Alg. 6, gathered from the interiors Omega^ib of the
 * blocks.  Unreachable nodes and barrier nodes (F = 0, Sec. 3.3) are +inf.
 * Errors: EIK_ESTATE before the first successful solve.
 */
eik_status eik_result(eik_ctx *ctx, void *psi_out, int out_on_device);

/*
 * eik_result_async -- eik_result without waiting for the copy: psi is put in
 * grid order on the device (the call waits for that kernel, a few ms at
 * 1024^3, so that a solve queued next on another context's stream starts
 * after it) and, for a host psi_out, the copy to it is queued on the context's
 * stream.  psi_out holds the result after eik_sync(ctx) or any later blocking
 * call on ctx; host psi_out should be pinned.  Two contexts used in turn
 * overlap one's host copies with the other's solve.  Errors as eik_result.
 */
eik_status eik_result_async(eik_ctx *ctx, void *psi_out, int out_on_device);

/*
 * eik_sync -- wait for everything queued on the context's stream (speed
 * uploads, result copies, a solve in flight; that solve's statistics still
 * come from eik_wait).  Returns EIK_EINVAL if an eik_set_speed_async found a
 * bad F.
 */
eik_status eik_sync(eik_ctx *ctx);

/* eik_destroy -- wait for the work queued on the context's stream, then free the context and
 * everything it allocated: the block data of Sec. 2.3 (per-block psi, h/F, ghost layers and
 * flags), the work lists and the control block (NULL is a no-op). */
void eik_destroy(eik_ctx *ctx);

/* eik_last_error -- message of the last failure on ctx (or of the last failed
 * eik_create when ctx is NULL).  Valid until the next call on ctx.  (Error reporting has no
 * counterpart in the paper.) */
const char *eik_last_error(const eik_ctx *ctx);

/* eik_version -- library version string. */
const char *eik_version(void);

/*
 * One grid sharded across GPUs.  The blocks of Sec. 2.3 are cut into slabs of
 * whole 8^3-brick planes along z, one slab per GPU.  Each GPU holds its slab
 * plus one ghost brick plane beyond each cut (a context over that extended
 * part of the grid: node planes [z_lo, z_hi) of the full grid).  The restarts of Alg. 6 run in lockstep:
 * every GPU marches its own active bricks up to the same bound (bound_k is
 * preset by the stride, so it needs no exchange), then each cut's face layers
 * go to the GPU across it and are merged into its ghost plane (Alg. 5 across
 * the cut; a lowered face puts the adjacent brick on the next restart's list),
 * and the solve ends when no GPU has a brick listed.  The result is the same,
 * bit for bit, as one GPU's: the update is monotone, so the order of work does
 * not change the fixed point.  Every call waits for its work.
 *
 * eik_slab_set      ctx's grid is node planes [zoff, zoff + nz) of a grid of
 *                   nz_all planes (zoff a multiple of 8); mark its brick planes
 *                   [own_bz0, own_bz1) as this GPU's (0 <= own_bz0 < own_bz1 <=
 *                   ceil(nz/8)); the planes outside are ghosts, never marched
 *                   here.  Call it before eik_add_sources: the sources are then
 *                   given in the whole grid's coordinates (z in [0, (nz_all-1)h]),
 *                   and every part computes psi0 at its fixed nodes exactly as
 *                   one grid would.
 * eik_slab_begin    Alg. 1 and the work list of restart 1 (sources as added
 *                   with eik_add_sources, possibly none on this GPU), fixed
 *                   stride (finite, > 0), 8^3 blocks.
 * eik_slab_restart  one restart on this GPU; *pending (nullable) = bricks on
 *                   the next restart's list so far.
 * eik_slab_export   side 0: the z = 0 face layer of plane own_bz0 (for the GPU
 *                   below); side 1: the z = 7 face layer of plane own_bz1 - 1
 *                   (for the GPU above); into buf, DEVICE memory of
 *                   eik_slab_face_bytes(ctx) bytes owned by the caller.
 * eik_slab_import   the record the GPU across side exported (side 0: below,
 *                   into ghost plane own_bz0 - 1; side 1: above, into plane
 *                   own_bz1), DEVICE memory; *pending as above, imports counted.
 * eik_slab_end      finish (the psi of the own planes is then read with
 *                   eik_result, whose ghost planes hold no meaningful values).
 * Errors: EIK_EINVAL (planes, side, buffers, stride), EIK_ESTATE (order of
 * calls), EIK_ETIMEOUT (a device wait limit or the restart cap), EIK_ECUDA.
 */
int64_t eik_slab_face_bytes(const eik_ctx *ctx);
eik_status eik_slab_set(eik_ctx *ctx, int32_t own_bz0, int32_t own_bz1, int32_t zoff, int32_t nz_all);
eik_status eik_slab_begin(eik_ctx *ctx, double stride);
eik_status eik_slab_restart(eik_ctx *ctx, int64_t *pending);
eik_status eik_slab_export(eik_ctx *ctx, int32_t side, void *buf);
eik_status eik_slab_import(eik_ctx *ctx, int32_t side, const void *buf, int64_t *pending);
eik_status eik_slab_end(eik_ctx *ctx, eik_stats *stats);

/*
 * Restart-schedule network (no counterpart in the paper; the paper fixes the
 * stride).  A multilayer perceptron EIK_SCHED_INPUTS -> EIK_SCHED_HIDDEN (tanh)
 * -> EIK_SCHED_HIDDEN (tanh) -> EIK_SCHED_ACTIONS maps the front statistics of
 * restart k (eik_restart_rec.features) to a predicted log cost rate (device
 * milliseconds per unit of bound advance) for each action of the table
 * eik_sched_actions; the learned schedule takes the lowest.  Parameters are
 * EIK_SCHED_PARAMS floats: W1 (hidden x inputs, row-major), b1, W2, b2, W3, b3.
 * Changing the schedule changes which restart does which work, not psi.
 */
#define EIK_SCHED_INPUTS 10
#define EIK_SCHED_HIDDEN 32
#define EIK_SCHED_ACTIONS 12
#define EIK_SCHED_PARAMS (EIK_SCHED_HIDDEN * EIK_SCHED_INPUTS + EIK_SCHED_HIDDEN + \
                          EIK_SCHED_HIDDEN * EIK_SCHED_HIDDEN + EIK_SCHED_HIDDEN + \
                          EIK_SCHED_ACTIONS * EIK_SCHED_HIDDEN + EIK_SCHED_ACTIONS)

/* eik_sched_actions -- the action table: stride in units of h and block edge of each action (host). */
eik_status eik_sched_actions(double *stride_h, int32_t *block_dim, int32_t cap, int32_t *n);

/* eik_set_schedule -- load network weights (host, n = EIK_SCHED_PARAMS finite floats) into the
 * context for EIK_SCHED_LEARNED; w = NULL unloads them.  A new context holds the weights shipped
 * with the library (trained by the project on its own per-restart timings). */
eik_status eik_set_schedule(eik_ctx *ctx, const float *w, int32_t n);

/* eik_mlp_forward -- Y[B][ACTIONS] = network(X[B][INPUTS]); all DEVICE pointers; async on stream. */
eik_status eik_mlp_forward(const float *w, const float *X, int32_t B, float *Y, void *stream);

/* eik_mlp_grad -- loss = mean_s (Y[s][act[s]] - tgt[s])^2 and its gradient grad[PARAMS] with respect
 * to w; DEVICE pointers; work holds eik_mlp_work_floats(B) floats owned by the caller.  The sum over
 * samples runs in a fixed order, so the result is deterministic. */
eik_status eik_mlp_grad(const float *w, const float *X, const int32_t *act, const float *tgt, int32_t B,
                        float *grad, float *loss, float *work, void *stream);
int32_t eik_mlp_work_floats(int32_t B);

/* eik_mlp_adam -- one Adam step (Kingma and Ba, 2015) on n parameters, step number t >= 1; DEVICE. */
eik_status eik_mlp_adam(float *w, const float *grad, float *m, float *v, int32_t n, float lr, float b1,
                        float b2, float eps, int32_t t, void *stream);

/* eik_mlp_last_error -- message of the calling thread's last failed eik_mlp_* call. */
const char *eik_mlp_last_error(void);

/*
 * Batched solves -- no counterpart in the paper, which solves one grid at a
 * time.  Many independent grids, each with its own size, spacing, speed and
 * sources, are solved by one cooperative persistent launch: each restart
 * hands out one work queue holding the active blocks of every grid, all grids
 * share one grid barrier per restart, and grid s runs Alg. 6 with its own
 * block edge and stride (bound of restart k = k * stride_s).  Each grid gets
 * the solution eik_solve gives it (the schedule changes which restart does
 * which work, not the discrete solution).
 */
typedef struct eik_batch eik_batch;

typedef struct {
    int32_t dims[3];        /* nx, ny, nz >= 1; nx*ny*nz < 2^31 */
    double h;               /* grid spacing, finite and > 0 */
    const void *F;          /* nx*ny*nz speeds in the batch precision, x fastest, finite and >= 0; copied */
    int32_t F_on_device;    /* non-zero: F is device memory */
    int32_t nsrc;           /* >= 1 point sources */
    const double *xyz;      /* nsrc*3 physical coordinates in host memory, as in eik_add_sources */
} eik_batch_item;

typedef struct {
    int32_t block_dim;      /* block edge of the grid: 8 or 16 */
    double stride;          /* bound increment of the grid: finite and > 0 */
} eik_batch_tile;

typedef struct {
    int32_t ctas_per_sm;    /* CTAs per SM of the launch: 0 = the autotuned value, else the most that fit */
    double window;          /* as eik_params.window (0 = 2) */
    double fallback_tau;    /* as eik_params.fallback_tau (0 = 1/8) */
    int64_t max_restarts;   /* restart cap of the launch (0 = 1 << 24) */
    void *loop_events[2];   /* optional cudaEvent_t pair recorded right before and after the launch */
} eik_batch_params;

typedef struct {
    int64_t restarts;       /* restarts of the launch: the most any grid needed */
    int64_t marches;        /* block marches, summed over grids (a 16^3 block counts 8) */
    int64_t accepted;       /* band points accepted, summed over grids */
    int64_t solves;         /* upwind solves (Alg. 3), summed over grids */
    int64_t updates;        /* solves that lowered psi */
    int64_t fallbacks;      /* FP32 roots recomputed in double */
    int64_t rounds;         /* acceptance rounds */
    double device_ms;       /* device time of the launch (%globaltimer) */
    int32_t status;         /* eik_status of the device run */
    int32_t ctas;           /* CTAs of the launch */
} eik_batch_stats;

typedef struct {
    int32_t restarts;       /* last restart in which a block of this grid marched */
    int32_t block_dim;      /* block edge used */
    double stride;          /* stride used */
    double done_ms;         /* device time from the start of the launch to the end of that restart:
                               the grid's latency inside the batch */
    double rmin;            /* smallest h/F over the grid (the autotuner scales strides by it) */
    int64_t nbricks;        /* 8^3 bricks of the grid */
} eik_batch_solve_info;

/*
 * eik_batch_create -- lay out n grids (items) for batched solves.
 *   Speeds are copied into the batch; sources are set up once (Alg. 1).
 *   precision and stream as in eik_create.
 * Errors: EIK_EINVAL (an item's dims, h, F, sources; the message names the
 * item), EIK_ENOMEM, EIK_ECUDA, EIK_ENOTSUP (no cooperative launch).
 */
eik_status eik_batch_create(eik_batch **out, int32_t n, const eik_batch_item *items, eik_precision precision,
                            void *stream);

/* eik_batch_params_default -- defaults above. */
void eik_batch_params_default(eik_batch_params *p);

/*
 * eik_batch_solve -- solve every grid of the batch in one launch and wait.
 *   tiles   n tiles (host), or NULL: the autotuned tiles if eik_batch_autotune
 *           ran, else block edge 8 and stride 2h for every grid.
 *   params  nullable (defaults).   stats  nullable.
 * Errors: EIK_EINVAL (a bad tile or parameter), EIK_ETIMEOUT (restart cap or a
 * device wait limit), EIK_ESTATE (a solve in flight).
 */
eik_status eik_batch_solve(eik_batch *b, const eik_batch_tile *tiles, const eik_batch_params *params,
                           eik_batch_stats *stats);

/* eik_batch_solve_async / eik_batch_wait -- the same, split into queueing and waiting. */
eik_status eik_batch_solve_async(eik_batch *b, const eik_batch_tile *tiles, const eik_batch_params *params);
eik_status eik_batch_wait(eik_batch *b, eik_batch_stats *stats);

/* eik_batch_info -- per-grid record of the last solve into out[0..n-1] (host, cap >= n). */
eik_status eik_batch_info(eik_batch *b, eik_batch_solve_info *out, int32_t cap);

/* eik_batch_result -- psi of grid i (as eik_result: nx*ny*nz, batch precision, x fastest). */
eik_status eik_batch_result(eik_batch *b, int32_t i, void *psi_out, int out_on_device);

/*
 * eik_batch_autotune -- pick the tiles and CTAs per SM of this batch by timing
 * it on the device (each run is a full eik_batch_solve).  Candidates: stride of
 * grid s = c * h_s with c in {1.25, 1.5, 1.75, 2, 2.5, 3, 4}, or f * edge_s * rmin_s with
 * f in {0.5, 0.75, 1, 1.5, 2} (rmin_s = min h/F), block edge 16 for the grids
 * with at least m bricks, m in {never, 2048, 512, 0}, and every CTAs-per-SM
 * count that fits.  Search:
 * successive halving -- time every candidate once, keep the best third, time
 * the survivors twice as often, and so on until one is left (at most `rounds`
 * rounds; 0 = no limit).  A second stage then tiles grid by grid: the grids
 * that finish last under the winner (done_ms at or above the 50/75/90 %
 * quantile) get a stride 1.25, 1.5 or 2 times longer, or those that finish
 * first (at or below the 25/50/75 % quantile) one 0.5 or 0.75 times as long,
 * and the same halving picks among these fifteen and the winner.  The result
 * is kept in the batch for later solves
 * given tiles = NULL and ctas_per_sm = 0, and returned in tiles_out (n tiles,
 * nullable), ctas_per_sm (nullable) and best_ms (its median device time,
 * nullable).  The batch's psi afterwards is that of the last timed run.
 */
eik_status eik_batch_autotune(eik_batch *b, int32_t rounds, eik_batch_tile *tiles_out, int32_t *ctas_per_sm,
                              double *best_ms);

/* eik_batch_size -- number of grids, total 8^3 bricks, most CTAs per SM the launch can use (all nullable). */
eik_status eik_batch_size(const eik_batch *b, int32_t *n, int64_t *nbricks, int32_t *max_ctas_per_sm);

/* eik_batch_destroy -- free the batch (NULL is a no-op). */
void eik_batch_destroy(eik_batch *b);

/* eik_batch_last_error -- message of the last failure on b (or of the calling thread's last failed
 * eik_batch_create when b is NULL). */
const char *eik_batch_last_error(const eik_batch *b);

/*
 * eik_solve_noalloc -- one complete solve that allocates no device memory.
 *
 * No counterpart in the paper: this is a deployment entry point.  It serves
 * callers that cannot call cudaMalloc at solve time -- code that lives under
 * a memory pool or caching allocator it does not own (a cudaMalloc there
 * would take memory behind the allocator's back, or fail once the pool has
 * reserved the device), and embedders that must keep the process's device
 * footprint fixed.  All working memory of the solve lives in one fixed device
 * array inside the library (EIK_NOALLOC_SCRATCH_BYTES, 64 MiB), which every
 * GPU that loads the library holds until the process exits.
 *
 *   dims, h   grid as in eik_create; the grid's 8x8x8 bricks,
 *             ceil(nx/8)*ceil(ny/8)*ceil(nz/8), must not exceed
 *             EIK_NOALLOC_MAX_BRICKS (e.g. 160^3 or 128x128x256 fit).
 *   F         nx*ny*nz float speeds in DEVICE memory (x fastest), finite, >= 0.
 *   nsrc, xyz 1..EIK_NOALLOC_MAX_SOURCES point sources, host memory, as in
 *             eik_add_sources.
 *   params    nullable (defaults); checked as eik_solve_ex checks them, and
 *             stride must be > 0: fixed schedule and 8^3 blocks only
 *             (EIK_ENOTSUP otherwise, and for log_restarts, whose records
 *             would need memory); wait_polls and loop_events are honoured.
 *   psi_out   nx*ny*nz floats in DEVICE memory: the solution (FP32 mode only).
 *   stats     nullable.
 *   stream    cudaStream_t or NULL.  The call returns after the solve finished
 *             (it waits for the stream twice: once to read the speed check
 *             and the h/F of the source nodes, once at the end).
 * Errors: EIK_EINVAL for a grid above the limit (with a message saying so),
 * bad arguments or bad F; EIK_ETIMEOUT when the restart cap or a device wait
 * limit ends the solve (the next call is not affected);
 * eik_noalloc_last_error() describes the failure.
 *
 * The array's device address is looked up on the first call made with a
 * given device current: make that first call before any stream capture.
 * Every call shares the array and leaves its contents behind; each call
 * clears what must start empty.  Calls that overlap on the GPU (from two host
 * threads, or on two streams) race on the array and must not be issued.
 */
#define EIK_NOALLOC_SCRATCH_BYTES (64u << 20)
#define EIK_NOALLOC_MAX_BRICKS 8192
#define EIK_NOALLOC_MAX_SOURCES 64
eik_status eik_solve_noalloc(const int32_t dims[3], double h, const float *F, int32_t nsrc, const double *xyz,
                             const eik_params *params, float *psi_out, eik_stats *stats, void *stream);

/* eik_noalloc_last_error -- message of the calling thread's last failed eik_solve_noalloc. */
const char *eik_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
