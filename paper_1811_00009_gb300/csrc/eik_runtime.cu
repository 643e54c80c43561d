// Host runtime of libeik: the C ABI declared in include/eik.h.
//
// A context owns the device copy of h/F in brick layout, the two psi copies of
// every brick, the work lists and the control block of the restart loop.  A
// solve (Alg. 6) is: reset the per-brick state, set up the fixed nodes of the
// point sources (Alg. 1), run the cooperative restart-loop kernel, restore h/F
// at the fixed nodes.  Everything runs on the context's stream.
#include "eik.h"
#include "eik_host.h"
#include "eik_internal.cuh"
#include "eik_mlp.cuh"

#include "eik_sched_weights.inc"   // kSchedDefault: the shipped schedule-network weights (written by build.py)

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace eikg {
template <typename T>
cudaError_t launch_layout_speed(const T*, T*, int, int, int, int, int, int64_t, double, int*, int, cudaStream_t);
template <typename T>
cudaError_t launch_init_sources(int, const int32_t*, const int32_t*, const double*, int, const int32_t*, int,
                                const int32_t*, int, const int32_t*, T*, unsigned long long*, unsigned long long*,
                                int32_t*, int32_t*, T*, T*, int32_t*, int32_t*, cudaStream_t);
template <typename T>
cudaError_t launch_restore_r(int, const int32_t*, const int32_t*, const T*, T*, cudaStream_t);
template <typename T>
cudaError_t launch_gather_r(int, const int32_t*, const int32_t*, const T*, double*, cudaStream_t);
template <typename T>
cudaError_t launch_result(const T*, const unsigned long long*, T*, int, int, int, int, int, int, cudaStream_t);
template <typename T>
cudaError_t launch_slab_export(const T*, const unsigned long long*, const unsigned long long*, int, int, int, int, void*,
                               cudaStream_t);
template <typename T>
cudaError_t launch_slab_import(T*, unsigned long long*, unsigned long long*, int, int, int, int, const void*, int,
                               int32_t*, int64_t, Ctrl*, int32_t*, cudaStream_t);
int block32_edge_values();
cudaError_t block32_occupancy(int* per_sm);
cudaError_t block32_layout(const float*, int, int, int, float*, int, int, int64_t, cudaStream_t);
cudaError_t block32_init(int, const int32_t*, const int32_t*, const double*, int, const int32_t*, int, const int32_t*,
                         float*, unsigned*, unsigned long long*, int32_t*, float*, float*, int32_t*, cudaStream_t);
cudaError_t block32_restore(int, const int32_t*, const int32_t*, const float*, float*, cudaStream_t);
cudaError_t block32_result(const float*, const unsigned long long*, float*, int, int, int, int, int, cudaStream_t);
cudaError_t block32_loop(int, int, int, int64_t, float*, unsigned*, unsigned long long*, const float*, int32_t*,
                         int32_t*, int32_t*, Ctrl*, float, float, double, int64_t, long long, int, cudaStream_t);
template <typename T>
size_t loop_smem_bytes();
template <typename T>
cudaError_t loop_occupancy(int*);
template <typename T>
cudaError_t launch_restart_loop(const LoopParams<T>&, int, cudaStream_t);
}  // namespace eikg

using eikg::kBrick;
using eikg::kSlot;

struct eik_ctx {
    int nx = 0, ny = 0, nz = 0;
    double h = 0;
    eik_precision prec = EIK_FP32;
    cudaStream_t stream = nullptr;
    int BX = 0, BY = 0, BZ = 0;
    int64_t nbricks = 0;
    size_t esz = 4;
    void* rr = nullptr;
    void* slot = nullptr;
    unsigned long long* ups = nullptr;
    unsigned long long* stamp = nullptr;
    int32_t* queued = nullptr;     // kRing x nbricks (ring slots)
    int32_t* lists = nullptr;      // kRing x nbricks: the brick work lists by ring slot
    int32_t* done = nullptr;       // per brick
    int GX = 0, GY = 0, GZ = 0;
    int64_t ngroups = 0;
    int32_t* qgroup = nullptr;     // kRing x ngroups
    int32_t* glists = nullptr;     // kRing x ngroups
    eikg::Ctrl* ctrl = nullptr;
    // Mapped pinned host memory that kernels write directly, so that the host
    // reads small results after a stream synchronisation without a
    // device-to-host copy (which would queue behind another context's large
    // result copy on the copy engine)
    int* h_err = nullptr;          // number of the last upload that found a bad F
    int* d_err = nullptr;
    int upload_seq = 0;
    int check_seq = 0;             // upload whose flag is still to be read (speed_unchecked)
    double* h_gather = nullptr;    // h/F at the source candidates
    double* d_gather = nullptr;
    int gather_cap = 0;
    float* d_mlp = nullptr;        // schedule network weights (eik_set_schedule)
    eikg::RestartRec* log = nullptr;
    int64_t log_cap = 0;
    void* scratch = nullptr;       // per-solve tables of the fixed nodes
    size_t scratch_cap = 0;
    void* fstage = nullptr;        // staging for host speed uploads and host results
    size_t fstage_cap = 0;
    int nfix = 0;
    int32_t* d_fix_b = nullptr;
    int32_t* d_fix_p = nullptr;
    void* d_saved_r = nullptr;
    std::vector<double> src;
    bool solved = false;
    bool in_flight = false;
    bool speed_unchecked = false;  // an eik_set_speed_async whose validation flag is not read yet
    int64_t last_nr = 0;
    int tuned_block = 0;           // block edge picked by eik_autotune (0: not tuned)
    double tuned_stride = 0.0;     // stride picked by eik_autotune
    int loop_grid = 0;
    int sms = 0;
    eik_params params{};
    eikg::Ctrl host_ctrl{};
    std::string err;
    // part of a grid sharded in z across GPUs (eik_slab_*): the brick planes this context owns, and the
    // restart loop's parameters between the restarts of a sharded solve
    int own_bz0 = 0, own_bz1 = 0;
    int zoff = 0;                  // first node plane of this part in the whole grid
    int nz_all = 0;                // node planes of the whole grid (sources are in its coordinates)
    bool slab = false;
    bool slab_running = false;
    eikg::LoopParams<float> lp_f{};
    eikg::LoopParams<double> lp_d{};
    // 32^3 blocks (block_dim 32, FP32): their own layout, allocated on the first such solve
    struct {
        int NBX = 0, NBY = 0, NBZ = 0;
        int64_t nblk = 0;
        float* rr = nullptr;               // h/F in 32^3 blocks (from the brick layout)
        float* copy = nullptr;
        unsigned* ups = nullptr;
        unsigned long long* stamp = nullptr;
        int32_t* queued = nullptr;
        int32_t* lists = nullptr;
        int32_t* done = nullptr;
        bool rr_valid = false;
        int grid = 0;
    } b32;
    int last_edge = 8;                 // block edge of the last solve (where eik_result finds psi)
};

namespace {

std::string g_create_error;

eik_status fail(eik_ctx* c, eik_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

#define EIK_CK(ctx, call)                                                                                   \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? EIK_ENOMEM : EIK_ECUDA,                    \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                                \
    } while (0)

template <typename P>
cudaError_t dalloc(P** p, size_t bytes) {
    return cudaMalloc(reinterpret_cast<void**>(p), bytes < 16 ? 16 : bytes);
}

void free_all(eik_ctx* c) {
    void* ptrs[] = {c->rr,    c->slot,  c->ups,   c->stamp,   c->queued, c->lists, c->done, c->qgroup, c->glists,
                    c->ctrl,  c->log, c->scratch, c->fstage, c->d_mlp};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    void* p32[] = {c->b32.rr, c->b32.copy, c->b32.ups, c->b32.stamp, c->b32.queued, c->b32.lists, c->b32.done};
    for (void* p : p32)
        if (p) cudaFree(p);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->h_gather) cudaFreeHost(c->h_gather);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// The device staging buffer for host uploads and host results, grown to `bytes`.
eik_status ensure_stage(eik_ctx* c, size_t bytes) {
    if (bytes <= c->fstage_cap) return EIK_OK;
    if (c->fstage) cudaFree(c->fstage);
    c->fstage = nullptr;
    c->fstage_cap = 0;
    EIK_CK(c, cudaMalloc(&c->fstage, bytes));
    c->fstage_cap = bytes;
    return EIK_OK;
}

eik_status check_speed(eik_ctx* c);

// F (x fastest, caller memory) -> h/F in brick layout, with validation (checked
// here, or left for check_speed when `wait` is false).
eik_status upload_speed(eik_ctx* c, const void* F, int F_on_device, bool wait = true) {
    const size_t bytes = static_cast<size_t>(c->nx) * c->ny * c->nz * c->esz;
    const void* Fd = F;
    if (!F_on_device) {
        const eik_status st = ensure_stage(c, bytes);
        if (st != EIK_OK) return st;
        EIK_CK(c, cudaMemcpyAsync(c->fstage, F, bytes, cudaMemcpyHostToDevice, c->stream));
        Fd = c->fstage;
    }
    const int seq = ++c->upload_seq;
    c->b32.rr_valid = false;
    if (c->prec == EIK_FP32)
        EIK_CK(c, eikg::launch_layout_speed<float>(static_cast<const float*>(Fd), static_cast<float*>(c->rr), c->nx,
                                                   c->ny, c->nz, c->BX, c->BY, c->nbricks, c->h, c->d_err, seq,
                                                   c->stream));
    else
        EIK_CK(c, eikg::launch_layout_speed<double>(static_cast<const double*>(Fd), static_cast<double*>(c->rr),
                                                    c->nx, c->ny, c->nz, c->BX, c->BY, c->nbricks, c->h,
                                                    c->d_err, seq, c->stream));
    c->speed_unchecked = true;
    c->check_seq = seq;
    if (!wait) return EIK_OK;
    return check_speed(c);
}

// Read the validation flag of an asynchronous speed upload (waits for the
// stream's queued work).
eik_status check_speed(eik_ctx* c) {
    if (!c->speed_unchecked) return EIK_OK;
    EIK_CK(c, cudaStreamSynchronize(c->stream));
    const bool bad = *reinterpret_cast<volatile int*>(c->h_err) == c->check_seq;
    c->speed_unchecked = false;
    if (bad) {
        c->solved = false;
        return fail(c, EIK_EINVAL, "F must be finite and >= 0 everywhere");
    }
    return EIK_OK;
}

// psi of the last solve in grid order -> dst (device memory), queued on the stream.
cudaError_t queue_result(eik_ctx* c, void* dst) {
    if (c->last_edge == 32)
        return eikg::block32_result(c->b32.copy, c->b32.stamp, static_cast<float*>(dst), c->nx, c->ny, c->nz, c->b32.NBX,
                                    c->b32.NBY, c->stream);
    if (c->prec == EIK_FP32)
        return eikg::launch_result<float>(static_cast<const float*>(c->slot), c->stamp, static_cast<float*>(dst),
                                          c->nx, c->ny, 0, c->nz, c->BX, c->BY, c->stream);
    return eikg::launch_result<double>(static_cast<const double*>(c->slot), c->stamp, static_cast<double*>(dst),
                                       c->nx, c->ny, 0, c->nz, c->BX, c->BY, c->stream);
}


}  // namespace

extern "C" {

const char* eik_version(void) { return "eik-gb300 0.1 (sm_103a)"; }

const char* eik_last_error(const eik_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void eik_params_default(eik_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->stride = 0.0;
    p->block_dim = 8;
    p->schedule = EIK_SCHED_FIXED;
    p->window = 2.0;
    p->fallback_tau = 0.125;
    p->max_restarts = int64_t(1) << 24;
    p->log_restarts = 0;
    p->switch_margin = 0.02;
}

eik_status eik_create(eik_ctx** out, const int32_t dims[3], double h, const void* F, int F_on_device,
                      eik_precision precision, void* stream) {
    if (!out) return fail(nullptr, EIK_EINVAL, "eik_create: out is NULL");
    *out = nullptr;
    if (!dims) return fail(nullptr, EIK_EINVAL, "eik_create: dims is NULL");
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1)
        return fail(nullptr, EIK_EINVAL, "eik_create: every dimension must be >= 1");
    const int64_t N = int64_t(dims[0]) * dims[1] * dims[2];
    if (N >= (int64_t(1) << 31)) return fail(nullptr, EIK_EINVAL, "eik_create: nx*ny*nz must be < 2^31");
    if (!finite_pos(h)) return fail(nullptr, EIK_EINVAL, "eik_create: h must be finite and > 0");
    if (!F) return fail(nullptr, EIK_EINVAL, "eik_create: F is NULL");
    if (precision != EIK_FP32 && precision != EIK_FP64)
        return fail(nullptr, EIK_EINVAL, "eik_create: precision must be EIK_FP32 or EIK_FP64");

    eik_ctx* c = new (std::nothrow) eik_ctx();
    if (!c) return fail(nullptr, EIK_ENOMEM, "eik_create: host allocation failed");
    c->nx = dims[0];
    c->ny = dims[1];
    c->nz = dims[2];
    c->h = h;
    c->prec = precision;
    c->stream = static_cast<cudaStream_t>(stream);
    c->esz = precision == EIK_FP32 ? 4 : 8;
    c->BX = (c->nx + 7) / 8;
    c->BY = (c->ny + 7) / 8;
    c->BZ = (c->nz + 7) / 8;
    c->nbricks = int64_t(c->BX) * c->BY * c->BZ;
    c->GX = (c->BX + 1) / 2;
    c->GY = (c->BY + 1) / 2;
    c->GZ = (c->BZ + 1) / 2;
    c->ngroups = int64_t(c->GX) * c->GY * c->GZ;
    eik_params_default(&c->params);

    auto bail = [&](eik_status s, const std::string& m) {
        free_all(c);
        delete c;
        return fail(nullptr, s, m);
    };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bail(EIK_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
    if (!coop) return bail(EIK_ENOTSUP, "eik_create: device lacks cooperative launch");
    const size_t nb = static_cast<size_t>(c->nbricks);
    struct {
        void** p;
        size_t bytes;
    } allocs[] = {
        {&c->rr, nb * kBrick * c->esz},
        {&c->slot, nb * 2 * kSlot * c->esz},
        {reinterpret_cast<void**>(&c->ups), nb * 2 * 6 * sizeof(unsigned long long)},
        {reinterpret_cast<void**>(&c->stamp), nb * sizeof(unsigned long long)},
        {reinterpret_cast<void**>(&c->queued), eikg::kRing * nb * sizeof(int32_t)},
        {reinterpret_cast<void**>(&c->lists), eikg::kRing * nb * sizeof(int32_t)},
        {reinterpret_cast<void**>(&c->done), nb * sizeof(int32_t)},
        {reinterpret_cast<void**>(&c->qgroup), eikg::kRing * static_cast<size_t>(c->ngroups) * sizeof(int32_t)},
        {reinterpret_cast<void**>(&c->glists), eikg::kRing * static_cast<size_t>(c->ngroups) * sizeof(int32_t)},
        {reinterpret_cast<void**>(&c->ctrl), sizeof(eikg::Ctrl)},
    };
    for (auto& a : allocs) {
        e = dalloc(a.p, a.bytes);
        if (e != cudaSuccess)
            return bail(EIK_ENOMEM, std::string("eik_create: cudaMalloc of ") + std::to_string(a.bytes) +
                                        " bytes failed: " + cudaGetErrorString(e));
    }
    e = cudaHostAlloc(reinterpret_cast<void**>(&c->h_err), 64, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->d_err), c->h_err, 0);
    if (e != cudaSuccess) return bail(EIK_ENOMEM, std::string("eik_create: mapped host flag: ") + cudaGetErrorString(e));
    *c->h_err = 0;
    {
        const eik_status st = upload_speed(c, F, F_on_device);
        if (st != EIK_OK) {
            const std::string m = c->err;
            return bail(st, m);
        }
    }
    int per_sm = 0;
    e = (c->prec == EIK_FP32) ? eikg::loop_occupancy<float>(&per_sm) : eikg::loop_occupancy<double>(&per_sm);
    if (e != cudaSuccess || per_sm < 1)
        return bail(EIK_ECUDA, std::string("eik_create: occupancy query: ") + cudaGetErrorString(e));
    c->loop_grid = per_sm * c->sms;
    // every context starts with the shipped schedule network (eik_set_schedule replaces or unloads it)
    static_assert(EIK_SCHED_DEFAULT_COUNT == eikg::kParams, "shipped weights match the network");
    e = cudaMalloc(&c->d_mlp, sizeof(float) * eikg::kParams);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_mlp, kSchedDefault, sizeof(float) * eikg::kParams, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(EIK_ENOMEM, std::string("eik_create: schedule weights: ") + cudaGetErrorString(e));
    *out = c;
    return EIK_OK;
}

eik_status eik_set_schedule(eik_ctx* c, const float* w, int32_t n) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_set_schedule: ctx is NULL");
    if (c->in_flight) return fail(c, EIK_ESTATE, "eik_set_schedule: a solve is in flight");
    if (!w) {
        if (c->d_mlp) cudaFree(c->d_mlp);
        c->d_mlp = nullptr;
        return EIK_OK;
    }
    if (n != eikg::kParams) return fail(c, EIK_EINVAL, "eik_set_schedule: n must be EIK_SCHED_PARAMS");
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(w[i])) return fail(c, EIK_EINVAL, "eik_set_schedule: weights must be finite");
    if (!c->d_mlp) EIK_CK(c, cudaMalloc(&c->d_mlp, sizeof(float) * eikg::kParams));
    EIK_CK(c, cudaMemcpy(c->d_mlp, w, sizeof(float) * eikg::kParams, cudaMemcpyHostToDevice));
    return EIK_OK;
}

eik_status eik_set_speed(eik_ctx* c, const void* F, int F_on_device) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_set_speed: ctx is NULL");
    if (!F) return fail(c, EIK_EINVAL, "eik_set_speed: F is NULL");
    if (c->in_flight) return fail(c, EIK_ESTATE, "eik_set_speed: a solve is in flight (call eik_wait)");
    c->solved = false;
    c->speed_unchecked = false;     // an earlier asynchronous upload is superseded
    return upload_speed(c, F, F_on_device);
}

eik_status eik_set_speed_async(eik_ctx* c, const void* F, int F_on_device) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_set_speed_async: ctx is NULL");
    if (!F) return fail(c, EIK_EINVAL, "eik_set_speed_async: F is NULL");
    if (c->in_flight) return fail(c, EIK_ESTATE, "eik_set_speed_async: a solve is in flight (call eik_wait)");
    c->solved = false;
    return upload_speed(c, F, F_on_device, false);
}

eik_status eik_source_nodes(const int32_t dims[3], double h, const void* F, eik_precision precision, int32_t nsrc,
                            const double* xyz, int64_t* idx_out, double* psi0_out, int64_t cap, int64_t* n_out) {
    if (!dims || !F || !n_out || (nsrc > 0 && !xyz) || nsrc < 0)
        return fail(nullptr, EIK_EINVAL, "eik_source_nodes: NULL argument or nsrc < 0");
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || !finite_pos(h))
        return fail(nullptr, EIK_EINVAL, "eik_source_nodes: bad dims or h");
    if (precision != EIK_FP32 && precision != EIK_FP64)
        return fail(nullptr, EIK_EINVAL, "eik_source_nodes: bad precision");
    const int nx = dims[0], ny = dims[1], nz = dims[2];
    const int dd[3] = {nx, ny, nz};
    for (int s = 0; s < nsrc; ++s)
        for (int a = 0; a < 3; ++a) {
            const double v = xyz[3 * s + a];
            if (!std::isfinite(v) || v < -1e-9 * h || v > (dd[a] - 1) * h + 1e-9 * h)
                return fail(nullptr, EIK_EINVAL, "eik_source_nodes: source " + std::to_string(s) + " lies outside the grid");
        }
    // the candidates and their h/F as a solve sees them (h/F rounded as the speed re-layout rounds it)
    const eikh::Bricks geo{(nx + 7) / 8, (ny + 7) / 8, (nz + 7) / 8, 0};
    std::vector<eikh::Cand> cand;
    eikh::source_candidates(xyz, nsrc, nx, ny, nz, h, geo, cand);
    std::vector<double> r(cand.size());
    auto lin = [&](const eikh::Cand& c, int* i, int* j, int* k) {
        const int bx = c.b % geo.BX, by = (c.b / geo.BX) % geo.BY, bz = c.b / (geo.BX * geo.BY);
        *i = bx * 8 + (c.p & 7);
        *j = by * 8 + ((c.p >> 3) & 7);
        *k = bz * 8 + (c.p >> 6);
    };
    for (size_t t = 0; t < cand.size(); ++t) {
        int i, j, k;
        lin(cand[t], &i, &j, &k);
        const int64_t q = (static_cast<int64_t>(k) * ny + j) * nx + i;
        double rv = INFINITY;
        if (precision == EIK_FP32) {
            const float f = static_cast<const float*>(F)[q];
            if (!(f >= 0.0f) || !std::isfinite(f)) return fail(nullptr, EIK_EINVAL, "F must be finite and >= 0");
            if (f > 0.0f) rv = static_cast<double>(static_cast<float>(h) / f);
        } else {
            const double f = static_cast<const double*>(F)[q];
            if (!(f >= 0.0) || !std::isfinite(f)) return fail(nullptr, EIK_EINVAL, "F must be finite and >= 0");
            if (f > 0.0) rv = h / f;
        }
        r[t] = rv;
    }
    const std::vector<eikh::FixNode> uf = eikh::fixed_nodes(cand, r, h);
    *n_out = static_cast<int64_t>(uf.size());
    if (static_cast<int64_t>(uf.size()) > cap) return fail(nullptr, EIK_EINVAL, "eik_source_nodes: cap too small");
    for (size_t t = 0; t < uf.size(); ++t) {
        int i, j, k;
        lin(eikh::Cand{uf[t].b, uf[t].p, 0.0}, &i, &j, &k);
        if (idx_out) idx_out[t] = (static_cast<int64_t>(k) * ny + j) * nx + i;
        if (psi0_out) psi0_out[t] = uf[t].v;
    }
    return EIK_OK;
}

eik_status eik_add_sources(eik_ctx* c, int32_t n, const double* xyz) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_add_sources: ctx is NULL");
    if (c->in_flight) return fail(c, EIK_ESTATE, "eik_add_sources: a solve is in flight (call eik_wait)");
    if (n < 0) return fail(c, EIK_EINVAL, "eik_add_sources: n < 0");
    if (n > 0 && !xyz) return fail(c, EIK_EINVAL, "eik_add_sources: xyz is NULL");
    const int dims[3] = {c->nx, c->ny, c->slab ? c->nz_all : c->nz};    // (a part of a sharded grid: whole-grid z)
    const double tol = 1e-9 * c->h;
    for (int s = 0; s < n; ++s)
        for (int a = 0; a < 3; ++a) {
            const double v = xyz[3 * s + a];
            const double ext = (dims[a] - 1) * c->h;
            if (!std::isfinite(v) || v < -tol || v > ext + tol)
                return fail(c, EIK_EINVAL, "eik_add_sources: source " + std::to_string(s) + " lies outside the grid");
        }
    c->src.insert(c->src.end(), xyz, xyz + 3 * static_cast<size_t>(n));
    return EIK_OK;
}

eik_status eik_clear_sources(eik_ctx* c) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_clear_sources: ctx is NULL");
    if (c->in_flight) return fail(c, EIK_ESTATE, "eik_clear_sources: a solve is in flight");
    c->src.clear();
    return EIK_OK;
}

}  // extern "C"

namespace {

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

template <typename T>
eikg::LoopParams<T>& loop_params(eik_ctx* c);
template <>
eikg::LoopParams<float>& loop_params<float>(eik_ctx* c) { return c->lp_f; }
template <>
eikg::LoopParams<double>& loop_params<double>(eik_ctx* c) { return c->lp_d; }

// Set up a solve (Alg. 1, work lists, control block) and, unless `slab`, queue
// the whole restart loop.  With `slab` the context is one part of a grid
// sharded in z: the loop's parameters are kept for eik_slab_restart, which
// runs one restart at a time, and ghost bricks never go on a work list.
template <typename T>
eik_status queue_solve(eik_ctx* c, const eik_params& P, bool slab = false) {
    cudaStream_t s = c->stream;
    // ---- fixed nodes: candidates of every source, with their h/F from the device
    const eikh::Bricks geo{c->BX, c->BY, c->BZ, 0};
    std::vector<eikh::Cand> cand;
    const int nsrc = static_cast<int>(c->src.size() / 3);
    eikh::source_candidates(c->src.data(), nsrc, c->nx, c->ny, c->slab ? c->nz_all : c->nz, c->h, geo, cand,
                            c->slab ? c->zoff : 0, c->nz);
    const int nc = static_cast<int>(cand.size());
    std::vector<int32_t> cb(nc), cp(nc);
    for (int t = 0; t < nc; ++t) {
        cb[t] = cand[t].b;
        cp[t] = cand[t].p;
    }
    // scratch: candidate tables, then the fixed-node tables
    const size_t need = align_up(nc * 4) * 2 + align_up(nc * 8) + align_up(nc * 4) * 4 + align_up(nc * 8) +
                        align_up(nc * sizeof(T)) + 4096;
    if (need > c->scratch_cap) {
        if (c->scratch) cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_cap = 0;
        EIK_CK(c, cudaMalloc(&c->scratch, need));
        c->scratch_cap = need;
    }
    char* sp = static_cast<char*>(c->scratch);
    auto carve = [&](size_t bytes) {
        char* r = sp;
        sp += align_up(bytes);
        return r;
    };
    int32_t* d_cb = reinterpret_cast<int32_t*>(carve(nc * 4));
    int32_t* d_cp = reinterpret_cast<int32_t*>(carve(nc * 4));
    carve(nc * 8);
    std::vector<double> cr(nc);
    if (nc > 0) {
        if (nc > c->gather_cap) {
            if (c->h_gather) cudaFreeHost(c->h_gather);
            c->h_gather = nullptr;
            c->gather_cap = 0;
            EIK_CK(c, cudaHostAlloc(reinterpret_cast<void**>(&c->h_gather), static_cast<size_t>(nc) * 8,
                                    cudaHostAllocMapped));
            EIK_CK(c, cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->d_gather), c->h_gather, 0));
            c->gather_cap = nc;
        }
        EIK_CK(c, cudaMemcpyAsync(d_cb, cb.data(), nc * 4, cudaMemcpyHostToDevice, s));
        EIK_CK(c, cudaMemcpyAsync(d_cp, cp.data(), nc * 4, cudaMemcpyHostToDevice, s));
        EIK_CK(c, eikg::launch_gather_r<T>(nc, d_cb, d_cp, static_cast<const T*>(c->rr), c->d_gather, s));
        EIK_CK(c, cudaStreamSynchronize(s));
        for (int t = 0; t < nc; ++t) cr[t] = reinterpret_cast<volatile double*>(c->h_gather)[t];
    }
    const std::vector<eikh::FixNode> uf = eikh::fixed_nodes(cand, cr, c->h);
    std::vector<int32_t> sb, enq;
    eikh::first_active(uf, geo, sb, enq);
    if (slab) {                          // ghost bricks are marched by the GPU that owns them
        std::vector<int32_t> own;
        for (int32_t x : enq) {
            const int bz = x / (c->BX * c->BY);
            if (bz >= c->own_bz0 && bz < c->own_bz1) own.push_back(x);
        }
        enq.swap(own);
    }
    const bool groups = (P.block_dim == 16) || (P.schedule != EIK_SCHED_FIXED);
    std::vector<int32_t> genq;
    if (groups) genq = eikh::groups_of(enq, geo, c->GX, c->GY, 0);
    const int nfix = static_cast<int>(uf.size());
    std::vector<int32_t> fb(nfix), fp(nfix);
    std::vector<double> fv(nfix);
    for (int t = 0; t < nfix; ++t) {
        fb[t] = uf[t].b;
        fp[t] = uf[t].p;
        fv[t] = uf[t].v;
    }
    c->d_fix_b = reinterpret_cast<int32_t*>(carve(nfix * 4));
    c->d_fix_p = reinterpret_cast<int32_t*>(carve(nfix * 4));
    double* d_fv = reinterpret_cast<double*>(carve(nfix * 8));
    int32_t* d_sb = reinterpret_cast<int32_t*>(carve(sb.size() * 4));
    int32_t* d_enq = reinterpret_cast<int32_t*>(carve(enq.size() * 4));
    int32_t* d_genq = reinterpret_cast<int32_t*>(carve(genq.size() * 4));
    c->d_saved_r = carve(nfix * sizeof(T));
    c->nfix = nfix;
    if (nfix > 0) {
        EIK_CK(c, cudaMemcpyAsync(c->d_fix_b, fb.data(), nfix * 4, cudaMemcpyHostToDevice, s));
        EIK_CK(c, cudaMemcpyAsync(c->d_fix_p, fp.data(), nfix * 4, cudaMemcpyHostToDevice, s));
        EIK_CK(c, cudaMemcpyAsync(d_fv, fv.data(), nfix * 8, cudaMemcpyHostToDevice, s));
        EIK_CK(c, cudaMemcpyAsync(d_sb, sb.data(), sb.size() * 4, cudaMemcpyHostToDevice, s));
        EIK_CK(c, cudaMemcpyAsync(d_enq, enq.data(), enq.size() * 4, cudaMemcpyHostToDevice, s));
        if (!genq.empty())
            EIK_CK(c, cudaMemcpyAsync(d_genq, genq.data(), genq.size() * 4, cudaMemcpyHostToDevice, s));
    }
    // ---- Alg. 1 for every brick: untouched (psi = +inf) unless it holds fixed nodes
    const size_t nb = static_cast<size_t>(c->nbricks);
    EIK_CK(c, cudaMemsetAsync(c->stamp, 0xFF, nb * sizeof(unsigned long long), s));
    EIK_CK(c, cudaMemsetAsync(c->queued, 0xFF, eikg::kRing * nb * sizeof(int32_t), s));
    EIK_CK(c, cudaMemsetAsync(c->lists, 0xFF, eikg::kRing * nb * sizeof(int32_t), s));     // empty entries are -1
    EIK_CK(c, cudaMemsetAsync(c->done, 0, nb * sizeof(int32_t), s));
    if (groups) {
        EIK_CK(c, cudaMemsetAsync(c->qgroup, 0xFF, eikg::kRing * static_cast<size_t>(c->ngroups) * sizeof(int32_t), s));
        EIK_CK(c, cudaMemsetAsync(c->glists, 0xFF, eikg::kRing * static_cast<size_t>(c->ngroups) * sizeof(int32_t), s));
    }
    if (nfix > 0)
        EIK_CK(c, eikg::launch_init_sources<T>(nfix, c->d_fix_b, c->d_fix_p, d_fv, static_cast<int>(sb.size()), d_sb,
                                               static_cast<int>(enq.size()), d_enq, static_cast<int>(genq.size()),
                                               d_genq, static_cast<T*>(c->slot), c->ups, c->stamp, c->queued + nb,
                                               c->qgroup + c->ngroups, static_cast<T*>(c->rr),
                                               static_cast<T*>(c->d_saved_r), c->lists + nb, c->glists + c->ngroups, s));
    // ---- control block: restart 1 with bound_1 = 0 + stride
    eikg::Ctrl& H = c->host_ctrl;
    std::memset(&H, 0, sizeof(H));
    H.k = (enq.empty() && !slab) ? 0 : 1;
    H.action = -1;
    H.pend_action = -1;
    H.bound_prev = -1.0;
    H.stride = P.stride;
    H.bound = std::fmin(0.0 + P.stride, P.width);
    H.count[1] = static_cast<int32_t>(enq.size());
    H.gcount[1] = static_cast<int32_t>(genq.size());
    H.mode = (P.block_dim == 16) ? 16 : 8;
    H.r_rmin_bits = 0x7f800000u;
    H.done = (enq.empty() && !slab) ? 1 : 0;
    EIK_CK(c, cudaMemcpyAsync(c->ctrl, &H, sizeof(H), cudaMemcpyHostToDevice, s));
    if (P.log_restarts) {
        const int64_t want = std::min<int64_t>(P.max_restarts, int64_t(1) << 16);
        if (want > c->log_cap) {
            if (c->log) cudaFree(c->log);
            c->log = nullptr;
            c->log_cap = 0;
            EIK_CK(c, cudaMalloc(&c->log, sizeof(eikg::RestartRec) * want));
            c->log_cap = want;
        }
    }
    if (!enq.empty() || slab) {
        eikg::LoopParams<T> L{};
        L.nx = c->nx;
        L.ny = c->ny;
        L.nz = c->nz;
        L.BX = c->BX;
        L.BY = c->BY;
        L.BZ = c->BZ;
        L.nbricks = c->nbricks;
        L.slot = static_cast<T*>(c->slot);
        L.ups = c->ups;
        L.stamp = c->stamp;
        L.queued = c->queued;
        L.done = c->done;
        L.ngroups = c->ngroups;
        L.rr = static_cast<const T*>(c->rr);
        for (int r = 0; r < eikg::kRing; ++r) {
            L.list[r] = c->lists + r * nb;
            L.glist[r] = c->glists + r * c->ngroups;
        }
        L.early = 1;
        L.GX = c->GX;
        L.GY = c->GY;
        L.GZ = c->GZ;
        L.groups = groups ? 1 : 0;
        L.qgroup = c->qgroup;
        L.mode_fixed = (P.block_dim == 16) ? 16 : 8;
        L.ctrl = c->ctrl;
        L.log = P.log_restarts ? c->log : nullptr;
        L.log_cap = P.log_restarts ? c->log_cap : 0;
        L.window = P.window;
        L.window_f = static_cast<float>(P.window);
        L.fallback_tau = P.fallback_tau;
        L.max_restarts = P.max_restarts;
        L.width = P.width;
        L.wait_limit = P.wait_polls > 0 ? P.wait_polls : eikg::kWaitPolls;
        L.sched = P.schedule;
        L.mlp = (P.schedule == EIK_SCHED_LEARNED) ? c->d_mlp : nullptr;
        L.h = c->h;
        L.nmax = std::max(c->nx, std::max(c->ny, c->nz));
        L.seed = static_cast<uint32_t>(P.seed);
        L.margin = static_cast<float>(P.switch_margin);
        L.own_bz0 = 0;
        L.own_bz1 = c->BZ;
        if (slab) {
            L.pause = 1;                 // one restart per launch; the host exchanges faces in between
            L.early = 0;
            L.own_bz0 = c->own_bz0;
            L.own_bz1 = c->own_bz1;
            loop_params<T>(c) = L;
            return EIK_OK;
        }
        if (P.loop_events[0]) EIK_CK(c, cudaEventRecord(static_cast<cudaEvent_t>(P.loop_events[0]), s));
        EIK_CK(c, eikg::launch_restart_loop<T>(L, c->loop_grid, s));
        if (P.loop_events[1]) EIK_CK(c, cudaEventRecord(static_cast<cudaEvent_t>(P.loop_events[1]), s));
    }
    if (nfix > 0)
        EIK_CK(c, eikg::launch_restore_r<T>(nfix, c->d_fix_b, c->d_fix_p, static_cast<const T*>(c->d_saved_r),
                                            static_cast<T*>(c->rr), s));
    return EIK_OK;
}

// The solve with 32^3 blocks (FP32, fixed stride): its layout is allocated and
// h/F re-laid from the bricks on first use; Alg. 1 as in queue_solve, in the
// blocks' coordinates.
eik_status queue_solve32(eik_ctx* c, const eik_params& P) {
    cudaStream_t s = c->stream;
    auto& B = c->b32;
    if (!B.copy) {
        B.NBX = (c->nx + 31) / 32;
        B.NBY = (c->ny + 31) / 32;
        B.NBZ = (c->nz + 31) / 32;
        B.nblk = int64_t(B.NBX) * B.NBY * B.NBZ;
        const size_t nb = static_cast<size_t>(B.nblk);
        struct {
            void** p;
            size_t bytes;
        } allocs[] = {
            {reinterpret_cast<void**>(&B.rr), nb * 32768 * sizeof(float)},
            {reinterpret_cast<void**>(&B.copy), nb * 2 * static_cast<size_t>(eikg::block32_edge_values()) * sizeof(float)},
            {reinterpret_cast<void**>(&B.ups), nb * 2 * 6 * 32 * sizeof(unsigned)},
            {reinterpret_cast<void**>(&B.stamp), nb * sizeof(unsigned long long)},
            {reinterpret_cast<void**>(&B.queued), eikg::kRing * nb * sizeof(int32_t)},
            {reinterpret_cast<void**>(&B.lists), eikg::kRing * nb * sizeof(int32_t)},
            {reinterpret_cast<void**>(&B.done), nb * sizeof(int32_t)},
        };
        for (auto& a : allocs) {
            const cudaError_t e = dalloc(a.p, a.bytes);
            if (e != cudaSuccess) return fail(c, EIK_ENOMEM, std::string("32^3 blocks: cudaMalloc failed: ") + cudaGetErrorString(e));
        }
        int per_sm = 0;
        EIK_CK(c, eikg::block32_occupancy(&per_sm));
        if (per_sm < 1) return fail(c, EIK_ENOTSUP, "32^3 blocks: one CTA of 1024 threads does not fit an SM");
        B.grid = per_sm * c->sms;
    }
    if (!B.rr_valid) {
        EIK_CK(c, eikg::block32_layout(static_cast<const float*>(c->rr), c->BX, c->BY, c->BZ, B.rr, B.NBX, B.NBY, B.nblk, s));
        B.rr_valid = true;
    }
    // ---- fixed nodes (Alg. 1): candidates and their h/F from the brick layout, then block coordinates
    const eikh::Bricks geo{c->BX, c->BY, c->BZ, 0};
    std::vector<eikh::Cand> cand;
    const int nsrc = static_cast<int>(c->src.size() / 3);
    eikh::source_candidates(c->src.data(), nsrc, c->nx, c->ny, c->nz, c->h, geo, cand);
    const int nc = static_cast<int>(cand.size());
    std::vector<int32_t> cb(nc), cp(nc);
    for (int t = 0; t < nc; ++t) {
        cb[t] = cand[t].b;
        cp[t] = cand[t].p;
    }
    const size_t need = align_up(nc * 4) * 2 + align_up(static_cast<size_t>(nc) * 8) * 2 + align_up(nc * 4) * 4 +
                        align_up(nc * 7 * 4) + 4096;
    if (need > c->scratch_cap) {
        if (c->scratch) cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_cap = 0;
        EIK_CK(c, cudaMalloc(&c->scratch, need));
        c->scratch_cap = need;
    }
    char* sp = static_cast<char*>(c->scratch);
    auto carve = [&](size_t bytes) {
        char* r = sp;
        sp += align_up(bytes);
        return r;
    };
    int32_t* d_cb = reinterpret_cast<int32_t*>(carve(nc * 4));
    int32_t* d_cp = reinterpret_cast<int32_t*>(carve(nc * 4));
    std::vector<double> cr(nc);
    if (nc > 0) {
        if (nc > c->gather_cap) {
            if (c->h_gather) cudaFreeHost(c->h_gather);
            c->h_gather = nullptr;
            c->gather_cap = 0;
            EIK_CK(c, cudaHostAlloc(reinterpret_cast<void**>(&c->h_gather), static_cast<size_t>(nc) * 8,
                                    cudaHostAllocMapped));
            EIK_CK(c, cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->d_gather), c->h_gather, 0));
            c->gather_cap = nc;
        }
        EIK_CK(c, cudaMemcpyAsync(d_cb, cb.data(), nc * 4, cudaMemcpyHostToDevice, s));
        EIK_CK(c, cudaMemcpyAsync(d_cp, cp.data(), nc * 4, cudaMemcpyHostToDevice, s));
        EIK_CK(c, eikg::launch_gather_r<float>(nc, d_cb, d_cp, static_cast<const float*>(c->rr), c->d_gather, s));
        EIK_CK(c, cudaStreamSynchronize(s));
        for (int t = 0; t < nc; ++t) cr[t] = reinterpret_cast<volatile double*>(c->h_gather)[t];
    }
    const std::vector<eikh::FixNode> uf = eikh::fixed_nodes(cand, cr, c->h);
    struct Fix32 {
        int32_t b, p;
        double v;
    };
    std::vector<Fix32> f32;
    std::vector<int32_t> sb, enq;
    for (const auto& f : uf) {
        const int bx8 = f.b % c->BX, by8 = (f.b / c->BX) % c->BY, bz8 = f.b / (c->BX * c->BY);
        const int i = bx8 * 8 + (f.p & 7), j = by8 * 8 + ((f.p >> 3) & 7), k = bz8 * 8 + (f.p >> 6);
        const int bx = i >> 5, by = j >> 5, bz = k >> 5, x = i & 31, y = j & 31, z = k & 31;
        const int32_t b = (bz * B.NBY + by) * B.NBX + bx;
        f32.push_back({b, (z * 32 + y) * 32 + x, f.v});
        sb.push_back(b);
        enq.push_back(b);
        // neighbours whose ghost layer holds the fixed node (Alg. 1 over Xi^ib)
        if (x == 0 && bx > 0) enq.push_back(b - 1);
        if (x == 31 && bx < B.NBX - 1) enq.push_back(b + 1);
        if (y == 0 && by > 0) enq.push_back(b - B.NBX);
        if (y == 31 && by < B.NBY - 1) enq.push_back(b + B.NBX);
        if (z == 0 && bz > 0) enq.push_back(b - B.NBX * B.NBY);
        if (z == 31 && bz < B.NBZ - 1) enq.push_back(b + B.NBX * B.NBY);
    }
    std::sort(sb.begin(), sb.end());
    sb.erase(std::unique(sb.begin(), sb.end()), sb.end());
    std::sort(enq.begin(), enq.end());
    enq.erase(std::unique(enq.begin(), enq.end()), enq.end());
    const int nfix = static_cast<int>(f32.size());
    std::vector<int32_t> fb(nfix), fp(nfix);
    std::vector<double> fv(nfix);
    for (int t = 0; t < nfix; ++t) {
        fb[t] = f32[t].b;
        fp[t] = f32[t].p;
        fv[t] = f32[t].v;
    }
    c->d_fix_b = reinterpret_cast<int32_t*>(carve(nfix * 4));
    c->d_fix_p = reinterpret_cast<int32_t*>(carve(nfix * 4));
    double* d_fv = reinterpret_cast<double*>(carve(static_cast<size_t>(nfix) * 8));
    int32_t* d_sb = reinterpret_cast<int32_t*>(carve(sb.size() * 4));
    int32_t* d_enq = reinterpret_cast<int32_t*>(carve(enq.size() * 4));
    c->d_saved_r = carve(nfix * sizeof(float));
    c->nfix = nfix;
    if (nfix > 0) {
        EIK_CK(c, cudaMemcpyAsync(c->d_fix_b, fb.data(), nfix * 4, cudaMemcpyHostToDevice, s));
        EIK_CK(c, cudaMemcpyAsync(c->d_fix_p, fp.data(), nfix * 4, cudaMemcpyHostToDevice, s));
        EIK_CK(c, cudaMemcpyAsync(d_fv, fv.data(), nfix * 8, cudaMemcpyHostToDevice, s));
        EIK_CK(c, cudaMemcpyAsync(d_sb, sb.data(), sb.size() * 4, cudaMemcpyHostToDevice, s));
        EIK_CK(c, cudaMemcpyAsync(d_enq, enq.data(), enq.size() * 4, cudaMemcpyHostToDevice, s));
    }
    const size_t nb = static_cast<size_t>(B.nblk);
    EIK_CK(c, cudaMemsetAsync(B.stamp, 0xFF, nb * sizeof(unsigned long long), s));
    EIK_CK(c, cudaMemsetAsync(B.queued, 0xFF, eikg::kRing * nb * sizeof(int32_t), s));
    EIK_CK(c, cudaMemsetAsync(B.lists, 0xFF, eikg::kRing * nb * sizeof(int32_t), s));
    EIK_CK(c, cudaMemsetAsync(B.done, 0xFF, nb * sizeof(int32_t), s));
    if (nfix > 0)
        EIK_CK(c, eikg::block32_init(nfix, c->d_fix_b, c->d_fix_p, d_fv, static_cast<int>(sb.size()), d_sb,
                                     static_cast<int>(enq.size()), d_enq, B.copy, B.ups, B.stamp, B.queued + nb, B.rr,
                                     static_cast<float*>(c->d_saved_r), B.lists + nb, s));
    eikg::Ctrl& H = c->host_ctrl;
    std::memset(&H, 0, sizeof(H));
    H.k = enq.empty() ? 0 : 1;
    H.action = -1;
    H.pend_action = -1;
    H.bound_prev = -1.0;
    H.stride = P.stride;
    H.bound = std::fmin(P.stride, P.width);
    H.count[1] = static_cast<int32_t>(enq.size());
    H.mode = 32;
    H.r_rmin_bits = 0x7f800000u;
    H.done = enq.empty() ? 1 : 0;
    EIK_CK(c, cudaMemcpyAsync(c->ctrl, &H, sizeof(H), cudaMemcpyHostToDevice, s));
    if (!enq.empty()) {
        if (P.loop_events[0]) EIK_CK(c, cudaEventRecord(static_cast<cudaEvent_t>(P.loop_events[0]), s));
        EIK_CK(c, eikg::block32_loop(B.NBX, B.NBY, B.NBZ, B.nblk, B.copy, B.ups, B.stamp, B.rr, B.queued, B.lists, B.done,
                                     c->ctrl,
                                     static_cast<float>(P.window), static_cast<float>(P.fallback_tau), P.width,
                                     P.max_restarts, P.wait_polls > 0 ? P.wait_polls : eikg::kWaitPolls, B.grid, s));
        if (P.loop_events[1]) EIK_CK(c, cudaEventRecord(static_cast<cudaEvent_t>(P.loop_events[1]), s));
    }
    if (nfix > 0)
        EIK_CK(c, eikg::block32_restore(nfix, c->d_fix_b, c->d_fix_p, static_cast<const float*>(c->d_saved_r), B.rr, s));
    return EIK_OK;
}

eik_status check_params(eik_ctx* c, const eik_params* p) {
    if (!p) return fail(c, EIK_EINVAL, "params is NULL");
    eik_status code;
    if (const char* m = eikh::param_error(*p, &code)) return fail(c, code, m);
    if (p->schedule == EIK_SCHED_LEARNED && !c->d_mlp)
        return fail(c, EIK_ESTATE, "learned schedule requested but the weights were unloaded (eik_set_schedule)");
    return EIK_OK;
}

}  // namespace

extern "C" {

eik_status eik_solve_async(eik_ctx* c, const eik_params* params) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_solve_async: ctx is NULL");
    if (c->in_flight) return fail(c, EIK_ESTATE, "eik_solve_async: a solve is already in flight");
    if (!params) return fail(c, EIK_EINVAL, "params is NULL");
    eik_params P = *params;
    // stride 0: the learned schedule (its first two restarts advance the bound by 2h)
    if (P.stride == 0.0) {
        P.schedule = EIK_SCHED_LEARNED;
        P.stride = 2.0 * c->h;
    }
    eik_status st = check_params(c, &P);
    if (st != EIK_OK) return st;
    if (c->src.empty()) return fail(c, EIK_ESTATE, "eik_solve: no source added");
    st = check_speed(c);
    if (st != EIK_OK) return st;
    // block edge 0: under the learned schedule the network picks it from restart 3 on (8 before); under a
    // fixed stride the edge eik_autotune picked for this context, else 8
    if (P.block_dim == 0) P.block_dim = (P.schedule == EIK_SCHED_FIXED && c->tuned_block) ? c->tuned_block : 8;
    if (P.max_restarts == 0) P.max_restarts = int64_t(1) << 24;
    if (P.window == 0.0) P.window = 2.0;
    if (P.width == 0.0) P.width = INFINITY;
    c->params = P;
    if (P.block_dim == 32) {
        if (c->prec != EIK_FP32) return fail(c, EIK_ENOTSUP, "32^3 blocks are single precision only");
        if (P.schedule != EIK_SCHED_FIXED) return fail(c, EIK_ENOTSUP, "32^3 blocks take a fixed stride");
        if (P.log_restarts) return fail(c, EIK_ENOTSUP, "32^3 blocks keep no restart log");
        st = queue_solve32(c, P);
        c->last_edge = 32;
    } else {
        st = (c->prec == EIK_FP32) ? queue_solve<float>(c, P) : queue_solve<double>(c, P);
        c->last_edge = 8;
    }
    if (st != EIK_OK) return st;
    c->in_flight = true;
    c->solved = false;
    return EIK_OK;
}

eik_status eik_wait(eik_ctx* c, eik_stats* stats) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_wait: ctx is NULL");
    if (!c->in_flight) return fail(c, EIK_ESTATE, "eik_wait: no solve in flight");
    c->in_flight = false;
    EIK_CK(c, cudaStreamSynchronize(c->stream));
    eikg::Ctrl H{};
    EIK_CK(c, cudaMemcpy(&H, c->ctrl, sizeof(H), cudaMemcpyDeviceToHost));
    c->host_ctrl = H;
    c->last_nr = H.k;
    eik_status st = EIK_OK;
    if (H.status & (eikg::kStWaitTimeout | eikg::kStRestartCap | eikg::kStRoundCap)) {
        st = EIK_ETIMEOUT;
        c->err = std::string("solve stopped early: ") +
                 ((H.status & eikg::kStRestartCap) ? "restart cap reached " : "") +
                 ((H.status & eikg::kStWaitTimeout) ? "grid-barrier wait limit reached " : "") +
                 ((H.status & eikg::kStRoundCap) ? "march round cap reached" : "");
    } else if (!H.done) {
        st = EIK_ECUDA;
        c->err = "solve did not finish";
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->restarts = H.k;
        stats->marches = static_cast<int64_t>(H.marches);
        stats->accepted = static_cast<int64_t>(H.accepted);
        stats->solves = static_cast<int64_t>(H.solves);
        stats->updates = static_cast<int64_t>(H.updates);
        stats->fallbacks = static_cast<int64_t>(H.fallbacks);
        stats->rounds = static_cast<int64_t>(H.rounds);
        stats->device_ms = (H.t_end > H.t_begin) ? static_cast<double>(H.t_end - H.t_begin) * 1e-6 : 0.0;
        stats->final_bound = H.bound;
        stats->status = st;
        stats->block_dim = c->params.block_dim;
    }
    if (st == EIK_OK) c->solved = true;
    return st;
}

eik_status eik_solve_ex(eik_ctx* c, const eik_params* params, eik_stats* stats) {
    eik_status st = eik_solve_async(c, params);
    if (st != EIK_OK) return st;
    return eik_wait(c, stats);
}

eik_status eik_solve(eik_ctx* c, double stride, int32_t block_dim, eik_stats* stats) {
    eik_params p;
    eik_params_default(&p);
    p.stride = stride;
    p.block_dim = block_dim;
    return eik_solve_ex(c, &p, stats);
}

eik_status eik_autotune(eik_ctx* c, int32_t rounds, double* stride_out, int32_t* block_out, double* best_ms) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_autotune: ctx is NULL");
    if (c->in_flight) return fail(c, EIK_ESTATE, "eik_autotune: a solve is in flight");
    if (rounds < 0) return fail(c, EIK_EINVAL, "eik_autotune: rounds must be >= 0");
    if (c->src.empty()) return fail(c, EIK_ESTATE, "eik_autotune: no source added");
    struct Cand {
        double stride_h;
        int block;
        std::vector<double> ms;
    };
    std::vector<Cand> alive;
    for (double sh : {1.0, 1.5, 2.0, 2.5, 3.0, 4.0})
        for (int bd : {8, 16}) alive.push_back({sh, bd, {}});
    const eik_params keep = c->params;
    auto median = [](std::vector<double> v) {
        std::sort(v.begin(), v.end());
        return v[v.size() / 2];
    };
    int reps = 1;
    for (int round = 0; alive.size() > 1 && (rounds == 0 || round < rounds); ++round, reps *= 2) {
        for (auto& cd : alive) {
            for (int r = 0; r < reps; ++r) {
                eik_params P;
                eik_params_default(&P);
                P.stride = cd.stride_h * c->h;
                P.block_dim = cd.block;
                eik_stats st{};
                const eik_status e = eik_solve_ex(c, &P, &st);
                if (e == EIK_ETIMEOUT) {
                    cd.ms.push_back(INFINITY);
                    continue;
                }
                if (e != EIK_OK) {
                    c->params = keep;
                    return e;
                }
                cd.ms.push_back(st.device_ms);
            }
        }
        std::sort(alive.begin(), alive.end(), [&](const Cand& a, const Cand& b) { return median(a.ms) < median(b.ms); });
        const size_t next = std::max<size_t>(1, alive.size() / 3);
        alive.resize(next);
    }
    if (!std::isfinite(median(alive[0].ms))) return fail(c, EIK_ETIMEOUT, "eik_autotune: every candidate hit a cap");
    c->tuned_stride = alive[0].stride_h * c->h;
    c->tuned_block = alive[0].block;
    if (stride_out) *stride_out = c->tuned_stride;
    if (block_out) *block_out = c->tuned_block;
    if (best_ms) *best_ms = median(alive[0].ms);
    return EIK_OK;
}

int64_t eik_slab_face_bytes(const eik_ctx* c) {
    if (!c) return -1;
    const size_t rec = (c->prec == EIK_FP32) ? sizeof(eikg::FaceRec<float>) : sizeof(eikg::FaceRec<double>);
    return static_cast<int64_t>(rec) * c->BX * c->BY;
}

eik_status eik_slab_set(eik_ctx* c, int32_t own_bz0, int32_t own_bz1, int32_t zoff, int32_t nz_all) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_slab_set: ctx is NULL");
    if (c->in_flight || c->slab_running) return fail(c, EIK_ESTATE, "eik_slab_set: a solve is in flight");
    if (!(0 <= own_bz0 && own_bz0 < own_bz1 && own_bz1 <= c->BZ))
        return fail(c, EIK_EINVAL, "eik_slab_set: need 0 <= own_bz0 < own_bz1 <= brick planes of the grid");
    if (!(zoff >= 0 && zoff % 8 == 0 && zoff + c->nz <= nz_all))
        return fail(c, EIK_EINVAL, "eik_slab_set: need zoff >= 0, a multiple of 8, and zoff + nz <= nz_all");
    if (!c->src.empty()) return fail(c, EIK_ESTATE, "eik_slab_set: call it before adding sources");
    c->own_bz0 = own_bz0;
    c->own_bz1 = own_bz1;
    c->zoff = zoff;
    c->nz_all = nz_all;
    c->slab = true;
    return EIK_OK;
}

eik_status eik_slab_begin(eik_ctx* c, double stride) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_slab_begin: ctx is NULL");
    if (!c->slab) return fail(c, EIK_ESTATE, "eik_slab_begin: no slab set (eik_slab_set)");
    if (c->in_flight || c->slab_running) return fail(c, EIK_ESTATE, "eik_slab_begin: a solve is in flight");
    // (no source is fine: a slab without one starts with an empty work list and gets work through imports)
    if (!(stride > 0.0) || std::isinf(stride)) return fail(c, EIK_EINVAL, "eik_slab_begin: stride must be finite and > 0");
    eik_status st = check_speed(c);
    if (st != EIK_OK) return st;
    eik_params P;
    eik_params_default(&P);
    P.stride = stride;
    P.block_dim = 8;
    P.width = INFINITY;
    c->params = P;
    c->last_edge = 8;
    st = (c->prec == EIK_FP32) ? queue_solve<float>(c, P, true) : queue_solve<double>(c, P, true);
    if (st != EIK_OK) return st;
    c->slab_running = true;
    c->solved = false;
    return EIK_OK;
}

namespace {
// Entries of the next restart's brick list (after a restart, or after imports).
eik_status slab_pending(eik_ctx* c, int64_t* pending) {
    eikg::Ctrl H{};
    EIK_CK(c, cudaStreamSynchronize(c->stream));
    EIK_CK(c, cudaMemcpy(&H, c->ctrl, sizeof(H), cudaMemcpyDeviceToHost));
    c->host_ctrl = H;
    if (pending) *pending = H.count[H.k % eikg::kRing];
    if (H.status & (eikg::kStWaitTimeout | eikg::kStRestartCap | eikg::kStRoundCap))
        return fail(c, EIK_ETIMEOUT, "sharded solve stopped early (restart cap, round cap or a device wait limit)");
    return EIK_OK;
}
}  // namespace

eik_status eik_slab_restart(eik_ctx* c, int64_t* pending) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_slab_restart: ctx is NULL");
    if (!c->slab_running) return fail(c, EIK_ESTATE, "eik_slab_restart: no sharded solve begun (eik_slab_begin)");
    EIK_CK(c, cudaMemsetAsync(&c->ctrl->done, 0, sizeof(int32_t), c->stream));
    if (c->prec == EIK_FP32) EIK_CK(c, eikg::launch_restart_loop<float>(c->lp_f, c->loop_grid, c->stream));
    else EIK_CK(c, eikg::launch_restart_loop<double>(c->lp_d, c->loop_grid, c->stream));
    return slab_pending(c, pending);
}

eik_status eik_slab_export(eik_ctx* c, int32_t side, void* buf) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_slab_export: ctx is NULL");
    if (!c->slab_running) return fail(c, EIK_ESTATE, "eik_slab_export: no sharded solve begun");
    if (!buf || (side != 0 && side != 1)) return fail(c, EIK_EINVAL, "eik_slab_export: side must be 0 or 1, buf not NULL");
    const int bz = side == 0 ? c->own_bz0 : c->own_bz1 - 1, face = side == 0 ? 4 : 5;
    if (c->prec == EIK_FP32)
        EIK_CK(c, eikg::launch_slab_export<float>(static_cast<const float*>(c->slot), c->ups, c->stamp, c->BX, c->BY, bz,
                                                  face, buf, c->stream));
    else
        EIK_CK(c, eikg::launch_slab_export<double>(static_cast<const double*>(c->slot), c->ups, c->stamp, c->BX, c->BY,
                                                   bz, face, buf, c->stream));
    EIK_CK(c, cudaStreamSynchronize(c->stream));
    return EIK_OK;
}

eik_status eik_slab_import(eik_ctx* c, int32_t side, const void* buf, int64_t* pending) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_slab_import: ctx is NULL");
    if (!c->slab_running) return fail(c, EIK_ESTATE, "eik_slab_import: no sharded solve begun");
    if (!buf || (side != 0 && side != 1)) return fail(c, EIK_EINVAL, "eik_slab_import: side must be 0 or 1, buf not NULL");
    const int gbz = side == 0 ? c->own_bz0 - 1 : c->own_bz1, obz = side == 0 ? c->own_bz0 : c->own_bz1 - 1;
    if (gbz < 0 || gbz >= c->BZ) return fail(c, EIK_EINVAL, "eik_slab_import: no ghost plane on that side");
    const int k_next = c->host_ctrl.k, k_done = k_next - 1;
    const int sn = k_next % eikg::kRing;
    int32_t* list_next = c->lists + static_cast<int64_t>(sn) * c->nbricks;
    if (c->prec == EIK_FP32)
        EIK_CK(c, eikg::launch_slab_import<float>(static_cast<float*>(c->slot), c->ups, c->stamp, c->BX, c->BY, gbz, obz,
                                                  buf, k_done, c->queued, c->nbricks, c->ctrl, list_next, c->stream));
    else
        EIK_CK(c, eikg::launch_slab_import<double>(static_cast<double*>(c->slot), c->ups, c->stamp, c->BX, c->BY, gbz,
                                                   obz, buf, k_done, c->queued, c->nbricks, c->ctrl, list_next,
                                                   c->stream));
    return slab_pending(c, pending);
}

eik_status eik_slab_end(eik_ctx* c, eik_stats* stats) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_slab_end: ctx is NULL");
    if (!c->slab_running) return fail(c, EIK_ESTATE, "eik_slab_end: no sharded solve begun");
    c->slab_running = false;
    if (c->nfix > 0) {
        if (c->prec == EIK_FP32)
            EIK_CK(c, eikg::launch_restore_r<float>(c->nfix, c->d_fix_b, c->d_fix_p, static_cast<const float*>(c->d_saved_r),
                                                    static_cast<float*>(c->rr), c->stream));
        else
            EIK_CK(c, eikg::launch_restore_r<double>(c->nfix, c->d_fix_b, c->d_fix_p,
                                                     static_cast<const double*>(c->d_saved_r), static_cast<double*>(c->rr),
                                                     c->stream));
    }
    eik_status st = slab_pending(c, nullptr);
    const eikg::Ctrl& H = c->host_ctrl;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->restarts = H.k - 1;
        stats->marches = static_cast<int64_t>(H.marches);
        stats->accepted = static_cast<int64_t>(H.accepted);
        stats->solves = static_cast<int64_t>(H.solves);
        stats->updates = static_cast<int64_t>(H.updates);
        stats->fallbacks = static_cast<int64_t>(H.fallbacks);
        stats->rounds = static_cast<int64_t>(H.rounds);
        stats->final_bound = H.bound_prev;
        stats->status = st;
        stats->block_dim = 8;
    }
    if (st == EIK_OK) c->solved = true;
    return st;
}

eik_status eik_restart_log(eik_ctx* c, eik_restart_rec* out, int64_t cap, int64_t* n) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_restart_log: ctx is NULL");
    if (!n || (cap > 0 && !out)) return fail(c, EIK_EINVAL, "eik_restart_log: NULL output");
    if (c->in_flight) return fail(c, EIK_ESTATE, "eik_restart_log: a solve is in flight");
    if (!c->params.log_restarts || !c->log) {
        *n = 0;
        return EIK_OK;
    }
    int64_t cnt = std::min<int64_t>(c->last_nr, c->log_cap);
    cnt = std::min<int64_t>(cnt, cap);
    static_assert(sizeof(eik_restart_rec) == sizeof(eikg::RestartRec), "record layout");
    if (cnt > 0) EIK_CK(c, cudaMemcpy(out, c->log, sizeof(eik_restart_rec) * cnt, cudaMemcpyDeviceToHost));
    *n = cnt;
    return EIK_OK;
}

eik_status eik_result(eik_ctx* c, void* out, int out_on_device) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_result: ctx is NULL");
    if (!out) return fail(c, EIK_EINVAL, "eik_result: psi_out is NULL");
    if (c->in_flight) return fail(c, EIK_ESTATE, "eik_result: a solve is in flight (call eik_wait)");
    if (!c->solved) return fail(c, EIK_ESTATE, "eik_result: no successful solve yet");
    eik_status st = eik_result_async(c, out, out_on_device);
    if (st != EIK_OK) return st;
    EIK_CK(c, cudaStreamSynchronize(c->stream));
    return EIK_OK;
}

eik_status eik_result_async(eik_ctx* c, void* out, int out_on_device) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_result_async: ctx is NULL");
    if (!out) return fail(c, EIK_EINVAL, "eik_result_async: psi_out is NULL");
    if (c->in_flight) return fail(c, EIK_ESTATE, "eik_result_async: a solve is in flight (call eik_wait)");
    if (!c->solved) return fail(c, EIK_ESTATE, "eik_result_async: no successful solve yet");
    if (out_on_device) {
        EIK_CK(c, queue_result(c, out));
        return EIK_OK;
    }
    const size_t bytes = static_cast<size_t>(c->nx) * c->ny * c->nz * c->esz;
    const eik_status st = ensure_stage(c, bytes);
    if (st != EIK_OK) return st;
    EIK_CK(c, queue_result(c, c->fstage));
    // the conversion is done before returning, so that work the caller queues
    // next (another context's solve) cannot hold the SMs it needs; the copy to
    // host memory then runs on a copy engine
    EIK_CK(c, cudaStreamSynchronize(c->stream));
    EIK_CK(c, cudaMemcpyAsync(out, c->fstage, bytes, cudaMemcpyDeviceToHost, c->stream));
    return EIK_OK;
}

eik_status eik_sync(eik_ctx* c) {
    if (!c) return fail(nullptr, EIK_EINVAL, "eik_sync: ctx is NULL");
    EIK_CK(c, cudaStreamSynchronize(c->stream));
    return check_speed(c);
}

void eik_destroy(eik_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);     // a solve or an asynchronous copy may still use the buffers
    free_all(c);
    delete c;
}

}  // extern "C"
