// Batched solves: many independent grids in one cooperative persistent launch
// (no counterpart in the paper, which solves one grid at a time).
//
// The bricks of all grids form one index space (grid s owns the bricks
// [boff_s, boff_s + nbricks_s) and the groups [goff_s, goff_s + ngroups_s));
// per-brick and per-group tables give the owning grid.  Every restart of the
// launch hands out one shared work queue: first the 2x2x2 groups of the
// grids marched with 16^3 blocks (one CTA each), then the bricks of the grids
// marched with 8^3 blocks (one warp each).  Grid s runs Alg. 6 with its own
// stride: its bound at restart k is k * stride_s.  One grid barrier per
// restart serves all grids; a grid is finished after the last restart in
// which one of its blocks marched, and its latency is the end of that restart.
//
// Tile shapes (block edge and stride of each grid, CTAs per SM) are picked by
// eik_batch_autotune: successive halving over a candidate table, every
// candidate timed by running the whole batch on the device.
#include "eik.h"
#include "eik_host.h"
#include "eik_internal.cuh"
#include "eik_march.cuh"

#include <algorithm>
#include <cmath>
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
cudaError_t launch_gather_r(int, const int32_t*, const int32_t*, const T*, double*, cudaStream_t);
template <typename T>
cudaError_t launch_result(const T*, const unsigned long long*, T*, int, int, int, int, int, int, cudaStream_t);

// Restart bookkeeping of a batched launch (run by lane 0 of the warp that
// reaches the barrier last): end time of the restart, totals, exit test.
template <typename T>
__device__ void batch_restart_end(const LoopParams<T>& P) {
    Ctrl* C = P.ctrl;
    const int k = __ldcg(&C->k);
    const int par = k % kRing, s1 = (k + 1) % kRing;
    const int n_next = __ldcg(&C->count[s1]) + __ldcg(&C->gcount[s1]);
    const unsigned long long now = globaltimer();
    if (P.tend != nullptr && k - 1 < P.tend_cap) P.tend[k - 1] = now;
    C->marches += static_cast<unsigned long long>(__ldcg(&C->count[par])) +
                  8ull * static_cast<unsigned long long>(__ldcg(&C->gcount[par]));
    C->accepted += __ldcg(&C->r_accepted);
    C->solves += __ldcg(&C->r_solves);
    C->updates += __ldcg(&C->r_updates);
    C->fallbacks += __ldcg(&C->r_fallbacks);
    C->rounds += __ldcg(&C->r_rounds);
    C->r_accepted = 0;
    C->r_band = 0;
    C->r_solves = 0;
    C->r_updates = 0;
    C->r_fallbacks = 0;
    C->r_rounds = 0;
    C->used[par] = __ldcg(&C->count[par]);
    C->count[par] = 0;
    C->head[par] = 0;
    C->gcount[par] = 0;
    C->ghead[par] = 0;
    if (n_next == 0 || (__ldcg(&C->status) & kStWaitTimeout)) {
        // (no work left, or a wait somewhere ran out: no warp starts another restart)
        C->done = 1;
        C->t_end = now;
    } else if (k >= P.max_restarts) {
        C->done = 1;
        C->status |= kStRestartCap;
        C->t_end = now;
    } else {
        C->k = k + 1;
        C->t_restart = now;
    }
}

// bound_band of grid sv at restart j (Alg. 6 with bound_j = j * stride; -1 for
// j = 0, so that every finite value is in the first band), from the table the
// restart bookkeeping keeps three restarts ahead (read from L2: other SMs write it)
template <typename T>
__device__ __forceinline__ T batch_bound(const LoopParams<T>& P, int sv, int j) {
    return __ldcg(P.gbound + static_cast<int64_t>(j % kRing) * P.nsolves + sv);
}
// At the end of restart k (the last warp at the barrier, every lane): the
// bounds of restart k + 2, into the ring slot of restart k - 2
template <typename T>
__device__ __forceinline__ void batch_bounds_ahead(const LoopParams<T>& P, int k, int lane) {
    const int j = k + 2;
    for (int sv = lane; sv < P.nsolves; sv += 32)
        P.gbound[static_cast<int64_t>(j % kRing) * P.nsolves + sv] =
            bound_down<T>(static_cast<double>(j) * P.solves[sv].stride);
    __threadfence();
}

template <typename T>
__global__ void __launch_bounds__(kWarps * 32, 3) k_batch_loop(LoopParams<T> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ int s_arrived;
    __shared__ LoopState s_state[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<T>* SW = reinterpret_cast<WarpSmem<T>*>(smem_raw);
    LoopState& L = s_state[warp];              // the loop's bookkeeping, kept out of registers
    Ctrl* C = P.ctrl;
    if (threadIdx.x == 0) s_arrived = 0;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer();
        C->t_begin = t0;
        C->t_restart = t0;
    }
    if (lane == 0) L.claim = -1;
    MarchAcc acc{0u, 0u, 0, 0u, 0u, 0u, __int_as_float(0x7f800000), 0.0f};
    bool any = false;
    for (;;) {
        const int k = __ldcg(&C->k);
        const int s = k % kRing;
        const bool early_k = P.early != 0;
        if (P.early) clear_used_slot(P, k);
        // ---- 16^3 blocks: one CTA per group of 2x2x2 bricks (the CTA goes on only as a whole)
        if (!cta_go(C, true, lane, &s_arrived)) return;
        {
            const int n = __ldcg(&C->gcount[s]);
            for (;;) {
                __syncthreads();
                if (threadIdx.x == 0) {
                    const int i = atomicAdd(&C->ghead[s], 1);
                    s_item = -1;
                    if (i < n) s_item = __ldcg(P.glist[s] + i);
                }
                __syncthreads();
                const int g = s_item;
                if (g < 0) break;
                const int sv = __ldg(P.gsolve + g);
                const SolveDesc D = P.solves[sv];
                const Geo G{D.BX, D.BY, D.BZ, D.boff, D.GX, D.GY, D.goff, 2u};
                const int gl = g - D.goff;
                const int gx = gl % D.GX, gy = (gl / D.GX) % D.GY, gz = gl / (D.GX * D.GY);
                const int bx = 2 * gx + (warp & 1), by = 2 * gy + ((warp >> 1) & 1), bz = 2 * gz + (warp >> 2);
                const bool in = bx < D.BX && by < D.BY && bz < D.BZ;
                const int32_t b = in ? D.boff + (bz * D.BY + by) * D.BX + bx : -1;
                unsigned gmask = 0;
                if (in) {
                    if (warp & 1) gmask |= 1u;
                    else if (bx + 1 < D.BX) gmask |= 2u;
                    if (warp & 2) gmask |= 4u;
                    else if (by + 1 < D.BY) gmask |= 8u;
                    if (warp & 4) gmask |= 16u;
                    else if (bz + 1 < D.BZ) gmask |= 32u;
                }
                march<T, true>(P, G, SW, warp, b, gmask, k, batch_bound(P, sv, k - 1), batch_bound(P, sv, k), true,
                               pick<T>(P.window, P.window_f), lane, acc, early_k);
                if (threadIdx.x == 0) atomicMax(P.last_k + sv, k);
                any = true;
            }
        }
        // ---- 8^3 blocks, one warp per brick: this restart's list, then -- once
        // arrived at the barrier -- restart k+1's bricks whose neighbourhood has
        // finished restart k.  One march call site for both.
        if (lane == 0) {
            L.n = __ldcg(&C->count[s]);
            L.waiting = 0;
            L.polls = 0;
            L.nap = 256;
        }
        __syncwarp();
        for (;;) {
            int32_t b = -1;
            int kk = k;
            if (!L.waiting) {
                int i = -1;
                if (lane == 0) {
                    const int n = L.n;
                    if (L.claim >= 0 && L.claim < n) i = L.claim;    // claimed before the entry existed
                    else {
                        const int j = atomicAdd(&C->head[s], 1);
                        if (j < n) i = j;
                    }
                    L.claim = -1;
                }
                i = __shfl_sync(kFull, i, 0);
                if (i >= 0) b = take_entry(P.list[s], i, false, 0, lane);
                if (b < 0) {
                    if (any) flush_acc(C, acc, lane);
                    any = false;
                    unsigned gen;
                    if (barrier_arrive(C, lane, &gen)) {
                        batch_bounds_ahead(P, k, lane);
                        if (lane == 0) batch_restart_end<T>(P);
                        barrier_release(C, lane, gen);
                        break;
                    }
                    if (lane == 0) {
                        L.gen = gen;
                        L.waiting = 1;
                    }
                    __syncwarp();
                    continue;
                }
            } else {
                const int st = barrier_poll(C, lane, L.gen);
                if (st == 2) return;
                if (st == 1) break;
                if (early_k) {
                    int claim = L.claim;
                    b = early_entry(C, P.list[(k + 1) % kRing], (k + 1) % kRing, claim, P.wait_limit, lane);
                    if (lane == 0) L.claim = claim;
                }
                if (b >= 0) {
                    const SolveDesc D = P.solves[__ldg(P.bsolve + b)];
                    const Geo G{D.BX, D.BY, D.BZ, D.boff, D.GX, D.GY, D.goff, 1u};
                    if (!wait_ready(P, G, b, k, lane)) b = -2;
                }
                if (b == -2) {
                    give_up(C, lane);
                    return;
                }
                if (b < 0) {
                    int quit = 0;
                    unsigned nap = 0;
                    if (lane == 0) {
                        quit = ++L.polls > P.wait_limit;
                        nap = L.nap;
                        if (L.nap < 4096) L.nap <<= 1;
                    }
                    if (__shfl_sync(kFull, quit, 0)) {
                        give_up(C, lane);
                        return;
                    }
                    __nanosleep(__shfl_sync(kFull, nap, 0));
                    continue;
                }
                kk = k + 1;
                if (lane == 0) {
                    L.polls = 0;
                    L.nap = 256;
                }
            }
            __syncwarp();
            const int sv = __ldg(P.bsolve + b);
            const SolveDesc D = P.solves[sv];
            const Geo G{D.BX, D.BY, D.BZ, D.boff, D.GX, D.GY, D.goff, 1u};
            march<T, false>(P, G, SW, warp, b, 0u, kk, batch_bound(P, sv, kk - 1), batch_bound(P, sv, kk), true,
                            pick<T>(P.window, P.window_f), lane, acc, early_k || kk > k);
            if (lane == 0) atomicMax(P.last_k + sv, kk);
            any = true;
        }
        if (__ldcg(&C->done)) return;
    }
}

// Smallest positive finite h/F of n values, as the bit pattern of a double
// (for positive doubles the unsigned order of the bits is the numeric order).
template <typename T>
__global__ void k_rmin(const T* __restrict__ rr, int64_t n, unsigned long long* out) {
    __shared__ double s_m[32];
    double m = __longlong_as_double(0x7ff0000000000000LL);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double r = static_cast<double>(rr[t]);
        if (r > 0.0 && r < m) m = r;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) m = fmin(m, s_m[w]);
        atomicMin(out, static_cast<unsigned long long>(__double_as_longlong(m)));
    }
}

// Owner tables: brick -> grid and group -> grid.
__global__ void k_owner(int32_t* __restrict__ tab, int64_t n, const int32_t* __restrict__ first, int ngrids) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int lo = 0, hi = ngrids - 1;          // last grid whose first index <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        tab[t] = lo;
    }
}

template <typename T>
size_t batch_smem_bytes() {
    return sizeof(WarpSmem<T>) * kWarps;
}

template <typename T>
cudaError_t batch_occupancy(int* blocks_per_sm) {
    const size_t smem = batch_smem_bytes<T>();
    cudaError_t e = cudaFuncSetAttribute(k_batch_loop<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_loop<T>, kWarps * 32, smem);
}

template <typename T>
cudaError_t launch_batch_loop(const LoopParams<T>& P, int grid, cudaStream_t s) {
    LoopParams<T> copy = P;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_batch_loop<T>), dim3(grid), dim3(kWarps * 32),
                                       args, batch_smem_bytes<T>(), s);
}

}  // namespace eikg

using eikg::kBrick;
using eikg::kSlot;

namespace {

struct BGrid {
    int nx, ny, nz;
    double h;
    eikh::Bricks geo;
    int64_t nb;
    int GX, GY, GZ;
    int32_t goff;
    int64_t ng;
    std::vector<eikh::FixNode> fix;
    std::vector<int32_t> sb, enq, genq;   // global brick / group indices
    double rmin;                          // smallest h/F over the grid (+inf: none)
};

}  // namespace

struct eik_batch {
    int n = 0;
    eik_precision prec = EIK_FP32;
    size_t esz = 4;
    cudaStream_t stream = nullptr;
    int sms = 0;
    int per_sm_max = 0;
    std::vector<BGrid> g;
    int64_t nbricks = 0, ngroups = 0;
    void* rr = nullptr;
    void* slot = nullptr;
    unsigned long long* ups = nullptr;
    unsigned long long* stamp = nullptr;
    int32_t* queued = nullptr;     // kRing x nbricks (ring slots)
    int32_t* lists = nullptr;      // kRing x nbricks
    int32_t* done = nullptr;       // per brick
    int32_t* qgroup = nullptr;     // kRing x ngroups
    int32_t* glists = nullptr;     // kRing x ngroups
    eikg::Ctrl* ctrl = nullptr;
    int* err_flag = nullptr;
    eikg::SolveDesc* d_solves = nullptr;
    int32_t* bsolve = nullptr;
    int32_t* gsolve = nullptr;
    int32_t* last_k = nullptr;
    unsigned long long* tend = nullptr;
    int64_t tend_cap = 0;
    int32_t* d_fix_b = nullptr;
    int32_t* d_fix_p = nullptr;
    double* d_fix_v = nullptr;
    void* d_saved_r = nullptr;
    int32_t* d_sb = nullptr;
    int32_t* d_enq = nullptr;
    int32_t* d_genq = nullptr;
    unsigned long long* d_rmin = nullptr;
    void* gbound = nullptr;        // kRing x n bounds (LoopParams::gbound)
    int nfix = 0, nsb = 0;
    std::vector<eik_batch_tile> tuned;    // autotuned tiles (empty: none)
    int tuned_ctas = 0;
    std::vector<eik_batch_tile> cur;      // tiles of the last solve
    int cur_ctas = 0;
    bool in_flight = false;
    bool solved = false;
    eikg::Ctrl host_ctrl{};
    std::string err;
};

namespace {

thread_local std::string g_batch_create_error;

eik_status bfail(eik_batch* b, eik_status s, const std::string& m) {
    if (b) b->err = m;
    else g_batch_create_error = m;
    return s;
}

#define EIKB_CK(bt, call)                                                                                   \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return bfail((bt), e_ == cudaErrorMemoryAllocation ? EIK_ENOMEM : EIK_ECUDA,                    \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                               \
    } while (0)

void bfree_all(eik_batch* b) {
    void* ptrs[] = {b->rr,       b->slot,     b->ups,      b->stamp,  b->queued,  b->lists,   b->done,
                    b->qgroup,   b->glists,   b->ctrl,     b->err_flag, b->d_solves, b->bsolve,
                    b->gsolve,   b->last_k,   b->tend,     b->d_fix_b, b->d_fix_p, b->d_fix_v, b->d_saved_r,
                    b->d_sb,     b->d_enq,    b->d_genq,   b->d_rmin,   b->gbound};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

template <typename P>
cudaError_t balloc(P** p, size_t bytes) {
    return cudaMalloc(reinterpret_cast<void**>(p), bytes < 16 ? 16 : bytes);
}

// bound_band of restart j with the given stride in precision T, rounded down as
// the device's bound_down does (-1 for j = 0)
template <typename T>
T host_bound_down(int j, double stride);
template <>
float host_bound_down<float>(int j, double stride) {
    if (j == 0) return -1.0f;
    const double d = static_cast<double>(j) * stride;
    float f = static_cast<float>(d);
    if (static_cast<double>(f) > d) f = std::nextafter(f, -INFINITY);
    return f;
}
template <>
double host_bound_down<double>(int j, double stride) {
    return j == 0 ? -1.0 : static_cast<double>(j) * stride;
}

bool tile_ok(const eik_batch_tile& t) {
    return (t.block_dim == 8 || t.block_dim == 16) && std::isfinite(t.stride) && t.stride > 0.0;
}

// Speeds -> h/F in brick layout for every grid, fixed nodes, owner tables.
template <typename T>
eik_status batch_setup(eik_batch* b, const eik_batch_item* items) {
    cudaStream_t s = b->stream;
    EIKB_CK(b, cudaMemsetAsync(b->err_flag, 0, sizeof(int), s));
    void* stage = nullptr;
    size_t stage_cap = 0;
    auto release = [&]() {
        if (stage) cudaFree(stage);
        stage = nullptr;
    };
    for (int i = 0; i < b->n; ++i) {
        const BGrid& G = b->g[i];
        const size_t bytes = static_cast<size_t>(G.nx) * G.ny * G.nz * sizeof(T);
        const void* Fd = items[i].F;
        if (!items[i].F_on_device) {
            if (bytes > stage_cap) {
                cudaStreamSynchronize(s);
                release();
                stage_cap = 0;
                const cudaError_t e = cudaMalloc(&stage, bytes);
                if (e != cudaSuccess) return bfail(b, EIK_ENOMEM, "eik_batch_create: staging allocation failed");
                stage_cap = bytes;
            }
            cudaError_t e = cudaMemcpyAsync(stage, items[i].F, bytes, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                release();
                return bfail(b, EIK_ECUDA, std::string("eik_batch_create: speed upload: ") + cudaGetErrorString(e));
            }
            Fd = stage;
        }
        T* rr = static_cast<T*>(b->rr) + static_cast<int64_t>(G.geo.boff) * kBrick;
        cudaError_t e = eikg::launch_layout_speed<T>(static_cast<const T*>(Fd), rr, G.nx, G.ny, G.nz, G.geo.BX,
                                                     G.geo.BY, G.nb, G.h, b->err_flag, 1, s);
        if (e == cudaSuccess) {
            const int rg = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(1024, (G.nb * kBrick + 255) / 256)));
            eikg::k_rmin<T><<<rg, 256, 0, s>>>(rr, G.nb * kBrick, b->d_rmin + i);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && !items[i].F_on_device) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            release();
            return bfail(b, EIK_ECUDA, std::string("eik_batch_create: speed layout: ") + cudaGetErrorString(e));
        }
    }
    EIKB_CK(b, cudaStreamSynchronize(s));
    release();
    int bad = 0;
    EIKB_CK(b, cudaMemcpy(&bad, b->err_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) return bfail(b, EIK_EINVAL, "eik_batch_create: F must be finite and >= 0 everywhere");
    std::vector<unsigned long long> rbits(b->n);
    EIKB_CK(b, cudaMemcpy(rbits.data(), b->d_rmin, sizeof(unsigned long long) * b->n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < b->n; ++i) {
        double r;
        std::memcpy(&r, &rbits[i], sizeof(r));
        b->g[i].rmin = r;
    }

    // ---- fixed nodes of every grid: candidates, their h/F, then Alg. 1
    std::vector<eikh::Cand> cand;
    std::vector<size_t> cfirst(b->n + 1, 0);
    for (int i = 0; i < b->n; ++i) {
        const BGrid& G = b->g[i];
        eikh::source_candidates(items[i].xyz, items[i].nsrc, G.nx, G.ny, G.nz, G.h, G.geo, cand);
        cfirst[i + 1] = cand.size();
    }
    const int nc = static_cast<int>(cand.size());
    std::vector<int32_t> cb(nc), cp(nc);
    for (int t = 0; t < nc; ++t) {
        cb[t] = cand[t].b;
        cp[t] = cand[t].p;
    }
    std::vector<double> cr(nc);
    {
        int32_t *d_cb = nullptr, *d_cp = nullptr;
        double* d_cr = nullptr;
        cudaError_t e = balloc(&d_cb, nc * 4);
        if (e == cudaSuccess) e = balloc(&d_cp, nc * 4);
        if (e == cudaSuccess) e = balloc(&d_cr, nc * 8);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_cb, cb.data(), nc * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_cp, cp.data(), nc * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = eikg::launch_gather_r<T>(nc, d_cb, d_cp, static_cast<const T*>(b->rr), d_cr, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cr.data(), d_cr, nc * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (d_cb) cudaFree(d_cb);
        if (d_cp) cudaFree(d_cp);
        if (d_cr) cudaFree(d_cr);
        if (e != cudaSuccess) return bfail(b, EIK_ECUDA, std::string("eik_batch_create: sources: ") + cudaGetErrorString(e));
    }
    std::vector<int32_t> fb, fp, sb;
    std::vector<double> fv;
    size_t max_enq = 0, max_genq = 0;
    for (int i = 0; i < b->n; ++i) {
        BGrid& G = b->g[i];
        std::vector<eikh::Cand> ci(cand.begin() + cfirst[i], cand.begin() + cfirst[i + 1]);
        std::vector<double> ri(cr.begin() + cfirst[i], cr.begin() + cfirst[i + 1]);
        G.fix = eikh::fixed_nodes(ci, ri, G.h);
        eikh::first_active(G.fix, G.geo, G.sb, G.enq);
        G.genq = eikh::groups_of(G.enq, G.geo, G.GX, G.GY, G.goff);
        for (const auto& f : G.fix) {
            fb.push_back(f.b);
            fp.push_back(f.p);
            fv.push_back(f.v);
        }
        sb.insert(sb.end(), G.sb.begin(), G.sb.end());
        max_enq += G.enq.size();
        max_genq += G.genq.size();
    }
    b->nfix = static_cast<int>(fb.size());
    b->nsb = static_cast<int>(sb.size());
    EIKB_CK(b, balloc(&b->d_fix_b, fb.size() * 4));
    EIKB_CK(b, balloc(&b->d_fix_p, fp.size() * 4));
    EIKB_CK(b, balloc(&b->d_fix_v, fv.size() * 8));
    EIKB_CK(b, balloc(&b->d_saved_r, fb.size() * sizeof(T)));
    EIKB_CK(b, balloc(&b->d_sb, sb.size() * 4));
    EIKB_CK(b, balloc(&b->d_enq, max_enq * 4));
    EIKB_CK(b, balloc(&b->d_genq, max_genq * 4));
    if (!fb.empty()) {
        EIKB_CK(b, cudaMemcpy(b->d_fix_b, fb.data(), fb.size() * 4, cudaMemcpyHostToDevice));
        EIKB_CK(b, cudaMemcpy(b->d_fix_p, fp.data(), fp.size() * 4, cudaMemcpyHostToDevice));
        EIKB_CK(b, cudaMemcpy(b->d_fix_v, fv.data(), fv.size() * 8, cudaMemcpyHostToDevice));
        EIKB_CK(b, cudaMemcpy(b->d_sb, sb.data(), sb.size() * 4, cudaMemcpyHostToDevice));
    }

    // ---- owner tables
    std::vector<int32_t> bfirst(b->n), gfirst(b->n);
    for (int i = 0; i < b->n; ++i) {
        bfirst[i] = b->g[i].geo.boff;
        gfirst[i] = b->g[i].goff;
    }
    int32_t* d_first = nullptr;
    EIKB_CK(b, balloc(&d_first, b->n * 4 * 2));
    cudaError_t e = cudaMemcpy(d_first, bfirst.data(), b->n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_first + b->n, gfirst.data(), b->n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        eikg::k_owner<<<static_cast<int>(std::min<int64_t>(4096, (b->nbricks + 255) / 256)), 256, 0, s>>>(
            b->bsolve, b->nbricks, d_first, b->n);
        eikg::k_owner<<<static_cast<int>(std::min<int64_t>(4096, (b->ngroups + 255) / 256)), 256, 0, s>>>(
            b->gsolve, b->ngroups, d_first + b->n, b->n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_first);
    if (e != cudaSuccess) return bfail(b, EIK_ECUDA, std::string("eik_batch_create: owner tables: ") + cudaGetErrorString(e));
    return EIK_OK;
}

// Queue one batched solve with the given tiles on the batch's stream.
template <typename T>
eik_status batch_queue(eik_batch* b, const std::vector<eik_batch_tile>& tiles, int ctas_per_sm,
                       const eik_batch_params& P) {
    cudaStream_t s = b->stream;
    // descriptors and the first work lists follow each grid's block edge
    std::vector<eikg::SolveDesc> D(b->n);
    std::vector<int32_t> enq, genq;
    for (int i = 0; i < b->n; ++i) {
        const BGrid& G = b->g[i];
        eikg::SolveDesc& d = D[i];
        std::memset(&d, 0, sizeof(d));
        d.BX = G.geo.BX;
        d.BY = G.geo.BY;
        d.BZ = G.geo.BZ;
        d.boff = G.geo.boff;
        d.GX = G.GX;
        d.GY = G.GY;
        d.GZ = G.GZ;
        d.goff = G.goff;
        d.mode = tiles[i].block_dim;
        d.stride = tiles[i].stride;
        if (d.mode == 16) genq.insert(genq.end(), G.genq.begin(), G.genq.end());
        else enq.insert(enq.end(), G.enq.begin(), G.enq.end());
    }
    EIKB_CK(b, cudaMemcpyAsync(b->d_solves, D.data(), sizeof(eikg::SolveDesc) * b->n, cudaMemcpyHostToDevice, s));
    // bounds of restarts 0-2 (the kernel writes restart k + 2's at the end of restart k)
    std::vector<T> gb(static_cast<size_t>(eikg::kRing) * b->n);
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < b->n; ++i) gb[static_cast<size_t>(j) * b->n + i] = host_bound_down<T>(j, D[i].stride);
    EIKB_CK(b, cudaMemcpyAsync(b->gbound, gb.data(), sizeof(T) * gb.size(), cudaMemcpyHostToDevice, s));
    if (!enq.empty()) EIKB_CK(b, cudaMemcpyAsync(b->d_enq, enq.data(), enq.size() * 4, cudaMemcpyHostToDevice, s));
    if (!genq.empty())
        EIKB_CK(b, cudaMemcpyAsync(b->d_genq, genq.data(), genq.size() * 4, cudaMemcpyHostToDevice, s));
    // ---- Alg. 1 for every brick of every grid
    EIKB_CK(b, cudaMemsetAsync(b->stamp, 0xFF, static_cast<size_t>(b->nbricks) * 8, s));
    EIKB_CK(b, cudaMemsetAsync(b->queued, 0xFF, eikg::kRing * static_cast<size_t>(b->nbricks) * 4, s));
    EIKB_CK(b, cudaMemsetAsync(b->lists, 0xFF, eikg::kRing * static_cast<size_t>(b->nbricks) * 4, s));   // empty: -1
    EIKB_CK(b, cudaMemsetAsync(b->done, 0, static_cast<size_t>(b->nbricks) * 4, s));
    EIKB_CK(b, cudaMemsetAsync(b->qgroup, 0xFF, eikg::kRing * static_cast<size_t>(b->ngroups) * 4, s));
    EIKB_CK(b, cudaMemsetAsync(b->glists, 0xFF, eikg::kRing * static_cast<size_t>(b->ngroups) * 4, s));
    EIKB_CK(b, cudaMemsetAsync(b->last_k, 0, static_cast<size_t>(b->n) * 4, s));
    if (b->nfix > 0)
        EIKB_CK(b, eikg::launch_init_sources<T>(b->nfix, b->d_fix_b, b->d_fix_p, b->d_fix_v, b->nsb, b->d_sb,
                                                static_cast<int>(enq.size()), b->d_enq, static_cast<int>(genq.size()),
                                                b->d_genq, static_cast<T*>(b->slot), b->ups, b->stamp,
                                                b->queued + b->nbricks, b->qgroup + b->ngroups,
                                                static_cast<T*>(b->rr), static_cast<T*>(b->d_saved_r),
                                                b->lists + b->nbricks, b->glists + b->ngroups, s));
    eikg::Ctrl& H = b->host_ctrl;
    std::memset(&H, 0, sizeof(H));
    const bool work = !enq.empty() || !genq.empty();
    H.k = work ? 1 : 0;
    H.action = -1;
    H.pend_action = -1;
    H.count[1] = static_cast<int32_t>(enq.size());
    H.gcount[1] = static_cast<int32_t>(genq.size());
    H.r_rmin_bits = 0x7f800000u;
    H.done = work ? 0 : 1;
    EIKB_CK(b, cudaMemcpyAsync(b->ctrl, &H, sizeof(H), cudaMemcpyHostToDevice, s));
    if (work) {
        eikg::LoopParams<T> L{};
        L.slot = static_cast<T*>(b->slot);
        L.ups = b->ups;
        L.stamp = b->stamp;
        L.queued = b->queued;
        L.done = b->done;
        L.nbricks = b->nbricks;
        L.ngroups = b->ngroups;
        L.early = 1;
        L.rr = static_cast<const T*>(b->rr);
        for (int r = 0; r < eikg::kRing; ++r) {
            L.list[r] = b->lists + r * b->nbricks;
            L.glist[r] = b->glists + r * b->ngroups;
        }
        L.qgroup = b->qgroup;
        L.ctrl = b->ctrl;
        L.window = P.window;
        L.window_f = static_cast<float>(P.window);
        L.fallback_tau = P.fallback_tau;
        L.max_restarts = P.max_restarts;
        L.width = INFINITY;                    // full solves
        L.wait_limit = eikg::kWaitPolls;
        L.solves = b->d_solves;
        L.bsolve = b->bsolve;
        L.gsolve = b->gsolve;
        L.last_k = b->last_k;
        L.tend = b->tend;
        L.tend_cap = b->tend_cap;
        L.gbound = static_cast<T*>(b->gbound);
        L.nsolves = b->n;
        if (P.loop_events[0]) EIKB_CK(b, cudaEventRecord(static_cast<cudaEvent_t>(P.loop_events[0]), s));
        EIKB_CK(b, eikg::launch_batch_loop<T>(L, ctas_per_sm * b->sms, s));
        if (P.loop_events[1]) EIKB_CK(b, cudaEventRecord(static_cast<cudaEvent_t>(P.loop_events[1]), s));
    }
    b->cur = tiles;
    b->cur_ctas = ctas_per_sm;
    return EIK_OK;
}

void default_batch_params(eik_batch_params* p) {
    std::memset(p, 0, sizeof(*p));
    p->window = 2.0;
    p->fallback_tau = 0.125;
    p->max_restarts = int64_t(1) << 24;
}

eik_status resolve(eik_batch* b, const eik_batch_tile* tiles, const eik_batch_params* params,
                   std::vector<eik_batch_tile>& T, int& ctas, eik_batch_params& P) {
    default_batch_params(&P);
    if (params) {
        P = *params;
        if (P.window == 0.0) P.window = 2.0;
        if (P.fallback_tau == 0.0) P.fallback_tau = 0.125;
        if (P.max_restarts == 0) P.max_restarts = int64_t(1) << 24;
    }
    if (!(P.window >= 0.0) || !std::isfinite(P.window)) return bfail(b, EIK_EINVAL, "window must be finite and >= 0");
    if (!(P.fallback_tau >= 0.0) || !(P.fallback_tau <= 1.0))
        return bfail(b, EIK_EINVAL, "fallback_tau must lie in [0, 1]");
    if (P.max_restarts < 0) return bfail(b, EIK_EINVAL, "max_restarts must be >= 0");
    if (P.ctas_per_sm < 0 || P.ctas_per_sm > b->per_sm_max)
        return bfail(b, EIK_EINVAL,
                     "ctas_per_sm must lie in [0, " + std::to_string(b->per_sm_max) + "] on this device");
    T.resize(b->n);
    for (int i = 0; i < b->n; ++i) {
        if (tiles) T[i] = tiles[i];
        else if (!b->tuned.empty()) T[i] = b->tuned[i];
        else T[i] = eik_batch_tile{8, 2.0 * b->g[i].h};
        if (!tile_ok(T[i]))
            return bfail(b, EIK_EINVAL, "tile " + std::to_string(i) + ": block_dim must be 8 or 16 and stride finite, > 0");
    }
    ctas = P.ctas_per_sm;
    if (ctas == 0) ctas = b->tuned_ctas > 0 ? b->tuned_ctas : b->per_sm_max;
    return EIK_OK;
}

eik_status batch_finish(eik_batch* b, eik_batch_stats* stats) {
    EIKB_CK(b, cudaStreamSynchronize(b->stream));
    eikg::Ctrl H{};
    EIKB_CK(b, cudaMemcpy(&H, b->ctrl, sizeof(H), cudaMemcpyDeviceToHost));
    b->host_ctrl = H;
    eik_status st = EIK_OK;
    if (H.status & (eikg::kStWaitTimeout | eikg::kStRestartCap | eikg::kStRoundCap)) {
        st = EIK_ETIMEOUT;
        b->err = std::string("batched solve stopped early: ") +
                 ((H.status & eikg::kStRestartCap) ? "restart cap reached " : "") +
                 ((H.status & eikg::kStWaitTimeout) ? "grid-barrier wait limit reached " : "") +
                 ((H.status & eikg::kStRoundCap) ? "march round cap reached" : "");
    } else if (!H.done) {
        st = EIK_ECUDA;
        b->err = "batched solve did not finish";
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
        stats->status = st;
        stats->ctas = b->cur_ctas * b->sms;
    }
    b->solved = (st == EIK_OK);
    return st;
}

template <typename T>
eik_status batch_run_timed(eik_batch* b, const std::vector<eik_batch_tile>& tiles, int ctas,
                           const eik_batch_params& P, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    EIKB_CK(b, cudaEventRecord(e0, b->stream));
    eik_status st = batch_queue<T>(b, tiles, ctas, P);
    if (st != EIK_OK) return st;
    EIKB_CK(b, cudaEventRecord(e1, b->stream));
    st = batch_finish(b, nullptr);
    if (st != EIK_OK) return st;
    EIKB_CK(b, cudaEventElapsedTime(ms, e0, e1));
    return EIK_OK;
}

// Candidate table of the autotuner.  Stride of grid s: factor * h_s (per_h),
// or factor * edge * rmin_s with rmin_s = min h/F over the grid (the time a
// front at the largest speed takes to cross one block is edge * rmin_s; a
// larger stride lets the bound outrun what one exchange per restart carries);
// block edge 16 for the grids with at least `min16` bricks; launch with ctas
// CTAs per SM.
struct Cand {
    bool per_h;
    double factor;
    int64_t min16;
    int ctas;
};

std::vector<eik_batch_tile> tiles_of(const eik_batch* b, const Cand& c) {
    std::vector<eik_batch_tile> t(b->n);
    for (int i = 0; i < b->n; ++i) {
        const BGrid& G = b->g[i];
        const int e = (G.nb >= c.min16) ? 16 : 8;
        const double r = (std::isfinite(G.rmin) && G.rmin > 0.0) ? G.rmin : G.h;
        t[i] = eik_batch_tile{e, c.per_h ? c.factor * G.h : c.factor * e * r};
    }
    return t;
}

template <typename T>
eik_status autotune(eik_batch* b, int32_t rounds_cap, eik_batch_tile* tiles_out, int32_t* ctas_out, double* ms_out) {
    const double factors[] = {0.5, 0.75, 1.0, 1.5, 2.0};
    const double per_h[] = {1.25, 1.5, 1.75, 2.0, 2.5, 3.0, 4.0};
    const int64_t min16s[] = {INT64_MAX, 2048, 512, 0};
    std::vector<Cand> cands;
    for (int c = b->per_sm_max; c >= 1; --c)                 // the default tiles (8^3, 2h, all CTAs) first
        for (int64_t m : min16s) {
            for (double f : per_h) cands.push_back(Cand{true, f, m, c});
            for (double f : factors) cands.push_back(Cand{false, f, m, c});
        }
    eik_batch_params P;
    default_batch_params(&P);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    EIKB_CK(b, cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return bfail(b, EIK_ECUDA, "eik_batch_autotune: cudaEventCreate failed");
    }
    struct Score {
        size_t idx;
        std::vector<float> ms;
        float med() const {
            std::vector<float> v = ms;
            std::sort(v.begin(), v.end());
            return v[v.size() / 2];
        }
    };
    std::vector<Score> alive;
    for (size_t i = 0; i < cands.size(); ++i) alive.push_back(Score{i, {}});
    eik_status st = EIK_OK;
    float warm = 0.0f;
    st = batch_run_timed<T>(b, tiles_of(b, cands[0]), cands[0].ctas, P, e0, e1, &warm);   // warm-up
    int reps = 1, round = 0;
    while (st == EIK_OK && alive.size() > 1 && (rounds_cap <= 0 || round < rounds_cap)) {
        std::vector<Score> next;
        for (auto& a : alive) {
            bool ok = true;
            for (int r = 0; r < reps && ok; ++r) {
                float ms = 0.0f;
                const eik_status s1 = batch_run_timed<T>(b, tiles_of(b, cands[a.idx]), cands[a.idx].ctas, P, e0, e1, &ms);
                if (s1 == EIK_ETIMEOUT) ok = false;            // candidate hit a cap: drop it
                else if (s1 != EIK_OK) {
                    st = s1;
                    ok = false;
                } else {
                    a.ms.push_back(ms);
                }
            }
            if (st != EIK_OK) break;
            if (ok) next.push_back(a);
        }
        if (st != EIK_OK) break;
        std::sort(next.begin(), next.end(), [](const Score& x, const Score& y) { return x.med() < y.med(); });
        next.resize(std::max<size_t>(1, (next.size() + 2) / 3));
        alive.swap(next);
        reps *= 2;
        ++round;
    }
    if (st != EIK_OK || alive.empty()) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != EIK_OK) return st;
        return bfail(b, EIK_ETIMEOUT, "eik_batch_autotune: every candidate hit a cap");
    }
    std::sort(alive.begin(), alive.end(), [](const Score& x, const Score& y) {
        if (x.ms.empty() != y.ms.empty()) return !x.ms.empty();
        return !x.ms.empty() && x.med() < y.med();
    });
    const Cand& best = cands[alive[0].idx];
    std::vector<eik_batch_tile> win = tiles_of(b, best);
    float win_ms = alive[0].ms.empty() ? 0.0f : alive[0].med();

    // Stage 2, per grid: the launch lasts as long as its slowest grids.  The
    // grids that finish last under the stage-1 tiles (done_ms at or above a
    // quantile q of the grids) get a stride longer by a factor (fewer restarts
    // for them); or the grids that finish first (done_ms at or below q) get a
    // shorter one (less refresh work in the restarts all grids share, more
    // restarts for grids that are not the last to finish).  Candidates q x
    // factor, timed with the same successive halving against the stage-1 tiles.
    {
        float ms = 0.0f;
        st = batch_run_timed<T>(b, win, best.ctas, P, e0, e1, &ms);
        std::vector<eik_batch_solve_info> info(b->n);
        if (st == EIK_OK) st = eik_batch_info(b, info.data(), b->n);
        if (st == EIK_OK) {
            std::vector<double> done(b->n);
            for (int i = 0; i < b->n; ++i) done[i] = info[i].done_ms;
            std::vector<double> sorted = done;
            std::sort(sorted.begin(), sorted.end());
            std::vector<std::vector<eik_batch_tile>> tl{win};
            for (double q : {0.5, 0.75, 0.9})
                for (double f : {1.25, 1.5, 2.0}) {
                    const double thr = sorted[static_cast<size_t>(q * (b->n - 1))];
                    std::vector<eik_batch_tile> t = win;
                    for (int i = 0; i < b->n; ++i)
                        if (done[i] >= thr) t[i].stride *= f;
                    tl.push_back(t);
                }
            for (double q : {0.25, 0.5, 0.75})
                for (double f : {0.5, 0.75}) {
                    const double thr = sorted[static_cast<size_t>(q * (b->n - 1))];
                    std::vector<eik_batch_tile> t = win;
                    for (int i = 0; i < b->n; ++i)
                        if (done[i] <= thr) t[i].stride *= f;
                    tl.push_back(t);
                }
            std::vector<Score> alive2;
            for (size_t i = 0; i < tl.size(); ++i) alive2.push_back(Score{i, {}});
            int reps2 = 1, round2 = 0;
            while (st == EIK_OK && alive2.size() > 1 && (rounds_cap <= 0 || round2 < rounds_cap)) {
                std::vector<Score> next;
                for (auto& a : alive2) {
                    bool ok = true;
                    for (int r = 0; r < reps2 && ok; ++r) {
                        float m2 = 0.0f;
                        const eik_status s1 = batch_run_timed<T>(b, tl[a.idx], best.ctas, P, e0, e1, &m2);
                        if (s1 == EIK_ETIMEOUT) ok = false;
                        else if (s1 != EIK_OK) {
                            st = s1;
                            ok = false;
                        } else {
                            a.ms.push_back(m2);
                        }
                    }
                    if (st != EIK_OK) break;
                    if (ok) next.push_back(a);
                }
                if (st != EIK_OK) break;
                std::sort(next.begin(), next.end(), [](const Score& x, const Score& y) { return x.med() < y.med(); });
                next.resize(std::max<size_t>(1, (next.size() + 2) / 3));
                alive2.swap(next);
                reps2 *= 2;
                ++round2;
            }
            if (st == EIK_OK && !alive2.empty() && !alive2[0].ms.empty()) {
                std::sort(alive2.begin(), alive2.end(), [](const Score& x, const Score& y) { return x.med() < y.med(); });
                win = tl[alive2[0].idx];
                win_ms = alive2[0].med();
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != EIK_OK) return st;
    b->tuned = win;
    b->tuned_ctas = best.ctas;
    if (tiles_out) std::copy(b->tuned.begin(), b->tuned.end(), tiles_out);
    if (ctas_out) *ctas_out = best.ctas;
    if (ms_out) *ms_out = static_cast<double>(win_ms);
    return EIK_OK;
}

}  // namespace

extern "C" {

const char* eik_batch_last_error(const eik_batch* b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

void eik_batch_params_default(eik_batch_params* p) {
    if (p) default_batch_params(p);
}

eik_status eik_batch_create(eik_batch** out, int32_t n, const eik_batch_item* items, eik_precision precision,
                            void* stream) {
    if (!out) return bfail(nullptr, EIK_EINVAL, "eik_batch_create: out is NULL");
    *out = nullptr;
    if (n < 1 || !items) return bfail(nullptr, EIK_EINVAL, "eik_batch_create: need n >= 1 items");
    if (precision != EIK_FP32 && precision != EIK_FP64)
        return bfail(nullptr, EIK_EINVAL, "eik_batch_create: precision must be EIK_FP32 or EIK_FP64");
    int64_t nb = 0, ng = 0;
    for (int i = 0; i < n; ++i) {
        const eik_batch_item& it = items[i];
        const std::string w = "eik_batch_create: item " + std::to_string(i) + ": ";
        if (it.dims[0] < 1 || it.dims[1] < 1 || it.dims[2] < 1) return bfail(nullptr, EIK_EINVAL, w + "dims must be >= 1");
        if (int64_t(it.dims[0]) * it.dims[1] * it.dims[2] >= (int64_t(1) << 31))
            return bfail(nullptr, EIK_EINVAL, w + "nx*ny*nz must be < 2^31");
        if (!(std::isfinite(it.h) && it.h > 0.0)) return bfail(nullptr, EIK_EINVAL, w + "h must be finite and > 0");
        if (!it.F) return bfail(nullptr, EIK_EINVAL, w + "F is NULL");
        if (it.nsrc < 1 || !it.xyz) return bfail(nullptr, EIK_EINVAL, w + "needs nsrc >= 1 sources");
        const double tol = 1e-9 * it.h;
        for (int q = 0; q < it.nsrc; ++q)
            for (int a = 0; a < 3; ++a) {
                const double v = it.xyz[3 * q + a];
                if (!std::isfinite(v) || v < -tol || v > (it.dims[a] - 1) * it.h + tol)
                    return bfail(nullptr, EIK_EINVAL, w + "source " + std::to_string(q) + " lies outside the grid");
            }
        const int64_t BX = (it.dims[0] + 7) / 8, BY = (it.dims[1] + 7) / 8, BZ = (it.dims[2] + 7) / 8;
        nb += BX * BY * BZ;
        ng += ((BX + 1) / 2) * ((BY + 1) / 2) * ((BZ + 1) / 2);
    }
    if (nb >= (int64_t(1) << 31) / 2) return bfail(nullptr, EIK_EINVAL, "eik_batch_create: too many bricks in the batch");

    eik_batch* b = new (std::nothrow) eik_batch();
    if (!b) return bfail(nullptr, EIK_ENOMEM, "eik_batch_create: host allocation failed");
    auto bail = [&](eik_status s, const std::string& m) {
        bfree_all(b);
        delete b;
        return bfail(nullptr, s, m);
    };
    b->n = n;
    b->prec = precision;
    b->esz = precision == EIK_FP32 ? 4 : 8;
    b->stream = static_cast<cudaStream_t>(stream);
    b->g.resize(n);
    int64_t boff = 0, goff = 0;
    for (int i = 0; i < n; ++i) {
        BGrid& G = b->g[i];
        G.nx = items[i].dims[0];
        G.ny = items[i].dims[1];
        G.nz = items[i].dims[2];
        G.h = items[i].h;
        G.geo = eikh::Bricks{(G.nx + 7) / 8, (G.ny + 7) / 8, (G.nz + 7) / 8, static_cast<int32_t>(boff)};
        G.nb = int64_t(G.geo.BX) * G.geo.BY * G.geo.BZ;
        G.GX = (G.geo.BX + 1) / 2;
        G.GY = (G.geo.BY + 1) / 2;
        G.GZ = (G.geo.BZ + 1) / 2;
        G.goff = static_cast<int32_t>(goff);
        G.ng = int64_t(G.GX) * G.GY * G.GZ;
        G.rmin = 0.0;
        boff += G.nb;
        goff += G.ng;
    }
    b->nbricks = boff;
    b->ngroups = goff;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bail(EIK_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (!coop) return bail(EIK_ENOTSUP, "eik_batch_create: device lacks cooperative launch");
    const size_t nbz = static_cast<size_t>(b->nbricks), ngz = static_cast<size_t>(b->ngroups);
    b->tend_cap = int64_t(1) << 16;
    struct {
        void** p;
        size_t bytes;
    } allocs[] = {
        {&b->rr, nbz * kBrick * b->esz},
        {&b->slot, nbz * 2 * kSlot * b->esz},
        {reinterpret_cast<void**>(&b->ups), nbz * 2 * 6 * 8},
        {reinterpret_cast<void**>(&b->stamp), nbz * 8},
        {reinterpret_cast<void**>(&b->queued), eikg::kRing * nbz * 4},
        {reinterpret_cast<void**>(&b->lists), eikg::kRing * nbz * 4},
        {reinterpret_cast<void**>(&b->done), nbz * 4},
        {reinterpret_cast<void**>(&b->qgroup), eikg::kRing * ngz * 4},
        {reinterpret_cast<void**>(&b->glists), eikg::kRing * ngz * 4},
        {reinterpret_cast<void**>(&b->ctrl), sizeof(eikg::Ctrl)},
        {reinterpret_cast<void**>(&b->err_flag), sizeof(int)},
        {reinterpret_cast<void**>(&b->d_solves), sizeof(eikg::SolveDesc) * n},
        {reinterpret_cast<void**>(&b->bsolve), nbz * 4},
        {reinterpret_cast<void**>(&b->gsolve), ngz * 4},
        {reinterpret_cast<void**>(&b->last_k), static_cast<size_t>(n) * 4},
        {reinterpret_cast<void**>(&b->tend), static_cast<size_t>(b->tend_cap) * 8},
        {reinterpret_cast<void**>(&b->d_rmin), static_cast<size_t>(n) * 8},
        {&b->gbound, eikg::kRing * static_cast<size_t>(n) * b->esz},
    };
    for (auto& a : allocs) {
        e = balloc(a.p, a.bytes);
        if (e != cudaSuccess)
            return bail(EIK_ENOMEM, std::string("eik_batch_create: cudaMalloc of ") + std::to_string(a.bytes) +
                                        " bytes failed: " + cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(b->d_rmin, 0x7F, static_cast<size_t>(n) * 8, b->stream);   // 0x7F7F...: above every finite r
    if (e != cudaSuccess) return bail(EIK_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    {
        const eik_status st = (precision == EIK_FP32) ? batch_setup<float>(b, items) : batch_setup<double>(b, items);
        if (st != EIK_OK) {
            const std::string m = b->err;
            return bail(st, m);
        }
    }
    for (int i = 0; i < n; ++i)
        if (!(b->g[i].rmin < 1e300)) b->g[i].rmin = INFINITY;                            // no positive speed
    e = (precision == EIK_FP32) ? eikg::batch_occupancy<float>(&b->per_sm_max) : eikg::batch_occupancy<double>(&b->per_sm_max);
    if (e != cudaSuccess || b->per_sm_max < 1)
        return bail(EIK_ECUDA, std::string("eik_batch_create: occupancy query: ") + cudaGetErrorString(e));
    *out = b;
    return EIK_OK;
}

eik_status eik_batch_solve_async(eik_batch* b, const eik_batch_tile* tiles, const eik_batch_params* params) {
    if (!b) return bfail(nullptr, EIK_EINVAL, "eik_batch_solve_async: batch is NULL");
    if (b->in_flight) return bfail(b, EIK_ESTATE, "eik_batch_solve_async: a solve is already in flight");
    std::vector<eik_batch_tile> T;
    int ctas = 0;
    eik_batch_params P;
    eik_status st = resolve(b, tiles, params, T, ctas, P);
    if (st != EIK_OK) return st;
    st = (b->prec == EIK_FP32) ? batch_queue<float>(b, T, ctas, P) : batch_queue<double>(b, T, ctas, P);
    if (st != EIK_OK) return st;
    b->in_flight = true;
    b->solved = false;
    return EIK_OK;
}

eik_status eik_batch_wait(eik_batch* b, eik_batch_stats* stats) {
    if (!b) return bfail(nullptr, EIK_EINVAL, "eik_batch_wait: batch is NULL");
    if (!b->in_flight) return bfail(b, EIK_ESTATE, "eik_batch_wait: no solve in flight");
    b->in_flight = false;
    return batch_finish(b, stats);
}

eik_status eik_batch_solve(eik_batch* b, const eik_batch_tile* tiles, const eik_batch_params* params,
                           eik_batch_stats* stats) {
    const eik_status st = eik_batch_solve_async(b, tiles, params);
    if (st != EIK_OK) return st;
    return eik_batch_wait(b, stats);
}

eik_status eik_batch_info(eik_batch* b, eik_batch_solve_info* out, int32_t cap) {
    if (!b) return bfail(nullptr, EIK_EINVAL, "eik_batch_info: batch is NULL");
    if (!out || cap < b->n) return bfail(b, EIK_EINVAL, "eik_batch_info: out must hold n records");
    if (b->in_flight) return bfail(b, EIK_ESTATE, "eik_batch_info: a solve is in flight");
    if (!b->solved) return bfail(b, EIK_ESTATE, "eik_batch_info: no successful solve yet");
    std::vector<int32_t> lk(b->n);
    EIKB_CK(b, cudaMemcpy(lk.data(), b->last_k, sizeof(int32_t) * b->n, cudaMemcpyDeviceToHost));
    const int64_t nr = std::min<int64_t>(b->host_ctrl.k, b->tend_cap);
    std::vector<unsigned long long> te(std::max<int64_t>(nr, 1));
    if (nr > 0) EIKB_CK(b, cudaMemcpy(te.data(), b->tend, sizeof(unsigned long long) * nr, cudaMemcpyDeviceToHost));
    const unsigned long long t0 = b->host_ctrl.t_begin;
    for (int i = 0; i < b->n; ++i) {
        eik_batch_solve_info& r = out[i];
        std::memset(&r, 0, sizeof(r));
        r.restarts = lk[i];
        r.block_dim = b->cur[i].block_dim;
        r.stride = b->cur[i].stride;
        r.rmin = b->g[i].rmin;
        r.nbricks = b->g[i].nb;
        unsigned long long t = b->host_ctrl.t_end;
        if (lk[i] >= 1 && lk[i] <= nr) t = te[lk[i] - 1];
        r.done_ms = (lk[i] >= 1 && t > t0) ? static_cast<double>(t - t0) * 1e-6 : 0.0;
    }
    return EIK_OK;
}

eik_status eik_batch_result(eik_batch* b, int32_t i, void* out, int out_on_device) {
    if (!b) return bfail(nullptr, EIK_EINVAL, "eik_batch_result: batch is NULL");
    if (!out) return bfail(b, EIK_EINVAL, "eik_batch_result: psi_out is NULL");
    if (i < 0 || i >= b->n) return bfail(b, EIK_EINVAL, "eik_batch_result: index out of range");
    if (b->in_flight) return bfail(b, EIK_ESTATE, "eik_batch_result: a solve is in flight (call eik_batch_wait)");
    if (!b->solved) return bfail(b, EIK_ESTATE, "eik_batch_result: no successful solve yet");
    const BGrid& G = b->g[i];
    const size_t bytes = static_cast<size_t>(G.nx) * G.ny * G.nz * b->esz;
    void* dst = out;
    if (!out_on_device) EIKB_CK(b, cudaMalloc(&dst, bytes));
    const int64_t boff = G.geo.boff;
    cudaError_t e;
    if (b->prec == EIK_FP32)
        e = eikg::launch_result<float>(static_cast<const float*>(b->slot) + boff * 2 * kSlot, b->stamp + boff,
                                       static_cast<float*>(dst), G.nx, G.ny, 0, G.nz, G.geo.BX, G.geo.BY, b->stream);
    else
        e = eikg::launch_result<double>(static_cast<const double*>(b->slot) + boff * 2 * kSlot, b->stamp + boff,
                                        static_cast<double*>(dst), G.nx, G.ny, 0, G.nz, G.geo.BX, G.geo.BY, b->stream);
    if (e == cudaSuccess && !out_on_device) e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (!out_on_device) cudaFree(dst);
    if (e != cudaSuccess) return bfail(b, EIK_ECUDA, std::string("eik_batch_result: ") + cudaGetErrorString(e));
    return EIK_OK;
}

eik_status eik_batch_autotune(eik_batch* b, int32_t rounds, eik_batch_tile* tiles_out, int32_t* ctas_per_sm,
                              double* best_ms) {
    if (!b) return bfail(nullptr, EIK_EINVAL, "eik_batch_autotune: batch is NULL");
    if (b->in_flight) return bfail(b, EIK_ESTATE, "eik_batch_autotune: a solve is in flight");
    if (rounds < 0) return bfail(b, EIK_EINVAL, "eik_batch_autotune: rounds must be >= 0");
    return (b->prec == EIK_FP32) ? autotune<float>(b, rounds, tiles_out, ctas_per_sm, best_ms)
                                 : autotune<double>(b, rounds, tiles_out, ctas_per_sm, best_ms);
}

eik_status eik_batch_size(const eik_batch* b, int32_t* n, int64_t* nbricks, int32_t* max_ctas_per_sm) {
    if (!b) return bfail(nullptr, EIK_EINVAL, "eik_batch_size: batch is NULL");
    if (n) *n = b->n;
    if (nbricks) *nbricks = b->nbricks;
    if (max_ctas_per_sm) *max_ctas_per_sm = b->per_sm_max;
    return EIK_OK;
}

void eik_batch_destroy(eik_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);     // nothing queued may outlive the buffers
    bfree_all(b);
    delete b;
}

}  // extern "C"
