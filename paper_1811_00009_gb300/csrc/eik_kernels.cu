// Device kernels of libeik for one grid: the block-based restarted
// narrow-band fast marching method (J. Yang 2018, Alg. 6 with Algs. 1-5) on
// sm_103a.  The march itself (Algs. 2-5) is in eik_march.cuh.
//
// The restart loop of Alg. 6 runs in one cooperative persistent kernel with
// one grid-wide barrier per restart; the exchange step (Alg. 5) is fused into
// the start of the next march (see eik_internal.cuh for the double-copy
// layout that makes this race-free, the argument of Sec. 2.7).
#include "eik_internal.cuh"
#include "eik_march.cuh"
#include "eik_mlp.cuh"

#include <cfloat>
#include <cstdint>

namespace eikg {

// Features of the front after restart k for the schedule network (all O(1)):
// log-counts of marched bricks, band nodes, accepted nodes and solves; log of
// the largest and smallest speed over the marched bricks; the bound in grid
// lengths; log k; the stride in h; whether the blocks were 16^3.
__device__ inline void schedule_features(float* x, double active, double band, double accepted, double solves,
                                         double rmin, double rmax, double bound, double stride, int k, int mode,
                                         double h, int nmax) {
    // single precision throughout (the network is FP32; double logs are slow on this part)
    const float hf = static_cast<float>(h);
    x[0] = log1pf(static_cast<float>(active)) / 16.0f;
    x[1] = log1pf(static_cast<float>(band)) / 20.0f;
    x[2] = log1pf(static_cast<float>(accepted)) / 20.0f;
    x[3] = (rmin > 0.0 && rmin < 1e300) ? logf(hf / static_cast<float>(rmin)) : 0.0f;
    x[4] = (rmax > 0.0 && rmax < 1e300) ? logf(hf / static_cast<float>(rmax)) : 0.0f;
    x[5] = static_cast<float>(bound) / (hf * static_cast<float>(nmax));
    x[6] = log1pf(static_cast<float>(k)) / 8.0f;
    x[7] = static_cast<float>(stride) / hf / 4.0f;
    x[8] = (mode == 16) ? 1.0f : 0.0f;
    x[9] = log1pf(static_cast<float>(solves)) / 20.0f;
    for (int i = 0; i < kIn; ++i) {
        if (!(x[i] == x[i])) x[i] = 0.0f;
        x[i] = fminf(10.0f, fmaxf(-10.0f, x[i]));
    }
}

__device__ inline unsigned mix32(unsigned a) {
    a ^= a >> 16;
    a *= 0x7feb352du;
    a ^= a >> 15;
    a *= 0x846ca68bu;
    a ^= a >> 16;
    return a;
}

// Stride and block edge of restart k+1, known from the start of restart k: the
// schedules choose each restart's action one restart ahead (at the end of
// restart k-1), so that warps waiting at the barrier of restart k can march
// restart k+1's bricks early.  -1: restart k's own stride and block edge.
template <typename T>
__device__ __forceinline__ void next_restart_of(const LoopParams<T>& P, const Ctrl* C, double* stride, int* mode) {
    const int pa = __ldcg(&C->pend_action);
    if (pa >= 0) {
        *stride = action_stride_h(pa) * P.h;
        *mode = P.groups ? action_block(pa) : 8;
    } else {
        *stride = __ldcg(&C->stride);
        *mode = __ldcg(&C->mode);
    }
}

// Bookkeeping at the end of restart k (run by the warp that reaches the barrier
// last): statistics, exit test and the next bound of Alg. 6 (restart k+1 takes
// the action chosen at the end of restart k-1) and, for the learned schedule,
// the schedule network (one hidden unit per lane) choosing the stride and
// block edge of restart k+2 from the front after restart k.  `scratch` is the
// calling warp's shared tile (free while it waits at the barrier): the
// network's weights are staged there with coalesced loads.
template <typename T>
__device__ void restart_end(const LoopParams<T>& P, int lane, float* scratch) {
    static_assert(kHid == 32, "one hidden unit per lane");
    static_assert(sizeof(WarpSmem<T>) >= (kHid * (kIn + 1) + (kHid + kAct) * (kHid + 1)) * sizeof(float),
                  "the staged weights fit the warp's tile");
    __shared__ float s_x[kIn];
    __shared__ float s_h1[kHid];
    __shared__ float s_h2[kHid];
    __shared__ float s_y[kAct];
    Ctrl* C = P.ctrl;
    const int k = __ldcg(&C->k);
    const int mode = __ldcg(&C->mode);
    const int s = k % kRing, s1 = (k + 1) % kRing;
    const int n_this = (mode == 16) ? __ldcg(&C->gcount[s]) : __ldcg(&C->count[s]);
    if (lane == 0)
        schedule_features(s_x, static_cast<double>(n_this) * (mode == 16 ? 8 : 1),
                          static_cast<double>(__ldcg(&C->r_band)), static_cast<double>(__ldcg(&C->r_accepted)),
                          static_cast<double>(__ldcg(&C->r_solves)),
                          static_cast<double>(__uint_as_float(__ldcg(&C->r_rmin_bits))),
                          static_cast<double>(__uint_as_float(__ldcg(&C->r_rmax_bits))), __ldcg(&C->bound),
                          __ldcg(&C->stride), k, mode, P.h, P.nmax);
    __syncwarp();
    if (P.sched == 1 && P.mlp != nullptr) {
        // weight rows staged with a padded stride (11 and 33 floats), so that
        // the 32 lanes, one hidden unit each, read 32 different banks
        constexpr int kS1 = kIn + 1, kS2 = kHid + 1;
        float* w1 = scratch;
        float* w2 = w1 + kHid * kS1;
        float* w3 = w2 + kHid * kS2;
        for (int i = lane; i < kHid * kIn; i += 32) w1[(i / kIn) * kS1 + i % kIn] = __ldg(P.mlp + kOffW1 + i);
        for (int i = lane; i < kHid * kHid; i += 32) w2[(i >> 5) * kS2 + (i & 31)] = __ldg(P.mlp + kOffW2 + i);
        for (int i = lane; i < kAct * kHid; i += 32) w3[(i >> 5) * kS2 + (i & 31)] = __ldg(P.mlp + kOffW3 + i);
        const float b1 = __ldg(P.mlp + kOffB1 + lane), b2 = __ldg(P.mlp + kOffB2 + lane);
        const float b3 = lane < kAct ? __ldg(P.mlp + kOffB3 + lane) : 0.0f;
        __syncwarp();
        float a = b1;
        for (int j = 0; j < kIn; ++j) a += w1[lane * kS1 + j] * s_x[j];
        s_h1[lane] = tanhf(a);
        __syncwarp();
        a = b2;
        for (int j = 0; j < kHid; ++j) a += w2[lane * kS2 + j] * s_h1[j];
        s_h2[lane] = tanhf(a);
        __syncwarp();
        if (lane < kAct) {
            a = b3;
            for (int j = 0; j < kHid; ++j) a += w3[lane * kS2 + j] * s_h2[j];
            s_y[lane] = a;
        }
        __syncwarp();
    }
    if (lane != 0) return;
    // restart k+1: the action chosen one restart ago
    double next_stride;
    int next_mode;
    next_restart_of(P, C, &next_stride, &next_mode);
    const int next_action = __ldcg(&C->pend_action);
    // restart k+2: chosen now (-1: keep the stride and block edge)
    int action = -1;
    if (P.sched == 1 && P.mlp != nullptr) {
        action = 0;
        for (int a = 1; a < kAct; ++a)
            if (s_y[a] < s_y[action]) action = a;           // lowest predicted cost rate
        const int cur = next_action >= 0 ? next_action : __ldcg(&C->action);
        if (cur >= 0 && s_y[cur] - s_y[action] <= P.margin) action = cur;   // not worth a switch
        if (!(s_y[action] == s_y[action])) action = -1;    // network output unusable: keep the stride
    } else if (P.sched == 2) {
        action = static_cast<int>(mix32(P.seed * 0x9e3779b9u + static_cast<unsigned>(k)) % kAct);
    }
    // work for restart k+1: its brick list, or its group list (which a learned or
    // random schedule builds from the brick list only when the restart starts)
    const int n_next = __ldcg(&C->count[s1]) + ((next_mode == 16) ? __ldcg(&C->gcount[s1]) : 0);
    const unsigned long long now = globaltimer();
    const unsigned long long acc_a = __ldcg(&C->r_accepted), acc_band = __ldcg(&C->r_band);
    const unsigned long long acc_s = __ldcg(&C->r_solves);
    if (P.log != nullptr && k - 1 < P.log_cap) {
        RestartRec rec;
        rec.k = k;
        rec.active = n_this * (mode == 16 ? 8 : 1);
        rec.band = static_cast<int64_t>(acc_band);
        rec.accepted = static_cast<int64_t>(acc_a);
        rec.solves = static_cast<int64_t>(acc_s);
        rec.bound = __ldcg(&C->bound);
        rec.stride = __ldcg(&C->stride);
        rec.rmin = __uint_as_float(__ldcg(&C->r_rmin_bits));
        rec.rmax = __uint_as_float(__ldcg(&C->r_rmax_bits));
        rec.ms = static_cast<double>(now - __ldcg(&C->t_restart)) * 1e-6;
        rec.block_dim = mode;
        rec.next_action = action;
        for (int i = 0; i < kIn; ++i) rec.features[i] = s_x[i];
        P.log[k - 1] = rec;
    }
    C->marches += static_cast<unsigned long long>(n_this) * (mode == 16 ? 8ull : 1ull);
    C->accepted += acc_a;
    C->solves += acc_s;
    C->updates += __ldcg(&C->r_updates);
    C->fallbacks += __ldcg(&C->r_fallbacks);
    C->rounds += __ldcg(&C->r_rounds);
    C->r_accepted = 0;
    C->r_band = 0;
    C->r_solves = 0;
    C->r_updates = 0;
    C->r_fallbacks = 0;
    C->r_rounds = 0;
    C->r_rmin_bits = 0x7f800000u;
    C->r_rmax_bits = 0u;
    C->used[s] = __ldcg(&C->count[s]);
    C->count[s] = 0;
    C->head[s] = 0;
    C->gcount[s] = 0;
    C->ghead[s] = 0;
    if ((n_next == 0 && !P.pause) || (__ldcg(&C->status) & kStWaitTimeout)) {
        // (no work left, or a wait somewhere ran out: no warp starts another restart)
        C->done = 1;
        C->t_end = now;
    } else if (k >= P.max_restarts) {
        C->done = 1;
        C->status |= kStRestartCap;
        C->t_end = now;
    } else {
        // (a sharded grid pauses after every restart, its state set up for the next one: the host
        // imports the neighbours' faces, which may list more bricks, and decides whether to go on)
        if (P.pause) {
            C->done = 1;
            C->t_end = now;
        }
        const double bnd = __ldcg(&C->bound);
        C->k = k + 1;
        C->mode = next_mode;
        C->action = next_action;
        C->pend_action = action;
        C->stride = next_stride;
        C->bound_prev = bnd;
        C->bound = fmin(bnd + next_stride, P.width);   // bound_band <- min(bound_band + stride, width_band)
        C->t_restart = now;
    }
}

// Restart k's group list (ring slot s) from its brick list, by every thread of
// the launch, then a grid barrier; false if a wait ran out.  Out of line: it
// runs only at 16^3 restarts of a learned or random schedule.
__device__ __noinline__ bool groups_from_bricks(Ctrl* C, const int32_t* list, int32_t* qgroup, int32_t* glist, int s,
                                                int k, int BX, int BY, int GX, int GY, int lane, long long limit) {
    const int nb = __ldcg(&C->count[s]);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
        const int32_t x = __ldcg(list + i);
        const int bx = x % BX, by = (x / BX) % BY, bz = x / (BX * BY);
        const int32_t g = ((bz >> 1) * GY + (by >> 1)) * GX + (bx >> 1);
        if (atomicMax(qgroup + g, k) < k) {
            const int pos = atomicAdd(&C->gcount[s], 1);
            glist[pos] = g;
        }
    }
    __threadfence();
    return grid_sync(C, lane, limit);
}

template <typename T>
__global__ void __launch_bounds__(kWarps * 32, 3) k_restart_loop(LoopParams<T> P) {
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
    // Work lists the marches fill: the brick list, and for fixed 16^3 blocks
    // the group list too.  Under a learned or random schedule a 16^3 restart
    // builds its group list from its brick list when it starts (such restarts
    // are rare, and every enqueue would otherwise pay for the group list).
    const Geo G{P.BX, P.BY, P.BZ, 0, P.GX, P.GY, 0, (P.groups && P.sched == 0) ? 3u : 1u};
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer();
        C->t_begin = t0;
        C->t_restart = t0;
    }
    if (lane == 0) L.claim = -1;
    MarchAcc acc{0u, 0u, 0, 0u, 0u, 0u, __int_as_float(0x7f800000), 0.0f};
    bool any = false;                          // acc holds something to flush
    for (;;) {
        const int k = __ldcg(&C->k);
        const int mode = __ldcg(&C->mode);
        const int s = k % kRing;
        if (P.early) clear_used_slot(P, k);
        if (lane == 0) {
            L.bound = __ldcg(&C->bound);
            L.bprev = __ldcg(&C->bound_prev);
            double ns;
            int nm;
            next_restart_of(P, C, &ns, &nm);
            L.next_bound = fmin(L.bound + ns, P.width);         // restart k+1's bound
            L.bound_f = __double2float_rd(L.bound);
            L.bprev_f = __double2float_rd(L.bprev);
            L.next_f = __double2float_rd(L.next_bound);
            L.grow = L.bound < P.width;
            L.grow_next = L.next_bound < P.width;
            L.early = (P.early && mode == 8 && nm == 8) ? 1 : 0;
            L.n = (mode == 8) ? __ldcg(&C->count[s]) : 0;
            L.waiting = 0;
            L.polls = 0;
            L.nap = 256;
        }
        __syncwarp();
        if (mode == 16) {
            const bool ok = (G.lists & 2u) ||
                            groups_from_bricks(C, P.list[s], P.qgroup + static_cast<int64_t>(s) * P.ngroups,
                                               P.glist[s], s, k, P.BX, P.BY, P.GX, P.GY, lane, P.wait_limit);
            if (!cta_go(C, ok, lane, &s_arrived)) return;
            // one CTA per group of 2x2x2 bricks
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
                const int gx = g % P.GX, gy = (g / P.GX) % P.GY, gz = g / (P.GX * P.GY);
                const int bx = 2 * gx + (warp & 1), by = 2 * gy + ((warp >> 1) & 1), bz = 2 * gz + (warp >> 2);
                const bool in = bx < P.BX && by < P.BY && bz < P.BZ;
                const int32_t b = in ? (bz * P.BY + by) * P.BX + bx : -1;
                unsigned gmask = 0;
                if (in) {
                    if (warp & 1) gmask |= 1u;                     // -x neighbour in the group
                    else if (bx + 1 < P.BX) gmask |= 2u;           // +x
                    if (warp & 2) gmask |= 4u;
                    else if (by + 1 < P.BY) gmask |= 8u;
                    if (warp & 4) gmask |= 16u;
                    else if (bz + 1 < P.BZ) gmask |= 32u;
                }
                march<T, true>(P, G, SW, warp, b, gmask, k, pick<T>(L.bprev, L.bprev_f), pick<T>(L.bound, L.bound_f),
                               L.grow != 0, pick<T>(P.window, P.window_f), lane, acc, L.early != 0);
                any = true;
            }
        }
        // One warp per 8^3 brick: this restart's list, then -- once arrived at
        // the barrier -- restart k+1's bricks whose neighbourhood has finished
        // restart k (fixed stride and 8^3 blocks only; the next bound is then
        // known).  One march call site for both.
        for (;;) {
            int32_t b = -1, pf = -1;
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
                if (i >= 0) {
                    b = take_entry(P.list[s], i, false, 0, lane);
                    // the entry one launch-width further down, for the march to prefetch
                    const int i2 = i + static_cast<int>(gridDim.x) * kWarps;
                    if (i2 < L.n) pf = __ldcg(P.list[s] + i2);
                    if (pf >= P.nbricks) pf = -1;
                }
                if (b < 0) {
                    if (any) flush_acc(C, acc, lane);
                    any = false;
                    unsigned gen;
                    if (barrier_arrive(C, lane, &gen)) {
                        restart_end<T>(P, lane, reinterpret_cast<float*>(SW + warp));
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
                if (L.early) {
                    int claim = L.claim;
                    b = early_entry(C, P.list[(k + 1) % kRing], (k + 1) % kRing, claim, P.wait_limit, lane);
                    if (lane == 0) L.claim = claim;
                }
                if (b >= 0 && !wait_ready(P, G, b, k, lane)) b = -2;
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
            const bool ahead = kk > k;
            march<T, false>(P, G, SW, warp, b, 0u, kk,
                            ahead ? pick<T>(L.bound, L.bound_f) : pick<T>(L.bprev, L.bprev_f),
                            ahead ? pick<T>(L.next_bound, L.next_f) : pick<T>(L.bound, L.bound_f),
                            (ahead ? L.grow_next : L.grow) != 0, pick<T>(P.window, P.window_f), lane, acc,
                            L.early != 0 || ahead, pf);
            any = true;
        }
        if (__ldcg(&C->done)) return;
    }
}

// F (x fastest) -> h/F in brick layout; flags negative, NaN or infinite speeds.
template <typename T>
__global__ void k_layout_speed(const T* __restrict__ F, T* __restrict__ rr, int nx, int ny, int nz, int BX,
                               int BY, int64_t nbricks, double h, int* err, int seq) {
    const T INF = Num<T>::inf();
    // h/F in the working precision: one IEEE division in FP32 mode (a double
    // division per node would make this copy kernel FP64-bound on this part)
    const T hT = static_cast<T>(h);
    // one block per row (k, j) of the padded brick grid at a time, its threads
    // along x: each warp reads 128 contiguous bytes of F and writes 32-byte runs
    // of four bricks; padding nodes get +inf
    const int px = BX * 8, py = BY * 8;
    const int64_t rows = (nbricks / (static_cast<int64_t>(BX) * BY)) * 8 * py;
    int bad = 0;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int k = static_cast<int>(r / py), j = static_cast<int>(r - static_cast<int64_t>(k) * py);
        const bool inrow = j < ny && k < nz;
        const int64_t frow = inrow ? (static_cast<int64_t>(k) * ny + j) * nx : 0;
        T* out = rr + ((static_cast<int64_t>(k >> 3) * BY + (j >> 3)) * BX) * kBrick + ((k & 7) * 8 + (j & 7)) * 8;
        for (int i = threadIdx.x; i < px; i += blockDim.x) {
            T v = INF;
            if (inrow && i < nx) {
                const T f = __ldg(F + frow + i);
                if (!(f >= 0) || !(f < INF)) bad = 1;
                else if (f > 0) v = hT / f;
            }
            __stcs(out + (i >> 3) * kBrick + (i & 7), v);
        }
    }
    if (bad) *reinterpret_cast<volatile int*>(err) = seq;     // this upload's number marks a bad F
}

// Alg. 1 for the bricks that hold fixed nodes, and the work list of restart 1.
//   fix_b/fix_p/fix_v: fixed nodes (brick, node in brick, psi0); saved_r gets their h/F.
template <typename T>
__global__ void k_init_sources(int nfix, const int32_t* __restrict__ fix_b, const int32_t* __restrict__ fix_p,
                               const double* __restrict__ fix_v, int nsrcb, const int32_t* __restrict__ src_bricks,
                               int nenq, const int32_t* __restrict__ enq, int ngenq, const int32_t* __restrict__ genq,
                               T* slot, unsigned long long* ups, unsigned long long* stamp, int32_t* queued,
                               int32_t* qgroup, T* rr, T* saved_r, int32_t* list1, int32_t* glist1) {
    const T INF = Num<T>::inf();
    if (blockIdx.x < nsrcb) {
        const int32_t b = src_bricks[blockIdx.x];
        T* dst = slot + static_cast<int64_t>(b) * 2 * kSlot;            // copy 0
        for (int t = threadIdx.x; t < kSlot; t += blockDim.x) dst[t] = INF;
        __syncthreads();
        for (int t = threadIdx.x; t < nfix; t += blockDim.x) {
            if (fix_b[t] != b) continue;
            const int p = fix_p[t];
            const T v = static_cast<T>(fix_v[t]);
            dst[p] = v;
            const int x = p & 7, y = (p >> 3) & 7, z = p >> 6;
            if (x == 0) dst[kXF0 + z * 8 + y] = v;
            if (x == 7) dst[kXF7 + z * 8 + y] = v;
        }
        if (threadIdx.x < 6) ups[static_cast<int64_t>(b) * 2 * 6 + threadIdx.x] = 0ull;
        if (threadIdx.x == 0) stamp[b] = make_stamp(0, static_cast<int>(kNever), 0);   // "restart 0", copy 0
    } else {
        const int base = (blockIdx.x - nsrcb) * blockDim.x + threadIdx.x;
        if (base < nfix) {
            const int64_t g = static_cast<int64_t>(fix_b[base]) * kBrick + fix_p[base];
            saved_r[base] = rr[g];
            rr[g] = static_cast<T>(-1);
        }
        if (base < nenq) {
            list1[base] = enq[base];
            queued[enq[base]] = 1;
        }
        if (base < ngenq) {
            glist1[base] = genq[base];
            qgroup[genq[base]] = 1;
        }
    }
}

template <typename T>
__global__ void k_restore_r(int nfix, const int32_t* __restrict__ fix_b, const int32_t* __restrict__ fix_p,
                            const T* __restrict__ saved_r, T* rr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nfix) rr[static_cast<int64_t>(fix_b[t]) * kBrick + fix_p[t]] = saved_r[t];
}

// h/F of selected nodes (brick, node) for the host's source set-up.
template <typename T>
__global__ void k_gather_r(int n, const int32_t* __restrict__ nb_b, const int32_t* __restrict__ nb_p,
                           const T* __restrict__ rr, double* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = static_cast<double>(rr[static_cast<int64_t>(nb_b[t]) * kBrick + nb_p[t]]);
}

// Latest copy of every brick -> psi in x-fastest order, nodes z in [z_begin, z_end).
template <typename T>
__global__ void k_result(const T* __restrict__ slot, const unsigned long long* __restrict__ stamp, T* __restrict__ out, int nx,
                         int ny, int z_begin, int z_end, int BX, int BY) {
    const T INF = Num<T>::inf();
    // one block per grid row (k, j) at a time, its threads along x: 32-bit row
    // arithmetic, coalesced stores, 32-byte runs of each brick row read
    const int rows = ny * (z_end - z_begin);
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int kk = r / ny, j = r - kk * ny, k = z_begin + kk;
        const int64_t brow = (static_cast<int64_t>(k >> 3) * BY + (j >> 3)) * BX;
        const int prow = ((k & 7) * 8 + (j & 7)) * 8;
        T* o = out + static_cast<int64_t>(r) * nx;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int64_t b = brow + (i >> 3);
            const unsigned long long st = __ldg(stamp + b);
            o[i] = (st == kUntouched) ? INF : __ldcs(slot + (b * 2 + stamp_copy(st)) * kSlot + prow + (i & 7));
        }
    }
}

// FP32 with x-rows of a multiple of 4 nodes and 16-byte aligned buffers: the
// same two kernels moving four consecutive nodes per thread (one 16-byte load
// and store each; four nodes never straddle a brick row).
__global__ void k_layout_speed_x4(const float* __restrict__ F, float* __restrict__ rr, int nx, int ny, int nz,
                                  int BX, int BY, int64_t nbricks, float hT, int* err, int seq) {
    const float INF = __int_as_float(0x7f800000);
    const int px = BX * 8, py = BY * 8;
    const int64_t rows = (nbricks / (static_cast<int64_t>(BX) * BY)) * 8 * py;
    int bad = 0;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int k = static_cast<int>(r / py), j = static_cast<int>(r - static_cast<int64_t>(k) * py);
        const bool inrow = j < ny && k < nz;
        const int64_t frow = inrow ? (static_cast<int64_t>(k) * ny + j) * nx : 0;
        float* out = rr + ((static_cast<int64_t>(k >> 3) * BY + (j >> 3)) * BX) * kBrick + ((k & 7) * 8 + (j & 7)) * 8;
        for (int i = 4 * threadIdx.x; i < px; i += 4 * blockDim.x) {
            float4 v = make_float4(INF, INF, INF, INF);
            if (inrow && i < nx) {
                const float4 f = __ldg(reinterpret_cast<const float4*>(F + frow + i));
                const float fq[4] = {f.x, f.y, f.z, f.w};
                float vq[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    vq[e] = INF;
                    if (!(fq[e] >= 0.0f) || !(fq[e] < INF)) bad = 1;
                    else if (fq[e] > 0.0f) vq[e] = hT / fq[e];
                }
                v = make_float4(vq[0], vq[1], vq[2], vq[3]);
            }
            __stcs(reinterpret_cast<float4*>(out + (i >> 3) * kBrick + (i & 7)), v);
        }
    }
    if (bad) *reinterpret_cast<volatile int*>(err) = seq;
}

__global__ void k_result_x4(const float* __restrict__ slot, const unsigned long long* __restrict__ stamp,
                            float* __restrict__ out, int nx, int ny, int z_begin, int z_end, int BX, int BY) {
    const float INF = __int_as_float(0x7f800000);
    const int rows = ny * (z_end - z_begin);
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int kk = r / ny, j = r - kk * ny, k = z_begin + kk;
        const int64_t brow = (static_cast<int64_t>(k >> 3) * BY + (j >> 3)) * BX;
        const int prow = ((k & 7) * 8 + (j & 7)) * 8;
        float* o = out + static_cast<int64_t>(r) * nx;
        for (int i = 4 * threadIdx.x; i < nx; i += 4 * blockDim.x) {
            const int64_t b = brow + (i >> 3);
            const unsigned long long st = __ldg(stamp + b);
            const float4 v = (st == kUntouched)
                                 ? make_float4(INF, INF, INF, INF)
                                 : __ldcs(reinterpret_cast<const float4*>(slot + (b * 2 + stamp_copy(st)) * kSlot +
                                                                          prow + (i & 7)));
            *reinterpret_cast<float4*>(o + i) = v;
        }
    }
}

// A grid sharded in z across GPUs: the face layer of every brick of plane bz
// that a neighbouring GPU's bricks read (face 4: the z = 0 layer, read by the
// GPU below; face 5: the z = 7 layer, read by the GPU above), with the Upsilon
// mask of the brick's latest copy on that face.  One CTA of 64 threads per brick.
template <typename T>
__global__ void k_slab_export(const T* __restrict__ slot, const unsigned long long* __restrict__ ups,
                              const unsigned long long* __restrict__ stamp, int BX, int BY, int bz, int face,
                              FaceRec<T>* __restrict__ out) {
    const int bxy = blockIdx.x, t = threadIdx.x;
    const int64_t b = static_cast<int64_t>(bz) * BX * BY + bxy;
    const unsigned long long st = stamp[b];
    FaceRec<T>& R = out[bxy];
    if (st == kUntouched) {
        R.v[t] = Num<T>::inf();
        if (t == 0) {
            R.ups = 0ull;
            R.written = -1;
        }
        return;
    }
    const int64_t c = b * 2 + stamp_copy(st);
    R.v[t] = slot[c * kSlot + (face == 4 ? t : 7 * 64 + t)];
    if (t == 0) {
        R.ups = ups[c * 6 + face];
        R.written = stamp_latest(st);
    }
}

// The faces a neighbouring GPU exported -> the ghost plane gbz of this GPU's
// part of the grid (copy 0 of each ghost brick: the layer this GPU's bricks
// read, the Upsilon mask on that face, the stamp), after the restart k_done.
// A ghost face lowered in that restart puts the adjacent brick of plane obz on
// the work list of restart k_done + 1 (C of Alg. 4 across the GPUs' cut).
template <typename T>
__global__ void k_slab_import(T* __restrict__ slot, unsigned long long* __restrict__ ups,
                              unsigned long long* __restrict__ stamp, int BX, int BY, int gbz, int obz,
                              const FaceRec<T>* __restrict__ in, int k_done, int32_t* queued, int64_t nbricks,
                              Ctrl* C, int32_t* list_next) {
    const int bxy = blockIdx.x, t = threadIdx.x;
    const int64_t g = static_cast<int64_t>(gbz) * BX * BY + bxy;
    const FaceRec<T>& R = in[bxy];
    const bool below = gbz < obz;      // the ghost plane under this GPU's bricks: they read its z = 7 layer
    slot[g * 2 * kSlot + (below ? 7 * 64 + t : t)] = R.v[t];
    if (t != 0) return;
    ups[g * 2 * 6 + (below ? 5 : 4)] = R.ups;
    stamp[g] = (R.written < 0) ? kUntouched : make_stamp(R.written, static_cast<int>(kNever), 0);
    if (R.ups != 0ull && R.written == k_done) {
        const int k_next = k_done + 1, s = k_next % kRing;
        const int32_t x = static_cast<int32_t>(static_cast<int64_t>(obz) * BX * BY + bxy);
        if (atomicMax(queued + s * nbricks + x, k_next) < k_next) {
            const int pos = atomicAdd(&C->count[s], 1);
            list_next[pos] = x;
        }
    }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers (called from eik_runtime.cu)
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_layout_speed(const T* F, T* rr, int nx, int ny, int nz, int BX, int BY, int64_t nbricks,
                                double h, int* err, int seq, cudaStream_t s) {
    const int64_t rows = (nbricks / (static_cast<int64_t>(BX) * BY)) * 8 * (static_cast<int64_t>(BY) * 8);
    int grid = static_cast<int>(rows < 65535 * 4 ? rows : 65535 * 4);
    if (grid < 1) grid = 1;
    if constexpr (sizeof(T) == 4) {
        if (nx % 4 == 0 && reinterpret_cast<uintptr_t>(F) % 16 == 0) {
            k_layout_speed_x4<<<grid, 256, 0, s>>>(reinterpret_cast<const float*>(F), reinterpret_cast<float*>(rr), nx,
                                                   ny, nz, BX, BY, nbricks, static_cast<float>(h), err, seq);
            return cudaGetLastError();
        }
    }
    k_layout_speed<T><<<grid, 256, 0, s>>>(F, rr, nx, ny, nz, BX, BY, nbricks, h, err, seq);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_sources(int nfix, const int32_t* fix_b, const int32_t* fix_p, const double* fix_v,
                                int nsrcb, const int32_t* src_bricks, int nenq, const int32_t* enq, int ngenq,
                                const int32_t* genq, T* slot, unsigned long long* ups, unsigned long long* stamp,
                                int32_t* queued, int32_t* qgroup, T* rr, T* saved_r, int32_t* list1,
                                int32_t* glist1, cudaStream_t s) {
    int m = nfix > nenq ? nfix : nenq;
    m = m > ngenq ? m : ngenq;
    const int grid = nsrcb + (m + 255) / 256;
    k_init_sources<T><<<grid, 256, 0, s>>>(nfix, fix_b, fix_p, fix_v, nsrcb, src_bricks, nenq, enq, ngenq, genq,
                                           slot, ups, stamp, queued, qgroup, rr, saved_r, list1, glist1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restore_r(int nfix, const int32_t* fix_b, const int32_t* fix_p, const T* saved_r, T* rr,
                             cudaStream_t s) {
    if (nfix <= 0) return cudaSuccess;
    k_restore_r<T><<<(nfix + 255) / 256, 256, 0, s>>>(nfix, fix_b, fix_p, saved_r, rr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_r(int n, const int32_t* nb_b, const int32_t* nb_p, const T* rr, double* out,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_gather_r<T><<<(n + 255) / 256, 256, 0, s>>>(n, nb_b, nb_p, rr, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_result(const T* slot, const unsigned long long* stamp, T* out, int nx, int ny, int z_begin, int z_end,
                          int BX, int BY, cudaStream_t s) {
    const int64_t rows = static_cast<int64_t>(ny) * (z_end - z_begin);
    int grid = static_cast<int>(rows < 65535 * 4 ? rows : 65535 * 4);
    if (grid < 1) grid = 1;
    if constexpr (sizeof(T) == 4) {
        if (nx % 4 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0) {
            k_result_x4<<<grid, 256, 0, s>>>(reinterpret_cast<const float*>(slot), stamp, reinterpret_cast<float*>(out),
                                             nx, ny, z_begin, z_end, BX, BY);
            return cudaGetLastError();
        }
    }
    k_result<T><<<grid, 256, 0, s>>>(slot, stamp, out, nx, ny, z_begin, z_end, BX, BY);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_slab_export(const T* slot, const unsigned long long* ups, const unsigned long long* stamp, int BX,
                               int BY, int bz, int face, void* out, cudaStream_t s) {
    k_slab_export<T><<<BX * BY, 64, 0, s>>>(slot, ups, stamp, BX, BY, bz, face, static_cast<FaceRec<T>*>(out));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_slab_import(T* slot, unsigned long long* ups, unsigned long long* stamp, int BX, int BY, int gbz,
                               int obz, const void* in, int k_done, int32_t* queued, int64_t nbricks, Ctrl* C,
                               int32_t* list_next, cudaStream_t s) {
    k_slab_import<T><<<BX * BY, 64, 0, s>>>(slot, ups, stamp, BX, BY, gbz, obz, static_cast<const FaceRec<T>*>(in),
                                            k_done, queued, nbricks, C, list_next);
    return cudaGetLastError();
}

template <typename T>
size_t loop_smem_bytes() {
    return sizeof(WarpSmem<T>) * kWarps;
}

template <typename T>
cudaError_t loop_occupancy(int* blocks_per_sm) {
    const size_t smem = loop_smem_bytes<T>();
    cudaError_t e = cudaFuncSetAttribute(k_restart_loop<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_restart_loop<T>, kWarps * 32, smem);
}

template <typename T>
cudaError_t launch_restart_loop(const LoopParams<T>& P, int grid, cudaStream_t s) {
    LoopParams<T> copy = P;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_restart_loop<T>), dim3(grid),
                                       dim3(kWarps * 32), args, loop_smem_bytes<T>(), s);
}

#define EIKG_INSTANTIATE(T)                                                                                     \
    template cudaError_t launch_layout_speed<T>(const T*, T*, int, int, int, int, int, int64_t, double, int*,    \
                                                int, cudaStream_t);                                              \
    template cudaError_t launch_init_sources<T>(int, const int32_t*, const int32_t*, const double*, int,         \
                                                const int32_t*, int, const int32_t*, int, const int32_t*, T*,     \
                                                unsigned long long*, unsigned long long*, int32_t*, int32_t*, T*,  \
                                                T*, int32_t*, int32_t*, cudaStream_t);                            \
    template cudaError_t launch_restore_r<T>(int, const int32_t*, const int32_t*, const T*, T*, cudaStream_t);   \
    template cudaError_t launch_gather_r<T>(int, const int32_t*, const int32_t*, const T*, double*,              \
                                            cudaStream_t);                                                       \
    template cudaError_t launch_result<T>(const T*, const unsigned long long*, T*, int, int, int, int, int, int, \
                                          cudaStream_t);                                                         \
    template cudaError_t launch_slab_export<T>(const T*, const unsigned long long*, const unsigned long long*, int, \
                                               int, int, int, void*, cudaStream_t);                              \
    template cudaError_t launch_slab_import<T>(T*, unsigned long long*, unsigned long long*, int, int, int, int,   \
                                               const void*, int, int32_t*, int64_t, Ctrl*, int32_t*, cudaStream_t); \
    template size_t loop_smem_bytes<T>();                                                                        \
    template cudaError_t loop_occupancy<T>(int*);                                                                \
    template cudaError_t launch_restart_loop<T>(const LoopParams<T>&, int, cudaStream_t);

EIKG_INSTANTIATE(float)
EIKG_INSTANTIATE(double)

}  // namespace eikg
