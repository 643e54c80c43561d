// Device kernels of libeik: the block-based restarted narrow-band fast
// marching method (J. Yang 2018, Alg. 6 with Algs. 1-5) on sm_103a.
//
// One warp marches one 8x8x8 block (a "brick").  The brick's psi, h/F and its
// six ghost faces sit in shared memory; lane L owns the two x-rows
// (y = L & 7, z = 2*(L >> 3) + {0, 1}) as a 16-bit mask, plus the ghost nodes
// next to them.  The band (Sec. 2.1 BAND set) is a per-lane bit mask; a band
// node's value carries its sign bit set in shared memory so that any lane can
// tell a tentative value from an accepted (KNOWN) one with one load.
//
// Ordered extraction (Alg. 4) is done in rounds: each round takes the band
// minimum m with a warp reduction and accepts every band node with
// psi <= min(m + w, bound), w = omega * min(h/F) over the brick; the
// neighbours of the accepted nodes (Alg. 2) are compacted into a list and
// re-solved (Alg. 3) 32 at a time.  A lowered node rejoins the band, so an
// accepted node can be refreshed later exactly as a KNOWN_NEW node of the
// paper can.  With w = 0 this is the paper's one-node-at-a-time order.
//
// The restart loop of Alg. 6 runs in one cooperative persistent kernel with
// one grid-wide barrier per restart; the exchange step (Alg. 5) is fused into
// the start of the next march (see eik_internal.cuh for the double-copy
// layout that makes this race-free, the argument of Sec. 2.7).
#include "eik_internal.cuh"
#include "eik_mlp.cuh"

#include <cfloat>
#include <cstdint>

namespace eikg {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRoundCap = 1 << 20;

template <typename T>
struct Num;
template <>
struct Num<float> {
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};
template <>
struct Num<double> {
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000LL); }
};

__device__ __forceinline__ bool sgn(float v) { return (__float_as_uint(v) >> 31) != 0u; }
__device__ __forceinline__ bool sgn(double v) {
    return (static_cast<unsigned long long>(__double_as_longlong(v)) >> 63) != 0ull;
}
__device__ __forceinline__ float vabs(float v) { return fabsf(v); }
__device__ __forceinline__ double vabs(double v) { return fabs(v); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// Alg. 3: the upwind root for sorted upwind values a <= b <= c (b, c may be
// +inf) and r = h/F.  Alg. 3 solves a x^2 - 2 b x + c = 0 for the id
// smallest values, growing id while the root exceeds the next value.  Here
// the same root is written without cancellation: with k admitted values,
//   x = v_1 + (sum_i (v_i - v_1) + sqrt(D)) / k,
//   D = k r^2 - sum_{i<j} (v_i - v_j)^2          (Lagrange's identity),
// whose differences are exact.  Whenever a value is admitted D > r^2 in
// exact arithmetic, so D < tau*k*r^2 (tau < 1/3) only flags rounding trouble.
// ---------------------------------------------------------------------------
// The root never falls below the largest admitted value (causality of the
// upwind scheme; exact arithmetic guarantees it, rounding could break it by an
// ulp and let two nodes lower each other forever), hence the fmax clamps.
__device__ __forceinline__ double upwind_root(double a, double b, double c, double r) {
    double x = a + r;
    if (!(x > b)) return x;
    const double d = b - a;
    const double r2 = r * r;
    double D = 2.0 * r2 - d * d;
    x = fmax(a + (d + sqrt(fmax(D, 0.0))) * 0.5, b);
    if (!(x > c)) return x;
    const double e = c - a, g = c - b;
    D = 3.0 * r2 - (d * d + e * e + g * g);
    return fmax(a + (d + e + sqrt(fmax(D, 0.0))) / 3.0, c);
}

__device__ __forceinline__ float upwind_root_f32(float a, float b, float c, float r, float tau, int& fb) {
    float x = a + r;
    if (!(x > b)) return x;
    const float d = b - a;
    const float r2 = r * r;
    float D = 2.0f * r2 - d * d;
    if (!(r2 >= FLT_MIN) || !(D >= tau * 2.0f * r2)) {
        ++fb;
        return static_cast<float>(upwind_root(a, b, c, r));
    }
    x = fmaxf(a + (d + sqrtf(D)) * 0.5f, b);
    if (!(x > c)) return x;
    const float e = c - a, g = c - b;
    D = 3.0f * r2 - (d * d + e * e + g * g);
    if (!(D >= tau * 3.0f * r2)) {
        ++fb;
        return static_cast<float>(upwind_root(a, b, c, r));
    }
    return fmaxf(a + (d + e + sqrtf(D)) / 3.0f, c);
}

// Bounds arrive as doubles; a float node value v satisfies v <= b exactly when
// v <= (the largest float <= b), so the FP32 path compares in float (FP64
// throughput on this part is a small fraction of FP32).
template <typename T>
__device__ __forceinline__ T bound_down(double b);
template <>
__device__ __forceinline__ float bound_down<float>(double b) { return __double2float_rd(b); }
template <>
__device__ __forceinline__ double bound_down<double>(double b) { return b; }

template <typename T>
struct RootOf;
template <>
struct RootOf<float> {
    static __device__ __forceinline__ float go(float a, float b, float c, float r, float tau, int& fb) {
        return upwind_root_f32(a, b, c, r, tau, fb);
    }
};
template <>
struct RootOf<double> {
    static __device__ __forceinline__ double go(double a, double b, double c, double r, float, int&) {
        return upwind_root(a, b, c, r);
    }
};

// Per-warp shared memory.
constexpr int kBandCap = 896;      // 512 interior + 384 ghost nodes: every node at most once

template <typename T>
struct __align__(16) WarpSmem {
    T psi[1000];            // brick plus one ghost layer, index ((z+1)*10 + (y+1))*10 + (x+1)
    T r[kBrick];            // h/F, brick index
    uint16_t band[kBandCap];// the narrow band: halo indices of the pending nodes
    uint16_t list[kBrick];  // nodes to re-solve in the current round (brick index)
    uint32_t dirty[16];     // bit per brick node: neighbour of a node accepted this round
    uint32_t upd[16];       // bit per brick node: lowered in this march (Upsilon)
    uint32_t fxob[16];      // bit per brick node: fixed, barrier or padding node (never solved)
};

__device__ __forceinline__ int halo_of(int p) {
    const int x = p & 7, y = (p >> 3) & 7, z = p >> 6;
    return ((z + 1) * 10 + (y + 1)) * 10 + (x + 1);
}

template <typename T>
__device__ __forceinline__ void load8_cg(const T* g, T* out);
template <>
__device__ __forceinline__ void load8_cg<float>(const float* g, float* out) {
    const float4 a = __ldcg(reinterpret_cast<const float4*>(g));
    const float4 b = __ldcg(reinterpret_cast<const float4*>(g) + 1);
    out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
    out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
}
template <>
__device__ __forceinline__ void load8_cg<double>(const double* g, double* out) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double2 a = __ldcg(reinterpret_cast<const double2*>(g) + i);
        out[2 * i] = a.x;
        out[2 * i + 1] = a.y;
    }
}
template <typename T>
__device__ __forceinline__ void load8_ro(const T* g, T* out);
template <>
__device__ __forceinline__ void load8_ro<float>(const float* g, float* out) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(g));
    const float4 b = __ldg(reinterpret_cast<const float4*>(g) + 1);
    out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
    out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
}
template <>
__device__ __forceinline__ void load8_ro<double>(const double* g, double* out) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(g) + i);
        out[2 * i] = a.x;
        out[2 * i + 1] = a.y;
    }
}
template <typename T>
__device__ __forceinline__ void store8(T* g, const T* v);
template <>
__device__ __forceinline__ void store8<float>(float* g, const float* v) {
    reinterpret_cast<float4*>(g)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(g)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
template <>
__device__ __forceinline__ void store8<double>(double* g, const double* v) {
#pragma unroll
    for (int i = 0; i < 4; ++i) reinterpret_cast<double2*>(g)[i] = make_double2(v[2 * i], v[2 * i + 1]);
}
template <typename T>
__device__ __forceinline__ void load2_cg(const T* g, T& a, T& b);
template <>
__device__ __forceinline__ void load2_cg<float>(const float* g, float& a, float& b) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(g));
    a = v.x;
    b = v.y;
}
template <>
__device__ __forceinline__ void load2_cg<double>(const double* g, double& a, double& b) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(g));
    a = v.x;
    b = v.y;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = vmin(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = vmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ unsigned long long warp_or64(unsigned long long v) {
    const unsigned lo = __reduce_or_sync(kFull, static_cast<unsigned>(v));
    const unsigned hi = __reduce_or_sync(kFull, static_cast<unsigned>(v >> 32));
    return (static_cast<unsigned long long>(hi) << 32) | lo;
}

struct MarchAcc {
    unsigned accepted, band;                 // counted on lane 0
    int fallbacks;                           // per lane
    unsigned long long solves, updates, rounds;  // the same on every lane
    float rmin, rmax;                        // the same on every lane
};

// Halo index of ghost bit `bit` owned by this lane (see the G layout below).
__device__ __forceinline__ int ghost_halo(int bit, int y, int z0) {
    if (bit < 4) {
        const int z = z0 + (bit & 1);
        const int x = (bit & 2) ? 9 : 0;                 // x = -1 or x = 8
        return ((z + 1) * 10 + (y + 1)) * 10 + x;
    }
    if (bit < 20) {
        const int j = bit - 4, x = j & 7, z = z0 + (j >> 3);
        const int row = (y == 0) ? 0 : 9;                // y = -1 or y = 8
        return ((z + 1) * 10 + row) * 10 + (x + 1);
    }
    const int x = bit - 20;
    const int plane = (z0 == 0) ? 0 : 9;                 // z = -1 or z = 8
    return (plane * 10 + (y + 1)) * 10 + (x + 1);
}

// Face-local element u of face f (x faces: u = z*8+y, y faces: u = z*8+x,
// z faces: u = y*8+x): halo index of the ghost node beyond face f, and halo
// index of the brick's own boundary node on face f.
__device__ __forceinline__ int face_ghost_halo(int f, int u) {
    const int a = u & 7, c = u >> 3;
    if (f < 2) return ((c + 1) * 10 + (a + 1)) * 10 + (f == 0 ? 0 : 9);
    if (f < 4) return ((c + 1) * 10 + (f == 2 ? 0 : 9)) * 10 + (a + 1);
    return ((f == 4 ? 0 : 9) * 10 + (c + 1)) * 10 + (a + 1);
}
__device__ __forceinline__ int face_own_halo(int f, int u) {
    const int a = u & 7, c = u >> 3;
    if (f < 2) return ((c + 1) * 10 + (a + 1)) * 10 + (f == 0 ? 1 : 8);
    if (f < 4) return ((c + 1) * 10 + (f == 2 ? 1 : 8)) * 10 + (a + 1);
    return ((f == 4 ? 1 : 8) * 10 + (c + 1)) * 10 + (a + 1);
}

// Put brick x (and, if the block work list is kept, its block) on restart
// k+1's work lists, once per restart (the "queued" marks dedupe).
template <typename T>
__device__ __forceinline__ void enqueue_next(const LoopParams<T>& P, int k, int32_t x) {
    const int par = (k + 1) & 1;
    if (atomicMax(P.queued + x, k + 1) < k + 1) {
        const int pos = atomicAdd(&P.ctrl->count[par], 1);
        (par ? P.list1 : P.list0)[pos] = x;
    }
    if (!P.groups) return;
    const int bx = x % P.BX, by = (x / P.BX) % P.BY, bz = x / (P.BX * P.BY);
    const int32_t g = ((bz >> 1) * P.GY + (by >> 1)) * P.GX + (bx >> 1);
    if (atomicMax(P.qgroup + g, k + 1) < k + 1) {
        const int pos = atomicAdd(&P.ctrl->gcount[par], 1);
        (par ? P.glist1 : P.glist0)[pos] = g;
    }
}

// March_Narrow_Band (Alg. 4) of brick b at restart k, with the exchange of
// Alg. 5 for its ghost layer done first from the neighbours' copies as of the
// end of restart k-1.
//
// GROUP = false: one warp, one 8^3 block.  GROUP = true: the eight warps of the
// CTA march the 2x2x2 bricks of one 16^3 block together (warp w holds brick
// (w & 1, (w >> 1) & 1, w >> 2) of the group; b < 0 for a brick outside the
// grid, whose warp only takes part in the barriers).  The rounds then share
// one acceptance threshold, an accepted node marks the neighbouring warp's
// nodes across internal faces, and after every phase each warp refreshes its
// ghost layer on internal faces from the neighbouring warp's tile, so
// information crosses the internal faces within the restart as it does inside
// one block of the paper.
template <typename T, bool GROUP>
__device__ void march(const LoopParams<T>& P, WarpSmem<T>* SW, int warp, int32_t b, unsigned gmask, int k,
                      double bprev_d, double bound_d, int lane, MarchAcc& acc) {
    __shared__ double s_wmin[kWarps];
    WarpSmem<T>& S = SW[warp];
    const T INF = Num<T>::inf();
    const T bprev = bound_down<T>(bprev_d);
    const T bound = bound_down<T>(bound_d);
    const bool present = b >= 0;
    const int y = lane & 7, zp = lane >> 3, z0 = 2 * zp;
    const int BX = P.BX, BY = P.BY, BZ = P.BZ;
    const int bb = present ? b : 0;
    const int bx = bb % BX, by = (bb / BX) % BY, bz = bb / (BX * BY);
    const int pbase = (z0 * 8 + y) * 8;                          // brick index of (0, y, z0)
    const int hbase = ((z0 + 1) * 10 + (y + 1)) * 10 + 1;       // halo index of (0, y, z0)
    const unsigned lt = (1u << lane) - 1u;

    int nbr[6];
    nbr[0] = bx > 0 ? bb - 1 : -1;
    nbr[1] = bx < BX - 1 ? bb + 1 : -1;
    nbr[2] = by > 0 ? bb - BX : -1;
    nbr[3] = by < BY - 1 ? bb + BX : -1;
    nbr[4] = bz > 0 ? bb - BX * BY : -1;
    nbr[5] = bz < BZ - 1 ? bb + BX * BY : -1;

    unsigned long long st = kUntouched;
    unsigned FXOB = 0xFFFFu;
    T rlo = INF, rhi = 0;
    int n = 0;
    if (present) {
        // ---- load phase 1 (independent loads): stamps of the brick and its six
        // neighbours, and h/F of this lane's two rows
        st = __ldcg(P.stamp + b);
        unsigned long long wst[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) wst[f] = nbr[f] >= 0 ? __ldcg(P.stamp + nbr[f]) : kUntouched;
        // fixed nodes (r < 0) and barrier/padding nodes (r = +inf) are never solved
        FXOB = 0;
        {
            T row[8];
            const T* rs = P.rr + static_cast<int64_t>(b) * kBrick;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                load8_ro(rs + pbase + 64 * s, row);
                store8(S.r + pbase + 64 * s, row);
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const T r = row[x];
                    if (!(r > 0) || !(r < INF)) FXOB |= 1u << (8 * s + x);
                    else {
                        rlo = vmin(rlo, r);
                        rhi = vmax(rhi, r);
                    }
                }
            }
        }
        // ---- load phase 2: the brick's latest copy, and the ghost layer: the
        // neighbours' faces as of the end of restart k-1 with their Upsilon masks
        // (Alg. 5).  A neighbour that already marched in this restart is read from
        // its other copy.
        unsigned long long fups[6];
        T fv0[6], fv1[6];
        const int u = 2 * lane;                                   // face-local index of this lane's pair
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const unsigned long long w = wst[f];
            int sl = -1, written = -1;
            if (w != kUntouched) {
                if (stamp_latest(w) >= k) {
                    written = stamp_other(w);
                    sl = (written == static_cast<int>(kNever)) ? -1 : (stamp_copy(w) ^ 1);
                } else {
                    written = stamp_latest(w);
                    sl = stamp_copy(w);
                }
            }
            fups[f] = (sl >= 0 && written == k - 1)
                          ? __ldcg(P.ups + (static_cast<int64_t>(nbr[f]) * 2 + sl) * 6 + (f ^ 1))
                          : 0ull;
            fv0[f] = INF;
            fv1[f] = INF;
            if (sl >= 0) {
                const T* src = P.slot + (static_cast<int64_t>(nbr[f]) * 2 + sl) * kSlot;
                int off;
                if (f == 0) off = kXF7 + u;
                else if (f == 1) off = kXF0 + u;
                else if (f == 2) off = ((u >> 3) * 8 + 7) * 8 + (u & 7);
                else if (f == 3) off = ((u >> 3) * 8 + 0) * 8 + (u & 7);
                else if (f == 4) off = 7 * 64 + u;
                else off = u;
                load2_cg(src + off, fv0[f], fv1[f]);
            }
        }
        {
            T row[8];
            if (st == kUntouched) {
#pragma unroll
                for (int x = 0; x < 8; ++x) S.psi[hbase + x] = INF, S.psi[hbase + 100 + x] = INF;
            } else {
                const T* src = P.slot + (static_cast<int64_t>(b) * 2 + stamp_copy(st)) * kSlot;
                T row1[8];
                load8_cg(src + pbase, row);
                load8_cg(src + pbase + 64, row1);
#pragma unroll
                for (int x = 0; x < 8; ++x) S.psi[hbase + x] = row[x], S.psi[hbase + 100 + x] = row1[x];
            }
        }
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const int h0 = face_ghost_halo(f, u);
            S.psi[h0] = fv0[f];
            S.psi[h0 + (f < 2 ? 10 : 1)] = fv1[f];
        }
        __syncwarp();

        // ---- the band at the start of the march: finite nodes above the previous
        // bound, plus ghost nodes the neighbour lowered in restart k-1 (Upsilon)
        unsigned B = 0, G = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int hh = hbase + (j >> 3) * 100 + (j & 7);
            const T v = S.psi[hh];
            if (v < INF && v > bprev) {
                B |= 1u << j;
                S.psi[hh] = -v;
            }
        }
        auto mark_ghost = [&](int bit, unsigned long long um, int uu) {
            const int hh = ghost_halo(bit, y, z0);
            const T g = S.psi[hh];
            if (g < INF && (((um >> uu) & 1ull) || g > bprev)) {
                G |= 1u << bit;
                S.psi[hh] = -g;
            }
        };
        mark_ghost(0, fups[0], z0 * 8 + y);
        mark_ghost(1, fups[0], (z0 + 1) * 8 + y);
        mark_ghost(2, fups[1], z0 * 8 + y);
        mark_ghost(3, fups[1], (z0 + 1) * 8 + y);
        if (y == 0 || y == 7) {
            const unsigned long long um = (y == 0) ? fups[2] : fups[3];
#pragma unroll
            for (int j = 0; j < 16; ++j) mark_ghost(4 + j, um, (z0 + (j >> 3)) * 8 + (j & 7));
        }
        if (zp == 0 || zp == 3) {
            const unsigned long long um = (zp == 0) ? fups[4] : fups[5];
#pragma unroll
            for (int x = 0; x < 8; ++x) mark_ghost(20 + x, um, y * 8 + x);
        }
        __syncwarp();
        // ---- the band as a list shared by the warp (one entry per pending node)
        const int cnt = __popc(B) + __popc(G);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        n = __shfl_sync(kFull, incl, 31);
        int off = incl - cnt;
        for (unsigned m = B; m; m &= m - 1) {
            const int j = __ffs(m) - 1;
            S.band[off++] = static_cast<uint16_t>(hbase + (j >> 3) * 100 + (j & 7));
        }
        for (unsigned m = G; m; m &= m - 1) S.band[off++] = static_cast<uint16_t>(ghost_halo(__ffs(m) - 1, y, z0));
    }
    if (lane < 16) {
        S.dirty[lane] = 0u;
        S.upd[lane] = 0u;
        S.fxob[lane] = 0u;
    }
    __syncwarp();
    if (FXOB & 0xFFu) atomicOr(&S.fxob[pbase >> 5], (FXOB & 0xFFu) << (pbase & 31));
    if (FXOB >> 8) atomicOr(&S.fxob[(pbase + 64) >> 5], (FXOB >> 8) << ((pbase + 64) & 31));

    const T rmin_b = warp_min(rlo);
    if (present) {
        acc.rmin = fminf(acc.rmin, static_cast<float>(rmin_b));
        acc.rmax = fmaxf(acc.rmax, static_cast<float>(warp_max(rhi)));
    }
    T w;
    if constexpr (GROUP) {
        // one window for the group: omega times the smallest h/F of its bricks
        if (lane == 0) s_wmin[warp] = static_cast<double>(rmin_b);
        __syncthreads();
        double g = s_wmin[0];
#pragma unroll
        for (int i = 1; i < kWarps; ++i) g = fmin(g, s_wmin[i]);
        w = static_cast<T>(P.window * g);
        __syncthreads();
    } else {
        w = static_cast<T>(P.window * static_cast<double>(rmin_b));
    }
    const float tau = static_cast<float>(P.fallback_tau);

    // ghost layer on internal faces <- the neighbouring warps' boundary nodes
    auto refresh_internal = [&]() {
        if constexpr (GROUP) {
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (!((gmask >> f) & 1u)) continue;
                const WarpSmem<T>& NB = SW[warp ^ (1 << (f >> 1))];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int uu = 2 * lane + e;
                    S.psi[face_ghost_halo(f, uu)] = NB.psi[face_own_halo(f ^ 1, uu)];
                }
            }
            __syncwarp();
        }
    };

    // ---- rounds of windowed ordered acceptance (Alg. 4)
    int rounds = 0;
    for (;;) {
        T lmin = INF;
        for (int i = lane; i < n; i += 32) lmin = vmin(lmin, vabs(S.psi[S.band[i]]));
        T mn = warp_min(lmin);
        if constexpr (GROUP) {
            if (lane == 0) s_wmin[warp] = static_cast<double>(mn);
            __syncthreads();
            double g = s_wmin[0];
#pragma unroll
            for (int i = 1; i < kWarps; ++i) g = fmin(g, s_wmin[i]);
            mn = static_cast<T>(g);
            __syncthreads();
        }
        if (!(mn < INF) || !(mn <= bound)) break;   // band empty, or its minimum above the bound
        if (++rounds > kRoundCap) {
            atomicOr(&P.ctrl->status, kStRoundCap);
            break;
        }
        const T thr = vmin(mn + w, bound);
        // accept (Remove_Min of a window), keep the rest of the band in order,
        // and mark the accepted nodes' neighbours (Alg. 2)
        int kept = 0;
        for (int base = 0; base < n; base += 32) {
            const int i = base + lane;
            int hh = 0;
            bool keep = false, take = false;
            if (i < n) {
                hh = S.band[i];
                const T v = vabs(S.psi[hh]);
                if (v <= thr) {
                    take = true;
                    S.psi[hh] = v;
                } else {
                    keep = true;
                }
            }
            const unsigned km = __ballot_sync(kFull, keep);
            const unsigned tm = __ballot_sync(kFull, take);
            if (keep) S.band[kept + __popc(km & lt)] = static_cast<uint16_t>(hh);
            kept += __popc(km);
            if (lane == 0) acc.accepted += __popc(tm);
            if (take) {
                const int px = hh % 10 - 1, py = (hh / 10) % 10 - 1, pz = hh / 100 - 1;
                auto cand = [&](int x, int yy, int z) {
                    const bool ix = static_cast<unsigned>(x) < 8u, iy = static_cast<unsigned>(yy) < 8u,
                               iz = static_cast<unsigned>(z) < 8u;
                    if (ix && iy && iz) {
                        const int q = (z * 8 + yy) * 8 + x;
                        atomicOr(&S.dirty[q >> 5], 1u << (q & 31));
                    } else if (GROUP) {
                        // across an internal face: the neighbouring warp's node
                        int f = -1;
                        if (!ix && iy && iz) f = (x < 0) ? 0 : 1;
                        else if (ix && !iy && iz) f = (yy < 0) ? 2 : 3;
                        else if (ix && iy && !iz) f = (z < 0) ? 4 : 5;
                        if (f >= 0 && ((gmask >> f) & 1u)) {
                            const int q = (((z & 7) * 8) + (yy & 7)) * 8 + (x & 7);
                            atomicOr(&SW[warp ^ (1 << (f >> 1))].dirty[q >> 5], 1u << (q & 31));
                        }
                    }
                };
                cand(px - 1, py, pz);
                cand(px + 1, py, pz);
                cand(px, py - 1, pz);
                cand(px, py + 1, pz);
                cand(px, py, pz - 1);
                cand(px, py, pz + 1);
            }
        }
        n = kept;
        if constexpr (GROUP) {
            __syncthreads();
            refresh_internal();
            __syncthreads();
        } else {
            __syncwarp();
        }

        // candidates -> list of nodes to re-solve; never-solved nodes dropped
        const unsigned word = S.dirty[lane >> 1] & ~S.fxob[lane >> 1];
        const unsigned wd = (lane & 1) ? (word >> 16) : (word & 0xFFFFu);
        __syncwarp();
        if (lane < 16) S.dirty[lane] = 0u;
        const int cnt = __popc(wd);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        int off = incl - cnt;
        for (unsigned m = wd; m; m &= m - 1)
            S.list[off++] = static_cast<uint16_t>((lane >> 1) * 32 + (lane & 1) * 16 + __ffs(m) - 1);
        __syncwarp();
        acc.solves += total;

        // Alg. 3 for each listed node, 32 at a time; new values land after the reads
        for (int base = 0; base < total; base += 32) {
            const int idx = base + lane;
            bool imp = false, known = false;
            T xn = 0;
            int hq = 0, q = 0;
            if (idx < total) {
                q = S.list[idx];
                hq = halo_of(q);
                const T cur = S.psi[hq];
                const T c = vabs(cur);
                known = !sgn(cur);
                // KNOWN neighbours below the node's current value (Alg. 3's test)
                auto kn = [&](T v) -> T { return (sgn(v) || !(v < c)) ? INF : v; };
                T mx = vmin(kn(S.psi[hq - 1]), kn(S.psi[hq + 1]));
                T my = vmin(kn(S.psi[hq - 10]), kn(S.psi[hq + 10]));
                T mz = vmin(kn(S.psi[hq - 100]), kn(S.psi[hq + 100]));
                // reorder psi_1 <= psi_2 <= psi_3
                T lo = vmin(mx, my), hi = vmax(mx, my);
                T a0 = vmin(lo, mz);
                T t1 = vmax(lo, mz);
                T a1 = vmin(hi, t1), a2 = vmax(hi, t1);
                if (a0 < INF) {
                    xn = RootOf<T>::go(a0, a1, a2, S.r[q], tau, acc.fallbacks);
                    imp = xn < c;
                }
            }
            __syncwarp();
            // a lowered node is tagged BAND (Alg. 2): it joins the band unless already in it
            const bool add = imp && known;
            const unsigned am = __ballot_sync(kFull, add);
            if (imp) {
                S.psi[hq] = -xn;
                atomicOr(&S.upd[q >> 5], 1u << (q & 31));
            }
            if (add) S.band[n + __popc(am & lt)] = static_cast<uint16_t>(hq);
            n += __popc(am);
            acc.updates += __popc(__ballot_sync(kFull, imp));
            __syncwarp();
        }
        if constexpr (GROUP) {
            __syncthreads();
            refresh_internal();
        }
    }
    acc.rounds += rounds;
    if constexpr (GROUP) __syncthreads();
    if (!present) return;

    // ---- Upsilon: own face nodes lowered in this march, per face (face-local bit
    // masks); none on internal faces of a group, whose neighbours saw them live
    const unsigned U = ((S.upd[pbase >> 5] >> (pbase & 31)) & 0xFFu) |
                       (((S.upd[(pbase + 64) >> 5] >> ((pbase + 64) & 31)) & 0xFFu) << 8);
    unsigned long long um[6];
    um[0] = (static_cast<unsigned long long>(U & 1u) << (z0 * 8 + y)) |
            (static_cast<unsigned long long>((U >> 8) & 1u) << ((z0 + 1) * 8 + y));
    um[1] = (static_cast<unsigned long long>((U >> 7) & 1u) << (z0 * 8 + y)) |
            (static_cast<unsigned long long>((U >> 15) & 1u) << ((z0 + 1) * 8 + y));
    um[2] = (y == 0) ? (static_cast<unsigned long long>(U & 0xFFFFu) << (z0 * 8)) : 0ull;
    um[3] = (y == 7) ? (static_cast<unsigned long long>(U & 0xFFFFu) << (z0 * 8)) : 0ull;
    um[4] = (zp == 0) ? (static_cast<unsigned long long>(U & 0xFFu) << (y * 8)) : 0ull;
    um[5] = (zp == 3) ? (static_cast<unsigned long long>((U >> 8) & 0xFFu) << (y * 8)) : 0ull;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        um[f] = warp_or64(um[f]);
        if (GROUP && ((gmask >> f) & 1u)) um[f] = 0ull;
    }

    // ---- write the other copy, then publish it
    const int ns = (st == kUntouched) ? 0 : (stamp_copy(st) ^ 1);
    T* dst = P.slot + (static_cast<int64_t>(b) * 2 + ns) * kSlot;
    {
        T row[8];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
#pragma unroll
            for (int x = 0; x < 8; ++x) row[x] = vabs(S.psi[hbase + 100 * s + x]);
            store8(dst + pbase + 64 * s, row);
            dst[kXF0 + (z0 + s) * 8 + y] = row[0];
            dst[kXF7 + (z0 + s) * 8 + y] = row[7];
        }
    }
    if (lane < 6) P.ups[(static_cast<int64_t>(b) * 2 + ns) * 6 + lane] = um[lane];
    // No fence: nobody reads this copy before the grid barrier that ends the
    // restart (a reader that sees the new stamp takes the other copy).
    if (lane == 0)
        P.stamp[b] = make_stamp(k, st == kUntouched ? static_cast<int>(kNever) : stamp_latest(st), ns);

    // ---- activation for restart k+1 (A of Alg. 4/5, C of Alg. 4)
    if (lane == 6 && n > 0) enqueue_next(P, k, b);
    if (lane < 6 && um[lane] != 0ull && nbr[lane] >= 0) enqueue_next(P, k, nbr[lane]);
    if (lane == 0) acc.band += n;
}

// Features of the front after restart k for the schedule network (all O(1)):
// log-counts of marched bricks, band nodes, accepted nodes and solves; log of
// the largest and smallest speed over the marched bricks; the bound in grid
// lengths; log k; the stride in h; whether the blocks were 16^3.
__device__ inline void schedule_features(float* x, double active, double band, double accepted, double solves,
                                         double rmin, double rmax, double bound, double stride, int k, int mode,
                                         double h, int nmax) {
    x[0] = static_cast<float>(log1p(active) / 16.0);
    x[1] = static_cast<float>(log1p(band) / 20.0);
    x[2] = static_cast<float>(log1p(accepted) / 20.0);
    x[3] = (rmin > 0.0 && rmin < 1e300) ? static_cast<float>(log(h / rmin)) : 0.0f;
    x[4] = (rmax > 0.0 && rmax < 1e300) ? static_cast<float>(log(h / rmax)) : 0.0f;
    x[5] = static_cast<float>(bound / (h * nmax));
    x[6] = static_cast<float>(log1p(static_cast<double>(k)) / 8.0);
    x[7] = static_cast<float>(stride / h / 4.0);
    x[8] = (mode == 16) ? 1.0f : 0.0f;
    x[9] = static_cast<float>(log1p(solves) / 20.0);
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

// Grid barrier at the end of restart k.  The CTA arriving last does the
// restart bookkeeping of Alg. 6 (statistics, exit test, next bound) and, for
// the learned schedule, evaluates the schedule network with its threads to
// pick the stride and block edge of restart k+1, before releasing the others.
// Returns false when this CTA must leave the loop.
template <typename T>
__device__ bool end_of_restart(const LoopParams<T>& P) {
    __shared__ int s_last;
    __shared__ int s_ok;
    __shared__ float s_x[kIn];
    __shared__ float s_h1[kHid];
    __shared__ float s_h2[kHid];
    __shared__ float s_y[kAct];
    Ctrl* C = P.ctrl;
    __syncthreads();
    unsigned gen = 0;
    if (threadIdx.x == 0) {
        gen = ld_acquire(&C->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&C->bar_count, 1u);
        s_last = (arrived == gridDim.x - 1);
        s_ok = 1;
    }
    __syncthreads();
    if (s_last) {
        if (threadIdx.x == 0) {
            __threadfence();
            const int k = __ldcg(&C->k);
            const int mode = __ldcg(&C->mode);
            const int par = k & 1;
            const int n_this = (mode == 16) ? __ldcg(&C->gcount[par]) : __ldcg(&C->count[par]);
            schedule_features(s_x, static_cast<double>(n_this) * (mode == 16 ? 8 : 1),
                              static_cast<double>(__ldcg(&C->r_band)), static_cast<double>(__ldcg(&C->r_accepted)),
                              static_cast<double>(__ldcg(&C->r_solves)),
                              static_cast<double>(__uint_as_float(__ldcg(&C->r_rmin_bits))),
                              static_cast<double>(__uint_as_float(__ldcg(&C->r_rmax_bits))), __ldcg(&C->bound),
                              __ldcg(&C->stride), k, mode, P.h, P.nmax);
        }
        __syncthreads();
        if (P.sched == 1 && P.mlp != nullptr) {
            // the schedule network, one neuron per thread, layer by layer
            const float* w = P.mlp;
            const int t = threadIdx.x;
            if (t < kHid) {
                float a = w[kOffB1 + t];
                for (int j = 0; j < kIn; ++j) a += w[kOffW1 + t * kIn + j] * s_x[j];
                s_h1[t] = tanhf(a);
            }
            __syncthreads();
            if (t < kHid) {
                float a = w[kOffB2 + t];
                for (int j = 0; j < kHid; ++j) a += w[kOffW2 + t * kHid + j] * s_h1[j];
                s_h2[t] = tanhf(a);
            }
            __syncthreads();
            if (t < kAct) {
                float a = w[kOffB3 + t];
                for (int j = 0; j < kHid; ++j) a += w[kOffW3 + t * kHid + j] * s_h2[j];
                s_y[t] = a;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const int k = __ldcg(&C->k);
            const int par = k & 1;
            const int mode = __ldcg(&C->mode);
            const int n_this = (mode == 16) ? __ldcg(&C->gcount[par]) : __ldcg(&C->count[par]);
            // the next restart's stride and block edge
            double next_stride = __ldcg(&C->stride);
            int next_mode = P.mode_fixed;
            int action = -1;
            if (P.sched == 1 && P.mlp != nullptr) {
                action = 0;
                for (int a = 1; a < kAct; ++a)
                    if (s_y[a] < s_y[action]) action = a;           // lowest predicted cost rate
                const int cur = __ldcg(&C->action);
                if (cur >= 0 && s_y[cur] - s_y[action] <= P.margin) action = cur;   // not worth a switch
                if (!(s_y[action] == s_y[action])) action = -1;    // network output unusable: keep the fixed stride
            } else if (P.sched == 2) {
                action = static_cast<int>(mix32(P.seed * 0x9e3779b9u + static_cast<unsigned>(k)) % kAct);
            }
            if (action >= 0) {
                next_stride = action_stride_h(action) * P.h;
                next_mode = action_block(action);
            }
            if (!P.groups) next_mode = 8;
            const int n_next = (next_mode == 16) ? __ldcg(&C->gcount[par ^ 1]) : __ldcg(&C->count[par ^ 1]);
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
            C->count[par] = 0;
            C->head[par] = 0;
            C->gcount[par] = 0;
            C->ghead[par] = 0;
            if (n_next == 0) {
                C->done = 1;
                C->t_end = now;
            } else if (k >= P.max_restarts) {
                C->done = 1;
                C->status |= kStRestartCap;
                C->t_end = now;
            } else {
                const double bnd = __ldcg(&C->bound);
                C->k = k + 1;
                C->mode = next_mode;
                C->action = action;
                C->stride = next_stride;
                C->bound_prev = bnd;
                C->bound = bnd + next_stride;               // bound_band <- bound_band + stride (width = +inf)
                C->t_restart = now;
            }
            C->bar_count = 0;
            __threadfence();
            st_release(&C->bar_gen, gen + 1);
        }
    } else if (threadIdx.x == 0) {
        long long it = 0;
        while (ld_acquire(&C->bar_gen) == gen) {
            if (++it > P.wait_limit) {
                atomicOr(&C->status, kStWaitTimeout);
                s_ok = 0;
                break;
            }
            __nanosleep(64);
        }
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(kWarps * 32, 3) k_restart_loop(LoopParams<T> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<T>* SW = reinterpret_cast<WarpSmem<T>*>(smem_raw);
    Ctrl* C = P.ctrl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer();
        C->t_begin = t0;
        C->t_restart = t0;
    }
    for (;;) {
        const int k = __ldcg(&C->k);
        const double bound = __ldcg(&C->bound);
        const double bprev = __ldcg(&C->bound_prev);
        const int mode = __ldcg(&C->mode);
        const int par = k & 1;
        MarchAcc acc{0u, 0u, 0, 0ull, 0ull, 0ull, __int_as_float(0x7f800000), 0.0f};
        bool any = false;
        if (mode == 16) {
            // one CTA per group of 2x2x2 bricks
            const int n = __ldcg(&C->gcount[par]);
            const int32_t* list = par ? P.glist1 : P.glist0;
            for (;;) {
                __syncthreads();
                if (threadIdx.x == 0) {
                    const int i = atomicAdd(&C->ghead[par], 1);
                    s_item = (i < n) ? __ldcg(list + i) : -1;
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
                march<T, true>(P, SW, warp, b, gmask, k, bprev, bound, lane, acc);
                any = true;
            }
        } else {
            // one warp per brick
            const int n = __ldcg(&C->count[par]);
            const int32_t* list = par ? P.list1 : P.list0;
            for (;;) {
                int i = 0;
                if (lane == 0) i = atomicAdd(&C->head[par], 1);
                i = __shfl_sync(kFull, i, 0);
                if (i >= n) break;
                march<T, false>(P, SW, warp, __ldcg(list + i), 0u, k, bprev, bound, lane, acc);
                any = true;
            }
        }
        if (any) {
            const unsigned acc_a = __reduce_add_sync(kFull, acc.accepted);
            const unsigned acc_b = __reduce_add_sync(kFull, acc.band);
            const int fb = __reduce_add_sync(kFull, acc.fallbacks);
            if (lane == 0) {
                atomicAdd(&C->r_accepted, static_cast<unsigned long long>(acc_a));
                atomicAdd(&C->r_band, static_cast<unsigned long long>(acc_b));
                atomicAdd(&C->r_solves, acc.solves);
                atomicAdd(&C->r_updates, acc.updates);
                atomicAdd(&C->r_rounds, acc.rounds);
                atomicMin(&C->r_rmin_bits, __float_as_uint(acc.rmin));
                atomicMax(&C->r_rmax_bits, __float_as_uint(acc.rmax));
                if (fb) atomicAdd(&C->r_fallbacks, static_cast<unsigned long long>(fb));
            }
        }
        if (!end_of_restart<T>(P)) return;
        if (__ldcg(&C->done)) return;
    }
}

// F (x fastest) -> h/F in brick layout; flags negative, NaN or infinite speeds.
template <typename T>
__global__ void k_layout_speed(const T* __restrict__ F, T* __restrict__ rr, int nx, int ny, int nz, int BX,
                               int BY, int64_t nbricks, double h, int* err) {
    const int64_t total = nbricks * kBrick;
    const T INF = Num<T>::inf();
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = t >> 9;
        const int p = static_cast<int>(t & 511);
        const int bx = static_cast<int>(b % BX), by = static_cast<int>((b / BX) % BY),
                  bz = static_cast<int>(b / (static_cast<int64_t>(BX) * BY));
        const int i = bx * 8 + (p & 7), j = by * 8 + ((p >> 3) & 7), k = bz * 8 + (p >> 6);
        T r = INF;
        if (i < nx && j < ny && k < nz) {
            const T f = F[(static_cast<int64_t>(k) * ny + j) * nx + i];
            if (!(f >= 0) || !(f < INF)) atomicOr(err, 1);
            else if (f > 0) r = static_cast<T>(h / static_cast<double>(f));
        }
        rr[t] = r;
    }
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
    const int64_t plane = static_cast<int64_t>(nx) * ny;
    const int64_t total = plane * (z_end - z_begin);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int k = z_begin + static_cast<int>(t / plane);
        const int64_t rem = t % plane;
        const int j = static_cast<int>(rem / nx), i = static_cast<int>(rem % nx);
        const int64_t b = (static_cast<int64_t>(k >> 3) * BY + (j >> 3)) * BX + (i >> 3);
        const int p = ((k & 7) * 8 + (j & 7)) * 8 + (i & 7);
        const unsigned long long st = stamp[b];
        out[t] = (st == kUntouched) ? INF : slot[(b * 2 + stamp_copy(st)) * kSlot + p];
    }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers (called from eik_runtime.cu)
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_layout_speed(const T* F, T* rr, int nx, int ny, int nz, int BX, int BY, int64_t nbricks,
                                double h, int* err, cudaStream_t s) {
    const int64_t total = nbricks * kBrick;
    int grid = static_cast<int>((total + 255) / 256);
    if (grid > 65535 * 4) grid = 65535 * 4;
    k_layout_speed<T><<<grid, 256, 0, s>>>(F, rr, nx, ny, nz, BX, BY, nbricks, h, err);
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
    const int64_t total = static_cast<int64_t>(nx) * ny * (z_end - z_begin);
    int grid = static_cast<int>((total + 255) / 256);
    if (grid > 65535 * 4) grid = 65535 * 4;
    if (grid < 1) grid = 1;
    k_result<T><<<grid, 256, 0, s>>>(slot, stamp, out, nx, ny, z_begin, z_end, BX, BY);
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
                                                cudaStream_t);                                                   \
    template cudaError_t launch_init_sources<T>(int, const int32_t*, const int32_t*, const double*, int,         \
                                                const int32_t*, int, const int32_t*, int, const int32_t*, T*,     \
                                                unsigned long long*, unsigned long long*, int32_t*, int32_t*, T*,  \
                                                T*, int32_t*, int32_t*, cudaStream_t);                            \
    template cudaError_t launch_restore_r<T>(int, const int32_t*, const int32_t*, const T*, T*, cudaStream_t);   \
    template cudaError_t launch_gather_r<T>(int, const int32_t*, const int32_t*, const T*, double*,              \
                                            cudaStream_t);                                                       \
    template cudaError_t launch_result<T>(const T*, const unsigned long long*, T*, int, int, int, int, int, int, \
                                          cudaStream_t);                                                         \
    template size_t loop_smem_bytes<T>();                                                                        \
    template cudaError_t loop_occupancy<T>(int*);                                                                \
    template cudaError_t launch_restart_loop<T>(const LoopParams<T>&, int, cudaStream_t);

EIKG_INSTANTIATE(float)
EIKG_INSTANTIATE(double)

}  // namespace eikg
