// Device code shared by the restart-loop kernels (one grid, eik_kernels.cu;
// many grids, eik_batch.cu): the upwind root of Alg. 3, the per-warp shared
// memory of a march, and March_Narrow_Band (Alg. 4 with Algs. 2, 3 and the
// ghost exchange of Alg. 5).
//
// One warp marches one 8x8x8 block (a "brick").  The brick's psi, h/F and its
// six ghost faces sit in shared memory; lane L loads and writes back the two
// x-rows (y = L & 7, z = 2*(L >> 3) + {0, 1}) and face-local nodes 2L, 2L+1 of
// each ghost face.  The band (Sec. 2.1 BAND set) is a list of halo indices
// shared by the warp; a band node's value carries its sign bit set in shared
// memory so that any lane can tell a tentative value from an accepted (KNOWN)
// one with one load.
//
// Ordered extraction (Alg. 4) is done in rounds: each round accepts every band
// node with psi <= min(m + w, bound), m the band minimum, w = omega * min(h/F)
// over the brick; the accepted nodes' neighbours (Alg. 2) come from shifting a
// halo bit vector of the accepted nodes, are compacted into a list and
// re-solved (Alg. 3) 32 at a time.  A lowered node rejoins the band, so an
// accepted node can be refreshed later exactly as a KNOWN_NEW node of the
// paper can.  With w = 0 this is the paper's one-node-at-a-time order.
//
// The rest of the file is the restart loop's shared machinery: the work-list
// ring, the per-warp grid barrier and the early marches of the next restart.
#pragma once

#include "eik_internal.cuh"

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
__device__ __forceinline__ unsigned ubits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned long long ubits(double v) {
    return static_cast<unsigned long long>(__double_as_longlong(v));
}
__device__ __forceinline__ float from_bits(unsigned u) { return __uint_as_float(u); }
__device__ __forceinline__ double from_bits(unsigned long long u) {
    return __longlong_as_double(static_cast<long long>(u));
}
__device__ __forceinline__ float vabs(float v) { return fabsf(v); }
__device__ __forceinline__ double vabs(double v) { return fabs(v); }
// Min, max and order of values that are >= 0 or +inf (every use in the march):
// single precision on the FP32 units; double precision as integer operations on
// the bit patterns, which order like such values, keeping them off this part's
// narrow FP64 pipe.
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) {
    const unsigned long long x = ubits(a), y = ubits(b);
    return from_bits(x < y ? x : y);
}
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) {
    const unsigned long long x = ubits(a), y = ubits(b);
    return from_bits(x > y ? x : y);
}
__device__ __forceinline__ bool vlt(float a, float b) { return a < b; }
__device__ __forceinline__ bool vlt(double a, double b) { return ubits(a) < ubits(b); }

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
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// Alg. 3: the upwind root for sorted upwind values a <= b <= c (b, c may be
// +inf) and r = h/F.  Alg. 3 solves sum_i (x - v_i)^2 = r^2 (Eq. (2.1)-(2.2))
// for the id smallest values, growing id while the root exceeds the next
// value.  Equivalently the root is the x with G(x) = r^2, where
//   G(x) = sum_i max(x - v_i, 0)^2
// is non-decreasing in x and non-increasing in every v_i: a value v_i >= x
// adds nothing, which is the growth rule of Alg. 3.
//
// The result returned is the value x of the working precision at which
// G_fl(x) comes nearest r^2 from either side (root_search), G_fl being G
// evaluated with round-to-nearest operations in a fixed order (largest term
// first; no contraction).  Every operation in G_fl is monotone in its
// operands, so G_fl keeps both monotonicities, and the returned root is then
// a monotone function of (a, b, c): a neighbour that is lower can never give
// a higher root.  The discrete solution is the
// greatest fixed point of psi_p = min(psi_p, root_p(neighbours)) below the
// initial values (+inf off the sources); iterations of a monotone map from
// above reach that one fixed point in any order, so psi does not depend on
// the stride, the schedule, the block edge or the order of the marches, bit
// for bit.
//
// The search starts from a fast estimate of the root, written without
// cancellation: with k admitted values,
//   x = v_1 + (sum_i (v_i - v_1) + sqrt(D)) / k,
//   D = k r^2 - sum_{i<j} (v_i - v_j)^2          (Lagrange's identity),
// whose differences are exact.  Whenever a value is admitted D > r^2 in
// exact arithmetic, so D < tau*k*r^2 (tau < 1/3) only flags rounding trouble;
// the estimate is then taken in double precision.  The estimate is within an
// ulp or two of the result, so the search usually evaluates G_fl twice (at
// the estimate and one ulp away): it gallops outwards from the estimate until
// the result is bracketed, then bisects on the bit patterns (non-negative
// values order like their bits).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double clamp0(double D) { return (ubits(D) >> 63) ? 0.0 : D; }

__device__ __forceinline__ float gsum(float x, float a, float b, float c) {
    const float ta = fmaxf(__fsub_rn(x, a), 0.0f), tb = fmaxf(__fsub_rn(x, b), 0.0f);
    const float tc = fmaxf(__fsub_rn(x, c), 0.0f);
    return __fadd_rn(__fadd_rn(__fmul_rn(ta, ta), __fmul_rn(tb, tb)), __fmul_rn(tc, tc));
}
// (max with 0 by the sign bit: the FP64 pipe of this part is narrow)
__device__ __forceinline__ double gsum(double x, double a, double b, double c) {
    const double ta = clamp0(__dsub_rn(x, a)), tb = clamp0(__dsub_rn(x, b)), tc = clamp0(__dsub_rn(x, c));
    return __dadd_rn(__dadd_rn(__dmul_rn(ta, ta), __dmul_rn(tb, tb)), __dmul_rn(tc, tc));
}

template <typename T>
struct BitsOf;
template <>
struct BitsOf<float> {
    using U = unsigned;
    static constexpr U kInf = 0x7f800000u;
};
template <>
struct BitsOf<double> {
    using U = unsigned long long;
    static constexpr U kInf = 0x7ff0000000000000ull;
};

// The root: with hi the smallest value of precision T above a with
// gsum(hi) >= r2, and lo the value just below it (gsum(lo) < r2), the one of
// the two whose gsum is nearer r2 (lo on a tie of the distances is not taken).
// Near the root G is linear to far below an ulp of x, so this is the root
// rounded to nearest, without the upward drift that always taking hi would
// add at every step along a characteristic.  It stays monotone: lower values
// (b, c, a) raise gsum everywhere, so hi cannot move up, and if it stays put
// the distance r2 - gsum(lo) can only shrink and gsum(hi) - r2 only grow
// (rounded subtraction is monotone), so lo can only become more likely.
// Searched from the estimate x0 (out of line: the estimate is almost always
// within an ulp of the result, which root_near settles in two evaluations).
template <typename T>
__device__ __noinline__ T root_search(T x0, T a, T b, T c, T r2) {
    using U = typename BitsOf<T>::U;
    const U ua = ubits(a);
    U g = ubits(x0);
    if (!(g > ua) || g > BitsOf<T>::kInf) g = ua + 1;
    U lo, hi;                       // gsum(lo) < r2 <= gsum(hi); lo = a needs no evaluation (G(a) = 0)
    T glo, ghi;
    U step = 1;
    T gg = gsum(from_bits(g), a, b, c);
    if (gg >= r2) {
        hi = g;
        ghi = gg;
        for (;;) {
            const U cand = (hi - ua > step) ? hi - step : ua;
            if (cand == ua) {
                lo = ua;
                glo = 0;
                break;
            }
            const T gc = gsum(from_bits(cand), a, b, c);
            if (!(gc >= r2)) {
                lo = cand;
                glo = gc;
                break;
            }
            hi = cand;
            ghi = gc;
            step <<= 1;
        }
    } else {
        lo = g;
        glo = gg;
        for (;;) {
            const U cand = (BitsOf<T>::kInf - lo > step) ? lo + step : BitsOf<T>::kInf;
            const T gc = gsum(from_bits(cand), a, b, c);
            if (cand == BitsOf<T>::kInf || gc >= r2) {
                hi = cand;
                ghi = gc;
                break;
            }
            lo = cand;
            glo = gc;
            step <<= 1;
        }
    }
    while (hi - lo > 1) {
        const U mid = lo + ((hi - lo) >> 1);
        const T gm = gsum(from_bits(mid), a, b, c);
        if (gm >= r2) {
            hi = mid;
            ghi = gm;
        } else {
            lo = mid;
            glo = gm;
        }
    }
    return (r2 - glo < ghi - r2) ? from_bits(lo) : from_bits(hi);
}

// The same root when it lies within an ulp of the estimate x0, which is the
// usual case: G at x0 says on which side of the crossing x0 lies, G one value
// further that way closes the bracket.  Otherwise the general search.
template <typename T>
__device__ __forceinline__ T root_near(T x0, T a, T b, T c, T r2) {
    using U = typename BitsOf<T>::U;
    const U g = ubits(x0);
    if (g > ubits(a) && g < BitsOf<T>::kInf) {
        const T g0 = gsum(x0, a, b, c);
        const bool up = !(g0 >= r2);                 // x0 below the crossing
        const U g1 = up ? g + 1 : g - 1;
        const T x1 = from_bits(g1);
        const T gx1 = gsum(x1, a, b, c);
        if (up == (gx1 >= r2)) {
            const T glo = up ? g0 : gx1, ghi = up ? gx1 : g0;
            return (r2 - glo < ghi - r2) ? (up ? x0 : x1) : (up ? x1 : x0);
        }
    }
    return root_search<T>(x0, a, b, c, r2);
}

// The estimate (with the causality clamps: in exact arithmetic the root is not
// below the largest admitted value).  (The division by 3 as a product.)
__device__ __forceinline__ double root_estimate(double a, double b, double c, double r) {
    double x = a + r;
    if (!vlt(b, x)) return x;
    const double d = b - a;
    const double r2 = r * r;
    double D = 2.0 * r2 - d * d;
    x = vmax(a + (d + sqrt(clamp0(D))) * 0.5, b);
    if (!vlt(c, x)) return x;
    const double e = c - a, g = c - b;
    D = 3.0 * r2 - (d * d + e * e + g * g);
    return vmax(a + (d + e + sqrt(clamp0(D))) * (1.0 / 3.0), c);
}

__device__ __forceinline__ double upwind_root(double a, double b, double c, double r) {
    return root_near<double>(root_estimate(a, b, c, r), a, b, c, __dmul_rn(r, r));
}

// FP32: sqrt(D) as D * rsqrt(D) (the hardware reciprocal square root, a few
// ulp) and the division by 3 as a product; D >= tau*k*r^2 > 0 on this path
// (the max guards tau = 0).  When (h/F)^2 underflows single precision the whole
// root is taken in double precision and rounded (rounding is monotone too).
__device__ __forceinline__ float sqrt_f32(float D) { return D * rsqrtf(fmaxf(D, FLT_MIN)); }

// (the double-precision paths out of line: they almost never run, and inlined
// they would crowd the instruction cache around the hot solve loop)
static __device__ __noinline__ float root_in_double(float a, float b, float c, float r) {
    return static_cast<float>(upwind_root(a, b, c, r));
}
static __device__ __noinline__ float estimate_in_double(float a, float b, float c, float r) {
    return static_cast<float>(root_estimate(a, b, c, r));
}

__device__ __forceinline__ float upwind_root_f32(float a, float b, float c, float r, float tau, int& fb) {
    const float r2 = __fmul_rn(r, r);
    if (!(r2 >= FLT_MIN)) {
        ++fb;
        return root_in_double(a, b, c, r);
    }
    float x = a + r;
    if (x > b) {
        const float d = b - a;
        float D = 2.0f * r2 - d * d;
        if (!(D >= tau * 2.0f * r2)) {
            ++fb;
            x = estimate_in_double(a, b, c, r);
        } else {
            x = fmaxf(a + (d + sqrt_f32(D)) * 0.5f, b);
            if (x > c) {
                const float e = c - a, g = c - b;
                D = 3.0f * r2 - (d * d + e * e + g * g);
                if (!(D >= tau * 3.0f * r2)) {
                    ++fb;
                    x = estimate_in_double(a, b, c, r);
                } else {
                    x = fmaxf(a + (d + e + sqrt_f32(D)) * (1.0f / 3.0f), c);
                }
            }
        }
    }
    return root_near<float>(x, a, b, c, r2);
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

// The value of precision T among a double and its single-precision copy
// (prepared once per restart, so that marches do no double arithmetic).
template <typename T>
__device__ __forceinline__ T pick(double d, float f);
template <>
__device__ __forceinline__ float pick<float>(double, float f) { return f; }
template <>
__device__ __forceinline__ double pick<double>(double d, float) { return d; }

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
    uint16_t list[kBrick];  // nodes to re-solve in the current round (halo index)
    uint32_t mark[32];      // one warp: halo bit vector of the nodes accepted in this round;
                            // group of warps: bit per brick node, neighbour of a node accepted this round
    uint32_t upd[16];       // bit per brick node: lowered in this march (Upsilon)
    uint32_t fxob[16];      // bit per brick node: fixed, barrier or padding node (never solved)
};

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) of global memory
// into L2, without a destination or a completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

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

// Minimum over the warp of values that are >= 0 (+inf allowed): the bits of
// non-negative IEEE numbers order like unsigned integers, so one integer
// reduction (two for FP64: high words, then low words among the lanes holding
// the smallest high word) replaces the five shuffle-and-min steps.  A NaN sits
// above +inf as an integer and loses to any number, as it does in fmin.
__device__ __forceinline__ float warp_min_nn(float v) {
    return __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(v)));
}
__device__ __forceinline__ double warp_min_nn(double v) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v));
    const unsigned hi = static_cast<unsigned>(u >> 32), lo = static_cast<unsigned>(u);
    const unsigned mh = __reduce_min_sync(kFull, hi);
    const unsigned ml = __reduce_min_sync(kFull, hi == mh ? lo : 0xffffffffu);
    return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(mh) << 32) | ml));
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
    unsigned accepted;                       // per lane
    unsigned band;                           // counted on lane 0
    int fallbacks;                           // per lane
    unsigned updates;                        // per lane
    unsigned solves, rounds;                 // the same on every lane (one restart of one warp)
    float rmin, rmax;                        // the same on every lane
};

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

// Where a grid sits in the work space of a launch: its bricks are the global
// indices [boff, boff + BX*BY*BZ), its 2x2x2 groups [goff, goff + GX*GY*GZ).
// One grid per launch has boff = goff = 0.
struct Geo {
    int32_t BX, BY, BZ;
    int32_t boff;
    int32_t GX, GY;
    int32_t goff;
    uint32_t lists;            // bit 0: keep the brick work list; bit 1: keep the group work list
};

// Put brick x (global index; and, if the group work list is kept, its group)
// on restart k+1's work lists, once per restart (the "queued" marks dedupe).
template <typename T>
__device__ __forceinline__ void enqueue_next(const LoopParams<T>& P, const Geo& G, int k, int32_t x) {
    const int s = (k + 1) % kRing;
    if (P.pause) {                       // a sharded grid: ghost bricks belong to another GPU
        const int bz = (x - G.boff) / (G.BX * G.BY);
        if (bz < P.own_bz0 || bz >= P.own_bz1) return;
    }
    if ((G.lists & 1u) && atomicMax(P.queued + s * P.nbricks + x, k + 1) < k + 1) {
        const int pos = atomicAdd(&P.ctrl->count[s], 1);
        P.list[s][pos] = x;
    }
    if (!(G.lists & 2u)) return;
    const int xl = x - G.boff;
    const int bx = xl % G.BX, by = (xl / G.BX) % G.BY, bz = xl / (G.BX * G.BY);
    const int32_t g = G.goff + ((bz >> 1) * G.GY + (by >> 1)) * G.GX + (bx >> 1);
    if (atomicMax(P.qgroup + s * P.ngroups + g, k + 1) < k + 1) {
        const int pos = atomicAdd(&P.ctrl->gcount[s], 1);
        P.glist[s][pos] = g;
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
__device__ void march(const LoopParams<T>& P, const Geo& G, WarpSmem<T>* SW, int warp, int32_t b, unsigned gmask,
                      int k, T bprev, T bound, bool grow, T window, int lane, MarchAcc& acc, bool publish,
                      int32_t pf = -1) {
    __shared__ T s_wmin[kWarps];
    __shared__ T s_bmin[2][kWarps];            // group rounds: band minima, by round parity
    WarpSmem<T>& S = SW[warp];
    const T INF = Num<T>::inf();
    const bool present = b >= 0;
    const int y = lane & 7, zp = lane >> 3, z0 = 2 * zp;
    const int BX = G.BX, BY = G.BY, BZ = G.BZ;
    const int bb = present ? b : G.boff;                         // global index; coordinates are local
    const int bl = bb - G.boff;
    const int bx = bl % BX, by = (bl / BX) % BY, bz = bl / (BX * BY);
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
        // a brick further down this restart's list (pf >= 0): its stamp now, and
        // once it has landed (below) bulk L2 prefetches of its h/F and latest copy
        const unsigned long long pst = (pf >= 0 && lane == 0) ? __ldcg(P.stamp + pf) : kUntouched;
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
        if (pf >= 0 && lane == 0) {
            prefetch_l2(P.rr + static_cast<int64_t>(pf) * kBrick, kBrick * sizeof(T));
            if (pst != kUntouched)
                prefetch_l2(P.slot + (static_cast<int64_t>(pf) * 2 + stamp_copy(pst)) * kSlot, kSlot * sizeof(T));
        }
        // ---- the band at the start of the march (marked as the values land in
        // shared memory): the brick's finite nodes above the previous bound, and
        // the ghost nodes that are above it or that the neighbour lowered in
        // restart k-1 (Upsilon) -- the heap contents of Alg. 4 after Alg. 5.
        // Lane L marks its two rows (bits 0-15 of B) and face-local nodes 2L and
        // 2L+1 of each face (bits 2f and 2f+1 of G).
        unsigned B = 0, G = 0;
        if (st == kUntouched) {
#pragma unroll
            for (int x = 0; x < 8; ++x) S.psi[hbase + x] = INF, S.psi[hbase + 100 + x] = INF;
        } else {
            const T* src = P.slot + (static_cast<int64_t>(b) * 2 + stamp_copy(st)) * kSlot;
            T row[8], row1[8];
            load8_cg(src + pbase, row);
            load8_cg(src + pbase + 64, row1);
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const T v0 = row[x], v1 = row1[x];
                const bool b0 = v0 < INF && v0 > bprev, b1 = v1 < INF && v1 > bprev;
                S.psi[hbase + x] = b0 ? -v0 : v0;
                S.psi[hbase + 100 + x] = b1 ? -v1 : v1;
                B |= (b0 ? 1u : 0u) << x;
                B |= (b1 ? 1u : 0u) << (8 + x);
            }
        }
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const int h0 = face_ghost_halo(f, u);
            const T g0 = fv0[f], g1 = fv1[f];
            const bool b0 = g0 < INF && (((fups[f] >> u) & 1ull) || g0 > bprev);
            const bool b1 = g1 < INF && (((fups[f] >> (u + 1)) & 1ull) || g1 > bprev);
            S.psi[h0] = b0 ? -g0 : g0;
            S.psi[h0 + (f < 2 ? 10 : 1)] = b1 ? -g1 : g1;
            G |= ((b0 ? 1u : 0u) | (b1 ? 2u : 0u)) << (2 * f);
        }
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
        for (unsigned m = G; m; m &= m - 1) {
            const int j = __ffs(m) - 1, f = j >> 1;
            S.band[off++] = static_cast<uint16_t>(face_ghost_halo(f, u) + ((j & 1) ? (f < 2 ? 10 : 1) : 0));
        }
    }
    if (lane < 16) {
        S.mark[lane] = 0u;
        S.upd[lane] = 0u;
        S.fxob[lane] = 0u;
    }
    __syncwarp();
    if constexpr (GROUP) {
        if (FXOB & 0xFFu) atomicOr(&S.fxob[pbase >> 5], (FXOB & 0xFFu) << (pbase & 31));
        if (FXOB >> 8) atomicOr(&S.fxob[(pbase + 64) >> 5], (FXOB >> 8) << ((pbase + 64) & 31));
    }

    const T rmin_b = warp_min_nn(rlo);
    if (present) {
        acc.rmin = fminf(acc.rmin, static_cast<float>(rmin_b));
        acc.rmax = fmaxf(acc.rmax, static_cast<float>(warp_max(rhi)));
    }
    T w;
    if constexpr (GROUP) {
        // one window for the group: omega times the smallest h/F of its bricks
        if (lane == 0) s_wmin[warp] = rmin_b;
        __syncthreads();
        T g = s_wmin[0];
#pragma unroll
        for (int i = 1; i < kWarps; ++i) g = vmin(g, s_wmin[i]);
        w = window * g;
        __syncthreads();
    } else {
        w = window * rmin_b;
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

    // Alg. 3 for each listed node (halo index), 32 at a time; new values land
    // after the reads.  A lowered node is tagged BAND (Alg. 2) and joins the band
    // unless it is in it already.  Returns this lane's smallest lowered value.
    auto solve_list = [&](int total) -> T {
        T smin = INF;
        for (int base = 0; base < total; base += 32) {
            const int idx = base + lane;
            bool imp = false, known = false;
            T xn = 0;
            int hq = 0, q = 0;
            if (idx < total) {
                hq = S.list[idx];
                // brick index of the halo position: z = hq / 100, y = (hq % 100) / 10 (exact for hq < 1000)
                const int hz = (hq * 41) >> 12, rem = hq - 100 * hz, hy = (rem * 103) >> 10;
                q = hz * 64 + hy * 8 + (rem - 10 * hy) - 73;
                const T cur = S.psi[hq];
                const T c = vabs(cur);
                known = !sgn(cur);
                // KNOWN neighbours below the node's current value (Alg. 3's test): as
                // unsigned bit patterns every KNOWN (sign clear) value orders as its
                // value and every BAND value (sign set) lies above any KNOWN one
                // (per axis: the smaller bit pattern of the two neighbours is the
                // smaller KNOWN value if either is KNOWN; it counts if below c)
                const auto cb = ubits(c);
                auto axis = [&](T a, T b) -> T {
                    const auto ua = ubits(a), ub = ubits(b);
                    const auto m = ua < ub ? ua : ub;
                    return m < cb ? from_bits(m) : INF;
                };
                T mx = axis(S.psi[hq - 1], S.psi[hq + 1]);
                T my = axis(S.psi[hq - 10], S.psi[hq + 10]);
                T mz = axis(S.psi[hq - 100], S.psi[hq + 100]);
                // reorder psi_1 <= psi_2 <= psi_3
                T lo = vmin(mx, my), hi = vmax(mx, my);
                T a0 = vmin(lo, mz);
                T t1 = vmax(lo, mz);
                T a1 = vmin(hi, t1), a2 = vmax(hi, t1);
                if (vlt(a0, INF)) {
                    xn = RootOf<T>::go(a0, a1, a2, S.r[q], tau, acc.fallbacks);
                    imp = vlt(xn, c);
                }
            }
            __syncwarp();
            const bool add = imp && known;
            const unsigned am = __ballot_sync(kFull, add);
            if (imp) {
                S.psi[hq] = -xn;
                atomicOr(&S.upd[q >> 5], 1u << (q & 31));
                smin = vmin(smin, xn);
            }
            if (add) S.band[n + __popc(am & lt)] = static_cast<uint16_t>(hq);
            n += __popc(am);
            acc.updates += imp ? 1u : 0u;
            __syncwarp();
        }
        return smin;
    };
    // lane-distributed bit set -> S.list (ascending), returns the entry count
    auto compact = [&](unsigned bits, int first) -> int {
        const int cnt = __popc(bits);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        int off = incl - cnt;
        for (unsigned m = bits; m; m &= m - 1) S.list[off++] = static_cast<uint16_t>(first + __ffs(m) - 1);
        __syncwarp();
        return __shfl_sync(kFull, incl, 31);
    };

    // ---- rounds of windowed ordered acceptance (Alg. 4)
    int rounds = 0;
    if constexpr (GROUP) {
        for (;;) {
            T lmin = INF;
            for (int i = lane; i < n; i += 32) lmin = vmin(lmin, vabs(S.psi[S.band[i]]));
            T mn = warp_min_nn(lmin);
            // (two buffers by round parity: the barriers later in the round order
            // these reads before the writes two rounds on, so one barrier suffices)
            T* bm = s_bmin[rounds & 1];
            if (lane == 0) bm[warp] = mn;
            __syncthreads();
            T g = bm[0];
#pragma unroll
            for (int i = 1; i < kWarps; ++i) g = vmin(g, bm[i]);
            mn = g;
            if (!(mn < INF) || !(mn <= bound)) break;   // band empty, or its minimum above the bound
            if (++rounds > kRoundCap) {
                atomicOr(&P.ctrl->status, kStRoundCap);
                break;
            }
            const T thr = vmin(mn + w, bound);
            // accept (Remove_Min of a window), keep the rest of the band in order,
            // and mark the accepted nodes' neighbours (Alg. 2), across internal
            // faces in the neighbouring warp's tile
            int kept = 0;
            for (int base = 0; base < n; base += 32) {
                const int i = base + lane;
                int hh = 0;
                bool keep = false, take = false;
                if (i < n) {
                    hh = S.band[i];
                    const T v = vabs(S.psi[hh]);
                    if (!vlt(thr, v)) {
                        take = true;
                        S.psi[hh] = v;
                    } else {
                        keep = true;
                    }
                }
                const unsigned km = __ballot_sync(kFull, keep);
                if (keep) S.band[kept + __popc(km & lt)] = static_cast<uint16_t>(hh);
                kept += __popc(km);
                acc.accepted += take ? 1u : 0u;
                if (take) {
                    const int px = hh % 10 - 1, py = (hh / 10) % 10 - 1, pz = hh / 100 - 1;
                    auto cand = [&](int x, int yy, int z) {
                        const bool ix = static_cast<unsigned>(x) < 8u, iy = static_cast<unsigned>(yy) < 8u,
                                   iz = static_cast<unsigned>(z) < 8u;
                        if (ix && iy && iz) {
                            const int q = (z * 8 + yy) * 8 + x;
                            atomicOr(&S.mark[q >> 5], 1u << (q & 31));
                        } else {
                            int f = -1;
                            if (!ix && iy && iz) f = (x < 0) ? 0 : 1;
                            else if (ix && !iy && iz) f = (yy < 0) ? 2 : 3;
                            else if (ix && iy && !iz) f = (z < 0) ? 4 : 5;
                            if (f >= 0 && ((gmask >> f) & 1u)) {
                                const int q = (((z & 7) * 8) + (yy & 7)) * 8 + (x & 7);
                                atomicOr(&SW[warp ^ (1 << (f >> 1))].mark[q >> 5], 1u << (q & 31));
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
            __syncthreads();
            refresh_internal();
            __syncthreads();
            // candidates (brick bits, 16 per lane) -> list of halo indices; never-solved nodes dropped
            const unsigned word = S.mark[lane >> 1] & ~S.fxob[lane >> 1];
            const unsigned wd = (lane & 1) ? (word >> 16) : (word & 0xFFFFu);
            __syncwarp();
            if (lane < 16) S.mark[lane] = 0u;
            const int total = compact(wd, 16 * lane);   // brick indices
            for (int i = lane; i < total; i += 32) S.list[i] = static_cast<uint16_t>(halo_of(S.list[i]));
            __syncwarp();
            acc.solves += total;
            solve_list(total);
            // no barrier or refresh here: the next round's first barrier orders these
            // writes before any other warp's marks and reads, and the ghost layer is
            // refreshed after the next accept pass, before any solve reads it
        }
    } else {
        // Halo bit vectors, one 32-bit word per lane (bit j of lane L's word is
        // halo position 32L + j): `solv` marks the nodes that are solved (not
        // fixed, barrier or padding); S.mark collects each round's accepted
        // nodes, whose neighbours are the vector shifted by +-1, +-10, +-100.
        // Every shift lands an interior node's true neighbour or a ghost
        // position, and ghost positions are not in `solv`.
        S.mark[lane] = 0u;
        __syncwarp();
        {
            auto put = [&](int h0, unsigned bits) {
                if (!bits) return;
                atomicOr(&S.mark[h0 >> 5], bits << (h0 & 31));
                if ((h0 & 31) > 24) atomicOr(&S.mark[(h0 >> 5) + 1], bits >> (32 - (h0 & 31)));
            };
            put(hbase, ~FXOB & 0xFFu);
            put(hbase + 100, (~FXOB >> 8) & 0xFFu);
        }
        __syncwarp();
        const unsigned solv = S.mark[lane];
        __syncwarp();
        S.mark[lane] = 0u;
        __syncwarp();
        T lmin = INF;
        for (int i = lane; i < n; i += 32) lmin = vmin(lmin, vabs(S.psi[S.band[i]]));
        T mn = warp_min_nn(lmin);
        for (;;) {
            if (!(mn < INF) || !(mn <= bound)) break;   // band empty, or its minimum above the bound
            if (++rounds > kRoundCap) {
                atomicOr(&P.ctrl->status, kStRoundCap);
                break;
            }
            const T thr = vmin(mn + w, bound);
            // accept (Remove_Min of a window) and keep the rest of the band in
            // order, with the minimum of what is kept
            // (the next chunk's entries are loaded before this chunk's stores, which
            // only touch earlier band slots and the accepted nodes themselves)
            int kept = 0;
            T kmin = INF;
            int hh = 0;
            T v = INF;
            if (lane < n) {
                hh = S.band[lane];
                v = vabs(S.psi[hh]);
            }
            for (int base = 0; base < n; base += 32) {
                const bool valid = base + lane < n;
                int hh2 = 0;
                T v2 = INF;
                if (base + 32 + lane < n) {
                    hh2 = S.band[base + 32 + lane];
                    v2 = vabs(S.psi[hh2]);
                }
                const bool take = valid && !vlt(thr, v);
                const bool keep = valid && !take;
                if (take) {
                    S.psi[hh] = v;
                    atomicOr(&S.mark[hh >> 5], 1u << (hh & 31));
                }
                if (keep) kmin = vmin(kmin, v);
                const unsigned km = __ballot_sync(kFull, keep);
                if (keep) S.band[kept + __popc(km & lt)] = static_cast<uint16_t>(hh);
                kept += __popc(km);
                hh = hh2;
                v = v2;
            }
            if (lane == 0) acc.accepted += static_cast<unsigned>(n - kept);   // every entry is taken or kept
            n = kept;
            __syncwarp();
            // neighbours of the accepted nodes (Alg. 2) that are solved
            const unsigned W = S.mark[lane];
            unsigned wm1 = __shfl_up_sync(kFull, W, 1), wm3 = __shfl_up_sync(kFull, W, 3);
            unsigned wm4 = __shfl_up_sync(kFull, W, 4), wp1 = __shfl_down_sync(kFull, W, 1);
            unsigned wp3 = __shfl_down_sync(kFull, W, 3), wp4 = __shfl_down_sync(kFull, W, 4);
            if (lane < 1) wm1 = 0u;
            if (lane < 3) wm3 = 0u;
            if (lane < 4) wm4 = 0u;
            if (lane > 30) wp1 = 0u;
            if (lane > 28) wp3 = 0u;
            if (lane > 27) wp4 = 0u;
            const unsigned d = (__funnelshift_l(wm1, W, 1) | __funnelshift_l(wm1, W, 10) | __funnelshift_l(wm4, wm3, 4) |
                                __funnelshift_r(W, wp1, 1) | __funnelshift_r(W, wp1, 10) | __funnelshift_r(wp3, wp4, 4)) &
                               solv;
            S.mark[lane] = 0u;
            const int total = compact(d, 32 * lane);
            acc.solves += total;
            const T smin = solve_list(total);
            mn = warp_min_nn(vmin(kmin, smin));
        }
    }
    acc.rounds += rounds;
    if constexpr (GROUP) __syncthreads();
    if (!present) return;

    // ---- Upsilon: own face nodes lowered in this march, per face (face-local bit
    // masks); none on internal faces of a group, whose neighbours saw them live
    const unsigned U = ((S.upd[pbase >> 5] >> (pbase & 31)) & 0xFFu) |
                       (((S.upd[(pbase + 64) >> 5] >> ((pbase + 64) & 31)) & 0xFFu) << 8);
    unsigned long long um[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    // A march that lowered no value leaves the brick as its latest copy holds it
    // (which nodes are accepted follows from the bounds), so it writes nothing:
    // readers keep taking that copy, and its Upsilon masks, written in an earlier
    // restart, are not applied again.
    if (__any_sync(kFull, U != 0u)) {
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
    }

    // ---- activation for restart k+1 (A of Alg. 4/5, C of Alg. 4)
    // (once the bound has reached width_band, pending nodes above it stay tentative: Alg. 6's A flag)
    if (lane == 6 && n > 0 && grow) enqueue_next(P, G, k, b);
    if (lane < 6 && um[lane] != 0ull && nbr[lane] >= 0) enqueue_next(P, G, k, nbr[lane]);
    if (lane == 0) acc.band += n;
    // publish: the brick's restart-k march has finished (read by early marches
    // of its neighbours; the release store orders the warp's writes above it)
    if (publish) {
        __syncwarp();
        if (lane == 0) st_release(P.done + b, k);
    }
}

// Work-list entry i of ring slot s.  An early taker may get an index whose
// entry is not written yet (the enqueuer bumps the count, then stores): it
// waits for it (bounded; -1 on timeout).  Unwritten entries are -1: a slot is
// cleared at the start of the restart after the one that used it
// (clear_used_slot), before it is used again two restarts later.
__device__ __forceinline__ int32_t take_entry(const int32_t* list, int i, bool wait, long long limit, int lane) {
    if (!wait) return __ldcg(list + i);
    int32_t v = -1;
    if (lane == 0) {
        v = ld_acquire(list + i);
        for (long long it = 0; v < 0 && it < limit; ++it) {
            __nanosleep(32);
            v = ld_acquire(list + i);
        }
    }
    return __shfl_sync(0xffffffffu, v, 0);
}

// At the start of restart k: every thread of the launch clears its share of the
// brick list restart k-1 used (ring slot (k-1) mod kRing), coalesced.  The
// slot is next written in restart k+1 (by early marches of restart k+2 while
// waiting at its barrier) at the earliest, after every warp has arrived at the
// barrier of restart k and so has finished its share.
template <typename T>
__device__ __forceinline__ void clear_used_slot(const LoopParams<T>& P, int k) {
    const int sp = (k + kRing - 1) % kRing;
    const int m = __ldcg(&P.ctrl->used[sp]);
    int32_t* list = P.list[sp];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) list[i] = -1;
}

// Before an early march of brick b at restart k+1: wait until b and each of its
// six neighbours that is on restart k's work list has finished that march
// (bounded; false on timeout).  After it the march reads what it would read
// after the barrier of restart k.
template <typename T>
__device__ bool wait_ready(const LoopParams<T>& P, const Geo& G, int32_t b, int k, int lane) {
    int32_t x = -1;
    if (lane < 7) {
        const int bl = b - G.boff;
        const int bx = bl % G.BX, by = (bl / G.BX) % G.BY, bz = bl / (G.BX * G.BY);
        if (lane == 6) x = b;
        else if (lane == 0) x = bx > 0 ? b - 1 : -1;
        else if (lane == 1) x = bx < G.BX - 1 ? b + 1 : -1;
        else if (lane == 2) x = by > 0 ? b - G.BX : -1;
        else if (lane == 3) x = by < G.BY - 1 ? b + G.BX : -1;
        else if (lane == 4) x = bz > 0 ? b - G.BX * G.BY : -1;
        else x = bz < G.BZ - 1 ? b + G.BX * G.BY : -1;
    }
    bool need = x >= 0 && __ldcg(P.queued + (k % kRing) * P.nbricks + x) == k;
    unsigned nap = 128;
    for (long long it = 0;; ++it) {
        if (need && ld_acquire(P.done + x) >= k) need = false;
        if (!__any_sync(0xffffffffu, need)) break;
        if (it > P.wait_limit) return false;
        __nanosleep(nap);
        if (nap < 2048) nap <<= 1;
    }
    __syncwarp();
    return true;
}

// This warp's statistics of the restart -> the control block.
__device__ __forceinline__ void flush_acc(Ctrl* C, MarchAcc& acc, int lane) {
    const unsigned acc_a = __reduce_add_sync(0xffffffffu, acc.accepted);
    const unsigned acc_b = __reduce_add_sync(0xffffffffu, acc.band);
    const int fb = __reduce_add_sync(0xffffffffu, acc.fallbacks);
    const unsigned upd = __reduce_add_sync(0xffffffffu, acc.updates);
    if (lane == 0) {
        atomicAdd(&C->r_accepted, static_cast<unsigned long long>(acc_a));
        atomicAdd(&C->r_band, static_cast<unsigned long long>(acc_b));
        atomicAdd(&C->r_solves, static_cast<unsigned long long>(acc.solves));
        atomicAdd(&C->r_updates, static_cast<unsigned long long>(upd));
        atomicAdd(&C->r_rounds, static_cast<unsigned long long>(acc.rounds));
        atomicMin(&C->r_rmin_bits, __float_as_uint(acc.rmin));
        atomicMax(&C->r_rmax_bits, __float_as_uint(acc.rmax));
        if (fb) atomicAdd(&C->r_fallbacks, static_cast<unsigned long long>(fb));
    }
    acc = MarchAcc{0u, 0u, 0, 0u, 0u, 0u, __int_as_float(0x7f800000), 0.0f};
}

// Per-warp state of the restart loop, in shared memory (lane 0 writes it):
// the march needs every register it can get.
struct LoopState {
    double bound, bprev, next_bound;
    float bound_f, bprev_f, next_f;    // the same rounded down to single precision
    int grow, grow_next;       // bound, next_bound below width_band (pending nodes re-activate the block)
    int n;                     // length of this restart's brick list
    int early;                 // early work allowed while waiting at this restart's barrier
    int waiting;               // arrived at the barrier
    unsigned gen;              // barrier generation to wait past
    int polls;
    unsigned nap;
    int claim;                 // entry of the next restart's list claimed while waiting (-1: none)
};

// Grid barrier at the end of a restart, one warp at a time: every warp of the
// launch arrives on its own (lane 0's atomic), and the warp arriving last does
// the restart bookkeeping and then releases the others by bumping bar_gen.
// barrier_arrive returns true for that last warp; *gen gets the generation the
// others wait to see change.
__device__ __forceinline__ bool barrier_arrive(Ctrl* C, int lane, unsigned* gen) {
    unsigned g = 0;
    int last = 0;
    if (lane == 0) {
        g = ld_acquire(&C->bar_gen);
        __threadfence();
        last = atomicAdd(&C->bar_count, 1u) == gridDim.x * (blockDim.x >> 5) - 1;
        if (last) __threadfence();
    }
    *gen = __shfl_sync(0xffffffffu, g, 0);
    return __shfl_sync(0xffffffffu, last, 0) != 0;
}
__device__ __forceinline__ void barrier_release(Ctrl* C, int lane, unsigned gen) {
    __syncwarp();
    if (lane == 0) {
        C->bar_count = 0;
        __threadfence();
        st_release(&C->bar_gen, gen + 1);
    }
}
// 1: released; 2: a wait somewhere ran out (kStWaitTimeout); 0: keep waiting.
__device__ __forceinline__ int barrier_poll(Ctrl* C, int lane, unsigned gen) {
    int state = 0;
    if (lane == 0) {
        if (ld_acquire(&C->bar_gen) != gen) state = 1;
        else if (__ldcg(&C->status) & kStWaitTimeout) state = 2;
    }
    return __shfl_sync(0xffffffffu, state, 0);
}

// A warp that gives up on a wait: the status bit, made visible to every other
// warp of the launch before the warp leaves.
__device__ __forceinline__ void give_up(Ctrl* C, int lane) {
    if (lane == 0) {
        atomicOr(&C->status, kStWaitTimeout);
        __threadfence();
    }
    __syncwarp();
}

// Start of CTA-wide work (16^3 blocks) in a restart: whether the whole CTA may
// go on.  A warp that gives up on a wait (give_up) exits on its own, and an
// exiting thread releases a CTA barrier that waits only for it (the exit rule
// of PTX), so this vote completes whichever warps are still there.  Every
// thread of the CTA gets the same answer: false if a warp is missing, if a
// warp of the CTA brings ok = false, or if any wait of the launch has run out.
// The CTA then leaves as a whole, before its first CTA-wide march, and no
// thread is ever left waiting at a CTA barrier for a warp that has gone.
// s_arrived is a shared counter that starts at zero (and is zero again after).
__device__ __forceinline__ bool cta_go(const Ctrl* C, bool ok, int lane, int* s_arrived) {
    if (lane == 0) atomicAdd(s_arrived, 1);
    const int stop = __syncthreads_or((!ok || (__ldcg(&C->status) & kStWaitTimeout)) ? 1 : 0);
    const bool all = *reinterpret_cast<volatile int*>(s_arrived) == static_cast<int>(blockDim.x >> 5);
    __syncthreads();
    if (threadIdx.x == 0) *s_arrived = 0;
    return stop == 0 && all;
}

// A grid barrier inside a restart (no bookkeeping): every warp of the launch
// arrives; false if this or another wait ran out (the status then says so).
__device__ inline bool grid_sync(Ctrl* C, int lane, long long limit) {
    unsigned gen;
    if (barrier_arrive(C, lane, &gen)) {
        barrier_release(C, lane, gen);
        return true;
    }
    unsigned nap = 32;
    for (long long it = 0;; ++it) {
        const int st = barrier_poll(C, lane, gen);
        if (st == 1) return true;
        if (st == 2) return false;
        if (it > limit) {
            give_up(C, lane);
            return false;
        }
        __nanosleep(nap);
        if (nap < 1024) nap <<= 1;
    }
}

// While waiting at the barrier of restart k: the next entry of restart k+1's
// list (ring slot s1) for an early march, or -1.  A warp claims one index
// (atomicAdd on the slot's head) and keeps the claim until the list holds that
// entry; a claim still open at the release is settled by the claimer at the
// start of restart k+1 (settle_claim).
__device__ __forceinline__ int32_t early_entry(Ctrl* C, int32_t* list, int s1, int& claim, long long limit,
                                               int lane) {
    if (claim < 0) {
        if (lane == 0) claim = atomicAdd(&C->head[s1], 1);
        claim = __shfl_sync(0xffffffffu, claim, 0);
    }
    int have = 0;
    if (lane == 0) have = claim < __ldcg(&C->count[s1]);
    if (!__shfl_sync(0xffffffffu, have, 0)) return -1;
    const int32_t b = take_entry(list, claim, true, limit, lane);
    claim = -1;
    return b < 0 ? -2 : b;
}

}  // namespace eikg
