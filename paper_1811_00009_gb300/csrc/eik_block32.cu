// Blocks of 32^3 nodes, each marched by one CTA of 1024 threads (block_dim
// = 32; FP32).  The paper finds block edge 32 the best for parallel runs
// (Sec. 3.6): a larger block carries the front across more nodes within one
// restart, so fewer accepted values have to be refreshed when ghost layers
// change (Sec. 3.5).  A 32^3 tile with a one-node ghost layer (34^3 floats,
// 157 KB) fits one CTA's shared memory, and so do the bit masks of the march:
// one 32-bit word per x-row of the block (y + 32 z) holds the row's band
// (BAND of Sec. 2.1), the nodes accepted in a round, the nodes lowered in the
// march (Upsilon) and the nodes that are solved at all.  Thread t loads and
// writes back row t; in the rounds the rows are dealt out diagonally (see
// round_row) so that a front lying in a plane spreads over all warps.
//
// Data layout in HBM (one grid): blocks b = (bz*NBY + by)*NBX + bx of 32^3
// nodes, node p = (z*32 + y)*32 + x; the ragged last block of each axis is
// padded with barrier nodes.
//   rr[b][32768]          h/F (+inf: barrier or padding, -1: fixed source node)
//   copy[b][2][34816]     two copies of the block's psi: 32768 interior values,
//                         then the x = 0 and x = 31 layers (1024 each, index
//                         z*32 + y) stored contiguously for the neighbours
//   ups[b][2][6][32]      per copy and face, the face nodes lowered by the march
//                         that wrote it (Upsilon of Alg. 2/4): word c, bit a of
//                         face-local (a, c) = (y, z) for x faces, (x, z) for y
//                         faces, (x, y) for z faces
//   stamp[b], queued, lists as for the 8^3 bricks (eik_internal.cuh)
// A march at restart k reads its block's latest copy and the neighbours'
// copies as of the end of restart k-1 and writes the other copy, as the 8^3
// path does, so a march never reads what another march of its restart writes;
// an early march of restart k+1 starts only once its block and neighbours have
// finished restart k (their done marks), and then reads the same as after the
// barrier.
#include "eik_internal.cuh"
#include "eik_march.cuh"

#include <algorithm>
#include <cstdint>

namespace eikg {
namespace b32 {

constexpr int kE = 32;                 // block edge
constexpr int kN = kE * kE * kE;       // nodes per block
constexpr int kH = kE + 2;             // edge with the ghost layer
constexpr int kHN = kH * kH * kH;      // halo tile
constexpr int kCopy = kN + 2 * kE * kE;
constexpr int kX0 = kN, kX31 = kN + kE * kE;
constexpr int kT = 1024;               // threads per CTA: one per x-row
constexpr int kWL = 256;               // per warp: candidates of a solve pass

struct Params {
    int32_t NBX, NBY, NBZ;
    int32_t pad;
    int64_t nblk;
    float* copy;
    unsigned* ups;
    unsigned long long* stamp;
    const float* rr;
    int32_t* queued;                   // kRing x nblk
    int32_t* list[kRing];              // work lists by ring slot; entries not yet written are -1
    int32_t* done;                     // per block: last restart whose march of it finished (-1: none)
    Ctrl* ctrl;
    float window;                      // omega: acceptance window = omega * min(h/F) over the block
    float tau;                         // FP64 root fallback threshold
    double width;                      // width_band
    int64_t max_restarts;
    long long wait_limit;
};

struct __align__(16) Smem {
    float psi[kHN];                    // tile with ghost layer, index ((z+1)*34 + (y+1))*34 + (x+1)
    unsigned band[kT];                 // per row: band nodes
    unsigned acc[2][kT];               // per row: accepted in this round (by round parity)
    unsigned upd[kT];                  // per row: lowered in this march
    unsigned solv[kT];                 // per row: solved nodes
    unsigned gband[6][32];             // ghost faces: band nodes (face-local word c, bit a)
    unsigned gacc[2][6][32];           // ghost faces: accepted in this round
    unsigned mslot[3];                 // band minimum for round j (float bits) at [j % 3]
    unsigned wmin;                     // min h/F over the block's solved nodes (float bits)
    unsigned long long nst[8];         // stamps of the six neighbours and of the block itself
    unsigned short wl[32][kWL];        // per warp: candidates of a solve pass (node index)
    int facemask;
};

__device__ __forceinline__ int hx(int x, int y, int z) { return ((z + 1) * kH + (y + 1)) * kH + (x + 1); }

// Halo index of the ghost node of face f at face-local (a, c).
__device__ __forceinline__ int ghost_h(int f, int a, int c) {
    if (f == 0) return hx(-1, a, c);
    if (f == 1) return hx(kE, a, c);
    if (f == 2) return hx(a, -1, c);
    if (f == 3) return hx(a, kE, c);
    if (f == 4) return hx(a, c, -1);
    return hx(a, c, kE);
}

// Offset, in the copy of the neighbour across face f, of the node that face f's ghost (a, c) mirrors.
__device__ __forceinline__ int nbr_off(int f, int a, int c) {
    if (f == 0) return kX31 + c * kE + a;           // x = 31 layer of the -x neighbour (index z*32 + y)
    if (f == 1) return kX0 + c * kE + a;            // x = 0 layer of the +x neighbour
    if (f == 2) return (c * kE + 31) * kE + a;      // (x = a, y = 31, z = c)
    if (f == 3) return (c * kE + 0) * kE + a;       // (x = a, y = 0, z = c)
    if (f == 4) return (31 * kE + c) * kE + a;      // (x = a, y = c, z = 31)
    return c * kE + a;                              // (x = a, y = c, z = 0)
}

__device__ __forceinline__ void enqueue(const Params& P, int k, int32_t x) {
    const int s = (k + 1) % kRing;
    if (atomicMax(P.queued + static_cast<int64_t>(s) * P.nblk + x, k + 1) < k + 1) {
        const int pos = atomicAdd(&P.ctrl->count[s], 1);
        P.list[s][pos] = x;
    }
}

// Row of the rounds' thread mapping: lane l of warp w holds the x-row (y, z) =
// ((w + l) mod 32, l).  Every plane of constant y or constant z then spreads
// over all 32 warps (one row each), so a front lying in such a plane gives
// every warp the same share of a round's work.
__device__ __forceinline__ int round_row(int warp, int lane) { return lane * kE + ((warp + lane) & 31); }

// Alg. 3 for one candidate node (index idx = row*32 + x) of the tile: per axis
// the smaller KNOWN neighbour below the node's value (BAND values carry their
// sign bit and order above every KNOWN bit pattern, as in the 8^3 march), then
// the upwind root; a lower value makes the node BAND again.
__device__ __forceinline__ void solve_node(const Params& P, Smem& S, int32_t blk, int idx, float tau, int& fb,
                                           float& smin, unsigned& nupd) {
    const float INF = __int_as_float(0x7f800000);
    const int x = idx & 31, row = idx >> 5;
    const int hq = ((row >> 5) + 1) * kH * kH + ((row & 31) + 1) * kH + x + 1;
    const float r = __ldg(P.rr + static_cast<int64_t>(blk) * kN + idx);
    const float c = fabsf(S.psi[hq]);
    const unsigned cb = __float_as_uint(c);
    auto axis = [&](float p, float q) -> float {
        const unsigned up = __float_as_uint(p), uq = __float_as_uint(q);
        const unsigned mm = up < uq ? up : uq;
        return mm < cb ? __uint_as_float(mm) : INF;
    };
    const float mx = axis(S.psi[hq - 1], S.psi[hq + 1]);
    const float my = axis(S.psi[hq - kH], S.psi[hq + kH]);
    const float mz = axis(S.psi[hq - kH * kH], S.psi[hq + kH * kH]);
    const float lo = fminf(mx, my), hi = fmaxf(mx, my);
    const float a0 = fminf(lo, mz), t1 = fmaxf(lo, mz);
    const float a1 = fminf(hi, t1), a2 = fmaxf(hi, t1);
    if (a0 < INF) {
        const float xn = upwind_root_f32(a0, a1, a2, r, tau, fb);
        if (xn < c) {
            S.psi[hq] = -xn;                              // tentative again: BAND
            atomicOr(&S.upd[row], 1u << x);
            atomicOr(&S.band[row], 1u << x);
            smin = fminf(smin, xn);
            ++nupd;
        }
    }
}

// March_Narrow_Band (Alg. 4 with Algs. 2 and 3) of block blk at restart k, the
// exchange of Alg. 5 for its ghost layer done first from the neighbours'
// copies as of the end of restart k-1.  Rounds of windowed ordered acceptance
// as in the 8^3 march: accept every band node within w of the band minimum
// (and not above the bound), then re-solve their neighbours.  A round has two
// CTA barriers: after the acceptance (the accepted rows are read by the
// neighbouring rows' threads) and after the solves (the next round reads the
// lowered values and the band minimum, kept by an atomic minimum in shared
// memory).  Each warp enumerates its words of band nodes and candidates either
// bit by bit in each lane or row by row across its lanes, whichever takes
// fewer steps, and solves its own candidates from a list of its own.
__device__ void march32(const Params& P, Smem& S, int32_t blk, int k, float bprev, float bound, bool grow) {
    const float INF = __int_as_float(0x7f800000);
    const unsigned INFB = 0x7f800000u;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int bx = static_cast<int>(blk % P.NBX), by = static_cast<int>((blk / P.NBX) % P.NBY);
    const int bz = static_cast<int>(blk / (static_cast<int64_t>(P.NBX) * P.NBY));
    const int32_t plane = P.NBX * P.NBY;
    int32_t nbr[6];
    nbr[0] = bx > 0 ? blk - 1 : -1;
    nbr[1] = bx < P.NBX - 1 ? blk + 1 : -1;
    nbr[2] = by > 0 ? blk - P.NBX : -1;
    nbr[3] = by < P.NBY - 1 ? blk + P.NBX : -1;
    nbr[4] = bz > 0 ? blk - plane : -1;
    nbr[5] = bz < P.NBZ - 1 ? blk + plane : -1;

    // ---- load (thread t holds row t: y = lane, z = warp): the stamps, then the
    // block's latest copy and h/F of the row
    if (t < 7) S.nst[t] = (t == 6) ? __ldcg(P.stamp + blk) : (nbr[t] >= 0 ? __ldcg(P.stamp + nbr[t]) : kUntouched);
    if (t == 0) {
        S.mslot[0] = S.mslot[1] = S.mslot[2] = INFB;
        S.wmin = INFB;
        S.facemask = 0;
    }
    __syncthreads();
    const unsigned long long st = S.nst[6];
    float mn0 = INF, rlo = INF;
    {
        const int y = lane, z = warp, rb = hx(0, y, z);
        const float* rs = P.rr + static_cast<int64_t>(blk) * kN + (z * kE + y) * kE;
        const float* ps = (st == kUntouched) ? nullptr
                                              : P.copy + (static_cast<int64_t>(blk) * 2 + stamp_copy(st)) * kCopy +
                                                    (z * kE + y) * kE;
        float row[32];
        unsigned B = 0u, SV = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 rv = __ldg(reinterpret_cast<const float4*>(rs) + q);
            const float rq[4] = {rv.x, rv.y, rv.z, rv.w};
            float4 pv = make_float4(INF, INF, INF, INF);
            if (ps) pv = __ldcg(reinterpret_cast<const float4*>(ps) + q);
            const float pq[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int x = 4 * q + e;
                const float r = rq[e], v = pq[e];
                if (r > 0.0f && r < INF) {
                    SV |= 1u << x;
                    rlo = fminf(rlo, r);
                }
                const bool b = v < INF && v > bprev;
                if (b) {
                    B |= 1u << x;
                    mn0 = fminf(mn0, v);
                }
                row[x] = b ? -v : v;
            }
        }
#pragma unroll
        for (int x = 0; x < 32; ++x) S.psi[rb + x] = row[x];
        S.band[t] = B;
        S.solv[t] = SV;
        S.upd[t] = 0u;
    }
    // ---- the ghost layer (Alg. 5): the neighbours' boundary layers as of the end
    // of restart k-1, with their Upsilon masks; thread t loads face-local (a, c) =
    // (lane, warp) of every face.  A ghost node is band when it lies above the
    // previous bound or the neighbour lowered it in restart k-1.
    {
        const int a = lane, c = warp;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            float g = INF;
            unsigned um = 0u;
            if (nbr[f] >= 0) {
                const unsigned long long w = S.nst[f];
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
                if (sl >= 0) {
                    const int64_t cb = static_cast<int64_t>(nbr[f]) * 2 + sl;
                    g = __ldcg(P.copy + cb * kCopy + nbr_off(f, a, c));
                    if (written == k - 1) um = __ldcg(P.ups + (cb * 6 + (f ^ 1)) * 32 + c);
                }
            }
            const bool gb = g < INF && (((um >> a) & 1u) || g > bprev);
            S.psi[ghost_h(f, a, c)] = gb ? -g : g;
            const unsigned gw = __ballot_sync(kFull, gb);
            if (lane == 0) S.gband[f][c] = gw;
            if (gb) mn0 = fminf(mn0, g);
        }
    }
    mn0 = warp_min_nn(mn0);
    rlo = warp_min_nn(rlo);
    if (lane == 0) {
        if (mn0 < INF) atomicMin(&S.mslot[0], __float_as_uint(mn0));
        if (rlo < INF) atomicMin(&S.wmin, __float_as_uint(rlo));
    }
    __syncthreads();
    const float w = P.window * __uint_as_float(S.wmin);
    const float tau = P.tau;

    // ---- rounds (Alg. 4), thread mapping of round_row; lanes 0..5 of warp w also
    // hold the ghost row c = w of face f = lane
    const int r = round_row(warp, lane);
    const int ry = r & 31, rz = r >> 5;
    const unsigned sv = S.solv[r];
    const bool gowner = lane < 6;
    unsigned gbw = gowner ? S.gband[lane][warp] : 0u;
    unsigned short* wl = S.wl[warp];
    const unsigned lt = (1u << lane) - 1u;
    int rounds = 0, par = 0, fb = 0;
    unsigned nacc = 0u, nsolve = 0u, nupd = 0u;
    for (int j = 0;; ++j) {
        const float mn = __uint_as_float(S.mslot[j % 3]);
        if (!(mn < INF) || !(mn <= bound)) break;          // band empty, or its minimum above the bound
        if (++rounds > kRoundCap) {
            if (t == 0) atomicOr(&P.ctrl->status, kStRoundCap);
            break;
        }
        if (t == 0) S.mslot[(j + 2) % 3] = INFB;         // last read at the start of round j - 1
        const float thr = fminf(mn + w, bound);
        float kmin = INF;
        // accept (Remove_Min of a window) of this warp's rows
        const unsigned bw = S.band[r];
        unsigned aw = 0u;
        {
            const unsigned nzl = __ballot_sync(kFull, bw != 0u);
            const int most = __reduce_max_sync(kFull, static_cast<unsigned>(__popc(bw)));
            if (__popc(nzl) < most) {
                for (unsigned q = nzl; q; q &= q - 1) {
                    const int L = __ffs(q) - 1;
                    const unsigned wL = __shfl_sync(kFull, bw, L);
                    bool ac = false;
                    if ((wL >> lane) & 1u) {
                        const int h = hx(lane, (warp + L) & 31, L);
                        const float v = fabsf(S.psi[h]);
                        if (!(thr < v)) {
                            S.psi[h] = v;
                            ac = true;
                        } else {
                            kmin = fminf(kmin, v);
                        }
                    }
                    const unsigned a = __ballot_sync(kFull, ac);
                    if (lane == L) aw = a;
                }
            } else {
                const int hb = hx(0, ry, rz);
                for (unsigned m = bw; m; m &= m - 1) {
                    const int x = __ffs(m) - 1;
                    const float v = fabsf(S.psi[hb + x]);
                    if (!(thr < v)) {
                        S.psi[hb + x] = v;
                        aw |= 1u << x;
                    } else {
                        kmin = fminf(kmin, v);
                    }
                }
            }
        }
        S.band[r] = bw & ~aw;
        S.acc[par][r] = aw;
        nacc += __popc(aw);
        // the ghost rows, row by row across the lanes
        {
            unsigned ga = 0u;
            for (unsigned q = __ballot_sync(kFull, gbw != 0u); q; q &= q - 1) {
                const int L = __ffs(q) - 1;
                const unsigned wL = __shfl_sync(kFull, gbw, L);
                bool ac = false;
                if ((wL >> lane) & 1u) {
                    const int h = ghost_h(L, lane, warp);
                    const float v = fabsf(S.psi[h]);
                    if (!(thr < v)) {
                        S.psi[h] = v;
                        ac = true;
                    } else {
                        kmin = fminf(kmin, v);
                    }
                }
                const unsigned a = __ballot_sync(kFull, ac);
                if (lane == L) ga = a;
            }
            if (gowner) {
                gbw &= ~ga;
                S.gacc[par][lane][warp] = ga;
                nacc += __popc(ga);
            }
        }
        __syncthreads();
        // neighbours of the accepted nodes (Alg. 2) in this row: x +- 1 by shifts,
        // the rows at y +- 1 and z +- 1, and the ghost faces at the block's edges
        unsigned Cw = (aw << 1) | (aw >> 1);
        Cw |= (ry > 0) ? S.acc[par][r - 1] : S.gacc[par][2][rz];
        Cw |= (ry < 31) ? S.acc[par][r + 1] : S.gacc[par][3][rz];
        Cw |= (rz > 0) ? S.acc[par][r - 32] : S.gacc[par][4][ry];
        Cw |= (rz < 31) ? S.acc[par][r + 32] : S.gacc[par][5][ry];
        Cw |= (S.gacc[par][0][rz] >> ry) & 1u;
        Cw |= ((S.gacc[par][1][rz] >> ry) & 1u) << 31;
        Cw &= sv;
        // this warp's candidates -> its list (position = exclusive prefix over the
        // lanes, then bit order), solved kWL at a time by the warp's lanes
        float smin = INF;
        {
            const int cnt = __popc(Cw);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(kFull, incl, 31);
            const int base = incl - cnt;
            if (lane == 0) nsolve += static_cast<unsigned>(total);
            if (total > 0) {
                const unsigned nzl = __ballot_sync(kFull, Cw != 0u);
                const bool by_rows = __popc(nzl) < static_cast<int>(__reduce_max_sync(kFull, static_cast<unsigned>(cnt)));
                for (int done = 0; done < total; done += kWL) {
                    const int lim = done + kWL;
                    if (by_rows) {
                        for (unsigned q = nzl; q; q &= q - 1) {
                            const int L = __ffs(q) - 1;
                            const unsigned wL = __shfl_sync(kFull, Cw, L);
                            const int bL = __shfl_sync(kFull, base, L);
                            if ((wL >> lane) & 1u) {
                                const int pos = bL + __popc(wL & lt);
                                if (pos >= done && pos < lim)
                                    wl[pos - done] = static_cast<unsigned short>(round_row(warp, L) * 32 + lane);
                            }
                        }
                    } else {
                        int pos = base;
                        for (unsigned m = Cw; m; m &= m - 1, ++pos)
                            if (pos >= done && pos < lim)
                                wl[pos - done] = static_cast<unsigned short>(r * 32 + __ffs(m) - 1);
                    }
                    __syncwarp();
                    const int n = min(kWL, total - done);
                    for (int i = lane; i < n; i += 32) solve_node(P, S, blk, wl[i], tau, fb, smin, nupd);
                    __syncwarp();
                }
            }
        }
        // the next band minimum: of the kept band and of the lowered values
        {
            const float v = warp_min_nn(fminf(kmin, smin));
            if (lane == 0 && v < INF) atomicMin(&S.mslot[(j + 1) % 3], __float_as_uint(v));
        }
        __syncthreads();
        par ^= 1;
    }
    if (gowner) S.gband[lane][warp] = gbw;

    // ---- statistics of the march
    {
        const unsigned a_ = __reduce_add_sync(kFull, nacc), u_ = __reduce_add_sync(kFull, nupd);
        const unsigned s_ = __reduce_add_sync(kFull, nsolve);
        const int f_ = __reduce_add_sync(kFull, fb);
        if (lane == 0) {
            atomicAdd(&P.ctrl->r_accepted, static_cast<unsigned long long>(a_));
            atomicAdd(&P.ctrl->r_updates, static_cast<unsigned long long>(u_));
            atomicAdd(&P.ctrl->r_solves, static_cast<unsigned long long>(s_));
            if (f_) atomicAdd(&P.ctrl->r_fallbacks, static_cast<unsigned long long>(f_));
        }
        if (t == 0) atomicAdd(&P.ctrl->r_rounds, static_cast<unsigned long long>(rounds));
    }

    // ---- write the other copy when the march lowered a value (thread t: row t),
    // with the Upsilon masks of its faces; list the neighbours across faces with a
    // lowered node
    const int y = lane, z = warp, rb = hx(0, y, z);
    const unsigned U = S.upd[t];
    const bool lowered = __syncthreads_or(U != 0u) != 0;
    if (lowered) {
        const int ns = (st == kUntouched) ? 0 : (stamp_copy(st) ^ 1);
        const int64_t cb = static_cast<int64_t>(blk) * 2 + ns;
        float* dst = P.copy + cb * kCopy;
        float v[32];
#pragma unroll
        for (int x = 0; x < 32; ++x) v[x] = fabsf(S.psi[rb + x]);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            reinterpret_cast<float4*>(dst + (z * kE + y) * kE)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2],
                                                                               v[4 * q + 3]);
        dst[kX0 + z * kE + y] = v[0];
        dst[kX31 + z * kE + y] = v[31];
        unsigned* um = P.ups + cb * 6 * 32;
        const unsigned w0 = __ballot_sync(kFull, U & 1u), w1 = __ballot_sync(kFull, (U >> 31) & 1u);
        unsigned fm = 0u;
        if (lane == 0) {
            um[0 * 32 + z] = w0;
            um[1 * 32 + z] = w1;
            um[2 * 32 + z] = U;                                  // the y = 0 row of plane z
            fm |= (w0 ? 1u : 0u) | (w1 ? 2u : 0u) | (U ? 4u : 0u);
        }
        if (lane == 31) {
            um[3 * 32 + z] = U;                                  // the y = 31 row
            fm |= U ? 8u : 0u;
        }
        if (warp == 0) {
            um[4 * 32 + y] = U;                                  // plane z = 0, row y
            fm |= U ? 16u : 0u;
        }
        if (warp == 31) {
            um[5 * 32 + y] = U;
            fm |= U ? 32u : 0u;
        }
        if (fm) atomicOr(&S.facemask, static_cast<int>(fm));
        __syncthreads();
        // (no fence: nobody reads this copy before the grid barrier that ends the restart)
        if (t == 0)
            P.stamp[blk] = make_stamp(k, st == kUntouched ? static_cast<int>(kNever) : stamp_latest(st), ns);
    }
    // ---- activation for restart k+1 (A of Alg. 4/5, C of Alg. 4)
    const bool pending = __syncthreads_or(S.band[t] != 0u || (t < 192 && S.gband[t >> 5][t & 31] != 0u)) != 0;
    if (t == 0) {
        if (pending && grow) enqueue(P, k, blk);
        const int fm = S.facemask;
        for (int f = 0; f < 6; ++f)
            if (((fm >> f) & 1) && nbr[f] >= 0) enqueue(P, k, nbr[f]);
        // publish: the block's restart-k march has finished (read by early marches
        // of its neighbours; the CTA barriers above put every thread's writes before it)
        __threadfence();
        st_release(P.done + blk, k);
    }
}

// At the start of restart k every thread of the launch clears its share of the
// list restart k-1 used (ring slot (k-1) mod kRing) to -1.  That slot is next
// written by early marches of restart k+2, after the barrier of restart k.
__device__ __forceinline__ void clear_used32(const Params& P, int k) {
    const int sp = (k + kRing - 1) % kRing;
    const int m = __ldcg(&P.ctrl->used[sp]);
    int32_t* list = P.list[sp];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) list[i] = -1;
}

// Thread 0 of a CTA waiting at the barrier of restart k: claim an entry of
// restart k+1's list (only below its current length, so an entry is claimed
// only once it has been counted), wait until the enqueuer has written it, then
// until the block and each of its six neighbours that is on restart k's list
// have finished that march.  An early march then reads what it would read after
// the barrier.  Returns the block, -1 if there is nothing to claim, -2 if a
// wait ran out (bounded).
__device__ int32_t early_claim32(const Params& P, int k) {
    Ctrl* C = P.ctrl;
    const int s = k % kRing, s1 = (k + 1) % kRing;
    int h = __ldcg(&C->head[s1]);
    int i = -1;
    for (int tries = 0; tries < 64; ++tries) {
        if (h >= __ldcg(&C->count[s1])) return -1;
        const int prev = atomicCAS(&C->head[s1], h, h + 1);
        if (prev == h) {
            i = h;
            break;
        }
        h = prev;
    }
    if (i < 0) return -1;
    int32_t b = ld_acquire(P.list[s1] + i);
    for (long long it = 0; b < 0; ++it) {
        if (it > P.wait_limit) return -2;
        __nanosleep(32);
        b = ld_acquire(P.list[s1] + i);
    }
    const int bx = static_cast<int>(b % P.NBX), by = static_cast<int>((b / P.NBX) % P.NBY);
    const int bz = static_cast<int>(b / (static_cast<int64_t>(P.NBX) * P.NBY));
    const int32_t plane = P.NBX * P.NBY;
    const int32_t xs[7] = {b, bx > 0 ? b - 1 : -1, bx < P.NBX - 1 ? b + 1 : -1, by > 0 ? b - P.NBX : -1,
                           by < P.NBY - 1 ? b + P.NBX : -1, bz > 0 ? b - plane : -1, bz < P.NBZ - 1 ? b + plane : -1};
    for (int j = 0; j < 7; ++j) {
        const int32_t x = xs[j];
        if (x < 0 || __ldcg(P.queued + static_cast<int64_t>(s) * P.nblk + x) != k) continue;
        unsigned nap = 64;
        for (long long it = 0; ld_acquire(P.done + x) < k; ++it) {
            if (it > P.wait_limit) return -2;
            __nanosleep(nap);
            if (nap < 1024) nap <<= 1;
        }
    }
    return b;
}

// Bookkeeping at the end of restart k (thread 0 of the CTA that reaches the
// grid barrier last): statistics, the exit test and the next bound of Alg. 6.
__device__ void restart_end32(const Params& P) {
    Ctrl* C = P.ctrl;
    const int k = __ldcg(&C->k);
    const int s = k % kRing, s1 = (k + 1) % kRing;
    const int n_this = __ldcg(&C->count[s]), n_next = __ldcg(&C->count[s1]);
    const unsigned long long now = globaltimer();
    C->marches += 64ull * static_cast<unsigned long long>(n_this);     // in 8^3-brick equivalents
    C->accepted += __ldcg(&C->r_accepted);
    C->solves += __ldcg(&C->r_solves);
    C->updates += __ldcg(&C->r_updates);
    C->fallbacks += __ldcg(&C->r_fallbacks);
    C->rounds += __ldcg(&C->r_rounds);
    C->r_accepted = C->r_solves = C->r_updates = C->r_fallbacks = C->r_rounds = 0;
    C->used[s] = n_this;
    C->count[s] = 0;
    C->head[s] = 0;
    if (n_next == 0 || (__ldcg(&C->status) & kStWaitTimeout)) {
        C->done = 1;
        C->t_end = now;
    } else if (k >= P.max_restarts) {
        C->done = 1;
        C->status |= kStRestartCap;
        C->t_end = now;
    } else {
        const double bnd = __ldcg(&C->bound);
        C->k = k + 1;
        C->bound_prev = bnd;
        C->bound = fmin(bnd + __ldcg(&C->stride), P.width);    // bound_band <- min(bound_band + stride, width_band)
        C->t_restart = now;
    }
}

// The restart loop of Alg. 6 for 32^3 blocks: one persistent cooperative
// launch, one CTA of 1024 threads per SM; each restart every CTA takes blocks
// from the work list and marches them; one grid barrier (one arrival per CTA)
// ends the restart, and a CTA waiting there marches blocks of restart k+1 whose
// neighbourhood has finished restart k (the stride is fixed, so the next bound
// is known).  Every wait is bounded and CTA-uniform: thread 0 polls, writes the
// outcome to shared memory, and the whole CTA acts on it after a barrier.
__global__ void __launch_bounds__(kT, 1) k_loop32(Params P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    __shared__ int s_blk, s_state;
    Ctrl* C = P.ctrl;
    const int t = threadIdx.x;
    if (blockIdx.x == 0 && t == 0) {
        const unsigned long long t0 = globaltimer();
        C->t_begin = t0;
        C->t_restart = t0;
    }
    for (;;) {
        const int k = __ldcg(&C->k);
        const int s = k % kRing;
        const double bd = __ldcg(&C->bound), bp = __ldcg(&C->bound_prev);
        const double bn = fmin(bd + __ldcg(&C->stride), P.width);      // restart k+1's bound
        const float bound = __double2float_rd(bd), bprev = __double2float_rd(bp), bnext = __double2float_rd(bn);
        const bool grow = bd < P.width, grow_next = bn < P.width;
        clear_used32(P, k);
        // restart k's list
        for (;;) {
            if (t == 0) {
                const int i = atomicAdd(&C->head[s], 1);
                s_blk = (i < __ldcg(&C->count[s])) ? __ldcg(P.list[s] + i) : -1;
            }
            __syncthreads();
            const int32_t blk = s_blk;
            if (blk < 0) break;
            march32(P, S, blk, k, bprev, bound, grow);
            __syncthreads();
        }
        // the grid barrier; state 0: waiting, 1: released, 2: leave the loop
        unsigned gen = 0;
        long long polls = 0;
        unsigned nap = 32;
        if (t == 0) {
            gen = ld_acquire(&C->bar_gen);
            __threadfence();
            int state = 0;
            if (atomicAdd(&C->bar_count, 1u) == gridDim.x - 1) {
                __threadfence();
                restart_end32(P);
                C->bar_count = 0;
                __threadfence();
                st_release(&C->bar_gen, gen + 1);
                state = __ldcg(&C->done) ? 2 : 1;
            }
            s_state = state;
            s_blk = -1;
        }
        __syncthreads();
        int state = s_state;
        __syncthreads();          // every thread has read s_state before thread 0 writes it again
        while (state == 0) {
            if (t == 0) {
                int st = 0;
                int32_t b = -1;
                if (ld_acquire(&C->bar_gen) != gen) {
                    st = __ldcg(&C->done) ? 2 : 1;
                } else if (__ldcg(&C->status) & kStWaitTimeout) {
                    st = 2;
                } else if (++polls > P.wait_limit) {
                    atomicOr(&C->status, kStWaitTimeout);
                    __threadfence();
                    st = 2;
                } else {
                    b = early_claim32(P, k);
                    if (b == -2) {
                        atomicOr(&C->status, kStWaitTimeout);
                        __threadfence();
                        st = 2;
                        b = -1;
                    } else if (b >= 0) {
                        polls = 0;
                        nap = 32;
                    } else {
                        __nanosleep(nap);
                        if (nap < 2048) nap <<= 1;
                    }
                }
                s_state = st;
                s_blk = b;
            }
            __syncthreads();
            state = s_state;
            const int32_t blk = s_blk;
            __syncthreads();      // read before thread 0 writes again
            if (state == 0 && blk >= 0) march32(P, S, blk, k + 1, bound, bnext, grow_next);
        }
        if (state == 2) return;
    }
}

// h/F in 8^3 bricks -> h/F in 32^3 blocks (+inf beyond the brick grid).
__global__ void k_rr_to_32(const float* __restrict__ rr8, int BX, int BY, int BZ, float* __restrict__ rr32, int NBX,
                           int NBY, int64_t nblk) {
    const int64_t total = nblk * kN;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = q / kN;
        const int p = static_cast<int>(q - b * kN);
        const int x = p & 31, y = (p >> 5) & 31, z = p >> 10;
        const int bxx = static_cast<int>(b % NBX), byy = static_cast<int>((b / NBX) % NBY);
        const int bzz = static_cast<int>(b / (static_cast<int64_t>(NBX) * NBY));
        const int i = bxx * 32 + x, j = byy * 32 + y, k = bzz * 32 + z;
        float v = __int_as_float(0x7f800000);
        if (i < 8 * BX && j < 8 * BY && k < 8 * BZ) {
            const int64_t b8 = (static_cast<int64_t>(k >> 3) * BY + (j >> 3)) * BX + (i >> 3);
            v = rr8[b8 * kBrick + ((k & 7) * 8 + (j & 7)) * 8 + (i & 7)];
        }
        rr32[q] = v;
    }
}

// Alg. 1 for the blocks holding fixed nodes (copy 0: +inf but at the fixed
// nodes, no Upsilon, stamp of "restart 0"), h/F of the fixed nodes -> -1, and
// the work list of restart 1.
__global__ void k_init32(int nfix, const int32_t* __restrict__ fb, const int32_t* __restrict__ fp,
                         const double* __restrict__ fv, int nsb, const int32_t* __restrict__ sb, int nenq,
                         const int32_t* __restrict__ enq, float* copy, unsigned* ups, unsigned long long* stamp,
                         int32_t* queued1, float* rr, float* saved, int32_t* list1) {
    const float INF = __int_as_float(0x7f800000);
    if (blockIdx.x < nsb) {
        const int32_t b = sb[blockIdx.x];
        float* dst = copy + static_cast<int64_t>(b) * 2 * kCopy;
        for (int q = threadIdx.x; q < kCopy; q += blockDim.x) dst[q] = INF;
        __syncthreads();
        for (int q = threadIdx.x; q < nfix; q += blockDim.x) {
            if (fb[q] != b) continue;
            const int p = fp[q];
            const float v = static_cast<float>(fv[q]);
            dst[p] = v;
            const int x = p & 31, y = (p >> 5) & 31, z = p >> 10;
            if (x == 0) dst[kX0 + z * 32 + y] = v;
            if (x == 31) dst[kX31 + z * 32 + y] = v;
        }
        for (int q = threadIdx.x; q < 6 * 32; q += blockDim.x) ups[static_cast<int64_t>(b) * 2 * 6 * 32 + q] = 0u;
        if (threadIdx.x == 0) stamp[b] = make_stamp(0, static_cast<int>(kNever), 0);
    } else {
        const int q = (blockIdx.x - nsb) * blockDim.x + threadIdx.x;
        if (q < nfix) {
            const int64_t g = static_cast<int64_t>(fb[q]) * kN + fp[q];
            saved[q] = rr[g];
            rr[g] = -1.0f;
        }
        if (q < nenq) {
            list1[q] = enq[q];
            queued1[enq[q]] = 1;
        }
    }
}

__global__ void k_restore32(int nfix, const int32_t* __restrict__ fb, const int32_t* __restrict__ fp,
                            const float* __restrict__ saved, float* rr) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nfix) rr[static_cast<int64_t>(fb[q]) * kN + fp[q]] = saved[q];
}

// Latest copy of every block -> psi in x-fastest order.
__global__ void k_result32(const float* __restrict__ copy, const unsigned long long* __restrict__ stamp,
                           float* __restrict__ out, int nx, int ny, int nz, int NBX, int NBY) {
    const int rows = ny * nz;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int k = r / ny, j = r - k * ny;
        const int64_t brow = (static_cast<int64_t>(k >> 5) * NBY + (j >> 5)) * NBX;
        const int prow = ((k & 31) * 32 + (j & 31)) * 32;
        float* o = out + static_cast<int64_t>(r) * nx;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int64_t b = brow + (i >> 5);
            const unsigned long long st = __ldg(stamp + b);
            o[i] = (st == kUntouched) ? __int_as_float(0x7f800000)
                                      : __ldcs(copy + (b * 2 + stamp_copy(st)) * kCopy + prow + (i & 31));
        }
    }
}

}  // namespace b32

// ---------------------------------------------------------------------------
// Host side (called from eik_runtime.cu)
// ---------------------------------------------------------------------------
int block32_edge_values() { return b32::kCopy; }

cudaError_t block32_occupancy(int* per_sm) {
    cudaError_t e = cudaFuncSetAttribute(b32::k_loop32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sizeof(b32::Smem)));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, b32::k_loop32, b32::kT, sizeof(b32::Smem));
}

cudaError_t block32_layout(const float* rr8, int BX, int BY, int BZ, float* rr32, int NBX, int NBY, int64_t nblk,
                           cudaStream_t s) {
    b32::k_rr_to_32<<<4 * 152 * 4, 256, 0, s>>>(rr8, BX, BY, BZ, rr32, NBX, NBY, nblk);
    return cudaGetLastError();
}

cudaError_t block32_init(int nfix, const int32_t* fb, const int32_t* fp, const double* fv, int nsb, const int32_t* sb,
                         int nenq, const int32_t* enq, float* copy, unsigned* ups, unsigned long long* stamp,
                         int32_t* queued1, float* rr, float* saved, int32_t* list1, cudaStream_t s) {
    const int m = std::max(nfix, nenq);
    const int grid = nsb + (m + 255) / 256;
    if (grid == 0) return cudaSuccess;
    b32::k_init32<<<grid, 256, 0, s>>>(nfix, fb, fp, fv, nsb, sb, nenq, enq, copy, ups, stamp, queued1, rr, saved,
                                       list1);
    return cudaGetLastError();
}

cudaError_t block32_restore(int nfix, const int32_t* fb, const int32_t* fp, const float* saved, float* rr,
                            cudaStream_t s) {
    if (nfix <= 0) return cudaSuccess;
    b32::k_restore32<<<(nfix + 255) / 256, 256, 0, s>>>(nfix, fb, fp, saved, rr);
    return cudaGetLastError();
}

cudaError_t block32_result(const float* copy, const unsigned long long* stamp, float* out, int nx, int ny, int nz,
                           int NBX, int NBY, cudaStream_t s) {
    const int64_t rows = static_cast<int64_t>(ny) * nz;
    int grid = static_cast<int>(rows < 65535 * 4 ? rows : 65535 * 4);
    if (grid < 1) grid = 1;
    b32::k_result32<<<grid, 256, 0, s>>>(copy, stamp, out, nx, ny, nz, NBX, NBY);
    return cudaGetLastError();
}

cudaError_t block32_loop(int NBX, int NBY, int NBZ, int64_t nblk, float* copy, unsigned* ups,
                         unsigned long long* stamp, const float* rr, int32_t* queued, int32_t* lists, int32_t* done,
                         Ctrl* ctrl, float window, float tau, double width, int64_t max_restarts,
                         long long wait_limit, int grid, cudaStream_t s) {
    b32::Params P{};
    P.NBX = NBX;
    P.NBY = NBY;
    P.NBZ = NBZ;
    P.nblk = nblk;
    P.copy = copy;
    P.ups = ups;
    P.stamp = stamp;
    P.rr = rr;
    P.queued = queued;
    for (int r = 0; r < kRing; ++r) P.list[r] = lists + static_cast<int64_t>(r) * nblk;
    P.done = done;
    P.ctrl = ctrl;
    P.window = window;
    P.tau = tau;
    P.width = width;
    P.max_restarts = max_restarts;
    P.wait_limit = wait_limit;
    void* args[] = {&P};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(b32::k_loop32), dim3(grid), dim3(b32::kT), args,
                                       sizeof(b32::Smem), s);
}

}  // namespace eikg
