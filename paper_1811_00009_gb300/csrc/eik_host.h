// Host-side set-up shared by the one-grid runtime (eik_runtime.cu) and the
// batched runtime (eik_batch.cu): the fixed nodes of point sources (Alg. 1)
// and the blocks active at the first restart.
#pragma once

#include "eik.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

namespace eikh {

// Nodes of the cell containing coordinate s along one axis (Alg. 1, "on or
// adjacent to Gamma"): one node when s is within 1e-9 cells of a node.
inline int cell_nodes(double s, double h, int n, int out[2]) {
    const double t = s / h;
    const double tn = std::floor(t + 0.5);
    if (std::fabs(t - tn) <= 1e-9) {
        out[0] = std::min(std::max(static_cast<int>(tn), 0), n - 1);
        return 1;
    }
    const int i0 = std::min(std::max(static_cast<int>(std::floor(t)), 0), std::max(n - 2, 0));
    out[0] = i0;
    out[1] = std::min(i0 + 1, n - 1);
    return (out[1] == out[0]) ? 1 : 2;
}

// Brick geometry of one grid inside a launch's brick index space.
struct Bricks {
    int BX, BY, BZ;
    int32_t boff;
};

// A node next to a source: global brick, node in brick, distance to the source.
struct Cand {
    int32_t b, p;
    double dist;
};

// Every node of every cell that contains a source (xyz: n*3 coordinates), into
// out[0 .. 8*nsrc); returns the count.  (Fixed-size arrays: the allocation-free
// entry point uses these forms directly.)  A part of a grid sharded in z holds
// node planes [zoff, zoff + nz_part) of a grid of nz planes: the sources and
// the distances stay in the whole grid's coordinates (so every part computes
// the same psi0 as one grid would), and nodes outside the part are dropped.
inline int source_candidates_into(const double* xyz, int nsrc, int nx, int ny, int nz, double h, const Bricks& g,
                                  Cand* out, int zoff = 0, int nz_part = -1) {
    if (nz_part < 0) nz_part = nz;
    int n = 0;
    for (int q = 0; q < nsrc; ++q) {
        const double* xs = xyz + 3 * q;
        int ci[3][2], cn[3];
        cn[0] = cell_nodes(xs[0], h, nx, ci[0]);
        cn[1] = cell_nodes(xs[1], h, ny, ci[1]);
        cn[2] = cell_nodes(xs[2], h, nz, ci[2]);
        for (int a = 0; a < cn[2]; ++a)
            for (int bq = 0; bq < cn[1]; ++bq)
                for (int d = 0; d < cn[0]; ++d) {
                    const int i = ci[0][d], j = ci[1][bq], k = ci[2][a];
                    const int kl = k - zoff;
                    if (kl < 0 || kl >= nz_part) continue;
                    const double dx = i * h - xs[0], dy = j * h - xs[1], dz = k * h - xs[2];
                    Cand c;
                    c.b = g.boff + ((kl >> 3) * g.BY + (j >> 3)) * g.BX + (i >> 3);
                    c.p = ((kl & 7) * 8 + (j & 7)) * 8 + (i & 7);
                    c.dist = std::sqrt(dx * dx + dy * dy + dz * dz);
                    out[n++] = c;
                }
    }
    return n;
}

inline void source_candidates(const double* xyz, int nsrc, int nx, int ny, int nz, double h, const Bricks& g,
                              std::vector<Cand>& out, int zoff = 0, int nz_part = -1) {
    const size_t at = out.size();
    out.resize(at + 8 * static_cast<size_t>(nsrc > 0 ? nsrc : 0));
    const int n = source_candidates_into(xyz, nsrc, nx, ny, nz, h, g, out.data() + at, zoff, nz_part);
    out.resize(at + n);
}

struct FixNode {
    int32_t b, p;
    double v;
};

// Fixed nodes from the nc candidates and their h/F (r): psi0 = distance / F; a
// node on a source gets 0; a barrier node (F = 0) is not fixed; a node next
// to several sources keeps the smallest psi0.  Sorted by (brick, node), into
// out (room for nc); returns the count.
inline int fixed_nodes_into(const Cand* cand, int nc, const double* r, double h, FixNode* out) {
    int m = 0;
    for (int t = 0; t < nc; ++t) {
        double v;
        if (cand[t].dist == 0.0) v = 0.0;
        else if (std::isfinite(r[t]) && r[t] > 0.0) v = cand[t].dist * r[t] / h;
        else continue;
        out[m++] = FixNode{cand[t].b, cand[t].p, v};
    }
    std::sort(out, out + m, [](const FixNode& a, const FixNode& b) {
        return a.b != b.b ? a.b < b.b : (a.p != b.p ? a.p < b.p : a.v < b.v);
    });
    int u = 0;
    for (int t = 0; t < m; ++t)
        if (u == 0 || out[u - 1].b != out[t].b || out[u - 1].p != out[t].p) out[u++] = out[t];
    return u;
}

inline std::vector<FixNode> fixed_nodes(const std::vector<Cand>& cand, const std::vector<double>& r, double h) {
    std::vector<FixNode> out(cand.size());
    out.resize(fixed_nodes_into(cand.data(), static_cast<int>(cand.size()), r.data(), h, out.data()));
    return out;
}

// Bricks holding fixed nodes (sb, room for nfix), and the work list of
// restart 1 (enq, room for 7*nfix): those bricks and the neighbours whose
// ghost layer holds a fixed node (Alg. 1 runs over Xi^ib).  Fixed nodes must
// all lie in grid g and be sorted by brick.  Both outputs sorted, unique.
inline void first_active_into(const FixNode* fix, int nfix, const Bricks& g, int32_t* sb, int* nsb, int32_t* enq,
                              int* nenq) {
    int ns = 0, ne = 0;
    for (int t = 0; t < nfix; ++t) {
        const FixNode& f = fix[t];
        if (ns == 0 || sb[ns - 1] != f.b) sb[ns++] = f.b;
        enq[ne++] = f.b;
        const int x = f.p & 7, y = (f.p >> 3) & 7, z = f.p >> 6;
        const int bl = f.b - g.boff;
        const int bx = bl % g.BX, by = (bl / g.BX) % g.BY, bz = bl / (g.BX * g.BY);
        if (x == 0 && bx > 0) enq[ne++] = f.b - 1;
        if (x == 7 && bx < g.BX - 1) enq[ne++] = f.b + 1;
        if (y == 0 && by > 0) enq[ne++] = f.b - g.BX;
        if (y == 7 && by < g.BY - 1) enq[ne++] = f.b + g.BX;
        if (z == 0 && bz > 0) enq[ne++] = f.b - g.BX * g.BY;
        if (z == 7 && bz < g.BZ - 1) enq[ne++] = f.b + g.BX * g.BY;
    }
    std::sort(enq, enq + ne);
    *nenq = static_cast<int>(std::unique(enq, enq + ne) - enq);
    *nsb = ns;
}

inline void first_active(const std::vector<FixNode>& fix, const Bricks& g, std::vector<int32_t>& sb,
                         std::vector<int32_t>& enq) {
    sb.resize(fix.size());
    enq.resize(7 * fix.size());
    int ns = 0, ne = 0;
    first_active_into(fix.data(), static_cast<int>(fix.size()), g, sb.data(), &ns, enq.data(), &ne);
    sb.resize(ns);
    enq.resize(ne);
}

// The checks every solve entry point applies to eik_params (the learned
// schedule's weights are the caller's to check): nullptr if the parameters are
// valid, else the message, with the status in *code.
inline const char* param_error(const eik_params& p, eik_status* code) {
    *code = EIK_EINVAL;
    if (!(p.stride > 0.0)) return "stride must be > 0 (+inf allowed), or 0 for the learned schedule";
    if (p.block_dim != 0 && p.block_dim != 8 && p.block_dim != 16 && p.block_dim != 32) {
        *code = EIK_ENOTSUP;
        return "block_dim must be 8, 16 or 32 (or 0)";
    }
    if (p.schedule != EIK_SCHED_FIXED && p.schedule != EIK_SCHED_LEARNED && p.schedule != EIK_SCHED_RANDOM)
        return "schedule must be EIK_SCHED_FIXED, EIK_SCHED_LEARNED or EIK_SCHED_RANDOM";
    if (!(p.window >= 0.0) || !std::isfinite(p.window)) return "window must be finite and >= 0";
    if (!(p.fallback_tau >= 0.0) || !(p.fallback_tau <= 1.0)) return "fallback_tau must lie in [0, 1]";
    if (p.max_restarts < 0) return "max_restarts must be >= 0";
    if (!(p.width >= 0.0)) return "width must be >= 0 (0 = +inf)";
    if (p.wait_polls < 0) return "wait_polls must be >= 0 (0 = default)";
    *code = EIK_OK;
    return nullptr;
}

// The 2x2x2 groups (16^3 blocks) of a list of global bricks of grid g, whose
// groups start at goff (GX x GY x GZ groups).  Sorted, unique.
inline std::vector<int32_t> groups_of(const std::vector<int32_t>& bricks, const Bricks& g, int GX, int GY,
                                      int32_t goff) {
    std::vector<int32_t> out;
    for (int32_t b : bricks) {
        const int bl = b - g.boff;
        const int bx = bl % g.BX, by = (bl / g.BX) % g.BY, bz = bl / (g.BX * g.BY);
        out.push_back(goff + ((bz >> 1) * GY + (by >> 1)) * GX + (bx >> 1));
    }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    return out;
}

}  // namespace eikh
