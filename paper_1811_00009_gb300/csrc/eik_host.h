// Host-side set-up shared by the one-grid runtime (eik_runtime.cu) and the
// batched runtime (eik_batch.cu): the fixed nodes of point sources (Alg. 1)
// and the blocks active at the first restart.
#pragma once

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

// Every node of every cell that contains a source (xyz: n*3 coordinates).
inline void source_candidates(const double* xyz, int nsrc, int nx, int ny, int nz, double h, const Bricks& g,
                              std::vector<Cand>& out) {
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
                    const double dx = i * h - xs[0], dy = j * h - xs[1], dz = k * h - xs[2];
                    Cand c;
                    c.b = g.boff + ((k >> 3) * g.BY + (j >> 3)) * g.BX + (i >> 3);
                    c.p = ((k & 7) * 8 + (j & 7)) * 8 + (i & 7);
                    c.dist = std::sqrt(dx * dx + dy * dy + dz * dz);
                    out.push_back(c);
                }
    }
}

struct FixNode {
    int32_t b, p;
    double v;
};

// Fixed nodes from the candidates and their h/F (r): psi0 = distance / F; a
// node on a source gets 0; a barrier node (F = 0) is not fixed; a node next
// to several sources keeps the smallest psi0.  Sorted by (brick, node).
inline std::vector<FixNode> fixed_nodes(const std::vector<Cand>& cand, const std::vector<double>& r, double h) {
    std::vector<FixNode> fix;
    for (size_t t = 0; t < cand.size(); ++t) {
        double v;
        if (cand[t].dist == 0.0) v = 0.0;
        else if (std::isfinite(r[t]) && r[t] > 0.0) v = cand[t].dist * r[t] / h;
        else continue;
        fix.push_back({cand[t].b, cand[t].p, v});
    }
    std::sort(fix.begin(), fix.end(), [](const FixNode& a, const FixNode& b) {
        return a.b != b.b ? a.b < b.b : (a.p != b.p ? a.p < b.p : a.v < b.v);
    });
    std::vector<FixNode> uf;
    for (const auto& f : fix)
        if (uf.empty() || uf.back().b != f.b || uf.back().p != f.p) uf.push_back(f);
    return uf;
}

// Bricks holding fixed nodes (sb), and the work list of restart 1 (enq): those
// bricks and the neighbours whose ghost layer holds a fixed node (Alg. 1 runs
// over Xi^ib).  Fixed nodes must all lie in grid g.  Both sorted, unique.
inline void first_active(const std::vector<FixNode>& fix, const Bricks& g, std::vector<int32_t>& sb,
                         std::vector<int32_t>& enq) {
    for (const auto& f : fix) {
        if (sb.empty() || sb.back() != f.b) sb.push_back(f.b);
        enq.push_back(f.b);
        const int x = f.p & 7, y = (f.p >> 3) & 7, z = f.p >> 6;
        const int bl = f.b - g.boff;
        const int bx = bl % g.BX, by = (bl / g.BX) % g.BY, bz = bl / (g.BX * g.BY);
        if (x == 0 && bx > 0) enq.push_back(f.b - 1);
        if (x == 7 && bx < g.BX - 1) enq.push_back(f.b + 1);
        if (y == 0 && by > 0) enq.push_back(f.b - g.BX);
        if (y == 7 && by < g.BY - 1) enq.push_back(f.b + g.BX);
        if (z == 0 && bz > 0) enq.push_back(f.b - g.BX * g.BY);
        if (z == 7 && bz < g.BZ - 1) enq.push_back(f.b + g.BX * g.BY);
    }
    std::sort(enq.begin(), enq.end());
    enq.erase(std::unique(enq.begin(), enq.end()), enq.end());
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
