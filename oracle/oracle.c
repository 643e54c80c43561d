/*
 * Oracle for the block-based restarted narrow-band fast marching method
 * (J. Yang, "An easily-implemented, block-based fast marching method with
 * superior sequential and parallel performance", 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64, single source file.  It is
 * loaded by tests/, by the smoke check and by the CPU-baseline leg of the
 * benchmark, never by the product path.  It shares no code with the CUDA
 * library.
 *
 * What it computes: the solution of the Godunov upwind system, Eq. (2.1)
 * with the one-sided differences of Eq. (2.2), on a node-centred uniform grid,
 * for point sources.  orc_fmm is the sequential fast marching method of
 * Sec. 2.1 with the unified heap of Sec. 2.2 (Algs. 1-4 with one block and an
 * infinite bound).  orc_block_fmm is the paper's method, Alg. 6 with Algs. 1-5.
 *
 * Readings of the paper that this file takes:
 *  - point sources: the nodes of the cell containing a source are "on or
 *    adjacent to Gamma" (Alg. 1), psi0 = distance / F at that node;
 *  - Alg. 3's quadratic a*x^2 - 2*b*x + c = 0 is evaluated on values
 *    measured from the smallest upwind value (the same root, without the
 *    cancellation of b^2 - a*c at large psi); a negative discriminant, which
 *    exact arithmetic never produces, is clamped to zero, and so is a root
 *    below the largest admitted value (causality, see orc_solve_quadratic);
 *  - heap ties are broken by the point index;
 *  - barrier nodes (F = 0) are never solved (Sec. 3.3);
 *  - bound_band accumulates by repeated addition of the stride (Alg. 6).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_INF HUGE_VAL

/* ------------------------------------------------------------------ */
/* Sources (Alg. 1: points on or adjacent to Gamma)                    */
/* ------------------------------------------------------------------ */

/* Grid indices along one axis of the cell containing coordinate s.  A source
 * within 1e-9 cell widths of a node sits on that node (one index). */
static int axis_cell(double s, double h, int n, int out[2])
{
    double t = s / h;
    double tn = floor(t + 0.5);
    if (fabs(t - tn) <= 1e-9) {
        int i = (int)tn;
        if (i < 0) i = 0;
        if (i > n - 1) i = n - 1;
        out[0] = i;
        return 1;
    }
    int i0 = (int)floor(t);
    if (i0 > n - 2) i0 = n - 2;
    if (i0 < 0) i0 = 0;
    out[0] = i0;
    out[1] = i0 + 1;
    return 2;
}

typedef struct { int64_t idx; double v; } fixpair;

static int cmp_fixpair(const void *a, const void *b)
{
    const fixpair *x = (const fixpair *)a, *y = (const fixpair *)b;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return (x->v < y->v) ? -1 : (x->v > y->v);
}

int64_t orc_fix_nodes(int nx, int ny, int nz, double h, const double *F,
                      int nsrc, const double *src, int64_t *out_idx, double *out_psi0, int64_t cap)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || nsrc < 0) return ORC_EINVAL;
    int n[3] = {nx, ny, nz};
    fixpair *list = (fixpair *)malloc(sizeof(fixpair) * (size_t)(8 * (nsrc > 0 ? nsrc : 1)));
    if (!list) return ORC_ENOMEM;
    int64_t m = 0;
    for (int s = 0; s < nsrc; ++s) {
        int cell[3][2], cnt[3];
        for (int a = 0; a < 3; ++a) {
            double c = src[3 * s + a];
            double ext = (double)(n[a] - 1) * h;
            double tol = 1e-9 * h;
            if (!(c >= -tol && c <= ext + tol)) { free(list); return ORC_EINVAL; }
            cnt[a] = axis_cell(c, h, n[a], cell[a]);
        }
        for (int cz = 0; cz < cnt[2]; ++cz)
            for (int cy = 0; cy < cnt[1]; ++cy)
                for (int cx = 0; cx < cnt[0]; ++cx) {
                    int i = cell[0][cx], j = cell[1][cy], k = cell[2][cz];
                    int64_t idx = ((int64_t)k * ny + j) * nx + i;
                    double dx = i * h - src[3 * s + 0];
                    double dy = j * h - src[3 * s + 1];
                    double dz = k * h - src[3 * s + 2];
                    double dist = sqrt(dx * dx + dy * dy + dz * dz);
                    double f = F[idx];
                    double v;
                    if (dist == 0.0) v = 0.0;
                    else if (f > 0.0) v = dist / f;
                    else continue;            /* a barrier node cannot carry a finite psi0 */
                    list[m].idx = idx;
                    list[m].v = v;
                    ++m;
                }
    }
    qsort(list, (size_t)m, sizeof(fixpair), cmp_fixpair);
    int64_t u = 0;
    for (int64_t t = 0; t < m; ++t) {
        if (u > 0 && list[u - 1].idx == list[t].idx) continue;   /* sorted: first is the minimum */
        list[u++] = list[t];
    }
    if (u > cap) { free(list); return ORC_ECAP; }
    for (int64_t t = 0; t < u; ++t) {
        if (out_idx) out_idx[t] = list[t].idx;
        if (out_psi0) out_psi0[t] = list[t].v;
    }
    free(list);
    return u;
}

/* ------------------------------------------------------------------ */
/* Alg. 3: Solve_Quadratic                                              */
/* ------------------------------------------------------------------ */

double orc_solve_quadratic(double psi_c, const double nbv[6], const int nbk[6], double r2)
{
    double v[3];
    int nd = 0;
    for (int a = 0; a < 3; ++a) {
        /* upwind neighbour in this direction: a KNOWN one below psi_c, the smaller of the two */
        double lo = nbv[2 * a], hi = nbv[2 * a + 1];
        int d = 0;
        if (nbk[2 * a] && psi_c > lo) d = -1;
        if (nbk[2 * a + 1] && psi_c > hi) {
            if (d == 0 || hi < lo) d = 1;
        }
        if (d != 0) v[nd++] = (d < 0) ? lo : hi;
    }
    if (nd == 0) return ORC_INF;
    /* reorder psi_1 <= ... <= psi_nd */
    for (int i = 1; i < nd; ++i)
        for (int j = i; j > 0 && v[j] < v[j - 1]; --j) {
            double t = v[j]; v[j] = v[j - 1]; v[j - 1] = t;
        }
    int id = 1;
    for (;;) {
        /* a x^2 - 2 b x + c = 0 in the variable x - psi_1 */
        double a = (double)id, b = 0.0, c = 0.0;
        for (int i = 0; i < id; ++i) {
            double d = v[i] - v[0];
            b += d;
            c += d * d;
        }
        c -= r2;
        double disc = b * b - a * c;
        if (disc < 0.0) disc = 0.0;
        double t = v[0] + (b + sqrt(disc)) / a;
        /* Causality of the upwind scheme (Sec. 2.1): the root is never below the
         * largest admitted value.  The admission test of Alg. 3 guarantees this
         * in exact arithmetic; rounding can break it by an ulp when the last
         * admitted value sits right at the threshold, which would let two nodes
         * lower each other endlessly.  Enforce it. */
        if (t < v[id - 1]) t = v[id - 1];
        if (id < nd && t > v[id]) { ++id; continue; }
        return t;
    }
}

/* ------------------------------------------------------------------ */
/* Binary min-heap with a position index (Sec. 2.1: Insert_Heap,       */
/* Locate_Min, Remove_Min, Up_Heap), keyed by (psi, index).            */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t *a;     /* heap array of point indices */
    int32_t n;
    int32_t *pos;   /* pos[p] = slot of p in a, or -1 */
    const double *key;
} heap_t;

static inline int hless(const heap_t *H, int32_t x, int32_t y)
{
    double kx = H->key[x], ky = H->key[y];
    return kx < ky || (kx == ky && x < y);
}

static void heap_sift_up(heap_t *H, int32_t i)
{
    int32_t p = H->a[i];
    while (i > 0) {
        int32_t parent = (i - 1) >> 1;
        int32_t q = H->a[parent];
        if (!hless(H, p, q)) break;
        H->a[i] = q;
        H->pos[q] = i;
        i = parent;
    }
    H->a[i] = p;
    H->pos[p] = i;
}

static void heap_sift_down(heap_t *H, int32_t i)
{
    int32_t p = H->a[i];
    for (;;) {
        int32_t c = 2 * i + 1;
        if (c >= H->n) break;
        if (c + 1 < H->n && hless(H, H->a[c + 1], H->a[c])) ++c;
        if (!hless(H, H->a[c], p)) break;
        H->a[i] = H->a[c];
        H->pos[H->a[i]] = i;
        i = c;
    }
    H->a[i] = p;
    H->pos[p] = i;
}

static void heap_insert(heap_t *H, int32_t p)
{
    H->a[H->n] = p;
    H->pos[p] = H->n;
    ++H->n;
    heap_sift_up(H, H->n - 1);
}

static void heap_remove_min(heap_t *H)
{
    int32_t top = H->a[0];
    H->pos[top] = -1;
    --H->n;
    if (H->n > 0) {
        H->a[0] = H->a[H->n];
        H->pos[H->a[0]] = 0;
        heap_sift_down(H, 0);
    }
}

static inline void heap_insert_or_up(heap_t *H, int32_t p)
{
    if (H->pos[p] < 0) heap_insert(H, p);
    else heap_sift_up(H, H->pos[p]);
}

/* ------------------------------------------------------------------ */
/* Single-heap fast marching (Algs. 1-4, one block, infinite bound)    */
/* ------------------------------------------------------------------ */

static inline int is_known(uint8_t g) { return g == ORC_KNOWN_NEW || g == ORC_KNOWN_FIX; }

int orc_fmm(int nx, int ny, int nz, double h, const double *F,
            int nsrc, const double *src, double *psi,
            int64_t *log_idx, double *log_val, int64_t log_cap, int64_t *n_log)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0)) return ORC_EINVAL;
    int64_t N = (int64_t)nx * ny * nz;
    if (N > 0x7fffffffLL) return ORC_EINVAL;
    int64_t nfix_cap = 8 * (int64_t)(nsrc > 0 ? nsrc : 1);
    int64_t *fidx = (int64_t *)malloc(sizeof(int64_t) * nfix_cap);
    double *fval = (double *)malloc(sizeof(double) * nfix_cap);
    uint8_t *G = (uint8_t *)malloc((size_t)N);
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *ha = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!fidx || !fval || !G || !pos || !ha) {
        free(fidx); free(fval); free(G); free(pos); free(ha);
        return ORC_ENOMEM;
    }
    int64_t nfix = orc_fix_nodes(nx, ny, nz, h, F, nsrc, src, fidx, fval, nfix_cap);
    if (nfix < 0) {
        free(fidx); free(fval); free(G); free(pos); free(ha);
        return (int)nfix;
    }
    /* Alg. 1 */
    for (int64_t p = 0; p < N; ++p) { psi[p] = ORC_INF; G[p] = ORC_FAR; pos[p] = -1; }
    heap_t H = {ha, 0, pos, psi};
    for (int64_t t = 0; t < nfix; ++t) {
        psi[fidx[t]] = fval[t];
        G[fidx[t]] = ORC_KNOWN_FIX;
        heap_insert(&H, (int32_t)fidx[t]);
    }
    const double h2 = h * h;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    int64_t npop = 0;
    /* Alg. 4 with width_band = bound_band = +inf: the loop ends when the heap is empty */
    while (H.n > 0) {
        int32_t p = H.a[0];
        if (G[p] != ORC_KNOWN_FIX) G[p] = ORC_KNOWN_NEW;
        heap_remove_min(&H);
        if (log_idx && npop < log_cap) { log_idx[npop] = p; log_val[npop] = psi[p]; }
        ++npop;
        /* Alg. 2: Update_Neighbors(p) */
        int i = (int)(p % nx), j = (int)((p / nx) % ny), k = (int)(p / sz);
        for (int d = 0; d < 6; ++d) {
            int a = d >> 1, dir = (d & 1) ? 1 : -1;
            int ci = i + (a == 0 ? dir : 0), cj = j + (a == 1 ? dir : 0), ck = k + (a == 2 ? dir : 0);
            if (ci < 0 || ci >= nx || cj < 0 || cj >= ny || ck < 0 || ck >= nz) continue;
            int64_t q = ((int64_t)ck * ny + cj) * nx + ci;
            if (G[q] == ORC_KNOWN_FIX || !(psi[q] > psi[p])) continue;
            if (!(F[q] > 0.0)) continue;                    /* barrier: never solved */
            double nbv[6];
            int nbk[6];
            int qi[3] = {ci, cj, ck}, nn[3] = {nx, ny, nz};
            int64_t st[3] = {sx, sy, sz};
            for (int e = 0; e < 6; ++e) {
                int b = e >> 1, s = (e & 1) ? 1 : -1;
                int c = qi[b] + s;
                if (c < 0 || c >= nn[b]) { nbv[e] = ORC_INF; nbk[e] = 0; continue; }
                int64_t r = q + s * st[b];
                nbv[e] = psi[r];
                nbk[e] = is_known(G[r]);
            }
            double t = orc_solve_quadratic(psi[q], nbv, nbk, h2 / (F[q] * F[q]));
            if (t < psi[q]) {
                psi[q] = t;
                G[q] = ORC_BAND;
                heap_insert_or_up(&H, (int32_t)q);
            }
        }
    }
    if (n_log) *n_log = npop;
    free(fidx); free(fval); free(G); free(pos); free(ha);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Brute force: Jacobi iteration of the same local solve               */
/* ------------------------------------------------------------------ */

int orc_jacobi(int nx, int ny, int nz, double h, const double *F,
               int nsrc, const double *src, double *psi, int64_t max_sweeps, int64_t *sweeps)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0)) return ORC_EINVAL;
    int64_t N = (int64_t)nx * ny * nz;
    int64_t nfix_cap = 8 * (int64_t)(nsrc > 0 ? nsrc : 1);
    int64_t *fidx = (int64_t *)malloc(sizeof(int64_t) * nfix_cap);
    double *fval = (double *)malloc(sizeof(double) * nfix_cap);
    uint8_t *fixed = (uint8_t *)calloc((size_t)N, 1);
    double *nxt = (double *)malloc(sizeof(double) * (size_t)N);
    if (!fidx || !fval || !fixed || !nxt) {
        free(fidx); free(fval); free(fixed); free(nxt);
        return ORC_ENOMEM;
    }
    int64_t nfix = orc_fix_nodes(nx, ny, nz, h, F, nsrc, src, fidx, fval, nfix_cap);
    if (nfix < 0) {
        free(fidx); free(fval); free(fixed); free(nxt);
        return (int)nfix;
    }
    for (int64_t p = 0; p < N; ++p) psi[p] = ORC_INF;
    for (int64_t t = 0; t < nfix; ++t) { psi[fidx[t]] = fval[t]; fixed[fidx[t]] = 1; }
    const double h2 = h * h;
    int64_t it = 0;
    int rc = ORC_OK;
    for (;;) {
        if (it >= max_sweeps) { rc = ORC_ECAP; break; }
        ++it;
        int changed = 0;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int64_t p = ((int64_t)k * ny + j) * nx + i;
                    nxt[p] = psi[p];
                    if (fixed[p] || !(F[p] > 0.0)) continue;
                    int qi[3] = {i, j, k}, nn[3] = {nx, ny, nz};
                    int64_t st[3] = {1, nx, (int64_t)nx * ny};
                    double nbv[6];
                    int nbk[6];
                    for (int e = 0; e < 6; ++e) {
                        int b = e >> 1, s = (e & 1) ? 1 : -1;
                        int c = qi[b] + s;
                        if (c < 0 || c >= nn[b]) { nbv[e] = ORC_INF; nbk[e] = 0; continue; }
                        nbv[e] = psi[p + s * st[b]];
                        nbk[e] = 1;
                    }
                    double t = orc_solve_quadratic(psi[p], nbv, nbk, h2 / (F[p] * F[p]));
                    if (t < psi[p]) { nxt[p] = t; changed = 1; }
                }
        memcpy(psi, nxt, sizeof(double) * (size_t)N);
        if (!changed) break;
    }
    if (sweeps) *sweeps = it;
    free(fidx); free(fval); free(fixed); free(nxt);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Residual of Eq. (2.1)                                                */
/* ------------------------------------------------------------------ */

static double residual_one(double p, const double nb[6], double f, double h)
{
    if (!(f > 0.0) || isinf(p)) return 0.0;
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        /* max(D^- psi, -D^+ psi, 0) with the one-sided differences of Eq. (2.2) */
        double dm = (p - nb[2 * a]) / h;
        double dp = (p - nb[2 * a + 1]) / h;   /* -D^+ psi */
        double m = 0.0;
        if (dm > m) m = dm;
        if (dp > m) m = dp;
        s += m * m;
    }
    return fabs(s * f * f - 1.0);
}

double orc_residual(int nx, int ny, int nz, double h, const double *F, const double *psi,
                    const int64_t *skip_idx, int64_t n_skip, int64_t *n_checked)
{
    int64_t N = (int64_t)nx * ny * nz;
    uint8_t *skip = (uint8_t *)calloc((size_t)N, 1);
    if (!skip) return -1.0;
    for (int64_t t = 0; t < n_skip; ++t) skip[skip_idx[t]] = 1;
    double worst = 0.0;
    int64_t cnt = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t p = ((int64_t)k * ny + j) * nx + i;
                if (skip[p] || !(F[p] > 0.0) || isinf(psi[p])) continue;
                double nb[6];
                nb[0] = i > 0 ? psi[p - 1] : ORC_INF;
                nb[1] = i < nx - 1 ? psi[p + 1] : ORC_INF;
                nb[2] = j > 0 ? psi[p - nx] : ORC_INF;
                nb[3] = j < ny - 1 ? psi[p + nx] : ORC_INF;
                nb[4] = k > 0 ? psi[p - (int64_t)nx * ny] : ORC_INF;
                nb[5] = k < nz - 1 ? psi[p + (int64_t)nx * ny] : ORC_INF;
                double r = residual_one(psi[p], nb, F[p], h);
                if (r > worst) worst = r;
                ++cnt;
            }
    free(skip);
    if (n_checked) *n_checked = cnt;
    return worst;
}

void orc_residual_stencils(int64_t n, const double *stencil, const double *F, double h, double *out)
{
    for (int64_t s = 0; s < n; ++s) out[s] = residual_one(stencil[7 * s], stencil + 7 * s + 1, F[s], h);
}

/* ------------------------------------------------------------------ */
/* Block-based restarted narrow-band fast marching (Alg. 6)            */
/* ------------------------------------------------------------------ */

typedef struct {
    int o[3];         /* global index of the first interior node */
    int s[3];         /* interior extent */
    int e[3];         /* extent with one ghost layer on each side: s + 2 */
    int nb[6];        /* neighbouring blocks across faces x-, x+, y-, y+, z-, z+ (-1: none) */
    double *psi;      /* psi^ib on Xi^ib */
    uint8_t *G;       /* G^ib on Xi^ib */
    int32_t *pos;
    int32_t *ha;
    int32_t hn;
    uint8_t *ups;     /* Upsilon^ib membership on Xi^ib */
    int32_t *ups_list;
    int32_t ups_n;
    int active;       /* A^ib */
    uint8_t C[6];     /* C^ib(nb) for the neighbour across each face */
    int64_t pops, updates, ghost_updates;
} oblock;

static inline int32_t lidx(const oblock *B, int lx, int ly, int lz)
{
    return ((int32_t)lz * B->e[1] + ly) * B->e[0] + lx;
}

/* Alg. 2 inside block B for the point just popped (local index p). */
static void block_update_neighbors(oblock *B, int32_t p, const double *F, int nx, int ny, double h2)
{
    heap_t H = {B->ha, B->hn, B->pos, B->psi};
    int ex = B->e[0], ey = B->e[1];
    int lx = p % ex, ly = (p / ex) % ey, lz = p / (ex * ey);
    int l[3] = {lx, ly, lz};
    int32_t st[3] = {1, ex, ex * ey};
    for (int d = 0; d < 6; ++d) {
        int a = d >> 1, dir = (d & 1) ? 1 : -1;
        int c[3] = {l[0], l[1], l[2]};
        c[a] += dir;
        /* (l,m,n) must lie in Omega^ib: the interior, local 1..s */
        if (c[0] < 1 || c[0] > B->s[0] || c[1] < 1 || c[1] > B->s[1] || c[2] < 1 || c[2] > B->s[2]) continue;
        int32_t q = p + dir * st[a];
        if (B->G[q] == ORC_KNOWN_FIX || !(B->psi[q] > B->psi[p])) continue;
        int gi = B->o[0] + c[0] - 1, gj = B->o[1] + c[1] - 1, gk = B->o[2] + c[2] - 1;
        double f = F[((int64_t)gk * ny + gj) * nx + gi];
        if (!(f > 0.0)) continue;
        double nbv[6];
        int nbk[6];
        for (int e = 0; e < 6; ++e) {
            int b = e >> 1, s = (e & 1) ? 1 : -1;
            int32_t r = q + s * st[b];
            nbv[e] = B->psi[r];
            nbk[e] = is_known(B->G[r]);
        }
        double t = orc_solve_quadratic(B->psi[q], nbv, nbk, h2 / (f * f));
        if (t < B->psi[q]) {
            B->psi[q] = t;
            B->G[q] = ORC_BAND;
            H.n = B->hn;
            heap_insert_or_up(&H, q);
            B->hn = H.n;
            ++B->updates;
            /* q in Pi^ib: on a boundary layer that is a neighbour's ghost zone */
            int on = (c[0] == 1 && B->nb[0] >= 0) || (c[0] == B->s[0] && B->nb[1] >= 0) ||
                     (c[1] == 1 && B->nb[2] >= 0) || (c[1] == B->s[1] && B->nb[3] >= 0) ||
                     (c[2] == 1 && B->nb[4] >= 0) || (c[2] == B->s[2] && B->nb[5] >= 0);
            if (on && !B->ups[q]) { B->ups[q] = 1; B->ups_list[B->ups_n++] = q; }
        }
    }
}

/* Alg. 4: March_Narrow_Band(ib).  Sets C of neighbours at the end. */
static void block_march(oblock *blocks, int ib, double bound, double width,
                        const double *F, int nx, int ny, double h2)
{
    oblock *B = &blocks[ib];
    for (int32_t t = 0; t < B->ups_n; ++t) B->ups[B->ups_list[t]] = 0;   /* Upsilon <- empty */
    B->ups_n = 0;
    heap_t H = {B->ha, B->hn, B->pos, B->psi};
    for (;;) {
        if (B->hn == 0) { B->active = 0; break; }
        int32_t p = B->ha[0];
        if (B->psi[p] > bound) {
            if (B->psi[p] > width) B->active = 0;
            break;
        }
        if (B->G[p] != ORC_KNOWN_FIX) B->G[p] = ORC_KNOWN_NEW;
        H.n = B->hn;
        heap_remove_min(&H);
        B->hn = H.n;
        ++B->pops;
        block_update_neighbors(B, p, F, nx, ny, h2);
    }
    /* for every neighbour whose ghost zone meets Upsilon^ib: C^nb(ib) <- TRUE */
    int hit[6] = {0, 0, 0, 0, 0, 0};
    int ex = B->e[0], ey = B->e[1];
    for (int32_t t = 0; t < B->ups_n; ++t) {
        int32_t q = B->ups_list[t];
        int c[3] = {q % ex, (q / ex) % ey, q / (ex * ey)};
        for (int a = 0; a < 3; ++a) {
            if (c[a] == 1) hit[2 * a] = 1;
            if (c[a] == B->s[a]) hit[2 * a + 1] = 1;
        }
    }
    for (int f = 0; f < 6; ++f)
        if (hit[f] && B->nb[f] >= 0) blocks[B->nb[f]].C[f ^ 1] = 1;
}

/* Alg. 5: Integrate_Ghost_Cell_Data(ib). */
static void block_integrate(oblock *blocks, int ib, double width)
{
    oblock *B = &blocks[ib];
    heap_t H = {B->ha, B->hn, B->pos, B->psi};
    for (int f = 0; f < 6; ++f) {
        if (!B->C[f]) continue;
        const oblock *N = &blocks[B->nb[f]];
        int a = f >> 1;
        /* ghost layer of B on face f, and the matching boundary layer of N */
        int gl = (f & 1) ? B->s[a] + 1 : 0;
        int nl = (f & 1) ? 1 : N->s[a];
        int b1 = (a == 0) ? 1 : 0, b2 = (a == 2) ? 1 : 2;
        for (int u = 1; u <= B->s[b2]; ++u)
            for (int v = 1; v <= B->s[b1]; ++v) {
                int cb[3], cn[3];
                cb[a] = gl; cb[b1] = v; cb[b2] = u;
                cn[a] = nl; cn[b1] = v; cn[b2] = u;
                int32_t g = lidx(B, cb[0], cb[1], cb[2]);
                int32_t r = lidx(N, cn[0], cn[1], cn[2]);
                if (!N->ups[r]) continue;                    /* Theta^ib intersected with Upsilon^nb */
                if (B->psi[g] > N->psi[r]) {
                    B->psi[g] = N->psi[r];
                    B->G[g] = N->G[r];
                    H.n = B->hn;
                    heap_insert_or_up(&H, g);
                    B->hn = H.n;
                    ++B->ghost_updates;
                }
            }
    }
    for (int f = 0; f < 6; ++f) B->C[f] = 0;
    if (B->hn != 0 && B->psi[B->ha[0]] <= width) B->active = 1;
}

int orc_block_fmm(int nx, int ny, int nz, double h, const double *F,
                  int nsrc, const double *src, int dim_block,
                  double stride, double width, int nthreads, int64_t max_restarts,
                  double *psi_out, orc_block_stats *stats)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || dim_block < 1 || !(stride > 0.0)) return ORC_EINVAL;
    int n[3] = {nx, ny, nz};
    int m[3];
    for (int a = 0; a < 3; ++a) m[a] = (n[a] + dim_block - 1) / dim_block;
    int nblocks = m[0] * m[1] * m[2];
    int64_t nfix_cap = 8 * (int64_t)(nsrc > 0 ? nsrc : 1);
    int64_t *fidx = (int64_t *)malloc(sizeof(int64_t) * nfix_cap);
    double *fval = (double *)malloc(sizeof(double) * nfix_cap);
    oblock *blocks = (oblock *)calloc((size_t)nblocks, sizeof(oblock));
    if (!fidx || !fval || !blocks) { free(fidx); free(fval); free(blocks); return ORC_ENOMEM; }
    int64_t nfix = orc_fix_nodes(nx, ny, nz, h, F, nsrc, src, fidx, fval, nfix_cap);
    if (nfix < 0) { free(fidx); free(fval); free(blocks); return (int)nfix; }
    int rc = ORC_OK;
    for (int bz = 0; bz < m[2]; ++bz)
        for (int by = 0; by < m[1]; ++by)
            for (int bx = 0; bx < m[0]; ++bx) {
                int ib = (bz * m[1] + by) * m[0] + bx;
                oblock *B = &blocks[ib];
                int bc[3] = {bx, by, bz};
                for (int a = 0; a < 3; ++a) {
                    B->o[a] = bc[a] * dim_block;
                    B->s[a] = (bc[a] + 1) * dim_block <= n[a] ? dim_block : n[a] - B->o[a];
                    B->e[a] = B->s[a] + 2;
                }
                B->nb[0] = bx > 0 ? ib - 1 : -1;
                B->nb[1] = bx < m[0] - 1 ? ib + 1 : -1;
                B->nb[2] = by > 0 ? ib - m[0] : -1;
                B->nb[3] = by < m[1] - 1 ? ib + m[0] : -1;
                B->nb[4] = bz > 0 ? ib - m[0] * m[1] : -1;
                B->nb[5] = bz < m[2] - 1 ? ib + m[0] * m[1] : -1;
                size_t ne = (size_t)B->e[0] * B->e[1] * B->e[2];
                B->psi = (double *)malloc(sizeof(double) * ne);
                B->G = (uint8_t *)malloc(ne);
                B->pos = (int32_t *)malloc(sizeof(int32_t) * ne);
                B->ha = (int32_t *)malloc(sizeof(int32_t) * ne);
                B->ups = (uint8_t *)calloc(ne, 1);
                B->ups_list = (int32_t *)malloc(sizeof(int32_t) * ne);
                if (!B->psi || !B->G || !B->pos || !B->ha || !B->ups || !B->ups_list) rc = ORC_ENOMEM;
            }
    if (rc != ORC_OK) goto done;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    {
        const double h2 = h * h;
        /* Alg. 6: bound <- 0, C <- FALSE, Initialize_Heap(ib) for every block */
        double bound = 0.0;
#pragma omp parallel for schedule(static)
        for (int ib = 0; ib < nblocks; ++ib) {
            oblock *B = &blocks[ib];
            size_t ne = (size_t)B->e[0] * B->e[1] * B->e[2];
            for (size_t t = 0; t < ne; ++t) { B->psi[t] = ORC_INF; B->G[t] = ORC_FAR; B->pos[t] = -1; }
            B->hn = 0;
            B->active = 0;
            for (int f = 0; f < 6; ++f) B->C[f] = 0;
            heap_t H = {B->ha, 0, B->pos, B->psi};
            /* Alg. 1 over Xi^ib: ghost cells included */
            for (int64_t t = 0; t < nfix; ++t) {
                int64_t g = fidx[t];
                int gi = (int)(g % nx), gj = (int)((g / nx) % ny), gk = (int)(g / ((int64_t)nx * ny));
                int lx = gi - B->o[0] + 1, ly = gj - B->o[1] + 1, lz = gk - B->o[2] + 1;
                if (lx < 0 || lx >= B->e[0] || ly < 0 || ly >= B->e[1] || lz < 0 || lz >= B->e[2]) continue;
                int32_t q = lidx(B, lx, ly, lz);
                B->psi[q] = fval[t];
                B->G[q] = ORC_KNOWN_FIX;
                heap_insert(&H, q);
                B->active = 1;
            }
            B->hn = H.n;
        }
        int *list = (int *)malloc(sizeof(int) * (size_t)nblocks);
        if (!list) { rc = ORC_ENOMEM; goto done; }
        int64_t nr = 0, marches = 0, exchanges = 0;
        for (;;) {
            if (nr >= max_restarts) { rc = ORC_ECAP; break; }
            ++nr;
            bound = bound + stride;
            if (bound > width) bound = width;
            int cnt = 0;
            for (int ib = 0; ib < nblocks; ++ib) if (blocks[ib].active) list[cnt++] = ib;
            marches += cnt;
#pragma omp parallel for schedule(dynamic, 1)
            for (int t = 0; t < cnt; ++t) block_march(blocks, list[t], bound, width, F, nx, ny, h2);
            cnt = 0;
            for (int ib = 0; ib < nblocks; ++ib) {
                const uint8_t *C = blocks[ib].C;
                if (C[0] | C[1] | C[2] | C[3] | C[4] | C[5]) list[cnt++] = ib;
            }
            exchanges += cnt;
#pragma omp parallel for schedule(dynamic, 1)
            for (int t = 0; t < cnt; ++t) block_integrate(blocks, list[t], width);
            int any = 0;
            for (int ib = 0; ib < nblocks; ++ib) any |= blocks[ib].active;
            if (!any) break;
        }
        free(list);
        if (stats) {
            memset(stats, 0, sizeof(*stats));
            stats->nr = nr;
            stats->marches = marches;
            stats->exchanges = exchanges;
            for (int ib = 0; ib < nblocks; ++ib) {
                stats->pops += blocks[ib].pops;
                stats->updates += blocks[ib].updates;
                stats->ghost_updates += blocks[ib].ghost_updates;
            }
        }
        /* gather the interiors */
        for (int ib = 0; ib < nblocks; ++ib) {
            const oblock *B = &blocks[ib];
            for (int lz = 1; lz <= B->s[2]; ++lz)
                for (int ly = 1; ly <= B->s[1]; ++ly)
                    for (int lx = 1; lx <= B->s[0]; ++lx) {
                        int64_t g = ((int64_t)(B->o[2] + lz - 1) * ny + (B->o[1] + ly - 1)) * nx + (B->o[0] + lx - 1);
                        psi_out[g] = B->psi[lidx(B, lx, ly, lz)];
                    }
        }
    }
done:
    for (int ib = 0; ib < nblocks; ++ib) {
        oblock *B = &blocks[ib];
        free(B->psi); free(B->G); free(B->pos); free(B->ha); free(B->ups); free(B->ups_list);
    }
    free(blocks); free(fidx); free(fval);
    return rc;
}
