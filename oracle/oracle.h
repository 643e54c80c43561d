/*
 * The oracle's own declarations.  TEST INFRASTRUCTURE ONLY: only tests/, the
 * smoke check and bench.py's CPU-baseline leg load liboracle.so.  Nothing here
 * is shared with the CUDA library (no common headers, helpers or tables).
 *
 * Every array is a node-centred grid of nx*ny*nz points, x fastest:
 * idx = (k*ny + j)*nx + i, node (i,j,k) at physical (i*h, j*h, k*h).
 * Arithmetic is IEEE double, compiled with -ffp-contract=off.
 */
#ifndef EIK_ORACLE_H
#define EIK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status tags of Sec. 2.1 / 2.2 (FAR, BAND, KNOWN_NEW, KNOWN_FIX). */
enum { ORC_FAR = 0, ORC_BAND = 1, ORC_KNOWN_NEW = 2, ORC_KNOWN_FIX = 3 };

/* Error codes. */
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ECAP = -3 };

/* Nodes "on or adjacent to Gamma" for point sources (Alg. 1): the nodes of the
 * grid cell that contains each source, with psi0 = |x_node - x_s| / F_node,
 * minimum over sources.  Writes up to cap (index, psi0) pairs; returns the
 * count or an error code. */
int64_t orc_fix_nodes(int nx, int ny, int nz, double h, const double *F,
                      int nsrc, const double *src_xyz,
                      int64_t *out_idx, double *out_psi0, int64_t cap);

/* Alg. 3 for one point: per-axis upwind KNOWN neighbour, sort, grow id.
 * nbv/nbk: the six neighbours (x-, x+, y-, y+, z-, z+) value and KNOWN flag;
 * psi_c: the point's current value; r2 = h^2/F^2.  Returns +inf when no
 * neighbour qualifies. */
double orc_solve_quadratic(double psi_c, const double nbv[6], const int nbk[6], double r2);

/* Single-heap fast marching (Algs. 1, 2, 3, 4 with one block and
 * width_band = bound_band = +inf).  psi_out: nx*ny*nz.  If log_idx/log_val
 * are non-NULL they receive the acceptance sequence (index, value) of every
 * heap pop, up to log_cap entries; *n_log gets the number of pops. */
int orc_fmm(int nx, int ny, int nz, double h, const double *F,
            int nsrc, const double *src_xyz, double *psi_out,
            int64_t *log_idx, double *log_val, int64_t log_cap, int64_t *n_log);

/* Brute force: Jacobi sweeps psi <- min(psi, Solve_Quadratic over all
 * in-domain neighbours) from +inf (sources fixed) until nothing changes.
 * *sweeps gets the number of sweeps; returns ORC_ECAP if max_sweeps is hit. */
int orc_jacobi(int nx, int ny, int nz, double h, const double *F,
               int nsrc, const double *src_xyz, double *psi_out,
               int64_t max_sweeps, int64_t *sweeps);

/* Residual of Eq. (2.1) at every non-fixed node with F > 0 and finite psi:
 * |F^2 * sum_axes max((psi - min(nb-, nb+))/h, 0)^2 - 1|.  Nodes listed in
 * skip_idx (the fixed nodes) are skipped.  Returns the maximum; *n_checked
 * gets the number of nodes checked. */
double orc_residual(int nx, int ny, int nz, double h, const double *F, const double *psi,
                    const int64_t *skip_idx, int64_t n_skip, int64_t *n_checked);

/* The same residual at selected nodes only, from 7-point stencils supplied by
 * the caller: stencil[7*s + 0] = psi at node s, then x-, x+, y-, y+, z-, z+
 * (+inf outside the grid); F[s] its speed.  out[s] gets the residual
 * (0 for F == 0 or psi == inf). */
void orc_residual_stencils(int64_t n, const double *stencil, const double *F, double h, double *out);

/* Statistics of the block solver. */
typedef struct {
    int64_t nr;            /* restarts: iterations of the loop of Alg. 6 */
    int64_t marches;       /* calls of March_Narrow_Band */
    int64_t exchanges;     /* calls of Integrate_Ghost_Cell_Data */
    int64_t pops;          /* heap pops over all blocks */
    int64_t updates;       /* accepted Solve_Quadratic results */
    int64_t ghost_updates; /* ghost points lowered by the exchange */
} orc_block_stats;

/* Block-based restarted narrow-band fast marching (Alg. 6 with Algs. 1-5):
 * each axis split into pieces of dim_block nodes (the last one ragged), one
 * ghost layer per block, per-block heaps, march/exchange activation flags.
 * stride and width may be +inf.  nthreads <= 0 uses the OpenMP default.
 * Returns ORC_ECAP if max_restarts is reached. */
int orc_block_fmm(int nx, int ny, int nz, double h, const double *F,
                  int nsrc, const double *src_xyz, int dim_block,
                  double stride, double width, int nthreads, int64_t max_restarts,
                  double *psi_out, orc_block_stats *stats);

#ifdef __cplusplus
}
#endif
#endif
