/*
 * xdgprob.h -- generator of the agglomerated XDG-SIP linear system (the INPUT of the
 * multigrid solve).
 *
 * Kummer, Smuda, Weber, "BoSSS: a package for multigrid extended discontinuous Galerkin
 * methods" (arXiv 2003.02431):
 *   - Poisson problem with a jump in the diffusivity, Eq. (poisson-jump-problem-def), section 1.1
 *   - level set, species A = {phi<0}, B = {phi>0}, interface normal grad(phi)/|grad(phi)|, section 1.1
 *   - DG / XDG spaces, cut-cell mesh, jump and mean operators, section 2.1 (Definitions 2-5)
 *   - SIP bilinear form and right-hand side, Eqs. (DefSIP), (SIPrhs), section 2.2
 *   - cell agglomeration A_alpha, section 2.3
 *   - aggregation sequence, mapping onto the cut-cell mesh, level spaces, section 3.1
 *   - basis Phi^{X,lambda}, re-orthonormalisation S, transfer R^{X,lambda}, section 3.2,
 *     Eqs. (XdgMgBasis), (XDGrestrictionMatrix)
 *
 * The generator holds the discretisation only: geometry, cut-cell quadrature, agglomeration,
 * bases, assembly of the finest-level operator M^1 and right-hand side b^1, the aggregation
 * maps and the transfer blocks R^{X,lambda}. It performs none of the solve (no operator
 * apply, no smoothing, no Galerkin product, no factorisation of the operator, no Krylov).
 *
 * Plain C ABI; all arrays are owned by the handle and stay valid until xp_free().
 */
#ifndef XDGPROB_H
#define XDGPROB_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int D;              /* 2 or 3 */
  int N;              /* cells per direction */
  int k;              /* DG degree (total degree), Np = C(k+D, D) */
  int rhs_kind;       /* 0: u_s = phi*prod(cos(pi x_d))/mu_s; 1: u_s = phi/mu_s; 2: f = 1, g_D = 0 */
  int max_coarse_dof; /* stop coarsening once a level has at most this many DOF */
  int max_levels;     /* hard cap on the number of levels (>= 1) */
  int quad_q;         /* Gauss points per sub-interval in cut cells (0 = default) */
  int nthreads;       /* OpenMP threads (0 = default) */
  double lo, hi;      /* domain [lo,hi]^D */
  double c[3];        /* level-set sphere/circle centre */
  double R;           /* radius: phi = |x-c|^2 - R^2 */
  double muA, muB;    /* diffusivity in A = {phi<0} and B = {phi>0} */
  double alpha;       /* agglomeration threshold on the volume fraction */
  double ceta;        /* SIP penalty constant */
} xp_config;

typedef struct {
  int D, N, k, Np;
  int n_levels;
  int n_cells, n_cut_cells, n_parts, n_small, n_isolated;
  int64_t nnzb1;      /* non-zero blocks of M^1 */
  double volA, volB, areaI;  /* sums of the cut-cell quadrature (closed-form checks) */
  double h;
} xp_info;

void* xp_build(const xp_config* cfg, char* err, int errlen);
void  xp_free(void* h);
void  xp_get_info(void* h, xp_info* out);

/* per-level block counts and metadata (level in 1..n_levels) */
int      xp_level_nb(void* h, int level);
const int32_t* xp_level_rep(void* h, int level);     /* representative (minimum) background cell */
const int8_t*  xp_level_species(void* h, int level); /* 0 = A, 1 = B */
const double*  xp_level_volume(void* h, int level);  /* block volume */
const int8_t*  xp_level_cut(void* h, int level);     /* 1 if any member part is cut */

/* finest-level system (BSR: row_ptr[nb+1], col[nnzb], val[nnzb][Np][Np] row-major, b[nb][Np]) */
const int64_t* xp_row_ptr(void* h);
const int32_t* xp_col(void* h);
const double*  xp_val(void* h);
const double*  xp_rhs(void* h);

/* transfer from level l to l+1 (l in 1..n_levels-1): agg[nb_l] and R[nb_l][Np][Np],
 * R_f[m][n] = integral over fine block f of Phi^l_{f,m} Phi^{l+1}_{agg[f],n}. */
const int32_t* xp_agg(void* h, int level);
const double*  xp_R(void* h, int level);

/* direct assembly of a(.,.) and b(.) in the basis of level `level` (for Galerkin-consistency
 * checks): arrays are allocated with malloc and must be released with xp_release. */
int  xp_assemble_level(void* h, int level, int64_t** row_ptr, int32_t** col, double** val,
                       double** rhs, int64_t* nnzb);
void xp_release(void* p);

/* L2 error (squared) of the level-1 coefficient vector x against the manufactured solution,
 * and squared L2 norm of the exact solution; returns -1 if rhs_kind has no exact solution. */
int xp_l2_error(void* h, const double* x, double* err2, double* norm2);

/* per-block features of level-1 cut blocks for a learned smoother:
 * for every level-1 block: phi at the 2^D vertices of the representative cell,
 * volume fractions of A and B in that cell, writes 2^D + 2 doubles per block. */
void xp_block_features(void* h, double* out);

/* the same features for n given background cells (2^D + 2 doubles each) */
void xp_cell_features(void* h, int n, const int32_t* cells, double* out);

/* cells holding parts of both species: (cell, level-1 block of the A part, level-1 block of
 * the B part) per cell, ascending cell index; returns the count (out == NULL: count only). */
int xp_cut_cells(void* h, int32_t* out);

#ifdef __cplusplus
}
#endif
#endif
