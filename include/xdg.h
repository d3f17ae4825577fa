/*
 * xdg.h -- C ABI of libxdg: the multigrid-preconditioned solve of the agglomerated XDG
 * (extended discontinuous Galerkin, cut-cell) symmetric-interior-penalty Poisson system on
 * one GPU (sm_103a).
 *
 * Reference: F. Kummer, M. Smuda, J. Weber, "BoSSS: a package for multigrid extended
 * discontinuous Galerkin methods", arXiv 2003.02431.
 *
 * The operation each entry point performs is defined by the paper:
 *   - the system M^1 U = b^1 in per-cell block form: sec. 3.2 "Agglomeration Algebra",
 *     Eq. (GenericMatrixSystem); one Np x Np block per agglomerated cut cell, Np = C(k+D, D)
 *   - the aggregation maps and transfer blocks R^{X,lambda}: sec. 3.1-3.2,
 *     Eq. (XDGrestrictionMatrix) (Phi^{lambda+1} = Phi^lambda R^{X,lambda})
 *   - coarse operators M^{lambda+1} = (R^{X,lambda})^T M^lambda R^{X,lambda}:
 *     Eq. (XDGsysRestriction)
 *   - the level recursion (smoothing, restriction r_c = R^T r, coarse correction,
 *     prolongation z = R z_c, smoothing): Algorithm 4 (orthonormalisation multigrid) without
 *     its residual-minimisation steps, used here as a symmetric preconditioner
 *   - the smoother: damped block Jacobi, i.e. cell-local dense direct solves with the diagonal
 *     blocks (the per-cell dense solves of Algorithm 1, one-cell blocks of Algorithm 2)
 *   - the coarsest-level direct solve: sec. 3.3 (direct solver with a stored factorisation)
 *   - the Krylov outer method: sec. 3.3 (multigrid as preconditioner of a Krylov solver);
 *     here conjugate gradients, since M is symmetric positive definite (sec. 4)
 *
 * Conventions (all entry points):
 *   - Return value: XDG_OK (0) or an error code below; xdg_strerror() names it and
 *     xdg_last_error() gives the message of the most recent failure on the calling thread.
 *   - Vectors are FP64, block-ordered ([nb][Np], block b holds the Np modal coefficients of
 *     block b). "device" pointers are CUDA global-memory pointers on the handle's device,
 *     owned by the caller; "host" pointers are ordinary host memory owned by the caller.
 *   - Work is enqueued on the handle's stream (the stream given at creation). Entry points
 *     that return results to the host (xdg_solve, xdg_solve_host, xdg_get_info,
 *     xdg_export_level) synchronise that stream before returning; the others are
 *     asynchronous with respect to the host.
 *   - apply / smooth / restrict / prolong / coarse_solve / vcycle / solve allocate no memory:
 *     all work buffers belong to the handle and are allocated by xdg_create_hierarchy.
 *   - There is no CPU fallback: every step of the solve runs in libxdg's CUDA kernels. Calls
 *     fail with XDG_ECUDA when no usable GPU is present.
 *   - A handle is not thread-safe; concurrent calls on one handle must be serialised by the
 *     caller. Different handles are independent.
 *   - Kernels are launched with programmatic dependent launch (each kernel waits for its
 *     predecessor's completion before touching memory, but is dispatched while the
 *     predecessor drains). The environment variable XDG_PDL=0, read once per process, turns it
 *     off; results are bitwise the same either way.
 */
#ifndef XDG_H
#define XDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  XDG_OK = 0,
  XDG_EINVAL = 1,      /* invalid argument, inconsistent sizes or indices, unsupported Np */
  XDG_ECUDA = 2,       /* CUDA runtime error (no device, launch failure, ...) */
  XDG_ENOMEM = 3,      /* device memory allocation failed */
  XDG_ENOTCONV = 4,    /* iteration limit reached; x and info hold the last iterate */
  XDG_EBREAKDOWN = 5,  /* Krylov breakdown (non-positive curvature, non-finite values) or an
                          operator block that is not positive definite */
  XDG_ETIMEOUT = 6     /* the solve exceeded its time budget; x and info hold the last iterate */
};

/* storage precision of the operator blocks used by an apply or an inner solve.
 * XDG_PREC_F64_PAIR (xdg_apply and xdg_kernel_time on level 1 only): the FP64-accurate product
 * computed on the FP32 pipe from a copy of the operator as pairs of FP32 numbers (hi + lo,
 * scaled by a power of two per block) and double-float accumulation within each block, the
 * blocks summed in FP64; error a few units of 2^-48 relative to sum |M||x| per row. It is the
 * outer apply of the mixed-precision solves when xdg_hier_opts.outer_apply selects it. */
enum { XDG_PREC_F64 = 0, XDG_PREC_F32 = 1, XDG_PREC_BF16 = 2, XDG_PREC_F64_PAIR = 3 };

typedef struct xdg_hier* xdg_hier_t;

/* The linear system and its aggregation hierarchy, as host arrays (caller-owned; the library
 * deep-copies them to the device in xdg_create_hierarchy and keeps no reference).
 *   Np          block size (modes per block): 3, 4, 6, 10, 15, 20 (k = 1..3 in 2D and 3D, k = 4
 *               in 2D), with every kernel; 35 or 56 (k = 4, 5 in 3D), FP64 only: low_precision
 *               must be 0 (no FP32 / BF16 cycle, no pair apply, no symmetric storage), and neither
 *               the additive Schwarz smoother nor the learned correction exists for them
 *   n_levels    number of aggregation levels (>= 1); level 1 is the finest
 *   nb[l]       number of blocks on level l+1, l = 0..n_levels-1
 *   row_ptr     int64[nb[0]+1], BSR row pointer of M^1 (row_ptr[0] = 0, non-decreasing)
 *   col         int32[row_ptr[nb[0]]], block column indices, strictly increasing within a
 *               row; every row holds its diagonal block
 *   val         double[row_ptr[nb[0]] * Np * Np], blocks row-major (val[z][r][c])
 *   agg[l]      int32[nb[l]], coarse block (0..nb[l+1]-1) of every level-(l+1) block; every
 *               coarse block has at least one child; l = 0..n_levels-2
 *   R[l]        double[nb[l] * Np * Np]: R_f[m][n] = coefficient of coarse basis function n of
 *               block agg[f] in fine basis function m of block f (Eq. XDGrestrictionMatrix) */
typedef struct {
  int Np;
  int n_levels;
  const int64_t* nb;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  const int32_t* const* agg;
  const double* const* R;
} xdg_problem;

typedef struct {
  double omega;       /* > 0: smoother damping on every level; <= 0: omega_l = 4/(3 lambda_l),
                         lambda_l a Lanczos estimate of the largest eigenvalue of D_l^{-1} M_l */
  int lanczos_steps;  /* Lanczos steps for lambda_l (default 12 when <= 0) */
  int nu;             /* block-Jacobi sweeps before and after the coarse correction (>= 1) */
  int gamma;          /* coarse visits per level: 1 = V-cycle, 2 = W-cycle */
  int low_precision;  /* bit mask: 1 = FP32 copies of operators, block inverses and transfers;
                         2 = BF16 copies of operators and transfers (the cycle then still reads
                         FP32 operators and block inverses, see xdg_cycle) */
  int w_levels;       /* > 0: only the w_levels finest levels repeat their coarse correction
                         gamma times (V-cycle below); <= 0: all levels */
  int split_rows;     /* row mapping of the low-precision cycle kernels: 0 = autotuned per level
                         at creation (one block row per group of Np lanes, or one row per warp
                         with the warp's groups splitting the row, whichever sweeps faster);
                         1 = never split; 2 = split on every level */
  int fused_coarse;   /* low-precision cycle: the V-cycle of the small levels below the W levels
                         (from the first of them with at most 16384 blocks) as one persistent
                         launch: a cooperative grid with grid barriers between its steps, or a
                         single thread-block cluster of 16 (else 8) CTAs with hardware cluster
                         barriers. 0 = the fastest of per-step, grid and cluster launches
                         measured at creation, 1 = never, 2 = always the grid form, 3 = always
                         the cluster form (single problems only; batches launch every step) */
  int outer_apply;    /* operator apply q = M p of the flexible CG around a low-precision cycle:
                         0 = the FP32-pair product (XDG_PREC_F64_PAIR) if it measures faster at
                         creation, 1 = FP64, 2 = FP32 pairs (the FP64 solve uses FP64) */
  int symmetric;      /* level 1 also in symmetric storage (diagonal and right blocks; a left
                         block read as the transpose of its mirror, bitwise the same results,
                         about half the operator streamed from HBM), used by the low-precision
                         level-1 sweep and restriction and by the pair product when the operator
                         is exactly symmetric: 0 = where it measures faster at creation,
                         1 = never, 2 = always */
} xdg_hier_opts;

typedef struct {
  double tol;           /* stop when ||b - M x||_2 <= tol ||b||_2 (FP64 residual) */
  int maxit;            /* iteration limit (outer CG steps, or inner steps in total) */
  int check_every;      /* read the residual norm back every this many iterations (>= 1) */
  int precision;        /* XDG_PREC_F64: CG with the FP64 cycle; F32 / BF16: flexible CG
                           (FP64 residuals, updates and inner products) preconditioned by the
                           low-precision cycle (xdg_cycle) */
  double inner_tol;     /* reserved (ignored) */
  double time_budget_ms;/* > 0: return XDG_ETIMEOUT once exceeded (checked with the residual) */
} xdg_solve_opts;

typedef struct {
  int iterations;      /* CG iterations */
  int outer;           /* 1 (reserved) */
  double relres;       /* final ||b - M x||_2 / ||b||_2, recomputed in FP64 */
  double ms;           /* wall time of the call */
  int status;          /* same as the return value */
  int64_t launches;    /* CUDA kernels launched by the call (graph kernel nodes included) */
} xdg_solve_info;

#define XDG_MAX_LEVELS 24

typedef struct {
  int Np, n_levels;
  int64_t nb[XDG_MAX_LEVELS];
  int64_t nnzb[XDG_MAX_LEVELS];
  double omega[XDG_MAX_LEVELS];
  double lambda_max[XDG_MAX_LEVELS];
  int64_t coarse_n;       /* DOF of the coarsest level (dense direct solve) */
  size_t device_bytes;    /* device memory held by the handle */
  double setup_ms[3];     /* upload+validation, Galerkin products, factorisations+estimates */
  uint64_t split_mask;    /* bit l set: level l+1's low-precision row kernels split rows */
  int fused_level;        /* > 0: the low-precision cycle runs levels fused_level.. in one launch */
  int outer_pair;         /* 1: the mixed-precision solves apply M with FP32 pairs */
  int symmetric;          /* bit 0: symmetric storage of level 1 exists; bit 1: the
                             low-precision cycle reads it; bit 2: the pair product reads it */
  int fused_cluster;      /* > 0: the fused small levels run as one thread-block cluster of
                             this many CTAs (0: grid form or not fused) */
} xdg_hier_info;

/* Build the hierarchy on the current CUDA device: validate every index on the host
 * (EINVAL on the first inconsistency), copy the problem to the device, compute the coarse
 * operators (Galerkin products, Eq. XDGsysRestriction), the Cholesky factors of all diagonal
 * blocks, the damping estimates, the coarsest-level inverse, and record the cycle in a CUDA
 * graph. stream: cudaStream_t to bind to the handle; NULL makes the handle create and own a
 * non-blocking stream (graph capture needs a stream other than the legacy default stream).
 * On success *out owns all device memory of the hierarchy until xdg_destroy. */
int xdg_create_hierarchy(const xdg_problem* p, const xdg_hier_opts* o, void* stream,
                         xdg_hier_t* out);

/* Release all device memory and graphs of the handle (synchronises its stream). */
int xdg_destroy(xdg_hier_t h);

const char* xdg_strerror(int code);
const char* xdg_last_error(void);

/* Sizes and setup results (host struct, synchronises). */
int xdg_get_info(xdg_hier_t h, xdg_hier_info* info);

/* Copy the BSR operator of level `level` (1-based) into caller-allocated host arrays
 * (row_ptr[nb+1], col[nnzb], val[nnzb*Np*Np]; sizes from xdg_get_info). Level 1 returns the
 * uploaded operator, coarser levels the Galerkin products computed on the device. */
int xdg_export_level(xdg_hier_t h, int level, int64_t* row_ptr, int32_t* col, double* val);

/* y = M^level x (device vectors of length nb[level-1]*Np). prec selects the stored operator
 * (XDG_PREC_F64, or F32 / BF16 when built with low_precision; FP32 accumulation then), or
 * XDG_PREC_F64_PAIR on level 1 of a hierarchy that holds the pair copy (xdg_get_info's
 * outer_pair, or outer_apply = 2); x is split into scaled FP32 pairs in the handle's scratch. */
int xdg_apply(xdg_hier_t h, int level, const double* x, double* y, int prec);

/* Test of the bounded waits (no counterpart in the paper): on != 0 makes every grid barrier of
 * the fused small-level cycle (xdg_hier_opts.fused_coarse) wait for one CTA more than the
 * launch has. Each barrier then gives up after its poll limit (about 0.3 s), sets the error
 * word and lets the kernel finish; the solve returns XDG_ETIMEOUT ("a grid barrier timed out")
 * and the context stays usable. on = 0 restores the normal barriers. XDG_EINVAL when the
 * hierarchy runs no fused cycle. Synchronises. */
int xdg_test_barrier_timeout(xdg_hier_t h, int on);

/* r = b - M^level x (FP64, device vectors; r may equal b but not x), Eq. GenericMatrixSystem. */
int xdg_residual(xdg_hier_t h, int level, const double* b, const double* x, double* r);

/* Set the row mapping of the low-precision kernels on `level` (1-based): on != 0 splits each
 * block row over a warp's groups, 0 gives each group its own row (see
 * xdg_hier_opts.split_rows; creation autotunes it). Records the low-precision solve graphs
 * again. For reproducing a mapping, e.g. in a profiler where the autotuner's timings are not
 * representative. */
int xdg_set_split(xdg_hier_t h, int level, int on);

/* Replace the smoother damping of `level` (1 <= level < n_levels) by omega > 0 (default:
 * 4 / (3 lambda_l) from the Lanczos estimate), for every problem of a batch group. Records the
 * handle's solve graphs again (a batch records its own graphs at its next solve only if none
 * exists: change the damping of a batch's groups before its first solve). */
int xdg_set_damping(xdg_hier_t h, int level, double omega);

/* The damping of `level` (1 <= level < n_levels) for problem `problem` of the hierarchy (0 for
 * a single problem; the member index for a batch group), and the Lanczos estimate lambda_max it
 * came from (host outputs, either may be NULL). */
int xdg_get_damping(xdg_hier_t h, int level, int problem, double* omega, double* lambda_max);

/* Additive Schwarz smoother on `level` (1 <= level < n_levels), Algorithm Swz of sec. 3.3
 * ("An additive Schwarz method"), in place of block Jacobi. The caller gives the patches (the
 * sets I_i of the algorithm, here lists of the level's blocks), host arrays: patch i holds the
 * blocks patch_blocks[patch_ptr[i] .. patch_ptr[i+1]-1], strictly ascending, every block of the
 * level in at least one patch; patches may overlap; at most 512 / Np blocks per patch.
 * The block solver is exact: each patch matrix M_{P_i P_i} is factorised (Cholesky, FP64, on
 * the device) and inverted once; patches with bitwise equal matrices share the inverse (two
 * 64-bit hashes of the matrix and its size decide). A smoothing step is then
 *   x_out = x_in + omega S (b - M x_in),
 *   S r = alpha^{-1/2} .* sum_i E_i M_{P_i P_i}^{-1} E_i^T (alpha^{-1/2} .* r),
 * alpha = the number of patches holding each block: the algorithm's overlap scaling x ./ alpha,
 * applied as alpha^{-1/2} on both sides so that the cycle stays symmetric (the two agree when
 * alpha is the same for every block). The FP32 cycles use FP32 copies of the inverses.
 * omega = 4 / (3 lambda_max(S M)) from a Lanczos estimate in the M inner product (or the fixed
 * xdg_hier_opts.omega). Records the solve graphs again; levels at or below the fused small-level
 * cycle (xdg_hier_opts.fused_coarse) then launch step by step. n_patches = 0 restores block
 * Jacobi. Single problems with Np <= 32 only (XDG_EINVAL on a batch group or a wider block).
 * Allocates device memory for the patch data (released with the handle or the next call for
 * the level).
 * Errors: XDG_EINVAL (bad patches), XDG_EBREAKDOWN (a patch matrix not positive definite),
 * XDG_ENOMEM, XDG_ECUDA. */
int xdg_set_schwarz(xdg_hier_t h, int level, int64_t n_patches, const int64_t* patch_ptr,
                    const int32_t* patch_blocks);

typedef struct {
  int64_t n_patches;       /* 0: the level smooths with block Jacobi */
  int64_t n_slots;         /* patch memberships (sum of the patch sizes) */
  int64_t n_distinct;      /* distinct patch matrices (stored inverses) */
  int64_t inverse_entries; /* entries of the stored inverses (FP64, and again in FP32) */
  int max_dof;             /* largest patch (modes) */
  int overlap;             /* 1 when some block lies in more than one patch */
  size_t device_bytes;     /* device memory of the level's Schwarz data */
} xdg_schwarz_info;

int xdg_get_schwarz(xdg_hier_t h, int level, xdg_schwarz_info* info);

/* One damped smoothing step on `level`: x_out = x_in + omega D^{-1} (b - M x_in), the
 * diagonal blocks D solved with their Cholesky factors (block Jacobi), or
 * x_out = x_in + omega S (b - M x_in) on a level with the Schwarz smoother (xdg_set_schwarz).
 * x_in == NULL means x_in = 0. x_out must not alias x_in or b. */
int xdg_smooth(xdg_hier_t h, int level, const double* b, const double* x_in, double* x_out);

/* rc = (R^{X,level})^T (b - M^level x)  (x == NULL: rc = R^T b), level < n_levels. */
int xdg_restrict(xdg_hier_t h, int level, const double* b, const double* x, double* rc);

/* x_out = x_in + R^{X,level} zc  (x_out may equal x_in). */
int xdg_prolong(xdg_hier_t h, int level, const double* zc, const double* x_in, double* x_out);

/* z = (M^{n_levels})^{-1} r on the coarsest level (dense FP64 inverse from a Cholesky
 * factorisation computed on the device). */
int xdg_coarse_solve(xdg_hier_t h, const double* r, double* z);

/* x = B b: one symmetric multigrid cycle from a zero initial guess on level 1 (V- or W-cycle
 * per xdg_hier_opts.gamma). Replayed from the recorded CUDA graph. b and x are device
 * vectors and must not alias. */
int xdg_vcycle(xdg_hier_t h, const double* b, double* x);

/* x = B_prec b: one cycle as xdg_vcycle in low precision (sec. 3.3: single-precision solves
 * inside, double-precision residuals outside): FP32 vectors and FP32 accumulation; level
 * operators and block inverses (computed in FP64) read from their FP32 copies (entries
 * divided by one FP32 scale per block); transfer blocks read from the FP32
 * (prec = XDG_PREC_F32) or BF16 (prec = XDG_PREC_BF16) copy; the coarsest level keeps its
 * FP64 inverse. A BF16-rounded operator is not used inside the cycle: with 2^-9 relative
 * rounding per entry it is indefinite on the smooth modes of these systems
 * (2^-9 cond(M) >> 1). b and x are FP64 device vectors (rounded to FP32 on entry, widened
 * on exit). prec = XDG_PREC_F64 is xdg_vcycle. Needs the copy requested in
 * xdg_hier_opts.low_precision, else XDG_EINVAL. */
int xdg_cycle(xdg_hier_t h, int prec, const double* b, double* x);

/* Solve M^1 x = b (device vectors). x holds the initial guess on entry (resume from a
 * previous x to continue a solve). Returns XDG_OK when converged, XDG_ENOTCONV /
 * XDG_ETIMEOUT / XDG_EBREAKDOWN otherwise; info (optional) is filled in every case.
 * With check_every == 1 and no time budget the whole iteration loop runs on the device (a
 * CUDA graph whose conditional while node is set by the convergence check and bounded by
 * maxit): one launch and one read-back per solve. Otherwise the host launches one recorded
 * iteration graph per step and reads the residual norm every check_every steps. Both run the
 * same kernels with the same arithmetic. The mixed-precision solves apply M with the FP32-pair
 * product when xdg_hier_info.outer_pair is set. */
int xdg_solve(xdg_hier_t h, const double* b, double* x, const xdg_solve_opts* o,
              xdg_solve_info* info);

/* Orthonormalisation multigrid, Algorithm OrthoMG of sec. 3.3 with the residual minimisation of
 * Algorithm ResMinimi: on the finest level, passes of
 *   z = S r (pre-smoother), RM; r_c = R^T r, z_c = MG(0, r_c) on the next level, z = R z_c, RM;
 *   z = S r (post-smoother), RM
 * until ||r||_2 <= tol ||b||_2 or maxit passes. RM(x0, z, W, Z) orthogonalises w = M z against
 * the stored W (two classical Gram-Schmidt sweeps; in exact arithmetic the algorithm's
 * sequential loop), normalises w and z by 1/||w||, appends them and sets x = x0 + Z alpha,
 * r = r0 - W alpha with alpha = W^T r0 (applied one new column at a time), so the residual norm
 * never grows. S is the level's smoother without damping (RM chooses the step): the Schwarz
 * preconditioner of xdg_set_schwarz, else block Jacobi D^{-1}. On a coarser level MG(0, r_c)
 * runs coarse_passes passes from zero with a space of 3 coarse_passes directions (1: one pass
 * per visit; 2: a K-cycle); the coarsest level is solved directly. Readings of the algorithm:
 * the smoothers act on the current residual r (the printed Swz(b) with b fixed would add no new
 * direction), and the finest level keeps at most `restart` directions (then x0 := x,
 * r0 := b - M x recomputed, the space restarts; also when the updated residual meets the
 * tolerance but the recomputed one does not). A numerically dependent direction (||w|| <= 1e-14 ||M z|| after the
 * orthogonalisation) is stored as a zero column and changes nothing. FP64 throughout. b, x
 * device vectors; x holds x0 on entry. Single problems only. Allocates its work space on the
 * first call (restart + 6 passes levels' vectors), records one CUDA graph per pass shape, and
 * reads the residual norm back after every pass. info: iterations = passes. */
typedef struct {
  double tol;              /* stop when ||b - M x||_2 <= tol ||b||_2 */
  int maxit;               /* passes on the finest level */
  int restart;             /* directions kept on the finest level (>= 3; rounded down to a multiple of 3) */
  int coarse_passes;       /* passes per coarse-level visit, 1..4 */
  int smoother_precision;  /* XDG_PREC_F64, or XDG_PREC_F32: the smoothers from the FP32 copies of
                              their inverses (r rounded to FP32, S r widened; everything else FP64) */
} xdg_orthomg_opts;

int xdg_solve_orthomg(xdg_hier_t h, const double* b, double* x, const xdg_orthomg_opts* o,
                      xdg_solve_info* info);

/* p-multigrid on level 1, Algorithm pMultigrid of sec. 3.3, as a preconditioner of GMRES:
 *   x := 0; x[I_lo] := M_lo^{-1} b[I_lo]; r := b - M x; x[I_hi,j] += M_hi,j^{-1} r[I_hi,j] per block,
 * I_lo = the first n_lo modes of every block (the modes are graded by degree: n_lo = C(k_lo+D, D)
 * spans the polynomials of degree <= k_lo), I_hi,j the other modes of block j. The low-order
 * system M_lo (the leading n_lo x n_lo parts of the level-1 blocks) is solved, where the paper
 * uses a sparse direct solver, by this library's own solver on a hierarchy built from M_lo and
 * the leading parts of the transfer blocks (options lo_opts, may be NULL), to the relative
 * residual inner_tol within inner_maxit iterations (inner_precision as xdg_solve_opts.precision);
 * the high-order systems with the inverses of the trailing (Np - n_lo)^2 parts of the diagonal
 * blocks. The printed right-hand side of the high-order solves, b_hi,j, is read as the residual
 * r of the line before. n_lo must be one of 3, 4, 6, 10, 15, 20, 35, smaller than Np, with at
 * most 64 high-order modes (Np - n_lo <= 64).
 * Allocates device memory (the low-order hierarchy, inverses, vectors); a second call replaces
 * the first. Errors: XDG_EINVAL, XDG_EBREAKDOWN (a sub-block not positive definite), ENOMEM,
 * ECUDA. Single problems only. */
int xdg_pmg_setup(xdg_hier_t h, int n_lo, const xdg_hier_opts* lo_opts, double inner_tol, int inner_maxit,
                  int inner_precision);

/* z = PMG(r) (device vectors of level 1, z must not alias r); synchronises (the inner solve
 * reads its residual back). */
int xdg_pmg_apply(xdg_hier_t h, const double* r, double* z);

/* Flexible GMRES(restart) on M x = b (device vectors; x holds x0): right preconditioning by the
 * multigrid cycle (preconditioner 0, precision as xdg_solve_opts.precision: XDG_PREC_F64 the FP64
 * cycle, F32 / BF16 the low-precision one) or by the p-multigrid of xdg_pmg_setup
 * (preconditioner 1). The Krylov basis is orthogonalised with two classical Gram-Schmidt sweeps,
 * the Hessenberg least-squares problem solved with Givens rotations on the device; the residual
 * estimate is read after every step and the true residual recomputed at the end. Flexible (the
 * search directions are kept), so an inexact or changing preconditioner is allowed (Saad 1993).
 * Allocates (restart + 1) + restart vectors on the first call of a restart length; the steps
 * with preconditioner 0 are recorded as CUDA graphs. info: iterations = Arnoldi steps. */
typedef struct {
  double tol;          /* stop when ||b - M x||_2 <= tol ||b||_2 */
  int maxit;           /* Arnoldi steps in total */
  int restart;         /* steps per cycle, 1..200 */
  int preconditioner;  /* 0: multigrid cycle, 1: p-multigrid */
  int precision;       /* cycle precision (preconditioner 0) */
} xdg_gmres_opts;

int xdg_solve_gmres(xdg_hier_t h, const double* b, double* x, const xdg_gmres_opts* o, xdg_solve_info* info);

/* Same as xdg_solve with host vectors: copies b to the device, solves from x = 0 and copies
 * x back, all inside the call (the end-to-end path for callers without device memory). */
int xdg_solve_host(xdg_hier_t h, const double* b_host, double* x_host, const xdg_solve_opts* o,
                   xdg_solve_info* info);

/* Measured fused multiply-add throughput of the current GPU (a utility of the benchmark, no
 * counterpart in the paper): runs 8 independent FMA chains per thread over 8 CTAs of 256
 * threads per SM and stores 2 * FMAs / time in *tflops (FP64 for prec = XDG_PREC_F64, FP32
 * for XDG_PREC_F32). Allocates and frees a small device buffer; synchronises the device.
 * This is the denominator of the FP64 kernels' roofline: on GB300 an FP64 block-sparse
 * apply (0.25 flop/byte) is bound by the FP64 pipe, not by HBM. */
int xdg_fma_peak(int prec, double* tflops);

/* Benchmark utility (no counterpart in the paper): mean duration (*ms, CUDA events on the
 * handle's stream, after 3 warm-up launches, over reps launches; reps <= 0 means 20) of one
 * kernel of the cycle on `level`, and its algorithmic bytes per launch (*bytes: every stored
 * operator, inverse and transfer entry and scale read once, row pointers and columns once, each
 * vector read or written once). which: 0 = operator apply y = M x (the stored copy of
 * precision prec; XDG_PREC_F64_PAIR: the pair product on level 1 from an already split
 * vector), 1 = block-Jacobi sweep from a nonzero guess (level < n_levels),
 * 2 = residual and restriction phase 1, R^T (b - M x) per fine block (level < n_levels).
 * The low-precision sweep and restriction read the FP32 operator (see xdg_cycle), on level 1
 * from the symmetric storage when the cycle uses it (xdg_hier_info.symmetric, bit 1; the bytes
 * then count the compact storage), as does the pair product (bit 2). Uses the level's work
 * vectors (zeroed first); synchronises. */
int xdg_kernel_time(xdg_hier_t h, int which, int level, int prec, int reps, double* ms,
                    double* bytes);

/* ---------------------------------------------------------------------------------------------
 * Batches of independent problems.
 *
 * Each problem is solved exactly as by xdg_solve on its own hierarchy (sec. 3.3: Krylov method
 * preconditioned by the multigrid cycle of Algorithm 4 without residual minimisation; damping,
 * Lanczos estimate and coarsest inverse computed per problem), but all problems run in one
 * CUDA graph launch. Problems with the same Np and the same number of levels form a group; a
 * group is one block-diagonal union hierarchy (the problems' level operators, aggregation maps
 * and transfers concatenated), so every kernel of a cycle covers all problems of the group.
 * Krylov scalars (inner products, step lengths, convergence) are per problem; a problem that
 * has converged takes no further steps while the others continue. The iteration loop of each
 * group is a conditional (while) node of the graph, set on the device by the convergence check
 * and bounded by maxit, so the whole batched solve needs no host round trip. */
typedef struct xdg_batch* xdg_batch_t;

typedef struct {
  int iterations;  /* CG iterations of this problem */
  int status;      /* XDG_OK, XDG_ENOTCONV (maxit reached) or XDG_EBREAKDOWN */
  double relres;   /* ||b - M x||_2 / ||b||_2 of this problem, recomputed in FP64 */
} xdg_batch_result;

typedef struct {
  int n_problems, n_groups;
  int64_t total_dof;           /* length of the concatenated vectors */
  size_t device_bytes;
  double setup_ms;
  int64_t nodes_fixed[3];          /* kernel nodes of a recorded solve outside its loops and */
  int64_t nodes_per_iteration[3];  /* per loop iteration (all groups), by precision; 0 until
                                      the first solve of that precision */
} xdg_batch_info;

/* Build the hierarchies of n problems (layout of each as in xdg_problem; host arrays, deep
 * copied). Every index is validated against the problem's own sizes (EINVAL names the
 * problem). Supported: Np in {6, 10, 15, 20} (another Np: XDG_EINVAL, naming the problem, before
 * any CUDA call), at most 4096 DOF on each problem's coarsest
 * level, at most 65535 problems per group. opts apply to every problem (omega <= 0 gives each
 * problem its own Lanczos-based damping per level). stream: as in xdg_create_hierarchy (all
 * work of the batch is ordered on it). */
int xdg_create_batch(int n, const xdg_problem* probs, const xdg_hier_opts* o, void* stream,
                     xdg_batch_t* out);
int xdg_batch_destroy(xdg_batch_t b);
int xdg_batch_get_info(xdg_batch_t b, xdg_batch_info* info);

/* Group g (0-based, groups numbered by first appearance in the problem list): *h = its union
 * hierarchy (owned by the batch; the single-problem entry points apply to it, on vectors of the
 * group's problems concatenated in member order, and run on the batch's stream),
 * *n_members = number of problems, members[] (optional, n_members entries) = their indices in
 * the caller's list, in the order of the union. */
int xdg_batch_group(xdg_batch_t b, int g, xdg_hier_t* h, int* n_members, int* members);

/* Solve all problems: b and x are device vectors holding every problem's right-hand side and
 * initial guess (solution on return) concatenated in the caller's order (problem i at offset
 * sum_{j<i} nb_j[0] Np_j). o->precision: XDG_PREC_F64 gives CG with the FP64 cycle, F32 /
 * BF16 flexible CG with the low-precision cycle (as xdg_solve). o->tol and o->maxit apply to
 * every problem; check_every and time_budget_ms are not used (the loop runs on the device).
 * The first solve of a precision records its graph (outside any stream capture). info
 * (optional): iterations = largest per-problem count, relres = largest, status = worst,
 * launches = kernel nodes executed. results (optional): n entries. Returns XDG_OK when every
 * problem converged, else XDG_EBREAKDOWN if any broke down, else XDG_ENOTCONV. */
int xdg_solve_batch(xdg_batch_t b, const double* bvec, double* x, const xdg_solve_opts* o,
                    xdg_solve_info* info, xdg_batch_result* results);

/* Same with host vectors: copies b in, solves from x = 0, copies x out, inside the call. */
int xdg_solve_batch_host(xdg_batch_t b, const double* b_host, double* x_host,
                         const xdg_solve_opts* o, xdg_solve_info* info,
                         xdg_batch_result* results);

/* ---------------------------------------------------------------------------------------------
 * Learned cut-cell correction (an extension of the paper's smoothing step, not part of it).
 *
 * The paper's smoothers solve small local systems exactly (cell-local dense solves, Algorithm 1;
 * block Schwarz, sec. 3.3). Here a small network proposes a correction on each "unit" -- the
 * two level-1 blocks that hold the A and B parts of one cut background cell -- from the unit's
 * geometry and its residual after the multigrid cycle. The target is the exact local solve
 * delta* = M_uu^{-1} r_u, which minimises the energy of the true error over corrections on the
 * unit: ||e - delta||_M^2 - ||e||_M^2 = delta^T M_uu delta - 2 delta^T r_u (r = M e). In the
 * solve, a unit's correction is applied (damped by theta) only if this energy change is
 * negative; otherwise the plain cycle's result stands for that unit. With the correction
 * enabled the preconditioner is nonlinear and xdg_solve runs flexible CG in every precision.
 *
 * Network: n_in -> 64 -> 64 -> 64 -> n_out = 2 Np, GELU (x Phi(x)) on the hidden layers.
 * Parameters, FP32, flat and row-major: W1[n_in][64] b1[64] W2[64][64] b2[64] W3[64][64]
 * b3[64] W4[64][n_out] b4[n_out]; a layer computes a_out = act(a_in W + b). Inference in the
 * solve uses a BF16 copy of the parameters (FP32 arithmetic).
 * Coordinates: with X_a = L_a^{-1}, X_b = L_b^{-1} the inverse Cholesky factors of the
 * diagonal blocks M_aa, M_bb (the factors of the block-Jacobi smoother), the unit works on
 * rt = [X_a r_a; X_b r_b] and H = diag(X_a, X_b) M_uu diag(X_a, X_b)^T (identity diagonal
 * blocks), so that its target y* = H^{-1} rt is of order one whatever the scale of M.
 * Inputs of unit u: its geometry features (n_geo floats, given by the caller), then
 * rhat = rt / s with s = ||rt||_2; for output y the correction is delta = s diag(X_a, X_b)^T y
 * (y = rhat is a block-Jacobi step on the unit), and its energy change is
 * s^2 (y^T H y - 2 y^T rhat).
 * Training sample: inputs X, matrix H (FP32), rhat R, and c = rhat^T H^{-1} rhat; loss
 * (y^T H y - 2 y^T rhat) / c (-1 = the exact local solve, 0 = no gain), averaged over the
 * samples. */
typedef struct xdg_mlp* xdg_mlp_t;

typedef struct {
  int epochs;          /* passes over the samples */
  int batch;           /* samples per Adam step */
  float lr;            /* Adam step size */
  float beta1, beta2;  /* Adam moment decay (0: 0.9, 0.999) */
  float eps;           /* Adam epsilon (0: 1e-8) */
  uint64_t seed;       /* shuffling */
} xdg_train_opts;

/* Network with Glorot-uniform weights drawn from a counter-based generator (splitmix64 of
 * seed and entry index) and zero biases; 1 <= n_in, n_out <= 64. stream as in
 * xdg_create_hierarchy. */
int xdg_mlp_create(int n_in, int n_out, uint64_t seed, void* stream, xdg_mlp_t* out);
int xdg_mlp_destroy(xdg_mlp_t m);
int xdg_mlp_num_params(xdg_mlp_t m, int64_t* n);
/* FP32 parameters to / from host memory (n = xdg_mlp_num_params); set resets Adam's state. */
int xdg_mlp_get_params(xdg_mlp_t m, float* host, int64_t n);
int xdg_mlp_set_params(xdg_mlp_t m, const float* host, int64_t n);
/* Y[n][n_out] = network(X[n][n_in]) (device arrays); prec XDG_PREC_F32 or XDG_PREC_BF16
 * (parameters rounded to BF16, FP32 arithmetic). */
int xdg_mlp_forward(xdg_mlp_t m, int prec, int64_t n, const float* X, float* Y);
/* Mean loss over n samples (host *loss) and its gradient (device grad[num_params], optional)
 * with the current parameters. Device arrays: X[n][n_in], uid[n] (row of Mloc of each sample),
 * Mloc[*][n_out][n_out], R[n][n_out], C[n]. */
int xdg_mlp_loss_grad(xdg_mlp_t m, int n, const float* X, const int32_t* uid, const float* Mloc,
                      const float* R, const float* C, double* loss, float* grad);
/* Adam on minibatches of the samples (arrays as in xdg_mlp_loss_grad), reshuffled every epoch;
 * loss_per_epoch (host, optional) receives the mean training loss of each epoch. */
int xdg_mlp_train(xdg_mlp_t m, int n, const float* X, const int32_t* uid, const float* Mloc,
                  const float* R, const float* C, const xdg_train_opts* o, double* loss_per_epoch);

/* Units of the hierarchy's level 1: pairs[u] = (block of the A part, block of the B part) of a
 * cut cell (host int32[n_units][2], distinct blocks), geom = host float[n_units][n_geo]
 * geometry features; n_geo + 2 Np <= 64. Computes the unit matrices and their inverses
 * (EBREAKDOWN if one is not positive definite). Once per hierarchy. */
int xdg_units_setup(xdg_hier_t h, int n_units, const int32_t* pairs, int n_geo, const float* geom);
/* FP32 unit matrices in block-Jacobi coordinates (H above) into device
 * Mloc[n_units][2Np][2Np]. */
int xdg_units_local(xdg_hier_t h, float* Mloc);
/* Training samples of all units from the level-1 right-hand side r (device): z = B r with the
 * plain cycle of precision prec, then per unit, for the residual r - M z: X[u] (inputs),
 * R[u] (rhat) and C[u] (optimal decrease rhat^T H^{-1} rhat); device outputs. */
int xdg_units_samples(xdg_hier_t h, int prec, const double* r, float* X, float* R, float* C);
/* Use network m (a BF16 snapshot of its current parameters) with damping theta > 0 in the
 * preconditioner of xdg_solve; m = NULL switches the correction off. */
int xdg_learned_enable(xdg_hier_t h, xdg_mlp_t m, double theta);
/* One correction step on device vectors: z += theta * (kept corrections) for the residual
 * r - M z; *n_kept (optional, synchronises) = units whose correction was kept. */
int xdg_learned_step(xdg_hier_t h, const double* r, double* z, int* n_kept);

/* Residual restriction for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is an interface variant of xdg_restrict. It serves
 * callers that must not call cudaMalloc -- code running inside a memory pool or arena that
 * owns all device memory, plugins whose host forbids allocations after start-up, and
 * real-time loops where an allocation could block or fail. No handle is needed: the caller
 * passes every array, as device pointers, and the entry point allocates nothing (no
 * cudaMalloc, cudaFree or allocating library call).
 *
 *   rc = R^T (b - M x) for one level (x == NULL: rc = R^T b), with
 *   Np                  block size (3, 4, 6, 10, 15, 20, 35 or 56)
 *   nb_fine, nb_coarse  blocks on the fine and the coarse level
 *   row_ptr, col, val   fine-level BSR operator (layout as in xdg_problem)
 *   R                   double[nb_fine*Np*Np] transfer blocks
 *   child_ptr, child    children of every coarse block: int64[nb_coarse+1] and
 *                       int32[nb_fine]; the children of block C are child[child_ptr[C] ..
 *                       child_ptr[C+1]-1], ascending (the sum over them runs in this order)
 *   b, x                double[nb_fine*Np];  rc  double[nb_coarse*Np]
 *   stream              cudaStream_t the kernels are enqueued on (NULL: legacy stream)
 *
 * The stream and every pointer must belong to the current CUDA device. The entry point cannot
 * see the length of a device array, so the caller guarantees the layout: row_ptr[0] = 0,
 * row_ptr non-decreasing, every col entry < nb_fine, child_ptr[0] = 0 and
 * child_ptr[nb_coarse] = nb_fine, every child index < nb_fine, and every array at least as
 * long as stated above (val: row_ptr[nb_fine]*Np*Np entries). A violation makes the kernels
 * read or write out of bounds; only the sizes below are checked here.
 *
 * Scratch: a fixed device array of XDG_NOALLOC_MAX_ENTRIES doubles (8 MiB) inside the
 * library, holding R_f^T (b_f - M_f x) for every fine block. Every GPU that loads the
 * library holds this array until the process exits. nb_fine*Np above
 * XDG_NOALLOC_MAX_ENTRIES is rejected with XDG_EINVAL before any work is enqueued.
 * All calls share the array and it keeps the last call's contents; each call overwrites
 * every entry it reads, so nothing has to be cleared. Calls whose work overlaps on one GPU
 * (concurrent streams, or host threads without ordering) race on the array and give wrong
 * results: serialise them.
 * The first call on a device looks up the array's device address (once per device, with
 * that device current); make that first call outside any CUDA stream capture.
 * Errors: XDG_EINVAL (null pointer, unsupported Np, size over the maximum), XDG_ECUDA. */
#define XDG_NOALLOC_MAX_ENTRIES (1 << 20)
int xdg_restrict_noalloc(int Np, int64_t nb_fine, int64_t nb_coarse, const int64_t* row_ptr,
                         const int32_t* col, const double* val, const double* R,
                         const int64_t* child_ptr, const int32_t* child, const double* b,
                         const double* x, double* rc, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* XDG_H */
