/*
 * xdg_oracle.c -- plain, slow, FP64 CPU oracle of the XDG multigrid solve.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load this library. The CUDA library never links, calls or includes it, and it
 * includes nothing of the CUDA library.
 *
 * Kummer, Smuda, Weber, "BoSSS: a package for multigrid extended discontinuous Galerkin
 * methods", arXiv 2003.02431. What each function follows:
 *   or_bsr_spmv      the matrix form M^lambda U = b^lambda of the agglomerated system,
 *                    Eq. (GenericMatrixSystem), sec. 3.2 "Agglomeration Algebra"
 *   or_galerkin      M^{lambda+1} = (R^{X,lambda})^T M^lambda R^{X,lambda}, Eq. (XDGsysRestriction)
 *   or_restrict      r_c := (R^{X,lambda})^T r, restriction step of Algorithm 4 (OrthoMG)
 *   or_prolong       z := R^{X,lambda} z_c, prolongation step of Algorithm 4
 *   block Jacobi     per-cell dense direct solves of the blocks M_{I_j,I_j} (the cell-local
 *                    dense solves of Algorithm 1, used as a damped point-block smoother,
 *                    i.e. the one-cell, no-overlap case of the Schwarz blocks of Algorithm 2)
 *   coarse solve     direct solve on the coarsest level (sec. 3.3: sparse direct solver with a
 *                    stored factorisation); here a dense Cholesky factorisation
 *   or_vcycle        the level recursion of Algorithm 4 (pre-smoother, restrict, coarse
 *                    correction, prolong, post-smoother) without the residual-minimisation
 *                    steps: a symmetric V-cycle used as a preconditioner
 *   or_pcg           conjugate gradients preconditioned by the V-cycle (the paper pairs its
 *                    multigrid preconditioners with a Krylov method, sec. 3.3)
 *   lambda_max       Lanczos estimate of the largest eigenvalue of D^{-1} M, used to set the
 *                    smoother damping omega = 4/(3 lambda_max); the paper gives no damping rule.
 *
 * Plain loops only; OpenMP parallelises independent rows, nothing is blocked or fused.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define OR_MAXL 24

/* Threads of the OpenMP loops below (n >= 1); returns the number in use afterwards (1 when the
 * library was built without OpenMP). Lets a caller time the oracle single-threaded. */
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ---------------- operator apply ---------------- */

/* y = A x for a BSR matrix with Np x Np row-major blocks */
void or_bsr_spmv(int64_t nb, int Np, const int64_t* rp, const int32_t* col, const double* val,
                 const double* x, double* y) {
  const int64_t Np2 = (int64_t)Np * Np;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nb; ++i) {
    for (int r = 0; r < Np; ++r) {
      double s = 0.0;
      for (int64_t z = rp[i]; z < rp[i + 1]; ++z) {
        const double* blk = val + z * Np2;
        const double* xj = x + (int64_t)col[z] * Np;
        for (int c = 0; c < Np; ++c) s += blk[r * Np + c] * xj[c];
      }
      y[i * Np + r] = s;
    }
  }
}

/* r = b - A x */
void or_residual(int64_t nb, int Np, const int64_t* rp, const int32_t* col, const double* val,
                 const double* b, const double* x, double* r) {
  or_bsr_spmv(nb, Np, rp, col, val, x, r);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nb * Np; ++i) r[i] = b[i] - r[i];
}

/* ---------------- transfers ---------------- */

/* rc = R^T r : rc[agg[f]] += R_f^T r_f */
void or_restrict(int64_t nbf, int64_t nbc, int Np, const int32_t* agg, const double* R,
                 const double* r, double* rc) {
  const int64_t Np2 = (int64_t)Np * Np;
  memset(rc, 0, sizeof(double) * nbc * Np);
  for (int64_t f = 0; f < nbf; ++f) {
    const double* Rf = R + f * Np2;
    double* o = rc + (int64_t)agg[f] * Np;
    for (int n = 0; n < Np; ++n) {
      double s = 0.0;
      for (int m = 0; m < Np; ++m) s += Rf[m * Np + n] * r[f * Np + m];
      o[n] += s;
    }
  }
}

/* x += R zc : x_f += R_f zc[agg[f]] */
void or_prolong(int64_t nbf, int Np, const int32_t* agg, const double* R, const double* zc,
                double* x) {
  const int64_t Np2 = (int64_t)Np * Np;
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < nbf; ++f) {
    const double* Rf = R + f * Np2;
    const double* z = zc + (int64_t)agg[f] * Np;
    for (int m = 0; m < Np; ++m) {
      double s = 0.0;
      for (int n = 0; n < Np; ++n) s += Rf[m * Np + n] * z[n];
      x[f * Np + m] += s;
    }
  }
}

/* ---------------- Galerkin product ---------------- */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Mc = R^T M R. Output arrays are malloc'ed (release with or_free). Returns 0 on success. */
int or_galerkin(int64_t nbf, int64_t nbc, int Np, const int64_t* rp, const int32_t* col,
                const double* val, const int32_t* agg, const double* R, int64_t** rp_c,
                int32_t** col_c, double** val_c, int64_t* nnz_c) {
  const int64_t Np2 = (int64_t)Np * Np;
  /* children of every coarse block */
  int64_t* cp = (int64_t*)calloc(nbc + 1, sizeof(int64_t));
  int64_t* ch = (int64_t*)malloc(sizeof(int64_t) * (nbf > 0 ? nbf : 1));
  if (!cp || !ch) return -1;
  for (int64_t f = 0; f < nbf; ++f) cp[agg[f] + 1]++;
  for (int64_t I = 0; I < nbc; ++I) cp[I + 1] += cp[I];
  {
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (nbc > 0 ? nbc : 1));
    for (int64_t I = 0; I < nbc; ++I) pos[I] = cp[I];
    for (int64_t f = 0; f < nbf; ++f) ch[pos[agg[f]]++] = f;
    free(pos);
  }
  /* symbolic: coarse columns of every coarse row */
  int64_t* rc = (int64_t*)calloc(nbc + 1, sizeof(int64_t));
  int32_t** cols = (int32_t**)malloc(sizeof(int32_t*) * (nbc > 0 ? nbc : 1));
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t I = 0; I < nbc; ++I) {
    int64_t cnt = 0;
    for (int64_t t = cp[I]; t < cp[I + 1]; ++t) cnt += rp[ch[t] + 1] - rp[ch[t]];
    int32_t* lst = (int32_t*)malloc(sizeof(int32_t) * (cnt > 0 ? cnt : 1));
    int64_t n = 0;
    for (int64_t t = cp[I]; t < cp[I + 1]; ++t)
      for (int64_t z = rp[ch[t]]; z < rp[ch[t] + 1]; ++z) lst[n++] = agg[col[z]];
    qsort(lst, n, sizeof(int32_t), cmp_i32);
    int64_t u = 0;
    for (int64_t q = 0; q < n; ++q)
      if (u == 0 || lst[q] != lst[u - 1]) lst[u++] = lst[q];
    cols[I] = lst;
    rc[I + 1] = u;
  }
  for (int64_t I = 0; I < nbc; ++I) rc[I + 1] += rc[I];
  int64_t nnz = rc[nbc];
  int32_t* cc = (int32_t*)malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  double* vc = (double*)calloc((size_t)(nnz > 0 ? nnz : 1) * Np2, sizeof(double));
  if (!cc || !vc) return -1;
  /* numeric: block (I, J) += R_i^T M_ij R_j */
#pragma omp parallel
  {
    double* tmp = (double*)malloc(sizeof(double) * Np2);
#pragma omp for schedule(dynamic, 64)
    for (int64_t I = 0; I < nbc; ++I) {
      int64_t len = rc[I + 1] - rc[I];
      memcpy(cc + rc[I], cols[I], sizeof(int32_t) * len);
      for (int64_t t = cp[I]; t < cp[I + 1]; ++t) {
        int64_t i = ch[t];
        const double* Ri = R + i * Np2;
        for (int64_t z = rp[i]; z < rp[i + 1]; ++z) {
          int64_t j = col[z];
          const double* Mij = val + z * Np2;
          const double* Rj = R + j * Np2;
          int32_t J = agg[j];
          /* position of J in the row */
          int64_t lo = rc[I], hi = rc[I + 1] - 1;
          while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (cc[mid] < J) lo = mid + 1;
            else hi = mid;
          }
          double* dst = vc + lo * Np2;
          /* tmp = M_ij R_j */
          for (int a = 0; a < Np; ++a)
            for (int n = 0; n < Np; ++n) {
              double s = 0.0;
              for (int b = 0; b < Np; ++b) s += Mij[a * Np + b] * Rj[b * Np + n];
              tmp[a * Np + n] = s;
            }
          /* dst += R_i^T tmp */
          for (int m = 0; m < Np; ++m)
            for (int n = 0; n < Np; ++n) {
              double s = 0.0;
              for (int a = 0; a < Np; ++a) s += Ri[a * Np + m] * tmp[a * Np + n];
              dst[m * Np + n] += s;
            }
        }
      }
    }
    free(tmp);
  }
  for (int64_t I = 0; I < nbc; ++I) free(cols[I]);
  free(cols);
  free(cp);
  free(ch);
  *rp_c = rc;
  *col_c = cc;
  *val_c = vc;
  *nnz_c = nnz;
  return 0;
}

void or_free(void* p) { free(p); }

/* ---------------- dense helpers ---------------- */

/* in-place Cholesky (lower) of an n x n row-major matrix; returns 0 if SPD */
static int chol(int64_t n, double* A) {
  for (int64_t j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int64_t p = 0; p < j; ++p) s -= A[j * n + p] * A[j * n + p];
    if (!(s > 0.0)) return -1;
    double d = sqrt(s);
    A[j * n + j] = d;
    for (int64_t i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int64_t p = 0; p < j; ++p) t -= A[i * n + p] * A[j * n + p];
      A[i * n + j] = t / d;
    }
  }
  return 0;
}

/* x = (L L^T)^{-1} b */
static void chol_solve(int64_t n, const double* L, const double* b, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int64_t p = 0; p < i; ++p) s -= L[i * n + p] * x[p];
    x[i] = s / L[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int64_t p = i + 1; p < n; ++p) s -= L[p * n + i] * x[p];
    x[i] = s / L[i * n + i];
  }
}

/* ---------------- hierarchy ---------------- */

typedef struct {
  int64_t nb;
  int64_t* rp;
  int32_t* col;
  double* val;
  int owns;          /* rp/col/val allocated here (coarse levels) */
  double* Dchol;     /* Cholesky factors of the diagonal blocks */
  double lmax, omega;
  const int32_t* agg; /* to the next level */
  const double* R;
  double* w[4];      /* work vectors */
  /* additive Schwarz smoother (Algorithm Swz); npatch = 0: block Jacobi */
  int64_t npatch;
  int64_t* pptr;     /* patch i = blocks pblk[pptr[i] .. pptr[i+1]-1] */
  int32_t* pblk;
  int64_t* poff;     /* offset of patch i's Cholesky factor in pchol */
  double* pchol;     /* dense Cholesky factor of M restricted to each patch */
  double* pscale;    /* per block: 1/alpha (mode 0) or 1/sqrt(alpha) (mode 1) */
  int pmode;         /* 0: x ./ alpha after the sum; 1: alpha^{-1/2} on both sides */
} or_level;

typedef struct {
  int Np, nlev, nu, gamma;
  int wlev; /* levels l < wlev repeat their coarse correction gamma times */
  or_level L[OR_MAXL];
  double* cchol; /* dense Cholesky factor of the coarsest operator */
  int64_t nc;
  double* pv[5]; /* PCG vectors */
} or_hier;

/* a . b as contiguous chunks, one per thread, whose sums are added in thread order: a fixed
   order at a given thread count, so that a result repeats from run to run (an OpenMP reduction
   combines its partial sums in an unspecified order) */
#define OR_MAX_CHUNKS 512
static double dot(int64_t n, const double* a, const double* b) {
  double part[OR_MAX_CHUNKS];
  int nchunk = 1;
#ifdef _OPENMP
  nchunk = omp_get_max_threads();
  if (nchunk > OR_MAX_CHUNKS) nchunk = OR_MAX_CHUNKS;
#endif
#pragma omp parallel for schedule(static, 1) num_threads(nchunk)
  for (int c = 0; c < nchunk; ++c) {
    const int64_t i0 = n * c / nchunk, i1 = n * (c + 1) / nchunk;
    double s = 0.0;
    for (int64_t i = i0; i < i1; ++i) s += a[i] * b[i];
    part[c] = s;
  }
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[c];
  return s;
}

/* z_b = D_b^{-1} r_b for every block */
static void bj_apply(const or_level* L, int Np, const double* r, double* z) {
  const int64_t Np2 = (int64_t)Np * Np;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < L->nb; ++i) chol_solve(Np, L->Dchol + i * Np2, r + i * Np, z + i * Np);
}

/* dense M_{PP} of the blocks blk[0..n-1] of a level (row-major, (n Np)^2) */
static void gather_patch(const or_level* L, int Np, int64_t n, const int32_t* blk, double* A) {
  const int64_t m = n * Np, Np2 = (int64_t)Np * Np;
  memset(A, 0, sizeof(double) * m * m);
  for (int64_t a = 0; a < n; ++a) {
    const int64_t i = blk[a];
    for (int64_t z = L->rp[i]; z < L->rp[i + 1]; ++z)
      for (int64_t c = 0; c < n; ++c)
        if (L->col[z] == blk[c])
          for (int r = 0; r < Np; ++r)
            for (int q = 0; q < Np; ++q) A[(a * Np + r) * m + c * Np + q] = L->val[z * Np2 + r * Np + q];
  }
}

/* Additive Schwarz (Algorithm Swz) with exact block solves on the patches P_i (PMG with every
 * mode in the low-order set is the direct solve of M_{P_i P_i}):
 *   mode 0 (the algorithm as printed): z = (sum_i E_i M_ii^{-1} E_i^T r) ./ alpha,
 *   mode 1 (symmetric): z = alpha^{-1/2} .* sum_i E_i M_ii^{-1} E_i^T (alpha^{-1/2} .* r),
 * alpha = number of patches holding each block. The two agree when alpha is constant. */
static void swz_apply(const or_level* L, int Np, const double* r, double* z) {
  const int64_t n = L->nb * Np;
  double* rs = (double*)malloc(sizeof(double) * n);
  for (int64_t i = 0; i < n; ++i) {
    z[i] = 0.0;
    rs[i] = L->pmode ? L->pscale[i / Np] * r[i] : r[i];
  }
  for (int64_t p = 0; p < L->npatch; ++p) {
    const int64_t nbp = L->pptr[p + 1] - L->pptr[p], m = nbp * Np;
    const int32_t* blk = L->pblk + L->pptr[p];
    double* rp = (double*)malloc(sizeof(double) * m);
    double* xp = (double*)malloc(sizeof(double) * m);
    for (int64_t a = 0; a < nbp; ++a)
      for (int q = 0; q < Np; ++q) rp[a * Np + q] = rs[(int64_t)blk[a] * Np + q];
    chol_solve(m, L->pchol + L->poff[p], rp, xp);
    for (int64_t a = 0; a < nbp; ++a)
      for (int q = 0; q < Np; ++q) z[(int64_t)blk[a] * Np + q] += xp[a * Np + q];
    free(rp);
    free(xp);
  }
  for (int64_t i = 0; i < n; ++i) z[i] *= L->pscale[i / Np];
  free(rs);
}

/* the level's smoother preconditioner: block Jacobi or additive Schwarz */
static void smoother_apply(const or_level* L, int Np, const double* r, double* z) {
  if (L->npatch > 0) swz_apply(L, Np, r, z);
  else bj_apply(L, Np, r, z);
}

/* Counter-based start vector for the Lanczos estimate (Knuth multiplicative hash):
 * v_i = (((i+1) * 2654435761) mod 2^32) / 2^32 - 0.5 */
static double start_entry(int64_t i) {
  uint32_t h = (uint32_t)((uint64_t)(i + 1) * 2654435761ull);
  return (double)h / 4294967296.0 - 0.5;
}

/* largest eigenvalue of a symmetric tridiagonal matrix (bisection on Sturm counts) */
static double tridiag_max(int m, const double* a, const double* b) {
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
    if (a[i] - r < lo) lo = a[i] - r;
    if (a[i] + r > hi) hi = a[i] + r;
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    /* number of eigenvalues < mid */
    int cnt = 0;
    double q = a[0] - mid;
    if (q < 0) cnt++;
    for (int i = 1; i < m; ++i) {
      if (q == 0.0) q = 1e-300;
      q = a[i] - mid - b[i - 1] * b[i - 1] / q;
      if (q < 0) cnt++;
    }
    if (cnt >= m) hi = mid;
    else lo = mid;
    if (hi - lo <= 1e-15 * fabs(hi)) break;
  }
  return hi;
}

/* m-step Lanczos in the D inner product for the pencil (M, D) */
static double lambda_max(or_level* L, int Np, int m) {
  const int64_t n = L->nb * Np, Np2 = (int64_t)Np * Np;
  double* q = (double*)calloc(n, sizeof(double));
  double* qp = (double*)calloc(n, sizeof(double));
  double* u = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* Dw = (double*)malloc(sizeof(double) * n);
  double al[64], be[64];
  for (int64_t i = 0; i < n; ++i) q[i] = start_entry(i);
  /* D q: D_b = L_b L_b^T */
  for (int64_t b = 0; b < L->nb; ++b) {
    const double* Lc = L->Dchol + b * Np2;
    for (int r = 0; r < Np; ++r) {
      double s = 0.0;
      for (int c = 0; c < Np; ++c) {
        double d = 0.0; /* (L L^T)_{rc} */
        for (int p = 0; p <= (r < c ? r : c); ++p) d += Lc[r * Np + p] * Lc[c * Np + p];
        s += d * q[b * Np + c];
      }
      Dw[b * Np + r] = s;
    }
  }
  double nrm = sqrt(dot(n, q, Dw));
  for (int64_t i = 0; i < n; ++i) q[i] /= nrm;
  double bprev = 0.0;
  int steps = 0;
  for (int j = 0; j < m; ++j) {
    or_bsr_spmv(L->nb, Np, L->rp, L->col, L->val, q, u);
    al[j] = dot(n, q, u);
    bj_apply(L, Np, u, w);
    for (int64_t i = 0; i < n; ++i) w[i] -= al[j] * q[i] + bprev * qp[i];
    for (int64_t b = 0; b < L->nb; ++b) {
      const double* Lc = L->Dchol + b * Np2;
      for (int r = 0; r < Np; ++r) {
        double s = 0.0;
        for (int c = 0; c < Np; ++c) {
          double d = 0.0;
          for (int p = 0; p <= (r < c ? r : c); ++p) d += Lc[r * Np + p] * Lc[c * Np + p];
          s += d * w[b * Np + c];
        }
        Dw[b * Np + r] = s;
      }
    }
    steps = j + 1;
    double bj = sqrt(dot(n, w, Dw));
    be[j] = bj;
    if (!(bj > 1e-300)) break;
    for (int64_t i = 0; i < n; ++i) {
      qp[i] = q[i];
      q[i] = w[i] / bj;
    }
    bprev = bj;
  }
  double lm = tridiag_max(steps, al, be);
  free(q);
  free(qp);
  free(u);
  free(w);
  free(Dw);
  return lm;
}

/* m-step Lanczos for the largest eigenvalue of S M with S the symmetric Schwarz preconditioner
 * (S M is self-adjoint in the M inner product; one product with M and one application of S per
 * step). Same start vector as the block-Jacobi estimate. */
static double lambda_max_swz(or_level* L, int Np, int m) {
  const int64_t n = L->nb * Np;
  double* q = (double*)calloc(n, sizeof(double));
  double* qp = (double*)calloc(n, sizeof(double));
  double* u = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* v = (double*)malloc(sizeof(double) * n);
  double al[64], be[64];
  for (int64_t i = 0; i < n; ++i) q[i] = start_entry(i);
  or_bsr_spmv(L->nb, Np, L->rp, L->col, L->val, q, u);
  double nrm = sqrt(dot(n, q, u));
  for (int64_t i = 0; i < n; ++i) {
    q[i] /= nrm;
    u[i] /= nrm;
  }
  double bprev = 0.0;
  int steps = 0;
  for (int j = 0; j < m; ++j) {
    swz_apply(L, Np, u, w); /* w = S M q */
    al[j] = dot(n, u, w);   /* <q, S M q>_M */
    for (int64_t i = 0; i < n; ++i) w[i] -= al[j] * q[i] + bprev * qp[i];
    or_bsr_spmv(L->nb, Np, L->rp, L->col, L->val, w, v);
    steps = j + 1;
    double bj = sqrt(dot(n, w, v));
    be[j] = bj;
    if (!(bj > 1e-300)) break;
    for (int64_t i = 0; i < n; ++i) {
      qp[i] = q[i];
      q[i] = w[i] / bj;
      u[i] = v[i] / bj;
    }
    bprev = bj;
  }
  double lm = tridiag_max(steps, al, be);
  free(q);
  free(qp);
  free(u);
  free(w);
  free(v);
  return lm;
}

/* Build the hierarchy: level-1 operator plus per-level (agg, R). All input arrays must stay
 * alive while the hierarchy exists. omega > 0 fixes the damping on every level; otherwise
 * omega_l = 4/(3 lambda_max(D^{-1} M^l)) from lanczos_steps Lanczos steps.
 * Returns NULL on failure (not SPD). */
void* or_hier_create(int nlev, int Np, int64_t nb1, const int64_t* rp, const int32_t* col,
                     const double* val, const int64_t* nbs, const int32_t* const* aggs,
                     const double* const* Rs, double omega, int lanczos_steps, int nu,
                     int gamma) {
  if (nlev < 1 || nlev > OR_MAXL) return NULL;
  or_hier* H = (or_hier*)calloc(1, sizeof(or_hier));
  H->Np = Np;
  H->nlev = nlev;
  H->nu = nu < 1 ? 1 : nu;
  H->gamma = gamma < 1 ? 1 : gamma;
  H->wlev = OR_MAXL;
  const int64_t Np2 = (int64_t)Np * Np;
  H->L[0].nb = nb1;
  H->L[0].rp = (int64_t*)rp;
  H->L[0].col = (int32_t*)col;
  H->L[0].val = (double*)val;
  for (int l = 0; l < nlev; ++l) {
    or_level* L = &H->L[l];
    if (l > 0) {
      int64_t nnz;
      if (or_galerkin(H->L[l - 1].nb, nbs[l], Np, H->L[l - 1].rp, H->L[l - 1].col,
                      H->L[l - 1].val, aggs[l - 1], Rs[l - 1], &L->rp, &L->col, &L->val, &nnz))
        return NULL;
      L->nb = nbs[l];
      L->owns = 1;
    }
    if (l + 1 < nlev) {
      L->agg = aggs[l];
      L->R = Rs[l];
    }
    for (int t = 0; t < 4; ++t) L->w[t] = (double*)calloc(L->nb * Np, sizeof(double));
    if (l + 1 < nlev) {
      L->Dchol = (double*)malloc(sizeof(double) * L->nb * Np2);
      int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
      for (int64_t i = 0; i < L->nb; ++i) {
        double* Dc = L->Dchol + i * Np2;
        int64_t z = L->rp[i];
        while (z < L->rp[i + 1] && L->col[z] != i) ++z;
        if (z == L->rp[i + 1]) {
          bad |= 1;
          continue;
        }
        memcpy(Dc, L->val + z * Np2, sizeof(double) * Np2);
        if (chol(Np, Dc)) bad |= 1;
      }
      if (bad) return NULL;
      L->lmax = lambda_max(L, Np, lanczos_steps);
      L->omega = omega > 0 ? omega : 4.0 / (3.0 * L->lmax);
    }
  }
  /* coarsest level: dense Cholesky */
  or_level* C = &H->L[nlev - 1];
  H->nc = C->nb * Np;
  H->cchol = (double*)calloc((size_t)H->nc * H->nc, sizeof(double));
  for (int64_t i = 0; i < C->nb; ++i)
    for (int64_t z = C->rp[i]; z < C->rp[i + 1]; ++z)
      for (int r = 0; r < Np; ++r)
        for (int c = 0; c < Np; ++c)
          H->cchol[(i * Np + r) * H->nc + (int64_t)C->col[z] * Np + c] = C->val[z * Np2 + r * Np + c];
  if (chol(H->nc, H->cchol)) return NULL;
  for (int t = 0; t < 5; ++t) H->pv[t] = (double*)calloc(nb1 * Np, sizeof(double));
  return H;
}

void or_hier_free(void* h) {
  or_hier* H = (or_hier*)h;
  if (!H) return;
  for (int l = 0; l < H->nlev; ++l) {
    or_level* L = &H->L[l];
    if (L->owns) {
      free(L->rp);
      free(L->col);
      free(L->val);
    }
    free(L->Dchol);
    for (int t = 0; t < 4; ++t) free(L->w[t]);
    free(L->pptr);
    free(L->pblk);
    free(L->poff);
    free(L->pchol);
    free(L->pscale);
  }
  free(H->cchol);
  for (int t = 0; t < 5; ++t) free(H->pv[t]);
  free(H);
}

/* level information: nb, nnzb, omega, lambda_max; pointers to the level's BSR arrays */
int or_hier_level(void* h, int l, int64_t* nb, int64_t* nnzb, double* omega, double* lmax,
                  const int64_t** rp, const int32_t** col, const double** val) {
  or_hier* H = (or_hier*)h;
  if (l < 0 || l >= H->nlev) return -1;
  or_level* L = &H->L[l];
  *nb = L->nb;
  *nnzb = L->rp[L->nb];
  *omega = L->omega;
  *lmax = L->lmax;
  *rp = L->rp;
  *col = L->col;
  *val = L->val;
  return 0;
}

/* one damped smoothing step on level l: x += omega S (b - M x), S = D^{-1} (block Jacobi) or
 * the additive Schwarz preconditioner when the level has patches */
void or_smooth(void* h, int l, const double* b, double* x) {
  or_hier* H = (or_hier*)h;
  or_level* L = &H->L[l];
  const int Np = H->Np;
  const int64_t n = L->nb * Np;
  or_residual(L->nb, Np, L->rp, L->col, L->val, b, x, L->w[2]);
  smoother_apply(L, Np, L->w[2], L->w[3]);
  for (int64_t i = 0; i < n; ++i) x[i] += L->omega * L->w[3][i];
}

/* z = M_coarsest^{-1} r */
void or_coarse_solve(void* h, const double* r, double* z) {
  or_hier* H = (or_hier*)h;
  chol_solve(H->nc, H->cchol, r, z);
}

static void vcycle_rec(or_hier* H, int l, const double* b, double* x) {
  const int Np = H->Np;
  or_level* L = &H->L[l];
  const int64_t n = L->nb * Np;
  if (l == H->nlev - 1) {
    chol_solve(H->nc, H->cchol, b, x);
    return;
  }
  /* pre-smoothing from x = 0 */
  smoother_apply(L, Np, b, x);
  for (int64_t i = 0; i < n; ++i) x[i] *= L->omega;
  for (int s = 1; s < H->nu; ++s) or_smooth(H, l, b, x);
  /* restrict the residual */
  double* r = L->w[0];
  or_residual(L->nb, Np, L->rp, L->col, L->val, b, x, r);
  or_level* Lc = &H->L[l + 1];
  double* bc = (double*)malloc(sizeof(double) * Lc->nb * Np);
  double* zc = (double*)malloc(sizeof(double) * Lc->nb * Np);
  or_restrict(L->nb, Lc->nb, Np, L->agg, L->R, r, bc);
  /* coarse-grid correction: gamma steps of the coarse cycle from zero (gamma = 1: V-cycle,
   * gamma = 2: W-cycle); each step z_c += B_c (r_c - M_c z_c) keeps the cycle symmetric */
  vcycle_rec(H, l + 1, bc, zc);
  if (H->gamma > 1 && l + 2 < H->nlev && l < H->wlev) {
    double* rc2 = (double*)malloc(sizeof(double) * Lc->nb * Np);
    double* dz = (double*)malloc(sizeof(double) * Lc->nb * Np);
    for (int g = 1; g < H->gamma; ++g) {
      or_residual(Lc->nb, Np, Lc->rp, Lc->col, Lc->val, bc, zc, rc2);
      vcycle_rec(H, l + 1, rc2, dz);
      for (int64_t i = 0; i < Lc->nb * Np; ++i) zc[i] += dz[i];
    }
    free(rc2);
    free(dz);
  }
  or_prolong(L->nb, Np, L->agg, L->R, zc, x);
  free(zc);
  free(bc);
  /* post-smoothing */
  for (int s = 0; s < H->nu; ++s) or_smooth(H, l, b, x);
}

/* x = B b, one symmetric V-cycle from a zero initial guess */
void or_vcycle(void* h, const double* b, double* x) { vcycle_rec((or_hier*)h, 0, b, x); }

/* PCG on level 1 with the V-cycle preconditioner. x holds the initial guess on entry.
 * Stops when ||r||_2 <= tol ||b||_2 (recursive residual) or after maxit iterations.
 * hist (optional, maxit+1 entries) receives ||r||/||b|| per iteration.
 * Returns the number of iterations; *relres is the true final relative residual. */
int or_pcg(void* h, const double* b, double* x, double tol, int maxit, double* relres,
           double* hist) {
  or_hier* H = (or_hier*)h;
  or_level* L = &H->L[0];
  const int Np = H->Np;
  const int64_t n = L->nb * Np;
  double *r = H->pv[0], *z = H->pv[1], *p = H->pv[2], *q = H->pv[3];
  or_residual(L->nb, Np, L->rp, L->col, L->val, b, x, r);
  double bn = sqrt(dot(n, b, b));
  if (bn == 0.0) bn = 1.0;
  double rn = sqrt(dot(n, r, r));
  if (hist) hist[0] = rn / bn;
  int it = 0;
  if (rn / bn > tol) {
    or_vcycle(H, r, z);
    memcpy(p, z, sizeof(double) * n);
    double rho = dot(n, r, z);
    for (it = 1; it <= maxit; ++it) {
      or_bsr_spmv(L->nb, Np, L->rp, L->col, L->val, p, q);
      double alpha = rho / dot(n, p, q);
      for (int64_t i = 0; i < n; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      rn = sqrt(dot(n, r, r));
      if (hist) hist[it] = rn / bn;
      if (rn / bn <= tol) break;
      or_vcycle(H, r, z);
      double rho2 = dot(n, r, z);
      double beta = rho2 / rho;
      rho = rho2;
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (it > maxit) it = maxit;
  }
  or_residual(L->nb, Np, L->rp, L->col, L->val, b, x, r);
  *relres = sqrt(dot(n, r, r)) / bn;
  return it;
}

/* ---------------- low-precision block storage ---------------- */

/* Round a float to the nearest bfloat16 (ties to even) and widen it back: keep the upper 16
 * bits of the IEEE-754 single after adding half an ulp of bfloat16 plus the tie bit. */
static float bf16_round(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

/* Stored form of Np x Np blocks for the low-precision cycle: s = max |entry| rounded to float
 * (1 for a zero block), stored entry = entry / s rounded to float (prec 1) or to bfloat16
 * through float (prec 2). out receives s * stored in FP64, scales receives s. */
void or_quantize_blocks(int64_t nblk, int np2, int prec, const double* in, double* out, float* scales) {
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblk; ++b) {
    const double* a = in + b * np2;
    double m = 0.0;
    for (int e = 0; e < np2; ++e) m = fabs(a[e]) > m ? fabs(a[e]) : m;
    float s = m > 0.0 ? (float)m : 1.0f;
    scales[b] = s;
    for (int e = 0; e < np2; ++e) {
      float q = (float)(a[e] / (double)s);
      if (prec == 2) q = bf16_round(q);
      out[b * np2 + e] = (double)s * (double)q;
    }
  }
}

/* restrict the repeated coarse corrections to levels l < wlev (V-cycle below) */
void or_hier_set_wlev(void* h, int wlev) { ((or_hier*)h)->wlev = wlev; }

/* Additive Schwarz smoother on level l (Algorithm Swz, exact patch solves): patch i holds the
 * blocks pblk[pptr[i] .. pptr[i+1]-1] (every block of the level in at least one patch). The
 * dense matrices M_{P_i P_i} are factorised (Cholesky), alpha counted per block, and the damping
 * re-estimated: omega = 4/(3 lambda_max(S M)) with S in its symmetric form, unless the
 * hierarchy was built with a fixed omega. mode 0: x ./ alpha as printed; mode 1: alpha^{-1/2} on
 * both sides (a symmetric smoother, as CG needs). npatch = 0 restores block Jacobi.
 * Returns 0, -1 on invalid patches, -2 if a patch matrix is not positive definite. */
int or_hier_set_patches(void* h, int l, int64_t npatch, const int64_t* pptr, const int32_t* pblk, int mode,
                        int lanczos_steps, double omega_fixed) {
  or_hier* H = (or_hier*)h;
  if (l < 0 || l >= H->nlev - 1) return -1;
  or_level* L = &H->L[l];
  const int Np = H->Np;
  free(L->pptr);
  free(L->pblk);
  free(L->poff);
  free(L->pchol);
  free(L->pscale);
  L->pptr = NULL;
  L->pblk = NULL;
  L->poff = NULL;
  L->pchol = NULL;
  L->pscale = NULL;
  L->npatch = 0;
  if (npatch > 0) {
    const int64_t tot = pptr[npatch];
    int* cnt = (int*)calloc(L->nb, sizeof(int));
    for (int64_t k = 0; k < tot; ++k) {
      if (pblk[k] < 0 || pblk[k] >= L->nb) {
        free(cnt);
        return -1;
      }
      cnt[pblk[k]]++;
    }
    for (int64_t i = 0; i < L->nb; ++i)
      if (cnt[i] == 0) {
        free(cnt);
        return -1;
      }
    L->pptr = (int64_t*)malloc(sizeof(int64_t) * (npatch + 1));
    L->pblk = (int32_t*)malloc(sizeof(int32_t) * (tot > 0 ? tot : 1));
    L->poff = (int64_t*)malloc(sizeof(int64_t) * (npatch + 1));
    memcpy(L->pptr, pptr, sizeof(int64_t) * (npatch + 1));
    memcpy(L->pblk, pblk, sizeof(int32_t) * tot);
    L->poff[0] = 0;
    for (int64_t p = 0; p < npatch; ++p) {
      const int64_t m = (pptr[p + 1] - pptr[p]) * Np;
      L->poff[p + 1] = L->poff[p] + m * m;
    }
    L->pchol = (double*)malloc(sizeof(double) * (L->poff[npatch] > 0 ? L->poff[npatch] : 1));
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (int64_t p = 0; p < npatch; ++p) {
      const int64_t nbp = pptr[p + 1] - pptr[p];
      double* A = L->pchol + L->poff[p];
      gather_patch(L, Np, nbp, pblk + pptr[p], A);
      if (chol(nbp * Np, A)) bad |= 1;
    }
    L->pscale = (double*)malloc(sizeof(double) * L->nb);
    for (int64_t i = 0; i < L->nb; ++i) L->pscale[i] = 1.0 / sqrt((double)cnt[i]);
    free(cnt);
    L->npatch = npatch;
    L->pmode = 1;
    if (bad) return -2;
    L->lmax = lambda_max_swz(L, Np, lanczos_steps);
    if (mode == 0)
      for (int64_t i = 0; i < L->nb; ++i) L->pscale[i] *= L->pscale[i];
    L->pmode = mode;
  } else {
    L->lmax = lambda_max(L, Np, lanczos_steps);
  }
  L->omega = omega_fixed > 0 ? omega_fixed : 4.0 / (3.0 * L->lmax);
  return 0;
}

/* z = Swz(r) on level l with the patches of or_hier_set_patches (undamped) */
void or_schwarz(void* h, int l, const double* r, double* z) {
  or_hier* H = (or_hier*)h;
  swz_apply(&H->L[l], H->Np, r, z);
}

/* ---------------- orthonormalisation multigrid (Algorithms ResMinimi and OrthoMG) ---------------- */

/* Search space of a residual minimisation on one level: Z = (z_1..z_l), W = M Z with orthonormal
 * columns, and the coefficients alpha_i = w_i . r_0. */
typedef struct {
  int64_t n;
  int cap, l;
  double *W, *Z, *alpha;
} or_rm_space;

static void rm_init(or_rm_space* S, int64_t n, int cap) {
  S->n = n;
  S->cap = cap;
  S->l = 0;
  S->W = (double*)malloc(sizeof(double) * n * cap);
  S->Z = (double*)malloc(sizeof(double) * n * cap);
  S->alpha = (double*)malloc(sizeof(double) * cap);
}

static void rm_free(or_rm_space* S) {
  free(S->W);
  free(S->Z);
  free(S->alpha);
}

/* Algorithm ResMinimi: (x, r) = RM(x0, z, W, Z) on level `lev`. z is overwritten. The new
 * direction w = M z is orthogonalised against the columns of W one after another (the loop of
 * the algorithm: beta from the partly orthogonalised w), z follows with the same coefficients,
 * both are normalised by gamma = 1/|w| and appended; alpha_{l+1} = w . r0; then
 * x = x0 + Z alpha and r = r0 - W alpha. A direction that is numerically dependent on W
 * (|w| <= 1e-14 |M z| after the loop; the algorithm leaves this case open) is appended as a
 * zero column with alpha 0, which leaves x and r unchanged. */
static void rm_step(or_hier* H, int lev, or_rm_space* S, const double* x0, const double* r0, double* z,
                    double* x, double* r) {
  or_level* L = &H->L[lev];
  const int Np = H->Np;
  const int64_t n = S->n;
  if (S->l >= S->cap) return;
  double* w = S->W + (int64_t)S->l * n;
  or_bsr_spmv(L->nb, Np, L->rp, L->col, L->val, z, w);
  const double w0 = sqrt(dot(n, w, w));
  for (int i = 0; i < S->l; ++i) {
    const double* wi = S->W + (int64_t)i * n;
    const double* zi = S->Z + (int64_t)i * n;
    const double beta = dot(n, wi, w);
    for (int64_t k = 0; k < n; ++k) {
      w[k] -= beta * wi[k];
      z[k] -= beta * zi[k];
    }
  }
  const double nw = sqrt(dot(n, w, w));
  const double gamma = (nw > 1e-14 * w0) ? 1.0 / nw : 0.0;
  double* zn = S->Z + (int64_t)S->l * n;
  for (int64_t k = 0; k < n; ++k) {
    w[k] *= gamma;
    zn[k] = gamma * z[k];
  }
  S->alpha[S->l] = dot(n, w, r0);
  S->l++;
  for (int64_t k = 0; k < n; ++k) {
    double xs = x0[k], rs = r0[k];
    for (int i = 0; i < S->l; ++i) {
      xs += S->Z[(int64_t)i * n + k] * S->alpha[i];
      rs -= S->W[(int64_t)i * n + k] * S->alpha[i];
    }
    x[k] = xs;
    r[k] = rs;
  }
}

/* the smoother of Algorithm OrthoMG on a level: Swz (patches) or block Jacobi, undamped (the
 * residual minimisation picks the step length) */
static void omg_smoother(or_hier* H, int lev, const double* r, double* z) {
  smoother_apply(&H->L[lev], H->Np, r, z);
}

static int g_omg_passes = 1; /* passes of Algorithm OrthoMG on every coarse level */

/* Algorithm OrthoMG on a coarse level (x0 = 0, right-hand side b): `g_omg_passes` passes of
 * pre-smoother, RM, restriction, MG on the next level, prolongation, RM, post-smoother, RM, one
 * search space for all of them. On the coarsest level: the direct solve. x receives the result. */
static void omg_level(or_hier* H, int lev, const double* b, double* x) {
  const int Np = H->Np;
  or_level* L = &H->L[lev];
  const int64_t n = L->nb * Np;
  if (lev == H->nlev - 1) {
    chol_solve(H->nc, H->cchol, b, x);
    return;
  }
  or_level* C = &H->L[lev + 1];
  const int64_t nc = C->nb * Np;
  or_rm_space S;
  rm_init(&S, n, 3 * g_omg_passes);
  double* x0 = (double*)calloc(n, sizeof(double));
  double* r = (double*)malloc(sizeof(double) * n);
  double* z = (double*)malloc(sizeof(double) * n);
  double* rc = (double*)malloc(sizeof(double) * nc);
  double* zc = (double*)malloc(sizeof(double) * nc);
  memcpy(r, b, sizeof(double) * n); /* r0 = b - M 0 */
  memset(x, 0, sizeof(double) * n);
  for (int pass = 0; pass < g_omg_passes; ++pass) {
    omg_smoother(H, lev, r, z);
    rm_step(H, lev, &S, x0, b, z, x, r);
    or_restrict(L->nb, C->nb, Np, L->agg, L->R, r, rc);
    omg_level(H, lev + 1, rc, zc);
    memset(z, 0, sizeof(double) * n);
    or_prolong(L->nb, Np, L->agg, L->R, zc, z);
    rm_step(H, lev, &S, x0, b, z, x, r);
    omg_smoother(H, lev, r, z);
    rm_step(H, lev, &S, x0, b, z, x, r);
  }
  rm_free(&S);
  free(x0);
  free(r);
  free(z);
  free(rc);
  free(zc);
}

/* Algorithm OrthoMG on the finest level: x holds x0 on entry. Passes of (pre-smoother, RM,
 * coarse correction by one OrthoMG pass per coarser level, RM, post-smoother, RM) while
 * |r| > tol |b|, at most maxit passes. The search space of the finest level keeps every
 * direction up to `restart` columns; then x0 := x, r0 := b - M x (recomputed) and the space
 * starts empty again; the same when the updated residual meets the tolerance but the
 * recomputed one does not.
 * hist (optional, maxit+1 entries): |r|/|b| after each pass (hist[0]: initial).
 * Returns the passes made; *relres = the final |b - M x| / |b| (recomputed). */
int or_orthomg(void* h, const double* b, double* x, double tol, int maxit, int restart, double* relres,
               double* hist) {
  or_hier* H = (or_hier*)h;
  const int Np = H->Np;
  or_level* L = &H->L[0];
  const int64_t n = L->nb * Np;
  if (restart < 3) restart = 3;
  restart -= restart % 3;
  double* x0 = (double*)malloc(sizeof(double) * n);
  double* r0 = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  double* z = (double*)malloc(sizeof(double) * n);
  double bn = sqrt(dot(n, b, b));
  if (bn == 0.0) bn = 1.0;
  or_residual(L->nb, Np, L->rp, L->col, L->val, b, x, r0);
  memcpy(x0, x, sizeof(double) * n);
  memcpy(r, r0, sizeof(double) * n);
  double rn = sqrt(dot(n, r, r));
  if (hist) hist[0] = rn / bn;
  int it = 0;
  if (H->nlev == 1) { /* a single level: the direct solve */
    double* e = (double*)malloc(sizeof(double) * n);
    chol_solve(H->nc, H->cchol, r0, e);
    for (int64_t k = 0; k < n; ++k) x[k] += e[k];
    free(e);
    it = 1;
  } else {
    or_level* C = &H->L[1];
    const int64_t nc = C->nb * Np;
    double* rc = (double*)malloc(sizeof(double) * nc);
    double* zc = (double*)malloc(sizeof(double) * nc);
    or_rm_space S;
    rm_init(&S, n, restart);
    for (;;) {
      if (!(rn / bn > tol)) {
        /* the updated residual meets the tolerance: check the recomputed one; if rounding has
         * moved them apart, restart from x with the recomputed residual */
        or_residual(L->nb, Np, L->rp, L->col, L->val, b, x, z);
        const double tn = sqrt(dot(n, z, z));
        if (!(tn / bn > tol) || it >= maxit) break;
        memcpy(x0, x, sizeof(double) * n);
        memcpy(r0, z, sizeof(double) * n);
        memcpy(r, z, sizeof(double) * n);
        S.l = 0;
        rn = tn;
      }
      if (it >= maxit) break;
      if (S.l + 3 > S.cap) { /* restart: x0 := x, r0 := b - M x recomputed, the space empty */
        memcpy(x0, x, sizeof(double) * n);
        or_residual(L->nb, Np, L->rp, L->col, L->val, b, x, r0);
        memcpy(r, r0, sizeof(double) * n);
        S.l = 0;
      }
      omg_smoother(H, 0, r, z);
      rm_step(H, 0, &S, x0, r0, z, x, r);
      or_restrict(L->nb, C->nb, Np, L->agg, L->R, r, rc);
      omg_level(H, 1, rc, zc);
      memset(z, 0, sizeof(double) * n);
      or_prolong(L->nb, Np, L->agg, L->R, zc, z);
      rm_step(H, 0, &S, x0, r0, z, x, r);
      omg_smoother(H, 0, r, z);
      rm_step(H, 0, &S, x0, r0, z, x, r);
      rn = sqrt(dot(n, r, r));
      ++it;
      if (hist) hist[it] = rn / bn;
    }
    rm_free(&S);
    free(rc);
    free(zc);
  }
  or_residual(L->nb, Np, L->rp, L->col, L->val, b, x, r);
  *relres = sqrt(dot(n, r, r)) / bn;
  free(x0);
  free(r0);
  free(r);
  free(z);
  return it;
}

/* passes of Algorithm OrthoMG on each coarse level (1: one pass per visit; 2: a K-cycle) */
void or_set_orthomg_passes(int passes) { g_omg_passes = passes < 1 ? 1 : passes; }

/* Test access to Algorithm ResMinimi on level `lev`: k steps with the raw directions
 * zin[j*n .. j*n+n-1] (j = 0..k-1) from x0 (r0 = b - M x0); outputs x, r and the final W, Z
 * (k columns each, n x k column-major: column j at j*n). */
void or_rm_steps(void* h, int lev, int k, const double* zin, const double* b, const double* x0, double* x,
                 double* r, double* Wout, double* Zout) {
  or_hier* H = (or_hier*)h;
  or_level* L = &H->L[lev];
  const int64_t n = L->nb * H->Np;
  or_rm_space S;
  rm_init(&S, n, k);
  double* r0 = (double*)malloc(sizeof(double) * n);
  double* z = (double*)malloc(sizeof(double) * n);
  or_residual(L->nb, H->Np, L->rp, L->col, L->val, b, x0, r0);
  memcpy(x, x0, sizeof(double) * n);
  memcpy(r, r0, sizeof(double) * n);
  for (int j = 0; j < k; ++j) {
    memcpy(z, zin + (int64_t)j * n, sizeof(double) * n);
    rm_step(H, lev, &S, x0, r0, z, x, r);
  }
  memcpy(Wout, S.W, sizeof(double) * n * k);
  memcpy(Zout, S.Z, sizeof(double) * n * k);
  rm_free(&S);
  free(r0);
  free(z);
}

/* ---------------- p-multigrid (Algorithm pMultigrid) ---------------- */

/* PMG(b, k_lo, I) on level `lev`: the blocks I[0..nI-1] (ascending; nI < 0: every block), the
 * first n_lo modes of each block form the low-order set (the modes are graded by degree, so
 * they span the polynomials up to degree k_lo). Steps in the algorithm's order: x := 0; the
 * low-order system M_lo = M[I_lo, I_lo] solved directly (dense Cholesky here) with b[I_lo] and
 * added to x; r := b - M x; for every block j of I the high-order system M[I_hi,j, I_hi,j] solved
 * directly with r[I_hi,j] (reading the printed b_hi,j as the residual r of the line before) and
 * added to x. x has the level's length; entries outside I are zero. Returns 0, or -1 when a
 * system is not positive definite. */
int or_pmg(void* h, int lev, int n_lo, int64_t nI, const int32_t* I, const double* b, double* x) {
  or_hier* H = (or_hier*)h;
  or_level* L = &H->L[lev];
  const int Np = H->Np;
  const int64_t Np2 = (int64_t)Np * Np, n = L->nb * Np;
  const int nhi = Np - n_lo;
  int32_t* all = NULL;
  if (nI < 0) {
    nI = L->nb;
    all = (int32_t*)malloc(sizeof(int32_t) * nI);
    for (int64_t i = 0; i < nI; ++i) all[i] = (int32_t)i;
    I = all;
  }
  /* position of every block in I (-1: not in I) */
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * L->nb);
  for (int64_t i = 0; i < L->nb; ++i) pos[i] = -1;
  for (int64_t a = 0; a < nI; ++a) pos[I[a]] = a;
  for (int64_t k = 0; k < n; ++k) x[k] = 0.0;
  int rc = 0;
  /* low-order system */
  const int64_t m = nI * n_lo;
  double* A = (double*)calloc((size_t)m * m, sizeof(double));
  double* bl = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  double* xl = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  for (int64_t a = 0; a < nI; ++a) {
    const int64_t i = I[a];
    for (int64_t z = L->rp[i]; z < L->rp[i + 1]; ++z) {
      const int64_t c = pos[L->col[z]];
      if (c < 0) continue;
      for (int r = 0; r < n_lo; ++r)
        for (int q = 0; q < n_lo; ++q) A[(a * n_lo + r) * m + c * n_lo + q] = L->val[z * Np2 + r * Np + q];
    }
    for (int r = 0; r < n_lo; ++r) bl[a * n_lo + r] = b[i * Np + r];
  }
  if (m > 0) {
    if (chol(m, A)) rc = -1;
    else chol_solve(m, A, bl, xl);
  }
  if (rc == 0)
    for (int64_t a = 0; a < nI; ++a)
      for (int r = 0; r < n_lo; ++r) x[(int64_t)I[a] * Np + r] += xl[a * n_lo + r];
  /* residual and the cell-local high-order systems */
  double* res = (double*)malloc(sizeof(double) * n);
  or_residual(L->nb, Np, L->rp, L->col, L->val, b, x, res);
  double* D = (double*)malloc(sizeof(double) * (nhi > 0 ? nhi * nhi : 1));
  double* bh = (double*)malloc(sizeof(double) * (nhi > 0 ? nhi : 1));
  double* xh = (double*)malloc(sizeof(double) * (nhi > 0 ? nhi : 1));
  for (int64_t a = 0; rc == 0 && a < nI && nhi > 0; ++a) {
    const int64_t j = I[a];
    int64_t z = L->rp[j];
    while (z < L->rp[j + 1] && L->col[z] != j) ++z;
    for (int r = 0; r < nhi; ++r) {
      for (int q = 0; q < nhi; ++q) D[r * nhi + q] = L->val[z * Np2 + (n_lo + r) * Np + n_lo + q];
      bh[r] = res[j * Np + n_lo + r];
    }
    if (chol(nhi, D)) {
      rc = -1;
      break;
    }
    chol_solve(nhi, D, bh, xh);
    for (int r = 0; r < nhi; ++r) x[j * Np + n_lo + r] += xh[r];
  }
  free(A);
  free(bl);
  free(xl);
  free(res);
  free(D);
  free(bh);
  free(xh);
  free(pos);
  free(all);
  return rc;
}
