// Internal interface of the FP64 kernels for blocks wider than a warp (xdg_big.cu): Np = 35 and
// 56, the k = 4 and k = 5 spaces in 3D (arXiv 2003.02431, sec. 4 runs k = 5). The operations
// are those of the small-block kernel table (operator apply, block-Jacobi sweep, residual and
// restriction, prolongation, Galerkin product, diagonal-block inverses); each function enqueues
// one kernel on the stream and reports errors through cudaGetLastError. Mapping: one warp per
// block row, lane l owning rows l and l + 32 of the block.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace xdg {
namespace big {

// partial sums spmv_dot may write (its grid is capped at this)
constexpr int kMaxPartials = 4096;

struct Table {
  // y = M x (mode 0) or y = b - M x (mode 1); rows with act[i] == 0 skipped (act may be null)
  void (*spmv)(int grid, cudaStream_t, const uint8_t* act, int64_t nb, const int64_t* rp, const int32_t* col,
               const double* val, const double* x, const double* b, double* y, int mode);
  // xo = xi + omega_i Dinv_i (b - M xi)_i; xi == nullptr: xo = omega_i Dinv_i b_i
  void (*smooth)(int grid, cudaStream_t, int64_t nb, const int64_t* rp, const int32_t* col, const double* val,
                 const double* Dinv, double omega, const double* omr, const double* b, const double* xi, double* xo);
  // z_i = Dinv_i v_i
  void (*bjsolve)(int grid, cudaStream_t, int64_t nb, const double* Dinv, const double* v, double* z);
  // w_i = M_ii v_i (diag[i]: position of block (i, i))
  void (*diagmul)(int grid, cudaStream_t, int64_t nb, const int64_t* diag, const double* val, const double* v,
                  double* w);
  // t_f = R_f^T (b - M x)_f (x == nullptr: R_f^T b_f)
  void (*resid_rt)(int grid, cudaStream_t, int64_t nbf, const int64_t* rp, const int32_t* col, const double* val,
                   const double* R, const double* b, const double* x, double* t);
  // rc_C = sum of t_f over the children f of C (ascending)
  void (*gather)(int grid, cudaStream_t, int64_t nbc, const int64_t* cptr, const int32_t* ch, const double* t,
                 double* rc);
  // bc_C = sum of t_f over the children; xc_C = omega_C Dinv_C bc_C
  void (*gather_smooth0)(int grid, cudaStream_t, int64_t nbc, const int64_t* cptr, const int32_t* ch,
                         const double* t, const double* Dinv, double omega, const double* omr, double* bc,
                         double* xc);
  // xo_f = xi_f + R_f zc_{agg[f]}
  void (*prolong)(int grid, cudaStream_t, int64_t nbf, const int32_t* agg, const double* R, const double* zc,
                  const double* xi, double* xo);
  // coarse values (zero on entry) += R_i^T M_ij R_j into block (agg[i], agg[j])
  void (*galerkin)(int grid, cudaStream_t, int64_t nbc, const int64_t* cptr, const int32_t* ch, const int64_t* rp,
                   const int32_t* col, const double* val, const int32_t* agg, const double* R, const int64_t* crp,
                   const int32_t* ccol, double* cval);
  // Dinv_i = M_ii^{-1} via Cholesky; *err = 1 if a block is not positive definite
  void (*diag_inv)(cudaStream_t, int64_t nb, const int64_t* diag, const double* val, double* Dinv, int* err);
  // y = M x and partial[CTA] = that CTA's part of x . y; returns the number of CTAs (at most
  // kMaxPartials)
  int (*spmv_dot)(int grid, cudaStream_t, int64_t nb, const int64_t* rp, const int32_t* col, const double* val,
                  const double* x, double* y, double* partial);
};

// the table for np (35 or 56); false for other sizes
bool table_for(int np, Table* t);

}  // namespace big
}  // namespace xdg
