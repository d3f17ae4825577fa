// Internal interface of the multi-vector Krylov kernels (xdg_krylov.cu): Gram-Schmidt against a
// block of stored vectors, used by the residual minimisation of the orthonormalisation
// multigrid (arXiv 2003.02431, Algorithms ResMinimi and OrthoMG) and by the Arnoldi process of
// GMRES. Vectors are FP64, n entries; a block of l vectors is stored column after column
// (vector i at V + i n). Scalars live on the device, so a whole step needs no host round trip.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace xdg {
namespace kry {

// partial sums of beta_i = V_i . w (i < l) per CTA: part[blk * l + i]; grid = CTAs used
cudaError_t mdot_partial(cudaStream_t s, int grid, int64_t n, int l, const double* V, const double* w, double* part);
// beta[i] = sum over the grid's CTAs of part[blk * l + i] (fixed order); also acc[i] += beta[i]
// when acc != nullptr
cudaError_t mdot_final(cudaStream_t s, int grid, int l, const double* part, double* beta, double* acc);
// w -= sum_i beta_i V_i; z -= sum_i beta_i Z_i (Z may be null)
cudaError_t gs_update(cudaStream_t s, int grid, int64_t n, int l, const double* V, const double* Z,
                      const double* beta, double* w, double* z);
// gamma = 1/sqrt(*nrm2) if *nrm2 > (1e-14)^2 *w0sq, else 0 (a dependent direction); w *= gamma;
// zout = gamma * zin (zin, zout may be null); *gam_out = gamma (optional)
cudaError_t normalize(cudaStream_t s, int grid, int64_t n, const double* nrm2, const double* w0sq, double* w,
                      const double* zin, double* zout, double* gam_out);
// x += a z; r -= a w with a = *alpha
cudaError_t rm_update(cudaStream_t s, int grid, int64_t n, const double* alpha, const double* z, const double* w,
                      double* x, double* r);

// GMRES least-squares updates, one thread on the device. Column j of the Hessenberg matrix H
// ((m+1) x m, column-major, ld = m+1) holds h_{0..j,j}; hnorm2 = |w|^2 of the new Arnoldi
// vector. Sets h_{j+1,j}, applies the previous Givens rotations (cs, sn) to the column, forms
// rotation j and updates g (the rotated right-hand side, g[0] = beta at the start).
cudaError_t givens(cudaStream_t s, int j, int ld, double* H, double* cs, double* sn, double* g, const double* hnorm2);
// the Arnoldi start: beta = sqrt(*nrm2), g = (beta, 0, ...), *inv = 1/beta (0 if beta = 0)
cudaError_t gmres_start(cudaStream_t s, int m, const double* nrm2, double* g, double* inv);
// y = H(0..k-1, 0..k-1)^{-1} g(0..k-1) by back substitution, stored negated (ny = -y)
cudaError_t gmres_solve(cudaStream_t s, int k, int ld, const double* H, const double* g, double* ny);
// x *= *a (a device scalar)
cudaError_t scale(cudaStream_t s, int grid, int64_t n, const double* a, const double* x, double* y);

}  // namespace kry

// p-multigrid on one level (arXiv 2003.02431, Algorithm pMultigrid): the first n_lo modes of
// every Np-mode block form the low-order set (the bases are graded by degree).
namespace pmg {
// dst[z] = the leading n_lo x n_lo part of the Np x Np block src[z] (nblk blocks)
cudaError_t sub_blocks(cudaStream_t s, int64_t nblk, int np, int n_lo, const double* src, double* dst);
// lo[i][r] = v[i][r], r < n_lo (nb blocks)
cudaError_t take_lo(cudaStream_t s, int64_t nb, int np, int n_lo, const double* v, double* lo);
// z = 0 except z[i][r] = lo[i][r], r < n_lo
cudaError_t put_lo(cudaStream_t s, int64_t nb, int np, int n_lo, const double* lo, double* z);
// inverses of the trailing (np - n_lo)^2 parts of the diagonal blocks val[diag[i]] (Cholesky,
// then column by column); err[0] = 1 if one is not positive definite
cudaError_t hi_inverses(cudaStream_t s, int64_t nb, int np, int n_lo, const int64_t* diag, const double* val,
                        double* Hinv, int* err);
// z[i][n_lo + r] += sum_c Hinv[i][r][c] res[i][n_lo + c]
cudaError_t hi_apply(cudaStream_t s, int64_t nb, int np, int n_lo, const double* Hinv, const double* res, double* z);
}  // namespace pmg
}  // namespace xdg
