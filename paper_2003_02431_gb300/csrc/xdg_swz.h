// Internal interface between the host code of libxdg (xdg.cu) and the additive Schwarz
// kernels (xdg_swz.cu), compiled as separate translation units.
//
// Kummer, Smuda, Weber, arXiv 2003.02431, Algorithm Swz (additive Schwarz): the level's blocks
// are covered by patches P_i (they may overlap); the smoother's preconditioner is
//   S r = alpha^{-1/2} .* sum_i E_i (M_{P_i P_i})^{-1} E_i^T (alpha^{-1/2} .* r),
// alpha = the number of patches holding each block, with exact patch solves (the p-multigrid
// block solver of Algorithm pMultigrid with every mode in the low-order set). The symmetric
// alpha^{-1/2} scaling equals the printed x ./ alpha when alpha is the same for every block
// and keeps the cycle a symmetric preconditioner otherwise.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace xdg {
namespace swz {

// largest patch (modes of all its blocks) the kernels handle
constexpr int kMaxDof = 512;

// Two 64-bit hashes per patch of the dense patch matrix M_{PP} (its stored blocks, entry by
// entry with their positions) and the patch size: h[2p], h[2p+1]. Patches whose hashes and
// sizes agree share one inverse.
cudaError_t hash(int np, cudaStream_t s, int64_t npatch, const int64_t* pptr, const int32_t* pblk,
                 const int64_t* rp, const int32_t* col, const double* val, unsigned long long* h);

// Inverses of the patch matrices of the representatives rep[u0..u1) (one per distinct patch):
// M_{PP} gathered into work (FP64, woff[u - u0] offsets), factorised by Cholesky, inverted
// column by column into Ainv + ioff[u] (FP64, n x n, symmetric) and Ainv32 (FP32 copy).
// err[0] is set to 1 when a patch matrix is not positive definite.
cudaError_t factor(int np, cudaStream_t s, int64_t u0, int64_t u1, const int64_t* rep, const int64_t* pptr,
                   const int32_t* pblk, const int64_t* rp, const int32_t* col, const double* val,
                   const int64_t* ioff, double* work, const int64_t* woff, double* Ainv, float* Ainv32, int* err);

// Work item of the patch solves: count patches porder[start .. start+count-1] that share the
// stored inverse tid (n modes each). Items of one shared inverse stage it in shared memory once
// for all their patches.
struct Item {
  int64_t start;
  int32_t tid, count, n, pad;
};
// patches per item of a shared inverse
constexpr int kItemPatches = 64;

// Opt the patch-solve kernels of block size np into the shared memory they need (once per
// process and device, before the first launch or graph capture).
cudaError_t prepare(int np);

// Patch solves. For every patch p (one warp each): y = Ainv_{tid} (isq .* r)_{P_p}, then
//   out_mode 0: y into the patch's slots, out[(pptr[p] + a) Np + q]  (overlapping patches)
//   out_mode 1: out[blk Np + q] = om isq[blk] y                        (each block in one patch)
//   out_mode 2: out[blk Np + q] = xin[blk Np + q] + om isq[blk] y      (each block in one patch)
template <class T>
cudaError_t apply(int np, cudaStream_t s, int grid, int out_mode, int64_t nitem, const Item* items,
                  const int32_t* porder, const int64_t* pptr, const int32_t* pblk, const int64_t* ioff,
                  const T* Ainv, const T* isq, const T* r, T om, const T* xin, T* out, int maxdof,
                  int stage_n);
// (maxdof: the largest patch; stage_n: the largest shared inverse to stage in shared memory)

// out[i] = (xin[i] or 0) + om isq[i] sum of the block's slots y[bslot[k]] over
// k = bsptr[i] .. bsptr[i+1]-1 (ascending patch order)
template <class T>
cudaError_t accum(int np, cudaStream_t s, int grid, int64_t nb, const int64_t* bsptr, const int64_t* bslot,
                  const T* isq, const T* y, T om, const T* xin, T* out);

}  // namespace swz
}  // namespace xdg
