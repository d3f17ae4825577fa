// CUDA kernels of the XDG multigrid solve (sm_103a).
//
// Kummer, Smuda, Weber, arXiv 2003.02431: operator M^lambda in per-cell block form
// (Eq. GenericMatrixSystem), transfers R^{X,lambda} (Eq. XDGrestrictionMatrix), Galerkin
// coarse operators (Eq. XDGsysRestriction), the level recursion of Algorithm 4 and the
// cell-local dense solves used for smoothing (Algorithms 1, 2).
//
// Work mapping: a "group" of NP consecutive lanes owns one block row (lane r <-> row r of the
// block); a warp holds 32/NP groups working on consecutive block rows, so a warp streams
// contiguous block data with 16-byte loads. Within a group, dense Np x Np work uses
// register rows plus shuffles restricted to the group's lanes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "xdg_common.cuh"

namespace xdg {

template <int NP>
struct Grp {
  static constexpr int GPW = 32 / NP;              // groups per warp
  static constexpr int NT = NP * (NP + 1) / 2;     // packed lower triangle
};

__device__ __forceinline__ unsigned group_mask(int g, int np) {
  return (np == 32) ? 0xffffffffu : (((1u << np) - 1u) << (g * np));
}

// NP consecutive doubles -> registers (16-byte loads when the row is 16-byte aligned)
template <int NP>
__device__ __forceinline__ void ldrow(const double* __restrict__ p, double (&v)[NP]) {
  if constexpr (NP % 2 == 0) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int c = 0; c < NP / 2; ++c) {
      double2 t = __ldg(q + c);
      v[2 * c] = t.x;
      v[2 * c + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < NP; ++c) v[c] = __ldg(p + c);
  }
}

// blocks of a row whose loads are put in flight together: the column indices of a chunk are
// read first, so the dependent x-block loads of the chunk overlap (short rows of coarse levels
// run with few warps, where a block-by-block dependent chain is not hidden)
// blocks of a row whose loads are issued together (FP32 kernels: Np <= 10 and Np > 10)
#ifndef XDG_CH32_SMALL
#define XDG_CH32_SMALL 4
#endif
#ifndef XDG_CH32_LARGE
#define XDG_CH32_LARGE 2
#endif
template <int NP>
struct Chunk {
  static constexpr int F64 = NP <= 10 ? 2 : 1;
  static constexpr int F32 = NP <= 10 ? XDG_CH32_SMALL : XDG_CH32_LARGE;
};

// acc += A[z][r][:] . x[col[z]][:] over the block row (lane r), blocks in increasing z
template <int NP>
__device__ __forceinline__ double row_dot(int64_t z0, int64_t z1, int r, const int32_t* __restrict__ col,
                                          const double* __restrict__ val, const double* __restrict__ x) {
  constexpr int CH = Chunk<NP>::F64;
  double acc = 0.0;
  for (int64_t z = z0; z < z1; z += CH) {
    int32_t cc[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) cc[u] = (z + u < z1) ? __ldg(col + z + u) : -1;
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (cc[u] < 0) continue;
      double a[NP], xv[NP];
      ldrow<NP>(val + (z + u) * (NP * NP) + r * NP, a);
      ldrow<NP>(x + (int64_t)cc[u] * NP, xv);
#pragma unroll
      for (int c = 0; c < NP; ++c) acc = fma(a[c], xv[c], acc);
    }
  }
  return acc;
}

// ------------------------------------------------------------------------------------------
// operator apply: y = M x (MODE 0) or y = b - M x (MODE 1); act (optional): rows with
// act[i] == 0 are skipped (finished problems of a batch)
template <int NP, int MODE>
__global__ void __launch_bounds__(kThreads) k_spmv(int64_t nb, const int64_t* __restrict__ rp,
                                                  const int32_t* __restrict__ col,
                                                  const double* __restrict__ val,
                                                  const double* __restrict__ x,
                                                  const double* __restrict__ b,
                                                  double* __restrict__ y, const uint8_t* __restrict__ act) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
    if (act && !act[i]) continue;
    double acc = row_dot<NP>(__ldg(rp + i), __ldg(rp + i + 1), r, col, val, x);
    y[i * NP + r] = MODE ? b[i * NP + r] - acc : acc;
  }
}

// ------------------------------------------------------------------------------------------
// (W v)_r for an Np x Np row-major block W (lane r; v_c held by lane c of the group)
template <int NP>
__device__ __forceinline__ double block_gemv(const double* __restrict__ W, int r, int base, unsigned mask,
                                             double v) {
  double w[NP];
  ldrow<NP>(W + r * NP, w);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < NP; ++c) s = fma(w[c], __shfl_sync(mask, v, base + c), s);
  return s;
}

// damped block Jacobi: xo = xi + omega D^{-1} (b - M xi); ZERO: xi = 0 (no operator apply).
// Dinv holds the inverse of every diagonal block (from its Cholesky factor).
template <int NP, bool ZERO>
__global__ void __launch_bounds__(kThreads) k_smooth(int64_t nb, const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ col,
                                                    const double* __restrict__ val,
                                                    const double* __restrict__ Dinv, double omega,
                                                    const double* __restrict__ omr,
                                                    const double* __restrict__ b,
                                                    const double* __restrict__ xi,
                                                    double* __restrict__ xo) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
    double res = b[i * NP + r];
    if (!ZERO) res -= row_dot<NP>(__ldg(rp + i), __ldg(rp + i + 1), r, col, val, xi);
    double z = block_gemv<NP>(Dinv + i * (NP * NP), r, g * NP, mask, res);
    const double om = omr ? __ldg(omr + i) : omega;  // per-row damping in batches
    xo[i * NP + r] = ZERO ? om * z : fma(om, z, xi[i * NP + r]);
  }
}

// z = D^{-1} v (no damping, no operator); used by the Lanczos estimate
template <int NP>
__global__ void __launch_bounds__(kThreads) k_bjsolve(int64_t nb, const double* __restrict__ Dinv,
                                                     const double* __restrict__ v,
                                                     double* __restrict__ z) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW)
    z[i * NP + r] = block_gemv<NP>(Dinv + i * (NP * NP), r, g * NP, mask, v[i * NP + r]);
}

// w = D v with the diagonal blocks of M (diag[i] = position of block (i,i))
template <int NP>
__global__ void __launch_bounds__(kThreads) k_diagmul(int64_t nb, const int64_t* __restrict__ diag,
                                                     const double* __restrict__ val,
                                                     const double* __restrict__ v,
                                                     double* __restrict__ w) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
    double a[NP], xv[NP];
    ldrow<NP>(val + __ldg(diag + i) * (NP * NP) + r * NP, a);
    ldrow<NP>(v + i * NP, xv);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NP; ++c) s = fma(a[c], xv[c], s);
    w[i * NP + r] = s;
  }
}

// ------------------------------------------------------------------------------------------
// restriction, phase 1 (row-parallel): t_f = R_f^T res_f, res_f = b_f - (M x)_f (RESID) or b_f
template <int NP, bool RESID>
__global__ void __launch_bounds__(kThreads) k_resid_rt(int64_t nbf, const int64_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ val,
                                                      const double* __restrict__ R,
                                                      const double* __restrict__ b,
                                                      const double* __restrict__ x,
                                                      double* __restrict__ t) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  const int base = g * NP;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t f = warp * GPW + g; f < nbf; f += nw * GPW) {
    double res = b[f * NP + r];
    if (RESID) res -= row_dot<NP>(__ldg(rp + f), __ldg(rp + f + 1), r, col, val, x);
    const double* Rf = R + f * (NP * NP);
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < NP; ++m) s = fma(__ldg(Rf + m * NP + r), __shfl_sync(mask, res, base + m), s);
    t[f * NP + r] = s;
  }
}

// sum of t[f][r] over the children f = ch[q0..q1) in increasing q (child indices read in chunks
// of 8 so the value loads overlap)
template <int NP, class T, class A, bool COH = false>
__device__ __forceinline__ A child_sum(int64_t q0, int64_t q1, int r, const int32_t* __restrict__ ch,
                                       const T* __restrict__ t) {
  A s = 0;
  for (int64_t q = q0; q < q1; q += 8) {
    int32_t f[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) f[u] = (q + u < q1) ? __ldg(ch + q + u) : -1;
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if constexpr (COH) v[u] = (f[u] >= 0) ? __ldcg(t + (int64_t)f[u] * NP + r) : (T)0;
      else v[u] = (f[u] >= 0) ? t[(int64_t)f[u] * NP + r] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (f[u] >= 0) s += v[u];
  }
  return s;
}

// restriction, phase 2: rc[C] = sum of t_f over the children f of C, in increasing f
// (deterministic; one thread per coarse entry)
template <int NP>
__global__ void __launch_bounds__(kThreads) k_gather(int64_t nbc, const int64_t* __restrict__ cptr,
                                                    const int32_t* __restrict__ ch,
                                                    const double* __restrict__ t,
                                                    double* __restrict__ rc) {
  pdl_entry();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nbc * NP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t C = e / NP;
    const int r = (int)(e - C * NP);
    rc[e] = child_sum<NP, double, double>(__ldg(cptr + C), __ldg(cptr + C + 1), r, ch, t);
  }
}

// phase 2 fused with the first sweep of the coarse level from a zero guess:
// bc_C = sum over children of t_f; xc_C = omega D_C^{-1} bc_C (one group per coarse block)
template <int NP>
__global__ void __launch_bounds__(kThreads) k_gather_smooth0(int64_t nbc, const int64_t* __restrict__ cptr,
                                                            const int32_t* __restrict__ ch,
                                                            const double* __restrict__ t,
                                                            const double* __restrict__ Dinv, double omega,
                                                            const double* __restrict__ omr,
                                                            double* __restrict__ bc, double* __restrict__ xc) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t C = warp * GPW + g; C < nbc; C += nw * GPW) {
    double bv = child_sum<NP, double, double>(__ldg(cptr + C), __ldg(cptr + C + 1), r, ch, t);
    bc[C * NP + r] = bv;
    double w[NP];
    ldrow<NP>(Dinv + C * (NP * NP) + r * NP, w);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NP; ++c) s = fma(w[c], __shfl_sync(mask, bv, g * NP + c), s);
    xc[C * NP + r] = (omr ? __ldg(omr + C) : omega) * s;
  }
}

// xo_f = xi_f + R_f zc[agg[f]]  (xo may equal xi)
template <int NP>
__global__ void __launch_bounds__(kThreads) k_prolong(int64_t nbf, const int32_t* __restrict__ agg,
                                                     const double* __restrict__ R,
                                                     const double* __restrict__ zc,
                                                     const double* xi, double* xo) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t f = warp * GPW + g; f < nbf; f += nw * GPW) {
    double a[NP], z[NP];
    ldrow<NP>(R + f * (NP * NP) + r * NP, a);
    ldrow<NP>(zc + (int64_t)__ldg(agg + f) * NP, z);
    double s = 0.0;
#pragma unroll
    for (int n = 0; n < NP; ++n) s = fma(a[n], z[n], s);
    xo[f * NP + r] = xi[f * NP + r] + s;
  }
}

// ------------------------------------------------------------------------------------------
// Galerkin product M_c = R^T M R: one group per coarse row I accumulates, for every child i
// of I and every fine block (i, j), R_i^T M_ij R_j into the coarse block (I, agg[j]).
// The coarse values must be zero on entry.
template <int NP>
__global__ void __launch_bounds__(kThreads) k_galerkin(int64_t nbc, const int64_t* __restrict__ cptr,
                                                      const int32_t* __restrict__ ch,
                                                      const int64_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ val,
                                                      const int32_t* __restrict__ agg,
                                                      const double* __restrict__ R,
                                                      const int64_t* __restrict__ crp,
                                                      const int32_t* __restrict__ ccol,
                                                      double* __restrict__ cval) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  __shared__ double T[kThreads / 32][GPW][NP * NP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  double* Tg = T[wib][g];
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t I = warp * GPW + g; I < nbc; I += nw * GPW) {
    const int64_t c0 = __ldg(crp + I), c1 = __ldg(crp + I + 1);
    for (int64_t t = __ldg(cptr + I); t < __ldg(cptr + I + 1); ++t) {
      const int64_t i = __ldg(ch + t);
      const double* Ri = R + i * (NP * NP);
      for (int64_t z = __ldg(rp + i); z < __ldg(rp + i + 1); ++z) {
        const int64_t j = __ldg(col + z);
        const double* Rj = R + j * (NP * NP);
        const int32_t J = __ldg(agg + j);
        // T = M_ij R_j, lane r computes row r
        double m[NP];
        ldrow<NP>(val + z * (NP * NP) + r * NP, m);
#pragma unroll
        for (int n = 0; n < NP; ++n) {
          double s = 0.0;
#pragma unroll
          for (int a = 0; a < NP; ++a) s = fma(m[a], __ldg(Rj + a * NP + n), s);
          Tg[r * NP + n] = s;
        }
        __syncwarp(mask);
        // locate (I, J) in the coarse row
        int64_t lo = c0, hi = c1 - 1;
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          if (__ldg(ccol + mid) < J) lo = mid + 1;
          else hi = mid;
        }
        double* dst = cval + lo * (NP * NP) + r * NP;
        // row r of R_i^T T
        double ri[NP];
#pragma unroll
        for (int a = 0; a < NP; ++a) ri[a] = __ldg(Ri + a * NP + r);
#pragma unroll
        for (int n = 0; n < NP; ++n) {
          double s = 0.0;
#pragma unroll
          for (int a = 0; a < NP; ++a) s = fma(ri[a], Tg[a * NP + n], s);
          dst[n] += s;
        }
        __syncwarp(mask);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// inverse of every diagonal block D = L L^T (one thread per block): Cholesky factor L, then
// X = L^{-1} by forward substitution, then D^{-1} = X^T X (row-major, symmetric).
// err is set when a block is not positive definite.
template <int NP>
__global__ void k_diag_inv(int64_t nb, const int64_t* __restrict__ diag, const double* __restrict__ val,
                           double* __restrict__ Dinv, int* err) {
  pdl_entry();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double A[NP * NP];
  const double* src = val + diag[i] * (NP * NP);
  for (int e = 0; e < NP * NP; ++e) A[e] = src[e];
  for (int j = 0; j < NP; ++j) {
    double s = A[j * NP + j];
    for (int p = 0; p < j; ++p) s -= A[j * NP + p] * A[j * NP + p];
    if (!(s > 0.0)) {
      atomicOr(err, 1);
      return;
    }
    double d = sqrt(s);
    A[j * NP + j] = d;
    for (int q = j + 1; q < NP; ++q) {
      double t = A[q * NP + j];
      for (int p = 0; p < j; ++p) t -= A[q * NP + p] * A[j * NP + p];
      A[q * NP + j] = t / d;
    }
  }
  // X = L^{-1}, column by column (lower triangular)
  double X[NP * NP];
  for (int e = 0; e < NP * NP; ++e) X[e] = 0.0;
  for (int c = 0; c < NP; ++c)
    for (int q = c; q < NP; ++q) {
      double s = (q == c) ? 1.0 : 0.0;
      for (int p = c; p < q; ++p) s -= A[q * NP + p] * X[p * NP + c];
      X[q * NP + c] = s / A[q * NP + q];
    }
  // D^{-1} = X^T X: entry (r, c) = sum over q >= max(r, c) of X[q][r] X[q][c]
  double* dst = Dinv + i * (NP * NP);
  for (int r = 0; r < NP; ++r)
    for (int c = r; c < NP; ++c) {
      double s = 0.0;
      for (int q = c; q < NP; ++q) s += X[q * NP + r] * X[q * NP + c];
      dst[r * NP + c] = s;
      dst[c * NP + r] = s;
    }
}

// ------------------------------------------------------------------------------------------
// deterministic reductions and Krylov vector updates

constexpr int kRedBlocks = 608;  // 4 x 152 SMs; fixed so that the summation order is fixed

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < kThreads / 32) ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// partial[blockIdx] = sum over the block's grid-stride share of x_i y_i
__global__ void __launch_bounds__(kThreads) k_dot_partial(int64_t n, const double* __restrict__ x,
                                                         const double* __restrict__ y,
                                                         double* __restrict__ partial) {
  pdl_entry();
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out = sum of partial[0..np) in a fixed order
__global__ void __launch_bounds__(kThreads) k_sum_final(int np, const double* __restrict__ partial,
                                                       double* __restrict__ out) {
  pdl_entry();
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// PCG scalars kept on the device
struct PcgScal {
  double rz, rz_new, pq, rr, alpha, beta, zq;
  int bad;
};

// beta = rz_new / rz; rz = rz_new
__global__ void k_pcg_beta(PcgScal* S) {
  pdl_entry();
  double rn = S->rz_new;
  if (!(rn > 0.0) || !isfinite(rn)) {
    S->bad = 1;
    S->beta = 0.0;
  } else {
    S->beta = rn / S->rz;
  }
  S->rz = rn;
}

// x += alpha p; r -= alpha q; partial[] of r.r; rf (optional) = r rounded to FP32 (the input
// of a low-precision cycle)
__global__ void __launch_bounds__(kThreads) k_pcg_xr(int64_t n, const PcgScal* __restrict__ S,
                                                    const double* __restrict__ p,
                                                    const double* __restrict__ q, double* __restrict__ x,
                                                    double* __restrict__ r, double* __restrict__ partial,
                                                    float* __restrict__ rf) {
  pdl_entry();
  const double a = S->alpha;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    if (rf) rf[i] = (float)ri;
    s = fma(ri, ri, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// y = M x (block rows spread as in k_spmv) and partial[blockIdx.x] = this CTA's part of x . y
template <int NP>
__global__ void __launch_bounds__(kThreads) k_spmv_dot(int64_t nb, const int64_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col, const double* __restrict__ val,
                                                      const double* __restrict__ x, double* __restrict__ y,
                                                      double* __restrict__ partial) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  double d = 0.0;
  if (g < GPW) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
      const double acc = row_dot<NP>(__ldg(rp + i), __ldg(rp + i + 1), r, col, val, x);
      y[i * NP + r] = acc;
      d = fma(x[i * NP + r], acc, d);
    }
  }
  d = block_sum(d);
  if (threadIdx.x == 0) partial[blockIdx.x] = d;
}

// sum of partial[0..np) (stride, offset) in a fixed order by one CTA; valid in thread 0
__device__ __forceinline__ double sum_partials(int np, const double* __restrict__ partial, int stride, int off) {
  const int per = (np + blockDim.x - 1) / blockDim.x;
  const int i0 = threadIdx.x * per, i1 = min(np, i0 + per);
  double s = 0.0;
  for (int i = i0; i < i1; ++i) s += partial[i * stride + off];
  return block_sum(s);
}

// pq from the partial sums, then alpha = rz / pq (breakdown flagged)
__global__ void __launch_bounds__(kThreads) k_cg_alpha_final(int np, const double* __restrict__ partial,
                                                            PcgScal* S) {
  pdl_entry();
  const double pq = sum_partials(np, partial, 1, 0);
  if (threadIdx.x == 0) {
    S->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
      S->bad = 1;
      S->alpha = 0.0;
    } else {
      S->alpha = S->rz / pq;
    }
  }
}

// p = z + beta p
__global__ void __launch_bounds__(kThreads) k_pcg_p(int64_t n, const PcgScal* __restrict__ S,
                                                   const double* __restrict__ z, double* __restrict__ p) {
  pdl_entry();
  const double be = S->beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(be, p[i], z[i]);
}

__global__ void k_copy(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// y += a x (a on the host)
__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

}  // namespace xdg
