// FP64 kernels of the XDG multigrid for blocks wider than a warp: Np = 35 and 56, the k = 4 and
// k = 5 polynomial spaces in 3D (arXiv 2003.02431: operator apply of Eq. GenericMatrixSystem,
// transfers of Eq. XDGrestrictionMatrix, Galerkin coarse operators of Eq. XDGsysRestriction,
// the cell-local dense solves of the block-Jacobi smoother; sec. 4 uses k = 5).
//
// Mapping: one warp per block row; lane l owns rows l and l + 32 of the block (RPL = 2 rows per
// lane for both sizes). A lane streams its block row through registers eight columns at a time
// (16-byte loads when Np is even); the x block of a column is read by the whole warp (one
// broadcast per load). Block-times-vector products with a vector spread over the warp's lanes
// take entry c from lane c % 32, slot c / 32, by shuffles. Per entry the arithmetic order is that
// of the small-block kernels: blocks of a row in increasing position, columns in increasing
// order, one FMA chain per entry.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "xdg_big.h"
#include "xdg_common.cuh"

namespace xdg {
namespace big {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// resident CTAs per SM requested for the row kernels (caps their registers; unbounded, the fully
// unrolled block rows take up to 174 registers and one CTA per SM)
#ifndef XDG_BIG_MINB
#define XDG_BIG_MINB 3
#endif

template <int NP>
struct Shape {
  static_assert(NP > 32 && NP <= 64, "two block rows per lane");
  static constexpr int RPL = (NP + 31) / 32;  // block rows per lane
};

// v[c / 32] without indexing the register array by a run-time value
template <int NP>
__device__ __forceinline__ double slot(const double (&v)[Shape<NP>::RPL], int c) {
  return c < 32 ? v[0] : v[Shape<NP>::RPL - 1];
}

__device__ __forceinline__ int64_t warp_id() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t n_warps() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

// eight consecutive doubles p[c0 .. c0 + 8) that lie below NP (16-byte loads for even NP: every
// row of an even-sized block starts on a 16-byte boundary)
template <int NP>
__device__ __forceinline__ void ld8(const double* __restrict__ p, int c0, double (&v)[8]) {
  if constexpr (NP % 2 == 0) {
#pragma unroll
    for (int u = 0; u < 8; u += 2)
      if (c0 + u < NP) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(p + c0 + u));
        v[u] = t.x;
        v[u + 1] = t.y;
      }
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (c0 + u < NP) v[u] = __ldg(p + c0 + u);
  }
}

// acc + a[0 .. NP) . v[0 .. NP), one FMA chain in increasing column order
template <int NP>
__device__ __forceinline__ double dot_row(const double* __restrict__ a, const double* __restrict__ v, double acc) {
#pragma unroll 1
  for (int c0 = 0; c0 < NP; c0 += 8) {
    double av[8], xv[8];
    ld8<NP>(a, c0, av);
    ld8<NP>(v, c0, xv);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (c0 + u < NP) acc = fma(av[u], xv[u], acc);
  }
  return acc;
}

// acc_q += sum over the blocks z0 .. z1 of row i of A_z[r_q][:] . x[col[z]][:]  (r_q = lane + 32 q)
template <int NP>
__device__ __forceinline__ void row_dot(int64_t z0, int64_t z1, int lane, const int32_t* __restrict__ col,
                                        const double* __restrict__ val, const double* __restrict__ x,
                                        double (&acc)[Shape<NP>::RPL]) {
  for (int64_t z = z0; z < z1; ++z) {
    const double* xv = x + (int64_t)__ldg(col + z) * NP;
    const double* A = val + z * (NP * NP);
#pragma unroll
    for (int q = 0; q < Shape<NP>::RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < NP) acc[q] = dot_row<NP>(A + r * NP, xv, acc[q]);
    }
  }
}

// out_q = sum_c W[r_q][c] v_c, v_c held by lane c % 32 in slot c / 32 (called by all 32 lanes)
template <int NP>
__device__ __forceinline__ void block_gemv(const double* __restrict__ W, int lane, const double (&v)[Shape<NP>::RPL],
                                           double (&out)[Shape<NP>::RPL]) {
#pragma unroll
  for (int q = 0; q < Shape<NP>::RPL; ++q) out[q] = 0.0;
#pragma unroll 1
  for (int c0 = 0; c0 < NP; c0 += 8) {
    double vc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (c0 + u < NP) vc[u] = __shfl_sync(kFull, slot<NP>(v, c0 + u), (c0 + u) & 31);
#pragma unroll
    for (int q = 0; q < Shape<NP>::RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < NP) {
        double w[8];
        ld8<NP>(W + r * NP, c0, w);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c0 + u < NP) out[q] = fma(w[u], vc[u], out[q]);
      }
    }
  }
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// ------------------------------------------------------------------------------------------
// y = M x (MODE 0) or y = b - M x (MODE 1)
template <int NP, int MODE>
__global__ void __launch_bounds__(kThreads, XDG_BIG_MINB) k_spmv_big(int64_t nb, const int64_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col, const double* __restrict__ val,
                                                      const double* __restrict__ x, const double* __restrict__ b,
                                                      double* __restrict__ y, const uint8_t* __restrict__ act) {
  pdl_entry();
  constexpr int RPL = Shape<NP>::RPL;
  const int lane = threadIdx.x & 31;
  for (int64_t i = warp_id(); i < nb; i += n_warps()) {
    if (act && !act[i]) continue;
    double acc[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) acc[q] = 0.0;
    row_dot<NP>(__ldg(rp + i), __ldg(rp + i + 1), lane, col, val, x, acc);
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < NP) y[i * NP + r] = MODE ? b[i * NP + r] - acc[q] : acc[q];
    }
  }
}

// y = M x and partial[CTA] = the CTA's part of x . y
template <int NP>
__global__ void __launch_bounds__(kThreads, XDG_BIG_MINB) k_spmv_dot_big(int64_t nb, const int64_t* __restrict__ rp,
                                                          const int32_t* __restrict__ col,
                                                          const double* __restrict__ val,
                                                          const double* __restrict__ x, double* __restrict__ y,
                                                          double* __restrict__ partial) {
  pdl_entry();
  constexpr int RPL = Shape<NP>::RPL;
  const int lane = threadIdx.x & 31;
  double d = 0.0;
  for (int64_t i = warp_id(); i < nb; i += n_warps()) {
    double acc[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) acc[q] = 0.0;
    row_dot<NP>(__ldg(rp + i), __ldg(rp + i + 1), lane, col, val, x, acc);
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < NP) {
        y[i * NP + r] = acc[q];
        d = fma(x[i * NP + r], acc[q], d);
      }
    }
  }
  d = block_sum(d);
  if (threadIdx.x == 0) partial[blockIdx.x] = d;
}

// res_q = b - (M xi) on row i (ZERO: res = b)
template <int NP, bool ZERO>
__device__ __forceinline__ void row_residual(int64_t i, int lane, const int64_t* __restrict__ rp,
                                             const int32_t* __restrict__ col, const double* __restrict__ val,
                                             const double* __restrict__ b, const double* __restrict__ xi,
                                             double (&res)[Shape<NP>::RPL]) {
  constexpr int RPL = Shape<NP>::RPL;
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int r = lane + 32 * q;
    res[q] = r < NP ? b[i * NP + r] : 0.0;
  }
  if (!ZERO) {
    double acc[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) acc[q] = 0.0;
    row_dot<NP>(__ldg(rp + i), __ldg(rp + i + 1), lane, col, val, xi, acc);
#pragma unroll
    for (int q = 0; q < RPL; ++q) res[q] -= acc[q];
  }
}

// damped block Jacobi: xo = xi + omega D^{-1} (b - M xi); ZERO: xi = 0
template <int NP, bool ZERO>
__global__ void __launch_bounds__(kThreads, XDG_BIG_MINB) k_smooth_big(int64_t nb, const int64_t* __restrict__ rp,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const double* __restrict__ Dinv, double omega,
                                                        const double* __restrict__ omr, const double* __restrict__ b,
                                                        const double* __restrict__ xi, double* __restrict__ xo) {
  pdl_entry();
  constexpr int RPL = Shape<NP>::RPL;
  const int lane = threadIdx.x & 31;
  for (int64_t i = warp_id(); i < nb; i += n_warps()) {
    double res[RPL], z[RPL];
    row_residual<NP, ZERO>(i, lane, rp, col, val, b, xi, res);
    block_gemv<NP>(Dinv + i * (NP * NP), lane, res, z);
    const double om = omr ? __ldg(omr + i) : omega;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < NP) xo[i * NP + r] = ZERO ? om * z[q] : fma(om, z[q], xi[i * NP + r]);
    }
  }
}

// z = D^{-1} v
template <int NP>
__global__ void __launch_bounds__(kThreads, XDG_BIG_MINB) k_bjsolve_big(int64_t nb, const double* __restrict__ Dinv,
                                                         const double* __restrict__ v, double* __restrict__ z) {
  pdl_entry();
  constexpr int RPL = Shape<NP>::RPL;
  const int lane = threadIdx.x & 31;
  for (int64_t i = warp_id(); i < nb; i += n_warps()) {
    double vi[RPL], zi[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      vi[q] = r < NP ? v[i * NP + r] : 0.0;
    }
    block_gemv<NP>(Dinv + i * (NP * NP), lane, vi, zi);
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < NP) z[i * NP + r] = zi[q];
    }
  }
}

// w = D v with the diagonal blocks of M
template <int NP>
__global__ void __launch_bounds__(kThreads, XDG_BIG_MINB) k_diagmul_big(int64_t nb, const int64_t* __restrict__ diag,
                                                         const double* __restrict__ val, const double* __restrict__ v,
                                                         double* __restrict__ w) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  for (int64_t i = warp_id(); i < nb; i += n_warps()) {
    const double* A = val + __ldg(diag + i) * (NP * NP);
#pragma unroll
    for (int q = 0; q < Shape<NP>::RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < NP) w[i * NP + r] = dot_row<NP>(A + r * NP, v + i * NP, 0.0);
    }
  }
}

// restriction, phase 1: t_f = R_f^T res_f, res_f = b_f - (M x)_f (RESID) or b_f
template <int NP, bool RESID>
__global__ void __launch_bounds__(kThreads, XDG_BIG_MINB) k_resid_rt_big(int64_t nbf, const int64_t* __restrict__ rp,
                                                          const int32_t* __restrict__ col,
                                                          const double* __restrict__ val,
                                                          const double* __restrict__ R, const double* __restrict__ b,
                                                          const double* __restrict__ x, double* __restrict__ t) {
  pdl_entry();
  constexpr int RPL = Shape<NP>::RPL;
  const int lane = threadIdx.x & 31;
  for (int64_t f = warp_id(); f < nbf; f += n_warps()) {
    double res[RPL], s[RPL];
    row_residual<NP, !RESID>(f, lane, rp, col, val, b, x, res);
    const double* Rf = R + f * (NP * NP);
#pragma unroll
    for (int q = 0; q < RPL; ++q) s[q] = 0.0;
#pragma unroll 8
    for (int m = 0; m < NP; ++m) {
      const double rm = __shfl_sync(kFull, slot<NP>(res, m), m & 31);
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int r = lane + 32 * q;
        if (r < NP) s[q] = fma(__ldg(Rf + m * NP + r), rm, s[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < NP) t[f * NP + r] = s[q];
    }
  }
}

// sum of t[f][r] over the children f = ch[q0 .. q1), in increasing q
template <int NP>
__device__ __forceinline__ double child_sum(int64_t q0, int64_t q1, int r, const int32_t* __restrict__ ch,
                                            const double* __restrict__ t) {
  double s = 0.0;
  for (int64_t q = q0; q < q1; ++q) s += t[(int64_t)__ldg(ch + q) * NP + r];
  return s;
}

// restriction, phase 2: rc[C] = sum of t_f over the children of C (one thread per entry)
template <int NP>
__global__ void __launch_bounds__(kThreads) k_gather_big(int64_t nbc, const int64_t* __restrict__ cptr,
                                                        const int32_t* __restrict__ ch, const double* __restrict__ t,
                                                        double* __restrict__ rc) {
  pdl_entry();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nbc * NP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t C = e / NP;
    const int r = (int)(e - C * NP);
    rc[e] = child_sum<NP>(__ldg(cptr + C), __ldg(cptr + C + 1), r, ch, t);
  }
}

// phase 2 fused with the coarse level's first sweep from zero: bc = sum of the children's t,
// xc = omega D^{-1} bc
template <int NP>
__global__ void __launch_bounds__(kThreads, XDG_BIG_MINB) k_gather_smooth0_big(int64_t nbc, const int64_t* __restrict__ cptr,
                                                                const int32_t* __restrict__ ch,
                                                                const double* __restrict__ t,
                                                                const double* __restrict__ Dinv, double omega,
                                                                const double* __restrict__ omr,
                                                                double* __restrict__ bc, double* __restrict__ xc) {
  pdl_entry();
  constexpr int RPL = Shape<NP>::RPL;
  const int lane = threadIdx.x & 31;
  for (int64_t C = warp_id(); C < nbc; C += n_warps()) {
    const int64_t q0 = __ldg(cptr + C), q1 = __ldg(cptr + C + 1);
    double bv[RPL], z[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      bv[q] = r < NP ? child_sum<NP>(q0, q1, r, ch, t) : 0.0;
      if (r < NP) bc[C * NP + r] = bv[q];
    }
    block_gemv<NP>(Dinv + C * (NP * NP), lane, bv, z);
    const double om = omr ? __ldg(omr + C) : omega;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < NP) xc[C * NP + r] = om * z[q];
    }
  }
}

// xo_f = xi_f + R_f zc[agg[f]] (xo may equal xi)
template <int NP>
__global__ void __launch_bounds__(kThreads, XDG_BIG_MINB) k_prolong_big(int64_t nbf, const int32_t* __restrict__ agg,
                                                         const double* __restrict__ R, const double* __restrict__ zc,
                                                         const double* xi, double* xo) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  for (int64_t f = warp_id(); f < nbf; f += n_warps()) {
    const double* z = zc + (int64_t)__ldg(agg + f) * NP;
#pragma unroll
    for (int q = 0; q < Shape<NP>::RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < NP) {
        const double s = dot_row<NP>(R + f * (NP * NP) + r * NP, z, 0.0);
        xo[f * NP + r] = xi[f * NP + r] + s;
      }
    }
  }
}

// Galerkin product: one warp (CTA of 32 threads) per coarse row I; for every child i of I and
// every fine block (i, j): T = M_ij R_j into shared memory, then R_i^T T added to the coarse
// block (I, agg[j]). Coarse values are zero on entry.
template <int NP>
__global__ void __launch_bounds__(32) k_galerkin_big(int64_t nbc, const int64_t* __restrict__ cptr,
                                                    const int32_t* __restrict__ ch, const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ col, const double* __restrict__ val,
                                                    const int32_t* __restrict__ agg, const double* __restrict__ R,
                                                    const int64_t* __restrict__ crp,
                                                    const int32_t* __restrict__ ccol, double* __restrict__ cval) {
  pdl_entry();
  extern __shared__ double T[];  // NP x NP
  const int lane = threadIdx.x;
  for (int64_t I = blockIdx.x; I < nbc; I += gridDim.x) {
    const int64_t c0 = __ldg(crp + I), c1 = __ldg(crp + I + 1);
    for (int64_t tq = __ldg(cptr + I); tq < __ldg(cptr + I + 1); ++tq) {
      const int64_t i = __ldg(ch + tq);
      const double* Ri = R + i * (NP * NP);
      for (int64_t z = __ldg(rp + i); z < __ldg(rp + i + 1); ++z) {
        const int64_t j = __ldg(col + z);
        const double* Rj = R + j * (NP * NP);
        const double* Mz = val + z * (NP * NP);
        const int32_t J = __ldg(agg + j);
#pragma unroll
        for (int q = 0; q < Shape<NP>::RPL; ++q) {
          const int r = lane + 32 * q;
          if (r >= NP) continue;
          for (int n0 = 0; n0 < NP; n0 += 8) {
            double s[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) s[u] = 0.0;
            for (int a = 0; a < NP; ++a) {
              const double m = __ldg(Mz + r * NP + a);
#pragma unroll
              for (int u = 0; u < 8; ++u)
                if (n0 + u < NP) s[u] = fma(m, __ldg(Rj + a * NP + n0 + u), s[u]);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (n0 + u < NP) T[r * NP + n0 + u] = s[u];
          }
        }
        __syncwarp();
        int64_t lo = c0, hi = c1 - 1;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (__ldg(ccol + mid) < J) lo = mid + 1;
          else hi = mid;
        }
        double* dst = cval + lo * (NP * NP);
#pragma unroll
        for (int q = 0; q < Shape<NP>::RPL; ++q) {
          const int r = lane + 32 * q;
          if (r >= NP) continue;
          for (int n0 = 0; n0 < NP; n0 += 8) {
            double s[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) s[u] = 0.0;
            for (int a = 0; a < NP; ++a) {
              const double ri = __ldg(Ri + a * NP + r);
#pragma unroll
              for (int u = 0; u < 8; ++u)
                if (n0 + u < NP) s[u] = fma(ri, T[a * NP + n0 + u], s[u]);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (n0 + u < NP) dst[r * NP + n0 + u] += s[u];
          }
        }
        __syncwarp();
      }
    }
  }
}

// inverse of every diagonal block (one warp per block, the block and its factor in shared
// memory): Cholesky D = L L^T with the rows below the pivot spread over the lanes, X = L^{-1}
// one column per lane, D^{-1} = X^T X. *err = 1 for a block that is not positive definite (its
// inverse is left unwritten).
template <int NP>
__global__ void __launch_bounds__(32) k_diag_inv_big(int64_t nb, const int64_t* __restrict__ diag,
                                                    const double* __restrict__ val, double* __restrict__ Dinv,
                                                    int* err) {
  pdl_entry();
  extern __shared__ double sh[];
  double* A = sh;
  double* X = sh + NP * NP;
  const int lane = threadIdx.x;
  for (int64_t i = blockIdx.x; i < nb; i += gridDim.x) {
    const double* src = val + __ldg(diag + i) * (NP * NP);
    for (int e = lane; e < NP * NP; e += 32) A[e] = src[e];
    __syncwarp();
    bool ok = true;
    for (int j = 0; j < NP; ++j) {
      double s = A[j * NP + j];  // every lane computes the same pivot
      for (int p = 0; p < j; ++p) s -= A[j * NP + p] * A[j * NP + p];
      if (!(s > 0.0)) {
        ok = false;
        break;
      }
      const double d = sqrt(s);
      for (int q = j + 1 + lane; q < NP; q += 32) {
        double t = A[q * NP + j];
        for (int p = 0; p < j; ++p) t -= A[q * NP + p] * A[j * NP + p];
        A[q * NP + j] = t / d;
      }
      __syncwarp();
      if (lane == 0) A[j * NP + j] = d;
      __syncwarp();
    }
    if (!ok) {
      if (lane == 0) atomicOr(err, 1);
      __syncwarp();
      continue;
    }
    for (int c = lane; c < NP; c += 32)
      for (int q = c; q < NP; ++q) {
        double s = (q == c) ? 1.0 : 0.0;
        for (int p = c; p < q; ++p) s -= A[q * NP + p] * X[p * NP + c];
        X[q * NP + c] = s / A[q * NP + q];
      }
    __syncwarp();
    double* dst = Dinv + i * (NP * NP);
    for (int c = lane; c < NP; c += 32)
      for (int r = 0; r <= c; ++r) {
        double s = 0.0;
        for (int q = c; q < NP; ++q) s += X[q * NP + r] * X[q * NP + c];
        dst[r * NP + c] = s;
        dst[c * NP + r] = s;
      }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------
// launches: grid capped at one wave of resident CTAs (occupancy per kernel and device), with the
// programmatic-stream-serialization attribute unless XDG_PDL=0

bool pdl_on() {
  static const bool on = [] {
    const char* e = std::getenv("XDG_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

int wave(const void* k, int threads, size_t smem) {
  static std::mutex mu;
  struct Entry {
    const void* k;
    int dev, cap;
  };
  static std::vector<Entry> cache;
  int dev = 0, sms = 152, occ = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (auto& e : cache)
    if (e.k == k && e.dev == dev) return e.cap;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  cache.push_back(Entry{k, dev, occ * sms});
  return occ * sms;
}

template <class... P, class... A>
int launch(void (*k)(P...), int64_t grid, int threads, size_t smem, cudaStream_t s, A... a) {
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(grid, wave((const void*)k, threads, smem)));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_on() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, static_cast<P>(a)...);  // errors surface through cudaGetLastError
  return g;
}

template <int NP>
struct Impl {
  static void spmv(int grid, cudaStream_t s, const uint8_t* act, int64_t nb, const int64_t* rp, const int32_t* col,
                   const double* val, const double* x, const double* b, double* y, int mode) {
    if (mode) launch(k_spmv_big<NP, 1>, grid, kThreads, 0, s, nb, rp, col, val, x, b, y, act);
    else launch(k_spmv_big<NP, 0>, grid, kThreads, 0, s, nb, rp, col, val, x, b, y, act);
  }
  static void smooth(int grid, cudaStream_t s, int64_t nb, const int64_t* rp, const int32_t* col, const double* val,
                     const double* Dinv, double om, const double* omr, const double* b, const double* xi,
                     double* xo) {
    if (xi) launch(k_smooth_big<NP, false>, grid, kThreads, 0, s, nb, rp, col, val, Dinv, om, omr, b, xi, xo);
    else launch(k_smooth_big<NP, true>, grid, kThreads, 0, s, nb, rp, col, val, Dinv, om, omr, b, xi, xo);
  }
  static void bjsolve(int grid, cudaStream_t s, int64_t nb, const double* Dinv, const double* v, double* z) {
    launch(k_bjsolve_big<NP>, grid, kThreads, 0, s, nb, Dinv, v, z);
  }
  static void diagmul(int grid, cudaStream_t s, int64_t nb, const int64_t* dg, const double* val, const double* v,
                      double* w) {
    launch(k_diagmul_big<NP>, grid, kThreads, 0, s, nb, dg, val, v, w);
  }
  static void resid_rt(int grid, cudaStream_t s, int64_t nbf, const int64_t* rp, const int32_t* col,
                       const double* val, const double* R, const double* b, const double* x, double* t) {
    if (x) launch(k_resid_rt_big<NP, true>, grid, kThreads, 0, s, nbf, rp, col, val, R, b, x, t);
    else launch(k_resid_rt_big<NP, false>, grid, kThreads, 0, s, nbf, rp, col, val, R, b, x, t);
  }
  static void gather(int grid, cudaStream_t s, int64_t nbc, const int64_t* cptr, const int32_t* ch, const double* t,
                     double* rc) {
    launch(k_gather_big<NP>, grid, kThreads, 0, s, nbc, cptr, ch, t, rc);
  }
  static void gather_smooth0(int grid, cudaStream_t s, int64_t nbc, const int64_t* cptr, const int32_t* ch,
                             const double* t, const double* Dinv, double om, const double* omr, double* bc,
                             double* xc) {
    launch(k_gather_smooth0_big<NP>, grid, kThreads, 0, s, nbc, cptr, ch, t, Dinv, om, omr, bc, xc);
  }
  static void prolong(int grid, cudaStream_t s, int64_t nbf, const int32_t* agg, const double* R, const double* zc,
                      const double* xi, double* xo) {
    launch(k_prolong_big<NP>, grid, kThreads, 0, s, nbf, agg, R, zc, xi, xo);
  }
  static void galerkin(int, cudaStream_t s, int64_t nbc, const int64_t* cptr, const int32_t* ch, const int64_t* rp,
                       const int32_t* col, const double* val, const int32_t* agg, const double* R,
                       const int64_t* crp, const int32_t* ccol, double* cval) {
    launch(k_galerkin_big<NP>, nbc, 32, (size_t)NP * NP * sizeof(double), s, nbc, cptr, ch, rp, col, val, agg, R,
           crp, ccol, cval);
  }
  static void diag_inv(cudaStream_t s, int64_t nb, const int64_t* dg, const double* val, double* Dinv, int* err) {
    const size_t sm = 2 * (size_t)NP * NP * sizeof(double);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_diag_inv_big<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    launch(k_diag_inv_big<NP>, nb, 32, sm, s, nb, dg, val, Dinv, err);
  }
  static int spmv_dot(int grid, cudaStream_t s, int64_t nb, const int64_t* rp, const int32_t* col, const double* val,
                      const double* x, double* y, double* partial) {
    return launch(k_spmv_dot_big<NP>, std::min(grid, kMaxPartials), kThreads, 0, s, nb, rp, col, val, x, y, partial);
  }
  static Table make() {
    return Table{spmv, smooth, bjsolve, diagmul, resid_rt, gather, gather_smooth0, prolong, galerkin, diag_inv,
                 spmv_dot};
  }
};

}  // namespace

bool table_for(int np, Table* t) {
  switch (np) {
    case 35: *t = Impl<35>::make(); return true;
    case 56: *t = Impl<56>::make(); return true;
    default: return false;
  }
}

}  // namespace big
}  // namespace xdg
