// Low-precision variants of the cycle kernels: operator, block inverses and transfer blocks
// stored in FP32 or BF16 with one FP32 scale per Np x Np block (stored value = entry / scale),
// vectors in FP32, accumulation in FP32.
//
// Kummer, Smuda, Weber, arXiv 2003.02431, sec. 3.3: the low-order solves of the p-multigrid
// preconditioner may run in single precision as long as residuals are computed in double
// precision. Here the whole multigrid cycle (the preconditioner) runs in FP32/BF16 while the
// flexible CG around it keeps FP64 residuals and updates.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "xdg_kernels.cuh"

// minimum resident CTAs per SM requested for the FP32 row kernels
#ifndef XDG_LP_MINB
#define XDG_LP_MINB 1
#endif
// residual-restriction: load the transfer block's column before the row's dot product, so
// that its loads overlap the dot product's (measured faster at 64^3; the same prefetch of the
// block inverse slows the smoother down, which keeps its loads after the dot product)
#ifndef XDG_PREFETCH_EPI
#define XDG_PREFETCH_EPI 1
#endif

namespace xdg {

template <class T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<double>(double v) { return (float)v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// NP consecutive stored values -> FP32 registers (paired loads for even NP)
template <int NP, class T>
__device__ __forceinline__ void ldrow_f(const T* __restrict__ p, float (&v)[NP]) {
  if constexpr (std::is_same<T, float>::value && NP % 2 == 0) {
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int c = 0; c < NP / 2; ++c) {
      float2 t = __ldg(q + c);
      v[2 * c] = t.x;
      v[2 * c + 1] = t.y;
    }
  } else if constexpr (std::is_same<T, __nv_bfloat16>::value && NP % 2 == 0) {
    const __nv_bfloat162* q = reinterpret_cast<const __nv_bfloat162*>(p);
#pragma unroll
    for (int c = 0; c < NP / 2; ++c) {
      float2 t = __bfloat1622float2(q[c]);
      v[2 * c] = t.x;
      v[2 * c + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < NP; ++c) v[c] = to_f<T>(p[c]);
  }
}

// Loads of vectors that the same launch writes (the fused small-level cycle: COH = true) go
// through L2 only (__ldcg), which the barrier's fences make coherent across SMs; the read-only
// path (__ldg) serves vectors that no CTA writes during the launch (COH = false).
template <bool COH>
__device__ __forceinline__ float ldv(const float* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}
template <int NP, class VT, bool COH>
__device__ __forceinline__ void ldvec(const VT* __restrict__ p, float (&v)[NP]) {
  if constexpr (COH && std::is_same<VT, float>::value && NP % 2 == 0) {
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int c = 0; c < NP / 2; ++c) {
      float2 t = __ldcg(q + c);
      v[2 * c] = t.x;
      v[2 * c + 1] = t.y;
    }
  } else if constexpr (COH && std::is_same<VT, float>::value) {
#pragma unroll
    for (int c = 0; c < NP; ++c) v[c] = __ldcg(p + c);
  } else {
    ldrow_f<NP, VT>(p, v);
  }
}

// sum_z s_z (A_z[r][:] . x[col z][:]) in FP32
template <int NP, class TS, class VT, bool COH = false>
__device__ __forceinline__ float row_dot_lp(int64_t z0, int64_t z1, int r, const int32_t* __restrict__ col,
                                            const TS* __restrict__ val, const float* __restrict__ sc,
                                            const VT* __restrict__ x) {
  constexpr int CH = Chunk<NP>::F32;
  float acc = 0.0f;
  for (int64_t z = z0; z < z1; z += CH) {
    int32_t cc[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) cc[u] = (z + u < z1) ? __ldg(col + z + u) : -1;
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (cc[u] < 0) continue;
      float a[NP], xv[NP];
      ldrow_f<NP, TS>(val + (z + u) * (NP * NP) + r * NP, a);
      ldvec<NP, VT, COH>(x + (int64_t)cc[u] * NP, xv);
      float s = 0.0f;
#pragma unroll
      for (int c = 0; c < NP; ++c) s = fmaf(a[c], xv[c], s);
      acc = fmaf(__ldg(sc + z + u), s, acc);
    }
  }
  return acc;
}

// Split rows (small levels): the GPW groups of a warp share one block row, group g taking the
// blocks z0 + g, z0 + g + GPW, ...; split_sum adds the groups' partial sums in group order
// (the same value in every group). This shortens the per-row chain of dependent loads, which
// bounds the small levels, by the factor GPW.
template <int NP, class TS, class VT, bool COH = false>
__device__ __forceinline__ float row_dot_lp_part(int64_t z0, int64_t z1, int g, int r,
                                                 const int32_t* __restrict__ col, const TS* __restrict__ val,
                                                 const float* __restrict__ sc, const VT* __restrict__ x) {
  constexpr int GPW = Grp<NP>::GPW;
  constexpr int CH = Chunk<NP>::F32;
  float acc = 0.0f;
  for (int64_t z = z0 + g; z < z1; z += (int64_t)CH * GPW) {
    int32_t cc[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) cc[u] = (z + u * GPW < z1) ? __ldg(col + z + u * GPW) : -1;
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (cc[u] < 0) continue;
      const int64_t zz = z + u * GPW;
      float a[NP], xv[NP];
      ldrow_f<NP, TS>(val + zz * (NP * NP) + r * NP, a);
      ldvec<NP, VT, COH>(x + (int64_t)cc[u] * NP, xv);
      float s = 0.0f;
#pragma unroll
      for (int c = 0; c < NP; ++c) s = fmaf(a[c], xv[c], s);
      acc = fmaf(__ldg(sc + zz), s, acc);
    }
  }
  return acc;
}

template <int NP>
__device__ __forceinline__ float split_sum(float part, int r) {
  constexpr int GPW = Grp<NP>::GPW;
  constexpr unsigned M = (GPW * NP == 32) ? 0xffffffffu : ((1u << (GPW * NP)) - 1u);
  float t = __shfl_sync(M, part, r);
#pragma unroll
  for (int gg = 1; gg < GPW; ++gg) t += __shfl_sync(M, part, gg * NP + r);
  return t;
}

// y = M x (MODE 0) or b - M x (MODE 1); VT = vector type of x, b and y (float or double)
template <int NP, class TS, class VT, int MODE, bool SPL = false>
__global__ void __launch_bounds__(kThreads, XDG_LP_MINB) k_spmv_lp(int64_t nb, const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col,
                                                     const TS* __restrict__ val, const float* __restrict__ sc,
                                                     const VT* __restrict__ x, const VT* __restrict__ b,
                                                     VT* __restrict__ y) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if constexpr (SPL) {
    for (int64_t i = warp; i < nb; i += nw) {
      const float acc = split_sum<NP>(row_dot_lp_part<NP, TS, VT>(__ldg(rp + i), __ldg(rp + i + 1), g, r, col,
                                                                  val, sc, x), r);
      if (g == 0) y[i * NP + r] = MODE ? (VT)(to_f<VT>(b[i * NP + r]) - acc) : (VT)acc;
    }
  } else {
    for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
      float acc = row_dot_lp<NP, TS, VT>(__ldg(rp + i), __ldg(rp + i + 1), r, col, val, sc, x);
      y[i * NP + r] = MODE ? (VT)(to_f<VT>(b[i * NP + r]) - acc) : (VT)acc;
    }
  }
}

template <int NP, class TS>
__device__ __forceinline__ float block_gemv_lp(const TS* __restrict__ W, float s, int r, int base,
                                               unsigned mask, float v) {
  float w[NP];
  ldrow_f<NP, TS>(W + r * NP, w);
  float acc = 0.0f;
#pragma unroll
  for (int c = 0; c < NP; ++c) acc = fmaf(w[c], __shfl_sync(mask, v, base + c), acc);
  return s * acc;
}

__device__ __forceinline__ int64_t grid_warp() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t grid_warps() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }
__device__ __forceinline__ int64_t grid_thread() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t grid_threads() { return (int64_t)gridDim.x * blockDim.x; }

// The cycle's FP32 steps as functions of (warp index, number of warps) or (thread index, number
// of threads): the kernels below run one step per launch, the fused coarse cycle runs several
// steps in one launch with grid barriers between them.

// damped block Jacobi in FP32: xo = xi + omega D^{-1} (b - M xi). The block inverses are
// computed in FP64 and stored in FP32 in both modes: rounding the inverse of an ill-conditioned
// cut-cell block to BF16 loses it.
template <int NP, class TS, bool ZERO, bool SPL, bool COH = false>
__device__ __forceinline__ void smooth_lp_rows(int64_t warp, int64_t nw, int64_t nb, const int64_t* __restrict__ rp,
                                               const int32_t* __restrict__ col, const TS* __restrict__ val,
                                               const float* __restrict__ sc, const float* __restrict__ Dinv,
                                               const float* __restrict__ dsc, float omega,
                                               const float* __restrict__ omr, const float* __restrict__ b,
                                               const float* __restrict__ xi, float* __restrict__ xo,
                                               const uint8_t* __restrict__ act) {
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  if constexpr (SPL) {
    for (int64_t i = warp; i < nb; i += nw) {
      if (act && !act[i]) continue;
      float res = ldv<COH>(b + i * NP + r);
      if (!ZERO)
        res -= split_sum<NP>(row_dot_lp_part<NP, TS, float, COH>(__ldg(rp + i), __ldg(rp + i + 1), g, r, col, val,
                                                                 sc, xi), r);
      float z = block_gemv_lp<NP, float>(Dinv + i * (NP * NP), __ldg(dsc + i), r, g * NP, mask, res);
      const float om = omr ? __ldg(omr + i) : omega;
      if (g == 0) xo[i * NP + r] = ZERO ? om * z : fmaf(om, z, ldv<COH>(xi + i * NP + r));
    }
  } else {
    for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
      if (act && !act[i]) continue;
      float res = ldv<COH>(b + i * NP + r);
      if (!ZERO) res -= row_dot_lp<NP, TS, float, COH>(__ldg(rp + i), __ldg(rp + i + 1), r, col, val, sc, xi);
      float z = block_gemv_lp<NP, float>(Dinv + i * (NP * NP), __ldg(dsc + i), r, g * NP, mask, res);
      const float om = omr ? __ldg(omr + i) : omega;  // per-row damping in batches
      xo[i * NP + r] = ZERO ? om * z : fmaf(om, z, ldv<COH>(xi + i * NP + r));
    }
  }
}

template <int NP, class TS, bool ZERO, bool SPL = false>
__global__ void __launch_bounds__(kThreads, XDG_LP_MINB) k_smooth_lp(int64_t nb, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ col,
                                                       const TS* __restrict__ val, const float* __restrict__ sc,
                                                       const float* __restrict__ Dinv, const float* __restrict__ dsc,
                                                       float omega, const float* __restrict__ omr,
                                                       const float* __restrict__ b,
                                                       const float* __restrict__ xi, float* __restrict__ xo,
                                                       const uint8_t* __restrict__ act) {
  pdl_entry();
  smooth_lp_rows<NP, TS, ZERO, SPL>(grid_warp(), grid_warps(), nb, rp, col, val, sc, Dinv, dsc, omega, omr, b, xi,
                                    xo, act);
}

// restriction phase 1 in FP32: t_f = R_f^T (b_f - M_f x). The operator is read from its FP32
// copy in both modes (TA = float): a BF16-rounded operator is not positive definite on the
// smooth modes the coarse levels correct (2^-9 cond(M) >> 1); TR is the transfer storage.
template <int NP, class TA, class TR, bool RESID, bool SPL, bool COH = false>
__device__ __forceinline__ void resid_rt_lp_rows(int64_t warp, int64_t nw, int64_t nbf,
                                                 const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                 const TA* __restrict__ val, const float* __restrict__ sc,
                                                 const TR* __restrict__ R, const float* __restrict__ rsc,
                                                 const float* __restrict__ b, const float* __restrict__ x,
                                                 float* __restrict__ t, const uint8_t* __restrict__ act) {
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  const int base = g * NP;
  if constexpr (SPL) {
    for (int64_t f = warp; f < nbf; f += nw) {
      if (act && !act[f]) continue;
      float res = ldv<COH>(b + f * NP + r);
      if (RESID)
        res -= split_sum<NP>(row_dot_lp_part<NP, TA, float, COH>(__ldg(rp + f), __ldg(rp + f + 1), g, r, col, val,
                                                                 sc, x), r);
      const TR* Rf = R + f * (NP * NP);
      float s = 0.0f;
#pragma unroll
      for (int m = 0; m < NP; ++m) s = fmaf(to_f<TR>(Rf[m * NP + r]), __shfl_sync(mask, res, base + m), s);
      if (g == 0) t[f * NP + r] = __ldg(rsc + f) * s;
    }
  } else {
    for (int64_t f = warp * GPW + g; f < nbf; f += nw * GPW) {
      if (act && !act[f]) continue;
      const TR* Rf = R + f * (NP * NP);
      float rc[NP];
      if (XDG_PREFETCH_EPI) {
#pragma unroll
        for (int m = 0; m < NP; ++m) rc[m] = to_f<TR>(Rf[m * NP + r]);
      }
      float res = ldv<COH>(b + f * NP + r);
      if (RESID) res -= row_dot_lp<NP, TA, float, COH>(__ldg(rp + f), __ldg(rp + f + 1), r, col, val, sc, x);
      float s = 0.0f;
#pragma unroll
      for (int m = 0; m < NP; ++m)
        s = fmaf(XDG_PREFETCH_EPI ? rc[m] : to_f<TR>(Rf[m * NP + r]), __shfl_sync(mask, res, base + m), s);
      t[f * NP + r] = __ldg(rsc + f) * s;
    }
  }
}

template <int NP, class TA, class TR, bool RESID, bool SPL = false>
__global__ void __launch_bounds__(kThreads, XDG_LP_MINB) k_resid_rt_lp(int64_t nbf, const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col,
                                                         const TA* __restrict__ val, const float* __restrict__ sc,
                                                         const TR* __restrict__ R, const float* __restrict__ rsc,
                                                         const float* __restrict__ b, const float* __restrict__ x,
                                                         float* __restrict__ t, const uint8_t* __restrict__ act) {
  pdl_entry();
  resid_rt_lp_rows<NP, TA, TR, RESID, SPL>(grid_warp(), grid_warps(), nbf, rp, col, val, sc, R, rsc, b, x, t, act);
}

// ------------------------------------------------------------------------------------------
// Level 1 with symmetric storage. M = M^T (the SIP operator is symmetric, sec. 4) is kept as its
// diagonal and right-of-diagonal blocks only, in a compact BSR (urp, ucol, uval, usc: ascending
// columns, the diagonal block first in each row); a block left of the diagonal, (i, j) with
// j < i, is read as the transpose of its mirror (j, i) (SymL: per row i the columns j in
// ascending order and the mirror blocks' indices in the compact storage). A row's sum runs over
// its left blocks, then its diagonal and right blocks: ascending columns with the same values,
// scales and operation order as the full storage, so the results are bitwise those of the
// full-storage kernels. Mirror blocks belong to rows at most about one mesh plane apart, all of
// which are in flight together: the second read is an L2 hit and HBM streams about half the
// operator.
struct SymL {
  const int64_t* lrp;
  const int32_t* lcol;
  const int32_t* lblk;
};

// sum over the blocks of row i (lane r): left blocks transposed, then the stored ones
template <int NP>
__device__ __forceinline__ float row_dot_sym(int64_t i, int r, const int64_t* __restrict__ urp,
                                             const int32_t* __restrict__ ucol, const float* __restrict__ uval,
                                             const float* __restrict__ usc, SymL L, const float* __restrict__ x) {
  constexpr int CH = Chunk<NP>::F32;
  float acc = 0.0f;
  const int64_t l0 = __ldg(L.lrp + i), l1 = __ldg(L.lrp + i + 1);
  for (int64_t z = l0; z < l1; z += CH) {
    int32_t cc[CH], bb[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      cc[u] = (z + u < l1) ? __ldg(L.lcol + z + u) : -1;
      bb[u] = (z + u < l1) ? __ldg(L.lblk + z + u) : 0;
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (cc[u] < 0) continue;
      const float* B = uval + (int64_t)bb[u] * (NP * NP) + r;  // column r of the mirror block
      float a[NP], xv[NP];
#pragma unroll
      for (int c = 0; c < NP; ++c) a[c] = __ldg(B + c * NP);
      ldvec<NP, float, false>(x + (int64_t)cc[u] * NP, xv);
      float sv = 0.0f;
#pragma unroll
      for (int c = 0; c < NP; ++c) sv = fmaf(a[c], xv[c], sv);
      acc = fmaf(__ldg(usc + bb[u]), sv, acc);
    }
  }
  const int64_t z0 = __ldg(urp + i), z1 = __ldg(urp + i + 1);
  for (int64_t z = z0; z < z1; z += CH) {
    int32_t cc[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) cc[u] = (z + u < z1) ? __ldg(ucol + z + u) : -1;
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (cc[u] < 0) continue;
      float a[NP], xv[NP];
      ldrow_f<NP, float>(uval + (z + u) * (NP * NP) + r * NP, a);
      ldvec<NP, float, false>(x + (int64_t)cc[u] * NP, xv);
      float sv = 0.0f;
#pragma unroll
      for (int c = 0; c < NP; ++c) sv = fmaf(a[c], xv[c], sv);
      acc = fmaf(__ldg(usc + z + u), sv, acc);
    }
  }
  return acc;
}

// the block-Jacobi sweep of smooth_lp_rows (one row per group, nonzero guess) on the symmetric
// storage
// resident CTAs per SM requested for the symmetric-storage row kernels (their two loops need
// more registers than the full-storage ones; without the cap the restriction drops to 2 CTAs)
#ifndef XDG_SYM_MINB
#define XDG_SYM_MINB 4
#endif
template <int NP>
__global__ void __launch_bounds__(kThreads, XDG_SYM_MINB) k_smooth_lp_sym(
    int64_t nb, const int64_t* __restrict__ urp, const int32_t* __restrict__ ucol, const float* __restrict__ uval,
    const float* __restrict__ usc, SymL L, const float* __restrict__ Dinv, const float* __restrict__ dsc, float omega,
    const float* __restrict__ omr, const float* __restrict__ b, const float* __restrict__ xi, float* __restrict__ xo,
    const uint8_t* __restrict__ act) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  const int64_t warp = grid_warp(), nw = grid_warps();
  for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
    if (act && !act[i]) continue;
    float res = b[i * NP + r];
    res -= row_dot_sym<NP>(i, r, urp, ucol, uval, usc, L, xi);
    float z = block_gemv_lp<NP, float>(Dinv + i * (NP * NP), __ldg(dsc + i), r, g * NP, mask, res);
    const float om = omr ? __ldg(omr + i) : omega;
    xo[i * NP + r] = fmaf(om, z, xi[i * NP + r]);
  }
}

// restriction phase 1 of resid_rt_lp_rows (one row per group) on the symmetric storage
template <int NP, class TR>
__global__ void __launch_bounds__(kThreads, XDG_SYM_MINB) k_resid_rt_lp_sym(
    int64_t nbf, const int64_t* __restrict__ urp, const int32_t* __restrict__ ucol, const float* __restrict__ uval,
    const float* __restrict__ usc, SymL L, const TR* __restrict__ R, const float* __restrict__ rsc,
    const float* __restrict__ b, const float* __restrict__ x, float* __restrict__ t, const uint8_t* __restrict__ act) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  const int base = g * NP;
  const int64_t warp = grid_warp(), nw = grid_warps();
  for (int64_t f = warp * GPW + g; f < nbf; f += nw * GPW) {
    if (act && !act[f]) continue;
    const TR* Rf = R + f * (NP * NP);
    float rc[NP];
    if (XDG_PREFETCH_EPI) {
#pragma unroll
      for (int m = 0; m < NP; ++m) rc[m] = to_f<TR>(Rf[m * NP + r]);
    }
    float res = b[f * NP + r];
    res -= row_dot_sym<NP>(f, r, urp, ucol, uval, usc, L, x);
    float s = 0.0f;
#pragma unroll
    for (int m = 0; m < NP; ++m)
      s = fmaf(XDG_PREFETCH_EPI ? rc[m] : to_f<TR>(Rf[m * NP + r]), __shfl_sync(mask, res, base + m), s);
    t[f * NP + r] = __ldg(rsc + f) * s;
  }
}

// the compact storage's values gathered from the full copy (umap: full index of each block)
__global__ void k_gather_blocks(int64_t nblk, int np2, const int64_t* __restrict__ umap, const float* __restrict__ v,
                                const float* __restrict__ sc, float* __restrict__ uv, float* __restrict__ usc) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t z = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; z < nblk; z += nw) {
    const int64_t zf = __ldg(umap + z);
    for (int k = lane; k < np2; k += 32) uv[z * np2 + k] = v[zf * np2 + k];
    if (lane == 0) usc[z] = sc[zf];
  }
}

// flag (*bad = 1) any pair of mirror blocks (i, j), (j, i) of the FP64 operator that are not
// exact transposes of each other (pos: full index of every left block and of its mirror)
__global__ void k_check_mirror(int64_t npair, int np, const int64_t* __restrict__ pos, const double* __restrict__ val,
                               int* __restrict__ bad) {
  pdl_entry();
  const int64_t np2 = (int64_t)np * np;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < npair * np2; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / np2;
    const int rc = (int)(e - k * np2);
    const int rr = rc / np, cc = rc - rr * np;
    const int64_t zl = __ldg(pos + 2 * k), zu = __ldg(pos + 2 * k + 1);
    if (val[zl * np2 + rr * np + cc] != val[zu * np2 + cc * np + rr]) atomicOr(bad, 1);
  }
}

// restriction phase 2 in FP32 (children in ascending order)
template <int NP, bool COH = false>
__device__ __forceinline__ void gather_lp_elems(int64_t tid, int64_t nt, int64_t nbc, const int64_t* __restrict__ cptr,
                                                const int32_t* __restrict__ ch, const float* __restrict__ t,
                                                float* __restrict__ rc) {
  for (int64_t e = tid; e < nbc * NP; e += nt) {
    const int64_t C = e / NP;
    const int r = (int)(e - C * NP);
    rc[e] = child_sum<NP, float, float, COH>(__ldg(cptr + C), __ldg(cptr + C + 1), r, ch, t);
  }
}

template <int NP>
__global__ void __launch_bounds__(kThreads) k_gather_lp(int64_t nbc, const int64_t* __restrict__ cptr,
                                                       const int32_t* __restrict__ ch,
                                                       const float* __restrict__ t, float* __restrict__ rc) {
  pdl_entry();
  gather_lp_elems<NP>(grid_thread(), grid_threads(), nbc, cptr, ch, t, rc);
}

// phase 2 fused with the first sweep of the coarse level from a zero guess (FP32)
template <int NP, bool COH = false>
__device__ __forceinline__ void gather_smooth0_lp_rows(int64_t warp, int64_t nw, int64_t nbc,
                                                       const int64_t* __restrict__ cptr,
                                                       const int32_t* __restrict__ ch, const float* __restrict__ t,
                                                       const float* __restrict__ Dinv, const float* __restrict__ dsc,
                                                       float omega, const float* __restrict__ omr,
                                                       float* __restrict__ bc, float* __restrict__ xc) {
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  for (int64_t C = warp * GPW + g; C < nbc; C += nw * GPW) {
    float bv = child_sum<NP, float, float, COH>(__ldg(cptr + C), __ldg(cptr + C + 1), r, ch, t);
    bc[C * NP + r] = bv;
    float z = block_gemv_lp<NP, float>(Dinv + C * (NP * NP), __ldg(dsc + C), r, g * NP, mask, bv);
    xc[C * NP + r] = (omr ? __ldg(omr + C) : omega) * z;
  }
}

template <int NP>
__global__ void __launch_bounds__(kThreads) k_gather_smooth0_lp(int64_t nbc, const int64_t* __restrict__ cptr,
                                                               const int32_t* __restrict__ ch,
                                                               const float* __restrict__ t,
                                                               const float* __restrict__ Dinv,
                                                               const float* __restrict__ dsc, float omega,
                                                               const float* __restrict__ omr,
                                                               float* __restrict__ bc, float* __restrict__ xc) {
  pdl_entry();
  gather_smooth0_lp_rows<NP>(grid_warp(), grid_warps(), nbc, cptr, ch, t, Dinv, dsc, omega, omr, bc, xc);
}

// xo_f = xi_f + R_f zc[agg[f]] in FP32 (xo may equal xi)
template <int NP, class TS, bool COH = false>
__device__ __forceinline__ void prolong_lp_rows(int64_t warp, int64_t nw, int64_t nbf, const int32_t* __restrict__ agg,
                                                const TS* __restrict__ R, const float* __restrict__ rsc,
                                                const float* __restrict__ zc, const float* xi, float* xo,
                                                const uint8_t* __restrict__ act) {
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  for (int64_t f = warp * GPW + g; f < nbf; f += nw * GPW) {
    if (act && !act[f]) continue;
    float a[NP], z[NP];
    ldrow_f<NP, TS>(R + f * (NP * NP) + r * NP, a);
    ldvec<NP, float, COH>(zc + (int64_t)__ldg(agg + f) * NP, z);
    float s = 0.0f;
#pragma unroll
    for (int n = 0; n < NP; ++n) s = fmaf(a[n], z[n], s);
    xo[f * NP + r] = fmaf(__ldg(rsc + f), s, ldv<COH>(xi + f * NP + r));
  }
}

template <int NP, class TS>
__global__ void __launch_bounds__(kThreads) k_prolong_lp(int64_t nbf, const int32_t* __restrict__ agg,
                                                        const TS* __restrict__ R, const float* __restrict__ rsc,
                                                        const float* __restrict__ zc, const float* xi, float* xo,
                                                        const uint8_t* __restrict__ act) {
  pdl_entry();
  prolong_lp_rows<NP, TS>(grid_warp(), grid_warps(), nbf, agg, R, rsc, zc, xi, xo, act);
}

// stored copy of Np x Np blocks: scale s = max |entry| (as float, 1 for a zero block),
// stored entry = round(entry / s) to TS (round to nearest even; BF16 through FP32)
template <class TS>
__device__ __forceinline__ TS store_lp(double v);
template <>
__device__ __forceinline__ float store_lp<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 store_lp<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }

template <class TS>
__global__ void k_make_lp(int64_t nblk, int np2, const double* __restrict__ src, TS* __restrict__ dst,
                          float* __restrict__ scale) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (blk >= nblk) return;
  const double* s = src + blk * np2;
  double m = 0.0;
  for (int e = lane; e < np2; e += 32) m = fmax(m, fabs(s[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  float sf = (m > 0.0) ? (float)m : 1.0f;
  const double sd = (double)sf;
  for (int e = lane; e < np2; e += 32) dst[blk * np2 + e] = store_lp<TS>(s[e] / sd);
  if (lane == 0) scale[blk] = sf;
}

// act (optional): entries of rows i = e / np with act[i] == 0 are skipped
__global__ void k_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b,
                      const uint8_t* __restrict__ act, int np) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!act || act[i / np]) b[i] = (float)a[i];
}

__global__ void k_f2d(int64_t n, const float* __restrict__ a, double* __restrict__ b,
                      const uint8_t* __restrict__ act, int np) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!act || act[i / np]) b[i] = (double)a[i];
}

__global__ void k_axpy_f(int64_t n, float a, const float* __restrict__ x, float* __restrict__ y) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fmaf(a, x[i], y[i]);
}

__global__ void k_copy_f(int64_t n, const float* __restrict__ a, float* __restrict__ b) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// flexible CG (one previous direction kept): beta = -(z_new . q) / (p . q), q = M p
// end of a flexible-CG step: z = widened FP32 cycle result; per-CTA parts of r . z and z . q
// (partial[2 b], partial[2 b + 1])
__global__ void __launch_bounds__(kThreads) k_fcg_tail(int64_t n, const float* __restrict__ zf,
                                                      const double* __restrict__ r, const double* __restrict__ q,
                                                      double* __restrict__ z, double* __restrict__ partial) {
  pdl_entry();
  double a = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = (double)zf[i];
    z[i] = zi;
    a = fma(r[i], zi, a);
    c = fma(zi, q[i], c);
  }
  a = block_sum(a);
  c = block_sum(c);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = c;
  }
}

// the same partial sums of r . z and z . q for an FP64 z (the cycle's output after the learned
// correction was added to it)
__global__ void __launch_bounds__(kThreads) k_fcg_dots(int64_t n, const double* __restrict__ r,
                                                      const double* __restrict__ q, const double* __restrict__ z,
                                                      double* __restrict__ partial) {
  pdl_entry();
  double a = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = z[i];
    a = fma(r[i], zi, a);
    c = fma(zi, q[i], c);
  }
  a = block_sum(a);
  c = block_sum(c);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = c;
  }
}

// rz, zq from the partial sums, then the flexible-CG beta = -zq / pq
__global__ void __launch_bounds__(kThreads) k_fcg_beta_final(int np, const double* __restrict__ partial, PcgScal* S) {
  pdl_entry();
  const double rz = sum_partials(np, partial, 2, 0);
  const double zq = sum_partials(np, partial, 2, 1);
  if (threadIdx.x == 0) {
    S->rz = rz;
    S->zq = zq;
    const double pq = S->pq;
    if (!(pq > 0.0) || !isfinite(zq)) {
      S->bad = 1;
      S->beta = 0.0;
    } else {
      S->beta = -zq / pq;
    }
  }
}

__global__ void k_fcg_beta(PcgScal* S) {
  pdl_entry();
  double pq = S->pq, zq = S->zq;
  if (!(pq > 0.0) || !isfinite(zq)) {
    S->bad = 1;
    S->beta = 0.0;
  } else {
    S->beta = -zq / pq;
  }
}

}  // namespace xdg
