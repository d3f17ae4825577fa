// The level-1 operator apply of the outer Krylov method with FP64 accuracy on the FP32 pipe.
//
// GB300 executes FP64 fused multiply-adds at 1/64 of its FP32 rate, so the FP64 product
// q = M p (one FP64 FMA per block entry) is bound by the FP64 pipe, not by HBM. Here every
// number is held as an unevaluated sum of two FP32 numbers (hi + lo, "double-float": Dekker,
// "A floating-point technique for extending the available precision", Numer. Math. 18, 1971)
// scaled by a power of two per block:
//   M_z = 2^ea[z] (H_z + L_z),   x_j = 2^ex[j] (h_j + l_j),   H, L, h, l in FP32
// and each block's contribution M_z x_j is accumulated in double-float arithmetic:
//   a_h x_h exactly as p + e (Dekker's product: p = fl(a_h x_h), e = fma(a_h, x_h, -p)),
//   the cross terms a_h x_l + a_l x_h in FP32 (they are 2^-24 smaller), the running sum of the
//   p's with Knuth's TwoSum (its rounding error kept exactly), all errors summed in FP32;
// the block results are then scaled by 2^(ea+ex) (exact) and summed in FP64. Per block entry
// this is 12 FP32 operations and 0.2 FP64 operations (Np = 10); the bytes read equal those of
// the FP64 product (8 per entry). The error is a few units of 2^-48 relative to sum |a||x| of
// the row, against 2^-53 for FP64: ample for the outer method's residuals (its tolerances are
// above 1e-13) and checked against the oracle's FP64 product in the tests.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "xdg_kernels.cuh"
#include "xdg_kernels_lp.cuh"

namespace xdg {

// 2^k as a double, built from its bits (k clamped to the normal range)
__device__ __forceinline__ double pow2_d(int k) {
  k = max(-1022, min(1023, k));
  return __longlong_as_double((long long)(k + 1023) << 52);
}

// exponent e with |v| = f 2^e, f in [0.5, 1) (normal v); 0 for v = 0, inf or nan
__device__ __forceinline__ int exp_of(double v) {
  const long long b = __double_as_longlong(v);
  const int f = (int)((b >> 52) & 0x7ff);
  if (f == 0x7ff) return 0;
  if (f == 0) return v == 0.0 ? 0 : -1022;
  return f - 1022;
}

// v -> (hi, lo) with hi = fl32(v), lo = fl32(v - hi); v already scaled to about [0.5, 1)
__device__ __forceinline__ float2 split_df(double v) {
  const float h = __double2float_rn(v);
  const float l = __double2float_rn(v - (double)h);
  return make_float2(h, l);
}

// blocks of a row whose loads are issued together, and resident CTAs per SM requested
#ifndef XDG_CH_PAIR
#define XDG_CH_PAIR 4
#endif
#ifndef XDG_PAIR_MINB
#define XDG_PAIR_MINB 4
#endif

// x 2^k as a double, exactly, built from the float's bits (integer operations instead of an
// FP64-pipe conversion and multiply); false for zero-exponent (subnormal), infinite or NaN x,
// k outside the range pow2_d handles, or a result outside the normal range
__device__ __forceinline__ bool f2d_scaled(float x, int k, double& out) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  if ((u & 0x7fffffffu) == 0u) {
    out = __longlong_as_double((long long)sgn);
    return true;
  }
  if (e == 0u || e == 0xffu || k < -1022 || k > 1023) return false;
  const int E = (int)e - 127 + 1023 + k;
  if (E < 1 || E > 2046) return false;
  out = __longlong_as_double((long long)(sgn | ((unsigned long long)E << 52) |
                                         ((unsigned long long)(u & 0x7fffffu) << 29)));
  return true;
}

// split_df(v 2^-k) with the scaling and the widening of hi done by integer operations where the
// results are normal (bitwise the same pair; two FP64-pipe operations fewer per entry)
__device__ __forceinline__ float2 split_scaled(double v, int k) {
  const long long b = __double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7ff);
  double vs;
  if (v == 0.0) {
    vs = v;
  } else if (E != 0 && E != 0x7ff && -k >= -1022 && -k <= 1023 && E - k >= 1 && E - k <= 2046) {
    vs = __longlong_as_double((b & ~(0x7ffLL << 52)) | ((long long)(E - k) << 52));
  } else {
    vs = v * pow2_d(-k);
  }
  const float h = __double2float_rn(vs);
  double hd;
  if (!f2d_scaled(h, 0, hd)) hd = (double)h;
  const float l = __double2float_rn(__dsub_rn(vs, hd));
  return make_float2(h, l);
}

// Sum of a row's block results (hi + lo) 2^k in FP64. hi 2^k and lo 2^k are exact, so adding them
// equals the fused multiply-add fma((double)hi, 2^k, acc) bit for bit; they are built with
// integer operations (two FP64-pipe additions a block instead of two conversions and two FMAs:
// the FP64 pipe was 61 % busy with the conversions), with the FMA form as the fallback. A
// double-float sum relative to the row's first block, converted once per row, measured slower.
struct RowAcc {
  double acc = 0.0;
  __device__ __forceinline__ void add(float hi, float lo, int k) {
    double a, b;
    if (f2d_scaled(hi, k, a) && f2d_scaled(lo, k, b)) {
      acc = __dadd_rn(acc, a);
      acc = __dadd_rn(acc, b);
    } else {
      const double sc = pow2_d(k);
      acc = fma((double)hi, sc, acc);
      acc = fma((double)lo, sc, acc);
    }
  }
  __device__ __forceinline__ double result() const { return acc; }
};

// NP consecutive float2 -> registers (16-byte loads when the row is 16-byte aligned)
template <int NP>
__device__ __forceinline__ void ldrow_df(const float2* __restrict__ p, float2 (&v)[NP]) {
  if constexpr (NP % 2 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int c = 0; c < NP / 2; ++c) {
      const float4 t = __ldg(q + c);
      v[2 * c] = make_float2(t.x, t.y);
      v[2 * c + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int c = 0; c < NP; ++c) v[c] = __ldg(p + c);
  }
}

// sum_c a[c] x[c] of one block row in double-float arithmetic; result hi + lo (FP32 pair).
// The intrinsics (_rn) keep the compiler from contracting a product into a later sum, which
// would break the exactness of Dekker's product and of TwoSum.
template <int NP>
__device__ __forceinline__ void block_dot_df(const float2 (&a)[NP], const float2 (&x)[NP], float& hi, float& lo) {
  float s = 0.0f, c = 0.0f;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float p = __fmul_rn(a[k].x, x[k].x);
    float e = __fmaf_rn(a[k].x, x[k].x, -p);           // a_h x_h = p + e exactly
    e = __fmaf_rn(a[k].x, x[k].y, e);                   // + a_h x_l
    e = __fmaf_rn(a[k].y, x[k].x, e);                   // + a_l x_h
    const float t = __fadd_rn(s, p);                    // TwoSum(s, p) = t + e2 exactly
    const float bp = __fsub_rn(t, s);
    const float e2 = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, e2));
  }
  hi = s;
  lo = c;
}

// acc over the block row (lane r): blocks in increasing z, each block's double-float dot
// scaled by 2^(ea + ex) and added in FP64
template <int NP>
__device__ __forceinline__ double row_dot_df(int64_t z0, int64_t z1, int r, const int32_t* __restrict__ col,
                                             const float2* __restrict__ val2, const int* __restrict__ ea,
                                             const float2* __restrict__ x2, const int* __restrict__ ex) {
  constexpr int CH = NP <= 10 ? XDG_CH_PAIR : 1;
  RowAcc acc;
  for (int64_t z = z0; z < z1; z += CH) {
    int32_t cc[CH];
    int ee[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      cc[u] = (z + u < z1) ? __ldg(col + z + u) : -1;
      ee[u] = (z + u < z1) ? __ldg(ea + z + u) : 0;
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (cc[u] < 0) continue;
      float2 a[NP], xv[NP];
      ldrow_df<NP>(val2 + (z + u) * (NP * NP) + r * NP, a);
      ldrow_df<NP>(x2 + (int64_t)cc[u] * NP, xv);
      const int k = ee[u] + __ldg(ex + cc[u]);
      float hi, lo;
      block_dot_df<NP>(a, xv, hi, lo);
      acc.add(hi, lo, k);
    }
  }
  return acc.result();
}

// y = M x from the double-float operator and vector (rows spread as in k_spmv_dot) and
// partial[blockIdx.x] = this CTA's part of x . y (x in FP64)
template <int NP>
__global__ void __launch_bounds__(kThreads, XDG_PAIR_MINB) k_spmv_dot_df(int64_t nb, const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col,
                                                         const float2* __restrict__ val2, const int* __restrict__ ea,
                                                         const float2* __restrict__ x2, const int* __restrict__ ex,
                                                         const double* __restrict__ x, double* __restrict__ y,
                                                         double* __restrict__ partial, const uint8_t* __restrict__ act) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  double d = 0.0;
  if (g < GPW) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
      if (act && !act[i]) continue;  // rows of finished problems of a batch
      const double acc = row_dot_df<NP>(__ldg(rp + i), __ldg(rp + i + 1), r, col, val2, ea, x2, ex);
      if (y) y[i * NP + r] = acc;
      if (partial) d = fma(x[i * NP + r], acc, d);
    }
  }
  if (partial) {
    d = block_sum(d);
    if (threadIdx.x == 0) partial[blockIdx.x] = d;
  }
}

// the same product on the symmetric storage of level 1 (SymL, see k_smooth_lp_sym): left blocks
// as transposes of their mirrors, then the diagonal and right blocks; bitwise the full storage's
// result
template <int NP>
__device__ __forceinline__ double row_dot_df_sym(int64_t i, int r, const int64_t* __restrict__ urp,
                                                 const int32_t* __restrict__ ucol, const float2* __restrict__ uval2,
                                                 const int* __restrict__ uea, SymL L, const float2* __restrict__ x2,
                                                 const int* __restrict__ ex) {
  constexpr int CH = NP <= 10 ? XDG_CH_PAIR : 1;
  RowAcc acc;
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
      const float2* B = uval2 + (int64_t)bb[u] * (NP * NP) + r;  // column r of the mirror block
      float2 a[NP], xv[NP];
#pragma unroll
      for (int c = 0; c < NP; ++c) a[c] = __ldg(B + c * NP);
      ldrow_df<NP>(x2 + (int64_t)cc[u] * NP, xv);
      const int k = __ldg(uea + bb[u]) + __ldg(ex + cc[u]);
      float hi, lo;
      block_dot_df<NP>(a, xv, hi, lo);
      acc.add(hi, lo, k);
    }
  }
  const int64_t z0 = __ldg(urp + i), z1 = __ldg(urp + i + 1);
  for (int64_t z = z0; z < z1; z += CH) {
    int32_t cc[CH];
    int ee[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      cc[u] = (z + u < z1) ? __ldg(ucol + z + u) : -1;
      ee[u] = (z + u < z1) ? __ldg(uea + z + u) : 0;
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (cc[u] < 0) continue;
      float2 a[NP], xv[NP];
      ldrow_df<NP>(uval2 + (z + u) * (NP * NP) + r * NP, a);
      ldrow_df<NP>(x2 + (int64_t)cc[u] * NP, xv);
      const int k = ee[u] + __ldg(ex + cc[u]);
      float hi, lo;
      block_dot_df<NP>(a, xv, hi, lo);
      acc.add(hi, lo, k);
    }
  }
  return acc.result();
}

template <int NP>
__global__ void __launch_bounds__(kThreads, XDG_PAIR_MINB) k_spmv_dot_df_sym(int64_t nb, const int64_t* __restrict__ urp,
                                                             const int32_t* __restrict__ ucol,
                                                             const float2* __restrict__ uval2,
                                                             const int* __restrict__ uea, SymL L,
                                                             const float2* __restrict__ x2, const int* __restrict__ ex,
                                                             const double* __restrict__ x, double* __restrict__ y,
                                                             double* __restrict__ partial,
                                                             const uint8_t* __restrict__ act) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  double d = 0.0;
  if (g < GPW) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
      if (act && !act[i]) continue;
      const double acc = row_dot_df_sym<NP>(i, r, urp, ucol, uval2, uea, L, x2, ex);
      if (y) y[i * NP + r] = acc;
      if (partial) d = fma(x[i * NP + r], acc, d);
    }
  }
  if (partial) {
    d = block_sum(d);
    if (threadIdx.x == 0) partial[blockIdx.x] = d;
  }
}

// compact pair storage gathered from the full pair copy
__global__ void k_gather_blocks_df(int64_t nblk, int np2, const int64_t* __restrict__ umap,
                                   const float2* __restrict__ v, const int* __restrict__ ea, float2* __restrict__ uv,
                                   int* __restrict__ uea) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t z = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; z < nblk; z += nw) {
    const int64_t zf = __ldg(umap + z);
    for (int k = lane; k < np2; k += 32) uv[z * np2 + k] = v[zf * np2 + k];
    if (lane == 0) uea[z] = ea[zf];
  }
}

// operator blocks -> scaled double-float pairs: one warp per block, ea = exponent of the
// block's largest magnitude (so that the scaled entries are at most 1)
__global__ void k_make_df(int64_t nblk, int np2, const double* __restrict__ val, float2* __restrict__ val2,
                          int* __restrict__ ea) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t z = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; z < nblk; z += nw) {
    const double* a = val + z * np2;
    double m = 0.0;
    for (int k = lane; k < np2; k += 32) m = fmax(m, fabs(a[k]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int e = exp_of(m);
    const double s = pow2_d(-e);
    for (int k = lane; k < np2; k += 32) val2[z * np2 + k] = split_df(a[k] * s);
    if (lane == 0) ea[z] = e;
  }
}

// the block of NP entries of lane r's group: exponent of its largest magnitude (all lanes)
template <int NP>
__device__ __forceinline__ int group_exp(double v, unsigned mask) {
  const int e = (v == 0.0) ? -2147483647 : exp_of(v);
  const int m = __reduce_max_sync(mask, e);
  return m == -2147483647 ? 0 : m;
}

// conjugate-gradient direction p = z + beta p (first: p = z) in FP64, and its scaled
// double-float copy for k_spmv_dot_df (groups of NP lanes per block row)
template <int NP>
__global__ void __launch_bounds__(kThreads) k_pcg_p_df(int64_t nb, const PcgScal* __restrict__ S, int first,
                                                      const double* __restrict__ z, double* __restrict__ p,
                                                      float2* __restrict__ p2, int* __restrict__ ex) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  const double be = first ? 0.0 : S->beta;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
    const int64_t e = i * NP + r;
    const double v = first ? z[e] : fma(be, p[e], z[e]);
    p[e] = v;
    const int k = group_exp<NP>(v, mask);
    p2[e] = split_scaled(v, k);
    if (r == 0) ex[i] = k;
  }
}

// the same copy of a given vector x (no update)
template <int NP>
__global__ void __launch_bounds__(kThreads) k_split_df(int64_t nb, const double* __restrict__ x,
                                                      float2* __restrict__ x2, int* __restrict__ ex) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;
  if (g >= GPW) return;
  const unsigned mask = group_mask(g, NP);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp * GPW + g; i < nb; i += nw * GPW) {
    const int64_t e = i * NP + r;
    const double v = x[e];
    const int k = group_exp<NP>(v, mask);
    x2[e] = split_scaled(v, k);
    if (r == 0) ex[i] = k;
  }
}

}  // namespace xdg
