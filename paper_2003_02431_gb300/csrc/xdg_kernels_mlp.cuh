// Learned cut-cell correction: a small MLP per unit (the two species blocks of one cut
// background cell) maps the unit's geometry and residual to a correction of both blocks.
//
// Network: n_in -> 64 -> 64 -> 64 -> n_out (= 2 Np), GELU (erf form) on the hidden layers.
// Flat parameters (row-major): W1[n_in][64] b1[64] W2[64][64] b2[64] W3[64][64] b3[64]
// W4[64][n_out] b4[n_out]; a layer computes a_out = act(a_in W + b).
//
// Loss of a sample (unit u, residual r_u = s rhat, network output yhat, correction s yhat):
// the change of the energy norm of the true error, ||e - delta||_M^2 - ||e||_M^2 =
// delta^T M_uu delta - 2 delta^T r_u, divided by s^2 and by the optimal decrease
// c = rhat^T M_uu^{-1} rhat:  L = (yhat^T M_uu yhat - 2 yhat^T rhat) / c  (-1: exact local solve).
//
// Mapping: one warp per sample; lane l owns hidden units l and l + 32 and outputs l, l + 32;
// the layer inputs are broadcast by shuffles and the weights are read from shared memory
// (consecutive lanes read consecutive weights). FLOPs are ~12k FMA per sample: the network
// is tiny next to the solve and runs on the FP32 pipe; training gradients are summed over
// samples in a fixed order (deterministic).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "xdg_kernels.cuh"

namespace xdg {

constexpr int kHid = 64;

struct MlpDims {
  int n_in, n_out;
  int oW1, ob1, oW2, ob2, oW3, ob3, oW4, ob4, total;
};

inline MlpDims mlp_dims(int n_in, int n_out) {
  MlpDims d;
  d.n_in = n_in;
  d.n_out = n_out;
  d.oW1 = 0;
  d.ob1 = n_in * kHid;
  d.oW2 = d.ob1 + kHid;
  d.ob2 = d.oW2 + kHid * kHid;
  d.oW3 = d.ob2 + kHid;
  d.ob3 = d.oW3 + kHid * kHid;
  d.oW4 = d.ob3 + kHid;
  d.ob4 = d.oW4 + kHid * n_out;
  d.total = d.ob4 + n_out;
  return d;
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__device__ __forceinline__ float wload(const float* p, int i) { return p[i]; }
__device__ __forceinline__ float wload(const __nv_bfloat16* p, int i) { return __bfloat162float(p[i]); }

// a_out(l), a_out(l+32) = (a_in W + b) for a hidden layer of width 64; a_in held as two
// registers per lane (entries l and l + 32), n inputs
template <class W>
__device__ __forceinline__ void dense64(const W* __restrict__ w, const W* __restrict__ b, int n, float in0, float in1,
                                        int lane, float& o0, float& o1) {
  float a0 = wload(b, lane), a1 = wload(b, lane + 32);
  for (int i = 0; i < n; ++i) {
    const float xi = __shfl_sync(0xffffffffu, i < 32 ? in0 : in1, i & 31);
    a0 = fmaf(wload(w, i * kHid + lane), xi, a0);
    a1 = fmaf(wload(w, i * kHid + 32 + lane), xi, a1);
  }
  o0 = a0;
  o1 = a1;
}

// output layer: y(j) for j = lane and lane + 32 (< n_out)
template <class W>
__device__ __forceinline__ void dense_out(const W* __restrict__ w, const W* __restrict__ b, int n_out, float in0,
                                          float in1, int lane, float& y0, float& y1) {
  const bool h0 = lane < n_out, h1 = lane + 32 < n_out;
  float a0 = h0 ? wload(b, lane) : 0.f, a1 = h1 ? wload(b, lane + 32) : 0.f;
  for (int i = 0; i < kHid; ++i) {
    const float xi = __shfl_sync(0xffffffffu, i < 32 ? in0 : in1, i & 31);
    if (h0) a0 = fmaf(wload(w, i * n_out + lane), xi, a0);
    if (h1) a1 = fmaf(wload(w, i * n_out + 32 + lane), xi, a1);
  }
  y0 = a0;
  y1 = a1;
}

template <class W>
__device__ __forceinline__ void mlp_forward(const W* __restrict__ P, const MlpDims& d, float x0, float x1, int lane,
                                            float* z, float* a, float& y0, float& y1) {
  // z[0..5], a[0..5]: pre-activations and activations of the 3 hidden layers (2 per lane)
  dense64(P + d.oW1, P + d.ob1, d.n_in, x0, x1, lane, z[0], z[1]);
  a[0] = gelu_f(z[0]);
  a[1] = gelu_f(z[1]);
  dense64(P + d.oW2, P + d.ob2, kHid, a[0], a[1], lane, z[2], z[3]);
  a[2] = gelu_f(z[2]);
  a[3] = gelu_f(z[3]);
  dense64(P + d.oW3, P + d.ob3, kHid, a[2], a[3], lane, z[4], z[5]);
  a[4] = gelu_f(z[4]);
  a[5] = gelu_f(z[5]);
  dense_out(P + d.oW4, P + d.ob4, d.n_out, a[4], a[5], lane, y0, y1);
}

// parameters to shared memory: 16-byte loads for the aligned bulk, element loads for the tail
template <class W>
__device__ void stage_params(W* sp, const W* __restrict__ P, int total) {
  const int nvec = (int)(((size_t)total * sizeof(W)) / 16);
  const uint4* src = reinterpret_cast<const uint4*>(P);
  uint4* dst = reinterpret_cast<uint4*>(sp);
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = __ldg(src + i);
  for (int i = nvec * (int)(16 / sizeof(W)) + threadIdx.x; i < total; i += blockDim.x) sp[i] = P[i];
  __syncthreads();
}

// Y[s] = network(X[s]) (inference or parity checks); W = float or bf16 parameters
template <class W>
__global__ void __launch_bounds__(256) k_mlp_forward(int64_t n, MlpDims d, const W* __restrict__ P,
                                                    const float* __restrict__ X, float* __restrict__ Y) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sp = reinterpret_cast<W*>(smem_raw);
  stage_params(sp, P, d.total);
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n; s += nw) {
    const float* x = X + s * d.n_in;
    const float x0 = lane < d.n_in ? x[lane] : 0.f, x1 = lane + 32 < d.n_in ? x[lane + 32] : 0.f;
    float z[6], a[6], y0, y1;
    mlp_forward(sp, d, x0, x1, lane, z, a, y0, y1);
    if (lane < d.n_out) Y[s * d.n_out + lane] = y0;
    if (lane + 32 < d.n_out) Y[s * d.n_out + lane + 32] = y1;
  }
}

// One training pass over the samples idx[0..n) (idx == nullptr: 0..n-1): forward, loss and
// backward of every sample. Writes per sample s (position in the batch): A1..A3, dZ1..dZ3
// ([n][64] each), dY ([n][n_out]) and its loss; the gradient is the mean over the batch
// (dY carries the factor 1 / n).
struct MlpTrainBuf {
  float *A1, *A2, *A3, *dZ1, *dZ2, *dZ3, *dY;
  double* loss;
};

__global__ void __launch_bounds__(256) k_mlp_train_pass(int n, const int32_t* __restrict__ idx, MlpDims d,
                                                       const float* __restrict__ P, const float* __restrict__ X,
                                                       const int32_t* __restrict__ uid,
                                                       const float* __restrict__ Mloc,
                                                       const float* __restrict__ R, const float* __restrict__ C,
                                                       MlpTrainBuf T) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sp = reinterpret_cast<float*>(smem_raw);
  float* w4t = sp + d.total;            // W4^T [n_out][64]
  float* w3t = w4t + d.n_out * kHid;    // W3^T [64][64]
  float* w2t = w3t + kHid * kHid;       // W2^T [64][64]
  for (int i = threadIdx.x; i < d.total; i += blockDim.x) sp[i] = P[i];
  for (int e = threadIdx.x; e < kHid * d.n_out; e += blockDim.x) {
    const int i = e / d.n_out, j = e - i * d.n_out;
    w4t[j * kHid + i] = P[d.oW4 + e];
  }
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
    const int i = e >> 6, j = e & 63;
    w3t[j * kHid + i] = P[d.oW3 + e];
    w2t[j * kHid + i] = P[d.oW2 + e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int m = d.n_out;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n; s += nw) {
    const int g = idx ? idx[s] : s;
    const float* x = X + (int64_t)g * d.n_in;
    const float x0 = lane < d.n_in ? x[lane] : 0.f, x1 = lane + 32 < d.n_in ? x[lane + 32] : 0.f;
    float z[6], a[6], y0, y1;
    mlp_forward(sp, d, x0, x1, lane, z, a, y0, y1);
    // loss and dL/dy
    const float* M = Mloc + (int64_t)uid[g] * m * m;
    const float* r = R + (int64_t)g * m;
    const float c = C[g];
    float my0 = 0.f, my1 = 0.f;
    for (int k = 0; k < m; ++k) {
      const float yk = __shfl_sync(0xffffffffu, k < 32 ? y0 : y1, k & 31);
      if (lane < m) my0 = fmaf(M[lane * m + k], yk, my0);
      if (lane + 32 < m) my1 = fmaf(M[(lane + 32) * m + k], yk, my1);
    }
    const float r0 = lane < m ? r[lane] : 0.f, r1 = lane + 32 < m ? r[lane + 32] : 0.f;
    float part = (lane < m ? y0 * (my0 - 2.f * r0) : 0.f) + (lane + 32 < m ? y1 * (my1 - 2.f * r1) : 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const float sc = 2.f / (c * (float)n);
    const float dy0 = lane < m ? sc * (my0 - r0) : 0.f, dy1 = lane + 32 < m ? sc * (my1 - r1) : 0.f;
    // backward
    float da0 = 0.f, da1 = 0.f;
    for (int j = 0; j < m; ++j) {
      const float gj = __shfl_sync(0xffffffffu, j < 32 ? dy0 : dy1, j & 31);
      da0 = fmaf(w4t[j * kHid + lane], gj, da0);
      da1 = fmaf(w4t[j * kHid + 32 + lane], gj, da1);
    }
    const float d30 = da0 * gelu_df(z[4]), d31 = da1 * gelu_df(z[5]);
    da0 = da1 = 0.f;
    for (int j = 0; j < kHid; ++j) {
      const float gj = __shfl_sync(0xffffffffu, j < 32 ? d30 : d31, j & 31);
      da0 = fmaf(w3t[j * kHid + lane], gj, da0);
      da1 = fmaf(w3t[j * kHid + 32 + lane], gj, da1);
    }
    const float d20 = da0 * gelu_df(z[2]), d21 = da1 * gelu_df(z[3]);
    da0 = da1 = 0.f;
    for (int j = 0; j < kHid; ++j) {
      const float gj = __shfl_sync(0xffffffffu, j < 32 ? d20 : d21, j & 31);
      da0 = fmaf(w2t[j * kHid + lane], gj, da0);
      da1 = fmaf(w2t[j * kHid + 32 + lane], gj, da1);
    }
    const float d10 = da0 * gelu_df(z[0]), d11 = da1 * gelu_df(z[1]);
    const int64_t o = (int64_t)s * kHid;
    T.A1[o + lane] = a[0];
    T.A1[o + 32 + lane] = a[1];
    T.A2[o + lane] = a[2];
    T.A2[o + 32 + lane] = a[3];
    T.A3[o + lane] = a[4];
    T.A3[o + 32 + lane] = a[5];
    T.dZ1[o + lane] = d10;
    T.dZ1[o + 32 + lane] = d11;
    T.dZ2[o + lane] = d20;
    T.dZ2[o + 32 + lane] = d21;
    T.dZ3[o + lane] = d30;
    T.dZ3[o + 32 + lane] = d31;
    if (lane < m) T.dY[(int64_t)s * m + lane] = dy0;
    if (lane + 32 < m) T.dY[(int64_t)s * m + 32 + lane] = dy1;
    if (lane == 0) T.loss[s] = (double)(part / c);
  }
}

// partial[sl][p] = sum over the samples of slice sl of dL/dparam p (fixed order within slices)
__global__ void __launch_bounds__(256) k_mlp_grad_partial(int n, int nsl, const int32_t* __restrict__ idx, MlpDims d,
                                                         const float* __restrict__ X, MlpTrainBuf T,
                                                         float* __restrict__ partial) {
  pdl_entry();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int sl = blockIdx.y;
  if (p >= d.total) return;
  const int s0 = (int)((int64_t)n * sl / nsl), s1 = (int)((int64_t)n * (sl + 1) / nsl);
  // which layer and entry
  const float *A = nullptr, *G = nullptr;
  int i = -1, j, ncol = kHid, in_x = 0;
  if (p < d.ob1) {
    i = p / kHid; j = p - i * kHid; G = T.dZ1; in_x = 1;
  } else if (p < d.oW2) {
    j = p - d.ob1; G = T.dZ1;
  } else if (p < d.ob2) {
    const int e = p - d.oW2; i = e / kHid; j = e - i * kHid; A = T.A1; G = T.dZ2;
  } else if (p < d.oW3) {
    j = p - d.ob2; G = T.dZ2;
  } else if (p < d.ob3) {
    const int e = p - d.oW3; i = e / kHid; j = e - i * kHid; A = T.A2; G = T.dZ3;
  } else if (p < d.oW4) {
    j = p - d.ob3; G = T.dZ3;
  } else if (p < d.ob4) {
    const int e = p - d.oW4; i = e / d.n_out; j = e - i * d.n_out; A = T.A3; G = T.dY; ncol = d.n_out;
  } else {
    j = p - d.ob4; G = T.dY; ncol = d.n_out;
  }
  float acc = 0.f;
  for (int s = s0; s < s1; ++s) {
    const float gj = G[(int64_t)s * ncol + j];
    float ai = 1.f;
    if (i >= 0) ai = in_x ? X[(int64_t)(idx ? idx[s] : s) * d.n_in + i] : A[(int64_t)s * kHid + i];
    acc = fmaf(ai, gj, acc);
  }
  partial[(int64_t)sl * d.total + p] = acc;
}

__global__ void k_mlp_grad_final(int total, int nsl, const float* __restrict__ partial, float* __restrict__ grad) {
  pdl_entry();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= total) return;
  float acc = 0.f;
  for (int sl = 0; sl < nsl; ++sl) acc += partial[(int64_t)sl * total + p];
  grad[p] = acc;
}

// Adam (Kingma & Ba) with bias correction; t = step number (1-based)
__global__ void k_adam(int total, float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m1,
                       float* __restrict__ m2, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  pdl_entry();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= total) return;
  const float g = G[p];
  const float a = b1 * m1[p] + (1.f - b1) * g;
  const float v = b2 * m2[p] + (1.f - b2) * g * g;
  m1[p] = a;
  m2[p] = v;
  P[p] -= lr * (a / bc1) / (sqrtf(v / bc2) + eps);
}

__global__ void k_to_bf16(int total, const float* __restrict__ P, __nv_bfloat16* __restrict__ Q) {
  pdl_entry();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < total) Q[p] = __float2bfloat16_rn(P[p]);
}

// sum of n doubles in index order by one CTA (each thread a contiguous range, then the block
// sum in a fixed tree)
__global__ void __launch_bounds__(kThreads) k_sum_ordered(int n, const double* __restrict__ v, double* __restrict__ out,
                                                         int accumulate) {
  pdl_entry();
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int i0 = threadIdx.x * per, i1 = min(n, i0 + per);
  double acc = 0.0;
  for (int i = i0; i < i1; ++i) acc += v[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = accumulate ? *out + acc : acc;
}

// ------------------------------------------------------------------------------------------
// units on the hierarchy

// warp helpers on small shared-memory matrices (row stride ld)
// in-place lower Cholesky factor of A[0..n)[0..n); false if not positive definite
__device__ bool warp_chol(double* A, int n, int ld, int lane) {
  bool ok = true;
  for (int j = 0; j < n; ++j) {
    const double djj = A[j * ld + j];
    if (!(djj > 0.0)) ok = false;
    const double d = sqrt(djj > 0.0 ? djj : 1.0);
    __syncwarp();
    for (int i = j + 1 + lane; i < n; i += 32) A[i * ld + j] /= d;
    if (lane == 0) A[j * ld + j] = d;
    __syncwarp();
    for (int i = j + 1 + lane; i < n; i += 32)
      for (int k = j + 1; k <= i; ++k) A[i * ld + k] -= A[i * ld + j] * A[k * ld + j];
    __syncwarp();
  }
  return ok;
}
// X = L^{-1} for the lower factor L (columns owned by lanes)
__device__ void warp_trinv(const double* L, int ldl, double* X, int ldx, int n, int lane) {
  for (int c = lane; c < n; c += 32)
    for (int i = 0; i < n; ++i) {
      if (i < c) {
        X[i * ldx + c] = 0.0;
        continue;
      }
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) v -= L[i * ldl + k] * X[k * ldx + c];
      X[i * ldx + c] = v / L[i * ldl + i];
    }
  __syncwarp();
}

// Per unit (one warp): the inverse Cholesky factors X_a = L_a^{-1}, X_b = L_b^{-1} of the
// diagonal blocks M_aa, M_bb; the unit matrix in these coordinates,
// H = diag(X_a, X_b) M_uu diag(X_a, X_b)^T (identity diagonal blocks), in FP64 (Hm) and FP32
// (Mloc); and H^{-1} (Hinv). zidx[u][0..3]: positions of the blocks (a,a), (a,b), (b,a), (b,b)
// in val (-1: zero block). err: set when a matrix is not positive definite.
template <int NP>
__global__ void __launch_bounds__(32) k_unit_factor(int U, const int64_t* __restrict__ zidx,
                                                    const double* __restrict__ val, double* __restrict__ Linv,
                                                    double* __restrict__ Hm, float* __restrict__ Mloc,
                                                    double* __restrict__ Hinv, int* err) {
  pdl_entry();
  constexpr int m = 2 * NP, ld = m + 1;
  __shared__ double A[m * ld];
  __shared__ double W[m * ld];
  __shared__ double X[m * ld];
  const int u = blockIdx.x, lane = threadIdx.x;
  if (u >= U) return;
  for (int e = lane; e < m * m; e += 32) {
    const int r = e / m, c = e - r * m;
    const int q = (r >= NP) * 2 + (c >= NP);
    const int64_t z = zidx[(int64_t)u * 4 + q];
    A[r * ld + c] = z >= 0 ? val[z * NP * NP + (r % NP) * NP + (c % NP)] : 0.0;
    X[r * ld + c] = 0.0;
  }
  __syncwarp();
  bool ok = true;
  for (int h = 0; h < 2; ++h) {
    const int o = h * NP;
    for (int e = lane; e < NP * NP; e += 32) {
      const int r = e / NP, c = e - r * NP;
      W[r * ld + c] = A[(o + r) * ld + o + c];
    }
    __syncwarp();
    ok = warp_chol(W, NP, ld, lane) && ok;
    warp_trinv(W, ld, X + o * ld + o, ld, NP, lane);
  }
  for (int e = lane; e < 2 * NP * NP; e += 32) {
    const int h = e / (NP * NP), q = e - h * NP * NP, r = q / NP, c = q - r * NP;
    Linv[(int64_t)u * 2 * NP * NP + e] = X[(h * NP + r) * ld + h * NP + c];
  }
  // W = X A, then A = W X^T = H
  for (int e = lane; e < m * m; e += 32) {
    const int r = e / m, c = e - r * m;
    const int o = (r >= NP) ? NP : 0;
    double acc = 0.0;
    for (int k = o; k <= r; ++k) acc += X[r * ld + k] * A[k * ld + c];
    W[r * ld + c] = acc;
  }
  __syncwarp();
  for (int e = lane; e < m * m; e += 32) {
    const int r = e / m, c = e - r * m;
    const int o = (c >= NP) ? NP : 0;
    double acc = 0.0;
    for (int k = o; k <= c; ++k) acc += W[r * ld + k] * X[c * ld + k];
    A[r * ld + c] = acc;
  }
  __syncwarp();
  for (int e = lane; e < m * m; e += 32) {
    const int r = e / m, c = e - r * m;
    const double v = 0.5 * (A[r * ld + c] + A[c * ld + r]);  // exact symmetry
    Hm[(int64_t)u * m * m + e] = v;
    Mloc[(int64_t)u * m * m + e] = (float)v;
    W[r * ld + c] = v;
  }
  __syncwarp();
  ok = warp_chol(W, m, ld, lane) && ok;
  warp_trinv(W, ld, X, ld, m, lane);
  for (int e = lane; e < m * m; e += 32) {
    const int r = e / m, c = e - r * m;
    double acc = 0.0;
    for (int k = (r > c ? r : c); k < m; ++k) acc += X[k * ld + r] * X[k * ld + c];
    Hinv[(int64_t)u * m * m + e] = acc;
  }
  if (!ok && lane == 0) atomicOr(err, 1);
}

// y[i] = b[i] - (M x)[i] for the listed block rows i = rows[t], one row per warp: group g of
// the warp takes the row's blocks z0 + g, z0 + g + GPW, ... (two at a time, so their loads
// overlap) and the groups' partial sums are added in group order (fixed). The units' rows are
// scattered over the mesh and few; with one row per group each warp waited on one long chain of
// dependent loads (27.7 us for the 13k rows of the 64^3 units).
template <int NP>
__global__ void __launch_bounds__(kThreads) k_resid_rows_split(int64_t nr, const int32_t* __restrict__ rows,
                                                              const int64_t* __restrict__ rp,
                                                              const int32_t* __restrict__ col,
                                                              const double* __restrict__ val,
                                                              const double* __restrict__ x,
                                                              const double* __restrict__ b, double* __restrict__ y) {
  pdl_entry();
  constexpr int GPW = Grp<NP>::GPW;
  const int lane = threadIdx.x & 31;
  const int g = lane / NP, r = lane - g * NP;  // idle lanes (g == GPW) keep r < NP
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = warp; t < nr; t += nw) {
    const int64_t i = rows[t];
    const int64_t z0 = __ldg(rp + i), z1 = __ldg(rp + i + 1);
    double acc = 0.0;
    if (g < GPW) {
      for (int64_t z = z0 + g; z < z1; z += 2 * GPW) {
        const int64_t z2 = z + GPW;
        const int32_t c0 = __ldg(col + z), c1 = z2 < z1 ? __ldg(col + z2) : -1;
        double a0[NP], x0[NP], a1[NP], x1[NP];
        ldrow<NP>(val + z * (NP * NP) + r * NP, a0);
        ldrow<NP>(x + (int64_t)c0 * NP, x0);
        if (c1 >= 0) {
          ldrow<NP>(val + z2 * (NP * NP) + r * NP, a1);
          ldrow<NP>(x + (int64_t)c1 * NP, x1);
        }
#pragma unroll
        for (int c = 0; c < NP; ++c) acc = fma(a0[c], x0[c], acc);
        if (c1 >= 0) {
#pragma unroll
          for (int c = 0; c < NP; ++c) acc = fma(a1[c], x1[c], acc);
        }
      }
    }
    double tot = 0.0;
#pragma unroll
    for (int gg = 0; gg < GPW; ++gg) tot += __shfl_sync(0xffffffffu, acc, gg * NP + r);
    if (g == 0) y[i * NP + r] = b[i * NP + r] - tot;
  }
}

// one unit's residual in block-Jacobi coordinates, rt = [X_a r_a; X_b r_b]: entries lane and
// lane + 32, and s = ||rt||_2
template <int NP>
__device__ __forceinline__ void unit_residual(const int32_t* __restrict__ pairs, const double* __restrict__ Linv,
                                              int u, const double* __restrict__ r, int lane, double& r0, double& r1,
                                              double& s) {
  constexpr int m = 2 * NP;
  const int blk[2] = {pairs[2 * u], pairs[2 * u + 1]};
  const double* X = Linv + (int64_t)u * 2 * NP * NP;
  double out[2] = {0.0, 0.0};
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int e = lane + 32 * t;
    if (e < m) {
      const int h = e / NP, i = e - h * NP;
      const double* xr = X + h * NP * NP + i * NP;
      const double* rv = r + (int64_t)blk[h] * NP;
      double acc = 0.0;
      for (int k = 0; k <= i; ++k) acc = fma(xr[k], rv[k], acc);
      out[t] = acc;
    }
  }
  r0 = out[0];
  r1 = out[1];
  double q = r0 * r0 + r1 * r1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  s = sqrt(q);
}

// network input entry k of unit u: geometry features, then rhat
__device__ __forceinline__ float unit_input(const float* __restrict__ geom, int n_geo, int u, int k, double r0,
                                            double r1, double inv_s, int lane) {
  // every lane evaluates the shuffles (all lanes participate)
  const int j = k - n_geo;
  const double rj0 = __shfl_sync(0xffffffffu, r0, (j < 0 ? 0 : j) & 31);
  const double rj1 = __shfl_sync(0xffffffffu, r1, (j < 0 ? 0 : j) & 31);
  if (k < n_geo) return geom[(int64_t)u * n_geo + k];
  return (float)((j < 32 ? rj0 : rj1) * inv_s);
}

// training samples of every unit for the residual r (after a cycle): with rt the residual in
// block-Jacobi coordinates and rhat = rt / ||rt||: X[u] = [geom, rhat], R[u] = rhat,
// C[u] = rhat^T H^{-1} rhat (0 for a zero residual)
template <int NP>
__global__ void __launch_bounds__(256) k_unit_samples(int U, int n_geo, const int32_t* __restrict__ pairs,
                                                     const float* __restrict__ geom, const double* __restrict__ r,
                                                     const double* __restrict__ Linv, const double* __restrict__ Minv,
                                                     float* __restrict__ X, float* __restrict__ R,
                                                     float* __restrict__ C) {
  pdl_entry();
  constexpr int m = 2 * NP;
  const int lane = threadIdx.x & 31;
  const int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (u >= U) return;
  double r0, r1, s;
  unit_residual<NP>(pairs, Linv, u, r, lane, r0, r1, s);
  const double inv = s > 0.0 ? 1.0 / s : 0.0;
  const int n_in = n_geo + m;
  for (int k0 = 0; k0 < n_in; k0 += 32) {
    const int k = k0 + lane;
    float v = unit_input(geom, n_geo, u, k < n_in ? k : 0, r0, r1, inv, lane);
    if (k < n_in) X[(int64_t)u * n_in + k] = v;
  }
  if (lane < m) R[(int64_t)u * m + lane] = (float)(r0 * inv);
  if (lane + 32 < m) R[(int64_t)u * m + lane + 32] = (float)(r1 * inv);
  // c = rhat^T Minv rhat (rows lane and lane + 32 of Minv rhat, then a warp sum)
  const double* Mi = Minv + (int64_t)u * m * m;
  double row0 = 0.0, row1 = 0.0;
  for (int k = 0; k < m; ++k) {
    const double rk = __shfl_sync(0xffffffffu, k < 32 ? r0 : r1, k & 31) * inv;
    if (lane < m) row0 = fma(Mi[lane * m + k], rk, row0);
    if (lane + 32 < m) row1 = fma(Mi[(lane + 32) * m + k], rk, row1);
  }
  double q = (lane < m ? row0 * r0 * inv : 0.0) + (lane + 32 < m ? row1 * r1 * inv : 0.0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  if (lane == 0) C[u] = (float)q;
}

// learned correction of every unit for the residual r (after the cycle): y = network([geom,
// rhat]) with BF16 parameters (FP32 arithmetic), rhat = rt / s; the correction in block-Jacobi
// coordinates is s y, i.e. delta = s [X_a^T y_a; X_b^T y_b]. Kept when it lowers the error's
// energy: E = s^2 (y^T H y - 2 y^T rhat) = delta^T M_uu delta - 2 delta^T r_u < 0 (FP64).
// delta[u][0..m) = kept correction (zeros otherwise), keep[u], E[u].
//
// Mapping: sixteen lanes per unit (two units per warp, sixteen per CTA of eight warps) for the
// per-unit work (residual transform, energy, correction; sums over a unit's lanes by shuffles in
// a fixed order). The three hidden layers are dense products of the CTA's 16 x K activations
// with the K x 64 weights and run on the tensor cores (mma_layer below); the output layer
// (2 Np outputs) runs on the unit's lanes from an FP32 copy of the last hidden layer.
constexpr int kUnitLanes = 16;
constexpr int kUnitsPerWarp = 32 / kUnitLanes;
constexpr int kUnitWarps = 8;
constexpr int kUnitsPerCta = kUnitsPerWarp * kUnitWarps;  // = 16, the rows of one MMA tile
static_assert(kUnitsPerCta == 16 && kUnitWarps * 8 == kHid, "one 16-row tile, eight columns per warp");
constexpr int kActStride = 65;
constexpr int kTriStride = 72;  // BF16 activation rows: 36 words, so a fragment's rows hit distinct banks
// shared memory of k_unit_apply after the parameters: two activation buffers of three BF16
// parts, then the FP32 rows (last hidden layer, outputs)
constexpr size_t kUnitTriBytes = 2 * 3 * kUnitsPerCta * kTriStride * sizeof(__nv_bfloat16);
constexpr size_t kUnitActBytes = (size_t)kUnitsPerCta * 2 * kActStride * sizeof(float);

// One hidden layer for the CTA's 16 units on the tensor cores: out = GELU(in W + bias), 64
// outputs; warp w computes columns 8w .. 8w+7 for all 16 rows. in: three BF16 parts
// tin[p][row][k] (k < K, K a multiple of 16; entries past the layer's n_in are zero), W: BF16
// rows of 64 (rows >= kmax read as zero). The partial products of the lo, mid and hi parts go
// into one FP32 accumulator started at the bias. The result goes either to tout (three BF16
// parts, the next layer's input) or, FP32, to fout[row * 2 kActStride + col].
template <bool TRI_OUT>
__device__ __forceinline__ void mma_layer(const __nv_bfloat16* tin, int K, int kmax, const __nv_bfloat16* W,
                                          const __nv_bfloat16* bias, __nv_bfloat16* tout, float* fout) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int n0 = 8 * w, c0 = n0 + 2 * t;
  constexpr int PS = kUnitsPerCta * kTriStride;  // elements per part
  float d[4];
  d[0] = d[2] = __bfloat162float(bias[c0]);
  d[1] = d[3] = __bfloat162float(bias[c0 + 1]);
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t b[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int k = k0 + 2 * t + 8 * j;
      const __nv_bfloat16 w0 = k < kmax ? W[k * kHid + n0 + g] : zero;
      const __nv_bfloat16 w1 = k + 1 < kmax ? W[(k + 1) * kHid + n0 + g] : zero;
      b[j] = pack_bf16x2(w0, w1);
    }
#pragma unroll
    for (int p = 2; p >= 0; --p) {  // lo, mid, hi
      const __nv_bfloat16* A = tin + p * PS;
      uint32_t a[4];
      a[0] = *reinterpret_cast<const uint32_t*>(A + g * kTriStride + k0 + 2 * t);
      a[1] = *reinterpret_cast<const uint32_t*>(A + (g + 8) * kTriStride + k0 + 2 * t);
      a[2] = *reinterpret_cast<const uint32_t*>(A + g * kTriStride + k0 + 2 * t + 8);
      a[3] = *reinterpret_cast<const uint32_t*>(A + (g + 8) * kTriStride + k0 + 2 * t + 8);
      mma_16816_bf16(d, a, b);
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int row = g + 8 * (e >> 1), col = c0 + (e & 1);
    const float v = gelu_f(d[e]);
    if constexpr (TRI_OUT) {
      __nv_bfloat16 h, mdl, l;
      split_bf16x3(v, h, mdl, l);
      tout[row * kTriStride + col] = h;
      tout[PS + row * kTriStride + col] = mdl;
      tout[2 * PS + row * kTriStride + col] = l;
    } else {
      fout[row * 2 * kActStride + col] = v;
    }
  }
}

// sum over the kUnitLanes lanes of a unit (aligned groups of the warp)
__device__ __forceinline__ double unit_sum(double v) {
#pragma unroll
  for (int o = 1; o < kUnitLanes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int NP>
__global__ void __launch_bounds__(kUnitWarps * 32) k_unit_apply(int U, MlpDims d, int n_geo, const int32_t* __restrict__ pairs,
                                                   const float* __restrict__ geom, const double* __restrict__ r,
                                                   const __nv_bfloat16* __restrict__ P,
                                                   const double* __restrict__ Linv, const float* __restrict__ Hf,
                                                   double* __restrict__ delta, int* __restrict__ keep,
                                                   double* __restrict__ E) {
  pdl_entry();
  constexpr int m = 2 * NP;
  constexpr int T = (m + kUnitLanes - 1) / kUnitLanes;  // residual / output entries per lane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* sp = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  const int wbytes = ((d.total * 2 + 15) / 16) * 16;
  __nv_bfloat16* tri = reinterpret_cast<__nv_bfloat16*>(smem_raw + wbytes);
  float* act = reinterpret_cast<float*>(smem_raw + wbytes + kUnitTriBytes);
  stage_params(sp, P, d.total);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int uu = lane / kUnitLanes, q = lane % kUnitLanes;
  const int slot = w * kUnitsPerWarp + uu;
  float* A0 = act + slot * 2 * kActStride;
  float* A1 = A0 + kActStride;
  const int u = blockIdx.x * kUnitsPerCta + slot;
  const bool valid = u < U;
  // residual of the unit in block-Jacobi coordinates: entries e = q + 4 t
  double rt[T];
  double ss = 0.0;
  const double* X = Linv + (int64_t)(valid ? u : 0) * 2 * NP * NP;
  const int blk[2] = {valid ? pairs[2 * u] : 0, valid ? pairs[2 * u + 1] : 0};
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int e = q + kUnitLanes * t;
    double acc = 0.0;
    if (valid && e < m) {
      const int h = e / NP, i = e - h * NP;
      const double* xr = X + h * NP * NP + i * NP;
      const double* rv = r + (int64_t)blk[h] * NP;
      // the triangular row unrolled to NP (predicated): all loads issue before the first FMA
      double xk[NP], rk[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k)
        if (k <= i) {
          xk[k] = __ldg(xr + k);
          rk[k] = __ldg(rv + k);
        }
#pragma unroll
      for (int k = 0; k < NP; ++k)
        if (k <= i) acc = fma(xk[k], rk[k], acc);
    }
    rt[t] = acc;
    ss = fma(acc, acc, ss);
  }
  ss = unit_sum(ss);
  const double s = sqrt(ss);
  const double inv = s > 0.0 ? 1.0 / s : 0.0;
  // network input: the unit's row of the first activation buffer, three BF16 parts, zero from
  // n_in up to K1 (the first layer's K, a multiple of 16)
  constexpr int PS = kUnitsPerCta * kTriStride;
  const int K1 = (d.n_in + 15) & ~15;  // d.n_in = n_geo + m
  __nv_bfloat16* trow = tri + slot * kTriStride;
  for (int e = q; e < K1; e += kUnitLanes) {  // geometry features, then zeros past n_in
    if (e >= n_geo && e < d.n_in) continue;
    const float v = (e < n_geo && valid) ? geom[(int64_t)u * n_geo + e] : 0.f;
    split_bf16x3(v, trow[e], trow[PS + e], trow[2 * PS + e]);
  }
#pragma unroll
  for (int t = 0; t < T; ++t) {  // rhat entry q + kUnitLanes t, held by this lane
    const int k = q + kUnitLanes * t;
    if (k < m) split_bf16x3((float)(rt[t] * inv), trow[n_geo + k], trow[PS + n_geo + k], trow[2 * PS + n_geo + k]);
  }
  __syncthreads();
  // three hidden layers (GELU) on the tensor cores, the last one into FP32 rows A0
  __nv_bfloat16* tri0 = tri;
  __nv_bfloat16* tri1 = tri + 3 * PS;
  mma_layer<true>(tri0, K1, d.n_in, sp + d.oW1, sp + d.ob1, tri1, nullptr);
  __syncthreads();
  mma_layer<true>(tri1, kHid, kHid, sp + d.oW2, sp + d.ob2, tri0, nullptr);
  __syncthreads();
  mma_layer<false>(tri0, kHid, kHid, sp + d.oW3, sp + d.ob3, nullptr, act);
  __syncthreads();
  const float* in = A0;
  float* out = A1;
  // output layer: y_e, e = q + 4 t
  double y[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int e = q + kUnitLanes * t;
    float acc = 0.f;
    if (e < m) {
      acc = wload(sp + d.ob4, e);
      for (int i = 0; i < kHid; ++i) acc = fmaf(wload(sp + d.oW4, i * m + e), in[i], acc);
      out[e] = acc;
    }
    y[t] = (double)acc;
  }
  __syncwarp();
  // energy change s^2 (y^T H y - 2 y^T rhat), H from its FP32 copy (rows of 2 Np floats, 16-byte
  // aligned: 2 Np is a multiple of 4 for Np in {6, 10, 20}; element loads otherwise)
  const float* Hu = Hf + (int64_t)(valid ? u : 0) * m * m;
  double part = 0.0;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int e = q + kUnitLanes * t;
    if (valid && e < m) {
      float hy = 0.f;
      if constexpr (m % 4 == 0) {
        const float4* hr = reinterpret_cast<const float4*>(Hu + e * m);
#pragma unroll
        for (int k4 = 0; k4 < m / 4; ++k4) {
          const float4 h4 = __ldg(hr + k4);
          hy = fmaf(h4.x, out[4 * k4], hy);
          hy = fmaf(h4.y, out[4 * k4 + 1], hy);
          hy = fmaf(h4.z, out[4 * k4 + 2], hy);
          hy = fmaf(h4.w, out[4 * k4 + 3], hy);
        }
      } else {
#pragma unroll
        for (int k = 0; k < m; ++k) hy = fmaf(__ldg(Hu + e * m + k), out[k], hy);
      }
      part += y[t] * ((double)hy - 2.0 * rt[t] * inv);
    }
  }
  const double en = unit_sum(part) * ss;
  const bool kp = valid && (en < 0.0) && (s > 0.0);
  // delta = s X^T y per half: delta_e = s sum_{j >= i} X_h[j][i] y_{h NP + j}
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int e = q + kUnitLanes * t;
    if (valid && e < m) {
      const int h = e / NP, i = e - h * NP;
      double xj[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j)
        if (j >= i) xj[j] = __ldg(X + h * NP * NP + j * NP + i);
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j)
        if (j >= i) acc = fma(xj[j], (double)out[h * NP + j], acc);
      delta[(int64_t)u * m + e] = kp ? s * acc : 0.0;
    }
  }
  if (valid && q == 0) {
    keep[u] = kp;
    E[u] = en;
  }
}

// z[t] += theta * sum of the kept corrections of the units holding block t
// (tlist[tptr[i] .. tptr[i+1]) = 2 u + half for touched block tblk[i], ascending u)
template <int NP>
__global__ void k_unit_gather(int nt, const int32_t* __restrict__ tblk, const int64_t* __restrict__ tptr,
                              const int32_t* __restrict__ tlist, const double* __restrict__ delta, double theta,
                              double* __restrict__ z) {
  pdl_entry();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nt * NP) return;
  const int i = (int)(e / NP), c = (int)(e - (int64_t)i * NP);
  double acc = 0.0;
  for (int64_t q = tptr[i]; q < tptr[i + 1]; ++q) {
    const int uh = tlist[q];
    acc += delta[(int64_t)(uh >> 1) * 2 * NP + (uh & 1) * NP + c];
  }
  z[(int64_t)tblk[i] * NP + c] += theta * acc;
}

}  // namespace xdg
