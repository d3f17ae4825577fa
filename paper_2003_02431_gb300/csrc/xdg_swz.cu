// Additive Schwarz smoother kernels of libxdg (sm_103a): patch matrix hashing, factorisation
// and inversion at setup, and the patch solves of every smoothing step.
//
// Kummer, Smuda, Weber, arXiv 2003.02431, Algorithm Swz with exact patch solves (the
// p-multigrid block solver of Algorithm pMultigrid with every mode in the low-order set, i.e.
// a dense direct solve of M restricted to the patch). See xdg_swz.h for the operation.
//
// Work mapping of a smoothing step: one warp per patch. The patch's right-hand side
// (alpha^{-1/2}-scaled, n = blocks x Np values) is gathered into shared memory, then lane i
// accumulates rows i, i+32, ... of the stored inverse times it, reading the inverse column by
// column (32 consecutive entries per load instruction). Patches with bitwise equal matrices
// (away from the interface and the boundary most patches of a Cartesian mesh are) share one
// stored inverse, which then stays in L2 and L1: a step streams little more than the vectors.
#include <algorithm>

#include "xdg_common.cuh"
#include "xdg_swz.h"

namespace xdg {
namespace swz {
namespace {

constexpr int kWarps = 8;  // warps (patches in flight) per CTA of the patch kernels

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  // splitmix64 finaliser (Steele, Lea, Flood 2014)
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// position of block j among the patch's blocks pb[0..nbp) (ascending), -1 if absent
__device__ __forceinline__ int find_member(const int32_t* __restrict__ pb, int nbp, int32_t j) {
  int lo = 0, hi = nbp - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int32_t v = __ldg(pb + mid);
    if (v == j) return mid;
    if (v < j) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

template <int NP>
__global__ void __launch_bounds__(kThreads) k_swz_hash(int64_t npatch, const int64_t* __restrict__ pptr,
                                                      const int32_t* __restrict__ pblk,
                                                      const int64_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ val,
                                                      unsigned long long* __restrict__ h) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = w0; p < npatch; p += nw) {
    const int64_t p0 = pptr[p];
    const int nbp = (int)(pptr[p + 1] - p0);
    const int64_t n = (int64_t)nbp * NP;
    unsigned long long h1 = 0, h2 = 0;
    for (int a = 0; a < nbp; ++a) {
      const int32_t i = __ldg(pblk + p0 + a);
      for (int64_t z = __ldg(rp + i); z < __ldg(rp + i + 1); ++z) {
        const int c = find_member(pblk + p0, nbp, __ldg(col + z));
        if (c < 0) continue;
        for (int e = lane; e < NP * NP; e += 32) {
          const int r = e / NP, q = e - r * NP;
          const unsigned long long idx = (unsigned long long)((a * NP + r) * n + c * NP + q);
          const unsigned long long bits = (unsigned long long)__double_as_longlong(__ldg(val + z * (NP * NP) + e));
          h1 += mix64(bits ^ mix64(idx));
          h2 += mix64((bits + 0x632BE59BD9B4E019ull * (idx + 1)) ^ 0xD6E8FEB86659FD93ull);
        }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      h1 += __shfl_xor_sync(0xffffffffu, h1, o);
      h2 += __shfl_xor_sync(0xffffffffu, h2, o);
    }
    if (lane == 0) {
      h[2 * p] = h1 ^ mix64((unsigned long long)n);
      h[2 * p + 1] = h2 + mix64((unsigned long long)n + 7);
    }
  }
}

// one CTA per distinct patch: gather, Cholesky (lower, in place), inverse column by column,
// symmetrised, FP32 copy
template <int NP>
__global__ void __launch_bounds__(256) k_swz_factor(int64_t u0, int64_t u1, const int64_t* __restrict__ rep,
                                                   const int64_t* __restrict__ pptr,
                                                   const int32_t* __restrict__ pblk,
                                                   const int64_t* __restrict__ rp,
                                                   const int32_t* __restrict__ col,
                                                   const double* __restrict__ val,
                                                   const int64_t* __restrict__ ioff, double* __restrict__ work,
                                                   const int64_t* __restrict__ woff, double* __restrict__ Ainv,
                                                   float* __restrict__ Ainv32, int* __restrict__ err) {
  pdl_entry();
  __shared__ int bad;
  for (int64_t u = u0 + blockIdx.x; u < u1; u += gridDim.x) {
    const int64_t p = rep[u], p0 = pptr[p];
    const int nbp = (int)(pptr[p + 1] - p0);
    const int n = nbp * NP;
    double* W = work + woff[u - u0];
    double* X = Ainv + ioff[u];
    float* X32 = Ainv32 + ioff[u];
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) W[e] = 0.0;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int a = 0; a < nbp; ++a) {
      const int32_t i = pblk[p0 + a];
      for (int64_t z = rp[i]; z < rp[i + 1]; ++z) {
        const int c = find_member(pblk + p0, nbp, col[z]);
        if (c < 0) continue;
        for (int e = threadIdx.x; e < NP * NP; e += blockDim.x) {
          const int r = e / NP, q = e - r * NP;
          W[(int64_t)(a * NP + r) * n + c * NP + q] = val[z * (NP * NP) + e];
        }
      }
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      if (threadIdx.x == 0) {
        double d = W[(int64_t)k * n + k];
        if (!(d > 0.0)) {
          bad = 1;
          d = 1.0;
        }
        W[(int64_t)k * n + k] = sqrt(d);
      }
      __syncthreads();
      const double dk = W[(int64_t)k * n + k];
      for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) W[(int64_t)i * n + k] /= dk;
      __syncthreads();
      const int m = n - k - 1;
      for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
        const int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
        if (j <= i) W[(int64_t)i * n + j] -= W[(int64_t)i * n + k] * W[(int64_t)j * n + k];
      }
      __syncthreads();
    }
    if (bad) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
        X[e] = 0.0;
        X32[e] = 0.0f;
      }
      __syncthreads();
      continue;
    }
    // column j of the inverse: L y = e_j, then L^T x = y (stored at X + j n)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double* x = X + (int64_t)j * n;
      for (int i = 0; i < j; ++i) x[i] = 0.0;
      for (int i = j; i < n; ++i) {
        double s = (i == j) ? 1.0 : 0.0;
        for (int k = j; k < i; ++k) s -= W[(int64_t)i * n + k] * x[k];
        x[i] = s / W[(int64_t)i * n + i];
      }
      for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < n; ++k) s -= W[(int64_t)k * n + i] * x[k];
        x[i] = s / W[(int64_t)i * n + i];
      }
    }
    __syncthreads();
    // symmetrise (the two triangles come from different columns' substitutions)
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
      const int i = (int)(e / n), j = (int)(e % n);
      if (j > i) {
        const double s = 0.5 * (X[(int64_t)i * n + j] + X[(int64_t)j * n + i]);
        X[(int64_t)i * n + j] = s;
        X[(int64_t)j * n + i] = s;
      }
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) X32[e] = (float)X[e];
    __syncthreads();
  }
}

template <class T>
__device__ __forceinline__ T ldg_t(const T* p) {
  return __ldg(p);
}

// inverses staged in shared memory (two buffers) up to n = stage_max_n (others are read from
// global memory): 2 n^2 sizeof(T) <= ~100 KB, so that two CTAs fit on an SM
template <class T>
constexpr int stage_max_n() {
  return sizeof(T) == 8 ? 78 : 110;
}

// y = A (isq .* r)_P for one patch (one warp), A column-major n x n (the symmetric inverse);
// R = rows per lane = ceil(n / 32) as a compile-time constant (up to 8), so that the inner loop
// issues only the loads and FMAs of real rows; larger patches take the loop with R = 16 rows
// guarded at run time. np (modes per block) and the output form are run-time values: they
// only enter the gather and the scatter.
template <class T>
__device__ __forceinline__ void patch_gather(T* v, int64_t p0, int n, int np, const int32_t* __restrict__ pblk,
                                             const T* __restrict__ isq, const T* __restrict__ r) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < n; e += 32) {
    const int a = e / np, q = e - a * np;
    const int32_t b = __ldg(pblk + p0 + a);
    v[e] = ldg_t(isq + b) * r[(int64_t)b * np + q];
  }
  __syncwarp();
}

template <class T>
__device__ __forceinline__ void patch_store(int i, T acc, int64_t p0, int np, int out_mode,
                                            const int32_t* __restrict__ pblk, const T* __restrict__ isq, T om,
                                            const T* __restrict__ xin, T* __restrict__ out) {
  const int a = i / np, q = i - a * np;
  if (out_mode == 0) {
    out[(p0 + a) * np + q] = acc;
  } else {
    const int32_t b = __ldg(pblk + p0 + a);
    const int64_t o = (int64_t)b * np + q;
    const T y = om * ldg_t(isq + b) * acc;
    out[o] = (out_mode == 2) ? xin[o] + y : y;
  }
}

template <class T, int R>
__device__ __forceinline__ void patch_solve_r(const T* A, T* v, int64_t p0, int n, int np, int out_mode,
                                              const int32_t* __restrict__ pblk, const T* __restrict__ isq,
                                              const T* __restrict__ r, T om, const T* __restrict__ xin,
                                              T* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  patch_gather(v, p0, n, np, pblk, isq, r);
  // rows lane + 32k; a row beyond n reads row n - 1 (in bounds) and is not stored
  int row[R];
#pragma unroll
  for (int k = 0; k < R; ++k) row[k] = min(lane + 32 * k, n - 1);
  T acc[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = T(0);
  int j = 0;
  for (; j + 2 <= n; j += 2) {  // two columns per step: more loads in flight
    const T v0 = v[j], v1 = v[j + 1];
    const T* A0 = A + (int64_t)j * n;
    const T* A1 = A0 + n;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const T a0 = A0[row[k]], a1 = A1[row[k]];
      acc[k] = fma(a0, v0, acc[k]);
      acc[k] = fma(a1, v1, acc[k]);
    }
  }
  if (j < n) {
    const T v0 = v[j];
    const T* A0 = A + (int64_t)j * n;
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = fma(A0[row[k]], v0, acc[k]);
  }
#pragma unroll
  for (int k = 0; k < R; ++k)
    if (lane + 32 * k < n) patch_store(lane + 32 * k, acc[k], p0, np, out_mode, pblk, isq, om, xin, out);
  __syncwarp();
}

// patches of more than 256 modes: rows guarded at run time
template <class T>
__device__ __forceinline__ void patch_solve_big(const T* A, T* v, int64_t p0, int n, int np, int out_mode,
                                                const int32_t* __restrict__ pblk, const T* __restrict__ isq,
                                                const T* __restrict__ r, T om, const T* __restrict__ xin,
                                                T* __restrict__ out) {
  constexpr int RB = kMaxDof / 32;
  const int lane = threadIdx.x & 31;
  patch_gather(v, p0, n, np, pblk, isq, r);
  const int rows = (n + 31) >> 5;
  T acc[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) acc[k] = T(0);
  for (int j = 0; j < n; ++j) {
    const T vj = v[j];
    const T* Aj = A + (int64_t)j * n;
#pragma unroll
    for (int k = 0; k < RB; ++k) {
      const int i = lane + 32 * k;
      if (k < rows && i < n) acc[k] = fma(Aj[i], vj, acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < RB; ++k)
    if (k < rows && lane + 32 * k < n) patch_store(lane + 32 * k, acc[k], p0, np, out_mode, pblk, isq, om, xin, out);
  __syncwarp();
}

template <class T>
__device__ __forceinline__ void patch_solve(const T* A, T* v, int64_t p0, int n, int np, int out_mode,
                                            const int32_t* __restrict__ pblk, const T* __restrict__ isq,
                                            const T* __restrict__ r, T om, const T* __restrict__ xin,
                                            T* __restrict__ out) {
  switch ((n + 31) >> 5) {
#define R_(K) \
  case K: patch_solve_r<T, K>(A, v, p0, n, np, out_mode, pblk, isq, r, om, xin, out); break;
    R_(1) R_(2) R_(3) R_(4) R_(5) R_(6) R_(7) R_(8)
#undef R_
    default: patch_solve_big<T>(A, v, p0, n, np, out_mode, pblk, isq, r, om, xin, out); break;
  }
}

// one patch spread over the CTA: warp w adds the columns of its slice for rows lane + 32k,
// partial sums into part[w * vstride + i]; R rows per lane (R = 16: rows guarded at run time)
template <class T, int R>
__device__ __forceinline__ void split_cols(const T* A, const T* vc, T* part, int vstride, int n) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per = (n + kWarps - 1) / kWarps;
  const int j0 = wid * per, j1 = min(n, j0 + per);
  const int rows = (n + 31) >> 5;
  int row[R];
#pragma unroll
  for (int k = 0; k < R; ++k) row[k] = min(lane + 32 * k, n - 1);
  T acc[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = T(0);
  for (int j = j0; j < j1; ++j) {
    const T vj = vc[j];
    const T* Aj = A + (int64_t)j * n;
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (R <= 8 || k < rows) acc[k] = fma(Aj[row[k]], vj, acc[k]);
  }
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int i = lane + 32 * k;
    if ((R <= 8 || k < rows) && i < n) part[wid * vstride + i] = acc[k];
  }
}

// 16-byte asynchronous global -> shared copies (LDGSTS), completed by wait_group
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// start copying an n x n inverse (padded to 16 bytes; inverses start 16-byte aligned) into buf
template <class T>
__device__ __forceinline__ void stage_async(T* buf, const T* Ag, int n) {
  const int chunks = (int)(((size_t)n * n * sizeof(T) + 15) / 16);
  const char* src = reinterpret_cast<const char*>(Ag);
  char* dst = reinterpret_cast<char*>(buf);
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) cp_async16(dst + 16 * c, src + 16 * c);
}

// One CTA per work item, items of a CTA in a double-buffered pipeline: while the CTA solves the
// patches of one item from its inverse in shared memory, the next item's inverse streams in
// (asynchronous copies). An item of several patches (a shared inverse) gives each warp its own
// patches; an item of one patch (a distinct inverse) spreads the patch's rows over the CTA.
// Inverses larger than the staging buffer are read from global memory.
template <class T>
__global__ void __launch_bounds__(kWarps * 32) k_swz_apply(int64_t nitem, const Item* __restrict__ items,
                                                          const int32_t* __restrict__ porder,
                                                          const int64_t* __restrict__ pptr,
                                                          const int32_t* __restrict__ pblk,
                                                          const int64_t* __restrict__ ioff,
                                                          const T* __restrict__ Ainv, const T* __restrict__ isq,
                                                          const T* __restrict__ r, T om, const T* __restrict__ xin,
                                                          T* __restrict__ out, int vstride, int stage_n, int np,
                                                          int out_mode) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int sbuf = ((stage_n * stage_n + 3) / 4) * 4;  // elements per staging buffer (16-byte multiple)
  T* bufs = reinterpret_cast<T*>(sm_raw);
  T* vall = bufs + 2 * sbuf;
  T* vc = vall + kWarps * vstride;  // the CTA's vector (one-patch items)
  T* v = vall + (threadIdx.x >> 5) * vstride;
  const int wid = threadIdx.x >> 5;
  int buf = 0;
  int64_t it = blockIdx.x;
  if (it < nitem) {
    const Item I = items[it];
    if (I.n <= stage_n) stage_async(bufs, Ainv + __ldg(ioff + I.tid), I.n);
  }
  cp_async_commit();
  for (; it < nitem; it += gridDim.x) {
    const Item I = items[it];
    const int64_t nx = it + gridDim.x;
    if (nx < nitem) {
      const Item J = items[nx];
      if (J.n <= stage_n) stage_async(bufs + (buf ^ 1) * sbuf, Ainv + __ldg(ioff + J.tid), J.n);
    }
    cp_async_commit();
    cp_async_wait<1>();  // every group but the newest: this item's inverse is in
    __syncthreads();
    const T* A = (I.n <= stage_n) ? bufs + buf * sbuf : Ainv + __ldg(ioff + I.tid);
    if (I.count > 1) {
      for (int q = wid; q < I.count; q += kWarps) {
        const int64_t p0 = __ldg(pptr + __ldg(porder + I.start + q));
        patch_solve<T>(A, v, p0, I.n, np, out_mode, pblk, isq, r, om, xin, out);
      }
    } else {
      const int n = I.n;
      const int64_t p0 = __ldg(pptr + __ldg(porder + I.start));
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int a = e / np, q = e - a * np;
        const int32_t b = __ldg(pblk + p0 + a);
        vc[e] = ldg_t(isq + b) * r[(int64_t)b * np + q];
      }
      __syncthreads();
      // the columns split over the warps (short dependent chains), partial sums per warp in
      // the warps' vector space, added in warp order
      switch ((n + 31) >> 5) {
#define R_(K) \
  case K: split_cols<T, K>(A, vc, vall, vstride, n); break;
        R_(1) R_(2) R_(3) R_(4) R_(5) R_(6) R_(7) R_(8)
#undef R_
        default: split_cols<T, kMaxDof / 32>(A, vc, vall, vstride, n); break;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T acc = T(0);
        for (int w = 0; w < kWarps; ++w) acc += vall[w * vstride + i];
        patch_store(i, acc, p0, np, out_mode, pblk, isq, om, xin, out);
      }
    }
    __syncthreads();  // the buffer is refilled two items later
    buf ^= 1;
  }
  cp_async_wait<0>();
}

// dynamic shared memory a CTA may opt into (227 KB)
constexpr size_t kSmemOptIn = 232448;

template <int NP, class T, bool ZERO>
__global__ void __launch_bounds__(kThreads) k_swz_accum(int64_t nb, const int64_t* __restrict__ bsptr,
                                                       const int64_t* __restrict__ bslot,
                                                       const T* __restrict__ isq, const T* __restrict__ y, T om,
                                                       const T* __restrict__ xin, T* __restrict__ out) {
  pdl_entry();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nb * NP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / NP;
    const int q = (int)(e - i * NP);
    T s = T(0);
    for (int64_t k = __ldg(bsptr + i); k < __ldg(bsptr + i + 1); ++k) s += y[__ldg(bslot + k) * NP + q];
    const T d = om * ldg_t(isq + i) * s;
    out[e] = ZERO ? d : xin[e] + d;
  }
}

inline cudaLaunchConfig_t pdl_cfg(dim3 g, dim3 b, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <int NP>
cudaError_t hash_t(cudaStream_t s, int64_t npatch, const int64_t* pptr, const int32_t* pblk, const int64_t* rp,
                   const int32_t* col, const double* val, unsigned long long* h) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((npatch + 7) / 8, 4096));
  k_swz_hash<NP><<<(unsigned)blocks, kThreads, 0, s>>>(npatch, pptr, pblk, rp, col, val, h);
  return cudaGetLastError();
}

template <int NP>
cudaError_t factor_t(cudaStream_t s, int64_t u0, int64_t u1, const int64_t* rep, const int64_t* pptr,
                     const int32_t* pblk, const int64_t* rp, const int32_t* col, const double* val,
                     const int64_t* ioff, double* work, const int64_t* woff, double* Ainv, float* Ainv32, int* err) {
  if (u1 <= u0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>(u1 - u0, 65535);
  k_swz_factor<NP><<<(unsigned)blocks, 256, 0, s>>>(u0, u1, rep, pptr, pblk, rp, col, val, ioff, work, woff, Ainv,
                                                     Ainv32, err);
  return cudaGetLastError();
}

template <class T>
cudaError_t prepare_t() {
  return cudaFuncSetAttribute(k_swz_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemOptIn);
}

template <class T>
cudaError_t apply_t(int np, cudaStream_t s, int grid, int out_mode, int64_t nitem, const Item* items,
                    const int32_t* porder, const int64_t* pptr, const int32_t* pblk, const int64_t* ioff,
                    const T* Ainv, const T* isq, const T* r, T om, const T* xin, T* out, int maxdof, int stage_n) {
  cudaLaunchAttribute at[1];
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(grid, nitem));
  cudaLaunchConfig_t cfg = pdl_cfg(dim3(g), dim3(kWarps * 32), s, at);
  stage_n = std::min(stage_n, stage_max_n<T>());
  maxdof = (maxdof + 3) / 4 * 4;
  auto smem = [&](int sn) {
    return ((size_t)2 * ((sn * sn + 3) / 4 * 4) + (size_t)(kWarps + 1) * maxdof) * sizeof(T);
  };
  while (stage_n > 0 && smem(stage_n) > kSmemOptIn) --stage_n;
  cfg.dynamicSmemBytes = smem(stage_n);
  return cudaLaunchKernelEx(&cfg, k_swz_apply<T>, nitem, items, porder, pptr, pblk, ioff, Ainv, isq, r, om, xin, out,
                            maxdof, stage_n, np, out_mode);
}

template <int NP, class T>
cudaError_t accum_t(cudaStream_t s, int grid, int64_t nb, const int64_t* bsptr, const int64_t* bslot, const T* isq,
                    const T* y, T om, const T* xin, T* out) {
  cudaLaunchAttribute at[1];
  const int64_t need = (nb * NP + kThreads - 1) / kThreads;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(grid, need));
  cudaLaunchConfig_t cfg = pdl_cfg(dim3(g), dim3(kThreads), s, at);
  if (xin) return cudaLaunchKernelEx(&cfg, k_swz_accum<NP, T, false>, nb, bsptr, bslot, isq, y, om, xin, out);
  return cudaLaunchKernelEx(&cfg, k_swz_accum<NP, T, true>, nb, bsptr, bslot, isq, y, om, xin, out);
}

}  // namespace

#define XDG_SWZ_NP(X) X(6) X(10) X(15) X(20)

cudaError_t hash(int np, cudaStream_t s, int64_t npatch, const int64_t* pptr, const int32_t* pblk,
                 const int64_t* rp, const int32_t* col, const double* val, unsigned long long* h) {
  switch (np) {
#define C_(N) \
  case N: return hash_t<N>(s, npatch, pptr, pblk, rp, col, val, h);
    XDG_SWZ_NP(C_)
#undef C_
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t factor(int np, cudaStream_t s, int64_t u0, int64_t u1, const int64_t* rep, const int64_t* pptr,
                   const int32_t* pblk, const int64_t* rp, const int32_t* col, const double* val,
                   const int64_t* ioff, double* work, const int64_t* woff, double* Ainv, float* Ainv32, int* err) {
  switch (np) {
#define C_(N) \
  case N: return factor_t<N>(s, u0, u1, rep, pptr, pblk, rp, col, val, ioff, work, woff, Ainv, Ainv32, err);
    XDG_SWZ_NP(C_)
#undef C_
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prepare(int np) {
  if (np < 1 || np > 32) return cudaErrorInvalidValue;
  cudaError_t e = prepare_t<double>();
  return e == cudaSuccess ? prepare_t<float>() : e;
}

template <class T>
cudaError_t apply(int np, cudaStream_t s, int grid, int out_mode, int64_t nitem, const Item* items,
                  const int32_t* porder, const int64_t* pptr, const int32_t* pblk, const int64_t* ioff,
                  const T* Ainv, const T* isq, const T* r, T om, const T* xin, T* out, int maxdof, int stage_n) {
  if (np < 1 || np > 32) return cudaErrorInvalidValue;
  return apply_t<T>(np, s, grid, out_mode, nitem, items, porder, pptr, pblk, ioff, Ainv, isq, r, om, xin, out, maxdof,
                    stage_n);
}

template <class T>
cudaError_t accum(int np, cudaStream_t s, int grid, int64_t nb, const int64_t* bsptr, const int64_t* bslot,
                  const T* isq, const T* y, T om, const T* xin, T* out) {
  switch (np) {
#define C_(N) \
  case N: return accum_t<N, T>(s, grid, nb, bsptr, bslot, isq, y, om, xin, out);
    XDG_SWZ_NP(C_)
#undef C_
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t apply<double>(int, cudaStream_t, int, int, int64_t, const Item*, const int32_t*, const int64_t*,
                                   const int32_t*, const int64_t*, const double*, const double*, const double*,
                                   double, const double*, double*, int, int);
template cudaError_t apply<float>(int, cudaStream_t, int, int, int64_t, const Item*, const int32_t*, const int64_t*,
                                  const int32_t*, const int64_t*, const float*, const float*, const float*, float,
                                  const float*, float*, int, int);
template cudaError_t accum<double>(int, cudaStream_t, int, int64_t, const int64_t*, const int64_t*, const double*,
                                   const double*, double, const double*, double*);
template cudaError_t accum<float>(int, cudaStream_t, int, int64_t, const int64_t*, const int64_t*, const float*,
                                  const float*, float, const float*, float*);

}  // namespace swz
}  // namespace xdg
