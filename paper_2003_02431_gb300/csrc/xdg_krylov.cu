// Multi-vector Krylov kernels of libxdg (sm_103a); see xdg_krylov.h. All reductions run in a
// fixed order (per-CTA partial sums, then one CTA adding them in CTA order), so results are
// bitwise repeatable.
#include <algorithm>

#include "xdg_common.cuh"
#include "xdg_krylov.h"

namespace xdg {
namespace kry {
namespace {

constexpr int kVec = 8;  // stored vectors per sweep of the multi-dot (accumulators per thread)

__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double sh[32];
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  return s;  // valid in thread 0
}

// part[blockIdx.x * l + i] = this CTA's share of V_i . w; kVec vectors per pass over w
__global__ void __launch_bounds__(kThreads) k_mdot(int64_t n, int l, const double* __restrict__ V,
                                                  const double* __restrict__ w, double* __restrict__ part) {
  pdl_entry();
  for (int i0 = 0; i0 < l; i0 += kVec) {
    const int m = min(kVec, l - i0);
    double s[kVec];
#pragma unroll
    for (int u = 0; u < kVec; ++u) s[u] = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
      const double wk = w[k];
#pragma unroll
      for (int u = 0; u < kVec; ++u)
        if (u < m) s[u] = fma(__ldg(V + (int64_t)(i0 + u) * n + k), wk, s[u]);
    }
    for (int u = 0; u < m; ++u) {
      const double t = block_sum_d(s[u]);
      if (threadIdx.x == 0) part[(int64_t)blockIdx.x * l + i0 + u] = t;
    }
  }
}

__global__ void k_mdot_final(int grid, int l, const double* __restrict__ part, double* __restrict__ beta,
                             double* __restrict__ acc) {
  pdl_entry();
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < grid; ++b) s += part[(int64_t)b * l + i];
    beta[i] = s;
    if (acc) acc[i] += s;
  }
}

__global__ void __launch_bounds__(kThreads) k_gs_update(int64_t n, int l, const double* __restrict__ V,
                                                       const double* __restrict__ Z, const double* __restrict__ beta,
                                                       double* __restrict__ w, double* __restrict__ z) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double wk = w[k], zk = Z ? z[k] : 0.0;
    for (int i = 0; i < l; ++i) {
      const double b = __ldg(beta + i);
      wk = fma(-b, __ldg(V + (int64_t)i * n + k), wk);
      if (Z) zk = fma(-b, __ldg(Z + (int64_t)i * n + k), zk);
    }
    w[k] = wk;
    if (Z) z[k] = zk;
  }
}

__global__ void __launch_bounds__(kThreads) k_normalize(int64_t n, const double* __restrict__ nrm2,
                                                       const double* __restrict__ w0sq, double* __restrict__ w,
                                                       const double* __restrict__ zin, double* __restrict__ zout,
                                                       double* __restrict__ gam_out) {
  pdl_entry();
  const double q = *nrm2;
  const double g = (q > 1e-28 * *w0sq && q > 0.0) ? 1.0 / sqrt(q) : 0.0;
  if (gam_out && blockIdx.x == 0 && threadIdx.x == 0) *gam_out = g;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    w[k] *= g;
    if (zout) zout[k] = g * zin[k];
  }
}

__global__ void __launch_bounds__(kThreads) k_rm_update(int64_t n, const double* __restrict__ alpha,
                                                       const double* __restrict__ z, const double* __restrict__ w,
                                                       double* __restrict__ x, double* __restrict__ r) {
  pdl_entry();
  const double a = *alpha;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    x[k] = fma(a, z[k], x[k]);
    r[k] = fma(-a, w[k], r[k]);
  }
}

__global__ void k_givens(int j, int ld, double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ g, const double* __restrict__ hnorm2) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* h = H + (int64_t)j * ld;
  h[j + 1] = sqrt(fmax(*hnorm2, 0.0));
  for (int i = 0; i < j; ++i) {  // previous rotations
    const double a = h[i], b = h[i + 1];
    h[i] = cs[i] * a + sn[i] * b;
    h[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = h[j], b = h[j + 1];
  const double rr = hypot(a, b);
  const double c = rr > 0.0 ? a / rr : 1.0, s_ = rr > 0.0 ? b / rr : 0.0;
  cs[j] = c;
  sn[j] = s_;
  h[j] = rr;
  h[j + 1] = 0.0;
  const double gj = g[j];
  g[j] = c * gj;
  g[j + 1] = -s_ * gj;
}

__global__ void k_gmres_start(int m, const double* __restrict__ nrm2, double* __restrict__ g,
                              double* __restrict__ inv) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double beta = sqrt(fmax(*nrm2, 0.0));
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  *inv = beta > 0.0 ? 1.0 / beta : 0.0;
}

__global__ void k_gmres_solve(int k, int ld, const double* __restrict__ H, const double* __restrict__ g,
                              double* __restrict__ ny) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s += H[(int64_t)c * ld + i] * ny[c];  // ny holds -y
    const double d = H[(int64_t)i * ld + i];
    ny[i] = d != 0.0 ? -s / d : 0.0;
  }
}

__global__ void __launch_bounds__(kThreads) k_scale(int64_t n, const double* __restrict__ a,
                                                   const double* __restrict__ x, double* __restrict__ y) {
  pdl_entry();
  const double s = *a;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = s * x[k];
}

template <class K, class... A>
cudaError_t launch(K k, int grid, int threads, cudaStream_t s, A... a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::max(1, grid));
  cfg.blockDim = dim3(threads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, a...);
}

}  // namespace

cudaError_t mdot_partial(cudaStream_t s, int grid, int64_t n, int l, const double* V, const double* w, double* part) {
  if (l <= 0) return cudaSuccess;
  return launch(k_mdot, grid, kThreads, s, n, l, V, w, part);
}

cudaError_t mdot_final(cudaStream_t s, int grid, int l, const double* part, double* beta, double* acc) {
  if (l <= 0) return cudaSuccess;
  return launch(k_mdot_final, 1, 128, s, grid, l, part, beta, acc);
}

cudaError_t gs_update(cudaStream_t s, int grid, int64_t n, int l, const double* V, const double* Z, const double* beta,
                      double* w, double* z) {
  if (l <= 0) return cudaSuccess;
  return launch(k_gs_update, grid, kThreads, s, n, l, V, Z, beta, w, z);
}

cudaError_t normalize(cudaStream_t s, int grid, int64_t n, const double* nrm2, const double* w0sq, double* w,
                      const double* zin, double* zout, double* gam_out) {
  return launch(k_normalize, grid, kThreads, s, n, nrm2, w0sq, w, zin, zout, gam_out);
}

cudaError_t rm_update(cudaStream_t s, int grid, int64_t n, const double* alpha, const double* z, const double* w,
                      double* x, double* r) {
  return launch(k_rm_update, grid, kThreads, s, n, alpha, z, w, x, r);
}

cudaError_t givens(cudaStream_t s, int j, int ld, double* H, double* cs, double* sn, double* g, const double* hnorm2) {
  return launch(k_givens, 1, 32, s, j, ld, H, cs, sn, g, hnorm2);
}

cudaError_t gmres_start(cudaStream_t s, int m, const double* nrm2, double* g, double* inv) {
  return launch(k_gmres_start, 1, 32, s, m, nrm2, g, inv);
}

cudaError_t gmres_solve(cudaStream_t s, int k, int ld, const double* H, const double* g, double* ny) {
  return launch(k_gmres_solve, 1, 32, s, k, ld, H, g, ny);
}

cudaError_t scale(cudaStream_t s, int grid, int64_t n, const double* a, const double* x, double* y) {
  return launch(k_scale, grid, kThreads, s, n, a, x, y);
}

}  // namespace kry
}  // namespace xdg

namespace xdg {
namespace pmg {
namespace {

__global__ void k_sub_blocks(int64_t nblk, int np, int n_lo, const double* __restrict__ src, double* __restrict__ dst) {
  pdl_entry();
  const int64_t m2 = (int64_t)n_lo * n_lo;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nblk * m2; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = e / m2;
    const int k = (int)(e - z * m2), r = k / n_lo, c = k - r * n_lo;
    dst[e] = src[z * np * np + r * np + c];
  }
}

__global__ void k_take_lo(int64_t nb, int np, int n_lo, const double* __restrict__ v, double* __restrict__ lo) {
  pdl_entry();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nb * n_lo; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n_lo;
    lo[e] = v[i * np + (e - i * n_lo)];
  }
}

__global__ void k_put_lo(int64_t nb, int np, int n_lo, const double* __restrict__ lo, double* __restrict__ z) {
  pdl_entry();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nb * np; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / np;
    const int r = (int)(e - i * np);
    z[e] = r < n_lo ? lo[i * n_lo + r] : 0.0;
  }
}

// largest trailing (high-order) sub-block: k = 5 in 3D (56 modes) above k_lo = 1 (4 modes)
constexpr int kHiMax = 64;

// one CTA of 32 threads per block: the trailing sub-block in shared memory, Cholesky by one
// thread (m <= kHiMax), inverse columns by the threads
__global__ void k_hi_inv(int64_t nb, int np, int n_lo, const int64_t* __restrict__ diag,
                         const double* __restrict__ val, double* __restrict__ Hinv, int* __restrict__ err) {
  pdl_entry();
  __shared__ double A[kHiMax * kHiMax];
  __shared__ int bad;
  const int m = np - n_lo;
  for (int64_t i = blockIdx.x; i < nb; i += gridDim.x) {
    const double* B = val + diag[i] * np * np;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) A[e] = B[(n_lo + e / m) * np + n_lo + e % m];
    __syncthreads();
    if (threadIdx.x == 0) {
      bad = 0;
      for (int j = 0; j < m; ++j) {
        double d = A[j * m + j];
        for (int p = 0; p < j; ++p) d -= A[j * m + p] * A[j * m + p];
        if (!(d > 0.0)) {
          bad = 1;
          d = 1.0;
        }
        d = sqrt(d);
        A[j * m + j] = d;
        for (int r = j + 1; r < m; ++r) {
          double t = A[r * m + j];
          for (int p = 0; p < j; ++p) t -= A[r * m + p] * A[j * m + p];
          A[r * m + j] = t / d;
        }
      }
      if (bad) atomicExch(err, 1);
    }
    __syncthreads();
    double* X = Hinv + i * m * m;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {  // column j: L y = e_j, L^T x = y
      double y[kHiMax];
      for (int r = 0; r < m; ++r) {
        double t = (r == j) ? 1.0 : 0.0;
        for (int p = 0; p < r; ++p) t -= A[r * m + p] * y[p];
        y[r] = t / A[r * m + r];
      }
      for (int r = m - 1; r >= 0; --r) {
        double t = y[r];
        for (int p = r + 1; p < m; ++p) t -= A[p * m + r] * y[p];
        y[r] = t / A[r * m + r];
      }
      for (int r = 0; r < m; ++r) X[r * m + j] = y[r];
    }
    __syncthreads();
  }
}

__global__ void k_hi_apply(int64_t nb, int np, int n_lo, const double* __restrict__ Hinv,
                           const double* __restrict__ res, double* __restrict__ z) {
  pdl_entry();
  const int m = np - n_lo;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nb * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / m;
    const int r = (int)(e - i * m);
    const double* h = Hinv + i * m * m + r * m;
    const double* q = res + i * np + n_lo;
    double s = 0.0;
    for (int c = 0; c < m; ++c) s = fma(h[c], q[c], s);
    z[i * np + n_lo + r] += s;
  }
}

template <class K, class... A>
cudaError_t launch_n(K k, int64_t work, int threads, cudaStream_t s, A... a) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 152 * 16));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(threads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, a...);
}

}  // namespace

cudaError_t sub_blocks(cudaStream_t s, int64_t nblk, int np, int n_lo, const double* src, double* dst) {
  return launch_n(k_sub_blocks, nblk * n_lo * n_lo, kThreads, s, nblk, np, n_lo, src, dst);
}
cudaError_t take_lo(cudaStream_t s, int64_t nb, int np, int n_lo, const double* v, double* lo) {
  return launch_n(k_take_lo, nb * n_lo, kThreads, s, nb, np, n_lo, v, lo);
}
cudaError_t put_lo(cudaStream_t s, int64_t nb, int np, int n_lo, const double* lo, double* z) {
  return launch_n(k_put_lo, nb * np, kThreads, s, nb, np, n_lo, lo, z);
}
cudaError_t hi_inverses(cudaStream_t s, int64_t nb, int np, int n_lo, const int64_t* diag, const double* val,
                        double* Hinv, int* err) {
  if (np - n_lo < 1 || np - n_lo > kHiMax) return cudaErrorInvalidValue;
  return launch_n(k_hi_inv, nb * 32, 32, s, nb, np, n_lo, diag, val, Hinv, err);
}
cudaError_t hi_apply(cudaStream_t s, int64_t nb, int np, int n_lo, const double* Hinv, const double* res, double* z) {
  return launch_n(k_hi_apply, nb * (np - n_lo), kThreads, s, nb, np, n_lo, Hinv, res, z);
}

}  // namespace pmg
}  // namespace xdg
