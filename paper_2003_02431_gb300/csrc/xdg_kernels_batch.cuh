// Kernels for batches of independent problems solved in one hierarchy: the problems' level
// operators are concatenated block-diagonally; per-problem quantities (damping, coarsest
// inverses, Krylov scalars) are addressed through segment offsets. A single problem is the
// batch of one (one segment).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "xdg_kernels.cuh"

namespace xdg {

// segment containing position i: largest s with off[s] <= i (off ascending, nseg+1 entries)
__device__ __forceinline__ int find_seg(const int64_t* __restrict__ off, int nseg, int64_t i) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// part[s * spl + blockIdx.x] = partial sum of x_i y_i over slice blockIdx.x of segment
// s = blockIdx.y (spl slices per segment, fixed order); k_seg_sum adds the slices in order
__global__ void __launch_bounds__(kThreads) k_seg_dot(int nseg, const int64_t* __restrict__ off,
                                                     const double* __restrict__ x, const double* __restrict__ y,
                                                     double* __restrict__ part) {
  pdl_entry();
  const int s = blockIdx.y, spl = gridDim.x;
  if (s >= nseg) return;
  const int64_t lo = off[s], len = off[s + 1] - lo;
  const int64_t a = lo + len * blockIdx.x / spl, b = lo + len * (blockIdx.x + 1) / spl;
  double acc = 0.0;
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) acc = fma(x[i], y[i], acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[(int64_t)s * spl + blockIdx.x] = acc;
}
__global__ void k_seg_sum(int nseg, int spl, const double* __restrict__ part, double* __restrict__ out) {
  pdl_entry();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < spl; ++j) acc += part[(int64_t)s * spl + j];
    out[s] = acc;
  }
}

// x_i *= a[s(i)] ; y_i += a[s(i)] x_i  (segment-wise scalars; seg = entry -> segment via off)
__global__ void k_seg_scale(int64_t n, int nseg, const int64_t* __restrict__ off, const double* __restrict__ a,
                            double* __restrict__ x) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= a[find_seg(off, nseg, i)];
}
__global__ void k_seg_axpy(int64_t n, int nseg, const int64_t* __restrict__ off, const double* __restrict__ a,
                           const double* __restrict__ x, double* __restrict__ y) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a[find_seg(off, nseg, i)], x[i], y[i]);
}

// v_i = ((j+1) * 2654435761 mod 2^32) / 2^32 - 0.5 with j the index of i inside its segment
// (Knuth's multiplicative hash, restarted at every problem)
__global__ void k_hash_vector_seg(int64_t n, int nseg, const int64_t* __restrict__ off, double* __restrict__ v) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i - __ldg(off + find_seg(off, nseg, i));
    uint32_t h = (uint32_t)((uint64_t)(j + 1) * 2654435761ull);
    v[i] = (double)h / 4294967296.0 - 0.5;
  }
}

// ------------------------------------------------------------------------------------------
// coarsest level: one dense matrix per segment (problem); moff = offset of its matrix
__global__ void k_bsr_to_dense_seg(int64_t nb, int np, int nseg, const int64_t* __restrict__ sblk,
                                   const int64_t* __restrict__ moff, const int64_t* __restrict__ rp,
                                   const int32_t* __restrict__ col, const double* __restrict__ val,
                                   double* __restrict__ A) {
  pdl_entry();
  const int64_t i = blockIdx.x;
  if (i >= nb) return;
  const int s = find_seg(sblk, nseg, i);
  const int64_t b0 = sblk[s], n = (sblk[s + 1] - b0) * np, il = i - b0;
  const int np2 = np * np;
  double* As = A + moff[s];
  for (int64_t z = rp[i]; z < rp[i + 1]; ++z) {
    const int64_t cl = (int64_t)col[z] - b0;  // block-diagonal: columns stay inside the segment
    for (int e = threadIdx.x; e < np2; e += blockDim.x) {
      int r = e / np, c = e - r * np;
      As[(il * np + r) * n + cl * np + c] = val[z * np2 + e];
    }
  }
}

// right-looking Cholesky of every segment's matrix (one CTA per segment), lower triangle = L
__global__ void __launch_bounds__(1024) k_dense_chol_seg(int nseg, const int64_t* __restrict__ nn,
                                                        const int64_t* __restrict__ moff, double* A, int* err) {
  pdl_entry();
  const int s = blockIdx.x;
  if (s >= nseg) return;
  const int64_t n = nn[s];
  double* M = A + moff[s];
  __shared__ double djj;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int64_t j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double v = M[j * n + j];
      if (!(v > 0.0)) {
        bad = 1;
        v = 1.0;
      }
      djj = sqrt(v);
      M[j * n + j] = djj;
    }
    __syncthreads();
    if (bad) break;
    for (int64_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x) M[i * n + j] /= djj;
    __syncthreads();
    const int64_t m = n - j - 1;
    for (int64_t e = threadIdx.x; e < m * m; e += blockDim.x) {
      int64_t a = j + 1 + e / m, c = j + 1 + e % m;
      if (c <= a) M[a * n + c] -= M[a * n + j] * M[c * n + j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) atomicOr(err, 1);
}

// X_s = L_s^{-1}: column j of segment blockIdx.y (one thread per column)
__global__ void k_tri_inverse_seg(int nseg, const int64_t* __restrict__ nn, const int64_t* __restrict__ moff,
                                  const double* __restrict__ L, double* __restrict__ X) {
  pdl_entry();
  const int s = blockIdx.y;
  if (s >= nseg) return;
  const int64_t n = nn[s], j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double* Ls = L + moff[s];
  double* Xs = X + moff[s];
  for (int64_t i = 0; i < j; ++i) Xs[i * n + j] = 0.0;
  for (int64_t i = j; i < n; ++i) {
    double v = (i == j) ? 1.0 : 0.0;
    for (int64_t p = j; p < i; ++p) v -= Ls[i * n + p] * Xs[p * n + j];
    Xs[i * n + j] = v / Ls[i * n + i];
  }
}

// Minv_s = X_s^T X_s (16x16 tiles, blockIdx.z = segment)
__global__ void k_xtx_seg(int nseg, const int64_t* __restrict__ nn, const int64_t* __restrict__ moff,
                          const double* __restrict__ X, double* __restrict__ Minv) {
  pdl_entry();
  const int s = blockIdx.z;
  if (s >= nseg) return;
  const int64_t n = nn[s];
  if ((int64_t)blockIdx.x * 16 >= n || (int64_t)blockIdx.y * 16 >= n) return;
  const double* Xs = X + moff[s];
  __shared__ double As[16][17], Bs[16][17];
  const int64_t i = (int64_t)blockIdx.y * 16 + threadIdx.y, j = (int64_t)blockIdx.x * 16 + threadIdx.x;
  double acc = 0.0;
  for (int64_t k0 = 0; k0 < n; k0 += 16) {
    int64_t ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    int64_t ia = (int64_t)blockIdx.y * 16 + threadIdx.y;
    As[threadIdx.y][threadIdx.x] = (ka < n && ia < n) ? Xs[ka * n + ia] : 0.0;
    Bs[threadIdx.y][threadIdx.x] = (kb < n && j < n) ? Xs[kb * n + j] : 0.0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) acc = fma(As[threadIdx.y][q], Bs[q][threadIdx.x], acc);
    __syncthreads();
  }
  if (i < n && j < n) Minv[moff[s] + i * n + j] = acc;
}

// z = Minv_s r on every segment (one warp per row, rows row = warp, warp + nw, ...); VT = vector
// type (double or float)
template <class VT, bool COH = false>
__device__ __forceinline__ void gemv_seg_rows(int64_t warp, int64_t nw, int64_t ntot, int nseg,
                                              const int64_t* __restrict__ doff, const int64_t* __restrict__ moff,
                                              const double* __restrict__ Minv, const VT* __restrict__ r,
                                              VT* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  for (int64_t row = warp; row < ntot; row += nw) {
    const int s = find_seg(doff, nseg, row);
    const int64_t d0 = __ldg(doff + s), n = __ldg(doff + s + 1) - d0;
    const double* A = Minv + __ldg(moff + s) + (row - d0) * n;
    double acc = 0.0;
    for (int64_t c = lane; c < n; c += 32) {
      VT rv;
      if constexpr (COH) rv = __ldcg(r + d0 + c);
      else rv = r[d0 + c];
      acc = fma(__ldg(A + c), (double)rv, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[row] = (VT)acc;
  }
}

template <class VT>
__global__ void __launch_bounds__(kThreads) k_gemv_seg(int64_t ntot, int nseg, const int64_t* __restrict__ doff,
                                                      const int64_t* __restrict__ moff,
                                                      const double* __restrict__ Minv, const VT* __restrict__ r,
                                                      VT* __restrict__ z) {
  pdl_entry();
  gemv_seg_rows<VT>(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, ((int64_t)gridDim.x * blockDim.x) >> 5,
                    ntot, nseg, doff, moff, Minv, r, z);
}

// ------------------------------------------------------------------------------------------
// Batched conjugate gradients: every problem (segment) runs its own CG / flexible CG; level-1
// vectors are cut into chunks that never straddle two problems (cb: chunk boundaries, cseg:
// problem of every chunk, cfirst: first chunk of every problem), so that every per-problem
// inner product is a fixed-order sum of per-chunk partial sums (deterministic).

// solve controls read by the graph at run time (one device copy, written before each launch)
struct BatchCtl {
  const double* b;  // right-hand sides of all problems, concatenated in input order
  double* x;        // initial guesses in, solutions out (same layout)
  double tol2;      // squared relative tolerance
  int maxit;        // iteration limit
  int pad;
};

struct BatchScal {
  double *rz, *rr, *bb, *pq, *zq, *alpha, *beta;
  int *active, *bad, *iters;
  int* it;  // loop iterations executed (all problems)
};

// s_b[i], s_x[i] <- b, x of the problem's entry i - sdof[s] (ioff[s] = problem offset in b, x)
__global__ void k_batch_gather(int64_t n, int nseg, const int64_t* __restrict__ sdof,
                               const int64_t* __restrict__ ioff, const BatchCtl* __restrict__ ctl,
                               double* __restrict__ sb, double* __restrict__ sx) {
  pdl_entry();
  const double* b = ctl->b;
  const double* x = ctl->x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int s = find_seg(sdof, nseg, i);
    const int64_t j = __ldg(ioff + s) + (i - __ldg(sdof + s));
    sb[i] = b[j];
    sx[i] = x[j];
  }
}
__global__ void k_batch_scatter(int64_t n, int nseg, const int64_t* __restrict__ sdof,
                                const int64_t* __restrict__ ioff, const BatchCtl* __restrict__ ctl,
                                const double* __restrict__ sx) {
  pdl_entry();
  double* x = ctl->x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int s = find_seg(sdof, nseg, i);
    x[__ldg(ioff + s) + (i - __ldg(sdof + s))] = sx[i];
  }
}

// part[d * nchunk + c] = sum over chunk c of x_d y_d  (ND = 1 or 2 products)
template <int ND>
__global__ void __launch_bounds__(kThreads) k_chunk_dot(int nchunk, const int64_t* __restrict__ cb,
                                                       const double* __restrict__ x0, const double* __restrict__ y0,
                                                       const double* __restrict__ x1, const double* __restrict__ y1,
                                                       double* __restrict__ part) {
  pdl_entry();
  const int c = blockIdx.x;
  if (c >= nchunk) return;
  double a0 = 0.0, a1 = 0.0;
  for (int64_t i = cb[c] + threadIdx.x; i < cb[c + 1]; i += blockDim.x) {
    a0 = fma(x0[i], y0[i], a0);
    if (ND > 1) a1 = fma(x1[i], y1[i], a1);
  }
  a0 = block_sum(a0);
  if (ND > 1) a1 = block_sum(a1);
  if (threadIdx.x == 0) {
    part[c] = a0;
    if (ND > 1) part[nchunk + c] = a1;
  }
}

__device__ __forceinline__ double chunk_total(const int* __restrict__ cfirst, const double* __restrict__ part, int s) {
  double acc = 0.0;
  for (int c = cfirst[s]; c < cfirst[s + 1]; ++c) acc += part[c];
  return acc;
}

// start of a solve: rr, bb from the chunk sums of (r, r), (b, b); every problem active
__global__ void k_bcg_start(int nseg, int nchunk, const int* __restrict__ cfirst, const double* __restrict__ part,
                            BatchScal S) {
  pdl_entry();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
    S.rr[s] = chunk_total(cfirst, part, s);
    S.bb[s] = chunk_total(cfirst, part + nchunk, s);
    S.active[s] = 1;
    S.bad[s] = 0;
    S.iters[s] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *S.it = 0;
}

// pq = (p, q); alpha = rz / pq for active problems (0 for finished ones); counts the step
__global__ void k_bcg_alpha(int nseg, const int* __restrict__ cfirst, const double* __restrict__ part, BatchScal S) {
  pdl_entry();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
    const double pq = chunk_total(cfirst, part, s);
    S.pq[s] = pq;
    double a = 0.0;
    if (S.active[s]) {
      if (!(pq > 0.0) || !isfinite(pq)) {
        S.bad[s] = 1;
      } else {
        a = S.rz[s] / pq;
        S.iters[s] += 1;
      }
    }
    S.alpha[s] = a;
  }
}

// x += alpha_s p, r -= alpha_s q on chunk c of problem s = cseg[c]; part[c] = (r, r) on it.
// A finished problem (alpha_s = 0) is not touched: its p may hold values the row-masked
// kernels never wrote.
__global__ void __launch_bounds__(kThreads) k_bcg_xr(int nchunk, const int64_t* __restrict__ cb,
                                                    const int* __restrict__ cseg, const double* __restrict__ alpha,
                                                    const double* __restrict__ p, const double* __restrict__ q,
                                                    double* __restrict__ x, double* __restrict__ r,
                                                    double* __restrict__ part) {
  pdl_entry();
  const int c = blockIdx.x;
  if (c >= nchunk) return;
  const double a = alpha[cseg[c]];
  if (a == 0.0) {
    if (threadIdx.x == 0) part[c] = 0.0;
    return;
  }
  double acc = 0.0;
  for (int64_t i = cb[c] + threadIdx.x; i < cb[c + 1]; i += blockDim.x) {
    const double ri = fma(-a, q[i], r[i]);
    x[i] = fma(a, p[i], x[i]);
    r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[c] = acc;
}

// rr from the chunk sums (when part != nullptr); a problem stays active while
// rr > tol^2 bb and no breakdown occurred. One CTA. count != 0: one more loop iteration is
// counted. The loop condition (some problem active and it < maxit) goes to the graph's
// conditional handle when use_cond != 0.
__global__ void __launch_bounds__(1024) k_bcg_check(int nseg, const int* __restrict__ cfirst,
                                                   const double* __restrict__ part, BatchScal S,
                                                   const BatchCtl* __restrict__ ctl, int count,
                                                   cudaGraphConditionalHandle cond, int use_cond) {
  pdl_entry();
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const double t2 = ctl->tol2;
  int mine = 0;
  for (int s = threadIdx.x; s < nseg; s += blockDim.x) {
    double rr = S.rr[s];
    if (part) {
      rr = chunk_total(cfirst, part, s);
      S.rr[s] = rr;
    }
    const int a = S.active[s] && !S.bad[s] && isfinite(rr) && (rr > t2 * S.bb[s]);
    S.active[s] = a;
    if (!isfinite(rr)) S.bad[s] = 1;
    mine += a;
  }
  if (mine) atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    int it = *S.it + (count ? 1 : 0);
    *S.it = it;
    if (use_cond) cudaGraphSetConditional(cond, (cnt > 0 && it < ctl->maxit) ? 1u : 0u);
  }
}

// rz_new = (r, z) (and zq = (z, q) for flexible CG) from the chunk sums; beta:
// CG: rz_new / rz;  flexible CG: -zq / pq;  start != 0: beta = 0 (first direction p = z)
__global__ void k_bcg_beta(int nseg, int nchunk, const int* __restrict__ cfirst, const double* __restrict__ part,
                           int flexible, int start, BatchScal S) {
  pdl_entry();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
    const double rzn = chunk_total(cfirst, part, s);
    double be = 0.0;
    if (!start && S.active[s]) {
      if (flexible) {
        const double zq = chunk_total(cfirst, part + nchunk, s);
        S.zq[s] = zq;
        be = -zq / S.pq[s];
      } else {
        be = rzn / S.rz[s];
      }
      if (!isfinite(be)) {
        S.bad[s] = 1;
        be = 0.0;
      }
    }
    S.beta[s] = be;
    S.rz[s] = rzn;
  }
}

// p = z + beta_s p on chunk c (start != 0: p = z), for running problems only
__global__ void k_bcg_p(int nchunk, const int64_t* __restrict__ cb, const int* __restrict__ cseg,
                        const double* __restrict__ beta, int start, const double* __restrict__ z,
                        double* __restrict__ p, const int* __restrict__ active) {
  pdl_entry();
  const int c = blockIdx.x;
  if (c >= nchunk || !active[cseg[c]]) return;
  const double be = beta[cseg[c]];
  for (int64_t i = cb[c] + threadIdx.x; i < cb[c + 1]; i += blockDim.x) p[i] = start ? z[i] : fma(be, p[i], z[i]);
}

// act[i] = 1 while the problem of level-1 block i is running (sdof: DOF offsets of the problems)
__global__ void k_bcg_rowact(int64_t nb, int np, int nseg, const int64_t* __restrict__ sdof,
                             const int* __restrict__ active, uint8_t* __restrict__ act) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x)
    act[i] = (uint8_t)(active[find_seg(sdof, nseg, i * np)] != 0);
}

// device-side loop of a single-problem solve: one more iteration done; continue while the
// residual is above tolerance, no breakdown occurred and the iteration limit is not reached
struct LoopCtl {
  double tol2, bb;
  int maxit, it;
};
__global__ void k_cg_loop_check(const PcgScal* __restrict__ S, LoopCtl* c, cudaGraphConditionalHandle cond) {
  pdl_entry();
  const int it = c->it + 1;
  c->it = it;
  const double rr = S->rr;
  const bool go = !S->bad && isfinite(rr) && rr > c->tol2 * c->bb && it < c->maxit;
  cudaGraphSetConditional(cond, go ? 1u : 0u);
}

// per-problem results: res[3 g] = iterations, res[3 g + 1] = ||b - M x|| / ||b|| (true residual
// from the chunk sums), res[3 g + 2] = status (0 converged, 4 not converged, 5 breakdown);
// g = gidx[s], the problem's index in the caller's list; res[gslot] = loop iterations
__global__ void k_bcg_result(int nseg, const int* __restrict__ cfirst, const double* __restrict__ part,
                             const int* __restrict__ gidx, BatchScal S, double* __restrict__ res, int gslot) {
  pdl_entry();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
    const double rr = chunk_total(cfirst, part, s);
    const double bb = S.bb[s];
    const int g = gidx[s];
    res[3 * (int64_t)g] = (double)S.iters[s];
    res[3 * (int64_t)g + 1] = sqrt(rr) / (bb > 0.0 ? sqrt(bb) : 1.0);
    res[3 * (int64_t)g + 2] = S.bad[s] ? 5.0 : (S.active[s] ? 4.0 : 0.0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) res[gslot] = (double)*S.it;
}

}  // namespace xdg
