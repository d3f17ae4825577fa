// The small levels of the low-precision cycle in one persistent launch: a V-cycle from a given
// level down to the coarsest direct solve and back (the same steps, in the same order, as the
// launch-per-step cycle: smoothing sweeps, residual-restriction phases 1 and 2, the coarsest
// solve, prolongation), with a grid-wide barrier after every step. Small levels are bound by
// launch and ramp-up latency when every step is a kernel of its own; here the steps are
// separated only by the barrier.
//
// The kernel must run as a cooperative launch (all CTAs resident). Every barrier wait is
// bounded: after kBarrierSpins polls it sets the error word and every later barrier returns at
// once, so a failure ends the kernel in bounded time instead of hanging the GPU.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "xdg_kernels_batch.cuh"
#include "xdg_kernels_lp.cuh"

namespace xdg {

constexpr int kFusedMaxLevels = 24;
constexpr unsigned kBarrierSpins = 1u << 22;  // x 64 ns sleep: about 0.3 s per barrier at most

struct FusedLevel {
  int64_t nb;
  const int64_t* rp;
  const int32_t* col;
  const float* val;   // FP32 operator copy and its block scales
  const float* sc;
  const float* Dinv;  // FP32 block inverses and scales
  const float* dsc;
  float omega;
  int spl;            // split-row mapping of the row steps
  const void* R;      // transfer blocks to the next level (FP32 or BF16) and scales
  const float* rsc;
  const int32_t* agg;
  const int64_t* cptr;  // children of the next level's blocks
  const int32_t* ch;
  float *b, *x, *t, *s;
};

struct FusedCycle {
  int n;   // levels in the fused part, the last one the coarsest
  int nu;  // sweeps before and after the coarse correction
  FusedLevel L[kFusedMaxLevels];
  const double* Minv;  // coarsest level: FP64 inverses of the problems
  const int64_t* doff;
  const int64_t* moff;
  int nseg;
  int64_t nc;
  unsigned* bar;  // barrier counter (zero at launch)
  int* err;       // nonzero: a barrier gave up
  unsigned extra; // 0; 1 makes every barrier wait for one CTA more than the grid has (a test of
                  // the bounded wait: the barriers give up and report, nothing hangs)
};

__device__ __forceinline__ void fused_barrier(unsigned* bar, unsigned& phase, int* err, unsigned extra) {
  __syncthreads();
  ++phase;
  if (threadIdx.x == 0) {
    volatile int* verr = err;
    if (*verr == 0) {
      __threadfence();
      atomicAdd(bar, 1u);
      const unsigned target = phase * (gridDim.x + extra);
      volatile unsigned* vbar = bar;
      unsigned spins = 0;
      while (*vbar < target) {
        if (*verr != 0) break;
        if (++spins > kBarrierSpins) {
          atomicOr(err, 1);
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
  }
  __syncthreads();
}

// The same step separation for a launch that is one thread-block cluster: the hardware cluster
// barrier (arrive with release, wait with acquire semantics at cluster scope) orders the
// steps' global-memory writes before the next step's reads; those reads bypass L1 (.cg) as in
// the grid-wide form. No polling, so nothing to bound.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <bool CLUSTER>
__device__ __forceinline__ void step_barrier(unsigned* bar, unsigned& phase, int* err, unsigned extra) {
  if (CLUSTER) cluster_barrier();
  else fused_barrier(bar, phase, err, extra);
}

template <int NP, bool ZERO>
__device__ __forceinline__ void fused_smooth(const FusedLevel& V, int64_t warp, int64_t nw, const float* xi, float* xo) {
  if (V.spl)
    smooth_lp_rows<NP, float, ZERO, true, true>(warp, nw, V.nb, V.rp, V.col, V.val, V.sc, V.Dinv, V.dsc, V.omega, nullptr,
                                          V.b, xi, xo, nullptr);
  else
    smooth_lp_rows<NP, float, ZERO, false, true>(warp, nw, V.nb, V.rp, V.col, V.val, V.sc, V.Dinv, V.dsc, V.omega, nullptr,
                                           V.b, xi, xo, nullptr);
}

// pre0: the first sweep on the fused part's first level has been done (x holds it).
// CLUSTER: the launch is a single thread-block cluster (its CTAs separated by cluster
// barriers); otherwise a cooperative grid (grid-wide barriers).
template <int NP, class TS, bool CLUSTER>
__global__ void __launch_bounds__(kThreads) k_fused_vcycle(const FusedCycle* __restrict__ F, int pre0) {
  pdl_entry();
  const int64_t warp = grid_warp(), nw = grid_warps();
  const int64_t tid = grid_thread(), nt = grid_threads();
  const int n = F->n, nu = F->nu;
  unsigned* bar = F->bar;
  int* err = F->err;
  unsigned phase = 0;
  float* cur[kFusedMaxLevels];
  // down: pre-smoothing, residual-restriction
  for (int l = 0; l + 1 < n; ++l) {
    const FusedLevel& V = F->L[l];
    const FusedLevel& C = F->L[l + 1];
    float* c = V.x;
    float* o = V.t;
    if (l == 0 && !pre0) {
      fused_smooth<NP, true>(V, warp, nw, nullptr, c);
      step_barrier<CLUSTER>(bar, phase, err, F->extra);
    }
    for (int s = 1; s < nu; ++s) {
      fused_smooth<NP, false>(V, warp, nw, c, o);
      step_barrier<CLUSTER>(bar, phase, err, F->extra);
      float* tmp = c;
      c = o;
      o = tmp;
    }
    cur[l] = c;
    if (V.spl)
      resid_rt_lp_rows<NP, float, TS, true, true, true>(warp, nw, V.nb, V.rp, V.col, V.val, V.sc, (const TS*)V.R, V.rsc,
                                                  V.b, c, V.s, nullptr);
    else
      resid_rt_lp_rows<NP, float, TS, true, false, true>(warp, nw, V.nb, V.rp, V.col, V.val, V.sc, (const TS*)V.R, V.rsc,
                                                   V.b, c, V.s, nullptr);
    step_barrier<CLUSTER>(bar, phase, err, F->extra);
    if (l + 2 < n) {  // phase 2 and the coarse level's first sweep
      gather_smooth0_lp_rows<NP, true>(warp, nw, C.nb, V.cptr, V.ch, V.s, C.Dinv, C.dsc, C.omega, nullptr, C.b, C.x);
    } else {
      gather_lp_elems<NP, true>(tid, nt, C.nb, V.cptr, V.ch, V.s, C.b);
    }
    step_barrier<CLUSTER>(bar, phase, err, F->extra);
  }
  // coarsest direct solve (FP64 inverse)
  {
    const FusedLevel& C = F->L[n - 1];
    gemv_seg_rows<float, true>(warp, nw, F->nc, F->nseg, F->doff, F->moff, F->Minv, C.b, C.x);
    step_barrier<CLUSTER>(bar, phase, err, F->extra);
  }
  // up: prolongation, post-smoothing
  for (int l = n - 2; l >= 0; --l) {
    const FusedLevel& V = F->L[l];
    const FusedLevel& C = F->L[l + 1];
    float* x = V.x;
    float* after = (nu % 2 == 0) ? x : V.t;
    float* c = cur[l];
    prolong_lp_rows<NP, TS, true>(warp, nw, V.nb, V.agg, (const TS*)V.R, V.rsc, C.x, c, after, nullptr);
    step_barrier<CLUSTER>(bar, phase, err, F->extra);
    c = after;
    float* o = (c == x) ? V.t : x;
    for (int s = 0; s < nu; ++s) {
      fused_smooth<NP, false>(V, warp, nw, c, o);
      step_barrier<CLUSTER>(bar, phase, err, F->extra);
      float* tmp = c;
      c = o;
      o = tmp;
    }
    if (c != x) {
      for (int64_t e = tid; e < V.nb * NP; e += nt) x[e] = __ldcg(c + e);
      step_barrier<CLUSTER>(bar, phase, err, F->extra);
    }
  }
}

}  // namespace xdg
