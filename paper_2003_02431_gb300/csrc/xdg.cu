// libxdg: C ABI (include/xdg.h) of the multigrid-preconditioned XDG solve on one GPU.
//
// Kummer, Smuda, Weber, "BoSSS: a package for multigrid extended discontinuous Galerkin
// methods", arXiv 2003.02431: system in block form (Eq. GenericMatrixSystem), transfers
// (Eq. XDGrestrictionMatrix), Galerkin coarse operators (Eq. XDGsysRestriction), level
// recursion (Algorithm 4 without residual minimisation), block smoothing with cell-local dense
// solves (Algorithms 1-2), direct coarsest solve and Krylov outer method (sec. 3.3).
//
// Host code here validates inputs, owns device memory, computes sparsity patterns, records
// CUDA graphs and drives the iterations; every arithmetic step of the solve runs in the
// kernels of xdg_kernels.cuh.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/xdg.h"
#include "xdg_kernels.cuh"
#include "xdg_kernels_lp.cuh"
#include "xdg_kernels_batch.cuh"
#include "xdg_kernels_mlp.cuh"
#include "xdg_kernels_fused.cuh"
#include "xdg_kernels_df.cuh"
#include "xdg_swz.h"
#include "xdg_krylov.h"
#include "xdg_big.h"

using namespace xdg;

namespace {

thread_local std::string g_last_error;

void set_err(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      set_err("%s:%d: %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));      \
      return e_ == cudaErrorMemoryAllocation ? XDG_ENOMEM : XDG_ECUDA;                  \
    }                                                                                   \
  } while (0)

#define CKL()  CK(cudaGetLastError())

// in void helpers that only enqueue work: the error surfaces at the next cudaGetLastError
#define CK_VOID(call) (void)(call)

#define TRY(expr)          \
  do {                     \
    int rc_ = (expr);      \
    if (rc_) return rc_;   \
  } while (0)

using clk = std::chrono::steady_clock;
double ms_since(clk::time_point t0) {
  return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
}


// partial sums a reduction may produce (grids of the fused apply-and-dot are capped at this)
constexpr int kPartials = 4096;

// One full wave: the grid-stride kernels get at most (resident CTAs per SM) x SMs CTAs, so that
// no partial second wave of CTAs runs at the end of a launch (occupancy queried once per kernel
// and device: the cap is kept per (kernel, device ordinal), so GPUs of different models in one
// process each get their own).
int wave_cap(const void* k) {
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
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kThreads, 0) != cudaSuccess || occ < 1) occ = 1;
  const int cap = occ * sms;
  cache.push_back(Entry{k, dev, cap});
  return cap;
}
inline int fit_grid(const void* k, int grid) { return std::max(1, std::min(grid, wave_cap(k))); }

// Kernel launches: kl(kernel, grid, block, shared bytes, stream)(arguments). Each launch carries
// the programmatic-stream-serialization attribute (every kernel begins with griddepcontrol.wait,
// see pdl_entry), so that inside captured graphs a kernel's CTAs are dispatched while its
// predecessor drains. XDG_PDL=0 in the environment launches without it (plain serialization).
inline bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("XDG_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}
template <class... P>
struct KLaunch {
  void (*k)(P...);
  dim3 g, b;
  size_t sm;
  cudaStream_t s;
  template <class... A>
  void operator()(A&&... a) const {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, std::forward<A>(a)...);  // errors surface through cudaGetLastError
  }
};
template <class... P>
inline KLaunch<P...> kl(void (*k)(P...), dim3 g, dim3 b, size_t sm, cudaStream_t s) {
  return KLaunch<P...>{k, g, b, sm, s};
}
#define LFIT(G, S, ...) kl(__VA_ARGS__, fit_grid((const void*)&__VA_ARGS__, G), kThreads, 0, S)

// --------------------------------------------------------------------------------------------
// per-Np kernel table
struct Ops {
  int np;
  void (*spmv)(int grid, cudaStream_t, const uint8_t*, int64_t, const int64_t*, const int32_t*, const double*,
               const double*, const double*, double*, int mode);
  void (*smooth)(int grid, cudaStream_t, int64_t, const int64_t*, const int32_t*, const double*,
                 const double*, double, const double*, const double*, const double*, double*);
  void (*bjsolve)(int grid, cudaStream_t, int64_t, const double*, const double*, double*);
  void (*diagmul)(int grid, cudaStream_t, int64_t, const int64_t*, const double*, const double*, double*);
  void (*resid_rt)(int grid, cudaStream_t, int64_t, const int64_t*, const int32_t*, const double*,
                   const double*, const double*, const double*, double*);
  void (*gather)(int grid, cudaStream_t, int64_t, const int64_t*, const int32_t*, const double*, double*);
  void (*gather_smooth0)(int grid, cudaStream_t, int64_t, const int64_t*, const int32_t*, const double*,
                         const double*, double, const double*, double*, double*);
  void (*prolong)(int grid, cudaStream_t, int64_t, const int32_t*, const double*, const double*,
                  const double*, double*);
  void (*galerkin)(int grid, cudaStream_t, int64_t, const int64_t*, const int32_t*, const int64_t*,
                   const int32_t*, const double*, const int32_t*, const double*, const int64_t*,
                   const int32_t*, double*);
  void (*diag_inv)(cudaStream_t, int64_t, const int64_t*, const double*, double*, int*);
  int (*spmv_dot)(int grid, cudaStream_t, int64_t, const int64_t*, const int32_t*, const double*, const double*,
                  double*, double*);
  // FP32-pair (double-float) product and the direction update writing the pair copy
  int (*spmv_dot_df)(int grid, cudaStream_t, int64_t, const int64_t*, const int32_t*, const float2*, const int*,
                     const float2*, const int*, const double*, double*, double*, const uint8_t*);
  void (*pcg_p_df)(int grid, cudaStream_t, int64_t, const PcgScal*, int, const double*, double*, float2*, int*);
  void (*split_df)(int grid, cudaStream_t, int64_t, const double*, float2*, int*);
  int (*spmv_dot_df_sym)(int grid, cudaStream_t, int64_t, const int64_t*, const int32_t*, const float2*, const int*,
                         SymL, const float2*, const int*, const double*, double*, double*, const uint8_t*);
  int gpw;
};

template <int NP>
struct OpsT {
  static void spmv(int grid, cudaStream_t s, const uint8_t* act, int64_t nb, const int64_t* rp, const int32_t* col,
                   const double* val, const double* x, const double* b, double* y, int mode) {
    if (mode) LFIT(grid, s, k_spmv<NP, 1>)(nb, rp, col, val, x, b, y, act);
    else LFIT(grid, s, k_spmv<NP, 0>)(nb, rp, col, val, x, b, y, act);
  }
  static void smooth(int grid, cudaStream_t s, int64_t nb, const int64_t* rp, const int32_t* col,
                     const double* val, const double* Dinv, double om, const double* omr, const double* b,
                     const double* xi, double* xo) {
    if (xi) LFIT(grid, s, k_smooth<NP, false>)(nb, rp, col, val, Dinv, om, omr, b, xi, xo);
    else LFIT(grid, s, k_smooth<NP, true>)(nb, rp, col, val, Dinv, om, omr, b, xi, xo);
  }
  static void bjsolve(int grid, cudaStream_t s, int64_t nb, const double* Dinv, const double* v, double* z) {
    LFIT(grid, s, k_bjsolve<NP>)(nb, Dinv, v, z);
  }
  static void diagmul(int grid, cudaStream_t s, int64_t nb, const int64_t* dg, const double* val,
                      const double* v, double* w) {
    LFIT(grid, s, k_diagmul<NP>)(nb, dg, val, v, w);
  }
  static void resid_rt(int grid, cudaStream_t s, int64_t nbf, const int64_t* rp, const int32_t* col,
                       const double* val, const double* R, const double* b, const double* x, double* t) {
    if (x) LFIT(grid, s, k_resid_rt<NP, true>)(nbf, rp, col, val, R, b, x, t);
    else LFIT(grid, s, k_resid_rt<NP, false>)(nbf, rp, col, val, R, b, x, t);
  }
  static void gather(int grid, cudaStream_t s, int64_t nbc, const int64_t* cptr, const int32_t* ch,
                     const double* t, double* rc) {
    LFIT(grid, s, k_gather<NP>)(nbc, cptr, ch, t, rc);
  }
  static void gather_smooth0(int grid, cudaStream_t s, int64_t nbc, const int64_t* cptr, const int32_t* ch,
                             const double* t, const double* Dinv, double om, const double* omr, double* bc,
                             double* xc) {
    LFIT(grid, s, k_gather_smooth0<NP>)(nbc, cptr, ch, t, Dinv, om, omr, bc, xc);
  }
  static void prolong(int grid, cudaStream_t s, int64_t nbf, const int32_t* agg, const double* R,
                      const double* zc, const double* xi, double* xo) {
    LFIT(grid, s, k_prolong<NP>)(nbf, agg, R, zc, xi, xo);
  }
  static void galerkin(int grid, cudaStream_t s, int64_t nbc, const int64_t* cptr, const int32_t* ch,
                       const int64_t* rp, const int32_t* col, const double* val, const int32_t* agg,
                       const double* R, const int64_t* crp, const int32_t* ccol, double* cval) {
    LFIT(grid, s, k_galerkin<NP>)(nbc, cptr, ch, rp, col, val, agg, R, crp, ccol, cval);
  }
  static void diag_inv(cudaStream_t s, int64_t nb, const int64_t* dg, const double* val, double* Dinv,
                       int* err) {
    kl(k_diag_inv<NP>, (unsigned)((nb + 63) / 64), 64, 0, s)(nb, dg, val, Dinv, err);
  }
  // returns the grid used (= the number of partial sums written)
  static int spmv_dot(int grid, cudaStream_t s, int64_t nb, const int64_t* rp, const int32_t* col,
                      const double* val, const double* x, double* y, double* partial) {
    const int g = std::min(fit_grid((const void*)&k_spmv_dot<NP>, grid), kPartials);
    kl(k_spmv_dot<NP>, g, kThreads, 0, s)(nb, rp, col, val, x, y, partial);
    return g;
  }
  static int spmv_dot_df(int grid, cudaStream_t s, int64_t nb, const int64_t* rp, const int32_t* col,
                         const float2* v2, const int* ea, const float2* x2, const int* ex, const double* x, double* y,
                         double* partial, const uint8_t* act) {
    const int g = std::min(fit_grid((const void*)&k_spmv_dot_df<NP>, grid), kPartials);
    kl(k_spmv_dot_df<NP>, g, kThreads, 0, s)(nb, rp, col, v2, ea, x2, ex, x, y, partial, act);
    return g;
  }
  static void pcg_p_df(int grid, cudaStream_t s, int64_t nb, const PcgScal* S, int first, const double* z, double* p,
                       float2* p2, int* ex) {
    LFIT(grid, s, k_pcg_p_df<NP>)(nb, S, first, z, p, p2, ex);
  }
  static void split_df(int grid, cudaStream_t s, int64_t nb, const double* x, float2* x2, int* ex) {
    LFIT(grid, s, k_split_df<NP>)(nb, x, x2, ex);
  }
  static int spmv_dot_df_sym(int grid, cudaStream_t s, int64_t nb, const int64_t* urp, const int32_t* ucol,
                             const float2* uv2, const int* uea, SymL Ls, const float2* x2, const int* ex,
                             const double* x, double* y, double* partial, const uint8_t* act) {
    const int g = std::min(fit_grid((const void*)&k_spmv_dot_df_sym<NP>, grid), kPartials);
    kl(k_spmv_dot_df_sym<NP>, g, kThreads, 0, s)(nb, urp, ucol, uv2, uea, Ls, x2, ex, x, y, partial, act);
    return g;
  }
  static Ops make() {
    return Ops{NP, spmv, smooth, bjsolve, diagmul, resid_rt, gather, gather_smooth0, prolong, galerkin, diag_inv,
               spmv_dot, spmv_dot_df, pcg_p_df, split_df, spmv_dot_df_sym, Grp<NP>::GPW};
  }
};

static_assert(kPartials == big::kMaxPartials, "partial-sum buffers of the apply-and-dot kernels");

// Np = 35 and 56 (the k = 4 and 5 spaces in 3D): the warp-per-row kernels of xdg_big.cu, FP64
// only (no low-precision cycle, no pair or symmetric storage)
bool ops_big(int np, Ops* o) {
  big::Table t;
  if (!big::table_for(np, &t)) return false;
  *o = Ops{};
  o->np = np;
  o->spmv = t.spmv;
  o->smooth = t.smooth;
  o->bjsolve = t.bjsolve;
  o->diagmul = t.diagmul;
  o->resid_rt = t.resid_rt;
  o->gather = t.gather;
  o->gather_smooth0 = t.gather_smooth0;
  o->prolong = t.prolong;
  o->galerkin = t.galerkin;
  o->diag_inv = t.diag_inv;
  o->spmv_dot = t.spmv_dot;
  o->gpw = 1;
  return true;
}

// Np = 3 and 4 (the k = 1 spaces in 2D and 3D) exist for the low-order systems of the
// p-multigrid; they have FP64 kernels only
bool ops_for(int np, Ops* o) {
  switch (np) {
    case 35:
    case 56: return ops_big(np, o);
    case 3: *o = OpsT<3>::make(); return true;
    case 4: *o = OpsT<4>::make(); return true;
    case 6: *o = OpsT<6>::make(); return true;
    case 10: *o = OpsT<10>::make(); return true;
    case 15: *o = OpsT<15>::make(); return true;
    case 20: *o = OpsT<20>::make(); return true;
    default: return false;
  }
}

// per-(Np, storage type) kernel table of the low-precision cycle (vectors in FP32)
struct OpsLP {
  void (*make)(cudaStream_t, int64_t nblk, int np2, const double*, void*, float*);
  void (*spmv_f)(int, bool, cudaStream_t, int64_t, const int64_t*, const int32_t*, const void*, const float*,
                 const float*, const float*, float*, int mode);
  void (*spmv_d)(int, cudaStream_t, int64_t, const int64_t*, const int32_t*, const void*, const float*,
                 const double*, double*);
  void (*smooth)(int, bool, cudaStream_t, int64_t, const int64_t*, const int32_t*, const void*, const float*,
                 const void*, const float*, float, const float*, const float*, const float*, float*,
                 const uint8_t*);
  void (*resid_rt)(int, bool, cudaStream_t, int64_t, const int64_t*, const int32_t*, const void*, const float*,
                   const void*, const float*, const float*, const float*, float*, const uint8_t*);
  void (*gather)(int, cudaStream_t, int64_t, const int64_t*, const int32_t*, const float*, float*);
  void (*prolong)(int, cudaStream_t, int64_t, const int32_t*, const void*, const float*, const float*,
                  const float*, float*, const uint8_t*);
  void (*resid32)(int, bool, cudaStream_t, int64_t, const int64_t*, const int32_t*, const void*, const float*,
                  const float*, const float*, float*);
  void (*gather_smooth0)(int, cudaStream_t, int64_t, const int64_t*, const int32_t*, const float*, const float*,
                         const float*, float, const float*, float*, float*);
  cudaError_t (*fused)(cudaStream_t, int grid, const FusedCycle*, int pre0);
  int (*fused_occupancy)();
  cudaError_t (*fused_cluster)(cudaStream_t, int csize, const FusedCycle*, int pre0);
  bool (*fused_cluster_ok)(int csize);
  // level 1 on the symmetric storage (sweep from a nonzero guess; residual-restriction)
  void (*smooth_sym)(int, cudaStream_t, int64_t, const int64_t*, const int32_t*, const float*, const float*, SymL,
                     const float*, const float*, float, const float*, const float*, const float*, float*,
                     const uint8_t*);
  void (*resid_rt_sym)(int, cudaStream_t, int64_t, const int64_t*, const int32_t*, const float*, const float*, SymL,
                       const void*, const float*, const float*, const float*, float*, const uint8_t*);
  size_t elem;
};

template <int NP, class TS>
struct OpsLPT {
  static void make(cudaStream_t s, int64_t nblk, int np2, const double* src, void* dst, float* sc) {
    kl(k_make_lp<TS>, (unsigned)((nblk * 32 + 255) / 256), 256, 0, s)(nblk, np2, src, (TS*)dst, sc);
  }
  // spl: one block row per warp, the warp's groups splitting the row (small levels)
  static void spmv_f(int grid, bool spl, cudaStream_t s, int64_t nb, const int64_t* rp, const int32_t* col,
                     const void* val, const float* sc, const float* x, const float* b, float* y, int mode) {
    const TS* v = (const TS*)val;
    if (spl) {
      if (mode) LFIT(grid, s, k_spmv_lp<NP, TS, float, 1, true>)(nb, rp, col, v, sc, x, b, y);
      else LFIT(grid, s, k_spmv_lp<NP, TS, float, 0, true>)(nb, rp, col, v, sc, x, b, y);
    } else {
      if (mode) LFIT(grid, s, k_spmv_lp<NP, TS, float, 1>)(nb, rp, col, v, sc, x, b, y);
      else LFIT(grid, s, k_spmv_lp<NP, TS, float, 0>)(nb, rp, col, v, sc, x, b, y);
    }
  }
  static void spmv_d(int grid, cudaStream_t s, int64_t nb, const int64_t* rp, const int32_t* col,
                     const void* val, const float* sc, const double* x, double* y) {
    LFIT(grid, s, k_spmv_lp<NP, TS, double, 0>)(nb, rp, col, (const TS*)val, sc, x, nullptr, y);
  }
  // val: the FP32 operator copy (a BF16 operator is not usable in the sweeps, see k_resid_rt_lp)
  static void smooth(int grid, bool spl, cudaStream_t s, int64_t nb, const int64_t* rp, const int32_t* col,
                     const void* val, const float* sc, const void* Dinv, const float* dsc, float om,
                     const float* omr, const float* b, const float* xi, float* xo, const uint8_t* act) {
    const float* v = (const float*)val;
    const float* D = (const float*)Dinv;
    if (xi && spl)
      LFIT(grid, s, k_smooth_lp<NP, float, false, true>)(nb, rp, col, v, sc, D, dsc, om, omr, b, xi, xo, act);
    else if (xi)
      LFIT(grid, s, k_smooth_lp<NP, float, false>)(nb, rp, col, v, sc, D, dsc, om, omr, b, xi, xo, act);
    else
      LFIT(grid, s, k_smooth_lp<NP, float, true>)(nb, rp, col, v, sc, D, dsc, om, omr, b, xi, xo, act);
  }
  // val: the FP32 operator copy
  static void resid_rt(int grid, bool spl, cudaStream_t s, int64_t nbf, const int64_t* rp, const int32_t* col,
                       const void* val, const float* sc, const void* R, const float* rsc, const float* b,
                       const float* x, float* t, const uint8_t* act) {
    const float* v = (const float*)val;
    const TS* Rt = (const TS*)R;
    if (x && spl)
      LFIT(grid, s, k_resid_rt_lp<NP, float, TS, true, true>)(nbf, rp, col, v, sc, Rt, rsc, b, x, t, act);
    else if (x)
      LFIT(grid, s, k_resid_rt_lp<NP, float, TS, true>)(nbf, rp, col, v, sc, Rt, rsc, b, x, t, act);
    else
      LFIT(grid, s, k_resid_rt_lp<NP, float, TS, false>)(nbf, rp, col, v, sc, Rt, rsc, b, x, t, act);
  }
  // W-cycle coarse residual b - M x with the FP32 operator copy
  static void resid32(int grid, bool spl, cudaStream_t s, int64_t nb, const int64_t* rp, const int32_t* col,
                      const void* val, const float* sc, const float* x, const float* b, float* y) {
    const float* v = (const float*)val;
    if (spl) LFIT(grid, s, k_spmv_lp<NP, float, float, 1, true>)(nb, rp, col, v, sc, x, b, y);
    else LFIT(grid, s, k_spmv_lp<NP, float, float, 1>)(nb, rp, col, v, sc, x, b, y);
  }
  static void gather(int grid, cudaStream_t s, int64_t nbc, const int64_t* cptr, const int32_t* ch,
                     const float* t, float* rc) {
    LFIT(grid, s, k_gather_lp<NP>)(nbc, cptr, ch, t, rc);
  }
  static void prolong(int grid, cudaStream_t s, int64_t nbf, const int32_t* agg, const void* R, const float* rsc,
                      const float* zc, const float* xi, float* xo, const uint8_t* act) {
    LFIT(grid, s, k_prolong_lp<NP, TS>)(nbf, agg, (const TS*)R, rsc, zc, xi, xo, act);
  }
  static void gather_smooth0(int grid, cudaStream_t s, int64_t nbc, const int64_t* cptr, const int32_t* ch,
                             const float* t, const float* Dinv, const float* dsc, float om, const float* omr,
                             float* bc, float* xc) {
    LFIT(grid, s, k_gather_smooth0_lp<NP>)(nbc, cptr, ch, t, Dinv, dsc, om, omr, bc, xc);
  }
  // the V-cycle of the small levels in one cooperative launch (all CTAs resident)
  static cudaError_t fused(cudaStream_t s, int grid, const FusedCycle* F, int pre0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fused_vcycle<NP, TS, false>, F, pre0);
  }
  static int fused_occupancy() {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_vcycle<NP, TS, false>, kThreads, 0) != cudaSuccess)
      occ = 0;
    return occ;
  }
  // the same cycle as one thread-block cluster of csize CTAs (csize <= 16)
  static cudaError_t fused_cluster(cudaStream_t s, int csize, const FusedCycle* F, int pre0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)csize);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fused_vcycle<NP, TS, true>, F, pre0);
  }
  // whether a cluster of csize CTAs of the cluster kernel can be resident
  static bool fused_cluster_ok(int csize) {
    if (csize > 8 &&
        cudaFuncSetAttribute(k_fused_vcycle<NP, TS, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)csize);
    cfg.blockDim = dim3(kThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_fused_vcycle<NP, TS, true>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return n >= 1;
  }
  static void smooth_sym(int grid, cudaStream_t s, int64_t nb, const int64_t* urp, const int32_t* ucol,
                         const float* uval, const float* usc, SymL Ls, const float* Dinv, const float* dsc, float om,
                         const float* omr, const float* b, const float* xi, float* xo, const uint8_t* act) {
    LFIT(grid, s, k_smooth_lp_sym<NP>)(nb, urp, ucol, uval, usc, Ls, Dinv, dsc, om, omr, b, xi, xo, act);
  }
  static void resid_rt_sym(int grid, cudaStream_t s, int64_t nbf, const int64_t* urp, const int32_t* ucol,
                           const float* uval, const float* usc, SymL Ls, const void* R, const float* rsc,
                           const float* b, const float* x, float* t, const uint8_t* act) {
    LFIT(grid, s, k_resid_rt_lp_sym<NP, TS>)(nbf, urp, ucol, uval, usc, Ls, (const TS*)R, rsc, b, x, t, act);
  }
  static OpsLP get() {
    return OpsLP{make, spmv_f, spmv_d, smooth, resid_rt, gather, prolong, resid32, gather_smooth0, fused,
                 fused_occupancy, fused_cluster, fused_cluster_ok, smooth_sym, resid_rt_sym, sizeof(TS)};
  }
};

// prec: XDG_PREC_F32 or XDG_PREC_BF16
bool ops_lp_for(int np, int prec, OpsLP* o) {
  const bool bf = prec == XDG_PREC_BF16;
  switch (np) {
    case 6: *o = bf ? OpsLPT<6, __nv_bfloat16>::get() : OpsLPT<6, float>::get(); return true;
    case 10: *o = bf ? OpsLPT<10, __nv_bfloat16>::get() : OpsLPT<10, float>::get(); return true;
    case 15: *o = bf ? OpsLPT<15, __nv_bfloat16>::get() : OpsLPT<15, float>::get(); return true;
    case 20: *o = bf ? OpsLPT<20, __nv_bfloat16>::get() : OpsLPT<20, float>::get(); return true;
    default: return false;
  }
}

// per-Np kernels of the learned cut-cell correction
struct OpsU {
  void (*factor)(cudaStream_t, int, const int64_t*, const double*, double*, double*, float*, double*, int*);
  void (*resid_rows)(int, cudaStream_t, int64_t, const int32_t*, const int64_t*, const int32_t*, const double*,
                     const double*, const double*, double*);
  void (*samples)(cudaStream_t, int, int, const int32_t*, const float*, const double*, const double*, const double*,
                  float*, float*, float*);
  void (*apply)(cudaStream_t, int, MlpDims, int, const int32_t*, const float*, const double*, const __nv_bfloat16*,
                const double*, const float*, double*, int*, double*);
  void (*gather)(cudaStream_t, int, const int32_t*, const int64_t*, const int32_t*, const double*, double, double*);
};

template <int NP>
struct OpsUT {
  static void factor(cudaStream_t s, int U, const int64_t* z, const double* v, double* Li, double* Hm, float* M,
                     double* Hi, int* e) {
    kl(k_unit_factor<NP>, U, 32, 0, s)(U, z, v, Li, Hm, M, Hi, e);
  }
  // one row per warp (k_resid_rows_split): the grid argument is ignored
  static void resid_rows(int, cudaStream_t s, int64_t nr, const int32_t* rows, const int64_t* rp,
                         const int32_t* col, const double* val, const double* x, const double* b, double* y) {
    const int64_t ctas = (nr + kThreads / 32 - 1) / (kThreads / 32);
    kl(k_resid_rows_split<NP>, fit_grid((const void*)&k_resid_rows_split<NP>, (int)std::min<int64_t>(ctas, 1 << 20)),
       kThreads, 0, s)(nr, rows, rp, col, val, x, b, y);
  }
  static void samples(cudaStream_t s, int U, int ng, const int32_t* pr, const float* geo, const double* r,
                      const double* Li, const double* Hi, float* X, float* R, float* C) {
    kl(k_unit_samples<NP>, (U + 7) / 8, 256, 0, s)(U, ng, pr, geo, r, Li, Hi, X, R, C);
  }
  static void apply(cudaStream_t s, int U, MlpDims d, int ng, const int32_t* pr, const float* geo, const double* r,
                    const __nv_bfloat16* W, const double* Li, const float* Hm, double* dl, int* kp, double* E) {
    // BF16 weights (<= 30.2 KB for n_in <= 64, n_out <= 40), the BF16 activation parts and
    // kUnitsPerCta units x 2 x 65 floats (up to 52.4 KB: above 48 KB the kernel's limit is raised)
    const size_t sm = (size_t)((d.total * 2 + 15) / 16) * 16 + kUnitTriBytes + kUnitActBytes;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_unit_apply<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kl(k_unit_apply<NP>, (U + kUnitsPerCta - 1) / kUnitsPerCta, kUnitWarps * 32, sm, s)(U, d, ng, pr, geo, r, W, Li,
                                                                                         Hm, dl, kp, E);
  }
  static void gather(cudaStream_t s, int nt, const int32_t* tb, const int64_t* tp, const int32_t* tl,
                     const double* dl, double th, double* z) {
    const int64_t n = (int64_t)nt * NP;
    kl(k_unit_gather<NP>, (unsigned)((n + 255) / 256), 256, 0, s)(nt, tb, tp, tl, dl, th, z);
  }
  static OpsU make() { return OpsU{factor, resid_rows, samples, apply, gather}; }
};

bool ops_u_for(int np, OpsU* o) {
  switch (np) {
    case 6: *o = OpsUT<6>::make(); return true;
    case 10: *o = OpsUT<10>::make(); return true;
    case 15: *o = OpsUT<15>::make(); return true;
    case 20: *o = OpsUT<20>::make(); return true;
    default: return false;
  }
}

// low-precision copy of one level
struct LevelLP {
  void* val = nullptr;       // operator in the storage precision (smoothing sweeps, apply)
  float* sc = nullptr;
  void* val32 = nullptr;     // FP32 operator (residuals that are restricted); == val in FP32 mode
  float* sc32 = nullptr;
  void* Dinv = nullptr;
  float* dsc = nullptr;
  void* R = nullptr;
  float* rsc = nullptr;
  float *b = nullptr, *x = nullptr, *t = nullptr, *r = nullptr, *dz = nullptr, *s = nullptr;
};

// --------------------------------------------------------------------------------------------
struct Level {
  int64_t nb = 0, nnzb = 0;
  std::vector<int64_t> h_rp, h_diag;
  std::vector<int32_t> h_col;
  int64_t* rp = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  int64_t* diag = nullptr;
  double* Dinv = nullptr;   // inverses of the diagonal blocks (levels above the coarsest)
  int32_t* agg = nullptr;  // to the next level
  double* R = nullptr;
  int64_t* cptr = nullptr;  // children of the next level's blocks
  int32_t* ch = nullptr;
  double *b = nullptr, *x = nullptr, *t = nullptr, *r = nullptr, *dz = nullptr;
  double* s = nullptr;       // restriction scratch R_f^T res_f (levels above the coarsest)
  double omega = 0.0, lmax = 0.0;
  bool spl = false;          // low-precision row kernels split rows across a warp (autotuned)
  // batches: damping per block row (one value per problem), problem offsets on this level
  double* omr = nullptr;
  float* omr_f = nullptr;
  std::vector<int64_t> hseg;   // block offsets of the problems (nprob + 1)
  int64_t* sdof = nullptr;     // DOF offsets of the problems (device, nprob + 1)
  std::vector<double> lmax_p, omega_p;
};

// learned cut-cell correction attached to a hierarchy (units on level 1)
struct Learned {
  int U = 0, n_geo = 0, nt = 0;
  int32_t* pairs = nullptr;   // [U][2] level-1 blocks (A part, B part)
  float* geom = nullptr;      // [U][n_geo] geometry features
  int64_t* zidx = nullptr;    // [U][4] positions of the blocks (a,a), (a,b), (b,a), (b,b) in val
  double* Linv = nullptr;     // [U][2][Np][Np] inverse Cholesky factors of M_aa, M_bb
  double* Hm = nullptr;       // [U][m][m] unit matrices in block-Jacobi coordinates
  float* Mloc = nullptr;      // [U][m][m] the same in FP32 (training)
  double* Minv = nullptr;     // [U][m][m] their inverses
  int32_t* tblk = nullptr;    // touched blocks (ascending)
  int64_t* tptr = nullptr;    // their (unit, half) lists
  int32_t* tlist = nullptr;
  double *res = nullptr, *delta = nullptr, *E = nullptr;
  int* keep = nullptr;
  __nv_bfloat16* W = nullptr; // BF16 snapshot of the network parameters
  int wcap = 0;
  MlpDims d{};
  double theta = 0.25;
  bool on = false;
  OpsU ops{};
  cudaGraphExec_t g_iter[3] = {nullptr, nullptr, nullptr};
  int64_t nodes[3] = {0, 0, 0};
};

// Additive Schwarz smoother of one level (Algorithm Swz with exact patch solves; kernels in
// xdg_swz.cu). Patches are caller-given block lists; the patch matrices' inverses are stored
// once per distinct matrix (tid[p] names the inverse of patch p).
struct SwzLevel {
  int64_t npatch = 0, nslot = 0, nuniq = 0, inv_entries = 0, nitem = 0;
  int maxdof = 0, stage_n = 0;
  swz::Item* items = nullptr;  // work items: patches grouped by their stored inverse
  int32_t* porder = nullptr;
  bool single = false;  // every block in exactly one patch: the solves write the result directly
  int64_t *pptr = nullptr, *ioff = nullptr, *bsptr = nullptr, *bslot = nullptr;
  int32_t *pblk = nullptr, *tid = nullptr;
  double *Ainv = nullptr, *isq = nullptr, *y = nullptr, *r = nullptr;
  float *Ainv32 = nullptr, *isq32 = nullptr, *y32 = nullptr, *r32 = nullptr;
  std::vector<int64_t> h_pptr;
  std::vector<int32_t> h_pblk;
  std::vector<void*> mem;
  size_t bytes = 0;
  ~SwzLevel() {
    for (void* q : mem) cudaFree(q);
  }
  template <class T>
  int alloc(T** p, size_t n) {
    void* q = nullptr;
    const size_t nbytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, nbytes);
    if (e != cudaSuccess) {
      set_err("cudaMalloc(%zu bytes): %s", nbytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? XDG_ENOMEM : XDG_ECUDA;
    }
    mem.push_back(q);
    bytes += nbytes;
    *p = static_cast<T*>(q);
    return XDG_OK;
  }
};

// One level of the orthonormalisation multigrid (Algorithms ResMinimi and OrthoMG): the search
// space Z, W = M Z (cap columns each), the level's right-hand side, iterate and residuals, and
// device scalars: sc[0] |w|^2, sc[1] |M z|^2, sc[2] alpha, sc[3 ..] Gram-Schmidt coefficients.
struct OmgLevel {
  int cap = 0, l = 0;
  double *W = nullptr, *Z = nullptr, *b = nullptr, *x = nullptr, *r = nullptr, *r0 = nullptr, *x0 = nullptr,
         *z = nullptr, *sc = nullptr, *part = nullptr;
  float *rf = nullptr, *zf = nullptr;  // the residual and the smoother's result in FP32
};

}  // namespace

struct xdg_hier {
  int Np = 0, nlev = 0, nu = 1, gamma = 1, wlev = 1 << 20, dev = 0, sms = 152;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Ops ops{};
  std::vector<Level> L;
  std::vector<std::unique_ptr<SwzLevel>> swz;  // additive Schwarz smoother per level (else block Jacobi)
  double omega_fixed = 0.0;                    // xdg_hier_opts.omega
  int lanczos_m = 12;                          // xdg_hier_opts.lanczos_steps
  bool has_swz(int l) const { return l < (int)swz.size() && swz[l]; }
  double* Minv = nullptr;       // dense inverses of the coarsest level, one per problem
  int64_t nc = 0;               // DOF of the coarsest level (all problems)
  int nprob = 1;                // problems in the hierarchy (a batch when > 1)
  int64_t* cs_doff = nullptr;   // coarsest level: DOF offset of every problem (nprob + 1)
  int64_t* cs_moff = nullptr;   // offset of every problem's inverse in Minv
  BatchScal B{};                // per-problem Krylov scalars (batches)
  double* h_bsc = nullptr;      // pinned host scalars (nprob; setup)
  double* spart = nullptr;      // slice sums of the per-problem setup reductions (nprob * 64)
  // level-1 chunks that never straddle two problems: cb boundaries (nchunk + 1), cseg problem
  // of every chunk, cfirst first chunk of every problem (nprob + 1), cpart 2 partial sums each
  int nchunk = 0;
  int64_t* cb = nullptr;
  int* cseg = nullptr;
  int* cfirst = nullptr;
  double* cpart = nullptr;
  int64_t* ioff = nullptr;      // offset of every problem in the caller's concatenated vectors
  int* gidx = nullptr;          // index of every problem in the caller's list
  Learned lr;                   // learned cut-cell correction (off unless enabled)
  // device-side iteration loops of the solve, by precision and learned correction off/on
  cudaGraphExec_t g_loop[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  int64_t loop_nodes[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  LoopCtl* lctl = nullptr;
  LoopCtl* hlctl = nullptr;
  int record_loop(int prec);
  void drop_loops() {
    for (auto& a : g_loop)
      for (auto& g : a) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
      }
  }
  uint8_t* act1 = nullptr;      // batches: 1 for the level-1 blocks of running problems
  const uint8_t* cur_act = nullptr;  // row mask of the level-1 cycle kernels (while recording a batch)
  cudaStream_t body_stream = nullptr;
  int64_t bnodes_fixed[3] = {0, 0, 0};  // kernel nodes of a recorded batched solve outside
  int64_t bnodes_body[3] = {0, 0, 0};   // its loop, and inside one loop iteration
  double *s_b = nullptr, *s_x = nullptr, *s_r = nullptr, *s_z = nullptr, *s_p = nullptr, *s_q = nullptr;
  // level 1 as scaled FP32 pairs (the outer apply of the mixed-precision solves) and the pair
  // copy of the direction p with its per-block exponents
  float2* val2 = nullptr;
  int* ea2 = nullptr;
  float2* p2 = nullptr;
  int* ex2 = nullptr;
  int pair_mode = 0;      // xdg_hier_opts.outer_apply
  bool pair_on = false;   // the mixed-precision iterations use the pair product
  int build_pair();
  int tune_pair();
  // level 1 in symmetric storage: diagonal and right blocks (compact BSR urp/ucol, umap = their
  // indices in the full storage), left blocks as mirrors (SymL); FP32 and pair values
  struct SymLevel {
    int64_t nu = 0, nl = 0;
    int64_t *urp = nullptr, *umap = nullptr, *lrp = nullptr;
    int32_t *ucol = nullptr, *lcol = nullptr, *lblk = nullptr;
    float* uval = nullptr;
    float* usc = nullptr;
    float2* uval2 = nullptr;
    int* uea = nullptr;
    SymL L() const { return SymL{lrp, lcol, lblk}; }
  } sy;
  int sym_mode = 0;        // xdg_hier_opts.symmetric
  bool sym_tried = false;
  bool sym_built = false;  // the operator of level 1 is exactly symmetric and its storage exists
  bool sym_on = false;     // the low-precision level-1 sweep and restriction read it
  bool sym_pair = false;   // the pair product reads it
  int build_sym();
  int tune_sym(int p);
  bool lvl1_sym(int l) const { return l == 0 && sym_on && !L[0].spl; }
  bool use_pair(int p) const { return pair_on && p != XDG_PREC_F64; }
  double* partial = nullptr;
  double* dsc = nullptr;       // device scalars for setup reductions
  PcgScal* S = nullptr;
  PcgScal* hS = nullptr;       // pinned host mirror
  double* hsc = nullptr;       // pinned host scalars
  cudaGraphExec_t g_cycle = nullptr;
  const double* g_cycle_b = nullptr;
  double* g_cycle_x = nullptr;
  cudaGraphExec_t g_iter = nullptr;
  int64_t iter_nodes = 0;      // kernel nodes in one recorded CG iteration
  int64_t cycle_nodes = 0;     // kernel nodes in the recorded cycle
  int64_t launches = 0;        // kernels launched outside graphs (counted by the helpers)
  // low-precision cycles, indexed by XDG_PREC_F32 (1) and XDG_PREC_BF16 (2)
  bool has_lp[3] = {false, false, false};
  OpsLP opl[3]{};
  std::vector<LevelLP> LP[3];
  cudaGraphExec_t g_iter_lp[3] = {nullptr, nullptr, nullptr};
  int64_t iter_lp_nodes[3] = {0, 0, 0};
  cudaGraphExec_t g_cyc_lp[3] = {nullptr, nullptr, nullptr};
  const double* g_cyc_lp_b[3] = {nullptr, nullptr, nullptr};
  double* g_cyc_lp_x[3] = {nullptr, nullptr, nullptr};
  int64_t cyc_lp_nodes[3] = {0, 0, 0};
  std::vector<void*> allocs;
  size_t bytes = 0;
  double setup_ms[3] = {0, 0, 0};

  ~xdg_hier() {
    if (stream) cudaStreamSynchronize(stream);
    delete pm.lo;
    if (g_cycle) cudaGraphExecDestroy(g_cycle);
    if (g_iter) cudaGraphExecDestroy(g_iter);
    for (int p = 0; p < 3; ++p) {
      if (g_iter_lp[p]) cudaGraphExecDestroy(g_iter_lp[p]);
      if (g_cyc_lp[p]) cudaGraphExecDestroy(g_cyc_lp[p]);
    }
    for (int p = 0; p < 3; ++p)
      if (lr.g_iter[p]) cudaGraphExecDestroy(lr.g_iter[p]);
    drop_loops();
    omg_drop_graphs();
    gm_drop();
    if (hlctl) cudaFreeHost(hlctl);
    for (void* p : allocs) cudaFree(p);
    if (h_bsc) cudaFreeHost(h_bsc);
    if (body_stream) cudaStreamDestroy(body_stream);
    if (hS) cudaFreeHost(hS);
    if (hsc) cudaFreeHost(hsc);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  template <class T>
  int alloc(T** p, size_t n) {
    void* q = nullptr;
    size_t nbytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, nbytes);
    if (e != cudaSuccess) {
      set_err("cudaMalloc(%zu bytes): %s", nbytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? XDG_ENOMEM : XDG_ECUDA;
    }
    allocs.push_back(q);
    bytes += nbytes;
    *p = static_cast<T*>(q);
    return XDG_OK;
  }

  int grid(int64_t rows) const {
    int64_t warps = (rows + ops.gpw - 1) / ops.gpw;
    int64_t blocks = (warps + (kThreads / 32) - 1) / (kThreads / 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sms * 8));
  }
  // grid of the low-precision row kernels of level l (split rows: one row per warp)
  int grid_lp(int l) const {
    const Level& V = L[l];
    if (!V.spl) return grid(V.nb);
    const int64_t blocks = (V.nb + (kThreads / 32) - 1) / (kThreads / 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sms * 16));
  }
  int vgrid(int64_t n) const {
    int64_t blocks = (n + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sms * 8));
  }

  // ---------------------------------------------------------------- building blocks
  void spmv(int l, const double* x, const double* b, double* y, int mode, const uint8_t* act = nullptr) {
    ++launches;
    Level& V = L[l];
    ops.spmv(grid(V.nb), stream, act, V.nb, V.rp, V.col, V.val, x, b, y, mode);
  }
  void smooth(int l, const double* b, const double* xi, double* xo) {
    if (has_swz(l)) {
      swz_smooth(l, b, xi, xo);
      return;
    }
    ++launches;
    Level& V = L[l];
    ops.smooth(grid(V.nb), stream, V.nb, V.rp, V.col, V.val, V.Dinv, V.omega, V.omr, b, xi, xo);
  }
  // Schwarz patch solves z = (om) S r (T = double: FP64 inverses; float: FP32 copies); xi: add
  // to xi (xi == nullptr: from zero)
  template <class T>
  void swz_solve(int l, const T* r, T om, const T* xi, T* xo) {
    SwzLevel& S = *swz[l];
    const T* Ai = std::is_same<T, double>::value ? (const T*)S.Ainv : (const T*)S.Ainv32;
    const T* isq = std::is_same<T, double>::value ? (const T*)S.isq : (const T*)S.isq32;
    if (S.single) {
      swz::apply<T>(Np, stream, sms * 4, xi ? 2 : 1, S.nitem, S.items, S.porder, S.pptr, S.pblk, S.ioff, Ai, isq, r,
                    om, xi, xo, S.maxdof, S.stage_n);
      ++launches;
    } else {
      T* y = std::is_same<T, double>::value ? (T*)S.y : (T*)S.y32;
      swz::apply<T>(Np, stream, sms * 4, 0, S.nitem, S.items, S.porder, S.pptr, S.pblk, S.ioff, Ai, isq, r, T(1),
                    nullptr, y, S.maxdof, S.stage_n);
      swz::accum<T>(Np, stream, sms * 8, L[l].nb, S.bsptr, S.bslot, isq, y, om, xi, xo);
      launches += 2;
    }
  }
  // xo = xi + omega S (b - M xi) with the level's Schwarz preconditioner (xi == nullptr: zero)
  void swz_smooth(int l, const double* b, const double* xi, double* xo) {
    Level& V = L[l];
    const double* r = b;
    if (xi) {
      ops.spmv(grid(V.nb), stream, nullptr, V.nb, V.rp, V.col, V.val, xi, b, swz[l]->r, 1);
      ++launches;
      r = swz[l]->r;
    }
    swz_solve<double>(l, r, V.omega, xi, xo);
  }
  void swz_smooth_lp(int p, int l, const float* b, const float* xi, float* xo) {
    Level& V = L[l];
    LevelLP& W = LP[p][l];
    const float* r = b;
    if (xi) {
      opl[p].resid32(grid_lp(l), V.spl, stream, V.nb, V.rp, V.col, W.val32, W.sc32, xi, b, swz[l]->r32);
      ++launches;
      r = swz[l]->r32;
    }
    swz_solve<float>(l, r, (float)V.omega, xi, xo);
  }
  int set_schwarz(int l, int64_t npatch, const int64_t* pptr, const int32_t* pblk);
  // orthonormalisation multigrid (xdg_solve_orthomg)
  std::vector<OmgLevel> omg;
  int omg_restart = 0, omg_passes = 0;
  std::vector<cudaGraphExec_t> omg_graphs;  // one recorded pass per start column of level 1
  int omg_grid() const { return std::min(kRedBlocks, sms * 2); }
  int omg_setup(int restart, int passes);
  void omg_drop_graphs() {
    for (auto& g : omg_graphs)
      if (g) cudaGraphExecDestroy(g);
    omg_graphs.clear();
  }
  // undamped smoother of Algorithm OrthoMG: z = S r (Schwarz) or D^{-1} r (block Jacobi), in
  // FP64 or (omg_f32) from the FP32 copies of the patch or block inverses, r rounded to FP32
  // and the result widened
  bool omg_f32 = false;
  void omg_smooth(int l, const double* r, double* z) {
    Level& V = L[l];
    OmgLevel& S = omg[l];
    const int64_t n = V.nb * Np;
    if (omg_f32) {
      kl(k_d2f, vgrid(n), kThreads, 0, stream)(n, r, S.rf, nullptr, Np);
      if (has_swz(l)) {
        swz_solve<float>(l, S.rf, 1.0f, nullptr, S.zf);
      } else {
        LevelLP& W = LP[1][l];
        opl[1].smooth(grid_lp(l), V.spl, stream, V.nb, V.rp, V.col, W.val32, W.sc32, W.Dinv, W.dsc, 1.0f, nullptr,
                      S.rf, nullptr, S.zf, nullptr);
        ++launches;
      }
      kl(k_f2d, vgrid(n), kThreads, 0, stream)(n, S.zf, z, nullptr, Np);
      launches += 2;
    } else if (has_swz(l)) {
      swz_solve<double>(l, r, 1.0, nullptr, z);
    } else {
      ops.bjsolve(grid(V.nb), stream, V.nb, V.Dinv, r, z);
      ++launches;
    }
  }
  // Algorithm ResMinimi: append z (orthogonalised, normalised) and w = M z to the level's space
  // and move x, r to the residual-minimising combination; two classical Gram-Schmidt sweeps
  void omg_rm(int l, double* x, double* r) {
    OmgLevel& S = omg[l];
    Level& V = L[l];
    const int64_t n = V.nb * Np;
    const int vg = vgrid(n);
    double* w = S.W + (int64_t)S.l * n;
    double* znew = S.Z + (int64_t)S.l * n;
    spmv(l, S.z, nullptr, w, 0);
    dot(n, w, w, S.sc + 1);
    for (int pass = 0; pass < 2 && S.l > 0; ++pass) {
      kry::mdot_partial(stream, omg_grid(), n, S.l, S.W, w, S.part);
      kry::mdot_final(stream, omg_grid(), S.l, S.part, S.sc + 3, nullptr);
      kry::gs_update(stream, vg, n, S.l, S.W, S.Z, S.sc + 3, w, S.z);
      launches += 3;
    }
    dot(n, w, w, S.sc);
    kry::normalize(stream, vg, n, S.sc, S.sc + 1, w, S.z, znew, nullptr);
    dot(n, w, S.r0, S.sc + 2);
    kry::rm_update(stream, vg, n, S.sc + 2, znew, w, x, r);
    launches += 2;
    ++S.l;
  }
  // one pass of Algorithm OrthoMG on level l with the level's x, r (x0 = 0 on coarse levels)
  void omg_pass(int l, double* x, double* r) {
    OmgLevel& S = omg[l];
    Level& V = L[l];
    const int64_t n = V.nb * Np;
    omg_smooth(l, r, S.z);
    omg_rm(l, x, r);
    restrict_(l, r, nullptr, omg[l + 1].b);
    omg_level(l + 1);
    CK_VOID(cudaMemsetAsync(S.z, 0, n * sizeof(double), stream));
    prolong(l, omg[l + 1].x, S.z, S.z);
    omg_rm(l, x, r);
    omg_smooth(l, r, S.z);
    omg_rm(l, x, r);
  }
  // Algorithm OrthoMG on a coarse level: x = MG(0, b) with omg_passes passes (the coarsest:
  // the direct solve)
  void omg_level(int l) {
    OmgLevel& S = omg[l];
    if (l == nlev - 1) {
      coarse(S.b, S.x);
      return;
    }
    const int64_t n = L[l].nb * Np;
    S.l = 0;
    CK_VOID(cudaMemcpyAsync(S.r0, S.b, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    CK_VOID(cudaMemcpyAsync(S.r, S.b, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    CK_VOID(cudaMemsetAsync(S.x, 0, n * sizeof(double), stream));
    for (int p = 0; p < omg_passes; ++p) omg_pass(l, S.x, S.r);
  }
  int solve_orthomg(const double* b, double* x, const xdg_orthomg_opts* o, xdg_solve_info* info);
  // flexible GMRES (xdg_solve_gmres): Arnoldi basis V (m+1 vectors), preconditioned Z (m), the
  // Hessenberg matrix and Givens rotations on the device, one recorded graph per Arnoldi step
  struct Gmres {
    int m = 0, prec = -1, kind = -1;
    double *V = nullptr, *Z = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *ny = nullptr,
           *sc = nullptr, *part = nullptr;
    std::vector<cudaGraphExec_t> step;
    int64_t step_nodes = 0;
  } gm;
  void gm_drop() {
    for (auto& g : gm.step)
      if (g) cudaGraphExecDestroy(g);
    gm.step.clear();
  }
  int solve_gmres(const double* b, double* x, const xdg_gmres_opts* o, xdg_solve_info* info);
  // the preconditioner of the flexible GMRES: kind 0 = the multigrid cycle of precision prec,
  // kind 1 = the p-multigrid of Algorithm pMultigrid
  void gm_precond(int kind, int prec, const double* v, double* z) {
    if (kind == 1) pmg_apply(v, z);
    else precond(prec, v, z);
  }
  // p-multigrid of level 1: the low-order hierarchy, the high-order block inverses, vectors
  struct Pmg {
    int n_lo = 0;
    xdg_hier* lo = nullptr;
    double *Hinv = nullptr, *blo = nullptr, *xlo = nullptr, *res = nullptr;
    xdg_solve_opts inner{};
    int last_rc = 0;
  } pm;
  bool pmg_ready() const { return pm.lo != nullptr; }
  int pmg_setup(int n_lo, const xdg_hier_opts* lo_opts, double inner_tol, int inner_maxit, int inner_prec);
  void pmg_apply(const double* v, double* z) {
    Level& V = L[0];
    const int64_t nb = V.nb;
    pmg::take_lo(stream, nb, Np, pm.n_lo, v, pm.blo);
    CK_VOID(cudaMemsetAsync(pm.xlo, 0, nb * pm.n_lo * sizeof(double), stream));
    const int rc = pm.lo->solve_dev(pm.blo, pm.xlo, &pm.inner, nullptr);
    if (rc != XDG_OK && rc != XDG_ENOTCONV) pm.last_rc = rc;
    pmg::put_lo(stream, nb, Np, pm.n_lo, pm.xlo, z);
    spmv(0, z, v, pm.res, 1);
    pmg::hi_apply(stream, nb, Np, pm.n_lo, pm.Hinv, pm.res, z);
    launches += 4;
  }
  const double* omg_graph_x = nullptr;  // the solution vector the recorded passes write
  int64_t omg_pass_nodes = 0;
  int lanczos_swz(int l, int m, double* lmax);
  int rerecord();
  void restrict_(int l, const double* b, const double* x, double* rc) {
    launches += 2;
    Level& V = L[l];
    Level& C = L[l + 1];
    ops.resid_rt(grid(V.nb), stream, V.nb, V.rp, V.col, V.val, V.R, b, x, V.s);
    ops.gather(vgrid(C.nb * Np), stream, C.nb, V.cptr, V.ch, V.s, rc);
  }
  void prolong(int l, const double* zc, const double* xi, double* xo) {
    ++launches;
    Level& V = L[l];
    ops.prolong(grid(V.nb), stream, V.nb, V.agg, V.R, zc, xi, xo);
  }
  void coarse(const double* r, double* z) {
    ++launches;
    int64_t blocks = (nc * 32 + kThreads - 1) / kThreads;
    kl(k_gemv_seg<double>, (unsigned)blocks, kThreads, 0, stream)(nc, nprob, cs_doff, cs_moff, Minv, r, z);
  }
  void dot(int64_t n, const double* a, const double* b, double* out) {
    launches += 2;
    kl(k_dot_partial, kRedBlocks, kThreads, 0, stream)(n, a, b, partial);
    kl(k_sum_final, 1, kThreads, 0, stream)(kRedBlocks, partial, out);
  }

  // one symmetric cycle on level l from a zero initial guess: x = B_l b. pre0: x already
  // holds the first sweep omega D^{-1} b (done by the fused restriction of the finer level)
  void cycle(int l, const double* b, double* x, bool pre0 = false) {
    if (l == nlev - 1) {
      coarse(b, x);
      return;
    }
    Level& V = L[l];
    Level& C = L[l + 1];
    // pre-smoothing: nu sweeps, the first one from x = 0
    double* cur = x;
    double* oth = V.t;
    if (!pre0) smooth(l, b, nullptr, cur);
    for (int s = 1; s < nu; ++s) {
      smooth(l, b, cur, oth);
      std::swap(cur, oth);
    }
    // coarse-grid correction: gamma cycles on the coarse level; above the coarsest level the
    // restriction's gather also does the coarse level's first sweep
    if (l + 2 < nlev && !has_swz(l + 1)) {
      ops.resid_rt(grid(V.nb), stream, V.nb, V.rp, V.col, V.val, V.R, b, cur, V.s);
      ops.gather_smooth0(grid(C.nb), stream, C.nb, V.cptr, V.ch, V.s, C.Dinv, C.omega, C.omr, C.b, C.x);
      launches += 2;
      cycle(l + 1, C.b, C.x, true);
    } else {
      restrict_(l, b, cur, C.b);
      cycle(l + 1, C.b, C.x);
    }
    if (gamma > 1 && l + 2 < nlev && l < wlev) {
      for (int g = 1; g < gamma; ++g) {
        spmv(l + 1, C.x, C.b, C.r, 1);
        cycle(l + 1, C.r, C.dz);
        kl(k_axpy, vgrid(C.nb * Np), kThreads, 0, stream)(C.nb * Np, 1.0, C.dz, C.x);
        ++launches;
      }
    }
    // prolongation into the buffer from which nu post-sweeps end in x
    // nu alternating post-sweeps starting in `after` end in x
    double* after = (nu % 2 == 0) ? x : V.t;
    prolong(l, C.x, cur, after);
    cur = after;
    oth = (cur == x) ? V.t : x;
    for (int s = 0; s < nu; ++s) {
      smooth(l, b, cur, oth);
      std::swap(cur, oth);
    }
    if (cur != x) {
      kl(k_copy, vgrid(V.nb * Np), kThreads, 0, stream)(V.nb * Np, cur, x);
      ++launches;
    }
  }

  // q = M p on level 1 with p . q into S->pq and alpha = rz / pq (3 launches)
  void apply_alpha(bool pair = false) {
    Level& V = L[0];
    const int g = (pair && sym_pair)
                      ? ops.spmv_dot_df_sym(grid(V.nb), stream, V.nb, sy.urp, sy.ucol, sy.uval2, sy.uea, sy.L(), p2,
                                            ex2, s_p, s_q, partial, nullptr)
                  : pair ? ops.spmv_dot_df(grid(V.nb), stream, V.nb, V.rp, V.col, val2, ea2, p2, ex2, s_p, s_q, partial,
                                           nullptr)
                         : ops.spmv_dot(grid(V.nb), stream, V.nb, V.rp, V.col, V.val, s_p, s_q, partial);
    kl(k_cg_alpha_final, 1, kThreads, 0, stream)(g, partial, S);
    launches += 2;
  }

  // one CG iteration on level 1 (buffers s_*), scalars in S
  void pcg_iteration() {
    const int64_t n = L[0].nb * Np;
    apply_alpha();
    launches += 4;  // x/r update, its sum, beta, direction
    kl(k_pcg_xr, kRedBlocks, kThreads, 0, stream)(n, S, s_p, s_q, s_x, s_r, partial, nullptr);
    kl(k_sum_final, 1, kThreads, 0, stream)(kRedBlocks, partial, &S->rr);
    cycle(0, s_r, s_z);
    dot(n, s_r, s_z, &S->rz_new);
    kl(k_pcg_beta, 1, 1, 0, stream)(S);
    kl(k_pcg_p, vgrid(n), kThreads, 0, stream)(n, S, s_z, s_p);
  }

  // ---------------------------------------------------------------- low-precision cycle
  void cycle_lp(int p, int l, const float* b, float* x, bool pre0 = false) {
    const OpsLP& o = opl[p];
    if (fused_on[p] && l == fused_start[p] && pre0 && b == LP[p][l].b && x == LP[p][l].x && fused_csize[p] > 0) {
      o.fused_cluster(stream, fused_csize[p], fdesc[p], 1);
      ++launches;
      return;
    }
    if (fused_on[p] && l == fused_start[p] && pre0 && b == LP[p][l].b && x == LP[p][l].x) {
      cudaMemsetAsync(fbar, 0, sizeof(unsigned), stream);
      o.fused(stream, fused_grid[p], fdesc[p], 1);
      ++launches;
      return;
    }
    if (l == nlev - 1) {
      ++launches;
      int64_t blocks = (nc * 32 + kThreads - 1) / kThreads;
      kl(k_gemv_seg<float>, (unsigned)blocks, kThreads, 0, stream)(nc, nprob, cs_doff, cs_moff, Minv, b, x);
      return;
    }
    Level& V = L[l];
    Level& C = L[l + 1];
    LevelLP& W = LP[p][l];
    LevelLP& WC = LP[p][l + 1];
    const float om = (float)V.omega;
    const uint8_t* act = (l == 0) ? cur_act : nullptr;  // finished problems of a batch are skipped
    float* cur = x;
    float* oth = W.t;
    const bool schwarz = has_swz(l);
    if (!pre0) {
      if (schwarz) {
        swz_smooth_lp(p, l, b, nullptr, cur);
      } else {
        o.smooth(grid_lp(l), V.spl, stream, V.nb, V.rp, V.col, W.val32, W.sc32, W.Dinv, W.dsc, om, V.omr_f, b,
                 nullptr, cur, act);
        ++launches;
      }
    }
    const bool sym = lvl1_sym(l);
    auto sweep = [&](const float* xi, float* xo) {  // counts its own launches
      if (schwarz) {
        swz_smooth_lp(p, l, b, xi, xo);
        return;
      }
      if (sym)
        o.smooth_sym(grid_lp(l), stream, V.nb, sy.urp, sy.ucol, sy.uval, sy.usc, sy.L(), (const float*)W.Dinv, W.dsc, om, V.omr_f,
                     b, xi, xo, act);
      else
        o.smooth(grid_lp(l), V.spl, stream, V.nb, V.rp, V.col, W.val32, W.sc32, W.Dinv, W.dsc, om, V.omr_f, b, xi,
                 xo, act);
      ++launches;
    };
    for (int s = 1; s < nu; ++s) {
      sweep(cur, oth);
      std::swap(cur, oth);
    }
    if (sym)
      o.resid_rt_sym(grid_lp(l), stream, V.nb, sy.urp, sy.ucol, sy.uval, sy.usc, sy.L(), W.R, W.rsc, b, cur, W.s, act);
    else
      o.resid_rt(grid_lp(l), V.spl, stream, V.nb, V.rp, V.col, W.val32, W.sc32, W.R, W.rsc, b, cur, W.s, act);
    launches += 2;
    if (l + 2 < nlev && !has_swz(l + 1)) {
      o.gather_smooth0(grid(C.nb), stream, C.nb, V.cptr, V.ch, W.s, (const float*)WC.Dinv, WC.dsc, (float)C.omega,
                       C.omr_f, WC.b, WC.x);
      cycle_lp(p, l + 1, WC.b, WC.x, true);
    } else {
      o.gather(vgrid(C.nb * Np), stream, C.nb, V.cptr, V.ch, W.s, WC.b);
      cycle_lp(p, l + 1, WC.b, WC.x);
    }
    if (gamma > 1 && l + 2 < nlev && l < wlev) {
      for (int g = 1; g < gamma; ++g) {
        o.resid32(grid_lp(l + 1), C.spl, stream, C.nb, C.rp, C.col, WC.val32, WC.sc32, WC.x, WC.b, WC.r);
        cycle_lp(p, l + 1, WC.r, WC.dz);
        kl(k_axpy_f, vgrid(C.nb * Np), kThreads, 0, stream)(C.nb * Np, 1.0f, WC.dz, WC.x);
        launches += 2;
      }
    }
    float* after = (nu % 2 == 0) ? x : W.t;
    o.prolong(grid(V.nb), stream, V.nb, V.agg, W.R, W.rsc, WC.x, cur, after, act);
    ++launches;
    cur = after;
    oth = (cur == x) ? W.t : x;
    for (int s = 0; s < nu; ++s) {
      sweep(cur, oth);
      std::swap(cur, oth);
    }
    if (cur != x) {
      kl(k_copy_f, vgrid(V.nb * Np), kThreads, 0, stream)(V.nb * Np, cur, x);
      ++launches;
    }
  }

  // z = B_p r for FP64 vectors: round r to FP32, run the low-precision cycle, widen the result
  void cycle_lp_d(int p, const double* r, double* z) {
    const int64_t n = L[0].nb * Np;
    LevelLP& W = LP[p][0];
    kl(k_d2f, vgrid(n), kThreads, 0, stream)(n, r, W.b, cur_act, Np);
    cycle_lp(p, 0, W.b, W.x);
    kl(k_f2d, vgrid(n), kThreads, 0, stream)(n, W.x, z, cur_act, Np);
    launches += 2;
  }

  // z += theta * (kept learned corrections of the units) for the residual r - M z
  void learned_apply(const double* r, double* z) {
    Level& V = L[0];
    lr.ops.resid_rows(grid(lr.nt), stream, lr.nt, lr.tblk, V.rp, V.col, V.val, z, r, lr.res);
    lr.ops.apply(stream, lr.U, lr.d, lr.n_geo, lr.pairs, lr.geom, lr.res, lr.W, lr.Linv, lr.Mloc, lr.delta, lr.keep,
                 lr.E);
    lr.ops.gather(stream, lr.nt, lr.tblk, lr.tptr, lr.tlist, lr.delta, lr.theta, z);
    launches += 3;
  }
  // the preconditioner of the solve: cycle of precision p, then the learned correction when on
  void precond_full(int p, const double* r, double* z) {
    if (p == XDG_PREC_F64) cycle(0, r, z);
    else cycle_lp_d(p, r, z);
    if (lr.on) learned_apply(r, z);
  }

  // one flexible-CG iteration (FP64 operator, residual and updates; low-precision cycle):
  // q = M p with p . q; alpha; x, r updated with r . r and the FP32 copy of r; the cycle;
  // z widened with r . z and z . q; beta; p = z + beta p
  void fcg_iteration(int p) {
    const int64_t n = L[0].nb * Np;
    const bool pair = use_pair(p);
    apply_alpha(pair);
    if (p == XDG_PREC_F64) {  // FP64 cycle: generic tail
      kl(k_pcg_xr, kRedBlocks, kThreads, 0, stream)(n, S, s_p, s_q, s_x, s_r, partial, nullptr);
      kl(k_sum_final, 1, kThreads, 0, stream)(kRedBlocks, partial, &S->rr);
      launches += 2;
      precond_full(p, s_r, s_z);
      dot(n, s_r, s_z, &S->rz);
      dot(n, s_z, s_q, &S->zq);
      kl(k_fcg_beta, 1, 1, 0, stream)(S);
      ++launches;
    } else if (lr.on) {  // low-precision cycle, widened, plus the learned correction
      LevelLP& W = LP[p][0];
      kl(k_pcg_xr, kRedBlocks, kThreads, 0, stream)(n, S, s_p, s_q, s_x, s_r, partial, W.b);
      kl(k_sum_final, 1, kThreads, 0, stream)(kRedBlocks, partial, &S->rr);
      cycle_lp(p, 0, W.b, W.x);
      kl(k_f2d, vgrid(n), kThreads, 0, stream)(n, W.x, s_z, cur_act, Np);
      learned_apply(s_r, s_z);
      kl(k_fcg_dots, kRedBlocks, kThreads, 0, stream)(n, s_r, s_q, s_z, partial);
      kl(k_fcg_beta_final, 1, kThreads, 0, stream)(kRedBlocks, partial, S);
      launches += 5;
    } else {
      LevelLP& W = LP[p][0];
      kl(k_pcg_xr, kRedBlocks, kThreads, 0, stream)(n, S, s_p, s_q, s_x, s_r, partial, W.b);
      kl(k_sum_final, 1, kThreads, 0, stream)(kRedBlocks, partial, &S->rr);
      cycle_lp(p, 0, W.b, W.x);
      kl(k_fcg_tail, kRedBlocks, kThreads, 0, stream)(n, W.x, s_r, s_q, s_z, partial);
      kl(k_fcg_beta_final, 1, kThreads, 0, stream)(kRedBlocks, partial, S);
      launches += 4;
    }
    if (pair) ops.pcg_p_df(grid(L[0].nb), stream, L[0].nb, S, 0, s_z, s_p, p2, ex2);
    else kl(k_pcg_p, vgrid(n), kThreads, 0, stream)(n, S, s_z, s_p);
    ++launches;
  }

  int build_lp(int p);
  int tune_split(int p);
  bool tuned = false;
  int split_mode = 0;  // xdg_hier_opts.split_rows
  // small levels of the low-precision cycle as one persistent launch (levels fused_lc..)
  int fused_mode = 0;  // xdg_hier_opts.fused_coarse
  int fused_lc = -1;                // the first level the fused cycle may start at
  int fused_start[3] = {-1, -1, -1};  // the level it starts at, per precision (the descriptor's first)
  bool fused_on[3] = {false, false, false};
  int fused_grid[3] = {0, 0, 0};
  int fused_csize[3] = {0, 0, 0};  // > 0: the fused cycle runs as one cluster of this many CTAs
  FusedCycle* fdesc[3] = {nullptr, nullptr, nullptr};
  unsigned* fbar = nullptr;
  int* ferr = nullptr;
  unsigned fused_extra = 0;  // xdg_test_barrier_timeout
  int write_fused(int p, int start = -1);
  int tune_fused(int p);
  int fused_error();

  // which: 0 FP64 cycle, 1 FP64 CG iteration, 2 low-precision cycle, 3 flexible-CG iteration
  int capture(cudaGraphExec_t* out, int which, const double* b, double* x, int p = 0) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    const int64_t before = launches;
    if (which == 0) cycle(0, b, x);
    else if (which == 1) pcg_iteration();
    else if (which == 2) cycle_lp_d(p, b, x);
    else fcg_iteration(p);  // 3: low-precision cycle; 4: with the learned correction (lr.on)
    const int64_t recorded = launches - before;
    launches = before;
    if (which == 0) cycle_nodes = recorded;
    else if (which == 1) iter_nodes = recorded;
    else if (which == 2) cyc_lp_nodes[p] = recorded;
    else if (which == 3) iter_lp_nodes[p] = recorded;
    else lr.nodes[p] = recorded;
    cudaError_t e = cudaStreamEndCapture(stream, &g);
    if (e != cudaSuccess) {
      set_err("graph capture: %s", cudaGetErrorString(e));
      return XDG_ECUDA;
    }
    if (*out) cudaGraphExecDestroy(*out);
    *out = nullptr;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      set_err("graph instantiate: %s", cudaGetErrorString(e));
      return XDG_ECUDA;
    }
    return XDG_OK;
  }

  int sync() {
    CK(cudaStreamSynchronize(stream));
    return XDG_OK;
  }

  // host read of a device scalar
  int read_scalar(const double* d, double* h) {
    CK(cudaMemcpyAsync(hsc, d, sizeof(double), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    *h = hsc[0];
    return XDG_OK;
  }

  // out[s] = (x, y) restricted to problem s on level l (fixed-order slice sums)
  void seg_dot(int l, const double* x, const double* y, double* out) {
    const int spl = std::max(1, std::min(64, 4 * sms / nprob));
    kl(k_seg_dot, dim3((unsigned)spl, (unsigned)nprob), kThreads, 0, stream)(nprob, L[l].sdof, x, y, spart);
    kl(k_seg_sum, (nprob + 255) / 256, 256, 0, stream)(nprob, spl, spart, out);
  }
  int sgrid() const { return (nprob + 255) / 256; }
  // z = B r with the FP64 cycle (prec = F64) or the low-precision one
  void precond(int prec, const double* r, double* z) {
    if (prec == XDG_PREC_F64) cycle(0, r, z);
    else cycle_lp_d(prec, r, z);
  }

  std::vector<std::vector<int64_t>> seg_in;  // problem block offsets per level (set before build)
  int lanczos(int l, int m);
  int read_scalars(const double* d, int n, double* h);
  int build_batch(int n, const xdg_problem* probs, const xdg_hier_opts* o);
  void batch_iteration(int prec, const BatchCtl* ctl, cudaGraphConditionalHandle cond);
  int record_batch(int prec, const BatchCtl* ctl, double* res, int gslot);
  int build(const xdg_problem* p, const xdg_hier_opts* o);
  int solve_dev(const double* b, double* x, const xdg_solve_opts* o, xdg_solve_info* info);
};

namespace {

// largest eigenvalue of the symmetric tridiagonal matrix (a, b) by bisection on the number of
// negative pivots of T - s I
double tridiag_lambda_max(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    double rad = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - rad);
    hi = std::max(hi, a[i] + rad);
  }
  auto below = [&](double s) {
    int k = 0;
    double d = a[0] - s;
    if (d < 0) ++k;
    for (int i = 1; i < m; ++i) {
      if (d == 0.0) d = 1e-300;
      d = (a[i] - s) - b[i - 1] * b[i - 1] / d;
      if (d < 0) ++k;
    }
    return k;
  };
  for (int it = 0; it < 300 && hi - lo > 1e-15 * std::fabs(hi); ++it) {
    double mid = 0.5 * (lo + hi);
    if (below(mid) >= m) hi = mid;
    else lo = mid;
  }
  return hi;
}

}  // namespace

int xdg_hier::read_scalars(const double* d, int n, double* h) {
  CK(cudaMemcpyAsync(h_bsc, d, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  std::copy(h_bsc, h_bsc + n, h);
  return XDG_OK;
}

// m-step Lanczos for the pencil (M_l, D_l) in the D inner product, run for every problem of
// the level at once (segment-wise scalars); the start vector restarts the counter-based hash
// at every problem. Result: V.lmax_p.
int xdg_hier::lanczos(int l, int m) {
  Level& V = L[l];
  const int64_t n = V.nb * Np;
  const int P = nprob;
  double *q = V.b, *qp = V.x, *u = V.t, *w = V.r, *Dw = V.dz;
  const int vg = vgrid(n);
  double* dv = B.alpha;  // device scratch of nprob doubles (free during setup)
  kl(k_hash_vector_seg, vg, kThreads, 0, stream)(n, P, V.sdof, q);
  CK(cudaMemsetAsync(qp, 0, n * sizeof(double), stream));
  ops.diagmul(grid(V.nb), stream, V.nb, V.diag, V.val, q, Dw);
  seg_dot(l, q, Dw, dv);
  std::vector<double> nrm2(P), fac(P), a(P), b2(P), bprev(P, 0.0), coef(P);
  TRY(read_scalars(dv, P, nrm2.data()));
  for (int s = 0; s < P; ++s) fac[s] = 1.0 / std::sqrt(nrm2[s]);
  auto put = [&](const std::vector<double>& h) -> int {
    std::copy(h.begin(), h.end(), h_bsc);
    CK(cudaMemcpyAsync(dv, h_bsc, P * sizeof(double), cudaMemcpyHostToDevice, stream));
    CK(cudaStreamSynchronize(stream));  // h_bsc is reused by the next transfer
    return XDG_OK;
  };
  TRY(put(fac));
  kl(k_seg_scale, vg, kThreads, 0, stream)(n, P, V.sdof, dv, q);
  std::vector<std::vector<double>> al(P), be(P);
  std::vector<char> live(P, 1);
  for (int j = 0; j < m; ++j) {
    spmv(l, q, nullptr, u, 0);
    seg_dot(l, q, u, dv);
    TRY(read_scalars(dv, P, a.data()));
    for (int s = 0; s < P; ++s)
      if (live[s]) al[s].push_back(a[s]);
    ops.bjsolve(grid(V.nb), stream, V.nb, V.Dinv, u, w);
    for (int s = 0; s < P; ++s) coef[s] = -a[s];
    TRY(put(coef));
    kl(k_seg_axpy, vg, kThreads, 0, stream)(n, P, V.sdof, dv, q, w);
    for (int s = 0; s < P; ++s) coef[s] = -bprev[s];
    TRY(put(coef));
    kl(k_seg_axpy, vg, kThreads, 0, stream)(n, P, V.sdof, dv, qp, w);
    ops.diagmul(grid(V.nb), stream, V.nb, V.diag, V.val, w, Dw);
    seg_dot(l, w, Dw, dv);
    TRY(read_scalars(dv, P, b2.data()));
    CKL();
    bool any = false;
    for (int s = 0; s < P; ++s) {
      double bj = std::sqrt(std::max(b2[s], 0.0));
      if (live[s]) be[s].push_back(bj);
      if (!(bj > 1e-300)) live[s] = 0;
      fac[s] = live[s] ? 1.0 / bj : 0.0;
      bprev[s] = live[s] ? bj : 0.0;
      any = any || live[s];
    }
    if (!any) break;
    kl(k_copy, vg, kThreads, 0, stream)(n, q, qp);
    kl(k_copy, vg, kThreads, 0, stream)(n, w, q);
    TRY(put(fac));
    kl(k_seg_scale, vg, kThreads, 0, stream)(n, P, V.sdof, dv, q);
  }
  CKL();
  V.lmax_p.resize(P);
  for (int s = 0; s < P; ++s) V.lmax_p[s] = tridiag_lambda_max(al[s], be[s]);
  return XDG_OK;
}

int xdg_hier::build(const xdg_problem* p, const xdg_hier_opts* o) {
  auto t0 = clk::now();
  Np = p->Np;
  nlev = p->n_levels;
  if (nlev < 1 || nlev > XDG_MAX_LEVELS) {
    set_err("n_levels = %d outside 1..%d", nlev, XDG_MAX_LEVELS);
    return XDG_EINVAL;
  }
  if (!ops_for(Np, &ops)) {
    set_err("block size Np = %d not supported (3, 4, 6, 10, 15, 20, 35, 56)", Np);
    return XDG_EINVAL;
  }
  nu = o && o->nu > 0 ? o->nu : 1;
  gamma = o && o->gamma > 0 ? o->gamma : 1;
  wlev = o && o->w_levels > 0 ? o->w_levels : (1 << 20);
  split_mode = o ? o->split_rows : 0;
  fused_mode = o ? o->fused_coarse : 0;
  pair_mode = o ? o->outer_apply : 0;
  sym_mode = o ? o->symmetric : 0;
  const int lsteps = o && o->lanczos_steps > 0 ? o->lanczos_steps : 12;
  lanczos_m = lsteps;
  omega_fixed = (o && o->omega > 0.0) ? o->omega : 0.0;
  const int64_t Np2 = (int64_t)Np * Np;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  L.resize(nlev);
  // ------------------------------------------------------------------ validation (host)
  for (int l = 0; l < nlev; ++l) {
    if (p->nb[l] <= 0 || p->nb[l] > INT32_MAX) {
      set_err("level %d: nb = %lld", l + 1, (long long)p->nb[l]);
      return XDG_EINVAL;
    }
    L[l].nb = p->nb[l];
  }
  {
    Level& V = L[0];
    const int64_t nb = V.nb;
    if (!p->row_ptr || !p->col || !p->val) {
      set_err("null operator arrays");
      return XDG_EINVAL;
    }
    if (p->row_ptr[0] != 0) {
      set_err("row_ptr[0] = %lld", (long long)p->row_ptr[0]);
      return XDG_EINVAL;
    }
    V.h_rp.assign(p->row_ptr, p->row_ptr + nb + 1);
    for (int64_t i = 0; i < nb; ++i)
      if (V.h_rp[i + 1] < V.h_rp[i]) {
        set_err("row_ptr decreases at row %lld", (long long)i);
        return XDG_EINVAL;
      }
    V.nnzb = V.h_rp[nb];
    V.h_col.assign(p->col, p->col + V.nnzb);
    V.h_diag.assign(nb, -1);
    for (int64_t i = 0; i < nb; ++i)
      for (int64_t z = V.h_rp[i]; z < V.h_rp[i + 1]; ++z) {
        int32_t c = V.h_col[z];
        if (c < 0 || c >= nb || (z > V.h_rp[i] && c <= V.h_col[z - 1])) {
          set_err("col[%lld] = %d invalid or not increasing in row %lld", (long long)z, c, (long long)i);
          return XDG_EINVAL;
        }
        if (c == i) V.h_diag[i] = z;
      }
    for (int64_t i = 0; i < nb; ++i)
      if (V.h_diag[i] < 0) {
        set_err("row %lld has no diagonal block", (long long)i);
        return XDG_EINVAL;
      }
    for (int64_t e = 0; e < V.nnzb * Np2; ++e)
      if (!std::isfinite(p->val[e])) {
        set_err("val[%lld] is not finite", (long long)e);
        return XDG_EINVAL;
      }
  }
  for (int l = 0; l + 1 < nlev; ++l) {
    if (!p->agg || !p->R || !p->agg[l] || !p->R[l]) {
      set_err("level %d: null transfer arrays", l + 1);
      return XDG_EINVAL;
    }
    std::vector<int64_t> cnt(L[l + 1].nb, 0);
    for (int64_t f = 0; f < L[l].nb; ++f) {
      int32_t a = p->agg[l][f];
      if (a < 0 || a >= L[l + 1].nb) {
        set_err("level %d: agg[%lld] = %d out of range", l + 1, (long long)f, a);
        return XDG_EINVAL;
      }
      cnt[a]++;
    }
    for (int64_t c = 0; c < L[l + 1].nb; ++c)
      if (cnt[c] == 0) {
        set_err("level %d: coarse block %lld has no child", l + 2, (long long)c);
        return XDG_EINVAL;
      }
    for (int64_t e = 0; e < L[l].nb * Np2; ++e)
      if (!std::isfinite(p->R[l][e])) {
        set_err("level %d: R[%lld] is not finite", l + 1, (long long)e);
        return XDG_EINVAL;
      }
  }
  // ------------------------------------------------------------------ symbolic hierarchy (host)
  std::vector<std::vector<int64_t>> h_cptr(nlev);
  std::vector<std::vector<int32_t>> h_ch(nlev);
  for (int l = 0; l + 1 < nlev; ++l) {
    Level& F = L[l];
    Level& C = L[l + 1];
    const int32_t* agg = p->agg[l];
    auto& cp = h_cptr[l];
    auto& chl = h_ch[l];
    cp.assign(C.nb + 1, 0);
    for (int64_t f = 0; f < F.nb; ++f) cp[agg[f] + 1]++;
    for (int64_t c = 0; c < C.nb; ++c) cp[c + 1] += cp[c];
    chl.resize(F.nb);
    std::vector<int64_t> pos(cp.begin(), cp.end() - 1);
    for (int64_t f = 0; f < F.nb; ++f) chl[pos[agg[f]]++] = (int32_t)f;  // children ascending
    // coarse sparsity: agg of the fine columns of all children
    C.h_rp.assign(C.nb + 1, 0);
    std::vector<int32_t> cols;
    std::vector<std::vector<int32_t>> rows(C.nb);
    for (int64_t c = 0; c < C.nb; ++c) {
      cols.clear();
      for (int64_t t = cp[c]; t < cp[c + 1]; ++t) {
        int64_t f = chl[t];
        for (int64_t z = F.h_rp[f]; z < F.h_rp[f + 1]; ++z) cols.push_back(agg[F.h_col[z]]);
      }
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      rows[c] = cols;
      C.h_rp[c + 1] = C.h_rp[c] + (int64_t)cols.size();
    }
    C.nnzb = C.h_rp[C.nb];
    C.h_col.resize(C.nnzb);
    C.h_diag.assign(C.nb, -1);
    for (int64_t c = 0; c < C.nb; ++c) {
      std::copy(rows[c].begin(), rows[c].end(), C.h_col.begin() + C.h_rp[c]);
      for (int64_t z = C.h_rp[c]; z < C.h_rp[c + 1]; ++z)
        if (C.h_col[z] == c) C.h_diag[c] = z;
      if (C.h_diag[c] < 0) {
        set_err("level %d: coarse block %lld couples not with itself", l + 2, (long long)c);
        return XDG_EINVAL;
      }
    }
  }
  nc = L[nlev - 1].nb * Np;
  // problem segments per level (a single problem is one segment)
  if ((int)seg_in.size() != nlev) {
    seg_in.assign(nlev, std::vector<int64_t>());
    for (int l = 0; l < nlev; ++l) seg_in[l] = {0, L[l].nb};
  }
  nprob = (int)seg_in[0].size() - 1;
  std::vector<int64_t> h_csd(nprob + 1, 0), h_csm(nprob + 1, 0);
  for (int s = 0; s < nprob; ++s) {
    const int64_t ns = (seg_in[nlev - 1][s + 1] - seg_in[nlev - 1][s]) * Np;
    if (ns > 4096 || ns <= 0) {
      set_err("problem %d: coarsest level has %lld DOF; 1..4096 are supported", s, (long long)ns);
      return XDG_EINVAL;
    }
    h_csd[s + 1] = h_csd[s] + ns;
    h_csm[s + 1] = h_csm[s] + ns * ns;
  }
  const int64_t minv_len = h_csm[nprob];
  // ------------------------------------------------------------------ device memory
  if (!stream) {
    CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    own_stream = true;
  }
  for (int l = 0; l < nlev; ++l) {
    Level& V = L[l];
    const int64_t n = V.nb * Np;
    TRY(alloc(&V.rp, V.nb + 1));
    TRY(alloc(&V.col, V.nnzb));
    TRY(alloc(&V.val, V.nnzb * Np2));
    TRY(alloc(&V.diag, V.nb));
    TRY(alloc(&V.b, n));
    TRY(alloc(&V.x, n));
    TRY(alloc(&V.t, n));
    TRY(alloc(&V.r, n));
    TRY(alloc(&V.dz, n));
    CK(cudaMemcpyAsync(V.rp, V.h_rp.data(), (V.nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(V.col, V.h_col.data(), std::max<int64_t>(V.nnzb, 0) * sizeof(int32_t),
                       cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(V.diag, V.h_diag.data(), V.nb * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    if (l + 1 < nlev) {
      TRY(alloc(&V.Dinv, V.nb * Np2));
      TRY(alloc(&V.s, n));
      TRY(alloc(&V.agg, V.nb));
      TRY(alloc(&V.R, V.nb * Np2));
      TRY(alloc(&V.cptr, L[l + 1].nb + 1));
      TRY(alloc(&V.ch, V.nb));
      CK(cudaMemcpyAsync(V.agg, p->agg[l], V.nb * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
      CK(cudaMemcpyAsync(V.R, p->R[l], V.nb * Np2 * sizeof(double), cudaMemcpyHostToDevice, stream));
      CK(cudaMemcpyAsync(V.cptr, h_cptr[l].data(), (L[l + 1].nb + 1) * sizeof(int64_t),
                         cudaMemcpyHostToDevice, stream));
      CK(cudaMemcpyAsync(V.ch, h_ch[l].data(), V.nb * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    }
  }
  CK(cudaMemcpyAsync(L[0].val, p->val, L[0].nnzb * Np2 * sizeof(double), cudaMemcpyHostToDevice, stream));
  const int64_t n1 = L[0].nb * Np;
  TRY(alloc(&s_b, n1));
  TRY(alloc(&s_x, n1));
  TRY(alloc(&s_r, n1));
  TRY(alloc(&s_z, n1));
  TRY(alloc(&s_p, n1));
  TRY(alloc(&s_q, n1));
  TRY(alloc(&partial, 2 * (size_t)kPartials));
  TRY(alloc(&dsc, 8));
  TRY(alloc(&S, 1));
  TRY(alloc(&Minv, minv_len));
  TRY(alloc(&cs_doff, nprob + 1));
  TRY(alloc(&cs_moff, nprob + 1));
  CK(cudaMemcpyAsync(cs_doff, h_csd.data(), (nprob + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(cs_moff, h_csm.data(), (nprob + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  for (int l = 0; l < nlev; ++l) {
    Level& V = L[l];
    V.hseg = seg_in[l];
    std::vector<int64_t> d(nprob + 1);
    for (int s = 0; s <= nprob; ++s) d[s] = V.hseg[s] * Np;
    TRY(alloc(&V.sdof, nprob + 1));
    CK(cudaMemcpyAsync(V.sdof, d.data(), (nprob + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  }
  {
    // per-problem Krylov scalars and the level-1 chunks of the batched reductions
    double** f[] = {&B.rz, &B.rr, &B.bb, &B.pq, &B.zq, &B.alpha, &B.beta};
    for (double** q : f) TRY(alloc(q, nprob));
    TRY(alloc(&B.active, nprob));
    TRY(alloc(&B.bad, nprob));
    TRY(alloc(&B.iters, nprob));
    TRY(alloc(&B.it, 1));
    TRY(alloc(&act1, L[0].nb));
    TRY(alloc(&spart, (size_t)nprob * 64));
    CK(cudaMallocHost(&h_bsc, (nprob + 1) * sizeof(double)));
    const int64_t target = std::max<int64_t>(1, n1 / (4 * (int64_t)sms));
    const int64_t ch = std::min<int64_t>(65536, std::max<int64_t>(2048, (target + 1023) / 1024 * 1024));
    std::vector<int64_t> hcb(1, 0);
    std::vector<int> hcs, hcf(1, 0);
    for (int s = 0; s < nprob; ++s) {
      const int64_t lo = seg_in[0][s] * Np, len = (seg_in[0][s + 1] - seg_in[0][s]) * Np;
      const int64_t m = std::max<int64_t>(1, (len + ch - 1) / ch);
      for (int64_t j = 1; j <= m; ++j) {
        hcb.push_back(lo + len * j / m);
        hcs.push_back(s);
      }
      hcf.push_back((int)hcs.size());
    }
    nchunk = (int)hcs.size();
    TRY(alloc(&cb, nchunk + 1));
    TRY(alloc(&cseg, nchunk));
    TRY(alloc(&cfirst, nprob + 1));
    TRY(alloc(&cpart, 2 * (size_t)nchunk));
    CK(cudaMemcpyAsync(cb, hcb.data(), (nchunk + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(cseg, hcs.data(), nchunk * sizeof(int), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(cfirst, hcf.data(), (nprob + 1) * sizeof(int), cudaMemcpyHostToDevice, stream));
    // caller layout: by default the problems in hierarchy order
    std::vector<int64_t> hio(nprob);
    std::vector<int> hgi(nprob);
    for (int s = 0; s < nprob; ++s) {
      hio[s] = seg_in[0][s] * Np;
      hgi[s] = s;
    }
    TRY(alloc(&ioff, nprob));
    TRY(alloc(&gidx, nprob));
    CK(cudaMemcpyAsync(ioff, hio.data(), nprob * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(gidx, hgi.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, stream));
    TRY(sync());
  }
  CK(cudaMallocHost(&hS, sizeof(PcgScal)));
  CK(cudaMallocHost(&hsc, 8 * sizeof(double)));
  int* derr = nullptr;
  TRY(alloc(&derr, 1));
  CK(cudaMemsetAsync(derr, 0, sizeof(int), stream));
  TRY(sync());
  setup_ms[0] = ms_since(t0);
  // ------------------------------------------------------------------ Galerkin products (device)
  t0 = clk::now();
  for (int l = 0; l + 1 < nlev; ++l) {
    Level& F = L[l];
    Level& C = L[l + 1];
    CK(cudaMemsetAsync(C.val, 0, C.nnzb * Np2 * sizeof(double), stream));
    ops.galerkin(grid(C.nb), stream, C.nb, F.cptr, F.ch, F.rp, F.col, F.val, F.agg, F.R, C.rp, C.col, C.val);
    CKL();
  }
  TRY(sync());
  setup_ms[1] = ms_since(t0);
  // ------------------------------------------------------------------ factorisations, damping
  t0 = clk::now();
  for (int l = 0; l + 1 < nlev; ++l) {
    Level& V = L[l];
    ops.diag_inv(stream, V.nb, V.diag, V.val, V.Dinv, derr);
    CKL();
  }
  {
    int h_err = 0;
    CK(cudaMemcpyAsync(&h_err, derr, sizeof(int), cudaMemcpyDeviceToHost, stream));
    TRY(sync());
    if (h_err) {
      set_err("a diagonal block is not positive definite");
      return XDG_EBREAKDOWN;
    }
  }
  for (int l = 0; l + 1 < nlev; ++l) {
    Level& V = L[l];
    TRY(lanczos(l, lsteps));
    V.omega_p.resize(nprob);
    for (int s = 0; s < nprob; ++s)
      V.omega_p[s] = (o && o->omega > 0.0) ? o->omega : 4.0 / (3.0 * V.lmax_p[s]);
    V.lmax = V.lmax_p[0];
    V.omega = V.omega_p[0];
    if (nprob > 1) {  // damping per block row
      std::vector<double> om(V.nb);
      std::vector<float> omf(V.nb);
      for (int s = 0; s < nprob; ++s)
        for (int64_t i = V.hseg[s]; i < V.hseg[s + 1]; ++i) {
          om[i] = V.omega_p[s];
          omf[i] = (float)V.omega_p[s];
        }
      TRY(alloc(&V.omr, V.nb));
      TRY(alloc(&V.omr_f, V.nb));
      CK(cudaMemcpyAsync(V.omr, om.data(), V.nb * sizeof(double), cudaMemcpyHostToDevice, stream));
      CK(cudaMemcpyAsync(V.omr_f, omf.data(), V.nb * sizeof(float), cudaMemcpyHostToDevice, stream));
      TRY(sync());
    }
  }
  {
    // coarsest level: dense Cholesky and explicit inverse of every problem's matrix
    Level& C = L[nlev - 1];
    double *A = nullptr, *X = nullptr;
    int64_t* cs_blk = nullptr;
    TRY(alloc(&A, minv_len));
    TRY(alloc(&X, minv_len));
    TRY(alloc(&cs_blk, nprob + 1));
    CK(cudaMemcpyAsync(cs_blk, C.hseg.data(), (nprob + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    CK(cudaMemsetAsync(A, 0, minv_len * sizeof(double), stream));
    kl(k_bsr_to_dense_seg, (unsigned)C.nb, 128, 0, stream)(C.nb, Np, nprob, cs_blk, cs_moff, C.rp, C.col, C.val, A);
    CK(cudaMemsetAsync(derr, 0, sizeof(int), stream));
    int64_t* cs_n = nullptr;
    TRY(alloc(&cs_n, nprob));
    int64_t nmax = 0;
    {
      std::vector<int64_t> hn(nprob);
      for (int s = 0; s < nprob; ++s) {
        hn[s] = h_csd[s + 1] - h_csd[s];
        nmax = std::max(nmax, hn[s]);
      }
      CK(cudaMemcpyAsync(cs_n, hn.data(), nprob * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    }
    kl(k_dense_chol_seg, (unsigned)nprob, 1024, 0, stream)(nprob, cs_n, cs_moff, A, derr);
    kl(k_tri_inverse_seg, dim3((unsigned)((nmax + 127) / 128), (unsigned)nprob), 128, 0, stream)(nprob, cs_n, cs_moff,
                                                                                                A, X);
    dim3 tb(16, 16), tg((unsigned)((nmax + 15) / 16), (unsigned)((nmax + 15) / 16), (unsigned)nprob);
    kl(k_xtx_seg, tg, tb, 0, stream)(nprob, cs_n, cs_moff, X, Minv);
    CKL();
    int h_err = 0;
    CK(cudaMemcpyAsync(&h_err, derr, sizeof(int), cudaMemcpyDeviceToHost, stream));
    TRY(sync());
    if (h_err) {
      set_err("coarsest operator is not positive definite");
      return XDG_EBREAKDOWN;
    }
    // scratch no longer needed
    for (auto it = allocs.begin(); it != allocs.end();) {
      if (*it == A || *it == X) {
        cudaFree(*it);
        it = allocs.erase(it);
      } else {
        ++it;
      }
    }
    bytes -= 2 * minv_len * sizeof(double);
  }
  TRY(capture(&g_iter, 1, nullptr, nullptr));
  if (o && (o->low_precision & 1)) TRY(build_lp(XDG_PREC_F32));
  if (o && (o->low_precision & 2)) TRY(build_lp(XDG_PREC_BF16));
  TRY(sync());
  setup_ms[2] = ms_since(t0);
  return XDG_OK;
}

// low-precision copies of every level (operator, block inverses, transfers: entry / block scale,
// rounded to FP32 or BF16) and FP32 work vectors; the FP64 originals stay resident
int xdg_hier::build_lp(int p) {
  if (!ops_lp_for(Np, p, &opl[p])) {
    set_err("no low-precision kernels for Np = %d", Np);
    return XDG_EINVAL;
  }
  const int np2 = Np * Np;
  const size_t el = opl[p].elem;
  LP[p].resize(nlev);
  for (int l = 0; l < nlev; ++l) {
    Level& V = L[l];
    LevelLP& W = LP[p][l];
    const int64_t n = V.nb * Np;
    char* raw = nullptr;
    TRY(alloc(&raw, V.nnzb * np2 * el));
    W.val = raw;
    TRY(alloc(&W.sc, V.nnzb));
    opl[p].make(stream, V.nnzb, np2, V.val, W.val, W.sc);
    if (p == XDG_PREC_F32) {
      W.val32 = W.val;
      W.sc32 = W.sc;
    } else if (has_lp[XDG_PREC_F32]) {  // share the FP32 copy
      W.val32 = LP[XDG_PREC_F32][l].val;
      W.sc32 = LP[XDG_PREC_F32][l].sc;
    } else {
      float* v32 = nullptr;
      TRY(alloc(&v32, V.nnzb * np2));
      TRY(alloc(&W.sc32, V.nnzb));
      kl(k_make_lp<float>, (unsigned)((V.nnzb * 32 + 255) / 256), 256, 0, stream)(V.nnzb, np2, V.val, v32,
                                                                                   W.sc32);
      W.val32 = v32;
    }
    TRY(alloc(&W.b, n));
    TRY(alloc(&W.x, n));
    TRY(alloc(&W.t, n));
    TRY(alloc(&W.r, n));
    TRY(alloc(&W.dz, n));
    if (l + 1 < nlev) {
      float* dinv = nullptr;  // FP32 in both modes
      TRY(alloc(&dinv, V.nb * np2));
      W.Dinv = dinv;
      TRY(alloc(&W.dsc, V.nb));
      kl(k_make_lp<float>, (unsigned)((V.nb * 32 + 255) / 256), 256, 0, stream)(V.nb, np2, V.Dinv, dinv, W.dsc);
      TRY(alloc(&raw, V.nb * np2 * el));
      W.R = raw;
      TRY(alloc(&W.rsc, V.nb));
      opl[p].make(stream, V.nb, np2, V.R, W.R, W.rsc);
      TRY(alloc(&W.s, n));
    }
    CKL();
  }
  TRY(sync());
  has_lp[p] = true;
  if (!tuned) {
    if (split_mode == 0) {
      TRY(tune_split(p));
    } else {
      for (int l = 0; l < nlev; ++l) L[l].spl = (split_mode == 2);
      tuned = true;
    }
  }
  if (!sym_tried && sym_mode != 1 && nlev > 1) {
    sym_tried = true;
    TRY(build_sym());
    if (sym_built) {
      if (sym_mode == 2) sym_on = !L[0].spl;
      else TRY(tune_sym(p));
    }
  }
  if (pair_mode != 1 && !val2) {
    TRY(build_pair());
    if (pair_mode == 2) {
      pair_on = true;
      sym_pair = sym_built && sym_mode == 2;
    }
    if (pair_mode != 2 || sym_mode == 0) TRY(tune_pair());
  }
  TRY(write_fused(p));
  if (fused_lc >= 0 && nprob == 1 && fused_mode != 1) {
    if (fused_mode == 2) {
      fused_on[p] = true;
    } else if (fused_mode == 3) {
      for (int cs : {16, 8})
        if (fused_csize[p] == 0 && opl[p].fused_cluster_ok(cs)) fused_csize[p] = cs;
      fused_on[p] = fused_csize[p] > 0;
    } else {
      TRY(tune_fused(p));
    }
  }
  TRY(capture(&g_iter_lp[p], 3, nullptr, nullptr, p));
  return XDG_OK;
}

// Autotuner of the low-precision row kernels: for every level with a smoother, time a sweep
// with one block row per group (rows spread over the warp's groups) and with one row per warp
// (the warp's groups splitting each row), and keep the faster (split only when >= 5 % faster).
// The same mapping then serves the residual-restriction and operator kernels of that level.
// CTAs per SM of the fused small-level cycle (fewer CTAs: cheaper grid barriers)
#ifndef XDG_FUSED_CTAS_PER_SM
#define XDG_FUSED_CTAS_PER_SM 4
#endif

// The fused small-level cycle of precision p: the first fused level is the first level below
// the W-cycle levels (at least level 2) with at most 16384 blocks, if it lies above the
// coarsest; the descriptor lists every fused level's arrays.
int xdg_hier::write_fused(int p, int start) {
  fused_lc = -1;
  const int lc = std::max(1, std::min(wlev, nlev));
  if (lc + 2 > nlev || L[lc].nb > 16384 || nlev - lc > kFusedMaxLevels) return XDG_OK;
  fused_lc = lc;
  if (start < 0) start = fused_start[p] >= lc ? fused_start[p] : lc;
  if (start + 2 > nlev) start = lc;
  fused_start[p] = start;
  if (!fbar) {
    TRY(alloc(&fbar, 1));
    TRY(alloc(&ferr, 1));
    CK(cudaMemsetAsync(ferr, 0, sizeof(int), stream));
  }
  if (!fdesc[p]) TRY(alloc(&fdesc[p], 1));
  FusedCycle h;
  std::memset(&h, 0, sizeof(h));
  h.n = nlev - start;
  h.nu = nu;
  for (int l = start; l < nlev; ++l) {
    Level& V = L[l];
    LevelLP& W = LP[p][l];
    FusedLevel& f = h.L[l - start];
    f.nb = V.nb;
    f.rp = V.rp;
    f.col = V.col;
    f.val = (const float*)W.val32;
    f.sc = W.sc32;
    f.Dinv = (const float*)W.Dinv;
    f.dsc = W.dsc;
    f.omega = (float)V.omega;
    f.spl = V.spl ? 1 : 0;
    f.R = W.R;
    f.rsc = W.rsc;
    f.agg = V.agg;
    f.cptr = V.cptr;
    f.ch = V.ch;
    f.b = W.b;
    f.x = W.x;
    f.t = W.t;
    f.s = W.s;
  }
  h.Minv = Minv;
  h.doff = cs_doff;
  h.moff = cs_moff;
  h.nseg = nprob;
  h.nc = nc;
  h.bar = fbar;
  h.err = ferr;
  h.extra = fused_extra;
  CK(cudaMemcpyAsync(fdesc[p], &h, sizeof(h), cudaMemcpyHostToDevice, stream));
  const int occ = opl[p].fused_occupancy();
  fused_grid[p] = std::max(1, std::min(occ, XDG_FUSED_CTAS_PER_SM)) * sms;
  if (occ < 1) fused_lc = -1;
  TRY(sync());
  return XDG_OK;
}

// time the low-precision cycle with the small levels launched per step, fused in one
// cooperative grid, and fused in one thread-block cluster of 16 or 8 CTAs; keep the fastest
// (a fused form only when >= 3 % faster than per step)
int xdg_hier::tune_fused(int p) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  LevelLP& W = LP[p][0];
  const int64_t n = L[0].nb * Np;
  CK(cudaMemsetAsync(W.r, 0, n * sizeof(float), stream));
  struct Cand {
    bool on;
    int csize, start;
  };
  // starts: the first level below the W levels, and (for a cluster, which has few SMs) the first
  // level with at most 1024 blocks if that lies lower and above the coarsest
  int lsmall = fused_lc;
  while (lsmall + 2 < nlev && L[lsmall].nb > 1024) ++lsmall;
  std::vector<Cand> cands = {{false, 0, fused_lc}, {true, 0, fused_lc}};
  for (int cs : {16, 8}) {
    if (!opl[p].fused_cluster_ok(cs)) continue;
    cands.push_back({true, cs, fused_lc});
    if (lsmall > fused_lc && L[lsmall].nb <= 1024) cands.push_back({true, cs, lsmall});
    break;
  }
  std::vector<float> ms(cands.size(), 0.f);
  int rc = XDG_OK;
  for (size_t v = 0; v < cands.size() && rc == XDG_OK; ++v) {
    fused_on[p] = cands[v].on;
    fused_csize[p] = cands[v].csize;
    if (cands[v].on) TRY(write_fused(p, cands[v].start));
    for (int k = 0; k < 2; ++k) cycle_lp(p, 0, W.r, W.dz);
    cudaEventRecord(e0, stream);
    for (int k = 0; k < 10; ++k) cycle_lp(p, 0, W.r, W.dz);
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms[v], e0, e1) != cudaSuccess)
      rc = XDG_ECUDA;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  fused_on[p] = false;
  fused_csize[p] = 0;
  if (rc) {
    set_err("fused-cycle tuning: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  TRY(fused_error());
  size_t best = 0;
  for (size_t v = 1; v < cands.size(); ++v)
    if (ms[v] < 0.97f * ms[0] && ms[v] < ms[best]) best = v;
  fused_on[p] = cands[best].on;
  fused_csize[p] = cands[best].csize;
  TRY(write_fused(p, cands[best].start));
  return XDG_OK;
}

// the error word of the fused cycle's barriers (XDG_ECUDA if one gave up; cleared)
int xdg_hier::fused_error() {
  if (!ferr) return XDG_OK;
  int h = 0;
  CK(cudaMemcpyAsync(&h, ferr, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  if (h) {
    cudaMemsetAsync(ferr, 0, sizeof(int), stream);
    set_err("fused small-level cycle: a grid barrier timed out");
    return XDG_ETIMEOUT;
  }
  return XDG_OK;
}

// Level 1 as scaled FP32 pairs (XDG_PREC_F64_PAIR) and the pair copy of the direction
int xdg_hier::build_pair() {
  Level& V = L[0];
  const int64_t np2 = (int64_t)Np * Np;
  TRY(alloc(&val2, V.nnzb * np2));
  TRY(alloc(&ea2, V.nnzb));
  TRY(alloc(&p2, V.nb * Np));
  TRY(alloc(&ex2, V.nb));
  kl(k_make_df, (unsigned)std::min<int64_t>((V.nnzb * 32 + 255) / 256, 65535 * 8), 256, 0, stream)(V.nnzb, (int)np2,
                                                                                                 V.val, val2, ea2);
  if (sym_built) {
    TRY(alloc(&sy.uval2, sy.nu * np2));
    TRY(alloc(&sy.uea, sy.nu));
    kl(k_gather_blocks_df, (unsigned)((sy.nu * 32 + 255) / 256), 256, 0, stream)(sy.nu, (int)np2, sy.umap, val2, ea2,
                                                                                 sy.uval2, sy.uea);
  }
  CKL();
  return sync();
}

// Outer apply: the FP64 product, the pair product and the pair product on the symmetric storage
// are timed with the direction update that precedes them in an iteration (FP64, or the update
// that also writes the pair copy). A pair variant is kept when it takes at least 3 % less time
// than the FP64 one (outer_apply = 0), the symmetric one when it is the faster pair variant
// (symmetric = 0).
int xdg_hier::tune_pair() {
  Level& V = L[0];
  const int64_t n = V.nb * Np;
  CK(cudaMemsetAsync(s_z, 0, n * sizeof(double), stream));
  CK(cudaMemsetAsync(s_p, 0, n * sizeof(double), stream));
  CK(cudaMemsetAsync(S, 0, sizeof(PcgScal), stream));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float ms[3] = {0.f, 0.f, 1e30f};
  const int nv = sym_built ? 3 : 2;
  int rc = XDG_OK;
  for (int v = 0; v < nv && rc == XDG_OK; ++v) {
    auto step = [&]() {
      if (v == 0) {
        kl(k_pcg_p, vgrid(n), kThreads, 0, stream)(n, S, s_z, s_p);
        ops.spmv_dot(grid(V.nb), stream, V.nb, V.rp, V.col, V.val, s_p, s_q, partial);
      } else {
        ops.pcg_p_df(grid(V.nb), stream, V.nb, S, 0, s_z, s_p, p2, ex2);
        if (v == 1)
          ops.spmv_dot_df(grid(V.nb), stream, V.nb, V.rp, V.col, val2, ea2, p2, ex2, s_p, s_q, partial, nullptr);
        else
          ops.spmv_dot_df_sym(grid(V.nb), stream, V.nb, sy.urp, sy.ucol, sy.uval2, sy.uea, sy.L(), p2, ex2, s_p, s_q,
                              partial, nullptr);
      }
    };
    for (int k = 0; k < 3; ++k) step();
    cudaEventRecord(e0, stream);
    for (int k = 0; k < 10; ++k) step();
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms[v], e0, e1) != cudaSuccess) rc = XDG_ECUDA;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    set_err("outer apply autotuning: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  const float best_pair = std::min(ms[1], ms[2]);
  if (pair_mode == 0) pair_on = best_pair < 0.97f * ms[0];
  if (sym_mode == 0) sym_pair = sym_built && ms[2] < ms[1];
  return XDG_OK;
}

// Symmetric storage of level 1 (see k_smooth_lp_sym), built when every left block has a right
// mirror and the two are exact transposes (checked on the device); the FP32 values are gathered
// from the low-precision copy of precision p, the pair values (when built) in build_pair.
int xdg_hier::build_sym() {
  Level& V = L[0];
  const int64_t nb = V.nb, np2 = (int64_t)Np * Np;
  std::vector<int64_t> urp(nb + 1, 0), umap, lrp(nb + 1, 0), pos;
  std::vector<int32_t> ucol, lcol, lblk;
  umap.reserve((V.nnzb + nb) / 2 + 1);
  ucol.reserve((V.nnzb + nb) / 2 + 1);
  for (int64_t i = 0; i < nb; ++i) {
    for (int64_t z = V.h_rp[i]; z < V.h_rp[i + 1]; ++z)
      if (V.h_col[z] >= i) {
        ucol.push_back(V.h_col[z]);
        umap.push_back(z);
      }
    urp[i + 1] = (int64_t)ucol.size();
  }
  for (int64_t i = 0; i < nb; ++i) {
    for (int64_t z = V.h_rp[i]; z < V.h_rp[i + 1] && V.h_col[z] < i; ++z) {
      const int32_t j = V.h_col[z];
      auto b0 = ucol.begin() + urp[j], b1 = ucol.begin() + urp[j + 1];
      auto it = std::lower_bound(b0, b1, (int32_t)i);
      if (it == b1 || *it != (int32_t)i) return XDG_OK;  // structurally not symmetric: full storage only
      const int64_t u = it - ucol.begin();
      lcol.push_back(j);
      lblk.push_back((int32_t)u);
      pos.push_back(z);
      pos.push_back(umap[u]);
    }
    lrp[i + 1] = (int64_t)lcol.size();
  }
  if ((int64_t)lcol.size() != (int64_t)ucol.size() - nb || (int64_t)ucol.size() > INT32_MAX) return XDG_OK;
  sy.nu = (int64_t)ucol.size();
  sy.nl = (int64_t)lcol.size();
  TRY(alloc(&sy.urp, nb + 1));
  TRY(alloc(&sy.umap, sy.nu));
  TRY(alloc(&sy.ucol, sy.nu));
  TRY(alloc(&sy.lrp, nb + 1));
  TRY(alloc(&sy.lcol, sy.nl));
  TRY(alloc(&sy.lblk, sy.nl));
  int64_t* dpos = nullptr;
  int* dbad = nullptr;
  TRY(alloc(&dpos, 2 * sy.nl));
  TRY(alloc(&dbad, 1));
  CK(cudaMemcpyAsync(sy.urp, urp.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(sy.umap, umap.data(), sy.nu * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(sy.ucol, ucol.data(), sy.nu * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(sy.lrp, lrp.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  if (sy.nl) {
    CK(cudaMemcpyAsync(sy.lcol, lcol.data(), sy.nl * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(sy.lblk, lblk.data(), sy.nl * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(dpos, pos.data(), 2 * sy.nl * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  }
  CK(cudaMemsetAsync(dbad, 0, sizeof(int), stream));
  if (sy.nl)
    kl(k_check_mirror, (unsigned)std::min<int64_t>((sy.nl * np2 + 255) / 256, 1 << 20), 256, 0, stream)(sy.nl, Np,
                                                                                                      dpos, V.val, dbad);
  int h_bad = 0;
  CK(cudaMemcpyAsync(&h_bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, stream));
  TRY(sync());
  if (h_bad) return XDG_OK;  // not exactly symmetric: full storage only
  // FP32 values from the low-precision copy (the cycle's operator)
  int p = has_lp[XDG_PREC_F32] ? XDG_PREC_F32 : XDG_PREC_BF16;
  const LevelLP& W = LP[p][0];
  TRY(alloc(&sy.uval, sy.nu * np2));
  TRY(alloc(&sy.usc, sy.nu));
  kl(k_gather_blocks, (unsigned)((sy.nu * 32 + 255) / 256), 256, 0, stream)(sy.nu, (int)np2, sy.umap,
                                                                            (const float*)W.val32, W.sc32, sy.uval,
                                                                            sy.usc);
  CKL();
  TRY(sync());
  sym_built = true;
  return XDG_OK;
}

// The level-1 sweep on the full and on the symmetric storage, timed as in tune_split; the
// symmetric one is kept when it is at least 3 % faster (the restriction follows the sweep).
int xdg_hier::tune_sym(int p) {
  Level& V = L[0];
  if (V.spl) {
    sym_on = false;
    return XDG_OK;
  }
  const OpsLP& o = opl[p];
  LevelLP& W = LP[p][0];
  const int64_t n = V.nb * Np;
  CK(cudaMemsetAsync(W.b, 0, n * sizeof(float), stream));
  CK(cudaMemsetAsync(W.x, 0, n * sizeof(float), stream));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float ms[2] = {0.f, 0.f};
  int rc = XDG_OK;
  for (int v = 0; v < 2 && rc == XDG_OK; ++v) {
    auto sweep = [&]() {
      if (v == 1)
        o.smooth_sym(grid_lp(0), stream, V.nb, sy.urp, sy.ucol, sy.uval, sy.usc, sy.L(), (const float*)W.Dinv, W.dsc,
                     (float)V.omega, V.omr_f, W.b, W.x, W.t, nullptr);
      else
        o.smooth(grid_lp(0), false, stream, V.nb, V.rp, V.col, W.val32, W.sc32, W.Dinv, W.dsc, (float)V.omega,
                 V.omr_f, W.b, W.x, W.t, nullptr);
    };
    for (int k = 0; k < 3; ++k) sweep();
    cudaEventRecord(e0, stream);
    for (int k = 0; k < 10; ++k) sweep();
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms[v], e0, e1) != cudaSuccess) rc = XDG_ECUDA;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    set_err("symmetric storage autotuning: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  sym_on = ms[1] < 0.97f * ms[0];
  return XDG_OK;
}

int xdg_hier::tune_split(int p) {
  const OpsLP& o = opl[p];
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = XDG_OK;
  for (int l = 0; l + 1 < nlev && rc == XDG_OK; ++l) {
    Level& V = L[l];
    LevelLP& W = LP[p][l];
    const int64_t n = V.nb * Np;
    if (cudaMemsetAsync(W.b, 0, n * sizeof(float), stream) != cudaSuccess ||
        cudaMemsetAsync(W.x, 0, n * sizeof(float), stream) != cudaSuccess) {
      rc = XDG_ECUDA;
      break;
    }
    float ms[2] = {0.f, 0.f};
    for (int v = 0; v < 2; ++v) {
      V.spl = (v == 1);
      auto sweep = [&]() {
        o.smooth(grid_lp(l), V.spl, stream, V.nb, V.rp, V.col, W.val32, W.sc32, W.Dinv, W.dsc, (float)V.omega,
                 V.omr_f, W.b, W.x, W.t, nullptr);
      };
      for (int k = 0; k < 3; ++k) sweep();
      cudaEventRecord(e0, stream);
      for (int k = 0; k < 10; ++k) sweep();
      cudaEventRecord(e1, stream);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms[v], e0, e1) != cudaSuccess) {
        rc = XDG_ECUDA;
        break;
      }
    }
    V.spl = ms[1] < 0.95f * ms[0];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    set_err("split autotuning: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  tuned = true;
  return XDG_OK;
}

// Host validation of problem s of a batch against its own sizes (no CUDA call).
// The recorded graphs hold the cycle's kernels and arguments (damping, smoother): drop them and
// record the iteration graphs again (cycle graphs are recorded at their next use).
int xdg_hier::rerecord() {
  drop_loops();
  omg_drop_graphs();  // recorded OrthoMG passes and GMRES steps hold the old smoothers
  gm_drop();
  TRY(capture(&g_iter, 1, nullptr, nullptr));
  for (int p = 1; p < 3; ++p)
    if (has_lp[p]) TRY(capture(&g_iter_lp[p], 3, nullptr, nullptr, p));
  if (g_cycle) cudaGraphExecDestroy(g_cycle);
  g_cycle = nullptr;
  g_cycle_b = nullptr;
  for (int p = 0; p < 3; ++p) {
    if (g_cyc_lp[p]) cudaGraphExecDestroy(g_cyc_lp[p]);
    g_cyc_lp[p] = nullptr;
    g_cyc_lp_b[p] = nullptr;
    if (lr.g_iter[p]) cudaGraphExecDestroy(lr.g_iter[p]);
    lr.g_iter[p] = nullptr;
  }
  return XDG_OK;
}

// m-step Lanczos for the largest eigenvalue of S M, S the level's Schwarz preconditioner: S M
// is self-adjoint in the M inner product, so the recursion runs in that inner product (one
// product with M and one application of S per step), from the same counter-based start vector
// as the block-Jacobi estimate. Single problems only.
int xdg_hier::lanczos_swz(int l, int m, double* lmax) {
  Level& V = L[l];
  const int64_t n = V.nb * Np;
  double *q = V.b, *qp = V.x, *u = V.t, *w = V.r, *v = V.dz;
  const int vg = vgrid(n);
  double* dv = B.alpha;  // device scratch (free outside solves)
  auto put = [&](double val) -> int {
    h_bsc[0] = val;
    CK(cudaMemcpyAsync(dv, h_bsc, sizeof(double), cudaMemcpyHostToDevice, stream));
    CK(cudaStreamSynchronize(stream));
    return XDG_OK;
  };
  auto get = [&](const double* x, const double* y, double* out) -> int {
    seg_dot(l, x, y, dv);
    return read_scalars(dv, 1, out);
  };
  kl(k_hash_vector_seg, vg, kThreads, 0, stream)(n, 1, V.sdof, q);
  CK(cudaMemsetAsync(qp, 0, n * sizeof(double), stream));
  spmv(l, q, nullptr, u, 0);
  double h = 0.0;
  TRY(get(q, u, &h));
  TRY(put(1.0 / std::sqrt(h)));
  kl(k_seg_scale, vg, kThreads, 0, stream)(n, 1, V.sdof, dv, q);
  kl(k_seg_scale, vg, kThreads, 0, stream)(n, 1, V.sdof, dv, u);
  std::vector<double> al, be;
  double bprev = 0.0;
  for (int j = 0; j < m; ++j) {
    swz_solve<double>(l, u, 1.0, nullptr, w);  // w = S M q
    double a = 0.0;
    TRY(get(u, w, &a));
    al.push_back(a);
    TRY(put(-a));
    kl(k_seg_axpy, vg, kThreads, 0, stream)(n, 1, V.sdof, dv, q, w);
    TRY(put(-bprev));
    kl(k_seg_axpy, vg, kThreads, 0, stream)(n, 1, V.sdof, dv, qp, w);
    spmv(l, w, nullptr, v, 0);
    double b2 = 0.0;
    TRY(get(w, v, &b2));
    CKL();
    const double bj = std::sqrt(std::max(b2, 0.0));
    be.push_back(bj);
    if (!(bj > 1e-300)) break;
    kl(k_copy, vg, kThreads, 0, stream)(n, q, qp);
    kl(k_copy, vg, kThreads, 0, stream)(n, w, q);
    kl(k_copy, vg, kThreads, 0, stream)(n, v, u);
    TRY(put(1.0 / bj));
    kl(k_seg_scale, vg, kThreads, 0, stream)(n, 1, V.sdof, dv, q);
    kl(k_seg_scale, vg, kThreads, 0, stream)(n, 1, V.sdof, dv, u);
    bprev = bj;
  }
  CKL();
  *lmax = tridiag_lambda_max(al, be);
  return XDG_OK;
}

// Install (npatch > 0) or remove (npatch == 0) the additive Schwarz smoother of level l:
// validate the patches, count alpha, find the distinct patch matrices, factor and invert them
// on the device, estimate the damping, record the graphs again.
int xdg_hier::set_schwarz(int l, int64_t npatch, const int64_t* pptr, const int32_t* pblk) {
  Level& V = L[l];
  TRY(sync());
  if ((int)swz.size() < nlev) swz.resize(nlev);
  swz[l].reset();
  if (npatch == 0) {  // back to block Jacobi with its own damping estimate
    TRY(lanczos(l, lanczos_m));
    V.lmax = V.lmax_p[0];
    V.omega = omega_fixed > 0.0 ? omega_fixed : 4.0 / (3.0 * V.lmax);
    V.lmax_p[0] = V.lmax;
    V.omega_p[0] = V.omega;
    return rerecord();
  }
  if (npatch < 0 || !pptr || !pblk || pptr[0] != 0) {
    set_err("xdg_set_schwarz: bad patch arrays");
    return XDG_EINVAL;
  }
  const int64_t nslot = pptr[npatch];
  std::vector<int> cnt(V.nb, 0);
  int maxdof = 0;
  for (int64_t p = 0; p < npatch; ++p) {
    const int64_t k = pptr[p + 1] - pptr[p];
    if (k < 1 || k * Np > swz::kMaxDof) {
      set_err("xdg_set_schwarz: patch %lld has %lld blocks (1..%d allowed for Np = %d)", (long long)p, (long long)k,
              swz::kMaxDof / Np, Np);
      return XDG_EINVAL;
    }
    maxdof = std::max<int>(maxdof, (int)(k * Np));
    for (int64_t q = pptr[p]; q < pptr[p + 1]; ++q) {
      const int32_t b = pblk[q];
      if (b < 0 || b >= V.nb || (q > pptr[p] && b <= pblk[q - 1])) {
        set_err("xdg_set_schwarz: patch %lld: block index %d out of range or not ascending", (long long)p, b);
        return XDG_EINVAL;
      }
      ++cnt[b];
    }
  }
  bool single = true;
  for (int64_t i = 0; i < V.nb; ++i) {
    if (cnt[i] == 0) {
      set_err("xdg_set_schwarz: block %lld is in no patch", (long long)i);
      return XDG_EINVAL;
    }
    single = single && cnt[i] == 1;
  }
  auto S = std::make_unique<SwzLevel>();
  S->npatch = npatch;
  S->nslot = nslot;
  S->maxdof = maxdof;
  S->single = single;
  S->h_pptr.assign(pptr, pptr + npatch + 1);
  S->h_pblk.assign(pblk, pblk + nslot);
  // alpha^{-1/2} per block; slots of every block in ascending patch order
  std::vector<double> isq(V.nb);
  std::vector<float> isq32(V.nb);
  for (int64_t i = 0; i < V.nb; ++i) {
    isq[i] = 1.0 / std::sqrt((double)cnt[i]);
    isq32[i] = (float)isq[i];
  }
  std::vector<int64_t> bsptr(V.nb + 1, 0), bslot(nslot);
  for (int64_t q = 0; q < nslot; ++q) bsptr[pblk[q] + 1]++;
  for (int64_t i = 0; i < V.nb; ++i) bsptr[i + 1] += bsptr[i];
  {
    std::vector<int64_t> pos(bsptr.begin(), bsptr.end() - 1);
    for (int64_t q = 0; q < nslot; ++q) bslot[pos[pblk[q]]++] = q;
  }
  const int64_t n = V.nb * Np;
  TRY(S->alloc(&S->pptr, npatch + 1));
  TRY(S->alloc(&S->pblk, nslot));
  TRY(S->alloc(&S->bsptr, V.nb + 1));
  TRY(S->alloc(&S->bslot, nslot));
  TRY(S->alloc(&S->isq, V.nb));
  TRY(S->alloc(&S->isq32, V.nb));
  TRY(S->alloc(&S->r, n));
  TRY(S->alloc(&S->r32, n));
  if (!single) {
    TRY(S->alloc(&S->y, nslot * Np));
    TRY(S->alloc(&S->y32, nslot * Np));
  }
  CK(cudaMemcpyAsync(S->pptr, pptr, (npatch + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(S->pblk, pblk, nslot * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(S->bsptr, bsptr.data(), (V.nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(S->bslot, bslot.data(), nslot * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(S->isq, isq.data(), V.nb * sizeof(double), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(S->isq32, isq32.data(), V.nb * sizeof(float), cudaMemcpyHostToDevice, stream));
  // distinct patch matrices: two 64-bit hashes and the size per patch
  std::vector<unsigned long long> hh(2 * npatch);
  {
    unsigned long long* dh = nullptr;
    TRY(S->alloc(&dh, 2 * npatch));
    CK(swz::hash(Np, stream, npatch, S->pptr, S->pblk, V.rp, V.col, V.val, dh));
    CK(cudaMemcpyAsync(hh.data(), dh, 2 * npatch * sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream));
    TRY(sync());
  }
  struct Key {
    unsigned long long a, b;
    int64_t n;
    bool operator<(const Key& o) const {
      return a != o.a ? a < o.a : (b != o.b ? b < o.b : n < o.n);
    }
  };
  std::map<Key, int32_t> uniq;
  std::vector<int32_t> tid(npatch);
  std::vector<int64_t> rep, ioff(1, 0);
  for (int64_t p = 0; p < npatch; ++p) {
    const int64_t m = (pptr[p + 1] - pptr[p]) * Np;
    auto it = uniq.emplace(Key{hh[2 * p], hh[2 * p + 1], m}, (int32_t)rep.size());
    if (it.second) {  // every inverse starts 16-byte aligned in FP32 (and FP64): padded to 4 entries
      rep.push_back(p);
      ioff.push_back(ioff.back() + (m * m + 3) / 4 * 4);
    }
    tid[p] = it.first->second;
  }
  const int64_t nu = (int64_t)rep.size();
  S->nuniq = nu;
  S->inv_entries = ioff.back();
  int64_t* drep = nullptr;
  int* derr = nullptr;
  TRY(S->alloc(&S->tid, npatch));
  TRY(S->alloc(&S->ioff, nu + 1));
  TRY(S->alloc(&drep, nu));
  TRY(S->alloc(&S->Ainv, ioff.back()));
  TRY(S->alloc(&S->Ainv32, ioff.back()));
  TRY(S->alloc(&derr, 1));
  CK(cudaMemcpyAsync(S->tid, tid.data(), npatch * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
  {
    // work items: the patches of every stored inverse, in chunks of kItemPatches
    std::vector<int32_t> porder(npatch);
    for (int64_t p = 0; p < npatch; ++p) porder[p] = (int32_t)p;
    std::stable_sort(porder.begin(), porder.end(), [&](int32_t a, int32_t b) { return tid[a] < tid[b]; });
    std::vector<swz::Item> items;
    for (int64_t q = 0; q < npatch;) {
      int64_t e = q;
      while (e < npatch && tid[porder[e]] == tid[porder[q]]) ++e;
      const int m = (int)((pptr[porder[q] + 1] - pptr[porder[q]]) * Np);
      for (int64_t c = q; c < e; c += swz::kItemPatches) {
        const int cnt = (int)std::min<int64_t>(swz::kItemPatches, e - c);
        items.push_back(swz::Item{c, tid[porder[q]], cnt, m, 0});
        if (cnt > 1) S->stage_n = std::max(S->stage_n, m);
      }
      q = e;
    }
    S->nitem = (int64_t)items.size();
    TRY(S->alloc(&S->items, items.size()));
    TRY(S->alloc(&S->porder, npatch));
    CK(cudaMemcpyAsync(S->items, items.data(), items.size() * sizeof(swz::Item), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(S->porder, porder.data(), npatch * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    TRY(sync());  // the host arrays are released at the end of this scope
  }
  CK(swz::prepare(Np));
  CK(cudaMemcpyAsync(S->ioff, ioff.data(), (nu + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(drep, rep.data(), nu * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(derr, 0, sizeof(int), stream));
  // factor and invert in chunks whose gathered matrices fit a bounded work array
  {
    const int64_t budget = std::max<int64_t>(64LL << 20, (int64_t)maxdof * maxdof);  // doubles
    double* work = nullptr;
    int64_t* dwoff = nullptr;
    const int64_t wcap = std::min<int64_t>(budget, ioff.back());
    cudaError_t e = cudaMalloc(&work, std::max<int64_t>(wcap, 1) * sizeof(double));
    if (e != cudaSuccess) {
      set_err("xdg_set_schwarz: work array: %s", cudaGetErrorString(e));
      return XDG_ENOMEM;
    }
    e = cudaMalloc(&dwoff, (nu + 1) * sizeof(int64_t));
    int rc = XDG_OK;
    if (e != cudaSuccess) {
      set_err("xdg_set_schwarz: %s", cudaGetErrorString(e));
      rc = XDG_ENOMEM;
    }
    std::vector<int64_t> woff;
    for (int64_t u0 = 0; rc == XDG_OK && u0 < nu;) {
      woff.assign(1, 0);
      int64_t u1 = u0;
      while (u1 < nu && woff.back() + (ioff[u1 + 1] - ioff[u1]) <= wcap) {
        woff.push_back(woff.back() + (ioff[u1 + 1] - ioff[u1]));
        ++u1;
      }
      e = cudaMemcpyAsync(dwoff, woff.data(), woff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess)
        e = swz::factor(Np, stream, u0, u1, drep, S->pptr, S->pblk, V.rp, V.col, V.val, S->ioff, work, dwoff, S->Ainv,
                        S->Ainv32, derr);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // woff and work are reused
      if (e != cudaSuccess) {
        set_err("xdg_set_schwarz: factorisation: %s", cudaGetErrorString(e));
        rc = XDG_ECUDA;
      }
      u0 = u1;
    }
    cudaFree(work);
    if (dwoff) cudaFree(dwoff);
    TRY(rc);
  }
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, stream));
  TRY(sync());
  if (herr) {
    set_err("xdg_set_schwarz: a patch matrix of level %d is not positive definite", l + 1);
    return XDG_EBREAKDOWN;
  }
  swz[l] = std::move(S);
  // the fused small-level cycle holds block-Jacobi steps: not for levels with Schwarz
  for (int q = 1; q < 3; ++q)
    if (fused_start[q] >= 0 && l >= fused_start[q]) fused_on[q] = false;
  double lm = 0.0;
  int rc = lanczos_swz(l, lanczos_m, &lm);
  if (rc) {
    swz[l].reset();
    return rc;
  }
  V.lmax = lm;
  V.omega = omega_fixed > 0.0 ? omega_fixed : 4.0 / (3.0 * lm);
  if (V.lmax_p.empty()) V.lmax_p.resize(1);
  if (V.omega_p.empty()) V.omega_p.resize(1);
  V.lmax_p[0] = V.lmax;
  V.omega_p[0] = V.omega;
  return rerecord();
}

// work space of the orthonormalisation multigrid: level 1 keeps `restart` directions, the
// coarser levels 3 per pass
int xdg_hier::omg_setup(int restart, int passes) {
  if (restart == omg_restart && passes == omg_passes && !omg.empty()) return XDG_OK;
  TRY(sync());
  omg_drop_graphs();
  omg.assign(nlev, OmgLevel{});
  omg_restart = restart;
  omg_passes = passes;
  for (int l = 0; l < nlev; ++l) {
    OmgLevel& S = omg[l];
    const int64_t n = L[l].nb * Np;
    TRY(alloc(&S.b, n));
    TRY(alloc(&S.x, n));
    if (l == nlev - 1) continue;
    S.cap = (l == 0) ? restart : 3 * passes;
    TRY(alloc(&S.W, (size_t)S.cap * n));
    TRY(alloc(&S.Z, (size_t)S.cap * n));
    TRY(alloc(&S.r, n));
    TRY(alloc(&S.r0, n));
    TRY(alloc(&S.x0, n));
    TRY(alloc(&S.z, n));
    TRY(alloc(&S.sc, 3 + S.cap));
    TRY(alloc(&S.part, (size_t)omg_grid() * S.cap));
    TRY(alloc(&S.rf, n));
    TRY(alloc(&S.zf, n));
  }
  return XDG_OK;
}

int xdg_hier::solve_orthomg(const double* b, double* x, const xdg_orthomg_opts* o, xdg_solve_info* info) {
  auto t0 = clk::now();
  const int restart = std::max(3, o->restart - o->restart % 3);
  const int passes = std::max(1, std::min(4, o->coarse_passes));
  TRY(omg_setup(restart, passes));
  if (omg_f32 != (o->smoother_precision == XDG_PREC_F32)) omg_drop_graphs();
  omg_f32 = o->smoother_precision == XDG_PREC_F32;
  OmgLevel& S = omg[0];
  Level& V = L[0];
  const int64_t n = V.nb * Np;
  const int64_t before = launches;
  double bn2 = 0.0, rn2 = 0.0;
  dot(n, b, b, dsc);
  TRY(read_scalar(dsc, &bn2));
  const double bn = bn2 > 0.0 ? std::sqrt(bn2) : 1.0;
  // (re)start from the current x: x0 := x, r0 := r := b - M x (recomputed), empty space
  auto restart_here = [&]() -> int {
    spmv(0, x, b, S.r0, 1);
    CK(cudaMemcpyAsync(S.r, S.r0, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    CK(cudaMemcpyAsync(S.x0, x, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    S.l = 0;
    return XDG_OK;
  };
  TRY(restart_here());
  dot(n, S.r, S.r, dsc);
  TRY(read_scalar(dsc, &rn2));
  int it = 0;
  if (nlev == 1) {
    coarse(S.r0, S.z);
    kl(k_axpy, vgrid(n), kThreads, 0, stream)(n, 1.0, S.z, x);
    it = 1;
  } else {
    omg_graphs.resize(restart / 3, nullptr);
    for (;;) {
      if (!(std::sqrt(rn2) > o->tol * bn)) {
        // the updated residual meets the tolerance: check the true one; if rounding has moved
        // them apart, restart from x with the true residual
        spmv(0, x, b, S.z, 1);
        dot(n, S.z, S.z, dsc);
        double t2 = 0.0;
        TRY(read_scalar(dsc, &t2));
        if (!(std::sqrt(t2) > o->tol * bn) || !std::isfinite(t2) || it >= o->maxit) break;
        TRY(restart_here());
        rn2 = t2;
      }
      if (it >= o->maxit || !std::isfinite(rn2)) break;
      if (S.l + 3 > S.cap) TRY(restart_here());
      // one pass, recorded once per start column of level 1 (and per x: the graph holds it)
      const int gi = S.l / 3;
      const int l_before = S.l;
      if (!omg_graphs[gi] || omg_graph_x != x) {
        if (omg_graph_x != x) {
          omg_drop_graphs();
          omg_graphs.resize(restart / 3, nullptr);
          omg_graph_x = x;
        }
        cudaGraph_t g = nullptr;
        const int64_t c0 = launches;
        CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        omg_pass(0, x, S.r);
        cudaError_t e = cudaStreamEndCapture(stream, &g);
        if (e != cudaSuccess) {
          set_err("orthomg graph capture: %s", cudaGetErrorString(e));
          return XDG_ECUDA;
        }
        e = cudaGraphInstantiate(&omg_graphs[gi], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          set_err("orthomg graph instantiate: %s", cudaGetErrorString(e));
          return XDG_ECUDA;
        }
        omg_pass_nodes = launches - c0;
      }
      S.l = l_before + 3;
      CK(cudaGraphLaunch(omg_graphs[gi], stream));
      ++it;
      dot(n, S.r, S.r, dsc);
      TRY(read_scalar(dsc, &rn2));
    }
  }
  // final residual recomputed
  spmv(0, x, b, S.z, 1);
  dot(n, S.z, S.z, dsc);
  TRY(read_scalar(dsc, &rn2));
  CKL();
  const double rel = std::sqrt(rn2) / bn;
  int rc = XDG_OK;
  if (!std::isfinite(rel)) rc = XDG_EBREAKDOWN;
  else if (rel > o->tol) rc = XDG_ENOTCONV;
  launches = before;
  if (info) {
    info->iterations = it;
    info->outer = 1;
    info->relres = rel;
    info->status = rc;
    info->ms = ms_since(t0);
    info->launches = (int64_t)it * omg_pass_nodes;
  }
  return rc;
}

// Flexible GMRES(m) (right preconditioning with a preconditioner that may change between
// applications, Saad 1993): Arnoldi with two classical Gram-Schmidt sweeps, Givens rotations and
// the least-squares solve on the device; the residual estimate |g_{j+1}| is read after every
// step; x += Z y at the end of every cycle of m steps.
int xdg_hier::solve_gmres(const double* b, double* x, const xdg_gmres_opts* o, xdg_solve_info* info) {
  auto t0 = clk::now();
  const int m = std::max(1, std::min(o->restart, 200));
  const int kind = o->preconditioner, prec = o->precision;
  Level& V0 = L[0];
  const int64_t n = V0.nb * Np;
  const int vg = vgrid(n), G = std::min(kRedBlocks, sms * 2);
  if (gm.m != m) {  // work space for this restart length
    TRY(sync());
    gm_drop();
    gm = Gmres{};
    gm.m = m;
    TRY(alloc(&gm.V, (size_t)(m + 1) * n));
    TRY(alloc(&gm.Z, (size_t)m * n));
    TRY(alloc(&gm.H, (size_t)(m + 1) * m));
    TRY(alloc(&gm.cs, m));
    TRY(alloc(&gm.sn, m));
    TRY(alloc(&gm.g, m + 1));
    TRY(alloc(&gm.ny, m + 1));
    TRY(alloc(&gm.sc, 4));
    TRY(alloc(&gm.part, (size_t)G * (m + 1)));
  }
  if (gm.prec != prec || gm.kind != kind || (int)gm.step.size() != m) {
    gm_drop();
    gm.step.assign(m, nullptr);
    gm.prec = prec;
    gm.kind = kind;
  }
  const int ld = m + 1;
  const int64_t before = launches;
  int64_t nodes = 0;
  double bn2 = 0.0;
  dot(n, b, b, dsc);
  TRY(read_scalar(dsc, &bn2));
  const double bn = bn2 > 0.0 ? std::sqrt(bn2) : 1.0;
  int it = 0;
  double est = 0.0;
  for (;;) {
    // (re)start: r = b - M x, normalised, is the first Arnoldi vector
    spmv(0, x, b, gm.V, 1);
    dot(n, gm.V, gm.V, gm.sc);
    kry::gmres_start(stream, m, gm.sc, gm.g, gm.sc + 1);
    CK(cudaMemsetAsync(gm.H, 0, (size_t)(m + 1) * m * sizeof(double), stream));
    TRY(read_scalar(gm.g, &est));
    if (!(est > o->tol * bn) || it >= o->maxit || !std::isfinite(est)) break;
    kry::scale(stream, vg, n, gm.sc + 1, gm.V, gm.V);
    int k = 0;
    // step j: z_j = P v_j, w = M z_j orthogonalised against v_0..v_j (H(:, j)), rotation j
    auto step = [&](int j) {
      double* vj = gm.V + (int64_t)j * n;
      double* zj = gm.Z + (int64_t)j * n;
      double* w = gm.V + (int64_t)(j + 1) * n;
      gm_precond(kind, prec, vj, zj);
      spmv(0, zj, nullptr, w, 0);
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice; H(:, j) accumulates
        kry::mdot_partial(stream, G, n, j + 1, gm.V, w, gm.part);
        kry::mdot_final(stream, G, j + 1, gm.part, gm.ny, gm.H + (int64_t)j * ld);
        kry::gs_update(stream, vg, n, j + 1, gm.V, nullptr, gm.ny, w, nullptr);
        launches += 3;
      }
      dot(n, w, w, gm.sc + 2);
      kry::givens(stream, j, ld, gm.H, gm.cs, gm.sn, gm.g, gm.sc + 2);
      kry::normalize(stream, vg, n, gm.sc + 2, gm.sc + 2, w, nullptr, nullptr, nullptr);
      launches += 2;
    };
    for (int j = 0; j < m && it < o->maxit; ++j) {
      if (kind == 1) {  // the p-multigrid's inner solve reads back: launched step by step
        const int64_t c0 = launches;
        pm.last_rc = 0;
        step(j);
        nodes += launches - c0;
        launches = c0;
        if (pm.last_rc) return pm.last_rc;
      } else if (!gm.step[j]) {  // record step j once
        cudaGraph_t g = nullptr;
        const int64_t c0 = launches;
        CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        step(j);
        cudaError_t e = cudaStreamEndCapture(stream, &g);
        if (e != cudaSuccess) {
          set_err("gmres graph capture: %s", cudaGetErrorString(e));
          return XDG_ECUDA;
        }
        e = cudaGraphInstantiate(&gm.step[j], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          set_err("gmres graph instantiate: %s", cudaGetErrorString(e));
          return XDG_ECUDA;
        }
        gm.step_nodes = launches - c0;
        launches = c0;
      }
      if (kind == 0) {
        CK(cudaGraphLaunch(gm.step[j], stream));
        nodes += gm.step_nodes;
      }
      ++it;
      k = j + 1;
      double gj = 0.0;
      TRY(read_scalar(gm.g + j + 1, &gj));
      est = std::fabs(gj);
      if (!(est > o->tol * bn) || !std::isfinite(est)) break;
    }
    // x += Z y, y = H^{-1} g on the k steps made
    kry::gmres_solve(stream, k, ld, gm.H, gm.g, gm.ny);
    kry::gs_update(stream, vg, n, k, gm.Z, nullptr, gm.ny, x, nullptr);
    if (!(est > o->tol * bn) || it >= o->maxit || !std::isfinite(est)) break;
  }
  // final residual recomputed
  spmv(0, x, b, gm.V, 1);
  double rn2 = 0.0;
  dot(n, gm.V, gm.V, dsc);
  TRY(read_scalar(dsc, &rn2));
  CKL();
  const double rel = std::sqrt(rn2) / bn;
  int rc = XDG_OK;
  if (!std::isfinite(rel)) rc = XDG_EBREAKDOWN;
  else if (rel > o->tol) rc = XDG_ENOTCONV;
  const int64_t outside = launches - before;
  launches = before;
  if (info) {
    info->iterations = it;
    info->outer = 1;
    info->relres = rel;
    info->status = rc;
    info->ms = ms_since(t0);
    info->launches = nodes + outside;
  }
  return rc;
}

int xdg_hier::pmg_setup(int n_lo, const xdg_hier_opts* lo_opts, double inner_tol, int inner_maxit, int inner_prec) {
  Ops lops;
  OpsLP lpl;
  if (inner_prec != XDG_PREC_F64 && !ops_lp_for(n_lo, inner_prec, &lpl)) {
    set_err("xdg_pmg_setup: a low-precision inner solve needs n_lo in 6, 10, 15, 20 (n_lo = %d)", n_lo);
    return XDG_EINVAL;
  }
  if (n_lo < 1 || n_lo >= Np || !ops_for(n_lo, &lops) || Np - n_lo > 64) {
    set_err("xdg_pmg_setup: n_lo = %d (Np = %d) not supported (3, 4, 6, 10, 15, 20, 35, below Np and at most 64 "
            "below it)", n_lo, Np);
    return XDG_EINVAL;
  }
  TRY(sync());
  delete pm.lo;
  pm = Pmg{};
  Level& V = L[0];
  const int64_t nb = V.nb;
  const int64_t m2 = (int64_t)n_lo * n_lo;
  // leading n_lo x n_lo parts of the level-1 operator and of every transfer block, to the host
  std::vector<double> hval((size_t)V.nnzb * m2);
  std::vector<std::vector<double>> hR(nlev - 1);
  std::vector<std::vector<int32_t>> hagg(nlev - 1);
  std::vector<int64_t> hnb(nlev);
  {
    int64_t biggest = V.nnzb;
    for (int l = 0; l + 1 < nlev; ++l) biggest = std::max(biggest, L[l].nb);
    double* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, std::max<int64_t>(1, biggest * m2) * sizeof(double));
    if (e != cudaSuccess) {
      set_err("xdg_pmg_setup: %s", cudaGetErrorString(e));
      return XDG_ENOMEM;
    }
    int rc = XDG_OK;
    auto take = [&](int64_t nblk, const double* src, double* dst) {
      cudaError_t ee = pmg::sub_blocks(stream, nblk, Np, n_lo, src, tmp);
      if (ee == cudaSuccess) ee = cudaMemcpyAsync(dst, tmp, nblk * m2 * sizeof(double), cudaMemcpyDeviceToHost, stream);
      if (ee == cudaSuccess) ee = cudaStreamSynchronize(stream);
      if (ee != cudaSuccess) {
        set_err("xdg_pmg_setup: %s", cudaGetErrorString(ee));
        rc = XDG_ECUDA;
      }
    };
    take(V.nnzb, V.val, hval.data());
    for (int l = 0; rc == XDG_OK && l + 1 < nlev; ++l) {
      hR[l].resize((size_t)L[l].nb * m2);
      take(L[l].nb, L[l].R, hR[l].data());
      hagg[l].resize(L[l].nb);
      if (cudaMemcpy(hagg[l].data(), L[l].agg, L[l].nb * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_err("xdg_pmg_setup: copying the aggregation map");
        rc = XDG_ECUDA;
      }
    }
    cudaFree(tmp);
    TRY(rc);
  }
  for (int l = 0; l < nlev; ++l) hnb[l] = L[l].nb;
  std::vector<const int32_t*> aggp(nlev);
  std::vector<const double*> Rp(nlev);
  for (int l = 0; l + 1 < nlev; ++l) {
    aggp[l] = hagg[l].data();
    Rp[l] = hR[l].data();
  }
  xdg_problem q{};
  q.Np = n_lo;
  q.n_levels = nlev;
  q.nb = hnb.data();
  q.row_ptr = V.h_rp.data();
  q.col = V.h_col.data();
  q.val = hval.data();
  q.agg = aggp.data();
  q.R = Rp.data();
  xdg_hier_opts lo{};
  if (lo_opts) lo = *lo_opts;
  else {
    lo.gamma = gamma;
    lo.w_levels = wlev < (1 << 20) ? wlev : 0;
  }
  lo.low_precision = (inner_prec == XDG_PREC_F64) ? 0 : (lo.low_precision | 1);
  auto child = new xdg_hier();
  child->stream = stream;
  child->own_stream = false;
  int rc = child->build(&q, &lo);
  if (rc) {
    delete child;
    return rc;
  }
  pm.lo = child;
  pm.n_lo = n_lo;
  pm.inner = xdg_solve_opts{inner_tol, inner_maxit, 1, inner_prec, 0.0, 0.0};
  const int m = Np - n_lo;
  int* derr = nullptr;
  TRY(alloc(&pm.Hinv, (size_t)nb * m * m));
  TRY(alloc(&pm.blo, (size_t)nb * n_lo));
  TRY(alloc(&pm.xlo, (size_t)nb * n_lo));
  TRY(alloc(&pm.res, (size_t)nb * Np));
  TRY(alloc(&derr, 1));
  CK(cudaMemsetAsync(derr, 0, sizeof(int), stream));
  CK(pmg::hi_inverses(stream, nb, Np, n_lo, V.diag, V.val, pm.Hinv, derr));
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, stream));
  TRY(sync());
  if (herr) {
    set_err("xdg_pmg_setup: a high-order diagonal sub-block is not positive definite");
    delete pm.lo;
    pm.lo = nullptr;
    return XDG_EBREAKDOWN;
  }
  gm_drop();  // recorded GMRES steps may hold the previous preconditioner
  return XDG_OK;
}

static int validate_problem(const xdg_problem& q, int s) {
  const int nl = q.n_levels;
  if (!q.nb || !q.row_ptr || !q.col || !q.val || (nl > 1 && (!q.agg || !q.R))) {
    set_err("problem %d: null arrays", s);
    return XDG_EINVAL;
  }
  if (nl < 1 || nl > XDG_MAX_LEVELS) {
    set_err("problem %d: n_levels = %d outside 1..%d", s, nl, XDG_MAX_LEVELS);
    return XDG_EINVAL;
  }
  for (int l = 0; l < nl; ++l)
    if (q.nb[l] <= 0 || q.nb[l] > INT32_MAX) {
      set_err("problem %d: level %d: nb = %lld", s, l + 1, (long long)q.nb[l]);
      return XDG_EINVAL;
    }
  if (q.row_ptr[0] != 0) {
    set_err("problem %d: row_ptr[0] = %lld", s, (long long)q.row_ptr[0]);
    return XDG_EINVAL;
  }
  for (int64_t i = 0; i < q.nb[0]; ++i) {
    if (q.row_ptr[i + 1] < q.row_ptr[i]) {
      set_err("problem %d: row_ptr decreases at row %lld", s, (long long)i);
      return XDG_EINVAL;
    }
    bool diag = false;
    for (int64_t z = q.row_ptr[i]; z < q.row_ptr[i + 1]; ++z) {
      const int32_t c = q.col[z];
      if (c < 0 || c >= q.nb[0] || (z > q.row_ptr[i] && c <= q.col[z - 1])) {
        set_err("problem %d: col[%lld] = %d out of range or not increasing in row %lld", s, (long long)z, c,
                (long long)i);
        return XDG_EINVAL;
      }
      diag = diag || c == i;
    }
    if (!diag) {
      set_err("problem %d: row %lld has no diagonal block", s, (long long)i);
      return XDG_EINVAL;
    }
  }
  for (int l = 0; l + 1 < nl; ++l) {
    if (!q.agg[l] || !q.R[l]) {
      set_err("problem %d: level %d: null transfer arrays", s, l + 1);
      return XDG_EINVAL;
    }
    std::vector<char> hit(q.nb[l + 1], 0);
    for (int64_t f = 0; f < q.nb[l]; ++f) {
      const int32_t a = q.agg[l][f];
      if (a < 0 || a >= q.nb[l + 1]) {
        set_err("problem %d: level %d: agg[%lld] = %d out of range", s, l + 1, (long long)f, a);
        return XDG_EINVAL;
      }
      hit[a] = 1;
    }
    for (int64_t c = 0; c < q.nb[l + 1]; ++c)
      if (!hit[c]) {
        set_err("problem %d: level %d: coarse block %lld has no child", s, l + 2, (long long)c);
        return XDG_EINVAL;
      }
  }
  return XDG_OK;
}

// Union of n problems with the same block size and depth: level operators, aggregation maps
// and transfers concatenated block-diagonally (problem s's blocks follow problem s-1's on every
// level). The problems must have passed validate_problem, so that the union couples no two
// problems.
int xdg_hier::build_batch(int n, const xdg_problem* probs, const xdg_hier_opts* o) {
  if (n < 1 || n > 65535 || !probs) {
    set_err("batch of %d problems (1..65535 per block size)", n);
    return XDG_EINVAL;
  }
  const int np = probs[0].Np, nl = probs[0].n_levels;
  const int64_t np2 = (int64_t)np * np;
  seg_in.assign(nl, std::vector<int64_t>(1, 0));
  for (int s = 0; s < n; ++s) {
    if (probs[s].Np != np || probs[s].n_levels != nl) {
      set_err("problem %d: Np = %d, n_levels = %d differ from the group's %d, %d", s, probs[s].Np,
              probs[s].n_levels, np, nl);
      return XDG_EINVAL;
    }
    for (int l = 0; l < nl; ++l) seg_in[l].push_back(seg_in[l].back() + probs[s].nb[l]);
  }
  if (seg_in[0].back() > INT32_MAX) {
    set_err("batch exceeds 2^31 blocks on level 1");
    return XDG_EINVAL;
  }
  // concatenation
  std::vector<int64_t> nb(nl), rp(1, 0);
  for (int l = 0; l < nl; ++l) nb[l] = seg_in[l][n];
  int64_t nnz = 0;
  for (int s = 0; s < n; ++s) nnz += probs[s].row_ptr[probs[s].nb[0]];
  std::vector<int32_t> col;
  std::vector<double> val;
  col.reserve(nnz);
  val.reserve(nnz * np2);
  rp.reserve(nb[0] + 1);
  std::vector<std::vector<int32_t>> agg(std::max(nl - 1, 0));
  std::vector<std::vector<double>> R(std::max(nl - 1, 0));
  for (int s = 0; s < n; ++s) {
    const xdg_problem& q = probs[s];
    const int64_t z0 = (int64_t)col.size(), b0 = seg_in[0][s], nz = q.row_ptr[q.nb[0]];
    for (int64_t i = 1; i <= q.nb[0]; ++i) rp.push_back(z0 + q.row_ptr[i]);
    for (int64_t z = 0; z < nz; ++z) col.push_back((int32_t)(b0 + q.col[z]));
    val.insert(val.end(), q.val, q.val + nz * np2);
    for (int l = 0; l + 1 < nl; ++l) {
      const int64_t c0 = seg_in[l + 1][s];
      for (int64_t f = 0; f < q.nb[l]; ++f) agg[l].push_back((int32_t)(c0 + q.agg[l][f]));
      R[l].insert(R[l].end(), q.R[l], q.R[l] + q.nb[l] * np2);
    }
  }
  std::vector<const int32_t*> aggp(std::max(nl - 1, 1), nullptr);
  std::vector<const double*> Rp(std::max(nl - 1, 1), nullptr);
  for (int l = 0; l + 1 < nl; ++l) {
    aggp[l] = agg[l].data();
    Rp[l] = R[l].data();
  }
  xdg_problem u{np, nl, nb.data(), rp.data(), col.data(), val.data(), aggp.data(), Rp.data()};
  return build(&u, o);
}

// One batched CG / flexible-CG step of every problem still running (finished problems take
// zero steps: alpha = 0). The loop condition is set by the convergence check.
void xdg_hier::batch_iteration(int prec, const BatchCtl* ctl, cudaGraphConditionalHandle cond) {
  const int flex = prec != XDG_PREC_F64;
  const int64_t nb1 = L[0].nb;
  if (use_pair(prec)) {  // q = M p from FP32 pairs: split p first (all rows; the product skips finished ones)
    ops.split_df(grid(nb1), stream, nb1, s_p, p2, ex2);
    if (sym_pair)
      ops.spmv_dot_df_sym(grid(nb1), stream, nb1, sy.urp, sy.ucol, sy.uval2, sy.uea, sy.L(), p2, ex2, s_p, s_q,
                          nullptr, act1);
    else
      ops.spmv_dot_df(grid(nb1), stream, nb1, L[0].rp, L[0].col, val2, ea2, p2, ex2, s_p, s_q, nullptr, act1);
    ++launches;
  } else {
    spmv(0, s_p, nullptr, s_q, 0, act1);
  }
  kl(k_chunk_dot<1>, nchunk, kThreads, 0, stream)(nchunk, cb, s_p, s_q, nullptr, nullptr, cpart);
  kl(k_bcg_alpha, sgrid(), 256, 0, stream)(nprob, cfirst, cpart, B);
  kl(k_bcg_xr, nchunk, kThreads, 0, stream)(nchunk, cb, cseg, B.alpha, s_p, s_q, s_x, s_r, cpart);
  kl(k_bcg_check, 1, 1024, 0, stream)(nprob, cfirst, cpart, B, ctl, 1, cond, 1);
  kl(k_bcg_rowact, vgrid(nb1), kThreads, 0, stream)(nb1, Np, nprob, L[0].sdof, B.active, act1);
  launches += 5;
  cur_act = act1;
  precond(prec, s_r, s_z);
  cur_act = nullptr;
  if (flex) kl(k_chunk_dot<2>, nchunk, kThreads, 0, stream)(nchunk, cb, s_r, s_z, s_z, s_q, cpart);
  else kl(k_chunk_dot<1>, nchunk, kThreads, 0, stream)(nchunk, cb, s_r, s_z, nullptr, nullptr, cpart);
  kl(k_bcg_beta, sgrid(), 256, 0, stream)(nprob, nchunk, cfirst, cpart, flex, 0, B);
  kl(k_bcg_p, nchunk, kThreads, 0, stream)(nchunk, cb, cseg, B.beta, 0, s_z, s_p, B.active);
  launches += 3;
}

// Records the whole batched solve into the capture running on `stream`: gather of b and x from
// the caller's vectors, start (r = b - M x, z = B r, p = z), the iteration loop as a
// conditional while node of the graph (its body one batch_iteration; the loop ends when no
// problem is running or after maxit iterations), per-problem results, scatter of x.
int xdg_hier::record_batch(int prec, const BatchCtl* ctl, double* res, int gslot) {
  const int64_t n = L[0].nb * Np;
  const int flex = prec != XDG_PREC_F64;
  const int64_t l0 = launches;
  kl(k_batch_gather, vgrid(n), kThreads, 0, stream)(n, nprob, L[0].sdof, ioff, ctl, s_b, s_x);
  spmv(0, s_x, s_b, s_r, 1);
  kl(k_chunk_dot<2>, nchunk, kThreads, 0, stream)(nchunk, cb, s_r, s_r, s_b, s_b, cpart);
  kl(k_bcg_start, sgrid(), 256, 0, stream)(nprob, nchunk, cfirst, cpart, B);
  launches += 3;
  cudaStreamCaptureStatus st;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(stream, &st, nullptr, &cg, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive) {
    set_err("record_batch: stream is not capturing");
    return XDG_ECUDA;
  }
  cudaGraphConditionalHandle cond;
  CK(cudaGraphConditionalHandleCreate(&cond, cg, 0, cudaGraphCondAssignDefault));
  kl(k_bcg_check, 1, 1024, 0, stream)(nprob, cfirst, nullptr, B, ctl, 0, cond, 1);
  kl(k_bcg_rowact, vgrid(L[0].nb), kThreads, 0, stream)(L[0].nb, Np, nprob, L[0].sdof, B.active, act1);
  launches += 2;
  cur_act = act1;
  precond(prec, s_r, s_z);
  cur_act = nullptr;
  kl(k_chunk_dot<1>, nchunk, kThreads, 0, stream)(nchunk, cb, s_r, s_z, nullptr, nullptr, cpart);
  kl(k_bcg_beta, sgrid(), 256, 0, stream)(nprob, nchunk, cfirst, cpart, flex, 1, B);
  kl(k_bcg_p, nchunk, kThreads, 0, stream)(nchunk, cb, cseg, B.beta, 1, s_z, s_p, B.active);
  launches += 3;
  CKL();
  // the loop
  CK(cudaStreamGetCaptureInfo(stream, &st, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  CK(cudaGraphAddNode(&wnode, cg, deps, nullptr, nd, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamUpdateCaptureDependencies(stream, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  if (!body_stream) CK(cudaStreamCreateWithFlags(&body_stream, cudaStreamNonBlocking));
  CK(cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaStream_t main_stream = stream;
  stream = body_stream;
  const int64_t lb = launches;
  batch_iteration(prec, ctl, cond);
  bnodes_body[prec] = launches - lb;
  stream = main_stream;
  cudaError_t e = cudaGetLastError();
  cudaGraph_t bout = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(body_stream, &bout);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    set_err("record_batch: loop body: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return XDG_ECUDA;
  }
  // results and scatter
  spmv(0, s_x, s_b, s_r, 1);
  kl(k_chunk_dot<1>, nchunk, kThreads, 0, stream)(nchunk, cb, s_r, s_r, nullptr, nullptr, cpart);
  kl(k_bcg_result, sgrid(), 256, 0, stream)(nprob, cfirst, cpart, gidx, B, res, gslot);
  kl(k_batch_scatter, vgrid(n), kThreads, 0, stream)(n, nprob, L[0].sdof, ioff, ctl, s_x);
  launches += 3;
  CKL();
  bnodes_fixed[prec] = launches - l0 - bnodes_body[prec];
  launches = l0;
  return XDG_OK;
}

// The solve's iteration loop as a graph: a conditional while node whose body is one CG /
// flexible-CG iteration (as recorded for the host loop) and the convergence check, which sets
// the loop condition; bounded by the iteration limit.
int xdg_hier::record_loop(int prec) {
  const int li = lr.on ? 1 : 0;
  if (!lctl) {
    TRY(alloc(&lctl, 1));
    CK(cudaMallocHost(&hlctl, sizeof(LoopCtl)));
  }
  if (!body_stream) CK(cudaStreamCreateWithFlags(&body_stream, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
  cudaStreamCaptureStatus st;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaGraphConditionalHandle cond;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t wnode;
  cudaError_t e = cudaStreamGetCaptureInfo(stream, &st, nullptr, &cg, &deps, nullptr, &nd);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, cg, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&wnode, cg, deps, nullptr, nd, &cp);
  }
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(stream, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(body_stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaStream_t main_stream = stream;
    stream = body_stream;
    const int64_t l0 = launches;
    if (prec == XDG_PREC_F64 && !lr.on) pcg_iteration();
    else fcg_iteration(prec);
    kl(k_cg_loop_check, 1, 1, 0, stream)(S, lctl, cond);
    loop_nodes[prec][li] = launches - l0 + 1;
    launches = l0;
    stream = main_stream;
    e = cudaGetLastError();
    cudaGraph_t bout = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(body_stream, &bout);
    if (e == cudaSuccess) e = e2;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(stream, &graph);
  if (e == cudaSuccess) e = e3;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g_loop[prec][li], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    set_err("solve loop graph: %s", cudaGetErrorString(e));
    return XDG_ECUDA;
  }
  return XDG_OK;
}

int xdg_hier::solve_dev(const double* b, double* x, const xdg_solve_opts* o, xdg_solve_info* info) {
  auto t0 = clk::now();
  const int64_t launches0 = launches;
  const int64_t n = L[0].nb * Np;
  const double tol = o ? o->tol : 1e-10;
  const int maxit = o && o->maxit > 0 ? o->maxit : 1000;
  const int every = o && o->check_every > 0 ? o->check_every : 1;
  const double budget = o ? o->time_budget_ms : 0.0;
  const int prec = o ? o->precision : XDG_PREC_F64;
  if (prec != XDG_PREC_F64 && (prec < 0 || prec > 2 || !has_lp[prec])) {
    set_err("precision %d requested but the hierarchy holds no such copy (xdg_hier_opts.low_precision)",
            prec);
    return XDG_EINVAL;
  }
  // FP64: CG with the FP64 cycle. FP32/BF16: flexible CG (FP64 operator, residuals and
  // updates) with the low-precision cycle as preconditioner.
  // with the learned correction the preconditioner is nonlinear: flexible CG in every precision
  if (lr.on && !lr.g_iter[prec]) TRY(capture(&lr.g_iter[prec], 4, nullptr, nullptr, prec));
  cudaGraphExec_t gi = lr.on ? lr.g_iter[prec] : (prec == XDG_PREC_F64) ? g_iter : g_iter_lp[prec];
  const int64_t gi_nodes = lr.on ? lr.nodes[prec] : (prec == XDG_PREC_F64) ? iter_nodes : iter_lp_nodes[prec];
  CK(cudaMemcpyAsync(s_b, b, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  CK(cudaMemcpyAsync(s_x, x, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  CK(cudaMemsetAsync(S, 0, sizeof(PcgScal), stream));
  // r = b - M x, z = B r, p = z, rz = r.z
  spmv(0, s_x, s_b, s_r, 1);
  dot(n, s_b, s_b, dsc);
  dot(n, s_r, s_r, &S->rr);
  precond_full(prec, s_r, s_z);
  if (use_pair(prec)) ops.pcg_p_df(grid(L[0].nb), stream, L[0].nb, S, 1, s_z, s_p, p2, ex2);
  else kl(k_copy, vgrid(n), kThreads, 0, stream)(n, s_z, s_p);
  ++launches;
  dot(n, s_r, s_z, &S->rz);
  CKL();
  double bb;
  TRY(read_scalar(dsc, &bb));
  const double bn = bb > 0 ? std::sqrt(bb) : 1.0;
  CK(cudaMemcpyAsync(hS, S, sizeof(PcgScal), cudaMemcpyDeviceToHost, stream));
  TRY(sync());
  int status = XDG_OK, it = 0;
  double rel = std::sqrt(hS->rr) / bn;
  if (!std::isfinite(rel)) status = XDG_EBREAKDOWN;
  int64_t loop_launches = 0;
  if (status == XDG_OK && rel > tol && budget <= 0 && every == 1) {
    // the whole iteration loop on the device: one graph launch, one read-back
    const int li = lr.on ? 1 : 0;
    if (!g_loop[prec][li]) TRY(record_loop(prec));
    hlctl->tol2 = tol * tol;
    hlctl->bb = bb > 0 ? bb : 1.0;
    hlctl->maxit = maxit;
    hlctl->it = 0;
    CK(cudaMemcpyAsync(lctl, hlctl, sizeof(LoopCtl), cudaMemcpyHostToDevice, stream));
    CK(cudaGraphLaunch(g_loop[prec][li], stream));
    CK(cudaMemcpyAsync(hS, S, sizeof(PcgScal), cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(hlctl, lctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, stream));
    TRY(sync());
    it = hlctl->it;
    loop_launches = (int64_t)it * loop_nodes[prec][li];
    rel = std::sqrt(hS->rr) / bn;
    if (hS->bad || !std::isfinite(rel)) status = XDG_EBREAKDOWN;
    else if (rel > tol) status = XDG_ENOTCONV;
  }
  while (status == XDG_OK && rel > tol) {
    if (it >= maxit) {
      status = XDG_ENOTCONV;
      break;
    }
    int todo = std::min(every, maxit - it);
    for (int k2 = 0; k2 < todo; ++k2) CK(cudaGraphLaunch(gi, stream));
    it += todo;
    CK(cudaMemcpyAsync(hS, S, sizeof(PcgScal), cudaMemcpyDeviceToHost, stream));
    TRY(sync());
    rel = std::sqrt(hS->rr) / bn;
    if (hS->bad || !std::isfinite(rel)) status = XDG_EBREAKDOWN;
    if (budget > 0 && ms_since(t0) > budget && rel > tol) status = XDG_ETIMEOUT;
  }
  if (prec != XDG_PREC_F64 && fused_on[prec]) TRY(fused_error());
  // true residual
  spmv(0, s_x, s_b, s_r, 1);
  dot(n, s_r, s_r, dsc);
  CK(cudaMemcpyAsync(x, s_x, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  double rr;
  TRY(read_scalar(dsc, &rr));
  if (info) {
    info->iterations = it;
    info->outer = 1;
    info->relres = std::sqrt(rr) / bn;
    info->ms = ms_since(t0);
    info->status = status;
    info->launches = launches - launches0 + (loop_launches ? loop_launches : (int64_t)it * gi_nodes);
  }
  if (status) set_err("solve stopped: %s after %d iterations (relres %.3e)", xdg_strerror(status), it,
                      std::sqrt(rr) / bn);
  return status;
}

// ============================================================================================
// Batches: problems grouped by (Np, depth); every group is one block-diagonal union hierarchy.
// One solve is one CUDA graph: the groups' recorded solves run as parallel branches, each with
// its iteration loop as a conditional node, so that the whole batch is a single launch.
struct xdg_batch {
  int n = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<std::unique_ptr<xdg_hier>> grp;
  std::vector<std::vector<int>> members;  // caller indices of every group, in hierarchy order
  std::vector<int64_t> off;               // DOF offset of every problem in the caller's vectors
  BatchCtl* ctl = nullptr;                // device controls
  BatchCtl* hctl = nullptr;               // pinned host mirror
  double* res = nullptr;                  // device results (3 n + groups)
  double* hres = nullptr;                 // pinned host mirror
  double *stage_b = nullptr, *stage_x = nullptr;  // device staging of the host-vector solve
  cudaGraphExec_t gx[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  std::vector<cudaStream_t> gstream;      // capture branch of every group
  std::vector<void*> allocs;
  size_t bytes = 0;
  double setup_ms = 0.0;

  ~xdg_batch() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto& g : gx)
      if (g) cudaGraphExecDestroy(g);
    grp.clear();
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (auto e : ev_join) cudaEventDestroy(e);
    for (auto q : gstream) cudaStreamDestroy(q);
    for (void* p : allocs) cudaFree(p);
    if (hctl) cudaFreeHost(hctl);
    if (hres) cudaFreeHost(hres);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
  template <class T>
  int alloc(T** p, size_t cnt) {
    void* q = nullptr;
    const size_t nbytes = std::max<size_t>(cnt, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, nbytes);
    if (e != cudaSuccess) {
      set_err("cudaMalloc(%zu bytes): %s", nbytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? XDG_ENOMEM : XDG_ECUDA;
    }
    allocs.push_back(q);
    bytes += nbytes;
    *p = static_cast<T*>(q);
    return XDG_OK;
  }

  // record the batched solve of precision prec (all groups) into gx[prec]
  int capture(int prec) {
    CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    int rc = XDG_OK;
    cudaError_t e = cudaEventRecord(ev_fork, stream);
    for (size_t g = 0; g < grp.size() && rc == XDG_OK && e == cudaSuccess; ++g) {
      xdg_hier& H = *grp[g];
      e = cudaStreamWaitEvent(gstream[g], ev_fork, 0);
      if (e != cudaSuccess) break;
      cudaStream_t keep = H.stream;
      H.stream = gstream[g];
      rc = H.record_batch(prec, ctl, res, 3 * n + (int)g);
      H.stream = keep;
      if (rc) break;
      e = cudaEventRecord(ev_join[g], gstream[g]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev_join[g], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(stream, &graph);
    if (rc == XDG_OK && (e != cudaSuccess || e2 != cudaSuccess)) {
      set_err("batch capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
      rc = XDG_ECUDA;
    }
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc;
    }
    if (gx[prec]) cudaGraphExecDestroy(gx[prec]);
    gx[prec] = nullptr;
    e = cudaGraphInstantiate(&gx[prec], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_err("batch graph instantiate: %s", cudaGetErrorString(e));
      return XDG_ECUDA;
    }
    return XDG_OK;
  }

  int solve(const double* b, double* x, const xdg_solve_opts* o, xdg_solve_info* info, xdg_batch_result* out) {
    auto t0 = clk::now();
    const int prec = o ? o->precision : XDG_PREC_F64;
    if (prec < 0 || prec > 2) {
      set_err("precision %d", prec);
      return XDG_EINVAL;
    }
    for (auto& g : grp)
      if (prec != XDG_PREC_F64 && !g->has_lp[prec]) {
        set_err("precision %d requested but the batch holds no such copy (xdg_hier_opts.low_precision)", prec);
        return XDG_EINVAL;
      }
    if (!gx[prec]) TRY(capture(prec));
    const double tol = o ? o->tol : 1e-10;
    hctl->b = b;
    hctl->x = x;
    hctl->tol2 = tol * tol;
    hctl->maxit = o && o->maxit > 0 ? o->maxit : 1000;
    CK(cudaMemcpyAsync(ctl, hctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, stream));
    CK(cudaGraphLaunch(gx[prec], stream));
    CK(cudaMemcpyAsync(hres, res, (3 * (size_t)n + grp.size()) * sizeof(double), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    int worst = XDG_OK, itmax = 0;
    double rmax = 0.0;
    int64_t nodes = 0;
    for (int i = 0; i < n; ++i) {
      const int it = (int)hres[3 * i], st = (int)hres[3 * i + 2];
      const double rr = hres[3 * i + 1];
      if (out) {
        out[i].iterations = it;
        out[i].relres = rr;
        out[i].status = st;
      }
      itmax = std::max(itmax, it);
      rmax = std::max(rmax, rr);
      if (st == XDG_EBREAKDOWN || (st == XDG_ENOTCONV && worst == XDG_OK)) worst = st;
    }
    for (size_t g = 0; g < grp.size(); ++g)
      nodes += grp[g]->bnodes_fixed[prec] + (int64_t)hres[3 * n + g] * grp[g]->bnodes_body[prec];
    if (info) {
      info->iterations = itmax;
      info->outer = 1;
      info->relres = rmax;
      info->ms = ms_since(t0);
      info->status = worst;
      info->launches = nodes;
    }
    if (worst) set_err("batched solve: %s (largest relres %.3e)", xdg_strerror(worst), rmax);
    return worst;
  }
};

// ============================================================================================
// The network of the learned correction: FP32 parameters (trained here), Adam moments, and
// batch work buffers.
struct xdg_mlp {
  MlpDims d{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *P = nullptr, *m1 = nullptr, *m2 = nullptr, *grad = nullptr, *partial = nullptr;
  __nv_bfloat16* Pb = nullptr;
  int nsl = 32;   // sample slices of the gradient reduction
  MlpTrainBuf T{};
  int cap = 0;    // samples the work buffers hold
  int32_t* idx = nullptr;
  int64_t idx_cap = 0;
  double* dloss = nullptr;   // [2]: batch loss, epoch sum
  double* hloss = nullptr;   // pinned
  int64_t step = 0;
  std::vector<void*> tbufs;  // work buffers (reallocated when a larger batch comes)
  std::vector<void*> allocs;

  ~xdg_mlp() {
    if (stream) cudaStreamSynchronize(stream);
    for (void* p : tbufs) cudaFree(p);
    for (void* p : allocs) cudaFree(p);
    if (hloss) cudaFreeHost(hloss);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
  template <class T_>
  int alloc(T_** p, size_t n, std::vector<void*>& list) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T_));
    if (e != cudaSuccess) {
      set_err("cudaMalloc: %s", cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? XDG_ENOMEM : XDG_ECUDA;
    }
    list.push_back(q);
    *p = static_cast<T_*>(q);
    return XDG_OK;
  }
  int ensure_batch(int n) {
    if (n <= cap) return XDG_OK;
    CK(cudaStreamSynchronize(stream));
    for (void* p : tbufs) cudaFree(p);
    tbufs.clear();
    const size_t h = (size_t)n * kHid;
    TRY(alloc(&T.A1, h, tbufs));
    TRY(alloc(&T.A2, h, tbufs));
    TRY(alloc(&T.A3, h, tbufs));
    TRY(alloc(&T.dZ1, h, tbufs));
    TRY(alloc(&T.dZ2, h, tbufs));
    TRY(alloc(&T.dZ3, h, tbufs));
    TRY(alloc(&T.dY, (size_t)n * d.n_out, tbufs));
    TRY(alloc(&T.loss, (size_t)n, tbufs));
    cap = n;
    return XDG_OK;
  }
  int ensure_idx(int64_t n) {
    if (n <= idx_cap) return XDG_OK;
    CK(cudaStreamSynchronize(stream));
    TRY(alloc(&idx, (size_t)n, allocs));
    idx_cap = n;
    return XDG_OK;
  }
  size_t train_smem() const { return (size_t)(d.total + d.n_out * kHid + 2 * kHid * kHid) * sizeof(float); }
  // forward, loss, backward and the gradient of the mean loss of samples idx[0..n) (or 0..n-1)
  int loss_grad(int n, const int32_t* ix, const float* X, const int32_t* uid, const float* Mloc, const float* R,
                const float* C) {
    TRY(ensure_batch(n));
    const size_t sm = train_smem();
    CK(cudaFuncSetAttribute(k_mlp_train_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int blocks = std::max(1, std::min((n + 7) / 8, 152 * 2));
    kl(k_mlp_train_pass, blocks, 256, sm, stream)(n, ix, d, P, X, uid, Mloc, R, C, T);
    dim3 gg((unsigned)((d.total + 255) / 256), (unsigned)nsl);
    kl(k_mlp_grad_partial, gg, 256, 0, stream)(n, nsl, ix, d, X, T, partial);
    kl(k_mlp_grad_final, (d.total + 255) / 256, 256, 0, stream)(d.total, nsl, partial, grad);
    kl(k_sum_ordered, 1, kThreads, 0, stream)(n, T.loss, dloss, 0);
    CKL();
    return XDG_OK;
  }
};

// ============================================================================================
extern "C" {

const char* xdg_strerror(int code) {
  switch (code) {
    case XDG_OK: return "XDG_OK";
    case XDG_EINVAL: return "XDG_EINVAL";
    case XDG_ECUDA: return "XDG_ECUDA";
    case XDG_ENOMEM: return "XDG_ENOMEM";
    case XDG_ENOTCONV: return "XDG_ENOTCONV";
    case XDG_EBREAKDOWN: return "XDG_EBREAKDOWN";
    case XDG_ETIMEOUT: return "XDG_ETIMEOUT";
    default: return "XDG_UNKNOWN";
  }
}

const char* xdg_last_error(void) { return g_last_error.c_str(); }

int xdg_create_hierarchy(const xdg_problem* p, const xdg_hier_opts* o, void* stream, xdg_hier_t* out) {
  if (!p || !out || !p->nb) {
    set_err("null argument");
    return XDG_EINVAL;
  }
  *out = nullptr;
  std::unique_ptr<xdg_hier> h(new xdg_hier());
  h->stream = static_cast<cudaStream_t>(stream);
  int rc = h->build(p, o);
  if (rc) return rc;
  *out = h.release();
  return XDG_OK;
}

int xdg_destroy(xdg_hier_t h) {
  delete h;
  return XDG_OK;
}

int xdg_get_info(xdg_hier_t h, xdg_hier_info* info) {
  if (!h || !info) {
    set_err("null argument");
    return XDG_EINVAL;
  }
  std::memset(info, 0, sizeof(*info));
  info->Np = h->Np;
  info->n_levels = h->nlev;
  for (int l = 0; l < h->nlev; ++l) {
    info->nb[l] = h->L[l].nb;
    info->nnzb[l] = h->L[l].nnzb;
    info->omega[l] = h->L[l].omega;
    info->lambda_max[l] = h->L[l].lmax;
  }
  info->coarse_n = h->nc;
  info->device_bytes = h->bytes;
  for (int i = 0; i < 3; ++i) info->setup_ms[i] = h->setup_ms[i];
  for (int l = 0; l < h->nlev && l < 64; ++l)
    if (h->L[l].spl) info->split_mask |= (uint64_t)1 << l;
  info->fused_level = h->fused_on[1] ? h->fused_start[1] + 1 : (h->fused_on[2] ? h->fused_start[2] + 1 : 0);
  info->fused_cluster = h->fused_on[1] ? h->fused_csize[1] : (h->fused_on[2] ? h->fused_csize[2] : 0);
  info->outer_pair = h->pair_on ? 1 : 0;
  info->symmetric = (h->sym_built ? 1 : 0) | (h->sym_on && !h->L[0].spl ? 2 : 0) | (h->sym_pair ? 4 : 0);
  return XDG_OK;
}

int xdg_export_level(xdg_hier_t h, int level, int64_t* row_ptr, int32_t* col, double* val) {
  if (!h || level < 1 || level > h->nlev) {
    set_err("bad level %d", level);
    return XDG_EINVAL;
  }
  Level& V = h->L[level - 1];
  const int64_t Np2 = (int64_t)h->Np * h->Np;
  if (row_ptr) std::copy(V.h_rp.begin(), V.h_rp.end(), row_ptr);
  if (col) std::copy(V.h_col.begin(), V.h_col.end(), col);
  if (val) {
    cudaError_t e = cudaMemcpyAsync(val, V.val, V.nnzb * Np2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      set_err("export: %s", cudaGetErrorString(e));
      return XDG_ECUDA;
    }
  }
  return XDG_OK;
}

int xdg_apply(xdg_hier_t h, int level, const double* x, double* y, int prec) {
  if (!h || level < 1 || level > h->nlev || !x || !y) {
    set_err("xdg_apply: bad arguments");
    return XDG_EINVAL;
  }
  if (prec == XDG_PREC_F64) {
    h->spmv(level - 1, x, nullptr, y, 0);
  } else if (prec == XDG_PREC_F64_PAIR) {
    if (level != 1 || !h->val2) {
      set_err("xdg_apply: the FP32-pair operator exists on level 1 only, and only when outer_apply != 1 with "
              "low_precision set");
      return XDG_EINVAL;
    }
    Level& V = h->L[0];
    h->ops.split_df(h->grid(V.nb), h->stream, V.nb, x, h->p2, h->ex2);
    h->ops.spmv_dot_df(h->grid(V.nb), h->stream, V.nb, V.rp, V.col, h->val2, h->ea2, h->p2, h->ex2, x, y, nullptr,
                       nullptr);
    h->launches += 2;
  } else {
    if (prec < 0 || prec > 2 || !h->has_lp[prec]) {
      set_err("xdg_apply: precision %d not stored (xdg_hier_opts.low_precision)", prec);
      return XDG_EINVAL;
    }
    Level& V = h->L[level - 1];
    LevelLP& W = h->LP[prec][level - 1];
    // vectors rounded to FP32 once (a per-element FP64 -> FP32 conversion inside the product
    // would run on the FP64 pipe); the level's FP32 work vectors r and dz hold x and y
    const int64_t n = V.nb * h->Np;
    kl(k_d2f, h->vgrid(n), kThreads, 0, h->stream)(n, x, W.r, nullptr, 1);
    h->opl[prec].spmv_f(h->grid_lp(level - 1), V.spl, h->stream, V.nb, V.rp, V.col, W.val, W.sc, W.r, nullptr,
                        W.dz, 0);
    kl(k_f2d, h->vgrid(n), kThreads, 0, h->stream)(n, W.dz, y, nullptr, 1);
    h->launches += 3;
  }
  CKL();
  return XDG_OK;
}

int xdg_set_schwarz(xdg_hier_t h, int level, int64_t n_patches, const int64_t* patch_ptr,
                    const int32_t* patch_blocks) {
  if (!h || level < 1 || level >= h->nlev || n_patches < 0) {
    set_err("xdg_set_schwarz: bad handle, level %d or patch count", level);
    return XDG_EINVAL;
  }
  if (h->nprob != 1) {
    set_err("xdg_set_schwarz: batch groups smooth with block Jacobi only");
    return XDG_EINVAL;
  }
  if (h->Np > 32) {
    set_err("xdg_set_schwarz: Np = %d: the patch solves exist for Np <= 32", h->Np);
    return XDG_EINVAL;
  }
  return h->set_schwarz(level - 1, n_patches, patch_ptr, patch_blocks);
}

int xdg_get_schwarz(xdg_hier_t h, int level, xdg_schwarz_info* info) {
  if (!h || level < 1 || level > h->nlev || !info) {
    set_err("xdg_get_schwarz: bad arguments");
    return XDG_EINVAL;
  }
  std::memset(info, 0, sizeof(*info));
  if (!h->has_swz(level - 1)) return XDG_OK;
  const SwzLevel& S = *h->swz[level - 1];
  info->n_patches = S.npatch;
  info->n_slots = S.nslot;
  info->n_distinct = S.nuniq;
  info->inverse_entries = S.inv_entries;
  info->max_dof = S.maxdof;
  info->overlap = S.single ? 0 : 1;
  info->device_bytes = S.bytes;
  return XDG_OK;
}

int xdg_solve_orthomg(xdg_hier_t h, const double* b, double* x, const xdg_orthomg_opts* o,
                      xdg_solve_info* info) {
  if (!h || !b || !x || !o || !(o->tol >= 0.0) || o->maxit < 0 || o->restart < 3 || o->coarse_passes < 1 ||
      o->coarse_passes > 4) {
    set_err("xdg_solve_orthomg: bad arguments");
    return XDG_EINVAL;
  }
  if (h->nprob != 1) {
    set_err("xdg_solve_orthomg: single problems only");
    return XDG_EINVAL;
  }
  if (o->smoother_precision != XDG_PREC_F64 && o->smoother_precision != XDG_PREC_F32) {
    set_err("xdg_solve_orthomg: smoother_precision must be XDG_PREC_F64 or XDG_PREC_F32");
    return XDG_EINVAL;
  }
  if (o->smoother_precision == XDG_PREC_F32 && !h->has_lp[XDG_PREC_F32]) {
    bool all_swz = true;
    for (int l = 0; l + 1 < h->nlev; ++l) all_swz = all_swz && h->has_swz(l);
    if (!all_swz) {
      set_err("xdg_solve_orthomg: an FP32 block-Jacobi smoother needs the FP32 copies (low_precision)");
      return XDG_EINVAL;
    }
  }
  return h->solve_orthomg(b, x, o, info);
}

int xdg_pmg_setup(xdg_hier_t h, int n_lo, const xdg_hier_opts* lo_opts, double inner_tol, int inner_maxit,
                  int inner_precision) {
  if (!h || !(inner_tol >= 0.0) || inner_maxit < 1 || inner_precision < 0 || inner_precision > 2) {
    set_err("xdg_pmg_setup: bad arguments");
    return XDG_EINVAL;
  }
  if (h->nprob != 1) {
    set_err("xdg_pmg_setup: single problems only");
    return XDG_EINVAL;
  }
  return h->pmg_setup(n_lo, lo_opts, inner_tol, inner_maxit, inner_precision);
}

int xdg_pmg_apply(xdg_hier_t h, const double* r, double* z) {
  if (!h || !r || !z || r == z || !h->pmg_ready()) {
    set_err("xdg_pmg_apply: bad arguments or no p-multigrid set up");
    return XDG_EINVAL;
  }
  h->pm.last_rc = 0;
  h->pmg_apply(r, z);
  CKL();
  TRY(h->sync());
  return h->pm.last_rc;
}

int xdg_solve_gmres(xdg_hier_t h, const double* b, double* x, const xdg_gmres_opts* o, xdg_solve_info* info) {
  if (!h || !b || !x || !o || !(o->tol >= 0.0) || o->maxit < 0 || o->restart < 1 || o->restart > 200 ||
      o->preconditioner < 0 || o->preconditioner > 1 || o->precision < 0 || o->precision > 2) {
    set_err("xdg_solve_gmres: bad arguments");
    return XDG_EINVAL;
  }
  if (h->nprob != 1) {
    set_err("xdg_solve_gmres: single problems only");
    return XDG_EINVAL;
  }
  if (o->preconditioner == 0 && o->precision != XDG_PREC_F64 && !h->has_lp[o->precision]) {
    set_err("xdg_solve_gmres: the hierarchy holds no copy of precision %d", o->precision);
    return XDG_EINVAL;
  }
  if (o->preconditioner == 1 && !h->pmg_ready()) {
    set_err("xdg_solve_gmres: no p-multigrid set up (xdg_pmg_setup)");
    return XDG_EINVAL;
  }
  return h->solve_gmres(b, x, o, info);
}

int xdg_test_barrier_timeout(xdg_hier_t h, int on) {
  if (!h) {
    set_err("xdg_test_barrier_timeout: null handle");
    return XDG_EINVAL;
  }
  bool any = false;
  for (int p = 1; p < 3; ++p) any = any || (h->fused_on[p] && h->fused_csize[p] == 0);
  if (!any) {
    set_err("xdg_test_barrier_timeout: the hierarchy runs no fused small-level cycle with grid barriers");
    return XDG_EINVAL;
  }
  TRY(h->sync());
  h->fused_extra = on ? 1u : 0u;
  for (int p = 1; p < 3; ++p)
    if (h->fused_on[p]) TRY(h->write_fused(p));
  return h->sync();
}

int xdg_residual(xdg_hier_t h, int level, const double* b, const double* x, double* r) {
  if (!h || level < 1 || level > h->nlev || !b || !x || !r || r == x) {
    set_err("xdg_residual: bad arguments");
    return XDG_EINVAL;
  }
  h->spmv(level - 1, x, b, r, 1);
  CKL();
  return XDG_OK;
}

int xdg_get_damping(xdg_hier_t h, int level, int problem, double* omega, double* lambda_max) {
  if (!h || level < 1 || level >= h->nlev || problem < 0 || problem >= h->nprob) {
    set_err("xdg_get_damping: bad level %d or problem %d", level, problem);
    return XDG_EINVAL;
  }
  const Level& V = h->L[level - 1];
  if (omega) *omega = V.omega_p.empty() ? V.omega : V.omega_p[problem];
  if (lambda_max) *lambda_max = V.lmax_p.empty() ? V.lmax : V.lmax_p[problem];
  return XDG_OK;
}

int xdg_set_split(xdg_hier_t h, int level, int on) {
  if (!h || level < 1 || level > h->nlev) {
    set_err("xdg_set_split: bad level %d", level);
    return XDG_EINVAL;
  }
  h->L[level - 1].spl = (on != 0);
  h->tuned = true;
  h->drop_loops();
  for (int p = 1; p < 3; ++p)
    if (h->has_lp[p]) TRY(h->write_fused(p));
  // the recorded low-precision graphs hold the launch shapes: record them again
  for (int p = 1; p < 3; ++p) {
    if (h->has_lp[p]) TRY(h->capture(&h->g_iter_lp[p], 3, nullptr, nullptr, p));
    if (h->g_cyc_lp[p]) cudaGraphExecDestroy(h->g_cyc_lp[p]);
    h->g_cyc_lp[p] = nullptr;
    h->g_cyc_lp_b[p] = nullptr;
  }
  for (int p = 0; p < 3; ++p) {
    if (h->lr.g_iter[p]) cudaGraphExecDestroy(h->lr.g_iter[p]);
    h->lr.g_iter[p] = nullptr;
  }
  return XDG_OK;
}

int xdg_set_damping(xdg_hier_t h, int level, double omega) {
  if (!h || level < 1 || level >= h->nlev || !(omega > 0.0) || !std::isfinite(omega)) {
    set_err("xdg_set_damping: bad level %d or omega %g", level, omega);
    return XDG_EINVAL;
  }
  Level& V = h->L[level - 1];
  V.omega = omega;
  std::fill(V.omega_p.begin(), V.omega_p.end(), omega);
  if (V.omr) {  // batch group: per-row damping of every problem
    std::vector<double> om(V.nb, omega);
    std::vector<float> omf(V.nb, (float)omega);
    CK(cudaMemcpyAsync(V.omr, om.data(), V.nb * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(V.omr_f, omf.data(), V.nb * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  // the recorded graphs hold the damping as a kernel argument: record them again
  return h->rerecord();
}

int xdg_smooth(xdg_hier_t h, int level, const double* b, const double* x_in, double* x_out) {
  if (!h || level < 1 || level >= h->nlev || !b || !x_out || x_out == x_in || x_out == b) {
    set_err("xdg_smooth: bad arguments");
    return XDG_EINVAL;
  }
  h->smooth(level - 1, b, x_in, x_out);
  CKL();
  return XDG_OK;
}

int xdg_restrict(xdg_hier_t h, int level, const double* b, const double* x, double* rc) {
  if (!h || level < 1 || level >= h->nlev || !b || !rc) {
    set_err("xdg_restrict: bad arguments");
    return XDG_EINVAL;
  }
  h->restrict_(level - 1, b, x, rc);
  CKL();
  return XDG_OK;
}

int xdg_prolong(xdg_hier_t h, int level, const double* zc, const double* x_in, double* x_out) {
  if (!h || level < 1 || level >= h->nlev || !zc || !x_in || !x_out) {
    set_err("xdg_prolong: bad arguments");
    return XDG_EINVAL;
  }
  h->prolong(level - 1, zc, x_in, x_out);
  CKL();
  return XDG_OK;
}

int xdg_coarse_solve(xdg_hier_t h, const double* r, double* z) {
  if (!h || !r || !z || r == z) {
    set_err("xdg_coarse_solve: bad arguments");
    return XDG_EINVAL;
  }
  h->coarse(r, z);
  CKL();
  return XDG_OK;
}

int xdg_vcycle(xdg_hier_t h, const double* b, double* x) {
  if (!h || !b || !x || b == x) {
    set_err("xdg_vcycle: bad arguments");
    return XDG_EINVAL;
  }
  if (!h->g_cycle || h->g_cycle_b != b || h->g_cycle_x != x) {
    TRY(h->capture(&h->g_cycle, 0, b, x));
    h->g_cycle_b = b;
    h->g_cycle_x = x;
  }
  CK(cudaGraphLaunch(h->g_cycle, h->stream));
  h->launches += h->cycle_nodes;
  return XDG_OK;
}

int xdg_cycle(xdg_hier_t h, int prec, const double* b, double* x) {
  if (prec == XDG_PREC_F64) return xdg_vcycle(h, b, x);
  if (!h || !b || !x || b == x || prec < 0 || prec > 2 || !h->has_lp[prec]) {
    set_err("xdg_cycle: bad arguments or precision %d not stored", prec);
    return XDG_EINVAL;
  }
  if (!h->g_cyc_lp[prec] || h->g_cyc_lp_b[prec] != b || h->g_cyc_lp_x[prec] != x) {
    TRY(h->capture(&h->g_cyc_lp[prec], 2, b, x, prec));
    h->g_cyc_lp_b[prec] = b;
    h->g_cyc_lp_x[prec] = x;
  }
  CK(cudaGraphLaunch(h->g_cyc_lp[prec], h->stream));
  h->launches += h->cyc_lp_nodes[prec];
  return XDG_OK;
}

int xdg_solve(xdg_hier_t h, const double* b, double* x, const xdg_solve_opts* o, xdg_solve_info* info) {
  if (!h || !b || !x) {
    set_err("xdg_solve: bad arguments");
    return XDG_EINVAL;
  }
  return h->solve_dev(b, x, o, info);
}

int xdg_solve_host(xdg_hier_t h, const double* b_host, double* x_host, const xdg_solve_opts* o,
                   xdg_solve_info* info) {
  if (!h || !b_host || !x_host) {
    set_err("xdg_solve_host: bad arguments");
    return XDG_EINVAL;
  }
  auto t0 = clk::now();
  const int64_t n = h->L[0].nb * h->Np;
  // the level-1 work vectors b, x of the hierarchy serve as device staging
  double* db = h->L[0].r;
  double* dx = h->L[0].dz;
  CK(cudaMemcpyAsync(db, b_host, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(dx, 0, n * sizeof(double), h->stream));
  int rc = h->solve_dev(db, dx, o, info);
  if (rc != XDG_OK && rc != XDG_ENOTCONV && rc != XDG_ETIMEOUT && rc != XDG_EBREAKDOWN) return rc;
  CK(cudaMemcpyAsync(x_host, dx, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (info) info->ms = ms_since(t0);
  return rc;
}

int xdg_create_batch(int n, const xdg_problem* probs, const xdg_hier_opts* o, void* stream, xdg_batch_t* out) {
  if (!out || !probs || n < 1) {
    set_err("xdg_create_batch: bad arguments (n = %d)", n);
    return XDG_EINVAL;
  }
  *out = nullptr;
  auto t0 = clk::now();
  for (int i = 0; i < n; ++i) {  // host only, before any CUDA call
    const int np = probs[i].Np;
    if (np != 6 && np != 10 && np != 15 && np != 20) {
      set_err("problem %d: Np = %d: batches take Np 6, 10, 15 or 20", i, np);
      return XDG_EINVAL;
    }
    TRY(validate_problem(probs[i], i));
  }
  std::unique_ptr<xdg_batch> bt(new xdg_batch());
  bt->n = n;
  bt->stream = static_cast<cudaStream_t>(stream);
  if (!bt->stream) {
    CK(cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking));
    bt->own_stream = true;
  }
  // groups by (Np, depth), in order of first appearance
  std::vector<std::pair<int, int>> key;
  std::vector<int> gof(n);
  bt->off.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    std::pair<int, int> k{probs[i].Np, probs[i].n_levels};
    int g = (int)(std::find(key.begin(), key.end(), k) - key.begin());
    if (g == (int)key.size()) {
      key.push_back(k);
      bt->members.emplace_back();
    }
    gof[i] = g;
    bt->members[g].push_back(i);
    bt->off[i + 1] = bt->off[i] + probs[i].nb[0] * probs[i].Np;
  }
  for (size_t g = 0; g < key.size(); ++g) {
    std::vector<xdg_problem> sub;
    for (int i : bt->members[g]) sub.push_back(probs[i]);
    std::unique_ptr<xdg_hier> h(new xdg_hier());
    h->stream = bt->stream;  // the groups work on the batch's stream (capture branches aside)
    int rc = h->build_batch((int)sub.size(), sub.data(), o);
    if (rc) {
      std::string m = g_last_error;
      set_err("group of Np = %d, %d levels (problems from %d): %s", key[g].first, key[g].second,
              bt->members[g][0], m.c_str());
      return rc;
    }
    // the group's problems in the caller's vectors
    const int P = (int)sub.size();
    std::vector<int64_t> io(P);
    for (int s = 0; s < P; ++s) io[s] = bt->off[bt->members[g][s]];
    CK(cudaMemcpyAsync(h->ioff, io.data(), P * sizeof(int64_t), cudaMemcpyHostToDevice, bt->stream));
    CK(cudaMemcpyAsync(h->gidx, bt->members[g].data(), P * sizeof(int), cudaMemcpyHostToDevice, bt->stream));
    CK(cudaStreamSynchronize(bt->stream));
    bt->bytes += h->bytes;
    bt->grp.push_back(std::move(h));
  }
  TRY(bt->alloc(&bt->ctl, 1));
  TRY(bt->alloc(&bt->res, 3 * (size_t)n + key.size()));
  TRY(bt->alloc(&bt->stage_b, bt->off[n]));
  TRY(bt->alloc(&bt->stage_x, bt->off[n]));
  CK(cudaMallocHost(&bt->hctl, sizeof(BatchCtl)));
  CK(cudaMallocHost(&bt->hres, (3 * (size_t)n + key.size()) * sizeof(double)));
  CK(cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming));
  for (size_t g = 0; g < key.size(); ++g) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    bt->ev_join.push_back(e);
    cudaStream_t q;
    CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
    bt->gstream.push_back(q);
  }
  bt->setup_ms = ms_since(t0);
  *out = bt.release();
  return XDG_OK;
}

int xdg_batch_destroy(xdg_batch_t bt) {
  delete bt;
  return XDG_OK;
}

int xdg_batch_get_info(xdg_batch_t bt, xdg_batch_info* info) {
  if (!bt || !info) {
    set_err("null argument");
    return XDG_EINVAL;
  }
  std::memset(info, 0, sizeof(*info));
  info->n_problems = bt->n;
  info->n_groups = (int)bt->grp.size();
  info->total_dof = bt->off[bt->n];
  info->device_bytes = bt->bytes;
  info->setup_ms = bt->setup_ms;
  for (int p = 0; p < 3; ++p)
    for (auto& g : bt->grp) {
      info->nodes_fixed[p] += g->bnodes_fixed[p];
      info->nodes_per_iteration[p] += g->bnodes_body[p];
    }
  return XDG_OK;
}

int xdg_batch_group(xdg_batch_t bt, int g, xdg_hier_t* h, int* n_members, int* members) {
  if (!bt || g < 0 || g >= (int)bt->grp.size()) {
    set_err("xdg_batch_group: bad group %d", g);
    return XDG_EINVAL;
  }
  if (h) *h = bt->grp[g].get();
  if (n_members) *n_members = (int)bt->members[g].size();
  if (members) std::copy(bt->members[g].begin(), bt->members[g].end(), members);
  return XDG_OK;
}

int xdg_solve_batch(xdg_batch_t bt, const double* b, double* x, const xdg_solve_opts* o, xdg_solve_info* info,
                    xdg_batch_result* results) {
  if (!bt || !b || !x || b == x) {
    set_err("xdg_solve_batch: bad arguments");
    return XDG_EINVAL;
  }
  return bt->solve(b, x, o, info, results);
}

int xdg_solve_batch_host(xdg_batch_t bt, const double* b_host, double* x_host, const xdg_solve_opts* o,
                         xdg_solve_info* info, xdg_batch_result* results) {
  if (!bt || !b_host || !x_host) {
    set_err("xdg_solve_batch_host: bad arguments");
    return XDG_EINVAL;
  }
  auto t0 = clk::now();
  const size_t nbytes = bt->off[bt->n] * sizeof(double);
  CK(cudaMemcpyAsync(bt->stage_b, b_host, nbytes, cudaMemcpyHostToDevice, bt->stream));
  CK(cudaMemsetAsync(bt->stage_x, 0, nbytes, bt->stream));
  int rc = bt->solve(bt->stage_b, bt->stage_x, o, info, results);
  if (rc != XDG_OK && rc != XDG_ENOTCONV && rc != XDG_EBREAKDOWN) return rc;
  CK(cudaMemcpyAsync(x_host, bt->stage_x, nbytes, cudaMemcpyDeviceToHost, bt->stream));
  CK(cudaStreamSynchronize(bt->stream));
  if (info) info->ms = ms_since(t0);
  return rc;
}

// ------------------------------------------------------------------------------ learned
static inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
// uniform in [-1, 1) from a counter
static inline double unit_uniform(uint64_t seed, uint64_t i) {
  return (double)(splitmix64(seed * 0x100000001B3ull + i) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

int xdg_mlp_create(int n_in, int n_out, uint64_t seed, void* stream, xdg_mlp_t* out) {
  if (!out || n_in < 1 || n_in > 64 || n_out < 1 || n_out > 64) {
    set_err("xdg_mlp_create: n_in = %d, n_out = %d (1..64 each)", n_in, n_out);
    return XDG_EINVAL;
  }
  *out = nullptr;
  std::unique_ptr<xdg_mlp> m(new xdg_mlp());
  m->d = mlp_dims(n_in, n_out);
  m->stream = static_cast<cudaStream_t>(stream);
  if (!m->stream) {
    CK(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
    m->own_stream = true;
  }
  const int tot = m->d.total;
  TRY(m->alloc(&m->P, tot, m->allocs));
  TRY(m->alloc(&m->m1, tot, m->allocs));
  TRY(m->alloc(&m->m2, tot, m->allocs));
  TRY(m->alloc(&m->grad, tot, m->allocs));
  TRY(m->alloc(&m->partial, (size_t)m->nsl * tot, m->allocs));
  TRY(m->alloc(&m->Pb, tot, m->allocs));
  TRY(m->alloc(&m->dloss, 2, m->allocs));
  CK(cudaMallocHost(&m->hloss, 2 * sizeof(double)));
  // Glorot-uniform weights from a counter-based generator, zero biases
  std::vector<float> h(tot, 0.0f);
  const int fan[4][2] = {{n_in, kHid}, {kHid, kHid}, {kHid, kHid}, {kHid, n_out}};
  const int off[4] = {m->d.oW1, m->d.oW2, m->d.oW3, m->d.oW4};
  for (int l = 0; l < 4; ++l) {
    const double a = std::sqrt(6.0 / (fan[l][0] + fan[l][1]));
    for (int e = 0; e < fan[l][0] * fan[l][1]; ++e) h[off[l] + e] = (float)(a * unit_uniform(seed, off[l] + e));
  }
  CK(cudaMemcpyAsync(m->P, h.data(), tot * sizeof(float), cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemsetAsync(m->m1, 0, tot * sizeof(float), m->stream));
  CK(cudaMemsetAsync(m->m2, 0, tot * sizeof(float), m->stream));
  CK(cudaStreamSynchronize(m->stream));
  *out = m.release();
  return XDG_OK;
}

int xdg_mlp_destroy(xdg_mlp_t m) {
  delete m;
  return XDG_OK;
}

int xdg_mlp_num_params(xdg_mlp_t m, int64_t* n) {
  if (!m || !n) {
    set_err("null argument");
    return XDG_EINVAL;
  }
  *n = m->d.total;
  return XDG_OK;
}

int xdg_mlp_get_params(xdg_mlp_t m, float* host, int64_t n) {
  if (!m || !host || n != m->d.total) {
    set_err("xdg_mlp_get_params: need %d entries", m ? m->d.total : 0);
    return XDG_EINVAL;
  }
  CK(cudaMemcpyAsync(host, m->P, n * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return XDG_OK;
}

int xdg_mlp_set_params(xdg_mlp_t m, const float* host, int64_t n) {
  if (!m || !host || n != m->d.total) {
    set_err("xdg_mlp_set_params: need %d entries", m ? m->d.total : 0);
    return XDG_EINVAL;
  }
  CK(cudaMemcpyAsync(m->P, host, n * sizeof(float), cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemsetAsync(m->m1, 0, n * sizeof(float), m->stream));
  CK(cudaMemsetAsync(m->m2, 0, n * sizeof(float), m->stream));
  CK(cudaStreamSynchronize(m->stream));
  m->step = 0;
  return XDG_OK;
}

int xdg_mlp_forward(xdg_mlp_t m, int prec, int64_t n, const float* X, float* Y) {
  if (!m || n < 0 || (n > 0 && (!X || !Y)) || (prec != XDG_PREC_F32 && prec != XDG_PREC_BF16)) {
    set_err("xdg_mlp_forward: bad arguments");
    return XDG_EINVAL;
  }
  if (n == 0) return XDG_OK;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 152 * 4));
  if (prec == XDG_PREC_F32) {
    const size_t sm = (size_t)m->d.total * sizeof(float);
    CK(cudaFuncSetAttribute(k_mlp_forward<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    kl(k_mlp_forward<float>, blocks, 256, sm, m->stream)(n, m->d, m->P, X, Y);
  } else {
    kl(k_to_bf16, (m->d.total + 255) / 256, 256, 0, m->stream)(m->d.total, m->P, m->Pb);
    const size_t sm = (size_t)m->d.total * sizeof(__nv_bfloat16);
    CK(cudaFuncSetAttribute(k_mlp_forward<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    kl(k_mlp_forward<__nv_bfloat16>, blocks, 256, sm, m->stream)(n, m->d, m->Pb, X, Y);
  }
  CKL();
  return XDG_OK;
}

int xdg_mlp_loss_grad(xdg_mlp_t m, int n, const float* X, const int32_t* uid, const float* Mloc, const float* R,
                      const float* C, double* loss, float* grad) {
  if (!m || n < 1 || !X || !uid || !Mloc || !R || !C) {
    set_err("xdg_mlp_loss_grad: bad arguments");
    return XDG_EINVAL;
  }
  TRY(m->loss_grad(n, nullptr, X, uid, Mloc, R, C));
  if (grad) CK(cudaMemcpyAsync(grad, m->grad, m->d.total * sizeof(float), cudaMemcpyDeviceToDevice, m->stream));
  CK(cudaMemcpyAsync(m->hloss, m->dloss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  if (loss) *loss = m->hloss[0] / n;
  return XDG_OK;
}

int xdg_mlp_train(xdg_mlp_t m, int n, const float* X, const int32_t* uid, const float* Mloc, const float* R,
                  const float* C, const xdg_train_opts* o, double* loss_per_epoch) {
  if (!m || n < 1 || !X || !uid || !Mloc || !R || !C || !o || o->epochs < 1 || o->batch < 1) {
    set_err("xdg_mlp_train: bad arguments");
    return XDG_EINVAL;
  }
  const int B = std::min(o->batch, n);
  TRY(m->ensure_idx(n));
  TRY(m->ensure_batch(B));
  std::vector<int32_t> perm(n);
  const float b1 = o->beta1 > 0 ? o->beta1 : 0.9f, b2 = o->beta2 > 0 ? o->beta2 : 0.999f;
  const float eps = o->eps > 0 ? o->eps : 1e-8f;
  for (int ep = 0; ep < o->epochs; ++ep) {
    // Fisher-Yates shuffle from a counter-based generator (seed, epoch)
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = n - 1; i > 0; --i) {
      const uint64_t r = splitmix64(o->seed * 0x9E3779B97F4A7C15ull + (uint64_t)ep * 0x100000001ull + i);
      std::swap(perm[i], perm[r % (uint64_t)(i + 1)]);
    }
    CK(cudaMemcpyAsync(m->idx, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, m->stream));
    CK(cudaMemsetAsync(m->dloss + 1, 0, sizeof(double), m->stream));
    for (int s0 = 0; s0 < n; s0 += B) {
      const int nb = std::min(B, n - s0);
      TRY(m->loss_grad(nb, m->idx + s0, X, uid, Mloc, R, C));
      kl(k_sum_ordered, 1, kThreads, 0, m->stream)(nb, m->T.loss, m->dloss + 1, 1);
      m->step += 1;
      const float bc1 = 1.f - std::pow(b1, (float)m->step), bc2 = 1.f - std::pow(b2, (float)m->step);
      kl(k_adam, (m->d.total + 255) / 256, 256, 0, m->stream)(m->d.total, m->P, m->grad, m->m1, m->m2, o->lr, b1, b2,
                                                              eps, bc1, bc2);
    }
    CKL();
    CK(cudaMemcpyAsync(m->hloss, m->dloss, 2 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));  // also keeps perm alive until its copy is done
    if (loss_per_epoch) loss_per_epoch[ep] = m->hloss[1] / n;
  }
  return XDG_OK;
}

int xdg_units_setup(xdg_hier_t h, int n_units, const int32_t* pairs, int n_geo, const float* geom) {
  if (!h || n_units < 1 || !pairs || n_geo < 0 || (n_geo > 0 && !geom) || n_geo + 2 * h->Np > 64) {
    set_err("xdg_units_setup: bad arguments (n_units %d, n_geo %d, Np %d)", n_units, n_geo, h ? h->Np : 0);
    return XDG_EINVAL;
  }
  Learned& U = h->lr;
  if (U.U) {
    set_err("xdg_units_setup: units already set");
    return XDG_EINVAL;
  }
  if (!ops_u_for(h->Np, &U.ops)) {
    set_err("xdg_units_setup: Np = %d not supported", h->Np);
    return XDG_EINVAL;
  }
  Level& V = h->L[0];
  const int Np = h->Np, m = 2 * Np;
  std::vector<int64_t> zi((size_t)n_units * 4, -1);
  auto find = [&](int64_t i, int64_t j) -> int64_t {
    auto b = V.h_col.begin() + V.h_rp[i], e = V.h_col.begin() + V.h_rp[i + 1];
    auto it = std::lower_bound(b, e, (int32_t)j);
    return (it != e && *it == j) ? (int64_t)(it - V.h_col.begin()) : -1;
  };
  std::vector<std::vector<int32_t>> lists(V.nb);
  for (int u = 0; u < n_units; ++u) {
    const int64_t a = pairs[2 * u], b = pairs[2 * u + 1];
    if (a < 0 || a >= V.nb || b < 0 || b >= V.nb || a == b) {
      set_err("xdg_units_setup: unit %d = (%lld, %lld) invalid", u, (long long)a, (long long)b);
      return XDG_EINVAL;
    }
    zi[4 * u] = find(a, a);
    zi[4 * u + 1] = find(a, b);
    zi[4 * u + 2] = find(b, a);
    zi[4 * u + 3] = find(b, b);
    lists[a].push_back(2 * u);
    lists[b].push_back(2 * u + 1);
  }
  std::vector<int32_t> tb, tl;
  std::vector<int64_t> tp(1, 0);
  for (int64_t i = 0; i < V.nb; ++i)
    if (!lists[i].empty()) {
      tb.push_back((int32_t)i);
      tl.insert(tl.end(), lists[i].begin(), lists[i].end());
      tp.push_back((int64_t)tl.size());
    }
  U.U = n_units;
  U.n_geo = n_geo;
  U.nt = (int)tb.size();
  TRY(h->alloc(&U.pairs, 2 * (size_t)n_units));
  TRY(h->alloc(&U.geom, (size_t)n_units * std::max(n_geo, 1)));
  TRY(h->alloc(&U.zidx, 4 * (size_t)n_units));
  TRY(h->alloc(&U.Linv, (size_t)n_units * 2 * Np * Np));
  TRY(h->alloc(&U.Hm, (size_t)n_units * m * m));
  TRY(h->alloc(&U.Mloc, (size_t)n_units * m * m));
  TRY(h->alloc(&U.Minv, (size_t)n_units * m * m));
  TRY(h->alloc(&U.tblk, tb.size()));
  TRY(h->alloc(&U.tptr, tp.size()));
  TRY(h->alloc(&U.tlist, tl.size()));
  TRY(h->alloc(&U.res, V.nb * (size_t)Np));
  TRY(h->alloc(&U.delta, (size_t)n_units * m));
  TRY(h->alloc(&U.E, (size_t)n_units));
  TRY(h->alloc(&U.keep, (size_t)n_units));
  cudaStream_t st = h->stream;
  CK(cudaMemcpyAsync(U.pairs, pairs, 2 * (size_t)n_units * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (n_geo > 0)
    CK(cudaMemcpyAsync(U.geom, geom, (size_t)n_units * n_geo * sizeof(float), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(U.zidx, zi.data(), zi.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(U.tblk, tb.data(), tb.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(U.tptr, tp.data(), tp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(U.tlist, tl.data(), tl.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(U.res, 0, V.nb * (size_t)Np * sizeof(double), st));
  int* derr = nullptr;
  TRY(h->alloc(&derr, 1));
  CK(cudaMemsetAsync(derr, 0, sizeof(int), st));
  U.ops.factor(st, n_units, U.zidx, V.val, U.Linv, U.Hm, U.Mloc, U.Minv, derr);
  CKL();
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr) {
    set_err("xdg_units_setup: a unit matrix is not positive definite");
    return XDG_EBREAKDOWN;
  }
  return XDG_OK;
}

int xdg_units_local(xdg_hier_t h, float* Mloc) {
  if (!h || !h->lr.U || !Mloc) {
    set_err("xdg_units_local: no units or null output");
    return XDG_EINVAL;
  }
  const size_t m = 2 * (size_t)h->Np;
  CK(cudaMemcpyAsync(Mloc, h->lr.Mloc, h->lr.U * m * m * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  return XDG_OK;
}

int xdg_units_samples(xdg_hier_t h, int prec, const double* r, float* X, float* R, float* C) {
  if (!h || !h->lr.U || !r || !X || !R || !C || prec < 0 || prec > 2 ||
      (prec != XDG_PREC_F64 && !h->has_lp[prec])) {
    set_err("xdg_units_samples: bad arguments, no units or precision %d not stored", prec);
    return XDG_EINVAL;
  }
  Learned& U = h->lr;
  Level& V = h->L[0];
  // z = B r with the plain cycle, then the residual r - M z on the units' rows
  double* z = h->s_q;  // solve work vector, free outside a solve
  if (prec == XDG_PREC_F64) h->cycle(0, r, z);
  else h->cycle_lp_d(prec, r, z);
  U.ops.resid_rows(h->grid(U.nt), h->stream, U.nt, U.tblk, V.rp, V.col, V.val, z, r, U.res);
  U.ops.samples(h->stream, U.U, U.n_geo, U.pairs, U.geom, U.res, U.Linv, U.Minv, X, R, C);
  h->launches += 2;
  CKL();
  return XDG_OK;
}

int xdg_learned_enable(xdg_hier_t h, xdg_mlp_t m, double theta) {
  if (!h) {
    set_err("null hierarchy");
    return XDG_EINVAL;
  }
  Learned& U = h->lr;
  h->drop_loops();
  for (int p = 0; p < 3; ++p)
    if (U.g_iter[p]) {
      cudaGraphExecDestroy(U.g_iter[p]);
      U.g_iter[p] = nullptr;
    }
  if (!m) {
    U.on = false;
    return XDG_OK;
  }
  if (!U.U || m->d.n_in != U.n_geo + 2 * h->Np || m->d.n_out != 2 * h->Np || !(theta > 0.0)) {
    set_err("xdg_learned_enable: network %d -> %d does not fit units of %d features, Np %d (or theta <= 0)",
            m->d.n_in, m->d.n_out, U.n_geo, h->Np);
    return XDG_EINVAL;
  }
  if (U.wcap < m->d.total) {
    TRY(h->alloc(&U.W, m->d.total));
    U.wcap = m->d.total;
  }
  CK(cudaStreamSynchronize(m->stream));
  kl(k_to_bf16, (m->d.total + 255) / 256, 256, 0, h->stream)(m->d.total, m->P, U.W);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  U.d = m->d;
  U.theta = theta;
  U.on = true;
  return XDG_OK;
}

int xdg_learned_step(xdg_hier_t h, const double* r, double* z, int* n_kept) {
  if (!h || !h->lr.on || !r || !z) {
    set_err("xdg_learned_step: learned correction not enabled or null vectors");
    return XDG_EINVAL;
  }
  h->learned_apply(r, z);
  CKL();
  if (n_kept) {
    std::vector<int> k(h->lr.U);
    CK(cudaMemcpyAsync(k.data(), h->lr.keep, h->lr.U * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int c = 0;
    for (int v : k) c += v;
    *n_kept = c;
  }
  return XDG_OK;
}

}  // extern "C"

// ============================================================================================
// Residual restriction without allocations (see xdg_restrict_noalloc in include/xdg.h).
// The scratch lives in a file-scope device array; host code only ever sees its host-side
// stand-in symbol, so the device address is looked up once per device and passed to the
// kernels.
static __device__ __align__(256) double g_noalloc_scratch[XDG_NOALLOC_MAX_ENTRIES];

namespace {
struct NoallocDev {
  bool ready = false;
  double* scratch = nullptr;
  int sms = 0;
};
std::mutex g_noalloc_mu;
NoallocDev g_noalloc_dev[128];
}  // namespace

extern "C" int xdg_restrict_noalloc(int Np, int64_t nb_fine, int64_t nb_coarse, const int64_t* row_ptr,
                                    const int32_t* col, const double* val, const double* R,
                                    const int64_t* child_ptr, const int32_t* child, const double* b,
                                    const double* x, double* rc, void* stream) {
  Ops ops;
  if (!ops_for(Np, &ops)) {
    set_err("xdg_restrict_noalloc: block size Np = %d not supported (3, 4, 6, 10, 15, 20, 35, 56)", Np);
    return XDG_EINVAL;
  }
  if (nb_fine <= 0 || nb_coarse <= 0 || !row_ptr || !col || !val || !R || !child_ptr || !child || !b || !rc) {
    set_err("xdg_restrict_noalloc: empty level or null pointer");
    return XDG_EINVAL;
  }
  if (nb_fine > XDG_NOALLOC_MAX_ENTRIES / Np) {
    set_err("xdg_restrict_noalloc: nb_fine*Np = %lld exceeds the fixed scratch of %d entries",
            (long long)nb_fine * Np, XDG_NOALLOC_MAX_ENTRIES);
    return XDG_EINVAL;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) {
    set_err("xdg_restrict_noalloc: device ordinal %d out of range", dev);
    return XDG_EINVAL;
  }
  NoallocDev st;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocDev& d = g_noalloc_dev[dev];
    if (!d.ready) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        set_err("xdg_restrict_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return XDG_ECUDA;
      }
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) {
        set_err("xdg_restrict_noalloc: %s", cudaGetErrorString(e));
        return XDG_ECUDA;
      }
      d.scratch = static_cast<double*>(p);
      d.sms = sms;
      d.ready = true;
    }
    st = d;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto grid_rows = [&](int64_t rows) {
    int64_t warps = (rows + ops.gpw - 1) / ops.gpw;
    int64_t blocks = (warps + (kThreads / 32) - 1) / (kThreads / 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)st.sms * 8));
  };
  auto grid_vec = [&](int64_t n) {
    int64_t blocks = (n + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)st.sms * 8));
  };
  ops.resid_rt(grid_rows(nb_fine), s, nb_fine, row_ptr, col, val, R, b, x, st.scratch);
  ops.gather(grid_vec(nb_coarse * Np), s, nb_coarse, child_ptr, child, st.scratch, rc);
  CKL();
  return XDG_OK;
}

// ============================================================================================
// FMA throughput probe (benchmark utility)
namespace {
template <class T>
__global__ void k_fma_probe(T* out, int iters) {
  T a0 = threadIdx.x * (T)1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
    a7 = a0 + 7;
  const T m = (T)0.9999999, c = (T)1e-7;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
  }
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

template <class T>
int fma_probe(int iters, double* tflops) {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  T* d = nullptr;
  CK(cudaMalloc(&d, sizeof(T) * (size_t)blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_probe<T><<<blocks, threads>>>(d, 64);
  cudaEventRecord(e0);
  k_fma_probe<T><<<blocks, threads>>>(d, iters);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_err("fma probe: %s", cudaGetErrorString(e));
    return XDG_ECUDA;
  }
  *tflops = 2.0 * 8.0 * blocks * threads * (double)iters / (ms * 1e-3) / 1e12;
  return XDG_OK;
}
}  // namespace

extern "C" int xdg_kernel_time(xdg_hier_t h, int which, int level, int prec, int reps, double* ms,
                               double* bytes) {
  const bool pair = prec == XDG_PREC_F64_PAIR;
  if (!h || level < 1 || level > h->nlev || which < 0 || which > 2 || (which > 0 && level >= h->nlev) ||
      prec < 0 || prec > 3 || (pair && (which != 0 || level != 1 || !h->val2)) ||
      (!pair && prec != XDG_PREC_F64 && !h->has_lp[prec])) {
    set_err("xdg_kernel_time: bad kernel %d, level %d or precision %d", which, level, prec);
    return XDG_EINVAL;
  }
  const int l = level - 1;
  Level& V = h->L[l];
  const int Np = h->Np;
  const int64_t n = V.nb * Np, np2 = (int64_t)Np * Np;
  cudaStream_t st = h->stream;
  const bool lp = prec != XDG_PREC_F64 && !pair;
  const double sv = lp ? 4.0 : 8.0;                        // vector entries
  const double sa = prec == XDG_PREC_F64 ? 8.0 : 4.0;      // operator read by smooth / restrict
  const double sap = prec == XDG_PREC_BF16 ? 2.0 : sa;     // operator read by apply
  const double sr = prec == XDG_PREC_BF16 ? 2.0 : sa;      // transfer blocks
  const double scal = lp ? 4.0 : 0.0;                      // per-block scales
  const double rows = 8.0 * (V.nb + 1) + 4.0 * V.nnzb;     // row pointer and columns
  // symmetric storage of level 1: compact row pointer and columns, left-block lists
  const xdg_hier::SymLevel& sy = h->sy;
  const double srows = 16.0 * (V.nb + 1) + 4.0 * sy.nu + 8.0 * sy.nl;
  const bool sym = lp && h->lvl1_sym(l) && which > 0;
  double by = 0.0;
  std::function<void()> launch;
  if (pair) {
    CK(cudaMemsetAsync(V.x, 0, n * sizeof(double), st));
    h->ops.split_df(h->grid(V.nb), st, V.nb, V.x, h->p2, h->ex2);
    // pairs (8 bytes) and an exponent per block; the split vector and its exponents; y in FP64
    if (h->sym_pair) {
      launch = [&]() {
        h->ops.spmv_dot_df_sym(h->grid(V.nb), st, V.nb, sy.urp, sy.ucol, sy.uval2, sy.uea, sy.L(), h->p2, h->ex2, V.x,
                               V.t, nullptr, nullptr);
      };
      by = srows + sy.nu * (np2 * 8.0 + 4.0) + n * 8.0 + V.nb * 4.0 + n * 8.0;
    } else {
      launch = [&]() {
        h->ops.spmv_dot_df(h->grid(V.nb), st, V.nb, V.rp, V.col, h->val2, h->ea2, h->p2, h->ex2, V.x, V.t, nullptr,
                           nullptr);
      };
      by = rows + V.nnzb * (np2 * 8.0 + 4.0) + n * 8.0 + V.nb * 4.0 + n * 8.0;
    }
  } else if (!lp) {
    CK(cudaMemsetAsync(V.b, 0, n * sizeof(double), st));
    CK(cudaMemsetAsync(V.x, 0, n * sizeof(double), st));
    if (which == 0) {
      launch = [&]() { h->ops.spmv(h->grid(V.nb), st, nullptr, V.nb, V.rp, V.col, V.val, V.x, nullptr, V.t, 0); };
      by = rows + V.nnzb * np2 * 8.0 + 2.0 * n * 8.0;
    } else if (which == 1) {
      launch = [&]() {
        h->ops.smooth(h->grid(V.nb), st, V.nb, V.rp, V.col, V.val, V.Dinv, V.omega, V.omr, V.b, V.x, V.t);
      };
      by = rows + V.nnzb * np2 * 8.0 + V.nb * np2 * 8.0 + 3.0 * n * 8.0;
    } else {
      launch = [&]() { h->ops.resid_rt(h->grid(V.nb), st, V.nb, V.rp, V.col, V.val, V.R, V.b, V.x, V.s); };
      by = rows + V.nnzb * np2 * 8.0 + V.nb * np2 * 8.0 + 3.0 * n * 8.0;
    }
  } else {
    LevelLP& W = h->LP[prec][l];
    const OpsLP& o = h->opl[prec];
    CK(cudaMemsetAsync(W.b, 0, n * sizeof(float), st));
    CK(cudaMemsetAsync(W.x, 0, n * sizeof(float), st));
    if (which == 0) {
      launch = [&]() {
        o.spmv_f(h->grid_lp(l), V.spl, st, V.nb, V.rp, V.col, W.val, W.sc, W.x, nullptr, W.t, 0);
      };
      by = rows + V.nnzb * (np2 * sap + scal) + 2.0 * n * sv;
    } else if (which == 1) {
      if (sym)
        launch = [&]() {
          o.smooth_sym(h->grid_lp(l), st, V.nb, sy.urp, sy.ucol, sy.uval, sy.usc, sy.L(), (const float*)W.Dinv, W.dsc,
                       (float)V.omega, V.omr_f, W.b, W.x, W.t, nullptr);
        };
      else
        launch = [&]() {
          o.smooth(h->grid_lp(l), V.spl, st, V.nb, V.rp, V.col, W.val32, W.sc32, W.Dinv, W.dsc, (float)V.omega,
                   V.omr_f, W.b, W.x, W.t, nullptr);
        };
      by = (sym ? srows + sy.nu * (np2 * 4.0 + scal) : rows + V.nnzb * (np2 * sa + scal)) +
           V.nb * (np2 * 4.0 + scal) + 3.0 * n * sv;
    } else {
      if (sym)
        launch = [&]() {
          o.resid_rt_sym(h->grid_lp(l), st, V.nb, sy.urp, sy.ucol, sy.uval, sy.usc, sy.L(), W.R, W.rsc, W.b, W.x, W.s,
                         nullptr);
        };
      else
        launch = [&]() {
          o.resid_rt(h->grid_lp(l), V.spl, st, V.nb, V.rp, V.col, W.val32, W.sc32, W.R, W.rsc, W.b, W.x, W.s,
                     nullptr);
        };
      by = (sym ? srows + sy.nu * (np2 * 4.0 + scal) : rows + V.nnzb * (np2 * sa + scal)) +
           V.nb * (np2 * sr + scal) + 3.0 * n * sv;
    }
  }
  const int R = reps > 0 ? reps : 20;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int k = 0; k < 3; ++k) launch();
  cudaEventRecord(e0, st);
  for (int k = 0; k < R; ++k) launch();
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_err("xdg_kernel_time: %s", cudaGetErrorString(e));
    return XDG_ECUDA;
  }
  if (ms) *ms = t / R;
  if (bytes) *bytes = by;
  return XDG_OK;
}

extern "C" int xdg_fma_peak(int prec, double* tflops) {
  if (!tflops) {
    set_err("xdg_fma_peak: null output");
    return XDG_EINVAL;
  }
  if (prec == XDG_PREC_F64) return fma_probe<double>(4096, tflops);
  if (prec == XDG_PREC_F32) return fma_probe<float>(65536, tflops);
  set_err("xdg_fma_peak: precision %d not probed", prec);
  return XDG_EINVAL;
}
