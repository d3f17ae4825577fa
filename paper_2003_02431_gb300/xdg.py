"""Thin ctypes binding of libxdg (include/xdg.h): argument marshalling only.

Every computation runs in the CUDA kernels of libxdg.so. Device vectors are torch CUDA
tensors (float64, contiguous) passed by data pointer; host vectors are numpy float64 arrays.
If libxdg.so cannot be loaded this module raises; it has no CPU fallback.

Entry points mirror the C names: create_hierarchy / destroy / get_info / export_level /
apply / smooth / restrict / prolong / coarse_solve / vcycle / solve / solve_host.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
LIB_PATH = os.path.join(_HERE, "libxdg.so")
_CSRC = os.path.join(_HERE, "csrc")
# translation units of libxdg (compiled in parallel, then linked) and every file they include
_UNITS = [os.path.join(_CSRC, "xdg.cu"), os.path.join(_CSRC, "xdg_swz.cu"), os.path.join(_CSRC, "xdg_krylov.cu"),
          os.path.join(_CSRC, "xdg_big.cu")]
_SRCS = _UNITS + [os.path.join(_CSRC, f) for f in sorted(os.listdir(_CSRC)) if f.endswith((".cuh", ".h"))] + [
    os.path.join(_ROOT, "include", "xdg.h")]

XDG_OK, XDG_EINVAL, XDG_ECUDA, XDG_ENOMEM, XDG_ENOTCONV, XDG_EBREAKDOWN, XDG_ETIMEOUT = range(7)
XDG_PREC_F64, XDG_PREC_F32, XDG_PREC_BF16, XDG_PREC_F64_PAIR = 0, 1, 2, 3
MAX_LEVELS = 24

NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC"]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libxdg.so in-tree for sm_103a with nvcc (cross-compiles without a GPU): every
    translation unit to an object file in parallel, then one shared library."""
    from concurrent.futures import ThreadPoolExecutor
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    nvcc = os.environ.get("NVCC", "nvcc")
    bdir = os.path.join(_HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    tag = "%d" % os.getpid()

    def compile_unit(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".%s.o" % tag)
        cmd = [nvcc] + NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-c", "-o", obj, src]
        subprocess.run(cmd, check=True)
        return obj

    with ThreadPoolExecutor(len(_UNITS)) as ex:
        objs = list(ex.map(compile_unit, _UNITS))
    tmp = LIB_PATH + ".tmp%s" % tag
    subprocess.run([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs, check=True)
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class XdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_NAMES.get(code, "XDG_%d" % code), msg))
        self.code = code


_NAMES = {0: "XDG_OK", 1: "XDG_EINVAL", 2: "XDG_ECUDA", 3: "XDG_ENOMEM", 4: "XDG_ENOTCONV",
          5: "XDG_EBREAKDOWN", 6: "XDG_ETIMEOUT"}


class Problem(C.Structure):
    _fields_ = [("Np", C.c_int), ("n_levels", C.c_int), ("nb", C.POINTER(C.c_int64)),
                ("row_ptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32)),
                ("val", C.POINTER(C.c_double)), ("agg", C.POINTER(C.POINTER(C.c_int32))),
                ("R", C.POINTER(C.POINTER(C.c_double)))]


class HierOpts(C.Structure):
    _fields_ = [("omega", C.c_double), ("lanczos_steps", C.c_int), ("nu", C.c_int),
                ("gamma", C.c_int), ("low_precision", C.c_int), ("w_levels", C.c_int), ("split_rows", C.c_int),
                ("fused_coarse", C.c_int), ("outer_apply", C.c_int), ("symmetric", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("check_every", C.c_int),
                ("precision", C.c_int), ("inner_tol", C.c_double), ("time_budget_ms", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer", C.c_int), ("relres", C.c_double),
                ("ms", C.c_double), ("status", C.c_int), ("launches", C.c_int64)]


class HierInfo(C.Structure):
    _fields_ = [("Np", C.c_int), ("n_levels", C.c_int), ("nb", C.c_int64 * MAX_LEVELS),
                ("nnzb", C.c_int64 * MAX_LEVELS), ("omega", C.c_double * MAX_LEVELS),
                ("lambda_max", C.c_double * MAX_LEVELS), ("coarse_n", C.c_int64),
                ("device_bytes", C.c_size_t), ("setup_ms", C.c_double * 3), ("split_mask", C.c_uint64),
                ("fused_level", C.c_int), ("outer_pair", C.c_int), ("symmetric", C.c_int),
                ("fused_cluster", C.c_int)]


class TrainOpts(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64)]


class BatchResult(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("relres", C.c_double)]


class BatchInfo(C.Structure):
    _fields_ = [("n_problems", C.c_int), ("n_groups", C.c_int), ("total_dof", C.c_int64),
                ("device_bytes", C.c_size_t), ("setup_ms", C.c_double),
                ("nodes_fixed", C.c_int64 * 3), ("nodes_per_iteration", C.c_int64 * 3)]


# (name, restype, argtypes) of every exported entry point
_vp, _dp, _ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
class SchwarzInfo(C.Structure):
    _fields_ = [("n_patches", C.c_int64), ("n_slots", C.c_int64), ("n_distinct", C.c_int64),
                ("inverse_entries", C.c_int64), ("max_dof", C.c_int), ("overlap", C.c_int),
                ("device_bytes", C.c_size_t)]


class OrthoMGOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("restart", C.c_int), ("coarse_passes", C.c_int),
                ("smoother_precision", C.c_int)]


class GmresOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("restart", C.c_int), ("preconditioner", C.c_int),
                ("precision", C.c_int)]


SIGNATURES = [
    ("xdg_create_hierarchy", C.c_int, [C.POINTER(Problem), C.POINTER(HierOpts), _vp, C.POINTER(_vp)]),
    ("xdg_destroy", C.c_int, [_vp]),
    ("xdg_set_schwarz", C.c_int, [_vp, _ip, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    ("xdg_get_schwarz", C.c_int, [_vp, _ip, C.POINTER(SchwarzInfo)]),
    ("xdg_solve_orthomg", C.c_int, [_vp, _vp, _vp, C.POINTER(OrthoMGOpts), C.POINTER(SolveInfo)]),
    ("xdg_pmg_setup", C.c_int, [_vp, _ip, C.POINTER(HierOpts), C.c_double, _ip, _ip]),
    ("xdg_pmg_apply", C.c_int, [_vp, _vp, _vp]),
    ("xdg_solve_gmres", C.c_int, [_vp, _vp, _vp, C.POINTER(GmresOpts), C.POINTER(SolveInfo)]),
    ("xdg_residual", C.c_int, [_vp, _ip, _vp, _vp, _vp]),
    ("xdg_test_barrier_timeout", C.c_int, [_vp, _ip]),
    ("xdg_strerror", C.c_char_p, [_ip]),
    ("xdg_last_error", C.c_char_p, []),
    ("xdg_get_info", C.c_int, [_vp, C.POINTER(HierInfo)]),
    ("xdg_export_level", C.c_int, [_vp, _ip, C.POINTER(C.c_int64), C.POINTER(C.c_int32), _dp]),
    ("xdg_apply", C.c_int, [_vp, _ip, _vp, _vp, _ip]),
    ("xdg_smooth", C.c_int, [_vp, _ip, _vp, _vp, _vp]),
    ("xdg_set_damping", C.c_int, [_vp, _ip, C.c_double]),
    ("xdg_set_split", C.c_int, [_vp, _ip, _ip]),
    ("xdg_get_damping", C.c_int, [_vp, _ip, _ip, _dp, _dp]),
    ("xdg_restrict", C.c_int, [_vp, _ip, _vp, _vp, _vp]),
    ("xdg_prolong", C.c_int, [_vp, _ip, _vp, _vp, _vp]),
    ("xdg_coarse_solve", C.c_int, [_vp, _vp, _vp]),
    ("xdg_vcycle", C.c_int, [_vp, _vp, _vp]),
    ("xdg_cycle", C.c_int, [_vp, _ip, _vp, _vp]),
    ("xdg_solve", C.c_int, [_vp, _vp, _vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
    ("xdg_solve_host", C.c_int, [_vp, _dp, _dp, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
    ("xdg_restrict_noalloc", C.c_int, [_ip, C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                      _vp]),
    ("xdg_fma_peak", C.c_int, [_ip, _dp]),
    ("xdg_kernel_time", C.c_int, [_vp, _ip, _ip, _ip, _ip, _dp, _dp]),
    ("xdg_mlp_create", C.c_int, [_ip, _ip, C.c_uint64, _vp, C.POINTER(_vp)]),
    ("xdg_mlp_destroy", C.c_int, [_vp]),
    ("xdg_mlp_num_params", C.c_int, [_vp, C.POINTER(C.c_int64)]),
    ("xdg_mlp_get_params", C.c_int, [_vp, C.POINTER(C.c_float), C.c_int64]),
    ("xdg_mlp_set_params", C.c_int, [_vp, C.POINTER(C.c_float), C.c_int64]),
    ("xdg_mlp_forward", C.c_int, [_vp, _ip, C.c_int64, _vp, _vp]),
    ("xdg_mlp_loss_grad", C.c_int, [_vp, _ip, _vp, _vp, _vp, _vp, _vp, _dp, _vp]),
    ("xdg_mlp_train", C.c_int, [_vp, _ip, _vp, _vp, _vp, _vp, _vp, C.POINTER(TrainOpts), _dp]),
    ("xdg_units_setup", C.c_int, [_vp, _ip, C.POINTER(C.c_int32), _ip, C.POINTER(C.c_float)]),
    ("xdg_units_local", C.c_int, [_vp, _vp]),
    ("xdg_units_samples", C.c_int, [_vp, _ip, _vp, _vp, _vp, _vp]),
    ("xdg_learned_enable", C.c_int, [_vp, _vp, C.c_double]),
    ("xdg_learned_step", C.c_int, [_vp, _vp, _vp, C.POINTER(C.c_int)]),
    ("xdg_create_batch", C.c_int, [_ip, C.POINTER(Problem), C.POINTER(HierOpts), _vp, C.POINTER(_vp)]),
    ("xdg_batch_destroy", C.c_int, [_vp]),
    ("xdg_batch_get_info", C.c_int, [_vp, C.POINTER(BatchInfo)]),
    ("xdg_batch_group", C.c_int, [_vp, _ip, C.POINTER(_vp), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("xdg_solve_batch", C.c_int, [_vp, _vp, _vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo),
                                  C.POINTER(BatchResult)]),
    ("xdg_solve_batch_host", C.c_int, [_vp, _dp, _dp, C.POINTER(SolveOpts), C.POINTER(SolveInfo),
                                       C.POINTER(BatchResult)]),
]


def fma_peak(prec=XDG_PREC_F64) -> float:
    """Measured FMA throughput (TFLOP/s) of the current GPU in FP64 or FP32."""
    out = C.c_double()
    _check(load().xdg_fma_peak(prec, C.byref(out)))
    return out.value

NOALLOC_MAX_ENTRIES = 1 << 20

_lib = None


def load():
    """Load libxdg.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        for name, rt, at in SIGNATURES:
            f = getattr(L, name)
            f.restype = rt
            f.argtypes = at
        _lib = L
    return _lib


def _check(rc):
    if rc != XDG_OK:
        raise XdgError(rc, load().xdg_last_error().decode())


def _dptr(t):
    """device pointer of a torch CUDA float64 tensor (None -> NULL)"""
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous() and t.dtype == _torch().float64):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _fptr(t, dtype=None):
    """device pointer of a contiguous CUDA tensor of float32 (or `dtype`)"""
    torch = _torch()
    dt = dtype or torch.float32
    if not (t.is_cuda and t.is_contiguous() and t.dtype == dt):
        raise ValueError("expected a contiguous %s CUDA tensor" % dt)
    return C.c_void_p(t.data_ptr())


def _torch():
    import torch
    return torch


class _Ordered:
    """Orders a library call after the work already queued on torch's current stream, and the
    work queued after it on torch's current stream after the call (event waits only)."""

    def __init__(self, h):
        self.h = h

    def __enter__(self):
        if self.h.stream is not None:
            self.h.stream.wait_stream(_torch().cuda.current_stream(self.h.stream.device))

    def __exit__(self, *a):
        if self.h.stream is not None:
            _torch().cuda.current_stream(self.h.stream.device).wait_stream(self.h.stream)


def _marshal(Np, nb, row_ptr, col, val, aggs, Rs, keep):
    """xdg_problem struct over contiguous copies of the arrays (kept alive in `keep`)."""

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a

    nl = len(nb)
    nb_a = arr(nb, np.int64)
    rp = arr(row_ptr, np.int64)
    cl = arr(col, np.int32)
    vl = arr(val, np.float64)
    ag = [arr(a, np.int32) for a in aggs]
    Rr = [arr(r, np.float64) for r in Rs]
    aggp = (C.POINTER(C.c_int32) * max(nl - 1, 1))(*[a.ctypes.data_as(C.POINTER(C.c_int32)) for a in ag])
    Rp = (C.POINTER(C.c_double) * max(nl - 1, 1))(*[r.ctypes.data_as(_dp) for r in Rr])
    keep += [aggp, Rp]
    return Problem(Np, nl, nb_a.ctypes.data_as(C.POINTER(C.c_int64)), rp.ctypes.data_as(C.POINTER(C.c_int64)),
                   cl.ctypes.data_as(C.POINTER(C.c_int32)), vl.ctypes.data_as(_dp), aggp, Rp)


class Hierarchy:
    """Owner of an xdg_hier_t handle.

    The handle works on its own CUDA stream (`self.stream`, a torch.cuda.Stream created here
    unless one is given); every call is ordered with torch's current stream by event waits."""

    def __init__(self, Np, nb, row_ptr, col, val, aggs, Rs, omega=0.0, lanczos_steps=12, nu=1,
                 gamma=1, low_precision=0, stream=None, w_levels=0, split_rows=0, fused_coarse=0, outer_apply=0,
                 symmetric=0):
        L = load()
        torch = _torch()
        if stream is None:
            stream = torch.cuda.Stream()
        self.stream = stream
        self._keep = []

        prob = _marshal(Np, nb, row_ptr, col, val, aggs, Rs, self._keep)
        opts = HierOpts(omega, lanczos_steps, nu, gamma, low_precision, w_levels, split_rows, fused_coarse,
                        outer_apply, symmetric)
        h = C.c_void_p()
        st = C.c_void_p(stream.cuda_stream)
        self._h = None
        with _Ordered(self):
            _check(L.xdg_create_hierarchy(C.byref(prob), C.byref(opts), st, C.byref(h)))
        self._keep = []
        self._h = h
        self.Np = Np
        self.nb = [int(x) for x in nb]
        self.n = self.nb[0] * Np

    @classmethod
    def from_problem(cls, prob, **kw):
        """From an xdg_problem.Problem (finest operator, maps and transfer blocks)."""
        return cls(prob.Np, prob.nb, prob.row_ptr, prob.col, prob.val, prob.agg, prob.R, **kw)

    # ------------------------------------------------------------------ queries
    def info(self) -> dict:
        i = HierInfo()
        _check(load().xdg_get_info(self._h, C.byref(i)))
        nl = i.n_levels
        return {"Np": i.Np, "n_levels": nl, "nb": list(i.nb[:nl]), "nnzb": list(i.nnzb[:nl]),
                "omega": list(i.omega[:nl]), "lambda_max": list(i.lambda_max[:nl]),
                "coarse_n": i.coarse_n, "device_bytes": i.device_bytes, "setup_ms": list(i.setup_ms),
                "split": [bool((i.split_mask >> l) & 1) for l in range(nl)], "fused_level": i.fused_level,
                "outer_pair": bool(i.outer_pair), "symmetric_built": bool(i.symmetric & 1),
                "symmetric_cycle": bool(i.symmetric & 2), "symmetric_pair": bool(i.symmetric & 4),
                "fused_cluster": i.fused_cluster}

    def export_level(self, level: int):
        _torch().cuda.synchronize(self.stream.device)
        inf = self.info()
        nb, nnz, Np = inf["nb"][level - 1], inf["nnzb"][level - 1], self.Np
        rp = np.zeros(nb + 1, np.int64)
        cl = np.zeros(max(nnz, 1), np.int32)
        vl = np.zeros(max(nnz, 1) * Np * Np)
        _check(load().xdg_export_level(self._h, level, rp.ctypes.data_as(C.POINTER(C.c_int64)),
                                       cl.ctypes.data_as(C.POINTER(C.c_int32)), vl.ctypes.data_as(_dp)))
        return rp, cl[:nnz], vl[:nnz * Np * Np].reshape(nnz, Np, Np)

    # ------------------------------------------------------------------ device entry points
    def apply(self, level, x, y, prec=XDG_PREC_F64):
        with _Ordered(self):
            _check(load().xdg_apply(self._h, level, _dptr(x), _dptr(y), prec))

    def set_split(self, level, on):
        with _Ordered(self):
            _check(load().xdg_set_split(self._h, level, int(bool(on))))

    def get_damping(self, level, problem=0):
        """(omega, lambda_max) of a level for one problem of the hierarchy."""
        om, lm = C.c_double(), C.c_double()
        _check(load().xdg_get_damping(self._h, level, problem, C.byref(om), C.byref(lm)))
        return om.value, lm.value

    def set_damping(self, level, omega):
        with _Ordered(self):
            _check(load().xdg_set_damping(self._h, level, omega))

    def set_schwarz(self, level, patches):
        """Additive Schwarz smoother on `level` (1-based) with patches = (ptr int64[n+1],
        blocks int32[ptr[n]]) host arrays, or None for block Jacobi (xdg_set_schwarz)."""
        with _Ordered(self):
            if patches is None:
                _check(load().xdg_set_schwarz(self._h, level, 0, None, None))
                return
            ptr = np.ascontiguousarray(patches[0], dtype=np.int64)
            blk = np.ascontiguousarray(patches[1], dtype=np.int32)
            _check(load().xdg_set_schwarz(self._h, level, len(ptr) - 1, ptr.ctypes.data_as(C.POINTER(C.c_int64)),
                                          blk.ctypes.data_as(C.POINTER(C.c_int32))))

    def solve_orthomg(self, b, x, tol=1e-10, maxit=500, restart=30, coarse_passes=1, smoother_precision=XDG_PREC_F64,
                      raise_on_error=True) -> dict:
        """Orthonormalisation multigrid (xdg_solve_orthomg); x holds x0 and receives the result."""
        o = OrthoMGOpts(tol, maxit, restart, coarse_passes, smoother_precision)
        info = SolveInfo()
        with _Ordered(self):
            rc = load().xdg_solve_orthomg(self._h, _dptr(b), _dptr(x), C.byref(o), C.byref(info))
        if raise_on_error and rc not in (XDG_OK,):
            _check(rc)
        return {f: getattr(info, f) for f, _ in SolveInfo._fields_}

    def test_barrier_timeout(self, on):
        """Make the fused cycle's grid barriers give up (xdg_test_barrier_timeout)."""
        with _Ordered(self):
            _check(load().xdg_test_barrier_timeout(self._h, 1 if on else 0))

    def residual(self, level, b, x, r):
        """r = b - M^level x (xdg_residual)."""
        with _Ordered(self):
            _check(load().xdg_residual(self._h, level, _dptr(b), _dptr(x), _dptr(r)))

    def pmg_setup(self, n_lo, inner_tol=1e-10, inner_maxit=500, inner_precision=XDG_PREC_F64, **lo_opts):
        """p-multigrid on level 1 with n_lo low-order modes per block (xdg_pmg_setup); lo_opts
        (omega, gamma, w_levels, ...) configure the low-order hierarchy, else the handle's cycle."""
        o = None
        if lo_opts:
            o = HierOpts(lo_opts.get("omega", 0.0), lo_opts.get("lanczos_steps", 12), lo_opts.get("nu", 1),
                         lo_opts.get("gamma", 1), lo_opts.get("low_precision", 0), lo_opts.get("w_levels", 0),
                         lo_opts.get("split_rows", 0), lo_opts.get("fused_coarse", 1), lo_opts.get("outer_apply", 1),
                         lo_opts.get("symmetric", 1))
        with _Ordered(self):
            _check(load().xdg_pmg_setup(self._h, n_lo, C.byref(o) if o is not None else None, inner_tol,
                                        inner_maxit, inner_precision))

    def pmg_apply(self, r, z):
        with _Ordered(self):
            _check(load().xdg_pmg_apply(self._h, _dptr(r), _dptr(z)))

    def solve_gmres(self, b, x, tol=1e-10, maxit=1000, restart=50, preconditioner=0, precision=XDG_PREC_F64,
                    raise_on_error=True) -> dict:
        """Flexible GMRES (xdg_solve_gmres); preconditioner 0 = multigrid cycle, 1 = p-multigrid."""
        o = GmresOpts(tol, maxit, restart, preconditioner, precision)
        info = SolveInfo()
        with _Ordered(self):
            rc = load().xdg_solve_gmres(self._h, _dptr(b), _dptr(x), C.byref(o), C.byref(info))
        if raise_on_error and rc != XDG_OK:
            _check(rc)
        return {f: getattr(info, f) for f, _ in SolveInfo._fields_}

    def schwarz_info(self, level) -> dict:
        i = SchwarzInfo()
        _check(load().xdg_get_schwarz(self._h, level, C.byref(i)))
        return {f: getattr(i, f) for f, _ in SchwarzInfo._fields_}

    KERNEL_APPLY, KERNEL_SMOOTH, KERNEL_RESTRICT = 0, 1, 2

    def kernel_time(self, which, level, prec=XDG_PREC_F64, reps=20):
        """(mean ms per launch, algorithmic bytes per launch) of one cycle kernel on a level."""
        ms, by = C.c_double(), C.c_double()
        with _Ordered(self):
            _check(load().xdg_kernel_time(self._h, which, level, prec, reps, C.byref(ms), C.byref(by)))
        return ms.value, by.value

    def smooth(self, level, b, x_in, x_out):
        with _Ordered(self):
            _check(load().xdg_smooth(self._h, level, _dptr(b), _dptr(x_in), _dptr(x_out)))

    def restrict(self, level, b, x, rc):
        with _Ordered(self):
            _check(load().xdg_restrict(self._h, level, _dptr(b), _dptr(x), _dptr(rc)))

    def prolong(self, level, zc, x_in, x_out):
        with _Ordered(self):
            _check(load().xdg_prolong(self._h, level, _dptr(zc), _dptr(x_in), _dptr(x_out)))

    def coarse_solve(self, r, z):
        with _Ordered(self):
            _check(load().xdg_coarse_solve(self._h, _dptr(r), _dptr(z)))

    def vcycle(self, b, x):
        with _Ordered(self):
            _check(load().xdg_vcycle(self._h, _dptr(b), _dptr(x)))

    def cycle(self, prec, b, x):
        with _Ordered(self):
            _check(load().xdg_cycle(self._h, prec, _dptr(b), _dptr(x)))

    def solve(self, b, x, tol=1e-10, maxit=1000, check_every=1, precision=XDG_PREC_F64, inner_tol=0.0,
              time_budget_ms=0.0, raise_on_error=True) -> dict:
        o = SolveOpts(tol, maxit, check_every, precision, inner_tol, time_budget_ms)
        info = SolveInfo()
        with _Ordered(self):
            rc = load().xdg_solve(self._h, _dptr(b), _dptr(x), C.byref(o), C.byref(info))
        if raise_on_error:
            _check(rc)
        return {"iterations": info.iterations, "outer": info.outer, "relres": info.relres,
                "ms": info.ms, "status": rc, "launches": info.launches}

    def solve_host(self, b_host, x_host, tol=1e-10, maxit=1000, check_every=1, precision=XDG_PREC_F64,
                   inner_tol=0.0, time_budget_ms=0.0, raise_on_error=True) -> dict:
        """b_host, x_host: numpy float64 arrays (pinned memory gives the fastest copies)."""
        for a in (b_host, x_host):
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host vectors must be contiguous float64")
        o = SolveOpts(tol, maxit, check_every, precision, inner_tol, time_budget_ms)
        info = SolveInfo()
        with _Ordered(self):
            rc = load().xdg_solve_host(self._h, b_host.ctypes.data_as(_dp), x_host.ctypes.data_as(_dp),
                                       C.byref(o), C.byref(info))
        if raise_on_error:
            _check(rc)
        return {"iterations": info.iterations, "outer": info.outer, "relres": info.relres,
                "ms": info.ms, "status": rc, "launches": info.launches}

    # ------------------------------------------------------------------ learned correction
    def units_setup(self, pairs, geom):
        """pairs int32 [U][2] (A block, B block of a cut cell), geom float32 [U][n_geo]."""
        pairs = np.ascontiguousarray(pairs, np.int32)
        geom = np.ascontiguousarray(geom, np.float32)
        self.n_units, self.n_geo = pairs.shape[0], (geom.shape[1] if geom.ndim == 2 else 0)
        with _Ordered(self):
            _check(load().xdg_units_setup(self._h, self.n_units, pairs.ctypes.data_as(C.POINTER(C.c_int32)),
                                          self.n_geo, geom.ctypes.data_as(C.POINTER(C.c_float))))

    def units_local(self):
        """FP32 unit matrices [U][2Np][2Np] (CUDA tensor)."""
        torch = _torch()
        m = 2 * self.Np
        out = torch.empty((self.n_units, m, m), dtype=torch.float32, device=self.stream.device)
        with _Ordered(self):
            _check(load().xdg_units_local(self._h, _fptr(out)))
        return out

    def units_samples(self, r, prec=XDG_PREC_F64):
        """(X, R, C) CUDA tensors of the training samples of all units for right-hand side r."""
        torch = _torch()
        m = 2 * self.Np
        dev = self.stream.device
        X = torch.empty((self.n_units, self.n_geo + m), dtype=torch.float32, device=dev)
        R = torch.empty((self.n_units, m), dtype=torch.float32, device=dev)
        Cc = torch.empty((self.n_units,), dtype=torch.float32, device=dev)
        with _Ordered(self):
            _check(load().xdg_units_samples(self._h, prec, _dptr(r), _fptr(X), _fptr(R), _fptr(Cc)))
        return X, R, Cc

    def learned_enable(self, mlp, theta=0.25):
        with _Ordered(self):
            _check(load().xdg_learned_enable(self._h, mlp._h if mlp is not None else None, theta))
        self._mlp = mlp

    def learned_step(self, r, z) -> int:
        k = C.c_int()
        with _Ordered(self):
            _check(load().xdg_learned_step(self._h, _dptr(r), _dptr(z), C.byref(k)))
        return k.value

    def destroy(self):
        if getattr(self, "_h", None):
            if not getattr(self, "_borrowed", None):
                load().xdg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _solve_result(rc, info, res):
    return {"iterations": info.iterations, "relres": info.relres, "ms": info.ms, "status": rc,
            "launches": info.launches,
            "problems": [{"iterations": r.iterations, "status": r.status, "relres": r.relres} for r in res]}


class Batch:
    """Owner of an xdg_batch_t: n independent problems solved in one graph launch.

    problems: list of xdg_problem.Problem (or objects with Np, nb, row_ptr, col, val, agg, R).
    Vectors are the problems' level-1 vectors concatenated in list order (`offsets`)."""

    def __init__(self, problems, omega=0.0, lanczos_steps=12, nu=1, gamma=1, low_precision=0,
                 w_levels=0, stream=None, split_rows=0, symmetric=0, outer_apply=0):
        L = load()
        torch = _torch()
        if stream is None:
            stream = torch.cuda.Stream()
        self.stream = stream
        keep = []
        arr = (Problem * len(problems))()
        for i, p in enumerate(problems):
            arr[i] = _marshal(p.Np, p.nb, p.row_ptr, p.col, p.val, p.agg, p.R, keep)
        opts = HierOpts(omega, lanczos_steps, nu, gamma, low_precision, w_levels, split_rows, 1, outer_apply,
                        symmetric)
        h = C.c_void_p()
        self._h = None
        with _Ordered(self):
            _check(L.xdg_create_batch(len(problems), arr, C.byref(opts), C.c_void_p(stream.cuda_stream),
                                      C.byref(h)))
        self._h = h
        self.n = len(problems)
        sizes = [int(p.nb[0]) * int(p.Np) for p in problems]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.total_dof = int(self.offsets[-1])

    def info(self) -> dict:
        i = BatchInfo()
        _check(load().xdg_batch_get_info(self._h, C.byref(i)))
        return {"n_problems": i.n_problems, "n_groups": i.n_groups, "total_dof": i.total_dof,
                "device_bytes": i.device_bytes, "setup_ms": i.setup_ms,
                "nodes_fixed": list(i.nodes_fixed), "nodes_per_iteration": list(i.nodes_per_iteration)}

    def group(self, g):
        """(Hierarchy view of group g's union hierarchy, list of member indices)."""
        h = C.c_void_p()
        m = C.c_int()
        _check(load().xdg_batch_group(self._h, g, C.byref(h), C.byref(m), None))
        mem = (C.c_int * max(m.value, 1))()
        _check(load().xdg_batch_group(self._h, g, None, None, mem))
        H = Hierarchy.__new__(Hierarchy)
        H._h, H._borrowed, H._owner, H.stream = h, True, self, self.stream
        inf = H.info()
        H.Np, H.nb = inf["Np"], inf["nb"]
        H.n = H.nb[0] * H.Np
        return H, list(mem[:m.value])

    def solve(self, b, x, tol=1e-10, maxit=1000, precision=XDG_PREC_F64, raise_on_error=True) -> dict:
        o = SolveOpts(tol, maxit, 1, precision, 0.0, 0.0)
        info = SolveInfo()
        res = (BatchResult * self.n)()
        with _Ordered(self):
            rc = load().xdg_solve_batch(self._h, _dptr(b), _dptr(x), C.byref(o), C.byref(info), res)
        if raise_on_error:
            _check(rc)
        return _solve_result(rc, info, res)

    def solve_host(self, b_host, x_host, tol=1e-10, maxit=1000, precision=XDG_PREC_F64,
                   raise_on_error=True) -> dict:
        for a in (b_host, x_host):
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host vectors must be contiguous float64")
        o = SolveOpts(tol, maxit, 1, precision, 0.0, 0.0)
        info = SolveInfo()
        res = (BatchResult * self.n)()
        with _Ordered(self):
            rc = load().xdg_solve_batch_host(self._h, b_host.ctypes.data_as(_dp), x_host.ctypes.data_as(_dp),
                                             C.byref(o), C.byref(info), res)
        if raise_on_error:
            _check(rc)
        return _solve_result(rc, info, res)

    def destroy(self):
        if getattr(self, "_h", None):
            load().xdg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Mlp:
    """Owner of an xdg_mlp_t: the network of the learned cut-cell correction."""

    def __init__(self, n_in, n_out, seed=0, stream=None):
        torch = _torch()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        self._h = None
        with _Ordered(self):
            _check(load().xdg_mlp_create(n_in, n_out, seed, C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h
        self.n_in, self.n_out = n_in, n_out
        n = C.c_int64()
        _check(load().xdg_mlp_num_params(h, C.byref(n)))
        self.n_params = n.value

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        with _Ordered(self):
            _check(load().xdg_mlp_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float)), self.n_params))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        with _Ordered(self):
            _check(load().xdg_mlp_set_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), self.n_params))

    def forward(self, X, prec=XDG_PREC_F32):
        torch = _torch()
        Y = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=X.device)
        with _Ordered(self):
            _check(load().xdg_mlp_forward(self._h, prec, X.shape[0], _fptr(X), _fptr(Y)))
        return Y

    def loss_grad(self, X, uid, Mloc, R, Cc):
        torch = _torch()
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        loss = C.c_double()
        with _Ordered(self):
            _check(load().xdg_mlp_loss_grad(self._h, X.shape[0], _fptr(X), _fptr(uid, torch.int32), _fptr(Mloc),
                                            _fptr(R), _fptr(Cc), C.byref(loss), _fptr(g)))
        return loss.value, g

    def train(self, X, uid, Mloc, R, Cc, epochs=20, batch=512, lr=1e-3, seed=1) -> np.ndarray:
        torch = _torch()
        hist = np.zeros(epochs)
        o = TrainOpts(epochs, batch, lr, 0.0, 0.0, 0.0, seed)
        with _Ordered(self):
            _check(load().xdg_mlp_train(self._h, X.shape[0], _fptr(X), _fptr(uid, torch.int32), _fptr(Mloc),
                                        _fptr(R), _fptr(Cc), C.byref(o), hist.ctypes.data_as(_dp)))
        return hist

    def destroy(self):
        if getattr(self, "_h", None):
            load().xdg_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def restrict_noalloc(Np, nb_fine, nb_coarse, row_ptr, col, val, R, child_ptr, child, b, x, rc, stream=None):
    """rc = R^T (b - M x) from caller-owned device tensors, with no allocation in the library
    (xdg_restrict_noalloc: fixed 8 MiB scratch, calls must not overlap on one GPU).
    row_ptr/child_ptr int64, col/child int32, the rest float64 CUDA tensors on the current
    device; x may be None. The C entry point cannot see the length of a device array, so every
    length is checked here, from tensor metadata and two scalar reads (row_ptr[nb_fine] and
    child_ptr[nb_coarse]), before anything is enqueued: a short array would make the kernels
    read or write past its end. Raises ValueError on a mismatch."""
    torch = _torch()
    cur = torch.cuda.current_device()
    if stream is None:
        stream = torch.cuda.current_stream()
    if stream.device.index != cur:
        raise ValueError("the stream must belong to the current device (cuda:%d)" % cur)
    Np, nb_fine, nb_coarse = int(Np), int(nb_fine), int(nb_coarse)
    if nb_fine <= 0 or nb_coarse <= 0:
        raise ValueError("nb_fine and nb_coarse must be positive")

    def p(t, dt, n, name):
        if t is None:
            return None
        if not (t.is_cuda and t.is_contiguous() and t.dtype == dt):
            raise ValueError("%s: expected a contiguous CUDA tensor of %s" % (name, dt))
        if t.device.index != cur:
            raise ValueError("%s: on cuda:%d, not on the current device cuda:%d" % (name, t.device.index, cur))
        if t.numel() < n:
            raise ValueError("%s: %d entries, at least %d needed" % (name, t.numel(), n))
        return C.c_void_p(t.data_ptr())

    f64, i64, i32 = torch.float64, torch.int64, torch.int32
    nf, nc = nb_fine * Np, nb_coarse * Np
    args = [p(row_ptr, i64, nb_fine + 1, "row_ptr"), p(col, i32, 1, "col"), p(val, f64, 0, "val"),
            p(R, f64, nf * Np, "R"), p(child_ptr, i64, nb_coarse + 1, "child_ptr"), p(child, i32, nb_fine, "child"),
            p(b, f64, nf, "b"), p(x, f64, nf, "x"), p(rc, f64, nc, "rc")]
    if None in args[:7] or args[8] is None:
        raise ValueError("only x may be None")
    nnzb = int(row_ptr[nb_fine].item())
    if nnzb < 0 or nnzb > col.numel() or val.numel() < nnzb * Np * Np:
        raise ValueError("row_ptr[nb_fine] = %d does not fit col (%d) and val (%d entries)"
                         % (nnzb, col.numel(), val.numel()))
    if int(child_ptr[nb_coarse].item()) != nb_fine:
        raise ValueError("child_ptr[nb_coarse] must equal nb_fine (every fine block is one child)")
    _check(load().xdg_restrict_noalloc(Np, nb_fine, nb_coarse, *args, C.c_void_p(stream.cuda_stream)))


# C-name aliases
def create_hierarchy(prob, **kw) -> Hierarchy:
    return Hierarchy.from_problem(prob, **kw)
