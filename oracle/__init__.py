"""CPU oracle of the XDG multigrid solve (plain FP64 C, ``xdg_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``. The CUDA library neither imports nor links anything here.

Kummer, Smuda, Weber, arXiv 2003.02431: Eq. (GenericMatrixSystem) (the operator),
Eq. (XDGsysRestriction) (Galerkin coarse operators), Algorithm 4 (level recursion: smoothing,
restriction, coarse correction, prolongation), sec. 3.3 (direct coarse solve, Krylov outer
method). The function-level citations are in the C source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xdg_oracle.c")
_LIB = os.path.join(_HERE, "libxdg_oracle.so")

_lib = None
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.or_bsr_spmv.argtypes = [C.c_int64, C.c_int, _i64p, _i32p, _dp, _dp, _dp]
        L.or_residual.argtypes = [C.c_int64, C.c_int, _i64p, _i32p, _dp, _dp, _dp, _dp]
        L.or_restrict.argtypes = [C.c_int64, C.c_int64, C.c_int, _i32p, _dp, _dp, _dp]
        L.or_prolong.argtypes = [C.c_int64, C.c_int, _i32p, _dp, _dp, _dp]
        L.or_galerkin.restype = C.c_int
        L.or_galerkin.argtypes = [C.c_int64, C.c_int64, C.c_int, _i64p, _i32p, _dp, _i32p, _dp,
                                  C.POINTER(_i64p), C.POINTER(_i32p), C.POINTER(_dp), _i64p]
        L.or_free.argtypes = [C.c_void_p]
        L.or_hier_create.restype = C.c_void_p
        L.or_hier_create.argtypes = [C.c_int, C.c_int, C.c_int64, _i64p, _i32p, _dp, _i64p,
                                     C.POINTER(_i32p), C.POINTER(_dp), C.c_double, C.c_int, C.c_int, C.c_int]
        L.or_hier_free.argtypes = [C.c_void_p]
        L.or_hier_level.restype = C.c_int
        L.or_hier_level.argtypes = [C.c_void_p, C.c_int, _i64p, _i64p, _dp, _dp,
                                    C.POINTER(_i64p), C.POINTER(_i32p), C.POINTER(_dp)]
        L.or_smooth.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
        L.or_coarse_solve.argtypes = [C.c_void_p, _dp, _dp]
        L.or_vcycle.argtypes = [C.c_void_p, _dp, _dp]
        L.or_pcg.restype = C.c_int
        L.or_pcg.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_int, _dp, _dp]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def bsr_spmv(row_ptr, col, val, x):
    """y = A x for BSR (row_ptr int64[nb+1], col int32[nnzb], val f64[nnzb,Np,Np])."""
    L = _load()
    nb, Np = len(row_ptr) - 1, val.shape[-1]
    x = _f64(x).reshape(-1)
    y = np.empty(nb * Np)
    L.or_bsr_spmv(nb, Np, _p(np.ascontiguousarray(row_ptr, np.int64), _i64p),
                  _p(np.ascontiguousarray(col, np.int32), _i32p), _p(_f64(val), _dp), _p(x, _dp), _p(y, _dp))
    return y.reshape(nb, Np)


def restrict(agg, R, r, nbc):
    L = _load()
    nbf, Np = R.shape[0], R.shape[-1]
    out = np.empty(nbc * Np)
    L.or_restrict(nbf, nbc, Np, _p(np.ascontiguousarray(agg, np.int32), _i32p), _p(_f64(R), _dp),
                  _p(_f64(r).reshape(-1), _dp), _p(out, _dp))
    return out.reshape(nbc, Np)


def prolong_add(agg, R, zc, x):
    """returns x + R zc"""
    L = _load()
    nbf, Np = R.shape[0], R.shape[-1]
    y = _f64(x).reshape(-1).copy()
    L.or_prolong(nbf, Np, _p(np.ascontiguousarray(agg, np.int32), _i32p), _p(_f64(R), _dp),
                 _p(_f64(zc).reshape(-1), _dp), _p(y, _dp))
    return y.reshape(nbf, Np)


def galerkin(row_ptr, col, val, agg, R, nbc):
    """Coarse operator R^T M R as (row_ptr, col, val)."""
    L = _load()
    nbf, Np = len(row_ptr) - 1, val.shape[-1]
    rp, cl, vl, nnz = _i64p(), _i32p(), _dp(), C.c_int64()
    rc = L.or_galerkin(nbf, nbc, Np, _p(np.ascontiguousarray(row_ptr, np.int64), _i64p),
                       _p(np.ascontiguousarray(col, np.int32), _i32p), _p(_f64(val), _dp),
                       _p(np.ascontiguousarray(agg, np.int32), _i32p), _p(_f64(R), _dp),
                       C.byref(rp), C.byref(cl), C.byref(vl), C.byref(nnz))
    if rc != 0:
        raise MemoryError("or_galerkin failed")
    z = nnz.value
    out = (np.ctypeslib.as_array(rp, shape=(nbc + 1,)).copy(),
           np.ctypeslib.as_array(cl, shape=(max(z, 1),))[:z].copy(),
           np.ctypeslib.as_array(vl, shape=(max(z, 1) * Np * Np,))[:z * Np * Np].reshape(z, Np, Np).copy())
    for p in (rp, cl, vl):
        L.or_free(C.cast(p, C.c_void_p))
    return out


class Hierarchy:
    """Oracle multigrid hierarchy built from a generated problem (xdg_problem.Problem)."""

    def __init__(self, prob, omega: float = 0.0, lanczos_steps: int = 12, nu: int = 1, n_levels=None,
                 gamma: int = 1):
        L = _load()
        self._L = L
        nl = prob.n_levels if n_levels is None else n_levels
        self.Np = prob.Np
        self.nlev = nl
        self._keep = [prob]  # the problem owns the level-1 and transfer arrays
        self._rp = np.ascontiguousarray(prob.row_ptr, np.int64)
        self._col = np.ascontiguousarray(prob.col, np.int32)
        self._val = _f64(prob.val)
        self._nbs = np.array(prob.nb[:nl], dtype=np.int64)
        self._aggs = [np.ascontiguousarray(a, np.int32) for a in prob.agg[:nl - 1]]
        self._Rs = [_f64(r) for r in prob.R[:nl - 1]]
        aggp = (_i32p * max(nl - 1, 1))(*[_p(a, _i32p) for a in self._aggs])
        Rp = (_dp * max(nl - 1, 1))(*[_p(r, _dp) for r in self._Rs])
        h = L.or_hier_create(nl, self.Np, prob.nb[0], _p(self._rp, _i64p), _p(self._col, _i32p),
                             _p(self._val, _dp), _p(self._nbs, _i64p), aggp, Rp, omega, lanczos_steps, nu,
                             gamma)
        if not h:
            raise RuntimeError("oracle hierarchy: operator not SPD")
        self._h = C.c_void_p(h)
        self.n = prob.nb[0] * self.Np

    def level(self, l: int) -> dict:
        nb, nnz, om, lm = C.c_int64(), C.c_int64(), C.c_double(), C.c_double()
        rp, cl, vl = _i64p(), _i32p(), _dp()
        if self._L.or_hier_level(self._h, l, C.byref(nb), C.byref(nnz), C.byref(om), C.byref(lm),
                                 C.byref(rp), C.byref(cl), C.byref(vl)) != 0:
            raise IndexError(l)
        n, z, Np = nb.value, nnz.value, self.Np
        return {"nb": n, "nnzb": z, "omega": om.value, "lmax": lm.value,
                "row_ptr": np.ctypeslib.as_array(rp, shape=(n + 1,)).copy(),
                "col": np.ctypeslib.as_array(cl, shape=(max(z, 1),))[:z].copy(),
                "val": np.ctypeslib.as_array(vl, shape=(max(z, 1) * Np * Np,))[:z * Np * Np].reshape(z, Np, Np).copy()}

    def vcycle(self, b):
        b = _f64(b).reshape(-1)
        x = np.empty_like(b)
        self._L.or_vcycle(self._h, _p(b, _dp), _p(x, _dp))
        return x

    def smooth(self, l, b, x):
        b = _f64(b).reshape(-1)
        y = _f64(x).reshape(-1).copy()
        self._L.or_smooth(self._h, l, _p(b, _dp), _p(y, _dp))
        return y

    def coarse_solve(self, r):
        r = _f64(r).reshape(-1)
        z = np.empty_like(r)
        self._L.or_coarse_solve(self._h, _p(r, _dp), _p(z, _dp))
        return z

    def set_patches(self, l, patches, mode=1, lanczos_steps=12, omega=0.0):
        """Additive Schwarz smoother (Algorithm Swz, exact patch solves) on level l (0-based):
        patches = (ptr int64[n+1], blocks int32[ptr[n]]) or None for block Jacobi. mode 0 divides
        the summed patch solutions by alpha (as printed), mode 1 scales by alpha^{-1/2} on both
        sides (symmetric). Re-estimates the level's damping from the Schwarz preconditioner."""
        L = self._L
        if not hasattr(L, "_swz_set"):
            L.or_hier_set_patches.restype = C.c_int
            L.or_hier_set_patches.argtypes = [C.c_void_p, C.c_int, C.c_int64, _i64p, _i32p, C.c_int, C.c_int,
                                              C.c_double]
            L.or_schwarz.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
            L._swz_set = True
        if patches is None:
            rc = L.or_hier_set_patches(self._h, l, 0, None, None, mode, lanczos_steps, omega)
        else:
            ptr = np.ascontiguousarray(patches[0], np.int64)
            blk = np.ascontiguousarray(patches[1], np.int32)
            self._keep.append((ptr, blk))
            rc = L.or_hier_set_patches(self._h, l, len(ptr) - 1, _p(ptr, _i64p), _p(blk, _i32p), mode,
                                       lanczos_steps, omega)
        if rc == -2:
            raise RuntimeError("oracle Schwarz: a patch matrix is not positive definite")
        if rc != 0:
            raise ValueError("oracle Schwarz: invalid patches")

    def schwarz(self, l, r):
        """z = Swz(r) on level l (undamped; the patches of set_patches)."""
        r = _f64(r).reshape(-1)
        z = np.empty_like(r)
        self._L.or_schwarz(self._h, l, _p(r, _dp), _p(z, _dp))
        return z

    def pcg(self, b, x0=None, tol=1e-10, maxit=500):
        """Returns (x, iterations, true relative residual, history)."""
        b = _f64(b).reshape(-1)
        x = np.zeros_like(b) if x0 is None else _f64(x0).reshape(-1).copy()
        rr = C.c_double()
        hist = np.zeros(maxit + 1)
        it = self._L.or_pcg(self._h, _p(b, _dp), _p(x, _dp), tol, maxit, C.byref(rr), _p(hist, _dp))
        return x, it, rr.value, hist[:it + 1]

    def orthomg(self, b, x0=None, tol=1e-10, maxit=500, restart=30):
        """Orthonormalisation multigrid (Algorithm OrthoMG with Algorithm ResMinimi) on the
        finest level; the finest level's search space restarts after `restart` directions.
        Returns (x, passes, true relative residual, residual history)."""
        L = self._L
        if not hasattr(L, "_omg_set"):
            L.or_orthomg.restype = C.c_int
            L.or_orthomg.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_int, C.c_int, _dp, _dp]
            L._omg_set = True
        b = _f64(b).reshape(-1)
        x = np.zeros_like(b) if x0 is None else _f64(x0).reshape(-1).copy()
        rr = C.c_double()
        hist = np.zeros(maxit + 1)
        it = L.or_orthomg(self._h, _p(b, _dp), _p(x, _dp), tol, maxit, restart, C.byref(rr), _p(hist, _dp))
        return x, it, rr.value, hist[:it + 1]

    def rm_steps(self, level, zs, b, x0):
        """Algorithm ResMinimi applied k times on `level` with the raw directions zs (k, n) from
        x0: returns (x, r, W (k, n), Z (k, n))."""
        L = self._L
        if not hasattr(L, "_rm_set"):
            L.or_rm_steps.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L._rm_set = True
        zs = _f64(zs)
        k, n = zs.shape
        b, x0 = _f64(b).reshape(-1), _f64(x0).reshape(-1)
        x, r = np.empty(n), np.empty(n)
        W, Z = np.empty((k, n)), np.empty((k, n))
        L.or_rm_steps(self._h, level, k, _p(zs, _dp), _p(b, _dp), _p(x0, _dp), _p(x, _dp), _p(r, _dp),
                      _p(W, _dp), _p(Z, _dp))
        return x, r, W, Z

    def pmg(self, level, n_lo, b, blocks=None):
        """Algorithm pMultigrid on `level` (0-based) with n_lo low-order modes per block, over the
        given block subset (None: every block): x = PMG(b, k_lo, I)."""
        L = self._L
        if not hasattr(L, "_pmg_set"):
            L.or_pmg.restype = C.c_int
            L.or_pmg.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, _i32p, _dp, _dp]
            L._pmg_set = True
        b = _f64(b).reshape(-1)
        x = np.empty_like(b)
        if blocks is None:
            rc = L.or_pmg(self._h, level, n_lo, -1, None, _p(b, _dp), _p(x, _dp))
        else:
            blk = np.ascontiguousarray(blocks, np.int32)
            rc = L.or_pmg(self._h, level, n_lo, len(blk), _p(blk, _i32p), _p(b, _dp), _p(x, _dp))
        if rc != 0:
            raise RuntimeError("oracle PMG: a system is not positive definite")
        return x

    def close(self):
        if getattr(self, "_h", None):
            self._L.or_hier_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def quantize_blocks(blocks, prec):
    """Dequantised FP64 values of the low-precision block storage (prec 1 = FP32, 2 = BF16)
    and the per-block scales."""
    L = _load()
    if not hasattr(L, "_q_set"):
        L.or_quantize_blocks.argtypes = [C.c_int64, C.c_int, C.c_int, _dp, _dp, C.POINTER(C.c_float)]
        L._q_set = True
    a = _f64(blocks)
    nblk, np2 = a.shape[0], a.shape[1] * a.shape[2]
    out = np.empty_like(a)
    sc = np.empty(nblk, dtype=np.float32)
    L.or_quantize_blocks(nblk, np2, prec, _p(a, _dp), _p(out, _dp), sc.ctypes.data_as(C.POINTER(C.c_float)))
    return out, sc


def set_orthomg_passes(passes: int) -> None:
    """Passes of Algorithm OrthoMG on every coarse level (1 = one pass per visit, 2 = K-cycle)."""
    L = _load()
    L.or_set_orthomg_passes.argtypes = [C.c_int]
    L.or_set_orthomg_passes(int(passes))


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops (n >= 1); returns the number now in use."""
    L = _load()
    L.or_set_threads.restype = C.c_int
    L.or_set_threads.argtypes = [C.c_int]
    return int(L.or_set_threads(int(n)))


def set_w_levels(h, wlev):
    """Repeat the coarse correction (gamma times) only on the wlev finest levels."""
    L = _load()
    L.or_hier_set_wlev.argtypes = [C.c_void_p, C.c_int]
    L.or_hier_set_wlev(h._h, wlev)
