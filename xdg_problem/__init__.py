"""Generator of the agglomerated XDG-SIP linear system: the input of the multigrid solve.

Kummer, Smuda, Weber, "BoSSS: a package for multigrid extended discontinuous Galerkin
methods" (arXiv 2003.02431), sections 1.1 (Poisson problem with a jump in mu), 2 (XDG space,
SIP form Eq. DefSIP and right-hand side Eq. SIPrhs, cell agglomeration), 3.1 (aggregation
sequence mapped onto the cut-cell mesh) and 3.2 (bases, re-orthonormalisation, transfer
matrices R^{X,lambda}).

The work is done by the C++ library ``libxdgprob.so`` built from ``xdgprob.cpp``; this module
marshals arguments and exposes the arrays as numpy views that live as long as the Problem.
It holds no part of the solve: the operator apply, smoothing, Galerkin products,
factorisations and Krylov iterations live in the CUDA library (and, independently, in the CPU
oracle used by the tests).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xdgprob.cpp")
_HDR = os.path.join(_HERE, "xdgprob.h")
_LIB = os.path.join(_HERE, "libxdgprob.so")


def build(force: bool = False) -> str:
    """Compile libxdgprob.so in-tree with g++ (OpenMP), unless it is up to date."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c++17", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [("D", C.c_int), ("N", C.c_int), ("k", C.c_int), ("rhs_kind", C.c_int),
                ("max_coarse_dof", C.c_int), ("max_levels", C.c_int), ("quad_q", C.c_int),
                ("nthreads", C.c_int), ("lo", C.c_double), ("hi", C.c_double),
                ("c", C.c_double * 3), ("R", C.c_double), ("muA", C.c_double),
                ("muB", C.c_double), ("alpha", C.c_double), ("ceta", C.c_double)]


class _Info(C.Structure):
    _fields_ = [("D", C.c_int), ("N", C.c_int), ("k", C.c_int), ("Np", C.c_int),
                ("n_levels", C.c_int), ("n_cells", C.c_int), ("n_cut_cells", C.c_int),
                ("n_parts", C.c_int), ("n_small", C.c_int), ("n_isolated", C.c_int),
                ("nnzb1", C.c_int64), ("volA", C.c_double), ("volB", C.c_double),
                ("areaI", C.c_double), ("h", C.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        vp = C.c_void_p
        L.xp_build.restype = vp
        L.xp_build.argtypes = [C.POINTER(_Cfg), C.c_char_p, C.c_int]
        L.xp_free.argtypes = [vp]
        L.xp_get_info.argtypes = [vp, C.POINTER(_Info)]
        for name, rt in [("xp_level_rep", C.POINTER(C.c_int32)), ("xp_level_species", C.POINTER(C.c_int8)),
                         ("xp_level_volume", C.POINTER(C.c_double)), ("xp_level_cut", C.POINTER(C.c_int8)),
                         ("xp_agg", C.POINTER(C.c_int32)), ("xp_R", C.POINTER(C.c_double))]:
            getattr(L, name).restype = rt
            getattr(L, name).argtypes = [vp, C.c_int]
        L.xp_level_nb.restype = C.c_int
        L.xp_level_nb.argtypes = [vp, C.c_int]
        L.xp_row_ptr.restype = C.POINTER(C.c_int64)
        L.xp_col.restype = C.POINTER(C.c_int32)
        L.xp_val.restype = C.POINTER(C.c_double)
        L.xp_rhs.restype = C.POINTER(C.c_double)
        for n in ("xp_row_ptr", "xp_col", "xp_val", "xp_rhs"):
            getattr(L, n).argtypes = [vp]
        L.xp_assemble_level.restype = C.c_int
        L.xp_assemble_level.argtypes = [vp, C.c_int, C.POINTER(C.POINTER(C.c_int64)),
                                        C.POINTER(C.POINTER(C.c_int32)), C.POINTER(C.POINTER(C.c_double)),
                                        C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.c_int64)]
        L.xp_release.argtypes = [vp]
        L.xp_l2_error.restype = C.c_int
        L.xp_l2_error.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.xp_block_features.argtypes = [vp, C.POINTER(C.c_double)]
        L.xp_cell_features.argtypes = [vp, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.xp_cut_cells.restype = C.c_int
        L.xp_cut_cells.argtypes = [vp, C.POINTER(C.c_int32)]
        _lib = L
    return _lib


@dataclass
class Config:
    """One synthetic XDG Poisson workload (sphere/circle interface on a Cartesian mesh)."""
    D: int = 2
    N: int = 16
    k: int = 2
    lo: float = 0.0
    hi: float = 1.0
    c: tuple = (0.5, 0.5, 0.5)
    R: float = 0.3
    muA: float = 1.0
    muB: float = 10.0
    alpha: float = 0.1
    ceta: float = 1.0
    rhs_kind: int = 0          # 0: phi*prod cos(pi x)/mu; 1: phi/mu (quadratic); 2: f=1, g_D=0
    max_coarse_dof: int = 2048
    max_levels: int = 16
    quad_q: int = 0
    nthreads: int = 0

    @property
    def Np(self) -> int:
        return math.comb(self.k + self.D, self.D)


# Workload definitions (seeded draws happen in tests/bench through numpy PCG64).
def config_2d_16(**kw) -> Config:
    """2D, unit square, 16^2 cells, circle (0.5,0.5) R=0.3, mu 1 inside / 10 outside, k=2."""
    base = dict(D=2, N=16, k=2, c=(0.5, 0.5, 0.0), R=0.3, muA=1.0, muB=10.0)
    base.update(kw)
    return Config(**base)


def config_3d_64(**kw) -> Config:
    """3D, unit cube, 64^3 cells, sphere centre (0.5,0.5,0.5) R=0.31, mu 1:1000, k=2, alpha=0.1."""
    base = dict(D=3, N=64, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1.0, muB=1000.0, alpha=0.1)
    base.update(kw)
    return Config(**base)


def config_paper_twin(N: int, k: int, alpha: float = 0.1, **kw) -> Config:
    """(-1,1)^3, sphere R=0.7 at the origin, mu 1:1000, f=1, g_D=0 (performance study)."""
    base = dict(D=3, N=N, k=k, lo=-1.0, hi=1.0, c=(0.0, 0.0, 0.0), R=0.7, muA=1.0,
                muB=1000.0, alpha=alpha, rhs_kind=2)
    base.update(kw)
    return Config(**base)


def batch_configs(n: int, seed: int = 20030244, N_range=(32, 128), ks=(2, 3, 4), R_range=(0.1, 0.3),
                  c_range=(0.3, 0.7), log10_mu_range=(0.0, 3.0), max_levels: int = 6) -> list:
    """n independent 2D problems, drawn from numpy PCG64(seed) in this order per problem:
    N ~ U{N_range}, k ~ U(ks), centre ~ U(c_range)^2, R ~ U(R_range), mu_B/mu_A = 10^U(log10_mu_range)
    (mu_A = 1 inside). Every problem gets max_levels aggregation levels (no coarse-size stop),
    so that problems of one block size share the depth of their hierarchy."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        k = int(ks[int(rng.integers(0, len(ks)))])
        cx, cy = (float(v) for v in rng.uniform(c_range[0], c_range[1], size=2))
        R = float(rng.uniform(*R_range))
        mu = float(10.0 ** rng.uniform(*log10_mu_range))
        out.append(Config(D=2, N=N, k=k, c=(cx, cy, 0.0), R=R, muA=1.0, muB=mu, max_coarse_dof=0,
                          max_levels=max_levels))
    return out


class Problem:
    """Assembled agglomerated XDG system plus its aggregation hierarchy (numpy views)."""

    def __init__(self, cfg: Config):
        L = _load()
        self.cfg = cfg
        c = _Cfg(cfg.D, cfg.N, cfg.k, cfg.rhs_kind, cfg.max_coarse_dof, cfg.max_levels,
                 cfg.quad_q, cfg.nthreads, cfg.lo, cfg.hi, (C.c_double * 3)(*cfg.c), cfg.R,
                 cfg.muA, cfg.muB, cfg.alpha, cfg.ceta)
        err = C.create_string_buffer(512)
        h = L.xp_build(C.byref(c), err, 512)
        if not h:
            raise RuntimeError("xdg_problem: " + err.value.decode())
        self._h = C.c_void_p(h)
        self._L = L
        info = _Info()
        L.xp_get_info(self._h, C.byref(info))
        self.info = {f: getattr(info, f) for f, _ in _Info._fields_}
        self.D, self.k, self.Np = info.D, info.k, info.Np
        self.n_levels = info.n_levels
        nb1 = L.xp_level_nb(self._h, 1)
        nnzb = info.nnzb1
        Np = self.Np
        self.row_ptr = np.ctypeslib.as_array(L.xp_row_ptr(self._h), shape=(nb1 + 1,))
        self.col = np.ctypeslib.as_array(L.xp_col(self._h), shape=(max(nnzb, 1),))[:nnzb]
        self.val = np.ctypeslib.as_array(L.xp_val(self._h), shape=(max(nnzb, 1) * Np * Np,))[
            :nnzb * Np * Np].reshape(nnzb, Np, Np)
        self.b = np.ctypeslib.as_array(L.xp_rhs(self._h), shape=(nb1 * Np,)).reshape(nb1, Np)
        self.nb = [L.xp_level_nb(self._h, l) for l in range(1, self.n_levels + 1)]
        self.agg, self.R = [], []
        for l in range(1, self.n_levels):
            n = self.nb[l - 1]
            self.agg.append(np.ctypeslib.as_array(L.xp_agg(self._h, l), shape=(n,)))
            self.R.append(np.ctypeslib.as_array(L.xp_R(self._h, l), shape=(n * Np * Np,)).reshape(n, Np, Np))

    def level_meta(self, level: int) -> dict:
        L, n = self._L, self.nb[level - 1]
        return {
            "rep": np.ctypeslib.as_array(L.xp_level_rep(self._h, level), shape=(n,)).copy(),
            "species": np.ctypeslib.as_array(L.xp_level_species(self._h, level), shape=(n,)).copy(),
            "volume": np.ctypeslib.as_array(L.xp_level_volume(self._h, level), shape=(n,)).copy(),
            "cut": np.ctypeslib.as_array(L.xp_level_cut(self._h, level), shape=(n,)).copy(),
        }

    def schwarz_patches(self, level: int = 1, offset: int = 0, species: str = "both"):
        """Patches of the additive Schwarz smoother on `level` from the background mesh: the
        blocks whose representative cell lies in one group of 2 cells per direction, groups
        shifted by `offset` cells (0 or 1; with 1 the boundary groups hold one cell in that
        direction), both species together (species="both") or one patch per species
        ("each"). Returns (ptr int64[n+1], blocks int32[ptr[n]]), blocks ascending in a patch,
        patches ordered by group then species."""
        meta = self.level_meta(level)
        rep, spc = meta["rep"].astype(np.int64), meta["species"].astype(np.int64)
        N, D = self.cfg.N, self.D
        idx = [(rep // N ** d) % N for d in range(D)]
        # cell coordinates on the level's Cartesian mesh: 2 cells per direction merge per
        # level, an odd trailing cell joining the last group
        n = N
        for _ in range(level - 1):
            idx = [np.minimum(c // 2, max(n // 2 - 1, 0)) for c in idx]
            n = max(n // 2, 1)
        G = n // 2 + 1
        key = np.zeros_like(rep)
        for d in reversed(range(D)):
            key = key * G + (idx[d] + offset) // 2
        if species == "each":
            key = key * 2 + spc
        order = np.lexsort((np.arange(len(rep)), key))
        k_sorted = key[order]
        starts = np.flatnonzero(np.r_[True, k_sorted[1:] != k_sorted[:-1]])
        ptr = np.r_[starts, len(order)].astype(np.int64)
        return ptr, order.astype(np.int32)

    def aggregate_patches(self, level: int = 1):
        """Patches = the children of every block of the next level (the aggregates of the
        aggregation sequence, one species each): (ptr, blocks) as in schwarz_patches."""
        agg = np.asarray(self.agg[level - 1])
        order = np.argsort(agg, kind="stable")
        ptr = np.zeros(self.nb[level] + 1, dtype=np.int64)
        np.add.at(ptr, agg + 1, 1)
        return np.cumsum(ptr), order.astype(np.int32)

    @property
    def dof(self) -> int:
        return self.nb[0] * self.Np

    def assemble_level(self, level: int):
        """Direct assembly of a_sip and b in the basis of `level` (row_ptr, col, val, rhs)."""
        L = self._L
        rp = C.POINTER(C.c_int64)()
        cl = C.POINTER(C.c_int32)()
        vl = C.POINTER(C.c_double)()
        rh = C.POINTER(C.c_double)()
        nnz = C.c_int64()
        if L.xp_assemble_level(self._h, level, C.byref(rp), C.byref(cl), C.byref(vl), C.byref(rh),
                               C.byref(nnz)) != 0:
            raise ValueError("bad level")
        n, Np, z = self.nb[level - 1], self.Np, nnz.value
        out = (np.ctypeslib.as_array(rp, shape=(n + 1,)).copy(),
               np.ctypeslib.as_array(cl, shape=(max(z, 1),))[:z].copy(),
               np.ctypeslib.as_array(vl, shape=(max(z, 1) * Np * Np,))[:z * Np * Np].reshape(z, Np, Np).copy(),
               np.ctypeslib.as_array(rh, shape=(n * Np,)).reshape(n, Np).copy())
        for p in (rp, cl, vl, rh):
            L.xp_release(C.cast(p, C.c_void_p))
        return out

    def l2_error(self, x) -> tuple[float, float]:
        """(||u_h - u||_L2, ||u||_L2) for a level-1 coefficient vector x."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
        e2, n2 = C.c_double(), C.c_double()
        if self._L.xp_l2_error(self._h, x.ctypes.data_as(C.POINTER(C.c_double)), C.byref(e2), C.byref(n2)) != 0:
            raise ValueError("no exact solution for this right-hand side")
        return math.sqrt(e2.value), math.sqrt(n2.value)

    def block_features(self) -> np.ndarray:
        """Per level-1 block: phi/h^2 at the 2^D vertices of the representative cell and the
        volume fractions of A and B in that cell."""
        nv = 1 << self.D
        out = np.zeros((self.nb[0], nv + 2))
        self._L.xp_block_features(self._h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def cut_cells(self) -> np.ndarray:
        """int32 [n_cut, 3]: (cell, level-1 block of the A part, level-1 block of the B part) of
        every background cell that holds both species, ascending cell index."""
        n = self._L.xp_cut_cells(self._h, None)
        out = np.zeros((max(n, 1), 3), np.int32)
        self._L.xp_cut_cells(self._h, out.ctypes.data_as(C.POINTER(C.c_int32)))
        return out[:n]

    def cell_features(self, cells) -> np.ndarray:
        """phi/h^2 at the 2^D vertices and the volume fractions of A and B of the given
        background cells ([len(cells), 2^D + 2])."""
        cells = np.ascontiguousarray(cells, np.int32)
        nv = 1 << self.D
        out = np.zeros((len(cells), nv + 2))
        self._L.xp_cell_features(self._h, len(cells), cells.ctypes.data_as(C.POINTER(C.c_int32)),
                                 out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def learned_units(self):
        """Units of the learned cut-cell correction: the distinct (A block, B block) pairs of
        the cut cells, in order of their first cell, with that cell's geometry features
        [phi / (2 R h) at the 2^D vertices (about the signed distance in cells), volume
        fractions of A and B, log10(mu_B / mu_A) / 3]. Returns (pairs int32 [U][2], geom
        float32 [U][2^D + 3], cells int32 [U])."""
        cc = self.cut_cells()
        seen, pairs, cells = set(), [], []
        for cell, a, b in cc:
            key = (int(a), int(b))
            if key not in seen:
                seen.add(key)
                pairs.append(key)
                cells.append(int(cell))
        pairs = np.array(pairs, np.int32).reshape(-1, 2)
        cells = np.array(cells, np.int32)
        f = self.cell_features(cells)
        nv = 1 << self.D
        h = (self.cfg.hi - self.cfg.lo) / self.cfg.N
        geom = np.zeros((len(cells), nv + 3), np.float32)
        geom[:, :nv] = f[:, :nv] * h / (2.0 * self.cfg.R)
        geom[:, nv:nv + 2] = f[:, nv:nv + 2]
        geom[:, nv + 2] = math.log10(self.cfg.muB / self.cfg.muA) / 3.0
        return pairs, geom, cells

    def close(self):
        if getattr(self, "_h", None):
            self._L.xp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
