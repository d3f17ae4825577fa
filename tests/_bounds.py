"""Element-wise comparisons of the CUDA path with the FP64 oracle.

Both sides compute the same FP64 expressions in different summation orders (and the GPU with
fused multiply-adds). For one product, entry i of M x then differs by at most about
2 n 2^-53 (|M||x|)_i, n the number of terms of the entry's sum (the classical bound
gamma_n = n u / (1 - n u) for a dot product, on each side); restriction, prolongation and one
smoothing step are short chains of such products and get the same kind of bound, with the
magnitudes carried through the chain on absolute values (computed here with the oracle's own
products on |M|, |R| and numpy for the dense per-block pieces). The comparison is entry by
entry, so that a wrong entry of a small-magnitude block row cannot hide under the norm of the
large ones.

A whole multigrid cycle cancels too much for such a running bound to mean anything (carried
through |I - omega D^-1 M| and the coarse inverses on absolute values, it exceeds the result
by many orders of magnitude), so cycles are compared block by block: the largest difference in
a block relative to that block's largest entry.
"""
import numpy as np

import oracle

U = 2.0 ** -53


def abs_apply(rp, col, val, x):
    """(|M||x|) for a BSR operator."""
    return oracle.bsr_spmv(rp, col, np.abs(val), np.abs(np.asarray(x).reshape(-1))).reshape(-1)


def row_terms(rp, Np):
    """Terms of the longest row sum of a BSR operator (blocks per row times Np)."""
    return int(np.max(np.diff(rp))) * Np


def diag_blocks(rp, col, val):
    nb = len(rp) - 1
    D = np.empty((nb,) + val.shape[1:])
    for i in range(nb):
        z = rp[i] + int(np.searchsorted(col[rp[i]:rp[i + 1]], i))
        D[i] = val[z]
    return D


def check(got, ref, bound, what=""):
    """|got_i - ref_i| <= bound_i for every entry (reports the count and the worst ratio)."""
    got, ref, bound = (np.asarray(a).reshape(-1) for a in (got, ref, bound))
    err = np.abs(got - ref)
    bad = err > bound
    assert not bad.any(), (what, int(bad.sum()), float(np.max(err / np.maximum(bound, 1e-300))))


def check_blocks(got, ref, Np, tol, what=""):
    """max_{i in block} |got_i - ref_i| <= tol max_{i in block} |ref_i| for every block."""
    d = np.abs(np.asarray(got).reshape(-1, Np) - np.asarray(ref).reshape(-1, Np)).max(axis=1)
    m = np.abs(np.asarray(ref).reshape(-1, Np)).max(axis=1)
    bad = d > tol * m
    assert not bad.any(), (what, int(bad.sum()), float(np.max(d / np.maximum(m, 1e-300))))


def apply_bound(rp, col, val, x):
    """Entry-wise bound on the difference of two FP64 evaluations of M x."""
    return 2 * (row_terms(rp, val.shape[-1]) + 2) * U * abs_apply(rp, col, val, x)


def restrict_bound(rp, col, val, agg, R, b, x, nbc):
    """Entry-wise bound for R^T (b - M x) (x None: R^T b)."""
    Np = R.shape[-1]
    mag = np.abs(np.asarray(b).reshape(-1))
    terms = 2
    if x is not None:
        mag = mag + abs_apply(rp, col, val, x)
        terms += row_terms(rp, Np)
    kids = int(np.max(np.bincount(np.asarray(agg), minlength=nbc)))
    out = oracle.restrict(agg, np.abs(R), mag, nbc).reshape(-1)
    return 2 * (terms + kids * Np + 2) * U * out


def prolong_bound(agg, R, zc, x):
    """Entry-wise bound for x + R zc."""
    Np = R.shape[-1]
    m = oracle.prolong_add(agg, np.abs(R), np.abs(zc), np.abs(x)).reshape(-1)
    return 2 * (Np + 2) * U * m


class SmoothBound:
    """Bound for one damped block-Jacobi step x + omega D^{-1} (b - M x) on a level.

    The residual is a product with |M|-magnitudes as above. The block solve is a Cholesky
    substitution on one side and a product with an explicit inverse (from the Cholesky factor)
    on the other; both have componentwise error at most c Np u |D^-1| |L| |L^T| |D^-1| |r|
    (Higham, Accuracy and Stability of Numerical Algorithms: componentwise backward error of
    Cholesky solves and of the inverse), which this bound adds per block."""

    def __init__(self, lv):
        self.lv = lv
        D = diag_blocks(lv["row_ptr"], lv["col"], lv["val"])
        self.Np = D.shape[-1]
        Di = np.abs(np.linalg.inv(D))
        Lf = np.abs(np.linalg.cholesky(D))
        self.Di = Di
        self.G = Di @ (Lf @ np.swapaxes(Lf, 1, 2)) @ Di

    def _blk(self, T, v):
        return np.einsum("bij,bj->bi", T, np.asarray(v).reshape(-1, self.Np)).reshape(-1)

    def __call__(self, omega, b, x):
        lv, Np = self.lv, self.Np
        b = np.abs(np.asarray(b).reshape(-1))
        x = np.abs(np.asarray(x).reshape(-1))
        m_r = b + abs_apply(lv["row_ptr"], lv["col"], lv["val"], x)
        E_r = (row_terms(lv["row_ptr"], Np) + 2) * m_r
        m_c = omega * self._blk(self.Di, m_r)
        E = omega * self._blk(self.Di, E_r) + 4 * Np * omega * self._blk(self.G, m_r) + (Np + 2) * m_c + x + m_c
        return 2 * U * E
