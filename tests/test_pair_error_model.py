"""Host check of the error bound that tests/test_gpu_pair.py asserts for the FP32-pair apply.

The pair product's arithmetic (per-block power-of-two scaling, hi + lo split of every operator
and vector entry, Dekker's exact product, the cross terms folded into its error, Knuth's
TwoSum over a block row, the errors summed in FP32, each block's hi and lo scaled back and
added in FP64) is written out here step by step in exact rational arithmetic, with every FP32
and FP64 operation rounded to nearest-even explicitly. Its result is compared with the exact
row sums for random, wide-range and cancelling inputs:

    |y_model - y_exact|_i <= ((9 + 2 Np^2) u^2 + 64 * 2^-53) (|M||x|)_i,   u = 2^-24

and the same model with one step left out (the cross terms, or the TwoSum error) must break the
bound on some of these inputs, so the bound is tight enough to catch such a mistake on the GPU.
No GPU and no code of the CUDA path: the model is written from the arithmetic it describes.
"""
from fractions import Fraction as F

import numpy as np
import pytest

U2 = 2.0 ** -48


def fl32(q):
    """q (exact rational) rounded to the nearest FP32 number, ties to even (no overflow here)."""
    if q == 0:
        return 0.0
    sign = -1.0 if q < 0 else 1.0
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if F(2) ** e > q:
        e -= 1
    ulp = max(e - 23, -149)
    scaled = q / F(2) ** ulp
    n = scaled.numerator // scaled.denominator
    r = scaled - n
    if r > F(1, 2) or (r == F(1, 2) and n % 2 == 1):
        n += 1
    return sign * float(n) * 2.0 ** ulp


def fl64(q):
    """q rounded to the nearest FP64 number (Python's conversion rounds to nearest-even)."""
    return float(q)


def exponent(m):
    """e with m = f 2^e, f in [0.5, 1) (0 for m = 0)."""
    return 0 if m == 0 else int(np.frexp(m)[1])


def split(v, k):
    vs = v * 2.0 ** -k  # exact: a power-of-two scaling of a normal double
    h = fl32(F(vs))
    return h, fl32(F(vs) - F(h))


def block_dot(a, x, cross=True, twosum_err=True):
    """sum_c a[c] x[c] for pairs a[c] = (hi, lo), x[c] = (hi, lo); returns (hi, lo) in FP32."""
    s = c = 0.0
    for (ah, al), (xh, xl) in zip(a, x):
        p = fl32(F(ah) * F(xh))
        e = fl32(F(ah) * F(xh) - F(p))  # exact: the product's rounding error
        if cross:
            e = fl32(F(ah) * F(xl) + F(e))
            e = fl32(F(al) * F(xh) + F(e))
        t = fl32(F(s) + F(p))
        bp = fl32(F(t) - F(s))
        e2 = fl32(F(fl32(F(s) - F(fl32(F(t) - F(bp))))) + F(fl32(F(p) - F(bp))))
        s = t
        c = fl32(F(c) + F(fl32(F(e) + F(e2)) if twosum_err else F(e)))
    return s, c


def pair_apply_row(blocks, xs, r, **kw):
    """Row r of sum_z M_z x_z over the blocks of one block row (FP64 blocks, FP64 x blocks)."""
    acc = 0.0
    for Mz, xz in zip(blocks, xs):
        ka, kx = exponent(np.abs(Mz).max()), exponent(np.abs(xz).max())
        a = [split(v, ka) for v in Mz[r]]
        xv = [split(v, kx) for v in xz]
        hi, lo = block_dot(a, xv, **kw)
        acc = fl64(F(hi) * F(2) ** (ka + kx) + F(acc))
        acc = fl64(F(lo) * F(2) ** (ka + kx) + F(acc))
    return acc


def exact_row(blocks, xs, r):
    return sum((F(float(a)) * F(float(b)) for Mz, xz in zip(blocks, xs) for a, b in zip(Mz[r], xz)), F(0))


def magnitude_row(blocks, xs, r):
    return float(sum(float(abs(a) * abs(b)) for Mz, xz in zip(blocks, xs) for a, b in zip(Mz[r], xz)))


def cases(Np, rng):
    nblk = 7
    out = []
    for kind in ("random", "wide", "cancel"):
        blocks = [rng.standard_normal((Np, Np)) for _ in range(nblk)]
        xs = [rng.standard_normal(Np) for _ in range(nblk)]
        if kind == "wide":  # block magnitudes over 2^+-300
            blocks = [B * 2.0 ** int(rng.integers(-300, 301)) for B in blocks]
            xs = [x * 2.0 ** int(rng.integers(-300, 301)) for x in xs]
        if kind == "cancel":  # a row sum far below sum |a||x|: the last block cancels the rest
            xs = [np.ones(Np) + 1e-9 * rng.standard_normal(Np) for _ in range(nblk)]
            tot = sum(B for B in blocks[:-1])
            blocks[-1] = -tot + 1e-10 * rng.standard_normal((Np, Np))
        out.append((kind, blocks, xs))
    return out


@pytest.mark.parametrize("Np", [6, 10])
def test_pair_model_within_bound(Np):
    rng = np.random.default_rng(100 + Np)
    bound_c = (9 + 2 * Np ** 2) * U2 + 64 * 2.0 ** -53
    for kind, blocks, xs in cases(Np, rng):
        for r in range(Np):
            y = pair_apply_row(blocks, xs, r)
            err = abs(F(y) - exact_row(blocks, xs, r))
            mag = magnitude_row(blocks, xs, r)
            assert float(err) <= bound_c * mag, (kind, r, float(err) / mag)


def test_bound_catches_a_dropped_step():
    """Leaving out the cross terms (or TwoSum's error) breaks the bound on these inputs."""
    Np = 6
    rng = np.random.default_rng(7)
    bound_c = (9 + 2 * Np ** 2) * U2 + 64 * 2.0 ** -53
    for kw in (dict(cross=False), dict(twosum_err=False)):
        worst = 0.0
        for kind, blocks, xs in cases(Np, rng):
            for r in range(Np):
                y = pair_apply_row(blocks, xs, r, **kw)
                err = abs(F(y) - exact_row(blocks, xs, r))
                worst = max(worst, float(err) / (bound_c * magnitude_row(blocks, xs, r)))
        assert worst > 1.0, (kw, worst)
