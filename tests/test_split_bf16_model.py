"""The split-operand scheme behind the tensor-core layers of the learned correction's inference
(k_unit_apply): an FP32 activation v is split into three BF16 numbers hi = bf16(v),
mid = bf16(v - hi), lo = bf16(v - hi - mid), and each hidden layer sums the products of the
three parts with the BF16 weights in FP32 accumulators.

Modelled exactly on the host (BF16 rounding = round to nearest even on the upper 16 bits of the
FP32 pattern; products and sums in float64 or exact rationals): the three parts sum to v
exactly for normal FP32 v, every product of a part with a BF16 weight is exact in FP32, so the
only rounding left is the FP32 accumulation itself -- the same as in the FP32 FMA chain the
layers replace. With two parts the residual would be up to 2^-17 |v| per activation, which a
test asserting FP32-level agreement would see."""
from fractions import Fraction

import numpy as np


def bf16(x):
    """Round float32 values to BF16 (nearest, ties to even), returned as float32."""
    x = np.asarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32)


def split3(v):
    v = np.asarray(v, dtype=np.float32)
    hi = bf16(v)
    r1 = (v - hi).astype(np.float32)
    mid = bf16(r1)
    lo = bf16((r1 - mid).astype(np.float32))
    return hi, mid, lo


def test_bf16_rounding_model():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.1415927, 65504.0], dtype=np.float32)
    r = bf16(x)
    # 1 + 2^-8 is the midpoint of 1 and 1 + 2^-7: ties to even gives 1
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == np.float32(1.0078125)
    assert abs(float(r[3]) + 3.140625) == 0.0
    # a BF16 number has at most 8 significant bits
    m, _ = np.frexp(r.astype(np.float64))
    assert np.all(m * 256 == np.round(m * 256))


def test_three_parts_sum_to_the_value_exactly():
    rng = np.random.default_rng(5)
    v = (rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    hi, mid, lo = split3(v)
    for p in (hi, mid, lo):
        assert np.array_equal(bf16(p), p)  # each part is a BF16 number
    s = hi.astype(np.float64) + mid.astype(np.float64) + lo.astype(np.float64)
    assert np.array_equal(s, v.astype(np.float64))
    # two parts leave up to about 2^-17 |v|
    two = hi.astype(np.float64) + mid.astype(np.float64)
    rel = np.abs(two - v) / np.abs(v)
    assert rel.max() > 2.0 ** -20 and rel.max() <= 2.0 ** -16


def test_products_with_bf16_weights_are_exact_in_fp32():
    rng = np.random.default_rng(6)
    v = rng.standard_normal(50000).astype(np.float32)
    w = bf16(rng.standard_normal(50000).astype(np.float32))
    for p in split3(v):
        prod64 = p.astype(np.float64) * w.astype(np.float64)
        assert np.array_equal(prod64.astype(np.float32).astype(np.float64), prod64)


def test_split_dot_matches_the_exact_dot_to_fp32_accumulation():
    """A 64-term layer sum: the sum of the 3 x 64 exact partial products equals the exact dot
    product of the FP32 activations and BF16 weights (checked in rationals); summed in FP32
    it is as close to the exact value as the FP32 FMA chain of the same terms."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        v = rng.standard_normal(64).astype(np.float32)
        w = bf16(rng.standard_normal(64).astype(np.float32))
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(v, w))
        parts = split3(v)
        split_exact = sum(Fraction(float(p[i])) * Fraction(float(w[i])) for p in parts for i in range(64))
        assert split_exact == exact
        acc = np.float32(0.0)
        for p in parts[::-1]:  # the kernel adds the small parts first
            for i in range(64):
                acc = np.float32(acc + np.float32(p[i] * w[i]))
        fma = np.float32(0.0)
        for i in range(64):
            fma = np.float32(float(fma) + float(v[i]) * float(w[i]))  # one rounding per step, as an FMA
        scale = float(np.sum(np.abs(v.astype(np.float64) * w)))
        err_split = abs(float(acc) - float(exact)) / scale
        err_fma = abs(float(fma) - float(exact)) / scale
        assert err_split <= 200 * 2.0 ** -24 and err_fma <= 100 * 2.0 ** -24
