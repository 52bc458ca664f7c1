"""The arithmetic of the tensor-core product (h2mg_apply_ex with TF32X3), on the CPU.

Each FP32 operand a is split into a head h = tf32(a) (11 significant bits, rounded to
nearest with ties away from zero: add half a unit of the 13 dropped bits to the bit
pattern and clear them) and a tail t = tf32(a - h); a b is formed as h_a h_b + h_a t_b +
t_a h_b. Pinned here against float64: the head is the nearest 11-bit value (error at most
2^-11 |a|); the head plus the tail recover a to 2^-22 |a|;
each product is within 2^-20 |a b| (the dropped t_a t_b is at most 2^-22 |a b|, the
roundings of the tails at most 2^-22 |a b| each); and a 64-term dot product of three
split products, summed in float64, is within 2^-20 sum |a_i b_i|.
"""
import numpy as np


def tf32(v):
    v = np.asarray(v, dtype=np.float32)
    b = v.view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def split(v):
    v = np.asarray(v, dtype=np.float32)
    h = tf32(v)
    return h, tf32(v - h)


def values(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) * 10.0 ** rng.integers(-8, 8, n)).astype(np.float32)


def test_head_is_a_rounded_tf32_value():
    v = values(200000, 1)
    h = tf32(v)
    assert not (h.view(np.uint32) & np.uint32(0x1FFF)).any()
    m, e = np.frexp(v.astype(np.float64))
    # the nearest 11-bit value, ties away from zero
    ref = np.sign(m) * np.floor(np.abs(m) * 2.0 ** 11 + 0.5) * 2.0 ** (e - 11)
    assert np.array_equal(h.astype(np.float64), ref)
    assert np.all(np.abs(v.astype(np.float64) - h) <= 2.0 ** -11 * np.abs(v.astype(np.float64)))


def test_head_and_tail_recover_the_value():
    v = values(200000, 2)
    h, t = split(v)
    err = np.abs(v.astype(np.float64) - h.astype(np.float64) - t.astype(np.float64))
    assert np.all(err <= 2.0 ** -22 * np.abs(v.astype(np.float64)))
    assert np.all(np.abs(t.astype(np.float64)) <= 2.0 ** -11 * np.abs(v.astype(np.float64)))


def test_three_products_reach_fp32_accuracy():
    a, b = values(200000, 3), values(200000, 4)
    ha, ta = (x.astype(np.float64) for x in split(a))
    hb, tb = (x.astype(np.float64) for x in split(b))
    exact = a.astype(np.float64) * b.astype(np.float64)
    approx = ha * hb + ha * tb + ta * hb
    assert np.all(np.abs(approx - exact) <= 2.0 ** -20 * np.abs(exact))
    # dropping the tails (one TF32 product) is far coarser
    assert np.max(np.abs(ha * hb - exact) / np.abs(exact)) > 2.0 ** -13


def test_split_dot_products():
    rng = np.random.default_rng(5)
    for _ in range(200):
        a = rng.standard_normal(64).astype(np.float32)
        b = rng.standard_normal(64).astype(np.float32)
        ha, ta = (x.astype(np.float64) for x in split(a))
        hb, tb = (x.astype(np.float64) for x in split(b))
        exact = float(a.astype(np.float64) @ b.astype(np.float64))
        approx = float(ha @ hb + ha @ tb + ta @ hb)
        scale = float(np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64)))
        assert abs(approx - exact) <= 2.0 ** -20 * scale
