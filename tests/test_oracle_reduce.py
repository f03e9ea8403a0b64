"""Pins for the oracle's reductions (C7).

The exact-sum oracle (a long fixed-point accumulator) is checked against
Python's math.fsum, which returns the correctly rounded sum of its doubles
(Shewchuk's algorithm): an independent library routine.  Integer sums are
checked against Python big integers reduced mod 2^64.
"""
import math
import random

import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs


def fsum32(a):
    return math.fsum(np.asarray(a, dtype=np.float32).astype(np.float64).tolist())


@pytest.mark.parametrize("gen", ["pm1", "lognormal", "uniform01"])
def test_exact_sum_vs_fsum(gen):
    n = 1 << 16
    a = {"pm1": inputs.f32_uniform_pm1, "lognormal": inputs.f32_lognormal_signed,
         "uniform01": inputs.f32_uniform01}[gen](n, 3)
    assert O.exact_sum_f32(a) == fsum32(a)


def test_exact_sum_vs_fsum_million_slice():
    a = inputs.f32_uniform_pm1(1 << 20, 0)
    assert O.exact_sum_f32(a) == fsum32(a)


def test_exact_sum_order_independent():
    a = inputs.f32_lognormal_signed(50000, 11)
    ref = O.exact_sum_f32(a)
    rng = np.random.default_rng(0)
    for _ in range(3):
        b = a.copy()
        rng.shuffle(b)
        assert O.exact_sum_f32(b) == ref


def test_exact_sum_hand_cases():
    f = np.float32
    assert O.exact_sum_f32(np.array([1e8, 1, -1e8], f)) == 1.0
    assert O.exact_sum_f32(np.array([], f)) == 0.0
    # ties to even: 1 + 2^-53 rounds to 1; 1 + 3*2^-53 rounds up to 1 + 2^-51
    assert O.exact_sum_f32(np.array([1.0, 2.0 ** -53], f)) == 1.0
    assert O.exact_sum_f32(np.array([1.0, 2.0 ** -53, 2.0 ** -52], f)) == 1.0 + 2.0 ** -51
    # just above the tie rounds up
    assert O.exact_sum_f32(np.array([1.0, 2.0 ** -53, 2.0 ** -80], f)) == 1.0 + 2.0 ** -52
    # subnormals and the top of the range
    tiny = np.float32(1e-45)
    assert O.exact_sum_f32(np.array([tiny, tiny, -tiny], f)) == float(tiny)
    big = np.float32(3e38)
    assert O.exact_sum_f32(np.array([big, big, big, -big], f)) == 2 * float(big)
    # exact cancellation to zero
    a = inputs.f32_uniform_pm1(1000, 1)
    assert O.exact_sum_f32(np.concatenate([a, -a])) == 0.0


def test_exact_sum_mixed_dynamic_range():
    rng = np.random.default_rng(9)
    e = rng.integers(-149, 127, size=20000)
    m = rng.uniform(1.0, 2.0, size=20000) * np.where(rng.random(20000) < 0.5, -1, 1)
    a = np.ldexp(m, e).astype(np.float32)
    a = a[np.isfinite(a)]
    assert O.exact_sum_f32(a) == fsum32(a)


def test_exact_dot_vs_fsum():
    x = inputs.f32_uniform01(30000, 0)
    y = inputs.f32_uniform01(30000, 1)
    ref = math.fsum((x.astype(np.float64) * y.astype(np.float64)).tolist())
    assert O.exact_dot_f32(x, y) == ref
    # extreme products: subnormal x subnormal and near-overflow squared
    x = np.array([1e-45, 3e38, -3e38, 1.0], np.float32)
    y = np.array([1e-45, 3e38, 3e38, 2.0 ** -149], np.float32)
    ref = math.fsum((x.astype(np.float64) * y.astype(np.float64)).tolist())
    assert O.exact_dot_f32(x, y) == ref


def test_exact_sum_bf16_vs_fsum():
    bits = inputs.bf16_uniform_pm1(40000, 2)
    vals = (bits.astype(np.uint32) << 16).view(np.float32)
    assert O.exact_sum_bf16(bits) == fsum32(vals)


def test_exact_sum_f64_combine():
    rng = random.Random(4)
    vals = [rng.uniform(-1e6, 1e6) for _ in range(5000)]
    assert O.exact_sum_f64(np.array(vals)) == math.fsum(vals)


def test_abs_sum():
    a = inputs.f32_uniform_pm1(10000, 5)
    assert O.exact_abs_sum_f32(a) == math.fsum(np.abs(a.astype(np.float64)).tolist())


def test_int_sums_wrap():
    a = inputs.int64_uniform(10000, 3)
    assert O.sum_int(a) == sum(int(v) for v in a)
    big = np.array([(1 << 63) - 1, 5, (1 << 63) - 2, -(1 << 63)], np.int64)
    s = sum(int(v) for v in big) % (1 << 64)
    s = s - (1 << 64) if s >= (1 << 63) else s
    assert O.sum_int(big) == s
    x = inputs.int32_uniform(10000, 0)
    assert O.sum_int(x) == sum(int(v) for v in x)


def test_max_min():
    for a in (inputs.f32_uniform_pm1(5000, 1), inputs.f32_lognormal_signed(5000, 2)):
        assert O.max_min(a, "max") == float(max(a.tolist()))
        assert O.max_min(a, "min") == float(min(a.tolist()))
    b = inputs.int64_uniform(5000, 3)
    assert O.max_min(b, "max") == max(b.tolist())
    assert O.max_min(b, "min") == min(b.tolist())
    c = inputs.int32_uniform(5000, 4)
    assert O.max_min(c, "max") == max(c.tolist())
    assert O.max_min(c, "min") == min(c.tolist())


def test_max_min_one_sided_single_and_empty():
    """Arrays entirely below zero (max) or above zero (min), single elements at
    the type's extremes, and the empty array, whose result is the identity of
    the operation in the result's type (OpenMP's initializer for max / min:
    the least / greatest value of the reduction item's type; integer data
    reduce into an int64 result, fp32 data into a double)."""
    f = np.abs(inputs.f32_uniform_pm1(3000, 5)) + np.float32(0.25)
    for a in (f, -f):
        assert O.max_min(a, "max") == float(max(a.tolist()))
        assert O.max_min(a, "min") == float(min(a.tolist()))
    for dt, lo, hi in ((np.int32, -(1 << 31), (1 << 31) - 1), (np.int64, -(1 << 63), (1 << 63) - 1)):
        pos = np.abs(inputs.int32_uniform(3000, 6)).astype(dt) + 1
        for a in (pos, -pos):
            assert O.max_min(a, "max") == max(a.tolist())
            assert O.max_min(a, "min") == min(a.tolist())
        for v in (lo, hi, -1, 1):
            one = np.array([v], dt)
            assert O.max_min(one, "max") == v and O.max_min(one, "min") == v
        empty = np.zeros(0, dt)
        assert O.max_min(empty, "max") == -(1 << 63) and O.max_min(empty, "min") == (1 << 63) - 1
    one = np.array([-3.5], np.float32)
    assert O.max_min(one, "max") == -3.5 and O.max_min(one, "min") == -3.5
    empty = np.zeros(0, np.float32)
    assert O.max_min(empty, "max") == float("-inf") and O.max_min(empty, "min") == float("inf")


def test_plain_sum_pins():
    """The plain fp64 loop (the CPU speed reference for the reductions, not the
    oracle of a GPU result): left to right, each fp32 value widened exactly
    and added with one fp64 rounding.
    * Integer-valued data whose partial sums stay below 2^53 are summed
      exactly, so the result equals the correctly rounded sum (math.fsum).
    * Order: [2^54, -2^54, 1, 1, 1] is 3 left to right; right to left the
      partial 3 - 2^54 rounds to 4 - 2^54 (spacing 2, ties to even) and the
      result is 4.
    * Accumulator width: [1, 1, 1, 1, 2^54, -2^54] is 4 in fp64 (2^54 + 4 is a
      double); an fp32 accumulator would round 2^54 + 4 to 2^54 and return 0.
    * Error bound of recursive summation: |plain - exact| <= (n - 1) u sum|x|
      with u = 2^-53 (first order in n u, n u << 1 here)."""
    f = np.float32
    a = np.arange(-5000, 7000, 3, dtype=f)
    assert O.plain_sum_f32(a) == fsum32(a)
    assert O.plain_sum_f32(np.array([2.0 ** 54, -2.0 ** 54, 1, 1, 1], f)) == 3.0
    assert O.plain_sum_f32(np.array([1, 1, 1, 1, 2.0 ** 54, -2.0 ** 54], f)) == 4.0
    assert O.plain_sum_f32(np.array([], f)) == 0.0
    for gen in (inputs.f32_uniform_pm1, inputs.f32_lognormal_signed):
        x = gen(100000, 21)
        err = abs(O.plain_sum_f32(x) - O.exact_sum_f32(x))
        assert err <= (x.size - 1) * 2.0 ** -53 * O.exact_abs_sum_f32(x)


def test_exact_sum_terms_split_across_slices():
    """The expansion of each slice's exact sum: its terms add up exactly
    (math.fsum) to the slice's correctly rounded sum's exact value, the first
    term is that rounded sum, terms do not overlap (each below half an ulp
    of the one before), and the terms of disjoint slices summed by the
    oracle's exact fp64 sum give the whole array's exact sum."""
    for gen, bf in ((inputs.f32_lognormal_signed, False), (inputs.f32_uniform_pm1, False),
                    (inputs.bf16_uniform_pm1, True)):
        a = gen(200003, 23)
        whole = O.exact_sum_bf16(a) if bf else O.exact_sum_f32(a)
        vals = (a.astype(np.uint32) << 16).view(np.float32) if bf else a
        cuts = [0, 1, 5000, 77777, 150000, a.size]
        terms = []
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            t = O.exact_sum_terms(a[lo:hi], bf16=bf)
            assert t.size >= 1
            assert t[0] == fsum32(vals[lo:hi])
            for u, v in zip(t[:-1], t[1:]):
                assert abs(v) <= math.ulp(u) / 2
            terms.extend(t.tolist())
        assert O.exact_sum_f64(np.array(terms)) == whole
        assert math.fsum(terms) == whole
    # a sum that needs more than one term: 1 + 2^-60 (fp32 values)
    t = O.exact_sum_terms(np.array([1.0, 2.0 ** -60], np.float32))
    assert t.tolist() == [1.0, 2.0 ** -60]
    assert O.exact_sum_terms(np.array([], np.float32)).size == 0
    assert O.exact_sum_terms(np.array([3.0, -3.0], np.float32)).size == 0
