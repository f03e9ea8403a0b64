"""Pins for the oracle's loop bodies (C6).

Each fp32 operation of a body is recomputed with exact rational arithmetic
(fractions.Fraction) and rounded to the nearest fp32 by a brute-force
nearest-neighbour search, so a dropped term, a wrong sign, a swapped operand
or a different parenthesisation in the oracle fails here.
"""
from fractions import Fraction

import numpy as np

import oracle as O
from paper_2106_03219_gb300 import inputs

F = np.float32


def rnd(fr):
    """Correctly rounded fp32 of an exact rational (ties to even)."""
    c = F(float(fr))
    best, bd = None, None
    for cand in (np.nextafter(c, F(-np.inf)), c, np.nextafter(c, F(np.inf))):
        d = abs(Fraction(float(cand)) - fr)
        if bd is None or d < bd or (d == bd and int(np.array(cand).view(np.uint32)) % 2 == 0):
            best, bd = cand, d
    return F(best)


def q(v):
    return Fraction(float(v))


def test_axpy_f32_exact_rounding():
    x = inputs.f32_uniform01(3000, 0)
    y = inputs.f32_uniform01(3000, 1)
    y[:5] = [1e-30, -0.75, 3e-8, 0.0, -1e-38]
    out = O.axpy_f32(3.0, x, y)
    for i in range(x.size):
        assert out[i] == rnd(3 * q(x[i]) + q(y[i])), i


def test_axpy_f32_other_alpha():
    x = inputs.f32_uniform_pm1(500, 2)
    y = inputs.f32_uniform_pm1(500, 3)
    out = O.axpy_f32(-0.3, x, y)
    a = q(F(-0.3))
    for i in range(x.size):
        assert out[i] == rnd(a * q(x[i]) + q(y[i]))


def test_axpy_i32_wraps():
    x = inputs.int32_uniform(4000, 0)
    y = inputs.int32_uniform(4000, 1)
    x[:4] = [2 ** 31 - 1, -2 ** 31, 2 ** 30, -7]
    y[:4] = [5, -1, 2 ** 31 - 1, 2 ** 31 - 1]
    out = O.axpy_i32(3, x, y)
    for i in range(x.size):
        v = (3 * int(x[i]) + int(y[i])) % (1 << 32)
        v = v - (1 << 32) if v >= (1 << 31) else v
        assert int(out[i]) == v


def stencil1d_exact(a, c0, c1):
    out = np.empty_like(a)
    n = a.size
    for i in range(n):
        if i == 0 or i == n - 1:
            out[i] = a[i]
        else:
            nb = rnd(q(a[i - 1]) + q(a[i + 1]))
            ce = rnd(q(c0) * q(a[i]))
            out[i] = rnd(q(c1) * q(nb) + q(ce))
    return out


def stencil2d_exact(a, c0, c1):
    ny, nx = a.shape
    out = np.empty_like(a)
    for r in range(ny):
        for c in range(nx):
            if r in (0, ny - 1) or c in (0, nx - 1):
                out[r, c] = a[r, c]
                continue
            ns = rnd(q(a[r - 1, c]) + q(a[r + 1, c]))
            ew = rnd(q(a[r, c + 1]) + q(a[r, c - 1]))
            s = rnd(q(ns) + q(ew))
            ce = rnd(q(c0) * q(a[r, c]))
            out[r, c] = rnd(q(c1) * q(s) + q(ce))
    return out


def test_stencil1d_exact():
    a = inputs.f32_uniform01(700, 4)
    assert np.array_equal(O.stencil1d3(a), stencil1d_exact(a, F(0.5), F(0.125)))
    b = inputs.f32_lognormal_signed(300, 5)
    assert np.array_equal(O.stencil1d3(b, 0.3, 0.7), stencil1d_exact(b, F(0.3), F(0.7)))


def test_stencil2d_exact_non_square():
    a = inputs.grid_f32(13, 29, 6)       # ny != nx: a transposed index fails
    assert np.array_equal(O.stencil2d5(a), stencil2d_exact(a, F(0.5), F(0.125)))
    b = inputs.f32_lognormal_signed(17 * 11, 7).reshape(17, 11)
    assert np.array_equal(O.stencil2d5(b, 0.25, 0.3), stencil2d_exact(b, F(0.25), F(0.3)))


def test_stencil_fixed_points():
    # with c0 = 1/2, c1 = 1/8 a 2-D field that is linear in (row, col) with
    # small integer values is reproduced exactly at every interior point
    # (1/8 * 4f + 1/2 * f = f), and the boundary is copied: output == input.
    r, c = np.meshgrid(np.arange(37), np.arange(23), indexing="ij")
    lin = (3 * r - 2 * c + 100).astype(F)
    assert np.array_equal(O.stencil2d5(lin), lin)
    # in 1-D the same weights give 1/8 * 2f + 1/2 * f = 3/4 f on a linear field
    line = (4 * np.arange(101) - 40).astype(F)
    out = O.stencil1d3(line)
    assert out[0] == line[0] and out[-1] == line[-1]
    assert np.array_equal(out[1:-1], (0.75 * line[1:-1]).astype(F))
    # a point source spreads 1/8 to each neighbour and keeps 1/2
    d = np.zeros((5, 5), F)
    d[2, 2] = 8.0
    out = O.stencil2d5(d)
    assert out[2, 2] == 4.0 and out[1, 2] == out[3, 2] == out[2, 1] == out[2, 3] == 1.0
    assert out.sum() == 8.0


def test_stencil_degenerate_shapes():
    for shape in [(1, 1), (1, 7), (7, 1), (2, 2), (2, 9), (3, 3)]:
        a = inputs.f32_uniform01(shape[0] * shape[1], 8).reshape(shape)
        out = O.stencil2d5(a)
        assert np.array_equal(out, stencil2d_exact(a, F(0.5), F(0.125)))
    for n in (1, 2, 3):
        a = inputs.f32_uniform01(n, 9)
        assert np.array_equal(O.stencil1d3(a), stencil1d_exact(a, F(0.5), F(0.125)))
