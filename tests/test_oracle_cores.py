"""The all-cores harness of the CPU baseline runs the oracle's own routines
on disjoint slices; its combined results equal the single-call oracle's
(exact sums bit for bit through the slices' exact expansions; axpy and the
banded 2-D stencil element for element)."""
import numpy as np

import oracle as O
from oracle import cores
from paper_2106_03219_gb300 import inputs


def test_slices_reproduce_the_single_call_oracle():
    pool = cores.Cores(3)
    try:
        a = inputs.f32_lognormal_signed(100003, 31)
        spec, _ = pool.share(a)
        _, terms = pool.run("exact_terms", [spec], a.size, extra=0)
        assert O.exact_sum_f64(np.concatenate(terms)) == O.exact_sum_f32(a)
        b = inputs.bf16_uniform_pm1(50001, 32)
        spec, _ = pool.share(b)
        _, terms = pool.run("exact_terms", [spec], b.size, extra=1)
        assert O.exact_sum_f64(np.concatenate(terms)) == O.exact_sum_bf16(b)
        x, y = inputs.f32_uniform01(30001, 0), inputs.f32_uniform01(30001, 1)
        sx, _ = pool.share(x)
        sy, vy = pool.share(y)
        pool.run("axpy_f32", [sx, sy], x.size, extra=3.0)
        assert np.array_equal(np.asarray(vy), O.axpy_f32(3.0, x, y))
        g = inputs.grid_f32(37, 52, 5)
        sg, _ = pool.share(g)
        so, vo = pool.share(np.zeros_like(g))
        pool.run("stencil2d", [sg, so], g.shape[0])
        assert np.array_equal(np.asarray(vo), O.stencil2d5(g))
        xi, yi = inputs.int32_uniform(9000, 2), inputs.int32_uniform(9000, 3)
        sxi, _ = pool.share(xi)
        syi, vyi = pool.share(yi)
        _, sums = pool.run("axpy_i32_sum", [sxi, syi], xi.size, extra=3)
        want = O.axpy_i32(3, xi, yi)
        assert np.array_equal(np.asarray(vyi), want)
        assert sum(sums) == O.sum_int(want)
    finally:
        pool.close()
