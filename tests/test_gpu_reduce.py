"""GPU parity: reductions.  Integer sums and max/min bit-exact; fp32 / bf16
sums within 1e-6 of the exact sum rounded to fp64 (relative to
max(|exact|, 2^-24 sum|x|)); bit-identical results run to run."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import dev, fp_sum_ok, host

pytestmark = pytest.mark.gpu


def _res(dtype="f64"):
    import torch
    return torch.zeros(1, dtype=torch.float64 if dtype == "f64" else torch.int64, device="cuda")


def _bf16_dev(bits):
    import torch
    return dev(bits.view(np.int16)).view(torch.bfloat16)


GT = [(1, 32), (3, 96), (608, 512), (152, 1024), (16384, 64)]


@pytest.mark.parametrize("n", [0, 1, 7, 1000, (1 << 20) + 5])
@pytest.mark.parametrize("G,T", GT)
def test_fp32_sum_small(rt, n, G, T):
    a = inputs.f32_lognormal_signed(n, 2)
    r = _res()
    rt.reduce(R.OP_SUM, dev(a), r, R.PREC_COMP_F64, G, T)
    ok, err, bound = fp_sum_ok(float(host(r)[0]), O.exact_sum_f32(a), O.exact_abs_sum_f32(a))
    assert ok, (err, bound)


@pytest.mark.parametrize("n", [0, 1, 9, 1000, (1 << 20) + 3])
@pytest.mark.parametrize("G,T", GT)
def test_int_sums_exact(rt, n, G, T):
    a64 = inputs.int64_uniform(n, 3)
    a32 = inputs.int32_uniform(n, 4)
    for a in (a64, a32):
        r = _res("i64")
        rt.reduce(R.OP_SUM, dev(a), r, 0, G, T)
        assert int(host(r)[0]) == O.sum_int(a)


@pytest.mark.parametrize("n", [1, 9, 1000, (1 << 20) + 3])
def test_max_min_exact(rt, n):
    for a in (inputs.f32_uniform_pm1(n, 1), inputs.f32_lognormal_signed(n, 2),
              inputs.int64_uniform(n, 3), inputs.int32_uniform(n, 4)):
        for op, name in ((R.OP_MAX, "max"), (R.OP_MIN, "min")):
            r = _res("f64" if a.dtype == np.float32 else "i64")
            rt.reduce(op, dev(a), r, 0, 37, 256)
            assert host(r)[0] == O.max_min(a, name)


@pytest.mark.parametrize("G,T", [(1, 32), (37, 256), (608, 512)])
def test_max_min_one_sided_and_empty(rt, G, T):
    """Arrays entirely below zero under max and above zero under min (a wrong
    starting value shows there), and n = 0, whose result is the identity in
    the result's type: -inf / +inf (fp32 data, double result),
    INT64_MIN / INT64_MAX (int32 and int64 data, int64 result).  The result
    buffer starts at a sentinel, so the launch must write it."""
    import torch
    f = np.abs(inputs.f32_uniform_pm1(5000, 5)) + np.float32(0.25)
    p32 = np.abs(inputs.int32_uniform(5000, 6)) + 1
    cases = [f, -f, p32, -p32, p32.astype(np.int64) << 20, -(p32.astype(np.int64) << 20),
             np.zeros(0, np.float32), np.zeros(0, np.int32), np.zeros(0, np.int64)]
    for a in cases:
        for op, name in ((R.OP_MAX, "max"), (R.OP_MIN, "min")):
            fl = a.dtype == np.float32
            r = torch.full((1,), 12345, dtype=torch.float64 if fl else torch.int64, device="cuda")
            rt.reduce(op, dev(a), r, 0, G, T)
            got = host(r)[0]
            assert (float(got) if fl else int(got)) == O.max_min(a, name), (a.dtype, a.size, name)
    assert rt.sync_status() == 0


def test_bf16_sum(rt):
    bits = inputs.bf16_uniform_pm1((1 << 20) + 11, 5)
    r = _res()
    rt.reduce(R.OP_SUM, _bf16_dev(bits), r, R.PREC_COMP_F64, 152, 512)
    vals = (bits.astype(np.uint32) << 16).view(np.float32)
    ok, err, bound = fp_sum_ok(float(host(r)[0]), O.exact_sum_bf16(bits),
                               O.exact_abs_sum_f32(vals))
    assert ok, (err, bound)


def test_reduction_deterministic(rt):
    a = dev(inputs.f32_uniform_pm1((1 << 22) + 1, 7))
    vals = set()
    for _ in range(5):
        r = _res()
        rt.reduce(R.OP_SUM, a, r, R.PREC_COMP_F64, 608, 512)
        vals.add(host(r)[0].tobytes())
    assert len(vals) == 1


def test_precision_variants_reported(rt):
    """The shipped compensated/fp64-combine variant meets the bound; the two
    comparison variants are run and their errors are only reported."""
    n = 1 << 22
    a = inputs.f32_uniform_pm1(n, 0)
    exact, asum = O.exact_sum_f32(a), O.exact_abs_sum_f32(a)
    ad = dev(a)
    errs = {}
    for prec in (R.PREC_COMP_F64, R.PREC_COMP_F32, R.PREC_NAIVE_F32):
        r = _res()
        rt.reduce(R.OP_SUM, ad, r, prec, 608, 512)
        errs[prec] = abs(float(host(r)[0]) - exact)
    assert fp_sum_ok(exact + errs[R.PREC_COMP_F64], exact, asum)[0]
    assert errs[R.PREC_COMP_F64] <= errs[R.PREC_NAIVE_F32]


def test_dot_reduction(rt):
    import torch
    n = (1 << 20) + 17
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    r = _res()
    xd, yd = dev(x), dev(y)
    for sched, chunk in ((R.SCHED_STATIC, 0), (R.SCHED_DYNAMIC, 256), (R.SCHED_AUTO, 0),
                         (R.SCHED_NONMONOTONIC, 64), (R.SCHED_NONMONOTONIC, 256)):
        rt.launch_region(R.loop_desc(R.BODY_DOT, n=n, x=xd, y=yd), sched, chunk, 148,
                         256, red=R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, r.data_ptr()))
        exact = O.exact_dot_f32(x, y)
        ok, err, bound = fp_sum_ok(float(host(r)[0]), exact, exact)
        assert ok, (sched, err, bound)


def test_axpy_f32_with_sum(rt):
    n = (1 << 20) + 1
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    xd, yd = dev(x), dev(y)
    r = _res()
    rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0), R.SCHED_STATIC, 0,
                     148, 256, red=R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, r.data_ptr()))
    ynew = O.axpy_f32(3.0, x, y)
    ok, err, bound = fp_sum_ok(float(host(r)[0]), O.exact_sum_f32(ynew), O.exact_sum_f32(ynew))
    assert ok, (err, bound)


# -- full size: n = 2^28 ---------------------------------------------------------

N_FULL = 1 << 28


@pytest.mark.parametrize("kind", ["pm1", "lognormal"])
def test_full_size_fp32(rt, kind):
    gen = inputs.f32_uniform_pm1 if kind == "pm1" else inputs.f32_lognormal_signed
    a = gen(N_FULL, 0)
    ad = dev(a)
    r = _res()
    rt.reduce(R.OP_SUM, ad, r, R.PREC_COMP_F64, 4 * rt.sm_count, 512)
    exact, asum = O.exact_sum_f32(a), O.exact_abs_sum_f32(a)
    ok, err, bound = fp_sum_ok(float(host(r)[0]), exact, asum)
    assert ok, (err, bound, exact)
    for op, name in ((R.OP_MAX, "max"), (R.OP_MIN, "min")):
        rt.reduce(op, ad, r, 0, 4 * rt.sm_count, 512)
        assert host(r)[0] == O.max_min(a, name)


def test_full_size_bf16_and_int64(rt):
    bits = inputs.bf16_uniform_pm1(N_FULL, 0)
    r = _res()
    rt.reduce(R.OP_SUM, _bf16_dev(bits), r, R.PREC_COMP_F64, 4 * rt.sm_count, 512)
    vals = (bits.astype(np.uint32) << 16).view(np.float32)
    ok, err, bound = fp_sum_ok(float(host(r)[0]), O.exact_sum_bf16(bits),
                               O.exact_abs_sum_f32(vals))
    assert ok, (err, bound)
    del vals
    a = inputs.int64_uniform(N_FULL, 0)
    ri = _res("i64")
    rt.reduce(R.OP_SUM, dev(a), ri, 0, 4 * rt.sm_count, 512)
    assert int(host(ri)[0]) == O.sum_int(a)


def test_precision_report_full_size(rt):
    """n = 2^28 fp32 (uniform [-1,1] and signed lognormal sigma = 3) and bf16
    (uniform [-1,1]): error of the three accumulation variants against the
    exact sum.  The shipped one
    (compensated fp32, fp64 combine) meets the bound; all three errors are
    written to precision_report.json in the folder that OMPRT_REPORT_DIR names,
    when it is set."""
    import json
    import os
    out = {}
    for kind, gen in (("pm1", inputs.f32_uniform_pm1), ("lognormal", inputs.f32_lognormal_signed)):
        a = gen(N_FULL, 0)
        exact, asum = O.exact_sum_f32(a), O.exact_abs_sum_f32(a)
        ad = dev(a)
        rec = {"exact": exact, "sum_abs": asum}
        for prec, name in ((R.PREC_COMP_F64, "comp_f32_combine_f64"),
                           (R.PREC_COMP_F32, "comp_f32_combine_f32"),
                           (R.PREC_NAIVE_F32, "naive_f32")):
            r = _res()
            rt.reduce(R.OP_SUM, ad, r, prec, 4 * rt.sm_count, 512)
            v = float(host(r)[0])
            rec[name] = {"value": v, "rel_err": abs(v - exact) / abs(exact),
                         "err_over_sum_abs": abs(v - exact) / asum}
        ok, err, bound = fp_sum_ok(rec["comp_f32_combine_f64"]["value"], exact, asum)
        assert ok, (kind, err, bound)
        out[kind] = rec
        del ad, a
    bits = inputs.bf16_uniform_pm1(N_FULL, 0)
    vals = (bits.astype(np.uint32) << 16).view(np.float32)
    exact, asum = O.exact_sum_bf16(bits), O.exact_abs_sum_f32(vals)
    del vals
    bd = _bf16_dev(bits)
    rec = {"exact": exact, "sum_abs": asum}
    for prec, name in ((R.PREC_COMP_F64, "comp_f32_combine_f64"),
                       (R.PREC_COMP_F32, "comp_f32_combine_f32"),
                       (R.PREC_NAIVE_F32, "naive_f32")):
        r = _res()
        rt.reduce(R.OP_SUM, bd, r, prec, 4 * rt.sm_count, 512)
        v = float(host(r)[0])
        rec[name] = {"value": v, "rel_err": abs(v - exact) / abs(exact),
                     "err_over_sum_abs": abs(v - exact) / asum}
    assert fp_sum_ok(rec["comp_f32_combine_f64"]["value"], exact, asum)[0]
    out["bf16_pm1"] = rec
    report_dir = os.environ.get("OMPRT_REPORT_DIR")
    if report_dir and os.path.isdir(report_dir):
        json.dump(out, open(os.path.join(report_dir, "precision_report.json"), "w"),
                  indent=1)
