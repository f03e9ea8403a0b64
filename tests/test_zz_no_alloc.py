"""The reduction entry point that allocates nothing (omprt_reduce_noalloc).

Some users of this library cannot allocate device memory at the point where
they need a reduction: code in a stream callback or an allocator hook, code
holding a lock that an allocation could need, or a process whose device
memory is owned and budgeted by another component.  For them the library
keeps the reduction's cross-team scratch in a fixed array of its own.

This test calls that entry point through the C ABI twice in a row per case
and checks every result against the CPU oracle: integer sums and max / min
bit for bit, fp32 and bf16 sums within 1e-6 * max(|exact|, 2^-24 * sum |x|)
of the exact sum rounded to fp64.  It also requires each result to equal,
bit for bit, the ordinary omprt_reduce run with the same teams and threads
(the two differ only in where the partials live).  Cases: n = 0 (the
identity of the operation), fp32 / bf16 / int32 / int64 data, sum, max and
min, the default team count (teams = 0, the whole scratch) and the maximum
of NOALLOC_MAX_TEAMS given explicitly.  It makes its own context for the
comparison call, so it runs the same alone in a fresh process or after the
other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _cases(inputs):
    bf = inputs.bf16_uniform_pm1((1 << 20) + 11, 14)
    return [
        ("f32 lognormal sum", inputs.f32_lognormal_signed((1 << 20) + 3, 11), "sum"),
        ("f32 U[-1,1] sum", inputs.f32_uniform_pm1(300007, 15), "sum"),
        ("bf16 sum", bf, "sum"),
        ("int32 sum", inputs.int32_uniform((1 << 20) + 7, 16), "sum"),
        ("int64 sum", inputs.int64_uniform((1 << 19) + 5, 12), "sum"),
        ("f32 max", inputs.f32_uniform_pm1(100003, 13), "max"),
        ("f32 min", inputs.f32_uniform_pm1(100019, 17), "min"),
        ("int64 min", inputs.int64_uniform(65541, 18), "min"),
        ("f32 empty sum", np.zeros(0, np.float32), "sum"),
        ("f32 empty max", np.zeros(0, np.float32), "max"),
        ("int32 empty sum", np.zeros(0, np.int32), "sum"),
        ("int64 empty min", np.zeros(0, np.int64), "min"),
    ]


def _oracle(O, a, op, is_bf16):
    """(expected value, sum |x| for the fp tolerance or None when exact)."""
    if op == "sum":
        if is_bf16:
            vals = (a.astype(np.uint32) << 16).view(np.float32)
            return O.exact_sum_bf16(a), O.exact_abs_sum_f32(vals)
        if a.dtype == np.float32:
            return O.exact_sum_f32(a), O.exact_abs_sum_f32(a)
        return O.sum_int(a), None
    return O.max_min(a, op), None


def test_noalloc_reduce_matches_oracle_twice():
    import torch
    import oracle as O
    from paper_2106_03219_gb300 import build_lib, inputs
    from paper_2106_03219_gb300 import omprt as R
    build_lib.build()
    rt = R.Runtime(0)
    ops = {"sum": R.OP_SUM, "max": R.OP_MAX, "min": R.OP_MIN}
    try:
        for name, a, op in _cases(inputs):
            is_bf16 = name.startswith("bf16")
            fl = a.dtype == np.float32 or is_bf16
            rdt = torch.float64 if fl else torch.int64
            t = torch.from_numpy(a.view(np.int16) if is_bf16 else a).cuda()
            if is_bf16:
                t = t.view(torch.bfloat16)
            want, abs_sum = _oracle(O, a, op, is_bf16)
            for teams, threads in ((0, 0), (R.NOALLOC_MAX_TEAMS, 256), (37, 1024)):
                ref = torch.full((1,), 12345, dtype=rdt, device="cuda")
                rt.reduce(ops[op], t, ref, R.PREC_COMP_F64, teams or R.NOALLOC_MAX_TEAMS,
                          threads or 512)
                ref_bits = ref.cpu().numpy().tobytes()
                for call in range(2):  # two calls in a row share the one scratch array
                    out = torch.full((1,), -1, dtype=rdt, device="cuda")
                    R.reduce_noalloc(ops[op], t, out, R.PREC_COMP_F64, teams, threads)
                    torch.cuda.synchronize()
                    got = out.cpu().numpy()
                    assert got.tobytes() == ref_bits, (name, teams, call)
                    if abs_sum is None:
                        assert (float(got[0]) if fl else int(got[0])) == want, (name, teams, call)
                    else:
                        bound = 1e-6 * max(abs(want), 2.0 ** -24 * abs_sum)
                        assert abs(float(got[0]) - want) <= bound, (name, teams, call)
        # a team count beyond the fixed scratch is refused, not clipped
        ad = torch.zeros(1000, device="cuda")
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(R.OmprtError):
            R.reduce_noalloc(R.OP_SUM, ad, out, R.PREC_COMP_F64, R.NOALLOC_MAX_TEAMS + 1, 256)
        assert rt.sync_status() == 0
    finally:
        rt.close()
