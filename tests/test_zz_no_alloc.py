"""The reduction entry point that allocates nothing (omprt_reduce_noalloc).

Some users of this library cannot allocate device memory at the point where
they need a reduction: they run while a CUDA graph is being captured, inside
a callback or an allocator hook, or in a process whose device memory belongs
to another component.  For them the library keeps the reduction's cross-team
scratch in a fixed array of its own.  This test calls that entry point
through the C ABI twice in a row and checks each result against the ordinary
omprt_reduce on the same data, within the tolerance the reduction tests use
(exact for integers and max/min).  It makes its own context for the
reference call, so it runs the same alone in a fresh process or after the
other tests.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_reduce_matches_context_reduce_twice():
    import torch
    from paper_2106_03219_gb300 import build_lib, inputs
    from paper_2106_03219_gb300 import omprt as R
    build_lib.build()
    rt = R.Runtime(0)
    try:
        cases = [
            (R.OP_SUM, inputs.f32_lognormal_signed((1 << 20) + 3, 11), torch.float64),
            (R.OP_SUM, inputs.int64_uniform((1 << 19) + 5, 12), torch.int64),
            (R.OP_MAX, inputs.f32_uniform_pm1(100003, 13), torch.float64),
        ]
        for op, a, rdt in cases:
            ad = torch.from_numpy(a).cuda()
            ref = torch.zeros(1, dtype=rdt, device="cuda")
            rt.reduce(op, ad, ref, R.PREC_COMP_F64, 1024, 256)
            refv = float(ref.cpu()[0]) if rdt == torch.float64 else int(ref.cpu()[0])
            for _ in range(2):                        # two calls in a row
                out = torch.full((1,), -1, dtype=rdt, device="cuda")
                R.reduce_noalloc(op, ad, out, R.PREC_COMP_F64, 1024, 256)
                torch.cuda.synchronize()
                if rdt == torch.float64:
                    got = float(out.cpu()[0])
                    assert abs(got - refv) <= 1e-6 * max(abs(refv), 2.0 ** -24 * a.size)
                else:
                    assert int(out.cpu()[0]) == refv
        # sizes beyond the fixed scratch are refused, not clipped
        ad = torch.zeros(1000, device="cuda")
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(R.OmprtError):
            R.reduce_noalloc(R.OP_SUM, ad, out, R.PREC_COMP_F64, R.NOALLOC_MAX_TEAMS + 1, 256)
        assert rt.sync_status() == 0
    finally:
        rt.close()
