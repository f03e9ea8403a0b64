"""What the learned schedule gains: the committed cost model (trained on the
runtime's own timings of 20k loops) picks configurations for loops it has
never seen (a fresh seed), and the measured total time of its picks is
compared with the plain heuristic's and with the per-loop best of the 12.
The model must beat the heuristic on the total by more than the spread of
repeated, interleaved timings."""
import json
import os

import numpy as np
import pytest

from paper_2106_03219_gb300 import learned
from paper_2106_03219_gb300 import omprt as R

pytestmark = pytest.mark.gpu


def test_learned_beats_heuristic_on_unseen_loops(rt):
    """800 loops the model has never seen (seed 2).  Each loop's model pick
    and heuristic pick are timed interleaved (5 of each, medians), and the
    whole set three times in fresh random orders.  The gain heuristic / model
    must exceed 1 in every round, and its mean must exceed 1 by more than
    three standard deviations of the rounds.  The oracle-best of the 12 bounds
    the model from below."""
    model = learned.Model.load()
    assert model is not None, "no committed cost model"
    buf = learned.LoopBuffers(1 << 24)
    kind, n = learned.make_loops(800, seed=2)
    n = np.minimum(n, 1 << 24)
    rep = learned.compare_picks(rt, model, kind, n, buf, reps=5, rounds=3)
    report_dir = os.environ.get("OMPRT_REPORT_DIR")
    if report_dir and os.path.isdir(report_dir):
        json.dump(rep, open(os.path.join(report_dir, "learned_gain.json"), "w"), indent=1)
    assert min(rep["gain_per_round"]) > 1.0, rep
    assert rep["gain_mean"] - 1.0 > 3.0 * rep["gain_std"], rep
    T = learned.time_loops(rt, kind[:200], n[:200], buf, reps=3)
    best = learned.evaluate(rt, model, kind[:200], n[:200], T, buf)
    assert best["model_total_ms"] >= best["best_total_ms"]
    # with the model removed the runtime falls back to the heuristic
    d, red = learned.loop_desc(int(kind[0]), int(n[0]), buf)
    assert rt.choose_config(d, red is not None) == learned.HEURISTIC


def test_learned_schedule_launch_is_exact(rt):
    """OMPRT_SCHED_LEARNED: the installed model picks a configuration inside
    the library and the loop runs under it with the same results as any
    other schedule (bit-exact axpy, reduction within 1e-6)."""
    import torch
    import oracle as O
    from paper_2106_03219_gb300 import inputs
    model = learned.Model.load()
    model.install(rt)
    try:
        for n in (1000, 1 << 16, (1 << 20) + 3):
            x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
            xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
            r = torch.zeros(1, dtype=torch.float64, device="cuda")
            d = R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0)
            k = rt.choose_config(d, True)
            assert 0 <= k < 12
            rt.launch_region(d, R.SCHED_LEARNED, 0, 0, 0,
                             red=R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, r.data_ptr()))
            ynew = O.axpy_f32(3.0, x, y)
            torch.cuda.synchronize()
            assert np.array_equal(yd.cpu().numpy().view(np.uint32), ynew.view(np.uint32))
            exact = O.exact_sum_f32(ynew)
            assert abs(float(r.cpu()[0]) - exact) <= 1e-6 * abs(exact)
        assert rt.sync_status() == 0
    finally:
        rt.set_cost_model(None)
