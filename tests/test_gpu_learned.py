"""What the learned schedule gains: the committed cost model (trained on the
runtime's own timings of 20k loops) picks configurations for loops it has
never seen (a fresh seed), and the measured total time of its picks is
compared with the plain heuristic's and with the per-loop best of the 12.
The model must beat the heuristic on the total."""
import json
import os

import numpy as np
import pytest

from paper_2106_03219_gb300 import learned
from paper_2106_03219_gb300 import omprt as R

pytestmark = pytest.mark.gpu


def test_learned_beats_heuristic_on_unseen_loops(rt):
    model = learned.Model.load()
    assert model is not None, "no committed cost model"
    buf = learned.LoopBuffers(1 << 24)
    kind, n = learned.make_loops(800, seed=2)
    n = np.minimum(n, 1 << 24)
    T = learned.time_loops(rt, kind, n, buf, reps=3)
    rep = learned.evaluate(rt, model, kind, n, T, buf)
    root = os.environ.get("GRAFT_REPO_ROOT", os.getcwd())
    if os.path.isdir(os.path.join(root, "gpurun_out")):
        json.dump(rep, open(os.path.join(root, "gpurun_out", "learned_gain.json"), "w"), indent=1)
    assert rep["model_total_ms"] < rep["heuristic_total_ms"], rep
    assert rep["model_total_ms"] >= rep["best_total_ms"]
    # with the model removed the runtime falls back to the heuristic
    d, red = learned.loop_desc(int(kind[0]), int(n[0]), buf)
    assert rt.choose_config(d, red is not None) == learned.HEURISTIC
