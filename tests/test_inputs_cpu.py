"""The seeded input generators (CPU): the counter-based form gives the same
bytes on the host and in a torch fill."""
import numpy as np


def test_counter_inputs_agree_between_numpy_and_torch():
    """The device fill and the host evaluation of the counter-based inputs give
    the same bytes, at indices on both sides of 2^31 and 2^32."""
    import torch
    from paper_2106_03219_gb300 import inputs
    for start in (0, (1 << 31) - 700, (1 << 32) - 1000, (1 << 33) + 3):
        t = torch.empty(3000, dtype=torch.float32)
        inputs.counter_f32_01_fill(t, 5, start=start, block=1024)
        want = inputs.counter_f32_01(np.arange(start, start + 3000), 5)
        assert np.array_equal(t.numpy().view(np.uint32), want.view(np.uint32))
    v = inputs.counter_f32_01(np.arange(1 << 16), 0)
    assert v.min() >= 0.0 and v.max() < 1.0
    assert abs(float(v.mean()) - 0.5) < 0.01           # roughly uniform
    assert len(np.unique(v)) > 60000                    # few collisions over 2^16 draws
    # different seeds give different streams
    assert not np.array_equal(v, inputs.counter_f32_01(np.arange(1 << 16), 1))


def test_batched_region_recipe():
    """The many-short-regions recipe (the stand-in for miniQMC's region
    launches): trip counts round(exp(N(ln 1e4, ln 10^2))) clipped to [100, 10^6],
    kinds uniform over three, disjoint slices starting on 64-element
    boundaries, the same bytes for the same seed."""
    from paper_2106_03219_gb300 import inputs
    n, kind, off = inputs.batched_regions(4096)
    assert n.dtype == np.int64 and kind.dtype == np.int32 and off.dtype == np.int64
    assert n.min() >= 100 and n.max() <= 1_000_000
    assert set(np.unique(kind).tolist()) == {0, 1, 2}
    assert np.all(off % 64 == 0) and off[0] == 0
    assert np.all(off[1:] >= off[:-1] + n[:-1])              # disjoint, in order
    assert np.all(off[1:] - (off[:-1] + n[:-1]) < 64)        # padding below one boundary
    med = float(np.median(n))
    assert 5e3 < med < 2e4                                    # centred on 1e4 in log space
    for k in range(3):
        assert abs(float((kind == k).mean()) - 1 / 3) < 0.03
    n2, kind2, off2 = inputs.batched_regions(4096)
    assert np.array_equal(n, n2) and np.array_equal(kind, kind2) and np.array_equal(off, off2)
    assert not np.array_equal(n, inputs.batched_regions(4096, seed=7)[0])


def test_learned_loop_recipe():
    """The cost model's loops: kinds uniform over the five loop kinds, trip
    counts log-uniform in [2^10, 2^26], one stream per seed."""
    from paper_2106_03219_gb300 import inputs
    kind, n = inputs.loop_set(20000, 0)
    assert n.min() >= 1 << 10 and n.max() <= 1 << 26
    lg = np.log2(n.astype(np.float64))
    assert abs(float(np.median(lg)) - 18.0) < 0.3             # log-uniform midpoint
    hist = np.histogram(lg, bins=8, range=(10, 26))[0] / n.size
    assert np.all(np.abs(hist - 1 / 8) < 0.02)
    for k in range(len(inputs.LOOP_KINDS)):
        assert abs(float((kind == k).mean()) - 1 / len(inputs.LOOP_KINDS)) < 0.02
    assert not np.array_equal(n, inputs.loop_set(20000, 1)[1])  # held-out set differs
