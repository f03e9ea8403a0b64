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
