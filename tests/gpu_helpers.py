"""Small helpers shared by the GPU parity tests (no runtime arithmetic)."""
import numpy as np


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def bits32(a):
    return np.ascontiguousarray(a).view(np.uint32)


def fp_sum_ok(gpu, exact, abs_sum, rel=1e-6):
    """|gpu - exact| <= rel * max(|exact|, 2^-24 * sum|x|) (the tolerance of
    the fp32 sums against the exact fp64 result)."""
    bound = rel * max(abs(exact), 2.0 ** -24 * abs_sum)
    return abs(gpu - exact) <= bound, abs(gpu - exact), bound
