"""Pins for the oracle's atomic inc (C8), shared-memory stack (C10) and MLP
cost model (C12)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            rows.append([int(v) for v in line.split()])
    return rows


# -- atomic inc (Sec. 3.1: v = x; x = x >= e ? 0 : x + 1; return v) ---------

def test_atomic_inc_golden():
    for x0, e, k, *rest in read_golden("atomic_inc.txt"):
        vals, final = O.atomic_inc_sequence(x0, e, k)
        assert vals == rest[:k]
        assert final == rest[k]


def test_atomic_inc_closed_form():
    # from x = 0, K increments leave K mod (e+1) and return each residue
    # K/(e+1) times when (e+1) divides K
    for e in (0, 1, 5, 127):
        K = 4 * (e + 1)
        vals, final = O.atomic_inc_sequence(0, e, K)
        assert final == K % (e + 1) == 0
        assert sorted(vals) == sorted(list(range(e + 1)) * 4)
        vals, final = O.atomic_inc_sequence(0, e, K + 3)
        assert final == (K + 3) % (e + 1)


# -- shared-memory stack (C10) ------------------------------------------------------

def test_stack_hand_trace():
    rows = read_golden("stack_trace.txt")
    S, Q = rows[0]
    ops = np.array([r[:2] for r in rows[1:-1]], np.int64)
    expect = np.array([r[2:4] for r in rows[1:-1]], np.int64)
    out, st = O.stack_replay(S, Q, ops)
    assert out.tolist() == expect.tolist()
    assert st == rows[-1][0]


@pytest.mark.parametrize("seed", range(6))
def test_stack_random_lifo_invariants(seed):
    S, Q = 1024, 2048
    ops = inputs.stack_trace(400, seed=seed, max_bytes=300)
    out, st = O.stack_replay(S, Q, ops)
    assert st & 2 == 0                       # a LIFO trace never breaks order
    live = {}
    nalloc = 0
    for (kind, arg), (a, b) in zip(ops.tolist(), out.tolist()):
        if kind == 0:
            r = ((max(arg, 1) + 15) // 16) * 16
            if a in (0, 1):
                cap = S if a == 0 else Q
                assert b % 16 == 0 and 0 <= b and b + r <= cap
                for (ra, rb, rr) in live.values():
                    if ra == a:
                        assert b + r <= rb or rb + rr <= b   # no overlap
                if a == 1:
                    # the shared stack really had no room
                    top = max([rb + rr for (ra, rb, rr) in live.values() if ra == 0] or [0])
                    assert top + r > S
            live[nalloc] = (a, b, r)
            nalloc += 1
        else:
            assert a == 0
            live.pop(arg)


def test_stack_order_violation_detected():
    ops = inputs.stack_trace(300, seed=3, max_bytes=100, bad_free=True)
    _, st = O.stack_replay(4096, 4096, ops)
    assert st & 2


# -- MLP (C12) ----------------------------------------------------------------------

def _rand_params(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.3, O.mlp_nparam())


def test_mlp_nparam():
    assert O.mlp_nparam() == 64 * 16 + 64 + 64 * 64 + 64 + 12 * 64 + 12


def test_mlp_forward_special_cases():
    p = np.zeros(O.mlp_nparam())
    b3 = np.arange(12) * 0.5 - 2
    p[-12:] = b3
    X = np.random.default_rng(0).normal(size=(7, 16))
    assert np.array_equal(O.mlp_forward(p, X), np.tile(b3, (7, 1)))
    # a single path: W1[0][3] = 2, W2[5][0] = 3, W3[7][5] = 4 -> y7 = 24 relu(x3)
    p = np.zeros(O.mlp_nparam())
    p[0 * 16 + 3] = 2.0
    off_w2 = 64 * 16 + 64
    p[off_w2 + 5 * 64 + 0] = 3.0
    off_w3 = off_w2 + 64 * 64 + 64
    p[off_w3 + 7 * 64 + 5] = 4.0
    Y = O.mlp_forward(p, X)
    assert np.allclose(Y[:, 7], 24 * np.maximum(X[:, 3], 0), rtol=0, atol=1e-15)
    assert np.all(np.delete(Y, 7, axis=1) == 0)


def test_mlp_zero_model_loss():
    p = np.zeros(O.mlp_nparam())
    rng = np.random.default_rng(1)
    X, Yt = rng.normal(size=(9, 16)), rng.normal(size=(9, 12))
    loss, g = O.mlp_loss_grad(p, X, Yt)
    assert np.isclose(loss, np.mean(Yt ** 2), rtol=1e-15)
    # only the output bias has a gradient at zero weights: -2 mean(target)
    assert np.allclose(g[-12:], -2 * Yt.mean(axis=0) / 12, rtol=1e-13)
    assert np.all(g[:-12] == 0)


def test_mlp_gradient_finite_differences():
    p = _rand_params(2)
    rng = np.random.default_rng(3)
    X, Yt = rng.normal(size=(6, 16)), rng.normal(size=(6, 12))
    _, g = O.mlp_loss_grad(p, X, Yt)
    idx = rng.choice(p.size, 200, replace=False)
    h = 1e-4

    def loss_at(i, d):
        q = p.copy()
        q[i] += d
        return O.mlp_loss_grad(q, X, Yt)[0]

    for i in idx:
        # fourth-order central difference: truncation O(h^4), rounding ~1e-12
        fd = (-loss_at(i, 2 * h) + 8 * loss_at(i, h) - 8 * loss_at(i, -h)
              + loss_at(i, -2 * h)) / (12 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3), (i, fd, g[i])


def test_adam_constant_gradient_closed_form():
    # with a constant gradient the bias-corrected moments are m^ = g and
    # v^ = g^2 at every step, so each step moves by lr * g / (|g| + eps)
    rng = np.random.default_rng(4)
    g = rng.normal(size=50)
    p0 = rng.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    lr, eps = 1e-3, 1e-8
    for t in range(1, 6):
        O.adam_step(p, g, m, v, t, lr=lr, eps=eps)
        expect = p0 - t * lr * g / (np.abs(g) + eps)
        assert np.allclose(p, expect, rtol=1e-12, atol=1e-15)
