"""Learned schedule selection: a 16 -> 64 -> 64 -> 12 MLP that predicts the
log run time of a loop under each of 12 schedule / chunk / teams
configurations, trained on timings the runtime takes of itself.

Pipeline (all device work through the C ABI):
  1. make_loops: loops of five kinds (axpy, dot, 1-D stencil, 2-D stencil,
     sum reduction), trip counts log-uniform in [2^10, 2^26].
  2. time_loops: each loop under each configuration, median of `reps`
     launches (CUDA events).  Features come from omprt_loop_features.
  3. train: MSE on standardised log time, Adam, forward / backward / update
     in the library's MLP kernels.
  4. evaluate: on held-out loops, the measured time of the configuration the
     installed model picks (host inference inside the library, with the
     heuristic as fallback) against the heuristic's pick and the per-loop
     best of the 12.
"""
import json
import os
import time

import numpy as np

from . import inputs
from . import omprt as R

PKG = os.path.dirname(os.path.abspath(__file__))
MODEL_PATH = os.path.join(PKG, "tuned", "cost_model_gb300.json")
HEURISTIC = 9
MAX_N = 1 << 26


class LoopBuffers:
    """Device buffers large enough for the largest loop; loops use prefixes."""

    def __init__(self, max_n=MAX_N):
        import torch
        self.x = torch.from_numpy(inputs.f32_uniform01(max_n, 0)).cuda()
        self.y = torch.from_numpy(inputs.f32_uniform01(max_n, 1)).cuda()
        self.out = torch.zeros(max_n, dtype=torch.float32, device="cuda")
        self.res = torch.zeros(1, dtype=torch.float64, device="cuda")


def loop_desc(kind, n, buf):
    """(descriptor, reduction or None) for a loop of LOOP_KINDS[kind] over n."""
    name = inputs.LOOP_KINDS[kind]
    red = R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, buf.res.data_ptr())
    if name == "axpy":
        return R.loop_desc(R.BODY_AXPY, n=n, x=buf.x, y=buf.y, alpha=1.0), None
    if name == "dot":
        return R.loop_desc(R.BODY_DOT, n=n, x=buf.x, y=buf.y), red
    if name == "stencil1d3":
        return R.loop_desc(R.BODY_STENCIL1D3, n=n, x=buf.x, out=buf.out), None
    if name == "stencil2d5":
        nx = 1 << max(0, int(np.log2(max(n, 1))) // 2)
        ny = max(1, n // nx)
        return R.loop_desc(R.BODY_STENCIL2D5, n=nx * ny, x=buf.x, out=buf.out, nx=nx,
                           ny=ny), None
    return R.loop_desc(R.BODY_NONE, n=n, x=buf.x, data_type=R.F32), red


def make_loops(count, seed):
    kind, n = inputs.loop_set(count, seed)
    return kind, np.minimum(n, MAX_N)


def features(rt, kind, n, buf):
    F = np.zeros((len(kind), R.MLP_IN), np.float32)
    for i, (k, m) in enumerate(zip(kind, n)):
        d, red = loop_desc(int(k), int(m), buf)
        F[i] = rt.loop_features(d, red is not None)
    return F


def time_loops(rt, kind, n, buf, reps=3, log=None):
    """times[i, k] = median ms of loop i under configuration k."""
    import torch
    cfgs = R.learned_configs()
    sms = rt.sm_count
    T = np.zeros((len(kind), len(cfgs)), np.float64)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps * len(cfgs) + 1)]
    t0 = time.time()
    for i, (k, m) in enumerate(zip(kind, n)):
        d, red = loop_desc(int(k), int(m), buf)
        for c, (sched, chunk, tps, thr) in enumerate(cfgs):   # warm every config once
            rt.launch_region(d, sched, chunk, tps * sms, thr, red=red, stream=stream)
        j = 0
        ev[0].record(stream)
        for c, (sched, chunk, tps, thr) in enumerate(cfgs):
            for _ in range(reps):
                rt.launch_region(d, sched, chunk, tps * sms, thr, red=red, stream=stream)
                j += 1
                ev[j].record(stream)
        ev[j].synchronize()
        for c in range(len(cfgs)):
            ts = [ev[c * reps + r].elapsed_time(ev[c * reps + r + 1]) for r in range(reps)]
            T[i, c] = float(np.median(ts))
        if log and i % 2000 == 0:
            log("timed %d / %d loops (%.1f s)" % (i, len(kind), time.time() - t0))
    assert rt.sync_status() == 0
    return T


class Model:
    def __init__(self, params, feat_mean, feat_std, y_mean, y_std):
        self.params = np.asarray(params, np.float32)
        self.feat_mean = np.asarray(feat_mean, np.float32)
        self.feat_std = np.asarray(feat_std, np.float32)
        self.y_mean = float(y_mean)
        self.y_std = float(y_std)

    def save(self, path=MODEL_PATH, extra=None):
        d = {"version": 1, "layout": "W1[64][16] b1 W2[64][64] b2 W3[12][64] b3, fp32",
             "params": self.params.tolist(), "feat_mean": self.feat_mean.tolist(),
             "feat_std": self.feat_std.tolist(), "y_mean": self.y_mean, "y_std": self.y_std}
        if extra:
            d.update(extra)
        os.makedirs(os.path.dirname(path), exist_ok=True)
        json.dump(d, open(path, "w"))

    @staticmethod
    def load(path=MODEL_PATH):
        if not os.path.exists(path):
            return None
        d = json.load(open(path))
        if d.get("version") != 1:
            return None
        return Model(d["params"], d["feat_mean"], d["feat_std"], d["y_mean"], d["y_std"])

    def install(self, rt):
        # outputs are log-times up to one affine map with positive scale, so
        # the argmin the library takes is the argmin of predicted time
        rt.set_cost_model(self.params, self.feat_mean, self.feat_std)


def init_params(seed=0):
    """He-style initial weights, zero biases."""
    g = np.random.default_rng(seed)
    p = np.zeros(R.MLP_NPARAM, np.float32)
    off = 0
    for fan_in, fan_out in ((16, 64), (64, 64), (64, 12)):
        w = g.normal(0, np.sqrt(2.0 / fan_in), size=fan_out * fan_in)
        p[off:off + w.size] = w
        off += w.size + fan_out
    return p


def train(rt, F, T, epochs=60, batch=256, lr=1e-3, seed=0, log=None):
    """Train on features F [N,16] and times T [N,12] (ms).  Returns Model."""
    import torch
    fm = F.mean(axis=0)
    fs = F.std(axis=0)
    fs[fs == 0] = 1.0
    Y = np.log(T)
    ym, ys = float(Y.mean()), float(Y.std())
    X = ((F - fm) / fs).astype(np.float32)
    Yn = ((Y - ym) / ys).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    p = dev(init_params(seed))
    grad = torch.zeros_like(p)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed)
    step = 0
    history = []
    for ep in range(epochs):
        # shuffle on the host and upload once per epoch: a batch is then a
        # contiguous slice, so every device step is one of the library's kernels
        perm = rng.permutation(len(X))
        Xd, Yd = dev(X[perm]), dev(Yn[perm])
        tot = 0.0
        nb = 0
        for s in range(0, len(X) - batch + 1, batch):
            xb, yb = Xd[s:s + batch], Yd[s:s + batch]
            rt.mlp_loss_grad(p, xb, yb, grad, loss)
            step += 1
            rt.mlp_adam(p, grad, m, v, step, lr=lr)
            tot += float(loss.item()) if nb % 50 == 0 else 0.0
            nb += 1
        history.append(tot)
        if log and ep % 10 == 0:
            log("epoch %d" % ep)
    model = Model(p.cpu().numpy(), fm, fs, ym, ys)
    return model, history


def evaluate(rt, model, kind, n, T, buf):
    """Measured time of the model's pick vs the heuristic and the per-loop best."""
    model.install(rt)
    picks = np.zeros(len(kind), np.int64)
    t0 = time.perf_counter()
    for i, (k, m) in enumerate(zip(kind, n)):
        d, red = loop_desc(int(k), int(m), buf)
        picks[i] = rt.choose_config(d, red is not None)
    decide_us = (time.perf_counter() - t0) / max(len(kind), 1) * 1e6
    rt.set_cost_model(None)
    rows = np.arange(len(kind))
    t_model = float(T[rows, picks].sum())
    t_heur = float(T[:, HEURISTIC].sum())
    t_best = float(T.min(axis=1).sum())
    return {"loops": int(len(kind)), "model_total_ms": t_model, "heuristic_total_ms": t_heur,
            "best_total_ms": t_best, "model_vs_heuristic": t_heur / t_model,
            "model_gap_to_best": t_model / t_best - 1.0,
            "heuristic_gap_to_best": t_heur / t_best - 1.0,
            "loops_model_faster": int((T[rows, picks] < T[:, HEURISTIC]).sum()),
            "loops_model_slower": int((T[rows, picks] > T[:, HEURISTIC]).sum()),
            "decision_us": decide_us}


def compare_picks(rt, model, kind, n, buf, reps=5, rounds=3, seed=0):
    """The model's pick against the heuristic's on the same loops, timed
    interleaved: for every loop, `reps` launches of the model's configuration
    alternate with `reps` of the heuristic's (CUDA events around each), and
    the loop's time under each is the median of its reps.  The whole set is
    timed `rounds` times, each in a fresh random loop order.  Returns the
    total time of each pick per round, the gain heuristic / model per round,
    and its mean and spread (sample standard deviation and range)."""
    import torch
    cfgs = R.learned_configs()
    sms = rt.sm_count
    model.install(rt)
    descs, picks = [], []
    try:
        for k, m in zip(kind, n):
            d, red = loop_desc(int(k), int(m), buf)
            descs.append((d, red))
            picks.append(rt.choose_config(d, red is not None))
    finally:
        rt.set_cost_model(None)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4 * reps + 1)]
    rng = np.random.default_rng(seed)
    tot_model, tot_heur = [], []
    for _ in range(rounds):
        tm = th = 0.0
        for i in rng.permutation(len(descs)):
            d, red = descs[i]
            run = [cfgs[picks[i]], cfgs[HEURISTIC]]
            for sched, chunk, tps, thr in run:  # warm both
                rt.launch_region(d, sched, chunk, tps * sms, thr, red=red, stream=stream)
            j = 0
            ev[0].record(stream)
            for _r in range(reps):
                for sched, chunk, tps, thr in run:
                    rt.launch_region(d, sched, chunk, tps * sms, thr, red=red, stream=stream)
                    j += 1
                    ev[j].record(stream)
            ev[j].synchronize()
            t = [ev[q].elapsed_time(ev[q + 1]) for q in range(j)]
            tm += float(np.median(t[0::2]))
            th += float(np.median(t[1::2]))
        tot_model.append(tm)
        tot_heur.append(th)
    assert rt.sync_status() == 0
    gain = [h / m for h, m in zip(tot_heur, tot_model)]
    return {"loops": len(descs), "reps": reps, "rounds": rounds,
            "model_total_ms": tot_model, "heuristic_total_ms": tot_heur,
            "gain_per_round": gain, "gain_mean": float(np.mean(gain)),
            "gain_std": float(np.std(gain, ddof=1)) if rounds > 1 else 0.0,
            "gain_range": [float(min(gain)), float(max(gain))],
            "loops_model_differs": int(sum(1 for p in picks if p != HEURISTIC))}


def main():
    import argparse
    import torch
    ap = argparse.ArgumentParser(description="time loops, train the cost model, evaluate")
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--test", type=int, default=2000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", default=MODEL_PATH)
    ap.add_argument("--report", default=None)
    args = ap.parse_args()
    torch.cuda.init()
    rt = R.Runtime(0)
    buf = LoopBuffers()
    ktr, ntr = make_loops(args.train, 0)
    kte, nte = make_loops(args.test, 1)
    Ftr = features(rt, ktr, ntr, buf)
    t0 = time.time()
    Ttr = time_loops(rt, ktr, ntr, buf, args.reps, log=print)
    Tte = time_loops(rt, kte, nte, buf, args.reps, log=print)
    t_time = time.time() - t0
    t0 = time.time()
    model, hist = train(rt, Ftr, Ttr, epochs=args.epochs, log=print)
    t_train = time.time() - t0
    rep = evaluate(rt, model, kte, nte, Tte, buf)
    rep.update({"train_loops": args.train, "timing_s": t_time, "train_s": t_train,
                "timed_launches": int((args.train + args.test) * 12 * args.reps)})
    model.save(args.out, extra={"report": rep})
    print(json.dumps(rep))
    if args.report:
        json.dump(rep, open(args.report, "w"), indent=1)
    rt.close()


if __name__ == "__main__":
    main()
