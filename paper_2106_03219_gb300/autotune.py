"""Autotuner: time region launch configurations on the device, keep the fastest.

The worksharing sweep times each (body, schedule) over the grid
teams x threads and records the fastest point; the table is what the
benchmark and the batched executor use.  Timing: CUDA events on the launching
stream, median of `reps` launches, with an L2 flush (a write of a buffer
larger than L2) before every timed launch.
"""
import json
import os
import statistics

PKG = os.path.dirname(os.path.abspath(__file__))
SWEEP_TABLE = os.path.join(PKG, "tuned", "sweep_gb300.json")

TEAMS = (148, 296, 592, 1184)
THREADS = (128, 256, 512, 1024)
SCHEDULES = [("static1", 1, 1), ("static8", 1, 8), ("static64", 1, 64), ("static", 0, 0),
             ("dynamic256", 2, 256), ("auto", 3, 0)]


def load_sweep_table(path=SWEEP_TABLE):
    if not os.path.exists(path):
        return None
    return json.load(open(path)).get("best")


class Timer:
    """Median device time of a launch callable, L2 flushed before each launch."""

    def __init__(self, torch, l2_bytes, reps=5):
        self.torch = torch
        self.reps = reps
        self.flush = torch.empty(max(2 * l2_bytes, 1 << 28) // 4, dtype=torch.float32,
                                 device="cuda")
        self.e0 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        self.e1 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]

    def __call__(self, fn):
        torch = self.torch
        s = torch.cuda.current_stream()
        fn()  # warm
        for k in range(self.reps):
            self.flush.zero_()
            self.e0[k].record(s)
            fn()
            self.e1[k].record(s)
        torch.cuda.synchronize()
        return statistics.median(self.e0[k].elapsed_time(self.e1[k]) for k in range(self.reps))


def sweep(rt, n_axpy=1 << 26, grid=4096, reps=5, teams=TEAMS, threads=THREADS, log=None):
    """The worksharing sweep: axpy (12 B/iter) and 2-D stencil (8 B/point)
    under every schedule at every (teams, threads).  Returns (rows, best)."""
    import torch
    from . import inputs
    from . import omprt as R

    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    timer = Timer(torch, l2, reps)
    x = torch.from_numpy(inputs.f32_uniform01(n_axpy, 0)).cuda()
    y = torch.from_numpy(inputs.f32_uniform01(n_axpy, 1)).cuda()
    g = torch.from_numpy(inputs.grid_f32(grid, grid, 0)).cuda()
    o = torch.empty_like(g)
    bodies = {
        "axpy": (R.loop_desc(R.BODY_AXPY, n=n_axpy, x=x, y=y, alpha=3.0), 12 * n_axpy),
        "stencil2d": (R.loop_desc(R.BODY_STENCIL2D5, n=grid * grid, x=g, out=o, nx=grid,
                                  ny=grid), 8 * grid * grid),
    }
    rows, best = [], {}
    for bname, (desc, nbytes) in bodies.items():
        for label, sched, chunk in SCHEDULES:
            for G in teams:
                for T in threads:
                    ms = timer(lambda: rt.launch_region(desc, sched, chunk, G, T))
                    gbs = nbytes / (ms * 1e-3) / 1e9
                    rows.append({"body": bname, "schedule": label, "teams": G, "threads": T,
                                 "ms": ms, "GBps": gbs})
                    key = "%s/%s" % (bname, label)
                    if key not in best or ms < best[key][2]:
                        best[key] = (G, T, ms)
                    if log:
                        log("%-10s %-11s G=%5d T=%5d %8.4f ms %8.1f GB/s" %
                            (bname, label, G, T, ms, gbs))
    assert rt.sync_status() == 0
    return rows, {k: [v[0], v[1]] for k, v in best.items()}


def main():
    import argparse
    import torch
    from . import omprt as R
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=SWEEP_TABLE)
    ap.add_argument("--rows", default=None, help="also write every measured point here")
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    torch.cuda.init()
    rt = R.Runtime(0)
    rows, best = sweep(rt, reps=args.reps, log=print)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    json.dump({"device": torch.cuda.get_device_name(0), "sm_count": rt.sm_count, "best": best},
              open(args.out, "w"), indent=1)
    if args.rows:
        json.dump(rows, open(args.rows, "w"), indent=0)
    rt.close()


if __name__ == "__main__":
    main()
