"""Autotuner: time region launch configurations on the device, keep the fastest.

The worksharing sweep times each (body, schedule) over the grid
teams x threads and records the fastest point; the table is what the
benchmark and the batched executor use.  The team counts include powers of
two besides multiples of the SM count (`team_grid`): with n a power of two they make every
team's block start on a 32-byte boundary, so per-thread chunks are whole
vectors.  Timing: CUDA events on the launching stream around launches that
go back to back over four copies of the buffers in turn (each launch's
inputs were last touched three launches earlier, more than L2 ago, and each
launch pays the write-back of the previous one's output, as in a stream of
such launches); the mean of `reps` rounds.
"""
import json
import os
import statistics

PKG = os.path.dirname(os.path.abspath(__file__))
SWEEP_TABLE = os.path.join(PKG, "tuned", "sweep_gb300.json")

# team counts: powers of two, and multiples of the device's SM count (see
# team_grid), where every SM gets the same number of teams
TEAMS_POW2 = (1024, 2048, 4096, 8192, 16384)
SM_MULTIPLES = (1, 2, 4, 8, 16, 32)


def team_grid(sm_count):
    """The sweep's team counts on a device of sm_count SMs."""
    return tuple(sorted(set(TEAMS_POW2) | {m * sm_count for m in SM_MULTIPLES}))
THREADS = (32, 64, 128, 256, 512, 1024)
SCHEDULES = [("static1", 1, 1), ("static8", 1, 8), ("static64", 1, 64), ("static", 0, 0),
             ("dynamic256", 2, 256), ("auto", 3, 0)]


BATCH_TABLE = os.path.join(PKG, "tuned", "batch_gb300.json")


def load_batch_table(path=BATCH_TABLE):
    """(chunk_elems, threads) for the batched executor; (8192, 256) untuned."""
    if not os.path.exists(path):
        return 8192, 256
    d = json.load(open(path))
    return int(d["chunk_elems"]), int(d["threads"])


def tune_batch(rt, rs, chunks=(2048, 4096, 8192, 16384, 32768, 65536), threads=(256, 512, 1024),
               reps=5):
    """Fastest (chunk_elems, threads) of the persistent kernel on a region set,
    timed under a CUDA graph."""
    import torch
    best = None
    rows = []
    s = torch.cuda.Stream()
    for c in chunks:
        for t in threads:
            b = rs.batch(rt, c)
            g = torch.cuda.CUDAGraph()
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                b.launch(0, t, stream=s)
            g.replay()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g.replay()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            rows.append({"chunk_elems": c, "threads": t, "ms": ms})
            if best is None or ms < best[2]:
                best = (c, t, ms)
            del g
            b.destroy()
    assert rt.sync_status() == 0
    return {"chunk_elems": best[0], "threads": best[1], "ms": best[2], "rows": rows}


def load_sweep_table(path=SWEEP_TABLE):
    if not os.path.exists(path):
        return None
    return json.load(open(path)).get("best")


def sweep(rt, n_axpy=1 << 26, grid=4096, reps=3, teams=None, threads=THREADS, log=None,
          nsets=4):
    """The worksharing sweep: axpy (12 B/iter) and 2-D stencil (8 B/point)
    under every schedule at every (teams, threads).  Returns (rows, best)."""
    import torch
    from . import inputs
    from . import omprt as R

    if teams is None:
        teams = team_grid(rt.sm_count)
    sets = []
    for _ in range(nsets):
        x = torch.from_numpy(inputs.f32_uniform01(n_axpy, 0)).cuda()
        y = torch.from_numpy(inputs.f32_uniform01(n_axpy, 1)).cuda()
        g = torch.from_numpy(inputs.grid_f32(grid, grid, 0)).cuda()
        o = torch.empty_like(g)
        sets.append({
            "axpy": R.loop_desc(R.BODY_AXPY, n=n_axpy, x=x, y=y, alpha=3.0),
            "stencil2d": R.loop_desc(R.BODY_STENCIL2D5, n=grid * grid, x=g, out=o, nx=grid,
                                     ny=grid)})
    nbytes = {"axpy": 12 * n_axpy, "stencil2d": 8 * grid * grid}
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows, best = [], {}
    for bname in ("axpy", "stencil2d"):
        for label, sched, chunk in SCHEDULES:
            for G in teams:
                for T in threads:
                    for st in sets:
                        rt.launch_region(st[bname], sched, chunk, G, T, stream=stream)
                    e0.record(stream)
                    for _ in range(reps):
                        for st in sets:
                            rt.launch_region(st[bname], sched, chunk, G, T, stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / (reps * nsets)
                    gbs = nbytes[bname] / (ms * 1e-3) / 1e9
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
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--batch", default=None, help="tune the batched executor, write here")
    args = ap.parse_args()
    torch.cuda.init()
    rt = R.Runtime(0)
    if args.batch:
        from . import batched
        rs = batched.RegionSet()
        res = tune_batch(rt, rs, reps=args.reps)
        json.dump(res, open(args.batch, "w"), indent=1)
        print(json.dumps({k: v for k, v in res.items() if k != "rows"}))
        rt.close()
        return
    rows, best = sweep(rt, reps=args.reps, log=print)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    json.dump({"device": torch.cuda.get_device_name(0), "sm_count": rt.sm_count, "best": best},
              open(args.out, "w"), indent=1)
    if args.rows:
        json.dump(rows, open(args.rows, "w"), indent=0)
    rt.close()


if __name__ == "__main__":
    main()
