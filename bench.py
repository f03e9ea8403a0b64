"""Benchmark: loop GB/s of the OpenMP device-runtime hot path on GB300.

One step = one pass of the worksharing workload: fp32 axpy y = 3x + y over
n = 2^26 and the 2-D 5-point stencil over a 4096 x 4096 fp32 grid, each run
as a "teams distribute parallel for" region under the six schedules
static(1), static(8), static(64), static (no chunk), dynamic(256) and auto,
at the teams / threads the tuning table gives for that schedule.

value     = algorithmic bytes of the step (12 B per axpy iteration, 8 B per
            stencil point) / device time of the step (CUDA events), the
            launches back to back on one stream, each free to start under the
            previous one's tail (launch overlap, the runtime's default); an
            event pair brackets the dominant kernel only.
launch_overlap = the same step with plain launches.
e2e       = the same bytes / time of a step through the C ABI with the inputs
            copied in from pinned host memory and the results copied back.
roofline  = the kernel with the largest share of the step: its algorithmic
            bytes per launch / its mean launch time, against the measured HBM
            copy bandwidth.
cpu_baseline / --impl reference = the CPU oracle on the same workload, on all
            host cores (one slice per core) and on one core.
kernels   = per-kernel event times in a pass of the step with every launch
            between its own event pair (serialised, about 1.5 us of event
            cost each); kernels_steady = each kernel alone, back to back over
            rotating buffer copies, with launch overlap and (plain_launches)
            without.

Launch: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference];
for N > 1 under torch.distributed.run, every rank runs the same workload on
its own GPU (weak scaling, no data-path collective; max time over ranks).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_AXPY = 1 << 26
GRID = 4096
AXPY_BYTES = 12 * N_AXPY
STENCIL_BYTES = 8 * GRID * GRID
METRIC = "loop GB/s vs HBM peak (worksharing sweep step: fp32 axpy 2^26 + 2D 5-point stencil 4096^2, 6 schedules)"
UNIT = "GB/s"

# (label, sched, chunk)
SCHEDULES = [("static1", 1, 1), ("static8", 1, 8), ("static64", 1, 64), ("static", 0, 0),
             ("dynamic256", 2, 256), ("auto", 3, 0)]


def _code_only(text):
    """Source text without C/C++ comments and whitespace, so that edits to
    documentation do not change the hash while any code change does."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r"\s+", "", text)


def source_hash():
    """Hash of the code of the kernels and the ABI header (profiles/traffic.json
    figures are used only while it matches)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2106_03219_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(_code_only(open(os.path.join(csrc, f)).read()).encode())
    h.update(_code_only(open(os.path.join(ROOT, "include", "omprt.h")).read()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def tuned_points(sm_count):
    """(teams, threads) per schedule label: the autotuner's table if one was
    committed for this source, else 4 teams per SM x 256 threads."""
    from paper_2106_03219_gb300 import autotune
    table = autotune.load_sweep_table()
    pts = {}
    for label, _, _ in SCHEDULES:
        for body in ("axpy", "stencil2d"):
            key = "%s/%s" % (body, label)
            if table and key in table:
                pts[key] = tuple(table[key])
            else:
                pts[key] = (4 * sm_count, 256)
    return pts


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        load = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(rows), "reasons": reasons}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws):
    """Largest value over all ranks (identity for one rank)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# -- CPU oracle legs --------------------------------------------------------------------
#
# The oracle as it stands, on the host: on every host core (disjoint slices in
# spawned worker processes, oracle/cores.py) and on one core.  These are
# reported baselines, not targets.

def oracle_step_one_core(x, y, grid):
    """One worksharing step on one core: fp32 axpy over x / y and the 2-D
    stencil over grid, once per schedule (the oracle is sequential, so every
    schedule runs the same loop).  Returns (seconds, algorithmic bytes)."""
    import oracle as O
    t0 = time.perf_counter()
    for _ in SCHEDULES:
        y[...] = O.axpy_f32(3.0, x, y)
        O.stencil2d5(grid)
    return time.perf_counter() - t0, (12 * x.size + 8 * grid.size) * len(SCHEDULES)


class CpuStep:
    """The worksharing step on all host cores: every schedule's axpy and
    stencil split into one contiguous slice (rows for the stencil) per core."""

    def __init__(self, pool, x, y, grid):
        self.pool = pool
        self.sx, _ = pool.share(x)
        self.sy, _ = pool.share(y)
        self.sg, _ = pool.share(grid)
        self.so, _ = pool.share(np.zeros_like(grid))
        self.n, self.ny = x.size, grid.shape[0]
        self.nbytes = (12 * x.size + 8 * grid.size) * len(SCHEDULES)

    def run(self):
        t = 0.0
        for _ in SCHEDULES:
            t += self.pool.run("axpy_f32", [self.sx, self.sy], self.n, extra=3.0)[0]
            t += self.pool.run("stencil2d", [self.sg, self.so], self.ny)[0]
        return t


def worksharing_inputs():
    from paper_2106_03219_gb300 import inputs
    return (inputs.f32_uniform01(N_AXPY, 0), inputs.f32_uniform01(N_AXPY, 1),
            inputs.grid_f32(GRID, GRID, 0))


def cpu_worksharing(pool, steps=3):
    """cpu_baseline of the main line: the full worksharing step (axpy 2^26 and
    the 4096^2 stencil, x 6 schedules) on all cores, best of `steps`, and on
    one core (one step)."""
    x, y, grid = worksharing_inputs()
    st = CpuStep(pool, x, y, grid)
    t_all = min(st.run() for _ in range(steps))
    t_one, nbytes = oracle_step_one_core(x, y.copy(), grid)
    return {"value": nbytes / t_all / 1e9, "unit": UNIT, "cores": pool.n, "kind": "oracle",
            "sample": "the full step (fp32 axpy n=2^26 + 2D stencil 4096x4096, x 6 schedules), "
                      "best of %d, oracle on %d cores (one slice per core)" % (steps, pool.n),
            "one_core": {"value": nbytes / t_one / 1e9, "unit": UNIT, "cores": 1,
                         "sample": "one full step, single-threaded oracle"}}


def cpu_single_region(pool):
    """Configuration 1 on the CPU: int32 axpy y = 3x + y over n = 2^20 and the
    int64 sum of the new y; median of 5 on one core, and on all cores."""
    import oracle as O
    from paper_2106_03219_gb300 import inputs
    n = 1 << 20
    x, y = inputs.int32_uniform(n, 0), inputs.int32_uniform(n, 1)
    ts = []
    for _ in range(5):
        t0 = time.perf_counter()
        yn = O.axpy_i32(3, x, y)
        O.sum_int(yn)
        ts.append(time.perf_counter() - t0)
    sx, _ = pool.share(x)
    ta = []
    for _ in range(5):
        sy, _ = pool.share(y)
        ta.append(pool.run("axpy_i32_sum", [sx, sy], n, extra=3)[0])
    t1, tall = statistics.median(ts), statistics.median(ta)
    return {"one_core_ms": t1 * 1e3, "one_core_GBps": 12 * n / t1 / 1e9,
            "all_cores_ms": tall * 1e3, "all_cores_GBps": 12 * n / tall / 1e9, "cores": pool.n}


def cpu_reductions(pool, arrays, gpu):
    """Exact sums of the reduction inputs on all cores (the oracle's exact
    expansions per slice, combined exactly), the error of every GPU variant
    against them, and the CPU baselines of the reduction: the exact oracle
    and the plain fp64 loop, on all cores and on one core (a 2^24 sample)."""
    import oracle as O
    out = {}
    for name, a in arrays.items():
        bf = name == "bf16_sum"
        if name == "int64_sum":
            want = O.sum_int(a)
            out[name] = {"exact": want, "gpu": gpu[name]["shipped"],
                         "bit_exact": gpu[name]["shipped"] == want}
            continue
        spec, _ = pool.share(a)
        t_exact, terms = pool.run("exact_terms", [spec], a.size, extra=1 if bf else 0)
        exact = O.exact_sum_f64(np.concatenate([np.asarray(t) for t in terms]))
        vals = (a.astype(np.uint32) << 16).view(np.float32) if bf else a
        sabs = O.exact_abs_sum_f32(vals[: 1 << 24]) * (a.size / min(a.size, 1 << 24))
        row = {"exact": exact, "abs_sum_estimate": sabs}
        for var in ("shipped", "comp_f32", "naive_f32"):
            v = gpu[name][var]
            err = abs(v - exact)
            row[var] = {"value": v, "rel_err": err / abs(exact) if exact else None,
                        "err_over_abs_sum": err / sabs if sabs else None,
                        "within_1e-6": err <= 1e-6 * max(abs(exact), 2.0 ** -24 * sabs)}
        if name == "fp32_pm1_sum":
            for op in ("max", "min"):
                got = gpu["fp32_" + op]["value"]
                gpu["fp32_" + op]["vs_oracle"] = {"oracle": O.max_min(a, op),
                                                  "bit_exact": got == O.max_min(a, op)}
            # CPU baselines of the reduction on this array (1 GiB of fp32)
            t_plain = pool.run("plain_sum", [spec], a.size)[0]
            s = a[: 1 << 24]
            t0 = time.perf_counter()
            O.exact_sum_f32(s)
            t1 = time.perf_counter()
            O.plain_sum_f32(s)
            t2 = time.perf_counter()
            row["cpu_baseline"] = {
                "exact_all_cores_GBps": a.nbytes / t_exact / 1e9,
                "plain_fp64_all_cores_GBps": a.nbytes / t_plain / 1e9,
                "exact_one_core_GBps": s.nbytes / (t1 - t0) / 1e9,
                "plain_fp64_one_core_GBps": s.nbytes / (t2 - t1) / 1e9,
                "cores": pool.n,
                "sample": "all cores: the whole n=2^28 array; one core: its first 2^24 elements"}
        out[name] = row
    return out


def cpu_batched(pool):
    """The 4096-region batch on the CPU: the oracle's per-region loop (axpy,
    exact dot, 1-D stencil), regions dealt round robin to the cores; and on
    one core."""
    import oracle as O
    from paper_2106_03219_gb300 import inputs
    n, kind, off = inputs.batched_regions()
    total = int(off[-1] + (n[-1] + 63) // 64 * 64)
    x, y = inputs.f32_uniform01(total, 0), inputs.f32_uniform01(total, 1)
    table = np.stack([kind.astype(np.int64), off.astype(np.int64), n.astype(np.int64)], 1)
    # deal regions so every core gets a similar number of iterations
    order = np.argsort(-n)
    owner = np.zeros(len(n), np.int64)
    load = np.zeros(pool.n)
    for r in order:
        k = int(np.argmin(load))
        owner[r] = k
        load[k] += n[r]
    perm = np.argsort(owner, kind="stable")
    tab = table[perm]
    cnt = np.bincount(owner, minlength=pool.n)
    cuts = np.r_[0, np.cumsum(cnt)]
    sx, _ = pool.share(x)
    sy, _ = pool.share(y)
    so, _ = pool.share(np.zeros(total, np.float32))
    st, _ = pool.share(tab)
    t_all = pool.run("regions", [sx, sy, so, st], len(n),
                     parts=list(zip(cuts[:-1].tolist(), cuts[1:].tolist())))[0]
    yy = y.copy()
    t0 = time.perf_counter()
    for k, o, m in table:
        if k == inputs.KIND_AXPY:
            yy[o:o + m] = O.axpy_f32(3.0, x[o:o + m], yy[o:o + m])
        elif k == inputs.KIND_DOT:
            O.exact_dot_f32(x[o:o + m], yy[o:o + m])
        else:
            O.stencil1d3(x[o:o + m])
    t_one = time.perf_counter() - t0
    from paper_2106_03219_gb300.batched import BYTES_PER_ITER
    nbytes = int(sum(BYTES_PER_ITER[int(k)] * int(m) for k, m in zip(kind, n)))
    return {"all_cores_regions_per_s": len(n) / t_all, "all_cores_GBps": nbytes / t_all / 1e9,
            "one_core_regions_per_s": len(n) / t_one, "one_core_GBps": nbytes / t_one / 1e9,
            "cores": pool.n}


def cpu_mlp(reps=20):
    """One FP64 training step of the cost model on the oracle (forward,
    loss, backward, Adam) on a batch of 256, one core.  A step is about 3
    MFLOP, too small to split across processes."""
    import oracle as O
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.1, O.mlp_nparam())
    X, Y = rng.normal(size=(256, 16)), rng.normal(size=(256, 12))
    m, v = np.zeros_like(p), np.zeros_like(p)
    ts = []
    for t in range(1, reps + 1):
        t0 = time.perf_counter()
        _, g = O.mlp_loss_grad(p, X, Y)
        O.adam_step(p, g, m, v, t)
        ts.append(time.perf_counter() - t0)
    return {"one_core_ms_per_step": statistics.median(ts) * 1e3, "batch": 256, "cores": 1}


def run_reference(args):
    """The reference arm: the CPU oracle on the host cores, on this bench's
    workload (the full worksharing step), with the same metric and unit."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import cores
    pool = cores.Cores()
    try:
        x, y, grid = worksharing_inputs()
        st = CpuStep(pool, x, y, grid)
        for _ in range(args.warmup):
            st.run()
        t = sum(st.run() for _ in range(args.steps))
        v = st.nbytes * args.steps / t / 1e9
        t_one, nbytes = oracle_step_one_core(x, y.copy(), grid)
    finally:
        pool.close()
    sample = ("per step: the full workload (fp32 axpy n=2^26 + 2D stencil 4096x4096, x 6 "
              "schedules), oracle on %d cores (one slice per core)" % pool.n)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_dict(None),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.n, "kind": "oracle",
                             "sample": sample,
                             "one_core": {"value": nbytes / t_one / 1e9, "unit": UNIT,
                                          "cores": 1, "sample": "one full step"}},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict(points):
    c = {"workload": "worksharing sweep step: fp32 axpy y=3x+y n=2^26 and 2D 5-point stencil "
                     "4096x4096 fp32 (uniform [0,1), seeds 0/1), each under schedules "
                     "static(1), static(8), static(64), static, dynamic(256), auto",
         "l2": "inputs larger than L2: every stencil launch follows an 805 MB axpy stream",
         "parallelism": "one GPU per rank, independent copies (weak scaling)"}
    if points:
        c["teams_threads"] = {k: list(v) for k, v in points.items()}
    return c


# -- GPU leg ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the reduction and batched-region measurements")
    ap.add_argument("--sets", type=int, default=1,
                    help="--single: rotate the launches over this many copies of the buffers")
    ap.add_argument("--single", default=None,
                    help="profiling aid: only launch plan entries whose name contains this "
                         "(e.g. axpy/auto), or one of reduce/fp32, reduce/bf16, reduce/int64, "
                         "batch; warmup + steps times, and print the mean time")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2106_03219_gb300 import build_lib, inputs
    from paper_2106_03219_gb300 import omprt as R

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build_lib.build()
    rt = R.Runtime(local)
    sms = rt.sm_count
    points = tuned_points(sms)
    stream = torch.cuda.current_stream()

    x = torch.from_numpy(inputs.f32_uniform01(N_AXPY, 0)).cuda()
    y = torch.from_numpy(inputs.f32_uniform01(N_AXPY, 1)).cuda()
    grid = torch.from_numpy(inputs.grid_f32(GRID, GRID, 0)).cuda()
    out = torch.empty_like(grid)

    def launches(xx, yy, gg, oo):
        L = []
        for label, sched, chunk in SCHEDULES:
            G, T = points["axpy/" + label]
            L.append(("axpy/" + label, AXPY_BYTES,
                      R.loop_desc(R.BODY_AXPY, n=N_AXPY, x=xx, y=yy, alpha=3.0), sched, chunk, G, T))
            G, T = points["stencil2d/" + label]
            L.append(("stencil2d/" + label, STENCIL_BYTES,
                      R.loop_desc(R.BODY_STENCIL2D5, n=GRID * GRID, x=gg, out=oo, nx=GRID,
                                  ny=GRID), sched, chunk, G, T))
        return L

    plan = launches(x, y, grid, out)
    if args.single and (args.single.startswith("reduce/") or args.single == "batch"):
        del x, y, grid, out, plan
        return run_single_extra(rt, R, torch, inputs, args)
    if args.single:
        return run_single(rt, torch, plan, args, launches, inputs)
    step_bytes = sum(b for _, b, *_ in plan)

    def new_events():
        return (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def run_step(record=None, only=None):
        """One step; record[i] brackets launch i with events (all launches, or
        launch `only` alone)."""
        for i, (name, _, desc, sched, chunk, G, T) in enumerate(plan):
            mark = record is not None and (only is None or i == only)
            if mark:
                record[i if only is None else 0][0].record(stream)
            rt.launch_region(desc, sched, chunk, G, T, stream=stream)
            if mark:
                record[i if only is None else 0][1].record(stream)

    for _ in range(args.warmup):
        run_step()
    torch.cuda.synchronize()
    assert rt.sync_status() == 0

    # Per-kernel breakdown, outside the timed region: each launch between its
    # own event pair.  An event between two launches orders them (the second
    # no longer overlaps the first one's tail) and costs about 1.5 us itself,
    # so these times include that and the step below carries events around
    # its dominant kernel only.
    evk = [[new_events() for _ in plan] for _ in range(args.steps)]
    for k in range(args.steps):
        run_step(evk[k])
    torch.cuda.synchronize()
    per = {}
    for i, (name, nbytes, *_rest) in enumerate(plan):
        ts = [evk[k][i][0].elapsed_time(evk[k][i][1]) for k in range(args.steps)]
        per[name] = (nbytes, statistics.mean(ts))
    dom = max(per, key=lambda k: per[k][1])
    dom_i = [p[0] for p in plan].index(dom)

    def timed_steps(ev):
        barrier(ws)
        torch.cuda.synchronize()
        t_start, t_end = new_events()
        t_start.record(stream)
        for k in range(args.steps):
            run_step(ev[k], only=dom_i)
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        return max_over_ranks(t_start.elapsed_time(t_end), ws) / args.steps

    ev = [[new_events()] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    ms_step = timed_steps(ev)
    clk = clocks.stop()
    value = step_bytes * ws / (ms_step * 1e-3) / 1e9
    assert rt.sync_status() == 0
    dom_ms = statistics.mean(ev[k][0][0].elapsed_time(ev[k][0][1]) for k in range(args.steps))

    # the same step with plain launches (no overlap of a launch with the
    # previous one's tail), for comparison; not the reported value
    rt.set_launch_overlap(False)
    ev_off = [[new_events()] for _ in range(args.steps)]
    ms_step_off = timed_steps(ev_off)
    rt.set_launch_overlap(True)
    assert rt.sync_status() == 0
    overlap_line = {"ms_per_step_plain_launches": ms_step_off,
                    "value_plain_launches": step_bytes * ws / (ms_step_off * 1e-3) / 1e9}

    peak, peak_kind = measured_peaks()
    achieved = per[dom][0] / (dom_ms * 1e-3) / 1e9
    traffic = traffic_for(dom)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s"}
    kernels = {k: {"ms": v[1], "GBps": v[0] / (v[1] * 1e-3) / 1e9,
                   "frac": v[0] / (v[1] * 1e-3) / 1e9 / peak} for k, v in per.items()}

    # end to end through the C ABI with host buffers
    e2e = measure_e2e(rt, R, torch, inputs, plan, points, args.e2e_steps, launches)
    e2e_val = max_over_ranks(e2e["ms"], ws)
    e2e_line = {"value": step_bytes * ws / (e2e_val * 1e-3) / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"]}

    # every kernel alone, back to back on rotating buffers (steady state)
    steady = measure_kernels_steady(rt, R, torch, launches, plan, peak) \
        if not args.no_extras else None
    single = measure_single_region(rt, R, torch, inputs) if not args.no_extras else None
    sharded_red = measure_sharded(rt, R, torch, inputs, ws, rank) if not args.no_extras else None
    red_gpu, red_arrays = measure_reductions(rt, R, torch, inputs) \
        if not args.no_extras else (None, None)
    batched_forms = measure_batched(rt) if not args.no_extras else None
    learned_eval = measure_learned(rt) if not args.no_extras else None

    cpu, cpu_legs = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import cores
        pool = cores.Cores()
        try:
            cpu = cpu_worksharing(pool)
            if not args.no_extras:
                cpu_legs = {"single_region": cpu_single_region(pool),
                            "batched": cpu_batched(pool), "mlp_step": cpu_mlp()}
                red_check = cpu_reductions(pool, red_arrays, red_gpu)
                for k, v in red_check.items():
                    red_gpu[k]["vs_oracle"] = v
        finally:
            pool.close()
    reductions = red_gpu
    del red_arrays
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic", "config": config_dict(points),
                "e2e": e2e_line, "roofline": roofline, "cpu_baseline": cpu,
                "gpu_launches": len(plan) * args.steps, "clocks": clk,
                "launch_overlap": overlap_line,
                "kernels": kernels, "kernels_steady": steady, "single_region": single,
                "sharded_reduction": sharded_red,
                "reductions": reductions, "batched": batched_forms, "learned": learned_eval,
                "cpu_legs": cpu_legs, "source_hash": source_hash()}
        print(json.dumps(line))
    rt.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_single_extra(rt, R, torch, inputs, args):
    """--single reduce/{fp32,bf16,int64}: the reduction of the bench's
    reductions leg (n = 2^28, 2 teams per SM x 512 threads); --single batch:
    one persistent launch over the 4096-region batch."""
    import numpy as np
    stream = torch.cuda.current_stream()
    if args.single == "batch":
        from paper_2106_03219_gb300 import batched
        from paper_2106_03219_gb300.autotune import load_batch_table
        chunk, threads = load_batch_table()
        rs = batched.RegionSet()
        b = rs.batch(rt, chunk)
        fn = lambda: b.launch(0, threads, stream=stream)
        nbytes = rs.algorithmic_bytes()
    else:
        n = 1 << 28
        gen = {"reduce/fp32": lambda: inputs.f32_uniform_pm1(n, 0),
               "reduce/bf16": lambda: inputs.bf16_uniform_pm1(n, 0).view(np.int16),
               "reduce/int64": lambda: inputs.int64_uniform(n, 0)}.get(args.single)
        if gen is None:
            raise SystemExit("unknown --single %r" % args.single)
        t = torch.from_numpy(gen()).cuda()
        if args.single == "reduce/bf16":
            t = t.view(torch.bfloat16)
        r = torch.zeros(1, dtype=torch.int64 if args.single == "reduce/int64" else torch.float64,
                        device="cuda")
        sms = rt.sm_count
        fn = lambda: rt.reduce(R.OP_SUM, t, r, R.PREC_COMP_F64, 2 * sms, 512, stream=stream)
        nbytes = t.numel() * t.element_size()
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    assert rt.sync_status() == 0
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"single": args.single, "ms": ms, "GBps": nbytes / (ms * 1e-3) / 1e9}))
    rt.close()
    return 0


def run_single(rt, torch, plan, args, launches, inputs):
    """--single NAME: the plan entries matching NAME, launched back to back.
    With --sets S > 1 launch k uses copy k mod S of the buffers, so that a
    launch's inputs were last touched S - 1 launches earlier (the steady state
    of kernels_steady: the previous launch's output still dirty in L2)."""
    names = [p[0] for p in plan]
    idx = [i for i, n in enumerate(names) if n == args.single] or \
        [i for i, n in enumerate(names) if args.single in n]
    if not idx:
        raise SystemExit("no plan entry matches %r" % args.single)
    plans = [plan]
    for k in range(1, max(1, args.sets)):
        xx = torch.from_numpy(inputs.f32_uniform01(N_AXPY, 0)).cuda()
        yy = torch.from_numpy(inputs.f32_uniform01(N_AXPY, 1)).cuda()
        gg = torch.from_numpy(inputs.grid_f32(GRID, GRID, k)).cuda()
        plans.append(launches(xx, yy, gg, torch.empty_like(gg)))
    sel = [plan[i] for i in idx]
    stream = torch.cuda.current_stream()
    count = [0]

    def launch_all():
        P = plans[count[0] % len(plans)]
        count[0] += 1
        for i in idx:
            name, _, desc, sched, chunk, G, T = P[i]
            rt.launch_region(desc, sched, chunk, G, T, stream=stream)

    for _ in range(args.warmup):
        launch_all()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        launch_all()
    e1.record(stream)
    torch.cuda.synchronize()
    assert rt.sync_status() == 0
    ms = e0.elapsed_time(e1) / args.steps
    nbytes = sum(p[1] for p in sel)
    print(json.dumps({"single": [p[0] for p in sel], "ms": ms,
                      "GBps": nbytes / (ms * 1e-3) / 1e9}))
    rt.close()
    return 0


def measure_reductions(rt, R, torch, inputs, n=1 << 28, reps=5):
    """GB/s of the reduction configuration: n = 2^28 sums (fp32 uniform and
    lognormal, bf16, int64) and fp32 max / min at the shipped precision
    (compensated fp32, fp64 combine), 2 teams per SM x 512 threads (every
    team resident: one wave); inputs
    (0.5-2 GB) are larger than L2.  The fp sums are also run at the two
    comparison precisions (compensated fp32 with an fp32 combine, plain fp32)
    for the error report.  Three warm-up launches, then the mean of `reps`.
    Returns (per-result dict, host arrays)."""
    out, arrays = {}, {}
    sms = rt.sm_count
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    resi = torch.zeros(1, dtype=torch.int64, device="cuda")
    peak, _ = measured_peaks()
    cases = [("fp32_pm1_sum", lambda: inputs.f32_uniform_pm1(n, 0), R.OP_SUM, res),
             ("fp32_lognormal_sum", lambda: inputs.f32_lognormal_signed(n, 0), R.OP_SUM, res),
             ("bf16_sum", lambda: inputs.bf16_uniform_pm1(n, 0), R.OP_SUM, res),
             ("int64_sum", lambda: inputs.int64_uniform(n, 0), R.OP_SUM, resi)]
    for name, gen, op, r in cases:
        a = gen()
        arrays[name] = a
        t = torch.from_numpy(a.view(np.int16) if name == "bf16_sum" else a).cuda()
        if name == "bf16_sum":
            t = t.view(torch.bfloat16)
        ops = [(name, op)] if name != "fp32_pm1_sum" else [(name, op), ("fp32_max", R.OP_MAX),
                                                           ("fp32_min", R.OP_MIN)]
        for label, o in ops:
            for _ in range(3):  # warm-up
                rt.reduce(o, t, r, R.PREC_COMP_F64, 2 * sms, 512)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                rt.reduce(o, t, r, R.PREC_COMP_F64, 2 * sms, 512)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = t.numel() * t.element_size() / (ms * 1e-3) / 1e9
            v = r.cpu()[0].item()
            if label in ("fp32_max", "fp32_min"):
                out[label] = {"ms": ms, "GBps": gbs, "frac": gbs / peak, "value": v}
                continue
            out[label] = {"ms": ms, "GBps": gbs, "frac": gbs / peak, "shipped": v}
            if o == R.OP_SUM and name != "int64_sum":
                for var, prec in (("comp_f32", R.PREC_COMP_F32), ("naive_f32", R.PREC_NAIVE_F32)):
                    rt.reduce(o, t, r, prec, 2 * sms, 512)
                    out[label][var] = r.cpu()[0].item()
        del t
    assert rt.sync_status() == 0
    return out, arrays


def measure_sharded(rt, R, torch, inputs, ws, rank, n=1 << 28, reps=5):
    """The reduction configuration's fp32 sum (n = 2^28, U[-1,1]) sharded over
    the ranks (strong scaling): rank r reduces its contiguous block on its own
    GPU, then one all-gather of 8 bytes per rank and the rank-order fp64
    combine.  Time: the slowest rank's local reduction (events, mean of
    `reps`) plus the exchange (host clock, barrier-to-barrier)."""
    from paper_2106_03219_gb300 import sharded
    s, c = sharded.rank_block(n, ws, rank)
    a = inputs.f32_uniform_pm1(n, 0)
    shard = torch.from_numpy(a[s:s + c]).cuda()
    del a
    sms = rt.sm_count
    stream = torch.cuda.current_stream()
    sharded.reduce_shard(rt, R.OP_SUM, shard, R.PREC_COMP_F64, 2 * sms, 512)
    torch.cuda.synchronize()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        rt.reduce(R.OP_SUM, shard, res, R.PREC_COMP_F64, 2 * sms, 512, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_local = max_over_ranks(e0.elapsed_time(e1) / reps, ws)
    v = res.item()
    barrier(ws)
    t0 = time.perf_counter()
    total = sharded.combine(sharded.gather_partials(v, False), R.OP_SUM, False)
    barrier(ws)
    ms_x = max_over_ranks((time.perf_counter() - t0) * 1e3, ws)
    assert rt.sync_status() == 0
    return {"n": n, "ranks": ws, "block": [s, c], "local_ms": ms_local, "exchange_ms": ms_x,
            "GBps": 4 * n / ((ms_local + ms_x) * 1e-3) / 1e9, "result": total,
            "scaling": "strong"}


def measure_single_region(rt, R, torch, inputs, reps=200):
    """Configuration 1: int32 axpy y = 3x + y over n = 2^20 with an int64 sum
    reduction, 4 teams x 128 threads, schedule(static).  Its 12.6 MB stay in
    L2 between back-to-back launches, so it is reported as time, GB/s and
    launch latency, not against the HBM roofline."""
    n = 1 << 20
    x = torch.from_numpy(inputs.int32_uniform(n, 0)).cuda()
    y = torch.from_numpy(inputs.int32_uniform(n, 1)).cuda()
    r = torch.zeros(1, dtype=torch.int64, device="cuda")
    desc = R.loop_desc(R.BODY_AXPY, n=n, x=x, y=y, alpha=3)
    red = R.ReduceDesc(R.OP_SUM, 0, r.data_ptr())
    stream = torch.cuda.current_stream()
    go = lambda: rt.launch_region(desc, R.SCHED_STATIC, 0, 4, 128, red=red, stream=stream)
    for _ in range(5):
        go()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        go()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # host cost of one call (argument checks + launch), no synchronisation
    t0 = time.perf_counter()
    for _ in range(reps):
        go()
    t_call = (time.perf_counter() - t0) / reps
    torch.cuda.synchronize()
    # one launch from the host call to its completion seen by the host
    lat = []
    for _ in range(50):
        t0 = time.perf_counter()
        go()
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0)
    assert rt.sync_status() == 0
    # the same launch on a fresh box stays 4 teams: G = 4 uses 4 of the SMs
    return {"n": n, "teams": 4, "threads": 128, "device_ms_per_launch": ms,
            "GBps": 12 * n / (ms * 1e-3) / 1e9, "host_call_us": t_call * 1e6,
            "launch_to_done_us": statistics.median(lat) * 1e6, "l2_resident": True}


def measure_kernels_steady(rt, R, torch, launches, plan, peak, nsets=4, reps=3):
    """Every kernel of the step alone, launched back to back over `nsets`
    copies of its buffers in turn (each launch's inputs were last touched
    three launches earlier, more than L2 ago), so each launch pays the
    write-back of the previous one's output as it would in a stream of its
    own kind.  In the step itself a stencil launch follows an 805 MB axpy and
    pays for the write-back of that axpy's dirty lines (up to L2's size),
    and the axpy after it pays less; these figures take that cross-charge
    out.  Launches overlap the previous one's tail (the runtime's default);
    `plain_launches` repeats the figures without that.
    `device_copy_of_the_grid` times a plain device copy of the stencil's
    134 MB the same way: the ceiling at that launch size for plain launches."""
    from paper_2106_03219_gb300 import inputs
    sets = []
    for k in range(nsets):
        xx = torch.from_numpy(inputs.f32_uniform01(N_AXPY, 0)).cuda()
        yy = torch.from_numpy(inputs.f32_uniform01(N_AXPY, 1)).cuda()
        gg = torch.from_numpy(inputs.grid_f32(GRID, GRID, 0)).cuda()
        oo = torch.empty_like(gg)
        sets.append(((xx, yy, gg, oo), launches(xx, yy, gg, oo)))
    stream = torch.cuda.current_stream()

    def alone(i):
        for _, L in sets:
            _, _, d, sched, chunk, G, T = L[i]
            rt.launch_region(d, sched, chunk, G, T, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            for _, L in sets:
                _, _, d, sched, chunk, G, T = L[i]
                rt.launch_region(d, sched, chunk, G, T, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / (reps * nsets)

    out, plain = {}, {}
    for i, (name, nbytes, *_r) in enumerate(plan):
        ms = alone(i)
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "GBps": gbs, "frac": gbs / peak}
    rt.set_launch_overlap(False)
    for i, (name, nbytes, *_r) in enumerate(plan):
        ms = alone(i)
        plain[name] = {"ms": ms, "frac": nbytes / (ms * 1e-3) / 1e9 / peak}
    rt.set_launch_overlap(True)
    out["plain_launches"] = plain
    assert rt.sync_status() == 0
    # the same-size ceiling: a plain device copy (torch's) of the stencil's
    # bytes, the grid in and out, launched the same way over the same buffers
    for (xx, yy, gg, oo), _ in sets:
        oo.copy_(gg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        for (xx, yy, gg, oo), _ in sets:
            oo.copy_(gg)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (reps * nsets)
    gbs = 8 * GRID * GRID / (ms * 1e-3) / 1e9
    out["device_copy_of_the_grid"] = {"ms": ms, "GBps": gbs, "frac": gbs / peak,
                                      "kernel": "torch copy_ (library, plain launches), "
                                                "not in the step"}
    del sets
    return out


def measure_batched(rt):
    """Regions/s of the 4096-region batch: persistent kernel vs one launch per
    region, eager and under CUDA graphs."""
    from paper_2106_03219_gb300 import batched
    from paper_2106_03219_gb300.autotune import load_batch_table
    chunk, threads = load_batch_table()
    rs = batched.RegionSet()
    r = batched.time_forms(rt, rs, reps=5, chunk_elems=chunk, threads=threads)
    del rs
    return r


def measure_learned(rt, count=2000, seed=1):
    """The committed cost model against the plain heuristic on held-out loops
    (seed 1, never used in training): each loop's two picks timed
    interleaved (5 launches each, medians), the whole set three times in
    fresh orders (gain mean and spread); and, from one timing of all 12
    configurations, the gap of each pick to the per-loop best."""
    from paper_2106_03219_gb300 import learned
    model = learned.Model.load()
    if model is None:
        return None
    buf = learned.LoopBuffers()
    kind, n = learned.make_loops(count, seed)
    rep = learned.compare_picks(rt, model, kind, n, buf, reps=5, rounds=3)
    T = learned.time_loops(rt, kind, n, buf, reps=3)
    rep["vs_best"] = learned.evaluate(rt, model, kind, n, T, buf)
    del buf
    return rep


def traffic_for(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, if it
    was taken on the current source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_hash") != source_hash():
        return None
    v = d.get("kernels", {}).get(kernel)
    return None if v is None else float(v)


def measure_e2e(rt, R, torch, inputs, plan, points, steps, launches):
    """Step time with H2D of the inputs from pinned memory and D2H of the
    results inside the timed region, every step.

    A streaming pipeline over three CUDA streams and NBUF device buffer
    sets: step k's H2D (copy stream) overlaps earlier steps' kernels
    (compute stream) and D2H (the link's other direction).  CUDA events
    order H2D -> kernels -> D2H within a step, and keep step k's H2D off a
    buffer set until step k - NBUF's D2H has read it."""
    NBUF = 3
    hx = torch.from_numpy(inputs.f32_uniform01(N_AXPY, 0)).pin_memory()
    hy = torch.from_numpy(inputs.f32_uniform01(N_AXPY, 1)).pin_memory()
    hg = torch.from_numpy(inputs.grid_f32(GRID, GRID, 0)).pin_memory()
    ry = torch.empty_like(hy).pin_memory()
    ro = torch.empty_like(hg).pin_memory()
    bufs = []
    for _ in range(NBUF):
        dx = torch.empty(N_AXPY, device="cuda")
        dy = torch.empty(N_AXPY, device="cuda")
        dg = torch.empty((GRID, GRID), device="cuda")
        do = torch.empty_like(dg)
        bufs.append((dx, dy, dg, do, launches(dx, dy, dg, do)))
    s_in, s_run, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()

    def pipeline(nsteps):
        done_out = [None] * NBUF  # last D2H event per buffer set
        for k in range(nsteps):
            dx, dy, dg, do, L = bufs[k % NBUF]
            if done_out[k % NBUF] is not None:
                s_in.wait_event(done_out[k % NBUF])
            with torch.cuda.stream(s_in):
                dg.copy_(hg, non_blocking=True)
                dx.copy_(hx, non_blocking=True)
                dy.copy_(hy, non_blocking=True)
            e_in = ev()
            e_in.record(s_in)
            s_run.wait_event(e_in)
            for name, _, desc, sched, chunk, G, T in L:
                rt.launch_region(desc, sched, chunk, G, T, stream=s_run)
            e_run = ev()
            e_run.record(s_run)
            s_out.wait_event(e_run)
            with torch.cuda.stream(s_out):
                ro.copy_(do, non_blocking=True)
                ry.copy_(dy, non_blocking=True)
            done_out[k % NBUF] = ev()
            done_out[k % NBUF].record(s_out)
        return done_out

    pipeline(NBUF)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s_in)
    last = pipeline(steps)
    for e in last:
        if e is not None:
            s_out.wait_event(e)
    t1.record(s_out)
    torch.cuda.synchronize()
    h2d = (hx.numel() + hy.numel() + hg.numel()) * 4
    d2h = (ry.numel() + ro.numel()) * 4
    return {"ms": t0.elapsed_time(t1) / steps, "h2d": h2d, "d2h": d2h}


if __name__ == "__main__":
    sys.exit(main())
