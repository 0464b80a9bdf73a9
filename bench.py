#!/usr/bin/env python
"""Benchmark of the GB300 NUHT: one JSON line on stdout (rank 0).

Workload (one step = the whole transform from unsorted device inputs):
    n = m = 1e6 points / frequencies, nu = 0, eps = 1e-12,
    r ~ U[0, 1], omega ~ U[0, 1e5], c ~ N(0, 1), FP64, seed 2 (+ rank),
    plan (domain check, device sort, subdivision, work lists) + execute
    (gather, local moments, type-3 spread / FFT / interpolation, local
    evaluation, direct blocks, scatter).
value = (n + m) * ranks / seconds per step (max over ranks), with the L2
flushed between timed steps.  `execute_only` repeats the measurement with the
plan reused.  `e2e` times nuht_transform_host: pinned host inputs -> device,
plan, execute, g back to the host.

--impl reference times the oracle (plain FP64 direct sum on the host cores)
on a bounded sample of output rows of the same workload, extrapolated to the
whole transform.
"""
import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "NUHT (n+m)/s at ε=1e-8 fp64 vs fp32-mixed; batched; % HBM roofline"
UNIT = "(n+m)/s"
L2_FLUSH_BYTES = 512 << 20
HBM_FALLBACK_GBS = 6800.0
DTYPE = ("df64: double-float (pairs of FP32, ~48-bit) tap, moment and Bessel arithmetic; "
         "64-bit fixed-point positions and phases; FP64 set-up and FP64 atomic accumulation")


def df_model_peak(dev):
    """Unit-count model of the double-float peak (context beside the measured
    one): the FP32 pipes issue 128 instructions per clock per SM and a
    compensated double-float multiply-add (TwoProduct + TwoSum + corrections)
    costs 12 of them, so FP64-equivalent FLOP/s = 2 x 128 x SMs x clock / 12.
    SMs from the device, the clock from MEASURED_PEAKS.json (sm_max_mhz).
    Returns (TFLOP/s, description)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except Exception:
        pass
    tf = 2 * 128 * sms * mhz * 1e6 / 12 / 1e12
    return tf, "128 FP32 instr/clk/SM x %d SMs x %.0f MHz / 12 instr x 2 FLOP" % (sms, mhz)


def measured_hbm_peak():
    """(GB/s, source): the machine's measured copy bandwidth, else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = float(json.load(open(path))["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback (no MEASURED_PEAKS.json)"


def probe_alu_peaks(dev):
    """Issue-rate probe of the arithmetic the kernels run (nuht_probe_alu), timed
    with CUDA events on this GPU: FP32 FMA, FP64 FMA and the double-float
    compensated multiply-add acc_fma, in TFLOP/s (2 FLOP per multiply-add)."""
    from paper_2411_09583_gb300.nuht import probe_alu
    out = {}
    for kind, iters in (("ffma", 1 << 20), ("dfma", 1 << 14), ("acc_fma", 1 << 17)):
        probe_alu(kind, 1 << 8)
        best = max(probe_alu(kind, iters)[2] for _ in range(3))
        out[kind + "_tflops"] = best / 1e12
    out["basis"] = ("nuht_probe_alu: 8 independent chains per thread, 4 CTAs x 256 threads per SM, "
                    "CUDA events, best of 3 launches; acc_fma is the double-float product added to a "
                    "compensated FP32 sum exactly as the execute kernels do it (FP64-equivalent FLOPs)")
    return out


def sampled_error(nu, r, omega, c, g, eps, rows, ref=None):
    """Worst max_k |g_k - oracle_k| / (eps ||c||_1) over the vectors, on the
    sampled output rows (the oracle's direct sum, outside any timed region).
    The accuracy contract is <= 10, i.e. err_over_tol <= 1."""
    import numpy as np

    import oracle
    if ref is None:
        ref = oracle.direct_rows(nu, r, omega, c, rows)
    gr = np.asarray(g)[rows]
    err = np.max(np.abs(gr - ref), axis=0)
    c1 = np.abs(np.asarray(c)).sum(axis=0)
    v = float(np.max(err / (eps * c1)))
    return {"err_over_eps_c1": v, "err_over_tol": v / 10.0, "rows": int(len(rows)),
            "against": "oracle direct sum on sampled rows"}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--m", type=int, default=1_000_000)
    ap.add_argument("--nu", type=int, default=0)
    ap.add_argument("--eps", type=float, default=1e-12)
    ap.add_argument("--omega-max", type=float, default=1e5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched / mixed-precision side measurements")
    ap.add_argument("--no-autotune", action="store_true",
                    help="library default options instead of the autotuned ones (min_size is chosen "
                         "from experiments, Algorithm 2)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target duration of the oracle sample")
    ap.add_argument("--only", choices=["large_grid", "mixed", "multi_vector"], default=None,
                    help="run one side workload alone and print its JSON (for profiling)")
    ap.add_argument("--opts", type=str, default=None,
                    help="plan options as JSON (e.g. '{\"min_size\": 2048}') instead of the autotuner's")
    return ap.parse_args(argv)


def workload_config(a):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return {"workload": "nuht_fp64_uniform_n%d_m%d_nu%d_eps%g" % (a.n, a.m, a.nu, a.eps),
            "parallelism": "replicas" if ws > 1 else "1 GPU",
            "n": a.n, "m": a.m, "nu": a.nu, "eps": a.eps,
            "r": "U[0,1]", "omega": "U[0,%g]" % a.omega_max, "c": "N(0,1) real",
            "seed": 2, "step": "plan+execute from unsorted device inputs",
            "l2": "flushed between timed steps (%d MiB write)" % (L2_FLUSH_BYTES >> 20)}


# ---------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws, device=None):
    """Largest value over all ranks (identity for a single process)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- oracle timing
def oracle_sample(a, r, omega, c, target_s):
    """Time the oracle on sampled output rows; returns (extrapolated (n+m)/s, rows, seconds)."""
    import numpy as np

    import oracle
    from paper_2411_09583_gb300.workloads import sample_rows
    oracle.build()
    probe = sample_rows(omega.size, 32, seed=1234)
    t0 = time.perf_counter()
    oracle.direct_rows(a.nu, r, omega, c, probe)
    dt = max(time.perf_counter() - t0, 1e-6)
    nrows = int(min(max(32, 32 * target_s / dt), omega.size, 20000))
    rows = sample_rows(omega.size, nrows, seed=4321)
    t0 = time.perf_counter()
    ref = oracle.direct_rows(a.nu, r, omega, c, rows)
    dt = time.perf_counter() - t0
    full = dt * omega.size / nrows
    return (r.size + omega.size) / full, nrows, dt, rows, ref


# ---------------------------------------------------------------- reference arm
def run_reference(a):
    import numpy as np

    from paper_2411_09583_gb300.workloads import uniform_problem
    r, omega, c = uniform_problem(a.n, a.m, omega_max=a.omega_max, seed=2)
    per_step = max(2.0, min(a.cpu_seconds, 120.0 / max(1, a.steps + a.warmup)))
    for _ in range(a.warmup):
        oracle_sample(a, r, omega, c, per_step * 0.3)
    vals, rows_used, secs = [], 0, 0.0
    for _ in range(a.steps):
        v, nrows, dt, _, _ = oracle_sample(a, r, omega, c, per_step)
        vals.append(v)
        rows_used, secs = nrows, secs + dt
    value = statistics.median(vals)
    cores = os.cpu_count()
    sample = ("oracle direct sum over all n points for %d random output rows per step, "
              "extrapolated to m rows" % rows_used)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * (a.n + a.m) / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(a),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- our arm
def _dominant_flops(stage, info, blocks, tab):
    """Algorithmic FP64 FLOPs of one launch of the stage: the work the method
    must do per unit (Sec. 3-4), not the kernels' own operation counts.

    asymptotic point or frequency: 2M w complex-by-real tap updates, 4 w Q flops
    (Q = 2M); local point or frequency: (L+1) term updates, 4 (L+1) flops;
    direct entry: one J_nu evaluation, counted as 150 flops."""
    w, Q, L = tab["w"], 2 * info["M"], info["L"]
    asy, loc, dirb = blocks[1], blocks[0], blocks[2]
    if stage == "asy_spread":
        units = float((asy[:, 3] - asy[:, 2] + 1).sum())
        return units * 4 * w * Q, units
    if stage == "asy_interp":
        units = float((asy[:, 1] - asy[:, 0] + 1).sum())
        return units * 4 * w * Q, units
    if stage == "local_moments":
        units = float((loc[:, 3] - loc[:, 2] + 1).sum())
        return units * 4 * (L + 1), units
    if stage == "local_eval":
        units = float((loc[:, 1] - loc[:, 0] + 1).sum())
        return units * 4 * (L + 1), units
    if stage == "direct":
        units = float(((dirb[:, 1] - dirb[:, 0] + 1) * (dirb[:, 3] - dirb[:, 2] + 1)).sum())
        return units * 150.0, units
    return None, None


def _code_only(text):
    """C/CUDA source without comments and blank lines (comment edits keep a
    capture valid; any code change invalidates it)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def source_hash(*names):
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_2411_09583_gb300", "csrc", nm), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def stored_traffic(kernel, workload, opts=None, units=None):
    """DRAM bytes per launch of the kernel from the committed ncu summary, if its
    sources are unchanged: as captured when the plan options are those of the
    capture, else scaled by the units the launch processes.  Returns (bytes,
    basis) or (None, reason)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None, "no capture"
    try:
        db = json.load(open(path))
        ent = db.get(kernel + "@" + workload) or db.get(kernel)
        if not ent or ent.get("workload") != workload:
            return None, "no capture of this kernel and workload"
        if ent.get("source_hash") != source_hash(*ent.get("sources", [])):
            return None, "kernel changed since the capture"
        if ent.get("opts", {}) == (opts or {}):
            return ent.get("bytes_per_launch"), "ncu capture of this launch configuration"
        if units and ent.get("units_per_launch"):
            return (ent["bytes_per_launch"] * units / ent["units_per_launch"],
                    "ncu capture at options %s scaled by units processed" % ent.get("opts"))
        return None, "captured at other options"
    except Exception as e:
        return None, "unreadable capture (%s)" % e


def run_batched(dev, steps):
    """256 uneven problems (n, m log-uniform in [1e3, 1e5], nu in 0..20, omega ~ U[0, m],
    eps = 1e-8) in one plan; execute replayed as one captured CUDA graph."""
    import numpy as np
    import torch

    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300.workloads import batch_problems
    probs = batch_problems(count=256, lo=1e3, hi=1e5, nu_max=20, seed=5)
    nus = [p[0] for p in probs]
    n = [p[1].size for p in probs]
    m = [p[2].size for p in probs]
    dr = torch.tensor(np.concatenate([p[1] for p in probs]), device=dev)
    dw = torch.tensor(np.concatenate([p[2] for p in probs]), device=dev)
    dc = torch.tensor(np.concatenate([p[3] for p in probs]), device=dev)
    units = int(sum(n) + sum(m))
    stream = torch.cuda.current_stream(dev)
    # options picked by the autotuner (execute time of the batch); the orders
    # differ between problems, so M stays per-problem (heuristic)
    from paper_2411_09583_gb300.autotune import autotune, candidates
    grid = candidates(nus, 1e-8, min_sizes=(512, 1024, 2048), spread_tiles=(0, 128), m_offsets=(0,))
    best, table = autotune(nus, dr, dw, dc, 1e-8, sizes=(n, m), objective="execute", reps=3, grid=grid)
    default_ms = [t for t, o in table if o == {"min_size": 1024, "spread_tile": 0, "m_terms": 0, "interp_tile": 0}]
    for _ in range(2):
        Plan.many(nus, dr, n, dw, m, 1e-8, **best).close()
    plan_ms = []
    for _ in range(max(3, steps // 4)):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        bp = Plan.many(nus, dr, n, dw, m, 1e-8, **best)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        plan_ms.append(s0.elapsed_time(s1))
        bp.close()
    bp = Plan.many(nus, dr, n, dw, m, 1e-8, **best)
    g = torch.empty(sum(m), dtype=torch.float64, device=dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(2):
            bp.execute(dc, out=g)
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bp.execute(dc, out=g)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize(dev)
    ex_ms = []
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(steps):
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        graph.replay()
        s1.record(stream)
        torch.cuda.synchronize(dev)
        ex_ms.append(s0.elapsed_time(s1))
    info = bp.info()
    bp.close()
    # the same batch with the local blocks in one persistent launch
    bpp = Plan.many(nus, dr, n, dw, m, 1e-8, persistent=True, **best)
    gp = torch.empty(sum(m), dtype=torch.float64, device=dev)
    with torch.cuda.stream(side):
        for _ in range(2):
            bpp.execute(dc, out=gp)
    stream.wait_stream(side)
    graph_p = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_p):
        bpp.execute(dc, out=gp)
    for _ in range(3):
        graph_p.replay()
    torch.cuda.synchronize(dev)
    exp_ms = []
    for _ in range(steps):
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        graph_p.replay()
        s1.record(stream)
        torch.cuda.synchronize(dev)
        exp_ms.append(s0.elapsed_time(s1))
    pers_status = bpp.status()
    bpp.close()
    exe = statistics.median(ex_ms)
    pl = statistics.median(plan_ms)
    # accuracy of the graph's result: 10 sampled rows of every problem
    gh = g.cpu().numpy()
    rng = np.random.default_rng(77)
    worst, off = 0.0, 0
    for nu_i, rr, ww, cc in probs:
        rows = np.sort(rng.choice(ww.size, size=min(10, ww.size), replace=False))
        e = sampled_error(nu_i, rr, ww, cc, gh[off:off + ww.size], 1e-8, rows)
        worst = max(worst, e["err_over_eps_c1"])
        off += ww.size
    return {"workload": "256 problems, n, m ~ 10^U[3,5], nu ~ U{0..20}, omega ~ U[0, m], eps 1e-8",
            "units_n_plus_m": units, "execute_graph_ms": exe, "plan_ms": pl,
            "value_execute": units / (exe * 1e-3), "value_plan_execute": units / ((exe + pl) * 1e-3),
            "unit": UNIT, "execute": "one CUDA graph replay (one launch per stage over all problems)",
            "autotuned_opts": best, "autotune_default_execute_ms": default_ms[0] if default_ms else None,
            "autotune_best_execute_ms": table[0][0],
            "execute_graph_ms_persistent_local": statistics.median(exp_ms),
            "persistent_status": pers_status,
            "blocks_local_asy_direct": [info["n_local"], info["n_asy"], info["n_direct"]],
            "error": {"err_over_eps_c1": worst, "err_over_tol": worst / 10.0, "rows": 10 * len(probs),
                      "against": "oracle direct sum, 10 sampled rows of every problem (worst problem)"}}


def run_mixed(dev, steps):
    """n = m = 4e6, nu = 1, r = 10^U[-3,0], omega ~ U[0, 4e4], complex c, eps = 1e-5:
    the FP32 mixed path and the FP64 path on the same problem (plan + execute)."""
    import torch

    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300.workloads import loguniform_problem, sample_rows
    r, omega, c = loguniform_problem(4_000_000, 4_000_000, omega_max=4e4, seed=4, complex_c=True)
    dr, dw, dc = (torch.tensor(x, device=dev) for x in (r, omega, c))
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    from paper_2411_09583_gb300.autotune import autotune, candidates
    out = {"workload": "n = m = 4e6, nu = 1, r = 10^U[-3,0], omega ~ U[0,4e4], complex c, eps 1e-5",
           "unit": UNIT}
    grid = candidates([1], 1e-5, min_sizes=(256, 512, 1024, 2048), spread_tiles=(0, 128), m_offsets=(0, 1))
    for prec in ("mixed", "fp64"):
        # options per precision from the autotuner (plan + execute), outside the timing
        opts, _ = autotune(1, dr, dw, dc, 1e-5, objective="plan+execute", reps=2, grid=grid, precision=prec)
        for _ in range(2):
            with Plan(1, dr, dw, 1e-5, precision=prec, **opts) as p:
                p.execute(dc)
        ms = []
        for _ in range(max(3, steps // 4)):
            flush.zero_()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            p = Plan(1, dr, dw, 1e-5, precision=prec, **opts)
            p.execute(dc)
            s1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(s0.elapsed_time(s1))
            p.close()
        t = statistics.median(ms)
        with Plan(1, dr, dw, 1e-5, precision=prec, **opts) as p:
            gh = p.execute(dc).cpu().numpy()
            asy_members = p.info()["asy_members"]
            ex = []
            for _ in range(max(3, steps // 4)):
                flush.zero_()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                p.execute(dc)
                s1.record(stream)
                torch.cuda.synchronize(dev)
                ex.append(s0.elapsed_time(s1))
        stages = {}
        for _ in range(3):
            flush.zero_()
            with Plan(1, dr, dw, 1e-5, precision=prec, timing="serial", **opts) as pt:
                pt.execute(dc)
                for k, v in pt.stage_times().items():
                    stages.setdefault(k, []).append(v)
        rows = sample_rows(omega.size, 100, seed=98)
        out[prec] = {"ms_per_step": t, "value": 8e6 / (t * 1e-3), "opts": opts,
                     "execute_ms": statistics.median(ex), "asy_members": asy_members,
                     "stage_ms_alone": {k: statistics.median(v) for k, v in stages.items()},
                     "error": sampled_error(1, r, omega, c, gh, 1e-5, rows)}
    return out


def run_grad(dev, steps):
    """n = m = 1e6, nu = 0, r ~ U[0,1], omega ~ U[0,1e5], eps = 1e-10: one step of
    L = 1/2 ||A c - g*||^2 with dL/dc (adjoint) and dL/dr (adjoints of orders nu +- 1),
    plans included."""
    import numpy as np
    import torch

    from paper_2411_09583_gb300 import Plan, nuht_autograd
    from paper_2411_09583_gb300.workloads import uniform_problem
    r, omega, c = uniform_problem(1_000_000, 1_000_000, omega_max=1e5, seed=6)
    dr, dw, dc = (torch.tensor(x, device=dev) for x in (r, omega, c))
    delta = torch.tensor(np.random.default_rng(7).standard_normal(c.size), device=dev)
    with Plan(0, dr, dw, 1e-10) as p:
        gstar = p.execute(dc + 0.01 * delta)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    from paper_2411_09583_gb300.autotune import autotune, candidates
    opts, _ = autotune(0, dr, dw, dc, 1e-10, objective="plan+execute", reps=2,
                       grid=candidates([0], 1e-10, min_sizes=(1024, 2048, 4096), spread_tiles=(0,),
                                       m_offsets=(0,)))

    def one():
        tc = dc.clone().requires_grad_(True)
        tr = dr.clone().requires_grad_(True)
        g = nuht_autograd(tc, tr, dw, 0, 1e-10, **opts)
        loss = 0.5 * ((g - gstar) ** 2).sum()
        loss.backward()
        return tc.grad, tr.grad

    for _ in range(2):
        one()
    ms = []
    for _ in range(max(3, steps // 4)):
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        one()
        s1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(s0.elapsed_time(s1))
    t = statistics.median(ms)
    # accuracy of the gradients on 100 sampled points: dL/dc_j = sum_k e_k J_nu(omega_k r_j)
    # within 10 eps ||e||_1, dL/dr_j = c_j sum_k e_k omega_k J_nu'(omega_k r_j) within
    # 10 eps |c_j| ||omega e||_1, with e = A c - g* from the same forward
    import oracle
    from paper_2411_09583_gb300.workloads import sample_rows
    gc, gr = one()
    with Plan(0, dr, dw, 1e-10, **opts) as p:
        e = (p.execute(dc) - gstar).cpu().numpy()
    cols = sample_rows(r.size, 100, seed=96)
    gc, gr = gc.cpu().numpy()[cols], gr.cpu().numpy()[cols]
    ref_c = oracle.direct_rows(0, omega, r, e, cols)
    we = omega * e
    ref_r = c[cols] * 0.5 * (oracle.direct_rows(-1, omega, r, we, cols) - oracle.direct_rows(1, omega, r, we, cols))
    err_c = float(np.max(np.abs(gc - ref_c)) / (1e-10 * np.abs(e).sum()))
    err_r = float(np.max(np.abs(gr - ref_r) / (1e-10 * np.abs(c[cols]) * np.abs(we).sum())))
    return {"workload": "n = m = 1e6, nu = 0, eps 1e-10, loss 1/2||A c - g*||^2, grads c and r",
            "error": {"grad_c_err_over_eps_e1": err_c, "grad_r_err_over_eps_c_we1": err_r,
                      "err_over_tol": max(err_c, err_r) / 10.0, "rows": 100,
                      "against": "oracle direct sums (orders nu, nu - 1, nu + 1) at 100 sampled points"},
            "ms_per_step": t, "value": 2e6 / (t * 1e-3), "unit": UNIT, "opts": opts,
            "step": "plan + forward + adjoint (dL/dc) + derivative plan (orders nu-1, nu+1 on the sorted points, no re-sort) and its adjoint (dL/dr)"}


def run_stress(dev, steps):
    """Sec. 5.1.1's cases with p = O(n), nu = 0, eps = 1e-8, n = m: the
    Fourier-Bessel grid and the exponential grid (the subdivision's worst
    case), plan + execute at n = 1e4, 1e5, 1e6 (the scaling with n of the
    paper's timing study), library default options."""
    import numpy as np
    import torch

    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300.workloads import exponential_grid, fourier_bessel_grid, sample_rows
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = {"workload": "nu = 0, eps 1e-8, n = m, Fourier-Bessel and exponential grids, c ~ N(0,1)",
           "unit": UNIT, "step": "plan + execute"}
    for name, grid in (("fourier_bessel", lambda n: fourier_bessel_grid(0, n)), ("exponential", exponential_grid)):
        res = {}
        for n in (10_000, 100_000, 1_000_000):
            r, omega = grid(n)
            c = np.random.default_rng(8).standard_normal(n)
            dr, dw, c = (torch.tensor(x, device=dev) for x in (r, omega, c))
            for _ in range(2):
                with Plan(0, dr, dw, 1e-8) as p:
                    p.execute(c)
            ms = []
            for _ in range(max(3, steps // 4)):
                flush.zero_()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                p = Plan(0, dr, dw, 1e-8)
                p.execute(c)
                s1.record(stream)
                torch.cuda.synchronize(dev)
                ms.append(s0.elapsed_time(s1))
                info = p.info()
                p.close()
            t = statistics.median(ms)
            with Plan(0, dr, dw, 1e-8) as p:
                gh = p.execute(c).cpu().numpy()
            rows = sample_rows(n, 100, seed=97)
            res["%.0e" % n] = {"ms_per_step": t, "value": 2 * n / (t * 1e-3),
                               "blocks_local_asy_direct": [info["n_local"], info["n_asy"], info["n_direct"]],
                               "error": sampled_error(0, r, omega, c.cpu().numpy(), gh, 1e-8, rows)}
        out[name] = res
    return out


def run_large_grid(dev, steps):
    """One asymptotic block with grids far larger than L2 (n = m = 4e6, r ~ U[1,2],
    omega ~ U[1e7,2e7], nu = 0): the spreading, FFT and interpolation kernels
    move their grids through HBM.  FP64 at eps 1e-12 and mixed at 1e-6: plan +
    execute, each stage alone, the error on sampled rows, and the stored ncu
    DRAM bytes per launch of the three kernels as GB/s over their times."""
    import torch

    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300.workloads import large_grid_problem, sample_rows
    r, omega, c = large_grid_problem()
    dr, dw, dc = (torch.tensor(x, device=dev) for x in (r, omega, c))
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    hbm_peak, hbm_src = measured_hbm_peak()
    out = {"workload": "one asymptotic block: n = m = 4e6, nu = 0, r ~ U[1,2], omega ~ U[1e7,2e7], c ~ N(0,1)",
           "unit": UNIT, "step": "plan + execute", "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src}
    for prec, eps in (("fp64", 1e-12), ("mixed", 1e-6)):
        with Plan(0, dr, dw, eps, precision=prec) as p:
            p.execute(dc)
            info = p.info()
        ms = []
        for _ in range(max(3, steps // 4)):
            flush.zero_()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            p = Plan(0, dr, dw, eps, precision=prec)
            g = p.execute(dc)
            s1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(s0.elapsed_time(s1))
            p.close()
        stages = {}
        for _ in range(3):
            flush.zero_()
            with Plan(0, dr, dw, eps, precision=prec, timing="serial") as pt:
                pt.execute(dc)
                for k, v in pt.stage_times().items():
                    stages.setdefault(k, []).append(v)
        stages = {k: statistics.median(v) for k, v in stages.items()}
        t = statistics.median(ms)
        res = {"eps": eps, "ms_per_step": t, "value": 8e6 / (t * 1e-3), "stage_ms_alone": stages,
               "grid_cells": info["asy_rows_cols"], "fft_points": info["fft_points"],
               "error": sampled_error(0, r, omega, c, g.cpu().numpy(), eps, sample_rows(omega.size, 60, seed=92))}
        wl = "large_grid_%s" % prec
        sfx = "" if prec == "fp64" else "_f32"
        hb = {}
        for stage, kerns in (("asy_spread", ["k_asy_spread" + sfx]), ("asy_interp", ["k_asy_interp" + sfx]),
                             ("asy_fft", ["k_asy_fft_pass_a", "k_asy_fft_pass_b"])):
            got = [stored_traffic(k, wl) for k in kerns]
            if all(tr for tr, _ in got):
                tr = sum(t for t, _ in got)
                gbs = tr / (stages[stage] * 1e-3) / 1e9
                hb[stage] = {"kernels": kerns, "dram_bytes": tr, "stage_ms": stages[stage], "gbs": gbs,
                             "frac": gbs / hbm_peak}
            else:
                hb[stage] = {"kernels": kerns, "dram_bytes": None, "basis": [b for _, b in got]}
        res["hbm"] = hb
        out[prec] = res
    return out


def run_multi_vector(dev, steps, nvec=16):
    """The n = m = 1e6, nu = 0, eps = 1e-12 workload with nvec coefficient vectors in
    one execute (plan reused), against one vector: per-vector throughput with the
    default pairs (vec_group 0) and with all nvec vectors in one group (their local
    and direct blocks' Bessel work shared), stage times of the grouped call, and
    the error of every vector on sampled rows."""
    import numpy as np
    import torch

    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300.workloads import sample_rows, uniform_problem
    r, omega, _ = uniform_problem(1_000_000, 1_000_000, omega_max=1e5, seed=2)
    C = np.random.default_rng(21).standard_normal((r.size, nvec))
    dr, dw, dC = (torch.tensor(x, device=dev) for x in (r, omega, C))
    dc1 = dC[:, 0].contiguous()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = {"workload": "n = m = 1e6, nu = 0, eps 1e-12, r ~ U[0,1], omega ~ U[0,1e5], %d vectors c ~ N(0,1)" % nvec,
           "unit": UNIT, "step": "execute (plan reused), L2 flushed"}

    def timed(p, x):
        for _ in range(2):
            p.execute(x)
        ms = []
        for _ in range(max(3, steps // 4)):
            flush.zero_()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            g = p.execute(x)
            s1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(s0.elapsed_time(s1))
        return statistics.median(ms), g

    grouped = "nvec_%d_group_%d" % (nvec, nvec)
    with Plan(0, dr, dw, 1e-12, min_size=2048) as p:
        for label, x in (("nvec_1", dc1), ("nvec_%d" % nvec, dC)):
            t, _ = timed(p, x)
            k = x.shape[1] if x.dim() > 1 else 1
            out[label] = {"ms": t, "value_per_vector": 2e6 / (t * 1e-3 / k), "vectors": k, "vec_group": "pairs"}
    with Plan(0, dr, dw, 1e-12, min_size=2048, vec_group=nvec) as p:
        t, g = timed(p, dC)
        out[grouped] = {"ms": t, "value_per_vector": 2e6 / (t * 1e-3 / nvec), "vectors": nvec,
                        "vec_group": nvec}
        gh = g.cpu().numpy()
    with Plan(0, dr, dw, 1e-12, min_size=2048, vec_group=nvec, timing="serial") as p:
        p.execute(dC)
        torch.cuda.synchronize(dev)
        out[grouped]["stage_ms_serial"] = p.stage_times()
    rows = sample_rows(omega.size, 60, seed=91)
    out["error"] = sampled_error(0, r, omega, C, gh, 1e-12, rows)
    base = out["nvec_1"]["value_per_vector"]
    out["per_vector_speedup"] = {"pairs": out["nvec_%d" % nvec]["value_per_vector"] / base,
                                 "group": out[grouped]["value_per_vector"] / base}
    return out


def run_ours(a):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2411_09583_gb300 import build_native
    build_native.build()
    from paper_2411_09583_gb300 import Plan, nuht as nuht_mod
    from paper_2411_09583_gb300.nuht import kernel_launch_count, transform_host
    from paper_2411_09583_gb300.workloads import uniform_problem

    seed = 2 + rank
    r, omega, c = uniform_problem(a.n, a.m, omega_max=a.omega_max, seed=seed)
    dr, dw, dc = (torch.tensor(x, device=dev) for x in (r, omega, c))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # plan options from the autotuner (min_size, spreading tile, M around the
    # heuristic), chosen before and outside the timed region
    opts, tuned = {}, None
    if a.opts:
        opts = json.loads(a.opts)
    elif not a.no_autotune:
        from paper_2411_09583_gb300.autotune import autotune, candidates
        grid = candidates([a.nu], a.eps, min_sizes=(1024, 2048, 4096, 8192), spread_tiles=(0, 128),
                          m_offsets=(0, 1))
        opts, table = autotune(a.nu, dr, dw, dc, a.eps, objective="plan+execute", reps=3, grid=grid)
        dflt = [t for t, o in table if o == {"min_size": 1024, "spread_tile": 0, "m_terms": 0, "interp_tile": 0}]
        tuned = {"opts": opts, "best_ms": table[0][0], "default_opts_ms": dflt[0] if dflt else None,
                 "candidates": len(grid), "objective": "plan+execute"}

    def step(timing=False):
        p = Plan(a.nu, dr, dw, a.eps, timing=timing, **opts)
        g = p.execute(dc)
        return p, g

    # measured arithmetic peaks of this GPU (outside the timed region), with
    # the SM clock sampled while the probes run
    psampler = ClockSampler(dev.index if dev.index is not None else 0)
    psampler.start()
    alu = probe_alu_peaks(dev)
    alu["clocks"] = psampler.stop()

    # warm-up
    for _ in range(max(a.warmup, 0)):
        p, g = step()
        p.close()
    torch.cuda.synchronize(dev)

    # timed: K whole transforms (plan + execute), L2 flushed between steps
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    stage_ms = {}
    launches0 = kernel_launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    info = blocks = None
    for i in range(a.steps):
        flush.zero_()
        ev[i][0].record(stream)
        p, g = step(timing=True)
        ev[i][1].record(stream)
        st = p.stage_times()
        for k, v in st.items():
            stage_ms.setdefault(k, []).append(v)
        if info is None:
            info = p.info()
            blocks = [p.blocks(k) for k in range(3)]
        p.close()
    torch.cuda.synchronize(dev)
    launches = kernel_launch_count() - launches0
    g_main = g.cpu().numpy()
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3, ws, dev)
    value = ws * a.steps * (a.n + a.m) / total_s

    # execute only (plan reused)
    p = Plan(a.nu, dr, dw, a.eps, **opts)
    for _ in range(2):
        p.execute(dc)
    exe_ms = []
    for i in range(a.steps):
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        p.execute(dc)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        exe_ms.append(s0.elapsed_time(s1))
    g_exec = p.execute(dc).cpu().numpy()
    p.close()
    exe_s = max_over_ranks(sum(exe_ms) / 1e3, ws, dev)

    # end to end through the host-buffer entry point (pinned memory)
    hr = torch.from_numpy(r).pin_memory().numpy()
    hw = torch.from_numpy(omega).pin_memory().numpy()
    hc = torch.from_numpy(c).pin_memory().numpy()
    hg = torch.empty(a.m, dtype=torch.float64).pin_memory().numpy()
    transform_host(a.nu, hr, hw, hc, a.eps, out=hg, **opts)
    e2e_ms = []
    for i in range(max(3, a.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize(dev)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        gh = transform_host(a.nu, hr, hw, hc, a.eps, out=hg, **opts)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms.append(s0.elapsed_time(s1))
    g_e2e = np.array(gh, copy=True)
    e2e_s = max_over_ranks(sum(e2e_ms) / 1e3, ws, dev)
    e2e_value = ws * len(e2e_ms) * (a.n + a.m) / e2e_s

    # each stage alone (outside the timed region): plans with serial stage
    # timing run every stage in order on one stream
    serial_ms = {}
    for _ in range(3):
        flush.zero_()
        p = Plan(a.nu, dr, dw, a.eps, timing="serial", **opts)
        p.execute(dc)
        for k, v in p.stage_times().items():
            serial_ms.setdefault(k, []).append(v)
        p.close()
    torch.cuda.synchronize(dev)
    mean_serial = {k: statistics.median(v) for k, v in serial_ms.items()}

    # dominant kernel (largest time alone) and its roofline (FP64 ALU bound),
    # achieved over its live launch duration in the timed steps
    mean_stage = {k: sum(v) / len(v) for k, v in stage_ms.items()}
    rated = ("asy_spread", "asy_interp", "local_moments", "local_eval", "direct")
    dom = max((k for k in mean_serial if k in rated), key=mean_serial.get)
    tab = {"w": info["nufft_width"], "deg": info["nufft_degree"]}
    flops, units = _dominant_flops(dom, info, blocks, tab)
    kernel_of = {"asy_spread": "k_asy_spread", "asy_interp": "k_asy_interp",
                 "local_moments": "k_local_moments", "local_eval": "k_local_eval",
                 "direct": "k_direct", "asy_fft": "k_asy_fft_small"}
    roof = None
    hbm_peak, hbm_src = measured_hbm_peak()
    if flops is not None:
        ach = flops / (mean_stage[dom] * 1e-3) / 1e12
        peak = alu["acc_fma_tflops"]
        roof = {"bound": "alu", "kernel": kernel_of.get(dom, dom), "stage": dom,
                "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak,
                "peak_source": "measured in this run (nuht_probe_alu, burst): FP64-equivalent FLOP/s of "
                               "the double-float compensated multiply-add acc_fma on the FP32 pipes; "
                               "FP32 FMA %.1f, FP64 FMA %.3f TFLOP/s measured beside it; unit-count model "
                               "%.3f (%s)" % ((alu["ffma_tflops"], alu["dfma_tflops"]) + df_model_peak(dev)),
                "algorithmic_flops_per_launch": flops, "units_per_launch": units,
                "launch_ms": mean_stage[dom], "launch_ms_alone": mean_serial[dom]}
        tr, basis = stored_traffic(kernel_of.get(dom, dom), workload_config(a)["workload"], opts, units)
        roof["traffic"] = tr
        roof["traffic_basis"] = basis
        if tr:
            gbs = tr / (mean_stage[dom] * 1e-3) / 1e9
            roof["hbm_gbs"] = gbs
            roof["hbm_frac"] = gbs / hbm_peak
    exe_ms_step = 1e3 * exe_s / a.steps
    compulsory = 8 * (2 * a.n + 2 * a.m)   # c, sorted r and omega read; g written
    hbm = {"peak_gbs": hbm_peak, "peak_source": hbm_src,
           "execute_compulsory_bytes": compulsory,
           "execute_gbs": compulsory / (exe_ms_step * 1e-3) / 1e9,
           "execute_frac": compulsory / (exe_ms_step * 1e-3) / 1e9 / hbm_peak,
           "dominant_kernel": roof["kernel"] if roof else None,
           "dominant_kernel_gbs": roof.get("hbm_gbs") if roof else None,
           "dominant_kernel_frac": roof.get("hbm_frac") if roof else None,
           "basis": "execute: compulsory bytes (c, sorted r and omega, g) over the execute-only time; "
                    "dominant kernel: ncu DRAM bytes per launch over its live launch time"}

    extra_batched = extra_mixed = extra_grad = extra_stress = extra_order = extra_det = extra_pers = None
    extra_large = extra_multi = None
    if not a.no_extra and ws == 1:
        # the same workload at the other order of the scaled plain-NUHT
        # configuration (nu = 10), same options and timing as the main line
        o_nu = 10 if a.nu != 10 else 0
        for _ in range(2):
            with Plan(o_nu, dr, dw, a.eps, **opts) as pw:
                pw.execute(dc)
        o_ms = []
        for _ in range(a.steps):
            flush.zero_()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            po = Plan(o_nu, dr, dw, a.eps, **opts)
            po.execute(dc)
            s1.record(stream)
            torch.cuda.synchronize(dev)
            o_ms.append(s0.elapsed_time(s1))
            po.close()
        with Plan(o_nu, dr, dw, a.eps, **opts) as pw:
            oi = pw.info()
            g_o = pw.execute(dc).cpu().numpy()
        from paper_2411_09583_gb300.workloads import sample_rows
        extra_order = {"nu": o_nu, "ms_per_step": statistics.median(o_ms),
                       "error": sampled_error(o_nu, r, omega, c, g_o, a.eps, sample_rows(a.m, 200, seed=95)),
                       "value": (a.n + a.m) / (statistics.median(o_ms) * 1e-3), "unit": UNIT,
                       "step": "plan + execute, same workload and options as the main line",
                       "M": oi["M"], "L": oi["L"], "z": oi["z"]}
        # the same workload in the deterministic mode (bitwise reproducible:
        # exact fixed-point accumulation instead of FP64 atomics)
        for _ in range(2):
            with Plan(a.nu, dr, dw, a.eps, deterministic=True, **opts) as pdt:
                pdt.execute(dc)
        d_ms, d_ex = [], []
        for _ in range(max(3, a.steps // 2)):
            flush.zero_()
            s0, s1, s2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            s0.record(stream)
            pdt = Plan(a.nu, dr, dw, a.eps, deterministic=True, **opts)
            s1.record(stream)
            g_d = pdt.execute(dc)
            s2.record(stream)
            torch.cuda.synchronize(dev)
            d_ms.append(s0.elapsed_time(s2))
            d_ex.append(s1.elapsed_time(s2))
            g_d2 = pdt.execute(dc)
            same = bool(torch.equal(g_d.view(torch.int64), g_d2.view(torch.int64)))
            pdt.close()
        from paper_2411_09583_gb300.workloads import sample_rows
        extra_det = {"ms_per_step": statistics.median(d_ms), "execute_ms": statistics.median(d_ex),
                     "value": (a.n + a.m) / (statistics.median(d_ms) * 1e-3), "unit": UNIT,
                     "repeat_bitwise_equal": same,
                     "error": sampled_error(a.nu, r, omega, c, g_d.cpu().numpy(), a.eps,
                                            sample_rows(a.m, 200, seed=93)),
                     "step": "plan + execute with deterministic=1, same workload and options as the main line"}
        # the local blocks in one persistent launch (device work queue with
        # bounded per-block waits) against the two launches: execute time and
        # the local stage alone (every stage in order on one stream)
        pers = {}
        for flag in (False, True):
            with Plan(a.nu, dr, dw, a.eps, persistent=flag, **opts) as pp_:
                for _ in range(2):
                    pp_.execute(dc)
                ex = []
                for _ in range(a.steps):
                    flush.zero_()
                    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    s0.record(stream)
                    pp_.execute(dc)
                    s1.record(stream)
                    torch.cuda.synchronize(dev)
                    ex.append(s0.elapsed_time(s1))
                st_ok = pp_.status()
            loc_alone = []
            for _ in range(3):
                flush.zero_()
                with Plan(a.nu, dr, dw, a.eps, persistent=flag, timing="serial", **opts) as pt:
                    pt.execute(dc)
                    stt = pt.stage_times()
                loc_alone.append(stt["local_moments"] + stt["local_eval"])
            pers["persistent" if flag else "two_launches"] = {
                "execute_ms": statistics.median(ex), "local_stage_ms_alone": statistics.median(loc_alone),
                "status": st_ok}
        extra_pers = pers
        extra_batched = run_batched(dev, a.steps)
        extra_mixed = run_mixed(dev, a.steps)
        extra_grad = run_grad(dev, a.steps)
        extra_stress = run_stress(dev, a.steps)
        extra_large = run_large_grid(dev, a.steps)
        extra_multi = run_multi_vector(dev, a.steps)

    line = None
    if rank == 0:
        cpu = None
        rows = ref = None
        if ws == 1 and not a.no_cpu_baseline:
            v, nrows, dt, rows, ref = oracle_sample(a, r, omega, c, a.cpu_seconds)
            cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "oracle direct sum over all n points for %d random output rows "
                             "(%.1f s), extrapolated to m rows" % (nrows, dt)}
        if rows is None:
            from paper_2411_09583_gb300.workloads import sample_rows
            rows = sample_rows(a.m, 200, seed=94)
            import oracle
            ref = oracle.direct_rows(a.nu, r, omega, c, rows)
        error = sampled_error(a.nu, r, omega, c, g_main, a.eps, rows, ref)
        error["execute_only"] = sampled_error(a.nu, r, omega, c, g_exec, a.eps, rows, ref)["err_over_eps_c1"]
        error["e2e"] = sampled_error(a.nu, r, omega, c, g_e2e, a.eps, rows, ref)["err_over_eps_c1"]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": 1e3 * total_s / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE, "data": "synthetic (seeded uniform r, omega; Gaussian c)",
                "error": error,
                "config": workload_config(a),
                "plan_opts": opts or "library defaults",
                "autotune": tuned,
                "clocks": clocks,
                "e2e": {"value": e2e_value, "unit": UNIT,
                        "h2d_bytes_per_step": 8 * (a.n + a.m + a.n),
                        "d2h_bytes_per_step": 8 * a.m},
                "gpu_launches": launches,
                "roofline": roof,
                "hbm": hbm,
                "alu_peaks": alu,
                "cpu_baseline": cpu,
                "execute_only": {"value": ws * a.steps * (a.n + a.m) / exe_s, "unit": UNIT,
                                 "ms_per_step": 1e3 * exe_s / a.steps},
                "stage_ms": mean_stage,
                "stage_ms_basis": "CUDA events around each stage on the stream it runs on, inside the timed "
                                  "steps; the local and direct blocks run concurrently with the asymptotic "
                                  "pipeline (which has stream priority), so their stage times overlap and "
                                  "include waiting for SM resources",
                "stage_ms_alone": mean_serial,
                "batched": extra_batched,
                "mixed_precision": extra_mixed,
                "differentiation": extra_grad,
                "stress": extra_stress,
                "other_order": extra_order,
                "deterministic": extra_det,
                "persistent_local": extra_pers,
                "large_grid": extra_large,
                "multi_vector": extra_multi,
                "plan": {"M": info["M"], "L": info["L"], "z": info["z"], "w": info["nufft_width"],
                         "blocks_local_asy_direct": [info["n_local"], info["n_asy"], info["n_direct"]],
                         "direct_entries": info["direct_entries"],
                         "asy_rows_cols": info["asy_rows_cols"],
                         "local_rows_cols": info["local_rows_cols"]}}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return line


def main(argv=None):
    a = parse_args(argv)
    ws, rank, _ = dist_env()
    if a.impl == "reference":
        if rank != 0:
            return 0
        run_reference(a)
        return 0
    if a.only:
        import torch
        from paper_2411_09583_gb300 import build_native
        build_native.build()
        fn = {"large_grid": run_large_grid, "mixed": run_mixed, "multi_vector": run_multi_vector}[a.only]
        print(json.dumps(fn(torch.device("cuda", 0), a.steps)))
        return 0
    run_ours(a)
    return 0


if __name__ == "__main__":
    sys.exit(main())
