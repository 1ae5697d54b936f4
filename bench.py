"""Benchmark: robust value iteration throughput (transition-updates/s) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

A step is one full finite-horizon query (K = 200 Bellman iterations, maximum
pessimistic reachability, as in the paper's Sec. 5 experiments) over one batch
of synthetic IMDPs already resident in HBM.  The metric is
    transition-updates/s = (stored transitions) x (iterations) / time,
summed over all ranks.  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "transition-updates/s (robust Bellman, O-maximization), max-pessimistic finite reachability K=200"
UNIT = "transition-updates/s"
PAPER_PIMDP2_RATE = 48106480 * 200 / 30.0  # Sec. 5: pimdp_2, 200 steps, 30 s on a GTX1060


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(name: str, rank: int, models: int = 0):
    from workloads import make_config
    from workloads.imdp_synth import CONFIGS
    c = dict(CONFIGS[name])
    kw = dict(seed=c["seed"] + 1000 * rank)
    if models and c["kind"] == "batch":
        kw["n_models"] = models
    return make_config(name, **kw)


def workload_config(name: str, m, horizon: int):
    from workloads.imdp_synth import CONFIGS
    c = dict(CONFIGS[name])
    if m.model_state_offsets is not None:
        c["n_models"] = len(m.model_state_offsets) - 1
    cfg = {"workload": name, "states": int(m.n_states), "columns": int(m.n_cols), "transitions": int(m.nnz),
           "horizon": horizon, "query": "maximize pessimistic reachability, finite horizon",
           "models": int(c.get("n_models", 1)), "l2": "inputs larger than L2 (%.2f GB resident model)" %
           (m.nnz * 20 / 1e9), "parallelism": "replicas"}
    return cfg


def reduce_across_ranks(elapsed_ms: float, kernel_ms: float, units: float, world: int, device):
    """Whole-job timing: the slowest rank's times (max) and every rank's units (sum).
    Works on any process group (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return elapsed_ms, kernel_ms, units
    import torch
    mx = torch.tensor([elapsed_ms, kernel_ms], dtype=torch.float64, device=device)
    sm = torch.tensor([units], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return float(mx[0]), float(mx[1]), float(sm[0])


def algorithmic_bytes_per_iteration(m, storage: str = "f64", exact_entries: int = 0, fixed=None) -> int:
    """rowval + lower + gap per transition; colptr + rem (+ shift and the
    correction offset) per column; stateptr + V read + V write per state. On
    32-bit storage a correction column's transitions keep 4 + 16 bytes. States
    in ``fixed`` (the reach / avoid targets, whose values Eq. 2 fixes) are
    read and written by no launch and are left out."""
    nnz, ncols, nst = int(m.nnz), int(m.n_cols), int(m.n_states)
    if fixed is not None and len(fixed):
        f = np.unique(np.asarray(fixed, np.int64))
        cols = np.asarray(m.stateptr, np.int64)
        ent = np.asarray(m.colptr, np.int64)
        nnz -= int((ent[cols[f + 1]] - ent[cols[f]]).sum())
        ncols -= int((cols[f + 1] - cols[f]).sum())
        nst -= int(f.size)
    if storage == "f32":
        return (12 * (nnz - exact_entries) + 20 * exact_entries + (20 if exact_entries else 16) * ncols
                + 20 * nst)
    return 20 * nnz + 12 * ncols + 20 * nst


def bellman_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("bellman.cu", "imdp_internal.h"):
        with open(os.path.join(ROOT, "paper_2401_04068_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """Per-launch DRAM bytes of the Bellman kernel from a committed ncu summary,
    only if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "bellman_step_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    rec = d.get(workload)
    if not rec or rec.get("source_hash") != bellman_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def cpu_baseline(m, horizon: int, budget_s: float = 12.0, sample_models: int = None):
    """The oracle as it stands, on host cores, over a bounded sample of the workload."""
    import oracle
    from workloads import concat_block_diagonal  # noqa: F401
    cores = os.cpu_count() or 1
    offs = m.model_state_offsets if m.model_state_offsets is not None else np.array([0, m.n_states])
    n_models = len(offs) - 1

    def sub(nm):
        # first nm models of the block-diagonal batch (or a prefix of one model's iterations)
        s_end = int(offs[nm])
        c_end = int(m.stateptr[s_end])
        e_end = int(m.colptr[c_end])
        return oracle.OracleIMDP(s_end, m.stateptr[:s_end + 1], m.colptr[:c_end + 1], m.rowval[:e_end],
                                 m.lower[:e_end], m.upper[:e_end]), e_end

    if n_models > 1:
        # calibrate on a few models (enough to occupy every thread), then size the
        # sample to the budget
        nc = min(n_models, max(4 * cores, 16))
        omc, _ = sub(nc)
        goalc = m.goal[m.goal < offs[nc]]
        t = time.perf_counter()
        oracle.value_iteration(omc, oracle.OracleSpec(horizon=horizon, reach=goalc), threads=cores)
        dt = max(time.perf_counter() - t, 1e-4) / nc
        nm = sample_models or int(max(1, min(n_models, budget_s / dt)))
        om, nz = sub(nm)
        goal = m.goal[m.goal < offs[nm]]
        iters = horizon
        sample = f"first {nm} of {n_models} models, K={iters}"
    else:
        om, nz = sub(1)
        goal = m.goal
        t = time.perf_counter()
        oracle.value_iteration(om, oracle.OracleSpec(horizon=1, reach=goal), threads=cores)
        dt = max(time.perf_counter() - t, 1e-4)
        iters = int(max(1, min(horizon, budget_s / dt)))
        sample = f"whole model, K={iters} of {horizon} iterations (cost per iteration is constant)"
    t = time.perf_counter()
    st, V, k, _, _ = oracle.value_iteration(om, oracle.OracleSpec(horizon=iters, reach=goal), threads=cores)
    el = time.perf_counter() - t
    return {"value": nz * iters / el, "unit": UNIT, "cores": cores if oracle.has_openmp() else 1, "kind": "oracle",
            "sample": sample, "seconds": round(el, 3)}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on a bounded sample of the same workload."""
    if rank != 0:
        return
    m = make_workload(args.workload, 0, args.models)
    cfg = workload_config(args.workload, m, args.horizon)
    per = []
    base = None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(m, args.horizon, budget_s=args.ref_budget)
        if i >= args.warmup:
            per.append(r["value"])
            base = r
    value = float(statistics.median(per)) if per else 0.0
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
           "cpu_baseline": dict(base, value=value) if base else None,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2401_04068_gb300 as g
    from paper_2401_04068_gb300 import build as pbuild

    torch.cuda.set_device(local_rank)
    if not os.path.exists(pbuild.LIB) or not pbuild.up_to_date():
        if rank == 0 or world == 1:
            pbuild.build()
    if world > 1:
        torch.distributed.barrier()
    g.load()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)

    m = make_workload(args.workload, rank, args.models)
    dtype = g.IMDP_F32 if args.dtype == "f32" else g.IMDP_F64
    model = g.create_model(m, dtype=dtype, stream=stream, budget=f32_budget(args))
    if args.infinite:
        spec = g.make_spec(infinite_time=True, eps=args.eps, horizon=1000000, reach=m.goal, pessimistic=True,
                           maximize=True)
    else:
        spec = g.make_spec(horizon=args.horizon, reach=m.goal, pessimistic=True, maximize=True)
    sess = g.imdp_session_create([model], [spec], want_policy=[1] if args.policy else None, stream=stream)
    # tuned on the query's own iterations: early iterations (many threshold
    # searches) and late ones (warm starts) favour different kernels
    launch = apply_launch(g, sess, args, stream, min(args.horizon, 200) if not args.infinite else 64)

    def one_step(ev=None):
        g.imdp_session_reset(sess, stream)
        if ev is not None:
            ev[0].record(stream)
        if args.infinite:
            g.imdp_session_run(sess, 32, stream)  # to convergence (max |V_k - V_k-1| < eps)
        else:
            g.imdp_session_step(sess, args.horizon, stream)
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    # correctness guard on the timed configuration: the run must reach K
    kk = [0]
    Vd = torch.empty(m.n_states, dtype=torch.float64, device=dev)
    g.imdp_session_read(sess, 0, Vd, kk, stream=stream)
    iters = kk[0]
    assert iters == args.horizon or (args.infinite and iters > 0), iters

    launches0 = g.imdp_session_launches(sess)
    clocks = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start.record(stream)
    for i in range(args.steps):
        one_step(kev[i])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev)
    launches = g.imdp_session_launches(sess) - launches0
    my_units = float(m.nnz) * iters * args.steps
    elapsed_ms, kernel_ms, total_units = reduce_across_ranks(elapsed_ms, kernel_ms, my_units, world, dev)
    value = total_units / (elapsed_ms / 1e3)

    # e2e: through the public C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(m, k))).pin_memory()
               for k in ("stateptr", "colptr", "rowval", "lower", "upper")}
        Vh = torch.empty(m.n_states, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in pin.values())
        d2h = Vh.numel() * Vh.element_size()

        def e2e_step():
            mdl = g.imdp_create_csc(m.n_states, m.n_cols, m.nnz, pin["stateptr"], pin["colptr"], pin["rowval"],
                                    pin["lower"], pin["upper"], dtype=dtype, stream=stream)
            kk2 = [0]
            g.imdp_value_iteration(mdl, spec, Vh, kk2, stream=stream)
            mdl.close()
            return kk2[0]

        e2e_step()  # warm-up
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            assert e2e_step() == iters
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_s, _, _ = reduce_across_ranks(e2e_s, 0.0, 0.0, world, dev)
        e2e = {"value": float(m.nnz) * iters * args.e2e_steps * world / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps}

    if rank != 0:
        return
    peak, peak_kind = measured_peak_hbm()
    # correction entries of the fixed states are not read either; counting them is a slight overestimate
    alg_bytes = algorithmic_bytes_per_iteration(m, args.dtype, g.imdp_model_exact_columns(model)[1], fixed=m.goal)
    launch_ms = kernel_ms / max(1, launches)  # per launched iteration (includes any past convergence)
    n_tiles, n_wide, wide_entries = g.imdp_session_plan(sess)
    wide_share = wide_entries / max(1, m.nnz)
    kernel = "bellman_wide_kernel" if wide_share > 0.5 else KERNEL_NAMES.get(launch["kernel"], "bellman_step_kernel")
    achieved = alg_bytes / (launch_ms / 1e3) / 1e9
    traffic = recorded_traffic(args.workload + ("" if args.dtype == "f64" else ":f32"))
    cfg = workload_config(args.workload, m, args.horizon)
    metric = METRIC
    if args.infinite:
        metric = METRIC.replace("finite reachability K=200", "infinite-horizon reachability (to convergence)")
    if args.policy:
        metric += ", with the time-dependent policy"
    if args.infinite:
        cfg["horizon"] = f"infinite (eps {args.eps:g}); converged after {iters} iterations"
        cfg["query"] = "maximize pessimistic reachability, infinite horizon"
    if args.policy:
        cfg["policy"] = "time-dependent, K x n int32 written every iteration"
    cfg["storage"] = ("32-bit bounds (per-column scaled) and values, 32-bit arithmetic; correction columns exact"
                      if args.dtype == "f32" else "64-bit bounds (Q1.63), 64-bit arithmetic")
    cfg["launch"] = launch
    if args.dtype == "f32":
        n_exact, exact_entries, budget = g.imdp_model_exact_columns(model)
        cfg["error_bound_per_iteration"] = model.error_bound()  # guaranteed
        cfg["error_bound_horizon"] = model.error_bound() * iters
        cfg["correction_columns"] = {"columns": n_exact, "transitions": exact_entries,
                                     "share_of_transitions": exact_entries / max(1, m.nnz), "budget": budget}
    out = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak",
        # the paper's number is for its query only: pimdp_2, finite K = 200, no policy output
        "vs_baseline": (value / world / PAPER_PIMDP2_RATE)
        if (args.workload == "pimdp2" and args.horizon == 200 and not args.infinite and not args.policy) else None,
        "dtype": "u32" if args.dtype == "f32" else "u64", "data": "synthetic (seeded banded IMDPs shaped like the paper's benchmark table)",
        "config": cfg,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel,
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": launch_ms,
                     "plan": {"tiles": n_tiles, "wide_states": n_wide, "wide_entry_share": wide_share,
                              "launch": launch},
                     "timing": "CUDA events around each step's launches (both step kernels) / launches"},
        "clocks": clk,
        # step kernels (two per iteration when the model has wide states) + one value-reset kernel per step
        "gpu_launches": int(launches * (2 if n_wide > 0 else 1) + args.steps),
        "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(m, iters, budget_s=args.ref_budget)  # same per-iteration work
    print(json.dumps(out), flush=True)


TUNE_CACHE = os.path.join(ROOT, "paper_2401_04068_gb300", "tuned_gb300.json")


def f32_budget(args):
    """Per-iteration error budget of 32-bit storage (None: the library's default)."""
    return args.f32_budget if (args.dtype == "f32" and args.f32_budget > 0) else None


KERNEL_NAMES = {1: "bellman_step_kernel", 2: "bellman_direct_kernel", 3: "bellman_tiny_kernel",
                4: "bellman_slice_kernel"}


def parse_launch(text: str) -> dict:
    """'ring[:warps]', 'direct[:ctas_per_sm[:tile_entries[:wide_col]]]' or
    'slice[:ctas_per_sm]' -> launch fields."""
    parts = text.split(":")
    kind = {"ring": 1, "direct": 2, "slice": 4}[parts[0]]
    nums = [int(x) for x in parts[1:]]
    if kind == 1:
        keys = ["cta_warps", "tile_entries", "wide_col"]
    else:
        keys = ["ctas_per_sm", "tile_entries", "wide_col"]
    out = {"kernel": kind}
    out.update(dict(zip(keys, nums)))
    return out


def apply_launch(g, sess, args, stream, tune_iters: int) -> dict:
    """Launch configuration of the timed session: explicit (--launch), the
    autotuner's cached or freshly timed choice (--tune), or the rule."""
    if args.launch:
        g.imdp_session_set_launch(sess, stream=stream, **parse_launch(args.launch))
        how = "explicit"
    elif args.tune != "off":
        cache = args.tune_cache or TUNE_CACHE
        if args.tune == "fresh":
            cache = None
        _, ms = g.imdp_session_autotune(sess, tune_iters, cache, stream=stream)
        how = "autotuner (cached choice)" if ms == 0.0 else f"autotuner (timed now: {ms:.4f} ms per iteration)"
    else:
        how = "rule"
    out = g.imdp_session_get_launch(sess)
    out["chosen_by"] = how
    return out


def _gpu_setup(rank, world, local_rank):
    import torch
    import paper_2401_04068_gb300 as g
    from paper_2401_04068_gb300 import build as pbuild
    torch.cuda.set_device(local_rank)
    if not os.path.exists(pbuild.LIB) or not pbuild.up_to_date():
        if rank == 0 or world == 1:
            pbuild.build()
    if world > 1:
        torch.distributed.barrier()
    g.load()
    return torch.device("cuda", local_rank)


def run_polished(args, rank, world, local_rank):
    """Infinite horizon on 32-bit storage, polished on the 64-bit model
    (imdp_value_iteration_polished): one step = one whole query from V_0 to the
    64-bit stopping test; units = transitions x all iterations (both phases)."""
    import torch
    import paper_2401_04068_gb300 as g
    dev = _gpu_setup(rank, world, local_rank)
    stream = torch.cuda.Stream(device=dev)
    m = make_workload(args.workload, rank, args.models)
    m32 = g.create_model(m, dtype=g.IMDP_F32, stream=stream, budget=f32_budget(args))
    m64 = g.create_model(m, dtype=g.IMDP_F64, stream=stream)
    spec = g.make_spec(infinite_time=True, eps=args.eps, horizon=1000000, reach=m.goal, pessimistic=True,
                       maximize=True)
    launches = []
    for mdl in (m32, m64):  # the autotuner's configuration of each storage
        s_ = g.imdp_session_create([mdl], [spec], stream=stream)
        launches.append(apply_launch(g, s_, args, stream, 64))
        s_.close()
    Vd = torch.empty(m.n_states, dtype=torch.float64, device=dev)
    res = torch.empty(m.n_states, dtype=torch.float64, device=dev)

    def one_step():
        k = [0]
        st, k32 = g.imdp_value_iteration_polished(m32, m64, spec, Vd, k, res, stream=stream,
                                                  launch32=launches[0], launch64=launches[1])
        assert st == g.IMDP_OK
        return k32, k[0]

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    iters = []
    for _ in range(args.steps):
        iters.append(one_step())
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    my_units = float(m.nnz) * sum(k for _, k in iters)
    elapsed_ms, _, total_units = reduce_across_ranks(elapsed_ms, 0.0, my_units, world, dev)
    if rank != 0:
        return
    k32, k = iters[-1]
    cfg = workload_config(args.workload, m, args.horizon)
    cfg.update(horizon=f"infinite (eps {args.eps:g}); {k32} iterations on 32-bit storage, then {k - k32} "
                       f"on 64-bit (stopping test of the 64-bit path)",
               query="maximize pessimistic reachability, infinite horizon",
               storage="32-bit + correction to its fixed point, polished with 64-bit sweeps",
               launch={"f32": launches[0], "f64": launches[1]},
               error_bound_per_iteration_f32=m32.error_bound())
    out = {
        "metric": METRIC.replace("finite reachability K=200", "infinite-horizon reachability (to convergence)"),
        "value": total_units / (elapsed_ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32+u64",
        "data": "synthetic (seeded banded IMDPs shaped like the paper's benchmark table)", "config": cfg,
        "roofline": None, "clocks": clk, "e2e": None,
        "note": "each step creates its two sessions (imdp_value_iteration_polished), inside the timed region",
    }
    print(json.dumps(out), flush=True)


def run_uneven(args, rank, world, local_rank):
    """Heterogeneous batch: 10,000 problems of different shapes and horizons in one
    resident session; a step runs every problem to its own horizon."""
    import torch
    import paper_2401_04068_gb300 as g
    from workloads.imdp_synth import uneven_batch
    dev = _gpu_setup(rank, world, local_rank)
    stream = torch.cuda.Stream(device=dev)
    n = args.models or 10000
    t = time.perf_counter()
    ms, Ks = uneven_batch(n, seed=7 + 1000 * rank, threads=os.cpu_count() or 1)
    gen_s = time.perf_counter() - t
    dtype = g.IMDP_F32 if args.dtype == "f32" else g.IMDP_F64
    models = [g.create_model(m, dtype=dtype, stream=stream, budget=f32_budget(args)) for m in ms]
    specs = [g.make_spec(horizon=int(K), reach=m.goal, pessimistic=True, maximize=True) for m, K in zip(ms, Ks)]
    sess = g.imdp_session_create(models, specs, stream=stream)
    kmax = int(Ks.max())
    # tuned on 200 iterations: the batch runs to horizons of 50..500, and its
    # first iterations (threshold searches) favour other kernels than the rest
    launch = apply_launch(g, sess, args, stream, 200)

    def one_step(ev=None):
        g.imdp_session_reset(sess, stream)
        if ev is not None:
            ev[0].record(stream)
        g.imdp_session_step(sess, kmax, stream)
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    for i in (0, n // 2, n - 1):  # every problem stops at its own horizon
        kk = [0]
        Vd = torch.empty(ms[i].n_states, dtype=torch.float64, device=dev)
        g.imdp_session_read(sess, i, Vd, kk, stream=stream)
        assert kk[0] == int(Ks[i]), (i, kk[0], int(Ks[i]))
    launches0 = g.imdp_session_launches(sess)
    clocks = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0.record(stream)
    for i in range(args.steps):
        one_step(kev[i])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev)
    launches = g.imdp_session_launches(sess) - launches0
    nnz = np.array([m.nnz for m in ms], np.float64)
    my_units = float((nnz * Ks).sum()) * args.steps
    elapsed_ms, kernel_ms, total_units = reduce_across_ranks(elapsed_ms, kernel_ms, my_units, world, dev)
    if rank != 0:
        return
    peak, peak_kind = measured_peak_hbm()
    alg = sum(algorithmic_bytes_per_iteration(m, args.dtype, g.imdp_model_exact_columns(x)[1], fixed=m.goal)
              * int(K) for m, x, K in zip(ms, models, Ks))
    achieved = alg * args.steps / (kernel_ms / 1e3) / 1e9
    out = {
        "metric": METRIC.replace("K=200", "K per problem"), "value": total_units / (elapsed_ms / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32" if args.dtype == "f32" else "u64",
        "data": "synthetic (seeded banded IMDPs, per-problem shapes and horizons)",
        "config": {"workload": f"uneven_x{n}", "problems": n, "transitions": int(nnz.sum()),
                   "states": int(sum(m.n_states for m in ms)), "horizon": "U{50..500} per problem",
                   "max_horizon": kmax, "shapes": "states U{6..961}, actions U{1..4}, window U{2..min(400,n)}",
                   "l2": "inputs larger than L2 (%.1f GB resident)" % (nnz.sum() * 20 / 1e9),
                   "generation_s": round(gen_s, 1), "parallelism": "replicas", "launch": launch},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_kind": peak_kind,
                     "kernel": KERNEL_NAMES.get(launch["kernel"], "bellman_step_kernel"),
                     "note": "algorithmic bytes of every running problem summed over the step's launches"},
        "clocks": clk, "gpu_launches": int(launches + args.steps), "e2e": None,
    }
    print(json.dumps(out), flush=True)


def run_latency(args, rank, world, local_rank):
    """Single small model (the Sec. 3.1 worked example, K = 100, or the linear_5
    shape, K = 200): latency of one query. Three views: the public call
    imdp_value_iteration with a host output buffer (session set-up, launches and
    read-back inside), a resident session (reset + K launches + read to the host),
    and the device time of the K launches alone (CUDA events)."""
    import torch
    import paper_2401_04068_gb300 as g
    from workloads import make_config
    dev = _gpu_setup(rank, world, local_rank)
    stream = torch.cuda.Stream(device=dev)
    if args.workload == "worked_example":
        # the Sec. 3.1 model as the paper states it: dense interval matrices per
        # source state (rows = destinations, columns = actions), through the
        # dense creation call
        ex = json.load(open(os.path.join(ROOT, "tests", "golden", "worked_example.json")))
        n = ex["n_states"]
        n_actions = np.array([len(a) for a in ex["actions"]], np.int32)
        lo = np.array([col for s in range(n) for col in ex["lower"][s]], np.float64).T.copy(order="F")
        up = np.array([col for s in range(n) for col in ex["upper"][s]], np.float64).T.copy(order="F")
        model = g.imdp_create_dense(n, n_actions, lo.ravel(order="F"), up.ravel(order="F"), stream=stream)
        info = model.info()
        n_states, ncols, nnz = info["n_states"], info["n_cols"], info["nnz"]
        goal = np.array([x - 1 for x in ex["goal_1based"]], np.int32)
        K = ex["horizon"]
    else:
        m = make_config("linear5")
        K = 200
        n_states, ncols, nnz, goal = m.n_states, len(m.colptr) - 1, len(m.rowval), m.goal
        model = g.create_model(m, stream=stream)

    class _M:  # what the rest of the function reads
        pass
    m = _M()
    m.n_states, m.goal = n_states, goal
    spec = g.make_spec(horizon=K, reach=m.goal)
    Vh = torch.empty(m.n_states, dtype=torch.float64).pin_memory()
    kk = [0]
    n = max(args.steps, 20)

    def timed(fn, reps):
        out = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            out.append((time.perf_counter() - t) * 1e3)
        return out

    for _ in range(max(args.warmup, 3)):
        g.imdp_value_iteration(model, spec, Vh, kk, stream=stream)
    e2e = timed(lambda: g.imdp_value_iteration(model, spec, Vh, kk, stream=stream), n)
    assert kk[0] == K
    sess = g.imdp_session_create([model], [spec], stream=stream)

    def resident():
        g.imdp_session_reset(sess, stream)
        g.imdp_session_step(sess, K, stream)
        g.imdp_session_read(sess, 0, Vh, kk, stream=stream)

    for _ in range(3):
        resident()
    res = timed(resident, n)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    clocks = ClockSampler(local_rank)
    clocks.start()
    for a, b in ev:
        g.imdp_session_reset(sess, stream)
        a.record(stream)
        g.imdp_session_step(sess, K, stream)
        b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    dev_ms = [a.elapsed_time(b) for a, b in ev]
    pct = lambda xs, q: float(np.percentile(np.asarray(xs), q))
    if rank != 0:
        return
    out = {
        "metric": "query latency, one small model (K Bellman iterations per query)", "value": pct(e2e, 50),
        "unit": "ms per query", "n_gpus": world, "steps": n, "warmup": max(args.warmup, 3),
        "ms_per_step": pct(e2e, 50), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32" if args.dtype == "f32" else "u64", "data": "the paper's worked example (Sec. 3.1)" if args.workload == "worked_example"
        else "synthetic (seeded banded IMDP shaped like linear_5_states)",
        "config": {"workload": args.workload, "states": int(m.n_states), "columns": ncols, "transitions": nnz,
                   "horizon": K, "query": "maximize pessimistic reachability, finite horizon",
                   "parallelism": "replicas", "l2": "model resident in L2 (a few hundred bytes)"},
        "latency_ms": {
            "value_iteration_call": {"p50": pct(e2e, 50), "p99": pct(e2e, 99)},
            "resident_session_reset_step_read": {"p50": pct(res, 50), "p99": pct(res, 99)},
            "device_K_launches": {"p50": pct(dev_ms, 50), "p99": pct(dev_ms, 99),
                                  "us_per_iteration": pct(dev_ms, 50) * 1e3 / K},
        },
        "transition_updates_per_s": nnz * K / (pct(e2e, 50) / 1e3),
        "clocks": clk, "gpu_launches": int(K * n), "roofline": None,
        "e2e": {"value": pct(e2e, 50), "unit": "ms per query", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(m.n_states * 8)},
    }
    print(json.dumps(out), flush=True)


def run_served(args, rank, world, local_rank):
    """Continuous-batching server under a Poisson request stream: requests arrive at
    `--rate` per second; 70 % bring a new model (created on arrival, inside the
    measured latency), 30 % re-query a resident one. Arrivals are handled by a
    pool of `--client-threads` frontend threads (model creation + submit), each
    on its own stream. Latency = arrival to result."""
    import queue as _queue
    from concurrent.futures import Future, ThreadPoolExecutor
    import torch
    import paper_2401_04068_gb300 as g
    from workloads.imdp_synth import served_stream
    dev = _gpu_setup(rank, world, local_rank)
    stream = torch.cuda.Stream(device=dev)
    n_req = args.requests
    models_h, reqs = served_stream(n_req, seed=8 + 1000 * rank, threads=os.cpu_count() or 1)
    server = g.imdp_server_create(int(args.server_budget_gb * (1 << 30)))
    launch = {"kernel": 0, "chosen_by": "rule"}
    if args.launch:
        launch = parse_launch(args.launch)
        g.imdp_server_set_launch(server, **launch)
        launch["chosen_by"] = "explicit"
    # warm-up: one request through the whole path (module load, first graph)
    dtype = g.IMDP_F32 if args.dtype == "f32" else g.IMDP_F64
    w = g.create_model(models_h[0], dtype=dtype, stream=stream, budget=f32_budget(args))
    tk = g.imdp_server_submit(server, w, g.make_spec(horizon=10, reach=models_h[0].goal))
    assert g.imdp_server_wait(server, tk, 60000.0, np.zeros(models_h[0].n_states)) == g.IMDP_OK
    rng = np.random.default_rng(99 + rank)
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, n_req))
    dev_models = [None] * len(models_h)
    done = [None] * n_req
    q = _queue.Queue()

    def waiter():
        while True:
            item = q.get()
            if item is None:
                return
            i, tk, t_sub, n = item
            V = np.zeros(n)
            k = [0]
            lat = [0.0]
            st = g.imdp_server_wait(server, tk, 600000.0, V, k, lat)
            done[i] = (st, k[0], t_sub + lat[0] / 1e3)

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    create_s = []
    lag_s = []
    lock = threading.Lock()
    local = threading.local()
    # high priority: a new model's conversion kernel runs before the server's queued launches
    streams = [torch.cuda.Stream(device=dev, priority=-1) for _ in range(args.client_threads)]
    next_stream = [0]

    def model_for(mi):
        # the first request of a model creates it; later ones wait for that
        with lock:
            f = dev_models[mi]
            mine = f is None
            if mine:
                f = dev_models[mi] = Future()
        if mine:
            tc = time.perf_counter()
            f.set_result(g.create_model(models_h[mi], dtype=dtype, stream=local.stream, budget=f32_budget(args)))
            create_s.append(time.perf_counter() - tc)
        return f.result()

    def handle(i):
        if not hasattr(local, "stream"):
            torch.cuda.set_device(dev)
            with lock:
                local.stream = streams[next_stream[0] % len(streams)]
                next_stream[0] += 1
        mi, K, pess, goal = reqs[i]
        model = model_for(mi)
        spec = g.make_spec(horizon=K, reach=goal, pessimistic=pess)
        t_sub = time.perf_counter()
        q.put((i, g.imdp_server_submit(server, model, spec), t_sub, models_h[mi].n_states))

    pool = ThreadPoolExecutor(max_workers=args.client_threads)
    clocks = ClockSampler(local_rank)
    clocks.start()
    t0 = time.perf_counter()
    futs = []
    for i in range(n_req):
        delay = t0 + arrivals[i] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        else:
            lag_s.append(-delay)
        futs.append(pool.submit(handle, i))
    for f in futs:
        f.result()
    pool.shutdown()
    q.put(None)
    th.join()
    clk = clocks.stop()
    lat = np.array([(d[2] - (t0 + a)) * 1e3 for d, a in zip(done, arrivals)])
    ok = all(d[0] == g.IMDP_OK and d[1] == r[1] for d, r in zip(done, reqs))
    span = max(d[2] for d in done) - t0
    units = float(sum(models_h[r[0]].nnz * r[1] for r in reqs))
    stats = g.imdp_server_stats(server)
    server.close()
    if rank != 0:
        return
    out = {
        "metric": "served robust value iteration: transition-updates/s and arrival-to-result latency",
        "value": units / span, "unit": UNIT, "n_gpus": world, "steps": n_req, "warmup": 1,
        "ms_per_step": span * 1e3 / n_req, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32" if args.dtype == "f32" else "u64", "data": "synthetic (seeded banded IMDPs, log-uniform shapes)",
        "config": {"workload": f"served_poisson{int(args.rate)}", "requests": n_req, "rate_per_s": args.rate,
                   "launch": launch,
                   "storage": ("32-bit + correction, per-iteration budget %g (guaranteed %g at K = 500)"
                               % (args.f32_budget or 5e-9, 500 * (args.f32_budget or 5e-9)))
                   if args.dtype == "f32" else "64-bit",
                   "new_models": len(models_h), "client_threads": args.client_threads,
                   "shapes": "states log-U[50,4000], actions U{1..3}, "
                   "window log-U[3,700], K U{100..500}", "server_budget_gb": args.server_budget_gb,
                   "all_ok": bool(ok)},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                       "p99": float(np.percentile(lat, 99)), "mean": float(lat.mean()), "max": float(lat.max())},
        # the stream's own rate: work of all requests over the span of their arrivals
        "offered_updates_per_s": units / float(arrivals[-1]),
        # the worker's time: device time of the launches against its wall time (the rest is
        # read-back, retirement, admission and table uploads between chunks)
        "server": dict(stats, device_busy=stats["device_ms"] / max(1e-9, stats["wall_ms"])),
        "client": {"model_create_ms_mean": 1e3 * float(np.mean(create_s)) if create_s else 0.0,
                   "model_create_s_total": float(np.sum(create_s)),
                   "submits_behind_schedule": len(lag_s),
                   "max_lag_ms": 1e3 * float(max(lag_s)) if lag_s else 0.0},
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)


def run_state_sharded(args, rank, world, local_rank):
    """One model (default: the pimdp_2 shape) split by states over the ranks; every
    rank iterates its slice and the ranks all-gather the iterates after each step
    (strong scaling: the total work is fixed)."""
    import torch
    import paper_2401_04068_gb300 as g
    from paper_2401_04068_gb300.sharded import SliceRunner, gather_slices
    dev = _gpu_setup(rank, world, local_rank)
    m = make_workload(args.workload, 0, args.models)  # the same model on every rank
    dtype = g.IMDP_F32 if args.dtype == "f32" else g.IMDP_F64
    bounds = g.imdp_partition_states(m.n_states, m.stateptr, m.colptr, world)
    lengths = np.diff(bounds)
    runner = SliceRunner(m, bounds, rank, dict(horizon=args.horizon, reach=m.goal), dtype)
    # each slice's session takes the autotuner's configuration for its own shape
    launch = apply_launch(g, runner.session, args, None, min(args.horizon, 200))

    def one_step():
        runner.reset()
        for _ in range(args.horizon):
            own = runner.step()
            if world > 1:
                runner.put(gather_slices(own, lengths, rank))

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        one_step()
    t1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    V = np.zeros(m.n_states)
    k = [0]
    runner.read(V, k)
    assert k[0] == args.horizon
    units = float(m.nnz) * args.horizon * args.steps  # the whole model, once
    elapsed_ms, _, _ = reduce_across_ranks(elapsed_ms, 0.0, 0.0, world, dev)
    if rank != 0:
        return
    cfg = workload_config(args.workload, m, args.horizon)
    cfg.update(parallelism=f"state-sharded x{world}", partition=[int(x) for x in bounds], launch=launch)
    out = {
        "metric": METRIC, "value": units / (elapsed_ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u32" if args.dtype == "f32" else "u64",
        "data": "synthetic (seeded banded IMDP shaped like the paper's benchmark table)", "config": cfg,
        "clocks": clk, "exchange_bytes_per_step": int(8 * m.n_states * args.horizon) if world > 1 else 0,
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pendulum240_x4096")
    ap.add_argument("--horizon", type=int, default=200)
    ap.add_argument("--models", type=int, default=0, help="override the number of models of a batch workload")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"], help="storage of the transition bounds")
    ap.add_argument("--f32-budget", type=float, default=0.0,
                    help="32-bit storage: per-iteration error budget of the correction stage (0: library default)")
    ap.add_argument("--launch", default="", help="explicit launch configuration, e.g. ring:24, direct:4:1024 or slice:4")
    ap.add_argument("--tune", default="cache", choices=["cache", "fresh", "off"],
                    help="autotuner: cached choice (timing only shapes missing from the cache), time now, or rule")
    ap.add_argument("--tune-cache", default="", help="autotuner cache file (default: the package's GB300 table)")
    ap.add_argument("--requests", type=int, default=2000, help="served workload: number of requests")
    ap.add_argument("--rate", type=float, default=2000.0, help="served workload: Poisson arrival rate per second")
    ap.add_argument("--server-budget-gb", type=float, default=16.0, help="served workload: HBM budget of the server")
    ap.add_argument("--client-threads", type=int, default=4, help="served workload: frontend threads")
    ap.add_argument("--policy", action="store_true", help="also synthesize the time-dependent policy (K x n)")
    ap.add_argument("--infinite", action="store_true", help="infinite horizon: iterate until max |dV| < eps")
    ap.add_argument("--polish", action="store_true",
                    help="with --infinite: 32-bit storage to its fixed point, then 64-bit sweeps")
    ap.add_argument("--eps", type=float, default=1e-6, help="convergence tolerance of --infinite")
    ap.add_argument("--shard", default="problems", choices=["problems", "states"],
                    help="multi-GPU split: independent problems per rank (default) or one model's states")
    args = ap.parse_args()
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        if args.workload.startswith("uneven"):
            run_uneven(args, rank, world, local_rank)
        elif args.workload in ("worked_example", "linear5"):
            run_latency(args, rank, world, local_rank)
        elif args.workload.startswith("served"):
            run_served(args, rank, world, local_rank)
        elif args.shard == "states":
            run_state_sharded(args, rank, world, local_rank)
        elif args.polish:
            run_polished(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
