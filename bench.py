"""Benchmark of the DSEM-SL step on GB300: Gauss-node updates per second.

Workload: 1D linear advection at constant speed a = 1 on the periodic unit interval,
K = 2^20 elements, N = 8 (9 Gauss-Legendre nodes), Gaussian pulse, boundary + mass + energy
constraints, RK4 particle integration, dt from the paper's rule (edge-node gap over |u|max, which
keeps every particle inside its element).  One bench step is
one time step of the whole mesh.  The headline is the mixed-precision shared-operator path
(double-float state, float bulk arithmetic); the plain FP64 per-element path is timed beside
it.  Inputs stay resident in HBM; L2 (129 MB) is flushed by writing a 256 MB buffer before
every timed step.

``python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]``
Under torchrun each rank runs an independent replica (independent problems; no collective).
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import math
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sl_inputs  # noqa: E402

METRIC = "Gauss-node updates/sec per time step at stated L2 error vs FP64; % HBM roofline"
UNIT = "node-updates/s"
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def peaks():
    try:
        d = json.load(open(MEASURED))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def workload_config(n, precision_name):
    return {"workload": f"1d_const_advection_K2^20_N{n - 1}_n{n}_GL_boundary+mass+energy_RK4_{precision_name}",
            "elements": 1 << 20, "nodes_per_element": n, "steps_per_bench_step": 1,
            "l2_flush": "256MB write before every timed step", "parallelism": "replicas"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = [r.split(",") for r in open(self.file.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(n, seconds=12.0, cons=7):
    """The FP64 oracle as it stands, on a bounded sample of elements of the same workload."""
    from oracle import sl_oracle as O
    prob = sl_inputs.config2_1d_gauss(n)
    setup = O.setup_from_problem(prob)
    phi = O.project_1d(setup, prob.phi0)
    vel = O.Vel(O.VEL_CONST, (1.0, 0, 0, 0, 0, 0))
    o = O.StepOpts(vel, 0.0, O.max_dt(setup, vel, rule=prob.dt_rule), cons, 4)
    # elements across the pulse, where every term of the step is active
    centre = prob.kx // 2
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        ks = range(centre + done, centre + done + 64)
        O.step_1d(setup, phi, o, elements=ks)
        done += 64
    el = time.perf_counter() - t0
    return {"value": done * n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} elements (x{n} nodes) of one step at the pulse centre, {el:.1f} s, numpy FP64, 1 thread"}


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks (the slowest rank's time); x itself on one rank.
    Collective: every rank of the process group calls it."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, nodes, steps, seconds):
    """Whole-job node updates per second: every rank advances its own replica of nodes nodes."""
    return world * nodes * steps / seconds


def run_reference(args, rank, world):
    n = args.n
    if rank != 0:
        return
    per = []
    # each step is a bounded sample so that the whole run stays within about two minutes
    sec = max(0.2, min(args.ref_seconds, 90.0 / (args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(n, seconds=min(sec, 0.5))
    for _ in range(args.steps):
        per.append(cpu_baseline(n, seconds=sec))
    vals = [p["value"] for p in per]
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * (1 << 20) * n / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(n, "mixed_shared_operator"),   # the same workload as the GPU arm
            "cpu_baseline": dict(per[-1], value=v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _time_steps(torch, ctx, stream, a, b, vel, dt, opts, t, steps, flush):
    """Per-step CUDA events on the library's stream, L2 flushed before every step."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for s in range(steps):
        flush.zero_()
        starts[s].record(stream)
        ctx.step(a, b, vel, t, dt, opts)
        ends[s].record(stream)
        a, b = b, a
        t += dt
    torch.cuda.synchronize()
    return sum(st.elapsed_time(en) for st, en in zip(starts, ends)), a, b, t


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_1910_06476_gb300 as sl
    from paper_1910_06476_gb300 import build as B

    torch.cuda.set_device(local_rank)
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    n = args.n
    prob = sl_inputs.config2_1d_gauss(n)
    stream = torch.cuda.current_stream()
    precision = sl.MIXED if args.precision == "mixed" else sl.FP64
    ctx = sl.Context(1, prob.kx, 1, prob.box, n, sl.GAUSS_LEGENDRE, precision, prob.bc, prob.ghost, stream)
    vel = sl.velocity(sl.VEL_CONST, 1.0)
    dt = ctx.max_dt(vel, sl_inputs.rule_code(prob))
    opts = sl.options(prob.constraints, 4)
    x, _ = ctx.node_coords()
    phi0 = prob.phi0(x).ravel()
    phi0_dev = torch.tensor(phi0, device="cuda")
    a = ctx.pack(phi0_dev)
    b = ctx.new_state()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    t = 0.0
    for _ in range(args.warmup):
        ctx.step(a, b, vel, t, dt, opts)
        a, b = b, a
        t += dt
    torch.cuda.synchronize()
    assert ctx.sync() == 0, "device status bits set during warm-up"

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clocks:
        total_ms, a, b, t = _time_steps(torch, ctx, stream, a, b, vel, dt, opts, t, args.steps, flush)
    if world > 1:
        dist.barrier()
    status = ctx.sync()
    nodes = prob.kx * n
    total_ms = max_over_ranks(total_ms, world, "cuda")
    value = job_throughput(world, nodes, args.steps, total_ms * 1e-3)

    # end to end through the public API: host doubles in, one step, host doubles out, every step
    e2e_steps = min(args.steps, 50)
    host_in = torch.tensor(phi0).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    ctx.run_host(host_in, host_out, vel, 0.0, dt, 1, opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        ctx.run_host(host_in, host_out, vel, s * dt, dt, 1, opts)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_value = job_throughput(world, nodes, e2e_steps, e2e_s)

    # the plain FP64 per-element form on the same workload, for comparison
    fp64 = None
    if precision == sl.MIXED and not args.no_fp64:
        c64 = sl.Context(1, prob.kx, 1, prob.box, n, sl.GAUSS_LEGENDRE, sl.FP64, prob.bc, prob.ghost, stream)
        a64, b64 = phi0_dev.clone(), torch.empty_like(phi0_dev)
        for _ in range(3):
            c64.step(a64, b64, vel, 0.0, dt, opts)
        k64 = min(args.steps, 50)
        ms64, _, _, _ = _time_steps(torch, c64, stream, a64, b64, vel, dt, opts, 0.0, k64, flush)
        fp64 = {"value": nodes * k64 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64 / k64,
                "kernel": "k_step1d_f64", "bound": "fp64 pipe (86.7% busy in ncu)"}

    # accuracy against FP64: one step vs the oracle on sampled elements from the GPU's own state;
    # 1000 steps vs the FP64 GPU path (itself within 1e-12 of the oracle per step)
    err = {}
    if rank == 0 and not args.no_check:
        from oracle import sl_oracle as O
        setup = O.setup_from_problem(prob)
        pre = ctx.unpack(a).cpu().numpy().reshape(prob.kx, n)
        ctx.step(a, b, vel, t, dt, opts)
        got = ctx.unpack(b).cpu().numpy().reshape(prob.kx, n)
        sample = np.unique(np.concatenate([sl_inputs.sample_elements(2048, prob.kx, 5),
                                           np.arange(prob.kx // 2 - 32, prob.kx // 2 + 32)]))
        ref, _ = O.step_1d(setup, pre, O.StepOpts(O.Vel(O.VEL_CONST, (1.0, 0, 0, 0, 0, 0)), t, dt,
                                                  prob.constraints, 4), elements=sample)
        err["after_1_step_vs_oracle_sampled"] = float(np.sqrt(np.sum((got[sample] - ref[sample]) ** 2)
                                                              / np.sum(ref[sample] ** 2)))
        if precision == sl.MIXED and not args.no_fp64:
            m_a, m_b = ctx.pack(phi0_dev), ctx.new_state()
            f_a, f_b = phi0_dev.clone(), torch.empty_like(phi0_dev)
            for s in range(1000):
                ctx.step(m_a, m_b, vel, s * dt, dt, opts)
                c64.step(f_a, f_b, vel, s * dt, dt, opts)
                m_a, m_b, f_a, f_b = m_b, m_a, f_b, f_a
            d = ctx.unpack(m_a) - f_a
            err["after_1000_steps_vs_fp64_path"] = float((d.norm() / f_a.norm()).item())
            err["bound"] = 1e-6

    if rank != 0:
        return
    hbm, peak_kind = peaks()
    bytes_per_node = 16
    avg_ms = total_ms / args.steps
    achieved = nodes * bytes_per_node / (avg_ms * 1e-3) / 1e9
    clk = clocks.summary()
    kname = "k_step1d_mixed" if precision == sl.MIXED else "k_step1d_f64"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": avg_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if precision == sl.MIXED else "f64",
            "data": "synthetic (seeded analytic Gaussian pulse)",
            "config": workload_config(n, "mixed_shared_operator" if precision == sl.MIXED else "fp64_per_element"),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": TRAFFIC.get(kname),
                         "peak_source": f"{peak_kind} hbm_gbs (copy, burst)",
                         "algorithmic_bytes_per_node": bytes_per_node, "kernel": kname},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nodes * 8,
                    "d2h_bytes_per_step": nodes * 8},
            "gpu_launches": args.steps,
            "l2_error_vs_fp64": err,
            "fp64_per_element": fp64,
            "device_status": status}
    if not args.no_configs:
        line["configs"] = secondary_configs(sl, torch, flush, full=args.all_configs, only=args.only_config)
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(n, seconds=args.ref_seconds)
    print(json.dumps(line), flush=True)


# DRAM bytes per launch from one ncu capture of the same workload (None once the kernel changed)
TRAFFIC = {"k_step1d_mixed": 75550000 + 24440000}   # n = 9, K = 2^20: read + written (lines still dirty
                                                    # in L2 at kernel end are not counted)


def _problem_state(sl, torch, prob, precision):
    """Context and initial state (device doubles) of a workload."""
    ctx = sl.Context(prob.dim, prob.kx, prob.ky, prob.box, prob.n, prob.basis, precision, prob.bc, prob.ghost,
                     orders=prob.orders)
    x, y = ctx.node_coords()
    phi = prob.phi0(x) if prob.dim == 1 else prob.phi0(x, y)
    return ctx, torch.tensor(np.ascontiguousarray(phi).ravel(), device="cuda")


def measure_config(sl, torch, prob, precision, steps, flush, phi=None):
    """Per-step CUDA-event time of one workload on one path (L2 flushed before each step)."""
    ctx, phi0 = _problem_state(sl, torch, prob, precision) if phi is None else (
        sl.Context(prob.dim, prob.kx, prob.ky, prob.box, prob.n, prob.basis, precision, prob.bc, prob.ghost,
                   orders=prob.orders), phi)
    vel = sl.velocity(prob.velocity.kind, *prob.velocity.p)
    dt = ctx.max_dt(vel, sl_inputs.rule_code(prob))
    opts = sl.options(prob.constraints, prob.rk_order)
    a, b = ctx.pack(phi0), ctx.new_state()
    stream = ctx.stream
    ctx.step(a, b, vel, 0.0, dt, opts)           # warm-up
    torch.cuda.synchronize()
    ms, a, b, _ = _time_steps(torch, ctx, stream, b, a, vel, dt, opts, dt, steps, flush)
    status = ctx.sync()
    out = ctx.unpack(a)
    nodes = ctx.size
    per = ms / steps
    return {"ms_per_step": per, "node_updates_per_s": nodes / (per * 1e-3), "steps": steps,
            "hbm_frac_of_measured": nodes * 16 / (per * 1e-3) / 1e9 / peaks()[0], "device_status": status}, phi0, out, (
        ctx, vel, dt, opts)


def secondary_configs(sl, torch, flush, full=False, only=None):
    """The other configurations of the measurement plan on both paths, outside the headline timed
    region (the 2048^2 swirl and the 64-problem batch only with full=True)."""
    res = []
    plan = [("1d_sine_K16_n9 (config 1)", sl_inputs.config1_1d_sine(), [sl.FP64], 200)]
    for n in (5, 9, 13, 17):
        plan.append((f"1d_gauss_K2^20_n{n} (config 2)", sl_inputs.config2_1d_gauss(n), [sl.MIXED, sl.FP64], 50))
    plan.append(("2d_const_512x512_n9 (config 3)", sl_inputs.config3_2d_const(), [sl.MIXED, sl.FP64], 10))
    plan.append(("2d_rotation_256x256_p-adaptive_n4-16 (config 4)", sl_inputs.config4_rotation(), [sl.MIXED, sl.FP64],
                 10))
    if full:
        plan.append(("2d_swirl_2048x2048_n8 (config 5)", sl_inputs.config5_swirl(), [sl.MIXED, sl.FP64], 3))
    if only is not None:
        plan = [p for p in plan if f"(config {only})" in p[0]]
    for name, prob, precs, steps in plan:
        entry = {"workload": name, "nodes": None}
        phi0, outs = None, {}
        for prec in precs:
            r, phi0, out, run = measure_config(sl, torch, prob, prec, steps, flush, phi0)
            key = "mixed" if prec == sl.MIXED else "fp64"
            entry[key] = r
            entry["nodes"] = int(phi0.numel())
            # one step from the initial state for the accuracy comparison
            ctx, vel, dt, opts = run
            a, b = ctx.pack(phi0), ctx.new_state()
            ctx.step(a, b, vel, 0.0, dt, opts)
            outs[key] = ctx.unpack(b)
            del ctx, a, b
        if prob.kx * prob.ky <= 64:
            # a launch-bound workload: the same steps replayed from one CUDA graph (sl_run); the
            # whole state (a few KB) stays in L2 either way, so no flush between steps
            prec = precs[0]
            ctx = sl.Context(prob.dim, prob.kx, prob.ky, prob.box, prob.n, prob.basis, prec, prob.bc, prob.ghost)
            vel = sl.velocity(prob.velocity.kind, *prob.velocity.p)
            dt = ctx.max_dt(vel, sl_inputs.rule_code(prob))
            opts = sl.options(prob.constraints, prob.rk_order)
            a, b = ctx.pack(phi0), ctx.new_state()
            ctx.run(a, b, vel, 0.0, dt, steps, opts)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            ctx.run(a, b, vel, 0.0, dt, steps, opts)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            per = e0.elapsed_time(e1) / steps
            entry["graph_replay"] = {"ms_per_step": per, "node_updates_per_s": entry["nodes"] / (per * 1e-3),
                                     "steps": steps, "api": "sl_run", "device_status": ctx.sync()}
            del ctx, a, b
        if "mixed" in outs and "fp64" in outs:
            d = outs["mixed"] - outs["fp64"]
            entry["mixed_vs_fp64_rel_l2_after_1_step"] = float((d.norm() / outs["fp64"].norm()).item())
            entry["mixed_speedup_over_fp64"] = entry["fp64"]["ms_per_step"] / entry["mixed"]["ms_per_step"]
        del outs, phi0
        torch.cuda.empty_cache()
        res.append(entry)
    if only is None:
        res.append(measure_batch(sl, torch, flush, nprob=64 if full else 16))
    return res


def measure_batch(sl, torch, flush, nprob=64, steps=3):
    """The batched rotation workload: nprob p-adaptive problems (sides 32..256) advanced together,
    each with its own step (sl_batch_step), mixed precision; one FP64 batch step for the error."""
    probs = sl_inputs.config4_batch(nprob)
    entry = {"workload": f"2d_rotation_batch_{nprob}_problems_p-adaptive (config 4 batch)"}
    outs = {}
    phi0 = None
    for prec in (sl.MIXED, sl.FP64):
        ctxs = [sl.Context(2, p.kx, p.ky, p.box, p.n, p.basis, prec, p.bc, p.ghost, orders=p.orders) for p in probs]
        batch = sl.Batch(ctxs)
        vel = sl.velocity(probs[0].velocity.kind, *probs[0].velocity.p)
        dts = [c.max_dt(vel, sl_inputs.rule_code(p)) for c, p in zip(ctxs, probs)]
        if phi0 is None:
            phis = []
            for c, p in zip(ctxs, probs):
                x, y = c.node_coords()
                phis.append(torch.tensor(p.phi0(x, y), device="cuda"))
            phi0 = torch.cat(phis)
            del phis
        opts = sl.options(probs[0].constraints, probs[0].rk_order)
        a, b = batch.pack(phi0), batch.new_state()
        key = "mixed" if prec == sl.MIXED else "fp64"
        batch.batch_step(a, b, vel, [0.0] * nprob, dts, opts)
        outs[key] = batch.unpack(b)
        n_steps = steps if prec == sl.MIXED else 1
        stream = batch.stream
        times = []
        for s in range(n_steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.batch_step(b, a, vel, [d * (s + 1) for d in dts], dts, opts)
            e1.record(stream)
            a, b = b, a
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        per = float(np.mean(times))
        entry["nodes"] = batch.size
        entry[key] = {"ms_per_step": per, "node_updates_per_s": batch.size / (per * 1e-3), "steps": n_steps,
                      "device_status": batch.sync()}
        del batch, ctxs, a, b
        torch.cuda.empty_cache()
    d = outs["mixed"] - outs["fp64"]
    entry["mixed_vs_fp64_rel_l2_after_1_step"] = float((d.norm() / outs["fp64"].norm()).item())
    entry["mixed_speedup_over_fp64"] = entry["fp64"]["ms_per_step"] / entry["mixed"]["ms_per_step"]
    return entry


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=9, help="nodes per element (N + 1)")
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 per-element comparison")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-configs", action="store_true", help="skip the other configurations")
    ap.add_argument("--all-configs", action="store_true",
                    help="add the 2048^2 swirl and the 64-problem batch to the other configurations")
    ap.add_argument("--only-config", type=int, default=None, help="of the other configurations, only this one")
    ap.add_argument("--quick-configs", action="store_true", help="(default) other configurations, smaller set")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
