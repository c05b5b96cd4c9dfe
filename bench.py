"""Benchmark of the DSEM-SL step on GB300: Gauss-node updates per second.

Headline workload (the largest configuration that fits one GPU): 2D swirling deformation flow
u = sin^2(pi x) sin(2 pi y) cos(pi t / T), v = -sin^2(pi y) sin(2 pi x) cos(pi t / T), T = 5, on the
unit square with inflow faces (ghost 0; the walls carry no normal velocity), 2048 x 2048 elements,
N = 7 (n = 8 Gauss-Legendre nodes per direction, 268,435,456 nodes), cosine bell of radius 0.15
at (0.5, 0.75), boundary + mass + energy constraints, RK4 particle integration, half the paper's
time step (the paper's, the edge-node gap over |u|max, keeps every particle inside its element but
is the stability limit of this flow on fine meshes; half of it stays bounded).  One bench step
is one time step of the whole mesh: phase-1 and phase-2 launches of the general mixed-precision
kernels (double-float state, float bulk arithmetic, float-float mass).  Inputs stay resident in
HBM; each state buffer (2.1 GB) is larger than L2, and L2 (129 MB) is also flushed by writing a
256 MB buffer before every timed step.  The plain FP64 per-element form of the same step is timed
beside it; the other configurations follow under "configs".

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
# FP32 lanes of the GPU: 152 SMs x 128 FP32 units, two FLOPs per fused multiply-add
FP32_LANES = 152 * 128
HEAD_K, HEAD_N = 2048, 8


def peaks():
    try:
        d = json.load(open(MEASURED))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def workload_config(k=HEAD_K, n=HEAD_N, precision_name="mixed"):
    return {"workload": f"2d_swirl_{k}x{k}_N{n - 1}_n{n}_GL_boundary+mass+energy_RK4_half-paper-dt_{precision_name} (config 5)",
            "elements": k * k, "nodes_per_element": n * n, "nodes": k * k * n * n, "steps_per_bench_step": 1,
            "l2": "inputs larger than L2 (2.1 GB per state buffer) and a 256 MB write before every timed step",
            "parallelism": "replicas"}


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


# ----------------------------------------------------------------------------- CPU oracle leg


class _LazyRow:
    def __init__(self, parent, ey):
        self.parent, self.ey = parent, ey

    def __getitem__(self, ex):
        return self.parent.element(ex, self.ey)


class LazyState:
    """phi[ey][ex] of a 2D mesh, evaluated from the analytic initial data when an element is read
    (the oracle reads one element and its face neighbours per step)."""

    def __init__(self, setup, f):
        self.setup, self.f, self.cache = setup, f, {}

    def element(self, ex, ey):
        key = (ex, ey)
        if key not in self.cache:
            from oracle import sl_oracle as O
            X, Y = O.node_coords_2d(self.setup, ex, ey)
            self.cache[key] = self.f(X, Y)
        return self.cache[key]

    def __getitem__(self, ey):
        return _LazyRow(self, ey)


def _oracle_elements(args):
    """One oracle step, from the initial state at t = 0, of a list of elements of the headline
    workload (run in a worker process); returns ({(ex, ey): values}, seconds)."""
    k, n, elems, dt = args
    from oracle import sl_oracle as O
    prob = sl_inputs.config5_swirl(n=n, k=k)
    setup = O.setup_from_problem(prob)
    phi = LazyState(setup, prob.phi0)
    o = O.StepOpts(O.Vel(O.VEL_SWIRL, prob.velocity.p), 0.0, dt, prob.constraints, prob.rk_order)
    cache = {}
    out = {}
    t0 = time.perf_counter()
    for ex, ey in elems:
        out[(ex, ey)], _ = O.element_step_2d(setup, phi, ex, ey, o, cache)
    return out, time.perf_counter() - t0


def bell_elements(k, count, run):
    """A run of `count` consecutive elements along one row through the cosine bell (every term of the
    step is active there; consecutive elements share their neighbours' remaps).  Run r takes the row
    0.75 k + 7 r (mod 0.3 k, centred on the bell) and starts at column 0.5 k - count / 2."""
    span = max(1, int(0.3 * k))
    row = int(0.75 * k) - span // 2 + (7 * run) % span
    col = max(0, int(0.5 * k) - count // 2)
    return [(col + i, row) for i in range(count)]


def cpu_oracle_run(dt, per_worker, workers, k=HEAD_K, n=HEAD_N):
    """Time the FP64 oracle as it stands on a bounded sample of the headline workload: `workers`
    processes (spawned, one thread each), `per_worker` elements each.  Returns (results, rate in
    node updates/s, cores used, sample description)."""
    chunks = [(k, n, bell_elements(k, per_worker, w), dt) for w in range(workers)]
    t0 = time.perf_counter()
    if workers == 1:
        res = [_oracle_elements(chunks[0])]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_oracle_elements, chunks)
    wall = time.perf_counter() - t0
    merged = {}
    for r, _ in res:
        merged.update(r)
    nodes = len(merged) * n * n
    busy = max(s for _, s in res)
    rate = nodes / busy
    desc = (f"{len(merged)} elements of the 2048^2 swirl near the bell, one step from t = 0, numpy FP64, "
            f"{workers} process(es) x 1 thread, {busy:.1f} s of oracle time ({wall:.1f} s wall incl. start-up)")
    return merged, rate, workers, desc


def cpu_baseline(dt, seconds=12.0):
    """The oracle on the host cores: single-threaded and one process per core."""
    per_elem = 0.02
    n1 = max(8, int(seconds / 2 / per_elem))
    _, r1, _, d1 = cpu_oracle_run(dt, n1, 1)
    cores = os.cpu_count() or 1
    merged, rc, used, dc = cpu_oracle_run(dt, max(8, int(seconds / 2 / per_elem)), cores)
    return {"value": rc, "unit": UNIT, "cores": used, "kind": "oracle", "sample": dc,
            "single_thread": {"value": r1, "cores": 1, "sample": d1}, "host_nproc": cores}, merged


# ----------------------------------------------------------------------------- multi-rank helpers


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
    if rank != 0:
        return
    prob = sl_inputs.config5_swirl(n=HEAD_N, k=HEAD_K)
    dt = config_dt(prob)
    cores = os.cpu_count() or 1
    # each step a bounded sample of the workload, so that the whole run stays within a few minutes
    per = max(4, int(min(args.ref_seconds, 90.0 / (args.steps + args.warmup)) / 0.02))
    for _ in range(args.warmup):
        cpu_oracle_run(dt, 4, 1)
    vals, desc = [], ""
    for _ in range(args.steps):
        _, rate, used, desc = cpu_oracle_run(dt, per, cores)
        vals.append(rate)
    v = statistics.mean(vals)
    nodes = HEAD_K * HEAD_K * HEAD_N * HEAD_N
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * nodes / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(precision_name="mixed"),   # the same workload as the GPU arm
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dt(prob):
    """The configured time step of the swirl (half the paper's: half the edge-node gap over
    |u|max = 1) for the reference arm, which runs no GPU code: the Gauss-Legendre edge gap from
    numpy's nodes."""
    x, _ = np.polynomial.legendre.leggauss(prob.n)
    return 0.5 * 0.5 * (x[0] + 1.0) * (prob.box[1] - prob.box[0]) / prob.kx


# ----------------------------------------------------------------------------- GPU leg


def device_initial_state(torch, ctx, prob):
    """Initial data at the library's nodes (sl_nodes_weights; documented state layout), evaluated
    on the device: no host array of the full mesh."""
    xi, _ = ctx.nodes_weights()
    n, kx, ky = prob.n, prob.kx, prob.ky
    x0, x1, y0, y1 = prob.box
    hx, hy = (x1 - x0) / kx, (y1 - y0) / ky
    xi_t = torch.tensor(xi, device="cuda", dtype=torch.float64)
    ex = torch.arange(kx, device="cuda", dtype=torch.float64)
    ey = torch.arange(ky, device="cuda", dtype=torch.float64)
    out = torch.empty((ky, kx, n, n), device="cuda", dtype=torch.float64)
    X = x0 + (ex[:, None] + xi_t[None, :]) * hx          # [kx][n] (i)
    for r in range(0, ky, 256):
        Y = y0 + (ey[r:r + 256, None] + xi_t[None, :]) * hy  # [rows][n] (j)
        xx = X[None, :, None, :]
        yy = Y[:, None, :, None]
        rr = torch.sqrt((xx - 0.5) ** 2 + (yy - 0.75) ** 2)
        out[r:r + 256] = torch.where(rr < 0.15, 0.5 * (1.0 + torch.cos(math.pi * torch.clamp(rr, max=0.15) / 0.15)),
                                     torch.zeros_like(rr))
    return out.reshape(-1)


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


def flop_model(n, rk, nel, c):
    """Algorithmic FP32 operations of one step of the general mixed path (FMA = 2), counted from
    the steps of the method with the iteration counts the kernels report (sl_counters, per step):
      velocity evaluation at a displaced point (swirl, angle addition): 40;
      phase 1, per element: RK advection of n^2 particles, S stages x (velocity + 4); two Lagrange
      bases per particle, 2 x 5 n; the collocation iteration, per residual evaluation 2 n (n + 1)
      per particle plus a preconditioner pass of 4 n; traces 4 n x 2 n; psi^n and the float-float
      element mass, 30 per node; the sign of u.n at 4 n face points x distinct stage times
      (velocity each); per traced outflow foot: backward RK (S x (velocity + 4)), two bases and the
      evaluation 2 n (n + 1);
      phase 2, per element: interface values at 4 n face points (velocity + 20); the fit, 2 m per
      node (m = 4 n + 1 rows); per energy iteration 2 m + 10 per node plus 4 n x 2 n traces; the
      float-float write-back and mass refinement, 40 per node.
    Returns (phase-1 flops, phase-2 flops) per step."""
    nd = n * n
    S = rk
    sd = {1: 1, 2: 2, 3: 3, 4: 3}[rk]
    vel = 40
    m = 4 * n + 1
    el = max(c.get("elems", 0), 1)
    iters = c.get("solve_iters", 0) / el
    feet = c.get("feet", 0) / el
    pit = c.get("picard_iters", 0) / el
    p1 = (nd * S * (vel + 4) + nd * 2 * 5 * n + nd * iters * (2 * n * (n + 1) + 4 * n) + 4 * n * 2 * n + nd * 30
          + 4 * n * sd * vel + feet * (S * (vel + 4) + 2 * 5 * n + 2 * n * (n + 1)))
    p2 = 4 * n * (vel + 20) + nd * 2 * m + pit * (nd * (2 * m + 10) + 4 * n * 2 * n) + nd * 40
    return p1 * nel, p2 * nel


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
    k, n = args.k, HEAD_N
    prob = sl_inputs.config5_swirl(n=n, k=k)
    stream = torch.cuda.current_stream()
    ctx = sl.Context(2, k, k, prob.box, n, sl.GAUSS_LEGENDRE, sl.MIXED, prob.bc, prob.ghost, stream)
    vel = sl.velocity(sl.VEL_SWIRL, *prob.velocity.p)
    dt = ctx.max_dt(vel, sl_inputs.rule_code(prob))      # half the paper's step (stability limit)
    opts = sl.options(prob.constraints, prob.rk_order)
    phi0_dev = device_initial_state(torch, ctx, prob)
    a = ctx.pack(phi0_dev)
    b = ctx.new_state()
    tuned = autotune(sl, ctx, a, b, vel, 0.0, dt, opts)             # launch shapes (sl_tune)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # one step from t = 0 for the accuracy check against the oracle
    ctx.step(a, b, vel, 0.0, dt, opts)
    first = ctx.unpack(b) if (rank == 0 and not args.no_check) else None
    t = 0.0
    for _ in range(args.warmup):
        ctx.step(a, b, vel, t, dt, opts)
        a, b = b, a
        t += dt
    torch.cuda.synchronize()
    warm_bits = ctx.sync()
    assert warm_bits & ~sl.ST_PICARD_NOCONV == 0, f"device status bits {warm_bits} during warm-up"

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.counters()
    ctx.timing(True)
    with ClockSampler(local_rank) as clocks:
        total_ms, a, b, t = _time_steps(torch, ctx, stream, a, b, vel, dt, opts, t, args.steps, flush)
    if world > 1:
        dist.barrier()
    p1_ms, p2_ms, _, timed = ctx.timing_read()
    ctx.timing(False)
    counts = ctx.counters()
    status = ctx.sync()
    nodes = k * k * n * n
    nel = k * k
    total_ms = max_over_ranks(total_ms, world, "cuda")
    value = job_throughput(world, nodes, args.steps, total_ms * 1e-3)

    # end to end through the public API: host doubles in, one step, host doubles out, every step
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    host_in = phi0_dev.cpu().pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    ctx.run_host(host_in, host_out, vel, 0.0, dt, 1, opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        ctx.run_host(host_in, host_out, vel, s * dt, dt, 1, opts)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_value = job_throughput(world, nodes, e2e_steps, e2e_s)
    del host_in, host_out
    ctx.sync()

    # the plain FP64 per-element form on the same workload, and the mixed-vs-FP64 error
    fp64, err = None, {}
    if not args.no_fp64:
        c64 = sl.Context(2, k, k, prob.box, n, sl.GAUSS_LEGENDRE, sl.FP64, prob.bc, prob.ghost, stream)
        a64, b64 = phi0_dev.clone(), torch.empty_like(phi0_dev)
        m_a, m_b = ctx.pack(phi0_dev), ctx.new_state()
        nerr = args.fp64_steps
        for s in range(nerr):
            c64.step(a64, b64, vel, s * dt, dt, opts)
            ctx.step(m_a, m_b, vel, s * dt, dt, opts)
            a64, b64, m_a, m_b = b64, a64, m_b, m_a
        d = ctx.unpack(m_a) - a64
        err[f"after_{nerr}_steps_vs_fp64_path"] = float((d.norm() / a64.norm()).item())
        del m_a, m_b, d
        k64 = 2
        ms64, _, _, _ = _time_steps(torch, c64, stream, a64, b64, vel, dt, opts, nerr * dt, k64, flush)
        fp64 = {"value": nodes * k64 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64 / k64,
                "kernels": "k2d::k_p1<8>, k_p2<8> (FP64 pipe)", "device_status": c64.sync()}
        del c64, a64, b64
        torch.cuda.empty_cache()
    err["bound"] = 1e-6

    # CPU oracle: the baseline on the host cores, and the accuracy of the first GPU step on the
    # oracle's sample (elements near the bell, recomputed from the same initial data)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, merged = cpu_baseline(dt, seconds=args.ref_seconds)
        if first is not None:
            got = first.reshape(k, k, n, n)
            keys = sorted(merged)
            g = torch.stack([got[ey, ex] for ex, ey in keys]).cpu().numpy()
            r = np.stack([merged[key] for key in keys])
            err["after_1_step_vs_oracle_sampled"] = float(np.sqrt(np.sum((g - r) ** 2) / np.sum(r ** 2)))
            err["oracle_sample_elements"] = len(keys)

    if rank != 0:
        return
    hbm, peak_kind = peaks()
    avg_ms = total_ms / args.steps
    clk = clocks.summary()
    sm_mhz = clk.get("sm_mhz") or 2070.0
    per_step = {kk: v / max(args.steps, 1) for kk, v in counts.items()}
    f1, f2 = flop_model(n, prob.rk_order, nel, per_step)
    p1_avg, p2_avg = p1_ms / max(timed, 1), p2_ms / max(timed, 1)
    fp32_peak = FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    kern = [{"kernel": "k2m::k_p1<8> (advection, collocation, traces, face outflow)", "ms_per_launch": p1_avg,
             "algorithmic_tflop": f1 / 1e12, "achieved_tflops": f1 / (p1_avg * 1e-3) / 1e12,
             "alu_frac": f1 / (p1_avg * 1e-3) / 1e12 / fp32_peak,
             "hbm_frac": nodes * 8 / (p1_avg * 1e-3) / 1e9 / hbm},
            {"kernel": "k2m::k_p2<8> (interface values, targets, fit, energy, write-back)", "ms_per_launch": p2_avg,
             "algorithmic_tflop": f2 / 1e12, "achieved_tflops": f2 / (p2_avg * 1e-3) / 1e12,
             "alu_frac": f2 / (p2_avg * 1e-3) / 1e12 / fp32_peak,
             "hbm_frac": nodes * 8 / (p2_avg * 1e-3) / 1e9 / hbm}]
    dom = kern[0] if p1_avg >= p2_avg else kern[1]
    dom_ms = max(p1_avg, p2_avg)
    dom_f = f1 if p1_avg >= p2_avg else f2
    roof = {"bound": "alu", "achieved": dom_f / (dom_ms * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": dom_f / (dom_ms * 1e-3) / 1e12 / fp32_peak, "traffic": (TRAFFIC_PER_ELEMENT[dom["kernel"].split(" ")[0]] * nel
                        if dom["kernel"].split(" ")[0] in TRAFFIC_PER_ELEMENT else None),
            "kernel": dom["kernel"], "ms_per_launch": dom_ms,
            "peak_source": f"FP32: {FP32_LANES} lanes x 2 x median SM clock {sm_mhz:.0f} MHz under load (unit counts)",
            "flop_model": "bench.flop_model (algorithmic FP32 operations from the measured iteration counts)",
            "hbm": {"achieved": nodes * 16 / (avg_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": nodes * 16 / (avg_ms * 1e-3) / 1e9 / hbm, "algorithmic_bytes_per_node": 16,
                    "peak_source": f"{peak_kind} hbm_gbs (copy, burst)", "of": "whole step (both launches)"},
            "kernels": kern}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": avg_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (double-float state, float-float mass)",
            "data": "synthetic (seeded analytic cosine bell)",
            "config": dict(workload_config(k, n, "mixed"), dt=dt),
            "roofline": roof, "clocks": clk, "autotune": tuned,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nodes * 8, "d2h_bytes_per_step": nodes * 8,
                    "api": "sl_run_host (pinned host doubles in, one step, host doubles out)"},
            "gpu_launches": 2 * args.steps,
            "work_counters_per_step": per_step,
            "picard_noconv_elements_per_step": per_step.get("picard_noconv"),
            "l2_error_vs_fp64": err,
            "fp64_per_element": fp64,
            "mixed_speedup_over_fp64": (fp64["ms_per_step"] / avg_ms) if fp64 else None,
            "device_status": status}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if not args.no_configs:
        line["configs"] = secondary_configs(sl, torch, flush, full=args.all_configs, only=args.only_config)
    print(json.dumps(line), flush=True)


# DRAM bytes per launch from one ncu capture (read + written), scaled to the full mesh by the
# element count (traffic grows in proportion); None once the kernel has changed since
# DRAM bytes (read + write) per element of the dominant kernels, from one ncu capture of both at
# 512 x 512 (262,144 elements; traffic grows in proportion to the elements), multiplied by the
# element count of a launch.  Valid for the kernels as profiled; to be taken again after a change
# to them.
TRAFFIC_PER_ELEMENT = {"k2m::k_p1<8>": (139.418112e6 + 89.868288e6) / 262144,
                       "k2m::k_p2<8>": (272.105728e6 + 113.296384e6) / 262144}


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
    tuned = autotune(sl, ctx, a, b, vel, 0.0, dt, opts)             # launch shapes (sl_tune)
    ctx.step(a, b, vel, 0.0, dt, opts)           # warm-up
    torch.cuda.synchronize()
    ms, a, b, _ = _time_steps(torch, ctx, stream, b, a, vel, dt, opts, dt, steps, flush)
    status = ctx.sync()
    nodes = ctx.size
    per = ms / steps
    return {"ms_per_step": per, "node_updates_per_s": nodes / (per * 1e-3), "steps": steps,
            "hbm_frac_of_measured": nodes * 16 / (per * 1e-3) / 1e9 / peaks()[0], "device_status": status,
            "autotune": tuned}, phi0, (ctx, vel, dt, opts)


def tune_cache_path():
    """The autotuner's JSON cache: SL_TUNE_CACHE, else the user's cache directory (None when that
    cannot be created: the tuner then times without a cache)."""
    p = os.environ.get("SL_TUNE_CACHE")
    if not p:
        d = os.path.join(os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache")),
                         "paper_1910_06476_gb300")
        try:
            os.makedirs(d, exist_ok=True)
        except OSError:
            return None
        p = os.path.join(d, "tune.json")
    return p


def autotune(sl, ctx, a, b, vel, t, dt, opts):
    """sl_tune with the cache; a cache that cannot be read or written falls back to timing without
    one (the choice is then reported with the reason)."""
    try:
        return ctx.tune(a, b, vel, t, dt, opts, tune_cache_path())
    except sl.SlError as e:
        r = ctx.tune(a, b, vel, t, dt, opts, None)
        r["cache_error"] = str(e)
        return r


def secondary_configs(sl, torch, flush, full=False, only=None):
    """The other configurations of the measurement plan on both paths, outside the headline timed
    region (the 64-problem batch by graph replay; with full=True, also the 16-problem batch stepped
    problem by problem)."""
    res = []
    plan = [("1d_sine_K16_n9 (config 1)", sl_inputs.config1_1d_sine(), [sl.FP64], 200)]
    for n in (5, 9, 13, 17):
        plan.append((f"1d_gauss_K2^20_n{n} (config 2)", sl_inputs.config2_1d_gauss(n), [sl.MIXED, sl.FP64], 50))
    plan.append(("2d_const_512x512_n9 (config 3)", sl_inputs.config3_2d_const(), [sl.MIXED, sl.FP64], 10))
    plan.append(("2d_rotation_256x256_p-adaptive_n4-16 (config 4)", sl_inputs.config4_rotation(), [sl.MIXED, sl.FP64],
                 10))
    if only is not None:
        plan = [p for p in plan if f"(config {only})" in p[0]]
    for name, prob, precs, steps in plan:
        entry = {"workload": name, "nodes": None}
        phi0, outs = None, {}
        for prec in precs:
            r, phi0, run = measure_config(sl, torch, prob, prec, steps, flush, phi0)
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
        res.append(measure_batch_graph(sl, torch, flush, nprob=64))
        if full:
            res.append(measure_batch(sl, torch, flush, nprob=16))
    return res


def measure_batch_graph(sl, torch, flush, nprob=64, steps=10):
    """The 64-problem rotation batch (sides 32..256, p-adaptive) advanced by sl_run's captured graph
    (every problem with the same dt: the smallest limit over the problems), mixed precision; the
    same steps by sl_step for the graph's equality with stepping; one FP64 step for the error."""
    probs = sl_inputs.config4_batch(nprob)
    entry = {"workload": f"2d_rotation_batch_{nprob}_problems_p-adaptive (config 4 batch, sl_run graph replay)"}
    outs = {}
    phi0 = None
    for prec in (sl.MIXED, sl.FP64):
        ctxs = [sl.Context(2, p.kx, p.ky, p.box, p.n, p.basis, prec, p.bc, p.ghost, orders=p.orders) for p in probs]
        batch = sl.Batch(ctxs)
        vel = sl.velocity(probs[0].velocity.kind, *probs[0].velocity.p)
        dt = batch.max_dt(vel, sl_inputs.rule_code(probs[0]))
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
        batch.step(a, b, vel, 0.0, dt, opts)
        outs[key] = batch.unpack(b)
        entry["nodes"] = batch.size
        if prec == sl.MIXED:
            batch.run(a, b, vel, 0.0, dt, steps, opts)       # capture
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(batch.stream)
            batch.run(a, b, vel, 0.0, dt, steps, opts)
            e1.record(batch.stream)
            torch.cuda.synchronize()
            per = e0.elapsed_time(e1) / steps
            entry[key] = {"ms_per_step": per, "node_updates_per_s": batch.size / (per * 1e-3), "steps": steps,
                          "api": "sl_run", "device_status": batch.sync()}
        else:
            ms, _, _, _ = _time_steps(torch, batch, batch.stream, a, b, vel, dt, opts, dt, 1, flush)
            entry[key] = {"ms_per_step": ms, "node_updates_per_s": batch.size / (ms * 1e-3), "steps": 1,
                          "device_status": batch.sync()}
        del batch, ctxs, a, b
        torch.cuda.empty_cache()
    d = outs["mixed"] - outs["fp64"]
    entry["mixed_vs_fp64_rel_l2_after_1_step"] = float((d.norm() / outs["fp64"].norm()).item())
    entry["mixed_speedup_over_fp64"] = entry["fp64"]["ms_per_step"] / entry["mixed"]["ms_per_step"]
    return entry


def measure_batch(sl, torch, flush, nprob=16, steps=3):
    """The batched rotation workload with a step of its own per problem (sl_batch_step), mixed."""
    probs = sl_inputs.config4_batch(nprob)
    entry = {"workload": f"2d_rotation_batch_{nprob}_problems_p-adaptive (config 4 batch, sl_batch_step)"}
    ctxs = [sl.Context(2, p.kx, p.ky, p.box, p.n, p.basis, sl.MIXED, p.bc, p.ghost, orders=p.orders) for p in probs]
    batch = sl.Batch(ctxs)
    vel = sl.velocity(probs[0].velocity.kind, *probs[0].velocity.p)
    dts = [c.max_dt(vel, sl_inputs.rule_code(p)) for c, p in zip(ctxs, probs)]
    phis = []
    for c, p in zip(ctxs, probs):
        x, y = c.node_coords()
        phis.append(torch.tensor(p.phi0(x, y), device="cuda"))
    phi0 = torch.cat(phis)
    opts = sl.options(probs[0].constraints, probs[0].rk_order)
    a, b = batch.pack(phi0), batch.new_state()
    batch.batch_step(a, b, vel, [0.0] * nprob, dts, opts)
    times = []
    for s in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(batch.stream)
        batch.batch_step(b, a, vel, [d * (s + 1) for d in dts], dts, opts)
        e1.record(batch.stream)
        a, b = b, a
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    per = float(np.mean(times))
    entry["nodes"] = batch.size
    entry["mixed"] = {"ms_per_step": per, "node_updates_per_s": batch.size / (per * 1e-3), "steps": steps,
                      "device_status": batch.sync()}
    return entry


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=HEAD_K, help="elements per direction of the headline mesh")
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=3, help="steps of the mixed-vs-FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 per-element comparison")
    ap.add_argument("--no-configs", action="store_true", help="skip the other configurations")
    ap.add_argument("--all-configs", action="store_true", help="add the 16-problem batch stepped per problem")
    ap.add_argument("--only-config", type=int, default=None, help="of the other configurations, only this one")
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
