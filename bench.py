"""Benchmark of the Symanzik MD hot path on GB300.

One step = one pass of the whole hot path over one 32^3x64 lattice of FP32
compact links (w_a ~ N(0, 0.3^2), u0 = 0.87, beta = 6): one
lqcd_md_force_step call (staple planes, then the force on every link with the
momentum step p += dt f and the gauge action fused into the same pass),
then the link step U <- exp(i dt p.T) U (the coefficients are computed once
on the host).  value = 4V links / step time in Glink/s.
Inputs (403 MB of links, 268 MB of momenta, 268 MB of force) are larger
than the 129 MB L2, so no flush is needed between steps.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--force-variant V] [--profile-force WORKLOAD]
N > 1 runs as independent replicas, one lattice per rank (the path has no
exchange step on one lattice per GPU); value = links of all ranks / max time.
--impl reference times the FP64 CPU oracle on the host cores instead.
--profile-force WORKLOAD runs only W + K FP32 force calls (the staple-field
force with the fused momentum step and action) on that workload (a key of
synth.WORKLOADS, e.g. 16^3x32, or extents such as 32x16x16x16, drawn like
the 32^3x64 workload) and prints their mean time: the small case
that profiler captures run.  --profile-wilson WORKLOAD does the same for the
FP32 Wilson hopping operator and hopping-term force.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "32^3x64"
METRIC = "Symanzik force Glink/s at 32^3x64 FP32 vs FP64; % HBM roofline; dH error"
DT = 0.05
# Algorithmic work per link-force of the literal algorithm (48 staples = 180
# SU(3) products of 198 flops, 47 matrix additions of 18 flops, U t and the
# projection): 36.9 kflop; compulsory bytes: FP32 12-real link read (48 B) +
# 8-real force write (32 B).
FLOP_PER_LINK_FORCE = 36.9e3
# What the staple-field force executes per link (FP32, full staple planes,
# FMA = 2 flops; a compact link's row 2 rebuild = 42 flops; a product of two
# SU(3) matrices with its third row rebuilt from its first two and
# accumulated = 144 + 42 + 36 = 222; a plain accumulated product = 216):
#   staple planes: 6 staples per link, each two link rebuilds (84), rows 0
#     and 1 of the first product (132), rows 0 and 1 of the second (144) and
#     the staple's third row (42): 2412;
#   force pass: plaquette and rectangle chains 6 x (18 + 222 + 216) = 2736,
#     their two link products and scalings 552, the action's trace 78,
#     six d-terms of 5 x 222 + 216 + 2 x 42 = 1410 each (8460), U t and the
#     projection, momentum step and action share (~282): 12108.
EXECUTED_FLOP_PER_LINK_FORCE = 2412 + 12108
BYTES_PER_LINK_FORCE = {"f32": 80, "f64": 160}
# streaming kernels, compulsory bytes per link
BYTES_MOM_UPDATE = {"f32": 96, "f64": 192}     # read p, read f, write p
BYTES_LINK_UPDATE = {"f32": 128, "f64": 256}   # read U, read p, write U
# FP32 pipe peak from unit counts and the maximum SM clock: 152 SMs x 128
# FP32 lanes x 2 flop (FMA) x 2.070 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
CPU_SAMPLE_DIMS = (12, 12, 12, 12)
# Wilson fermion kernels (Sec. III), compulsory bytes in units of the real
# size R: the hopping operator reads x (24 R) and the 4 links of a site
# (48 R) and writes y (24 R) per site; the hopping-term force with the fused
# momentum step reads per link its link (12 R), a quarter of a site's X and Y
# (12 R) and the momenta (8 R), and writes the momenta (8 R).
WILSON_KAPPA = 0.1315
# thermalising FP32 trajectories before the same-start dH comparison
DH_THERM = 30
WILSON_REALS_PER_SITE_DSLASH = 96
WILSON_REALS_PER_LINK_FORCE = 40


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _source_digest() -> str:
    """Digest of the force kernels' code (comments and whitespace stripped,
    so that only a change of the code itself invalidates a recorded profile)."""
    h = hashlib.sha256()
    for f in ("force_sf.cu", "su3.cuh"):
        with open(os.path.join(ROOT, "paper_1808_02281_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "force_traffic_f32_32x32x32x64.json")


def _recorded_traffic():
    """DRAM bytes (read + write) per force call at the bench workload from the
    machine-readable record written beside the ncu summary, if it was taken
    on the current force kernel source (same digest); else None."""
    try:
        with open(TRAFFIC_RECORD) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("source_digest") != _source_digest():
        return None
    return float(rec["traffic_bytes_per_call"])


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) taken while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[2:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle

def oracle_step_rate(dims=CPU_SAMPLE_DIMS, steps: int = 1):
    """The FP64 CPU oracle running the same step (force, momentum step, link
    step, action) on a lattice drawn like the benchmark workload; returns
    links per second over ``steps`` steps and the seconds taken."""
    from oracle import oracle as O
    from paper_1808_02281_gb300 import synth
    w = synth.WORKLOADS[WORKLOAD]
    U = O.links_from_omega(synth.omega(dims, w["sigma"], w["seed"]))
    p = synth.momenta(dims, seed=1)
    c = O.coefficients(w["u0"])
    t0 = time.perf_counter()
    for _ in range(steps):
        f = O.gauge_force(dims, U, w["beta"], c)
        p = O.md_update_momenta(p, f, DT)
        U = O.md_update_links(U, p, DT)
        O.gauge_action(dims, U, w["beta"], c)
    dt = time.perf_counter() - t0
    return 4 * synth.volume(dims) * steps / dt, dt


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_replica(steps: int):
    """One worker of the all-cores oracle timing (a separate process)."""
    rate, secs = oracle_step_rate(steps=steps)
    return rate, secs


class OracleReplicas:
    """The oracle as it stands, one independent replica per host core: a
    process pool started with spawn (never forked from a process that holds
    a CUDA context); throughput = the sum of the replicas' rates."""

    def __init__(self, workers: int | None = None):
        from oracle import oracle as O
        O.build()                      # compiled once, before the workers load it
        self.workers = workers or host_cores()
        self.pool = multiprocessing.get_context("spawn").Pool(self.workers)

    def step(self, steps: int = 1):
        """(aggregate links/s, wall seconds) of `steps` oracle steps on every core."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_replica, [steps] * self.workers)
        return sum(r for r, _ in res), time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    reps = OracleReplicas()
    try:
        for _ in range(args.warmup):
            reps.step(1)
        rates, secs = [], []
        for _ in range(args.steps):
            r, s = reps.step(1)
            rates.append(r)
            secs.append(s)
    finally:
        reps.close()
    value = statistics.mean(rates) / 1e9
    sample = (f"per timed step, one oracle step (force, momentum step, link step, action) of a "
              f"{'x'.join(map(str, CPU_SAMPLE_DIMS))} lattice drawn like the {WORKLOAD} workload "
              f"(w_a ~ N(0, 0.3^2), u0 0.87) on each of {reps.workers} host cores, one "
              f"independent single-threaded replica per core; per-link work is volume independent")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Glink/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(secs) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_dims": list(CPU_SAMPLE_DIMS)},
        "cpu_baseline": {"value": value, "unit": "Glink/s", "cores": reps.workers,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Glink/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))
    return 0


# ------------------------------------------------- replicas on N ranks

class RankContext:
    """One process per GPU (torchrun): replicas of the workload, no data-path
    collective; only barriers and the max-over-ranks of timings."""

    def __init__(self, backend: str = "nccl"):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.backend = backend
        if self.world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, x: float, device=None) -> float:
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device or "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def replica_seed(seed: int, rank: int) -> int:
    """Each rank draws its own lattice (the same workload, another sample)."""
    return seed + rank


def weak_scaling_value(links_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Links of all ranks per second (Glink/s) over the slowest rank's time."""
    return world * links_per_rank * steps / (ms_max / 1e3) / 1e9


# ----------------------------------------------------------------- GPU arm

def run_ours(args):
    import torch

    from paper_1808_02281_gb300 import build as B
    from paper_1808_02281_gb300 import lqcd, synth

    ctx = RankContext("nccl")
    world, rank, local = ctx.world, ctx.rank, ctx.local
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        B.build()
    ctx.barrier()
    barrier = ctx.barrier

    w = synth.WORKLOADS[WORKLOAD]
    dims = w["dims"]
    V = synth.volume(dims)
    nlinks = 4 * V
    seed = replica_seed(w["seed"], rank)
    omega_np = synth.omega(dims, w["sigma"], seed)
    p_np = synth.momenta(dims, seed=1000 + seed)
    stream = torch.cuda.current_stream(dev)
    launches = {"n": 0}

    def make(prec):
        lat = lqcd.Lattice.symanzik(dims, w["beta"], w["u0"], prec)
        U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, omega_np, device=dev))
        mom = lqcd.algebra_to_device(lat, p_np, device=dev)
        force = lqcd.empty_algebra(lat, dev)
        S = torch.empty((), dtype=torch.float64, device=dev)
        ws = lqcd.make_workspace(lat, dev)
        return lat, U, mom, force, S, ws

    def step(lat, U, mom, force, S, ws, ev=None):
        if ev is not None:
            ev[0].record(stream)
        # force + momentum step + action in one call (staple planes, force pass, action sum)
        lqcd.md_force_step(lat, U, mom=mom, dt=DT, action=S, workspace=ws)
        if ev is not None:
            ev[1].record(stream)
        lqcd.md_update_links(lat, U, mom, DT)
        if ev is not None:
            ev[2].record(stream)
        launches["n"] += 4  # staple planes, force pass, action sum, link step

    tuned = {}

    def timed(prec, K, W, with_events):
        lat, U, mom, force, S, ws = make(prec)
        # set-up, untimed: pick the fastest force schedule on these links, or
        # take the one fixed on the command line (reproducible profiling)
        if args.force_variant >= 0:
            lqcd.set_force_variant(lat, args.force_variant)
            tuned[prec] = {"variant": args.force_variant, "fixed": True}
        else:
            best, ms_v = lqcd.autotune_force(lat, U, reps=3, workspace=ws)
            tuned[prec] = {"variant": best, "ms_per_variant": ms_v}
        for _ in range(W):
            step(lat, U, mom, force, S, ws)
        torch.cuda.synchronize(dev)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)] \
            if with_events else [None] * K
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches["n"] = 0
        barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        for k in range(K):
            step(lat, U, mom, force, S, ws, evs[k])
        stop.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms = start.elapsed_time(stop)
        n_launch = launches["n"]
        per = None
        if with_events:
            per = {"force": statistics.mean(e[0].elapsed_time(e[1]) for e in evs),
                   "links": statistics.mean(e[1].elapsed_time(e[2]) for e in evs)}
        S_val = float(S.item())
        del U, mom, force, S, ws
        torch.cuda.empty_cache()
        return ms, per, n_launch, S_val

    def max_over_ranks(x: float) -> float:
        return ctx.max_over_ranks(x, dev)

    # headline: FP32
    with ClockSampler(local) as clk:
        ms, per, n_launch, S32 = timed("f32", args.steps, args.warmup, True)
    ms = max_over_ranks(ms)
    clocks = clk.summary()
    value = weak_scaling_value(nlinks, world, args.steps, ms)
    # FP64 beside it (fewer steps: the FP64 pipe is narrow on this part)
    k64 = max(2, min(args.steps, 5))
    ms64, per64, _, S64 = timed("f64", k64, max(3, min(args.warmup, 3)), True)
    ms64 = max_over_ranks(ms64)

    # end to end through the public API with host buffers: every step's links
    # and momenta are copied from pinned host memory, and the step's results
    # -- the updated links, the updated momenta and the action -- are copied
    # back to pinned host memory.  As a user of the API would pipeline it,
    # three device buffer sets rotate: while step k computes (compute
    # stream), step k+1's inputs are copied in (input stream) and step k-1's
    # results are copied out (output stream).
    lat, U0, mom0, force, S0, ws = make("f32")
    U_host = U0.detach().to("cpu").pin_memory()
    mom_host = mom0.detach().to("cpu").pin_memory()
    U_out = torch.empty_like(U_host).pin_memory()
    mom_out = torch.empty_like(mom_host).pin_memory()
    K_e2e = max(3, args.steps)
    S_host = torch.empty(K_e2e, dtype=torch.float64).pin_memory()
    h2d = U_host.numel() * U_host.element_size() + mom_host.numel() * mom_host.element_size()
    d2h = h2d + 8
    NB = 3
    Ub = [U0] + [torch.empty_like(U0) for _ in range(NB - 1)]
    mb = [mom0] + [torch.empty_like(mom0) for _ in range(NB - 1)]
    Sb = [S0] + [torch.empty_like(S0) for _ in range(NB - 1)]
    in_stream, out_stream = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in range(NB)]   # inputs of buffer b on the device
    computed = [torch.cuda.Event() for _ in range(NB)]  # step on buffer b done
    drained = [torch.cuda.Event() for _ in range(NB)]  # results of buffer b on the host

    def put(b, used):
        if used[b]:
            in_stream.wait_event(drained[b])
        with torch.cuda.stream(in_stream):
            Ub[b].copy_(U_host, non_blocking=True)
            mb[b].copy_(mom_host, non_blocking=True)
            copied[b].record(in_stream)

    def e2e_run(K):
        used = [False] * NB
        put(0, used)
        for k in range(K):
            b = k % NB
            if k + 1 < K:
                put((k + 1) % NB, used)
            stream.wait_event(copied[b])
            step(lat, Ub[b], mb[b], force, Sb[b], ws)
            computed[b].record(stream)
            out_stream.wait_event(computed[b])
            with torch.cuda.stream(out_stream):
                U_out.copy_(Ub[b], non_blocking=True)
                mom_out.copy_(mb[b], non_blocking=True)
                S_host[k].copy_(Sb[b], non_blocking=True)
                drained[b].record(out_stream)
            used[b] = True
        stream.wait_stream(out_stream)

    e2e_run(2)
    torch.cuda.synchronize(dev)
    barrier()
    e_start, e_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    in_stream.wait_event(e_start)
    out_stream.wait_event(e_start)
    e2e_run(K_e2e)
    e_stop.record(stream)
    torch.cuda.synchronize(dev)
    assert all(np.isfinite(S_host.numpy())), "non-finite action in the end-to-end steps"
    assert bool(torch.isfinite(U_out).all()) and bool(torch.isfinite(mom_out).all())
    e_ms = max_over_ranks(e_start.elapsed_time(e_stop))
    del Ub, mb, Sb, U0, mom0, force, S0, ws
    torch.cuda.empty_cache()
    e2e_value = weak_scaling_value(nlinks, world, K_e2e, e_ms)

    # dH of one Omelyan trajectory (tau 0.5, dt 0.05) in FP32 and in FP64
    # from the same state: the synthetic start thermalised by FP32
    # trajectories, then the same links and momenta in both precisions (FP32
    # values promoted exactly); H = K + S in FP64 in both, so the difference
    # of the two dH is the error of the FP32 arithmetic alone
    from paper_1808_02281_gb300 import hmc
    recs = list(hmc.same_start_study(dims, 0.5, [0.05], "omelyan", seed, n_therm=DH_THERM,
                                     therm_tau=0.5, therm_dt=0.025, sigma=w["sigma"],
                                     u0=w["u0"], beta=w["beta"]))
    therm = [r for r in recs if r["phase"] == "thermalise"]
    study = [r for r in recs if r["phase"] == "study"][0]
    dh = {"integrator": "omelyan", "tau": 0.5, "dt": 0.05, "dims": list(dims),
          "start": f"w ~ N(0, {w['sigma']}^2) links thermalised by {DH_THERM} FP32 trajectories "
                   "(tau 0.5, dt 0.025, momentum refresh, no accept/reject), reunitarised in "
                   "FP64; then the same values in FP32 and FP64",
          "thermalise_action": [r["action"] for r in therm],
          "f32": study["dH_f32"], "f64": study["dH_f64"], "abs_err_f32": study["abs_diff"],
          "f32_with_f32_action": study["dH_f32_f32action"], "H0": study["H0"],
          "same_H0": study["H0_equal"],
          "seconds_f32": study["seconds_f32"], "seconds_f64": study["seconds_f64"]}
    torch.cuda.empty_cache()
    # the same FP32 trajectory captured as one CUDA graph, replayed
    st = hmc.initial_state(dims, "f32", w["sigma"], w["u0"], w["beta"], seed)
    g_traj = hmc.GraphTrajectory(st, 0.05, 10, "omelyan")
    g_traj.replay()
    torch.cuda.synchronize(dev)
    t_start, t_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    g_traj.replay()
    t_stop.record(stream)
    torch.cuda.synchronize(dev)
    dh["trajectory_graph_ms"] = t_start.elapsed_time(t_stop)
    t_start.record(stream)
    hmc.omelyan(st, 0.05, 10)
    t_stop.record(stream)
    torch.cuda.synchronize(dev)
    dh["trajectory_eager_ms"] = t_start.elapsed_time(t_stop)
    del st, g_traj
    torch.cuda.empty_cache()

    # uneven-volume batch: 4 each of 8^4, 12^3x24, 16^3x32, 24^3x48 (FP32)
    bs = hmc.initial_batch(synth.BATCH_DIMS, "f32", w["sigma"], w["u0"], w["beta"], seed)
    nl_batch = sum(4 * synth.volume(d) for d in bs.dims)
    actions = torch.empty(len(bs.dims), dtype=torch.float64, device=dev)

    def batch_step():
        lqcd.md_force_step_batched(bs.params, bs.dims, bs.links, mom=bs.mom, dt=DT,
                                   actions=actions, workspace=bs.workspace)
        lqcd.md_update_links_batched(bs.params, bs.dims, bs.links, bs.mom, DT)

    def single_steps():
        for c, d in enumerate(bs.dims):
            lat_c = bs.params.with_(dims=d)
            lqcd.md_force_step(lat_c, bs.links[c], mom=bs.mom[c], dt=DT, action=actions[c],
                               workspace=bs.workspace)
            lqcd.md_update_links(lat_c, bs.links[c], bs.mom[c], DT)

    def time_it(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        for _ in range(reps):
            fn()
        b_.record(stream)
        torch.cuda.synchronize(dev)
        return a_.elapsed_time(b_) / reps

    ms_batched = time_it(batch_step, 10)
    ms_single = time_it(single_steps, 10)
    g_batch = hmc.GraphBatchTrajectory(bs, DT, 20, "leapfrog")
    ms_graph = time_it(g_batch.replay, 3)
    ms_eager = time_it(lambda: hmc.batch_leapfrog(bs, DT, 20), 3)
    batch = {"lattices": len(bs.dims), "links": nl_batch,
             "step_ms_batched": ms_batched, "step_ms_per_lattice_calls": ms_single,
             "glinks_batched": nl_batch / (ms_batched / 1e3) / 1e9,
             "glinks_per_lattice_calls": nl_batch / (ms_single / 1e3) / 1e9,
             "trajectory": "leapfrog, 20 steps, dt 0.05",
             "trajectory_graph_ms": ms_graph, "trajectory_eager_ms": ms_eager}
    del bs, g_batch, actions
    torch.cuda.empty_cache()

    # the device: SM count, L2, and the measured FMA issue rates (FP32, FP64)
    props = torch.cuda.get_device_properties(dev)
    device = {"name": props.name, "sms": props.multi_processor_count,
              "l2_mb": getattr(props, "L2_cache_size", 0) / 2**20,
              "fma_tflops_f32": lqcd.measure_fma_rate("f32", device=dev),
              "fma_tflops_f64": lqcd.measure_fma_rate("f64", device=dev),
              "fma_note": "measured: every SM filled with independent FMA chains (lqcd_measure_fma_rate)"}

    # Wilson fermion force at the same lattice (Sec. III): Y = D X with the
    # hopping operator (kappa 0.1315, no clover term), then the hopping-term
    # force with the momentum step fused; each kernel timed alone with L2
    # flushed (a 256 MB write) between repetitions
    hbm_peak, peak_kind = _peaks()
    wilson = {"kappa": WILSON_KAPPA, "workload": WORKLOAD,
              "x": "Gaussian spinor, re/im ~ N(0, 1)", "peak_gbs": hbm_peak, "peak_kind": peak_kind}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def kernel_ms(fn, reps):
        for _ in range(3):
            fn()
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            fn()
            b_.record(stream)
            torch.cuda.synchronize(dev)
            tot += a_.elapsed_time(b_)
        return tot / reps

    for prec in ("f32", "f64"):
        lat = lqcd.Lattice(dims, prec)
        real = 4 if prec == "f32" else 8
        U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, omega_np, device=dev))
        X = lqcd.spinor_to_device(lat, synth.spinor(dims, 11 + seed), device=dev)
        Y = lqcd.empty_spinor(lat, dev)
        pm = lqcd.algebra_to_device(lat, p_np, device=dev)
        reps = 20 if prec == "f32" else 5
        ms_d = kernel_ms(lambda: lqcd.wilson_dslash(lat, U, X, 1.0, -WILSON_KAPPA, out=Y), reps)
        ms_f = kernel_ms(lambda: lqcd.wilson_hopping_force(lat, U, X, Y, coef=WILSON_KAPPA,
                                                          mom=pm, dt=DT), reps)
        gb_d = WILSON_REALS_PER_SITE_DSLASH * real * V / (ms_d / 1e3) / 1e9
        gb_f = WILSON_REALS_PER_LINK_FORCE * real * nlinks / (ms_f / 1e3) / 1e9
        wilson[prec] = {"dslash_ms": ms_d, "dslash_gbs": gb_d, "dslash_frac": gb_d / hbm_peak,
                        "force_ms": ms_f, "force_gbs": gb_f, "force_frac": gb_f / hbm_peak,
                        "step_ms": ms_d + ms_f,
                        "step_glinks": nlinks / ((ms_d + ms_f) / 1e3) / 1e9}
        del U, X, Y, pm
        torch.cuda.empty_cache()
    del flush
    torch.cuda.empty_cache()

    if rank != 0:
        ctx.close()
        return 0

    force_ms = per["force"]
    achieved_tflops = FLOP_PER_LINK_FORCE * nlinks / (force_ms / 1e3) / 1e12
    executed_tflops = EXECUTED_FLOP_PER_LINK_FORCE * nlinks / (force_ms / 1e3) / 1e12
    roofline = {
        "bound": "alu", "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": achieved_tflops / FP32_PEAK_TFLOPS, "traffic": _recorded_traffic(),
        "kernel": "force: staple_fields<float> + force_from_staples<float, true> + finish_sum "
                  "(one lqcd_md_force_step call, momentum step and action fused)",
        "units_per_launch": nlinks,
        "algorithmic_flop_per_unit": FLOP_PER_LINK_FORCE,
        "executed_flop_per_unit": EXECUTED_FLOP_PER_LINK_FORCE,
        "executed_achieved": executed_tflops,
        "executed_frac": executed_tflops / FP32_PEAK_TFLOPS,
        "algorithmic_bytes_per_unit": BYTES_PER_LINK_FORCE["f32"],
        "peak_note": "FP32 pipe: 152 SMs x 128 lanes x 2 flop x 2.070 GHz (unit counts and "
                     "maximum clock); 'achieved'/'frac' count the literal 180-product "
                     "algorithm's flops, 'executed_*' the flops the staple-field force "
                     "executes (63 SU(3) products per link): executed_frac is the FP32-pipe "
                     "utilisation",
        "hbm_frac_of_" + peak_kind: BYTES_PER_LINK_FORCE["f32"] * nlinks / (force_ms / 1e3) / 1e9
        / hbm_peak,
    }
    streaming = {
        "md_update_links": {
            "gbs": BYTES_LINK_UPDATE["f32"] * nlinks / (per["links"] / 1e3) / 1e9,
            "ms": per["links"]},
        "peak_gbs": hbm_peak, "peak_kind": peak_kind,
    }
    streaming["md_update_links"]["frac"] = streaming["md_update_links"]["gbs"] / hbm_peak
    cpu = None
    if world == 1 or rank == 0:
        rate1, secs1 = oracle_step_rate(steps=2)
        reps = OracleReplicas()
        try:
            rate_all, secs_all = reps.step(3)
        finally:
            reps.close()
        cpu = {"value": rate_all / 1e9, "unit": "Glink/s", "cores": reps.workers, "kind": "oracle",
               "sample": f"3 oracle steps (force, momentum step, link step, action) of a "
                         f"{'x'.join(map(str, CPU_SAMPLE_DIMS))} lattice drawn like the "
                         f"{WORKLOAD} workload on each of {reps.workers} host cores (one "
                         f"independent single-threaded replica per core, spawned processes), "
                         f"{secs_all:.1f} s",
               "single_core_value": rate1 / 1e9,
               "single_core_sample": f"2 steps on one core, {secs1:.1f} s"}
    out = {
        "metric": METRIC, "value": value, "unit": "Glink/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "dims": list(dims), "links": nlinks,
                   "precision": "f32 links, staples and accumulation; f64 action sum",
                   "step": "force with fused momentum step and action, then link step",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2 (403 MB links, 268 MB momenta, 268 MB force)"},
        "autotune": tuned,
        "force_glinks": nlinks / (force_ms / 1e3) / 1e9,
        "force_ms": force_ms,
        "f64": {"value": weak_scaling_value(nlinks, world, k64, ms64), "unit": "Glink/s",
                "ms_per_step": ms64 / k64, "force_ms": per64["force"],
                "force_glinks": nlinks / (per64["force"] / 1e3) / 1e9, "steps": k64},
        "action_f32": S32, "action_f64": S64,
        "dH": dh,
        "batch": batch,
        "wilson": wilson,
        "device": device,
        "roofline": roofline,
        "streaming": streaming,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "Glink/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": K_e2e,
                "results_copied_back": "updated links and momenta, and the action",
                "pipelining": "three device buffer sets: step k+1's inputs copied in and step "
                              "k-1's results copied out on two copy streams during step k"},
        "gpu_launches": n_launch,
        "clocks": clocks,
    }
    print(json.dumps(out))
    ctx.close()
    return 0


def _named_or_explicit_workload(name):
    """A workload of synth.WORKLOADS by name, or explicit extents "AxBxCxD"
    drawn like the 32^3x64 workload (sigma 0.3, u0 0.87, beta 6, seed 0)."""
    from paper_1808_02281_gb300 import synth

    if name in synth.WORKLOADS:
        return synth.WORKLOADS[name]
    dims = tuple(int(d) for d in name.lower().split("x"))
    if len(dims) != 4 or min(dims) < 1:
        raise SystemExit(f"unknown workload {name!r}: a name of synth.WORKLOADS or AxBxCxD")
    return dict(dims=dims, sigma=0.3, u0=0.87, beta=6.0, seed=0)


def run_profile_force(args):
    """W + K FP32 force calls (staple planes, force pass with the fused
    momentum step and action) on one workload, for profiler captures of a
    small case; prints the mean time of the K timed calls."""
    import torch

    from paper_1808_02281_gb300 import build as B
    from paper_1808_02281_gb300 import lqcd, synth

    B.build()
    w = _named_or_explicit_workload(args.profile_force)
    dims = w["dims"]
    lat = lqcd.Lattice.symanzik(dims, w["beta"], w["u0"], "f32")
    U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(dims, w["sigma"], w["seed"])))
    mom = lqcd.algebra_to_device(lat, synth.momenta(dims, seed=1000 + w["seed"]))
    S = torch.empty((), dtype=torch.float64, device="cuda")
    ws = lqcd.make_workspace(lat)
    if args.force_variant >= 0:
        lqcd.set_force_variant(lat, args.force_variant)
    for _ in range(args.warmup):
        lqcd.md_force_step(lat, U, mom=mom, dt=DT, action=S, workspace=ws)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        lqcd.md_force_step(lat, U, mom=mom, dt=DT, action=S, workspace=ws)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"profile_force": args.profile_force, "variant": lqcd.get_force_variant(lat),
                      "links": 4 * lat.V, "force_ms": ms, "action": float(S.item())}))
    return 0


def run_profile_wilson(args):
    """W + K launches each of the FP32 Wilson hopping operator (Y = X -
    kappa calD X) and of the hopping-term force with the fused momentum step
    on one workload, for profiler captures; prints their mean times."""
    import torch

    from paper_1808_02281_gb300 import build as B
    from paper_1808_02281_gb300 import lqcd, synth

    B.build()
    w = synth.WORKLOADS[args.profile_wilson]
    dims = w["dims"]
    lat = lqcd.Lattice(dims, "f32")
    U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(dims, w["sigma"], w["seed"])))
    X = lqcd.spinor_to_device(lat, synth.spinor(dims, 11))
    Y = lqcd.empty_spinor(lat)
    pm = lqcd.algebra_to_device(lat, synth.momenta(dims, seed=1000 + w["seed"]))
    out = {"profile_wilson": args.profile_wilson, "sites": lat.V}
    for name, fn in (("dslash", lambda: lqcd.wilson_dslash(lat, U, X, 1.0, -WILSON_KAPPA, out=Y)),
                     ("force", lambda: lqcd.wilson_hopping_force(lat, U, X, Y, coef=WILSON_KAPPA,
                                                                mom=pm, dt=DT))):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            fn()
        b.record()
        torch.cuda.synchronize()
        out[name + "_ms"] = a.elapsed_time(b) / args.steps
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--force-variant", type=int, default=-1,
                    help="fix the staple-field force schedule (0..8) instead of autotuning it "
                         "at set-up; -1 (default) autotunes")
    ap.add_argument("--profile-force", default=None, metavar="WORKLOAD",
                    help="only time FP32 force calls on this workload, a name of "
                         "synth.WORKLOADS or extents AxBxCxD (profiler captures)")
    ap.add_argument("--profile-wilson", default=None, metavar="WORKLOAD",
                    help="only time the FP32 Wilson kernels on this workload (profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_force:
        return run_profile_force(args)
    if args.profile_wilson:
        return run_profile_wilson(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
