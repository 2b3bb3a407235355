"""Benchmark: active-particle forces/s and interactions/s of the tree-gravity
force path on one GB300 (or N replicas under torchrun).

Workload (headline): Hernquist halo, N = 2^20 (M = G = a = 1, r <= 100 a),
softening h = 0.005, leaf bucket 16, all particles active.  One step is one
local time step of the paper's gravity path: tree construction from scratch
(keys, sort, nodes, FP64 monopoles) followed by the relative-criterion walk
(alpha = 0.0025) against |a| of the previous step.  Before timing, the first
force is computed with the geometric criterion (theta = 0.5), as the paper
prescribes for the very first force evaluation.

The periodic TreePM box (128^3 Zel'dovich lattice, PM 256^3) is measured
beside it and reported under "periodic_treepm".

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import collections
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "active-particle forces/s and interactions/s at p99 rel. force err <=5e-3; p50/p99 latency"
FLOPS_PER_INTERACTION = 20  # monopole pair term with potential, FP32: offset 3, r^2 5, rsqrt 1, products 3, acc 6, pot 1

# From the ncu capture of one k_walk_group launch of the headline step (its
# summary is under profiles/), valid only for the walk source it was taken
# from: DRAM bytes (read + write) and the pipe activity of that launch (the
# FMA pipe's busy cycles, counting the two-wide FP32 instructions, and the
# ALU pipe's instructions, both against their peaks)
WALK_TRAFFIC = {"bytes": 87.394048e6 + 14.233344e6,
                "fma_pipe_active": 0.43799987, "alu_pipe_inst": 0.54087898,
                "walk_cu_sha256": "b5647f3b414cb0904d1dbc84cd4b2a472a79d8c57a0d2e47584f9ecc2cc3b967"}


def walk_capture():
    """The capture's figures if walk.cu is the captured source, else None."""
    import hashlib

    path = os.path.join(ROOT, "paper_1909_04667_gb300", "csrc", "walk.cu")
    try:
        digest = hashlib.sha256(open(path, "rb").read()).hexdigest()
    except OSError:
        return None
    return WALK_TRAFFIC if digest == WALK_TRAFFIC["walk_cu_sha256"] else None

# ------------------------------------------------------------------ configs
HERNQUIST = dict(n=1 << 20, seed=W.CONFIG_SEEDS[2], h=0.005, G=1.0, bucket=16, theta=0.5, alpha=0.0025)
PLUMMER = dict(n=8192, h=0.01, G=1.0, bucket=8, theta=0.7)
SERVING = dict(seed=W.CONFIG_SEEDS[5], budget_gb=60, n_requests=10000, warmup_requests=4000, rate=200.0,
               load_factors=(1, 8), nmin=1 << 12, nmax=1 << 20, overcommit=1.5, bytes_per_particle=118,
               round_ids=1 << 21, accuracy_every=1000, accuracy_targets=1024, aold_cache_gb=2)
TIMEBINS = dict(nbins=8, seed=W.CONFIG_SEEDS[4], req_lo=64, req_hi=65536)
HIERARCHY = dict(nbins=8, dt_tick=0.005, c_grav=0.025)
ISOLATED = dict(pm_n=64, asmth=2.5, rcut=4.5)
ZELDOVICH = dict(ngrid=128, seed=W.CONFIG_SEEDS[3], pm_n=256, asmth=1.25, rcut=4.5, G=1.0, bucket=8, theta=0.5,
                 alpha=0.005)


def hernquist_inputs():
    pos, mass = W.hernquist(HERNQUIST["n"], HERNQUIST["seed"])
    return pos, mass


def zeldovich_inputs():
    return W.zeldovich(ZELDOVICH["ngrid"], ZELDOVICH["seed"])


def zeldovich_h():
    return (1.0 / ZELDOVICH["ngrid"]) / 40.0


def root_shift(step: int, base: int):
    return tuple(float(v) for v in W.root_shift(base * 1000 + step))


# ------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi clock / throttle samples, each stamped with its arrival time;
    started before the warm-up (nvidia-smi takes longer to start than a short
    timed region lasts), summarised over the samples inside the timed window
    (`window(t0, t1)`, host perf_counter times), else the nearest one."""

    def __init__(self, device: int):
        self.device = device
        self.samples = []
        self.t0 = self.t1 = None
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + q,
                                           "--format=csv,noheader,nounits", "-lms", "20"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self._proc = None
        return self

    def _read(self):
        for line in self._proc.stdout:
            self.samples.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def window(self, t0, t1):
        self.t0, self.t1 = t0, t1

    def __exit__(self, *a):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        picked = self.samples
        where = "whole run"
        if self.t0 is not None:
            inside = [x for x in self.samples if self.t0 <= x[0] <= self.t1 + 0.03]  # + pipe latency
            if inside:
                picked, where = inside, "timed region"
            else:
                mid = 0.5 * (self.t0 + self.t1)
                picked, where = [min(self.samples, key=lambda x: abs(x[0] - mid))], "nearest to the timed region"
        samples = [x[1] for x in picked]
        sm = [float(s[0]) for s in samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in samples for i in range(4)
                          if len(s) > 4 + i and s[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(samples), "sampled": where}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def l2_flush(buf):
    buf.zero_()


EXACT_SUMS = os.path.join(ROOT, "tests", "golden", "exact_sums.npz")
EXACT_DESC = {
    "hernquist": "FP64 softened direct sum (oracle), 4096 seeded targets",
    "zeldovich": "FP64 Ewald sum with neutralising background (oracle), 2048 seeded targets",
    "two_species": "FP64 direct sum with the larger of the two supports (oracle), 4096 seeded targets",
    "plummer": "FP64 softened direct sum (oracle), all 8192 particles",
}


def exact_sums():
    """The stored exact forces (tests/golden/make_exact_sums.py writes them
    with the FP64 oracle), or None."""
    try:
        with np.load(EXACT_SUMS) as f:
            return {k: f[k] for k in f.files}
    except Exception:
        return None


def error_stats(acc, exact) -> dict:
    """Relative force error |a - a_exact| / |a_exact| over the targets."""
    e = np.linalg.norm(np.asarray(acc, np.float64) - exact, axis=1) / np.linalg.norm(exact, axis=1)
    return {"p50": float(np.percentile(e, 50)), "p90": float(np.percentile(e, 90)),
            "p99": float(np.percentile(e, 99)), "max": float(e.max()), "targets": int(len(e)),
            "p99_within_5e-3": bool(np.percentile(e, 99) <= 5e-3)}


def accuracy_at(acc_dev, name) -> dict:
    """Accuracy of forces computed for all particles (device tensor, caller's
    order) against the stored exact sums of workload `name`."""
    ex = exact_sums()
    if ex is None or name + "_targets" not in ex:
        return {"unavailable": "stored exact sums missing (run tests/golden/make_exact_sums.py)"}
    tg = ex[name + "_targets"].astype(np.int64)
    import torch

    got = acc_dev[torch.from_numpy(tg).to(acc_dev.device)].cpu().numpy()
    return dict(error_stats(got, ex[name + "_acc"]), reference=EXACT_DESC[name])


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world):
    import torch

    import paper_1909_04667_gb300 as tpm
    from paper_1909_04667_gb300 import shard

    dev = torch.device("cuda", 0 if world == 1 else int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    props = torch.cuda.get_device_properties(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = tpm.Context(dev.index)
    cfg = HERNQUIST
    pos, mass = hernquist_inputs()
    n = len(pos)
    pos_d = torch.from_numpy(pos).to(dev)
    mass_d = torch.from_numpy(mass).to(dev)
    bp = lambda step: tpm.BuildParams(G=cfg["G"], h=cfg["h"], shift=root_shift(step, 2), leaf_bucket=cfg["bucket"])
    fp_bh = tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"])
    fp_rel = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MiB > 129 MB L2

    # first force: geometric criterion
    s = ctx.build_tree(pos_d, mass_d, bp(0))
    acc, pot, nint = s.compute_forces(fp=fp_bh)
    s.sync_status()  # the walk's device status (stack capacity) before timing anything
    s.release()
    a_old = torch.linalg.vector_norm(acc, dim=1).contiguous()
    acc_buf = torch.empty((n, 3), dtype=torch.float32, device=dev)
    pot_buf = torch.empty(n, dtype=torch.float32, device=dev)
    nint_buf = torch.empty(n, dtype=torch.int32, device=dev)

    def step(k, ev=None):
        if ev:
            ev[0].record(stream)
        sy = ctx.build_tree(pos_d, mass_d, bp(k))
        if ev:
            ev[1].record(stream)
        sy.compute_forces(a_old=a_old, fp=fp_rel, acc=acc_buf, pot=pot_buf, n_int=nint_buf)
        if ev:
            ev[2].record(stream)
        sy.release()

    clk = ClockSampler(dev.index).__enter__()
    t_wait = time.perf_counter()
    while not clk.samples and time.perf_counter() - t_wait < 5.0:  # the sampler is running
        time.sleep(0.01)
    for k in range(args.warmup):
        step(1 + k)
        a_old.copy_(torch.linalg.vector_norm(acc_buf, dim=1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_build, t_walk, t_step = [], [], []
    k0, c0 = tpm.launch_counts()
    t_host0 = time.perf_counter()
    for k in range(args.steps):
        l2_flush(flush)
        step(1000 + k, evs[k])
    torch.cuda.synchronize()
    clk.window(t_host0, time.perf_counter())
    clk.__exit__()
    k1, c1 = tpm.launch_counts()
    for e in evs:
        t_build.append(e[0].elapsed_time(e[1]))
        t_walk.append(e[1].elapsed_time(e[2]))
        t_step.append(e[0].elapsed_time(e[2]))
    if world > 1:
        torch.distributed.barrier()
    ms = shard.max_over_ranks(sum(t_step) / len(t_step), device=dev)
    interactions = int(nint_buf.to(torch.int64).sum().item())
    walk_ms = statistics.mean(t_walk)
    build_ms = statistics.mean(t_build)
    # accuracy of the last timed step against the exact sum; the oracle walk's
    # floor on the same targets (same tree shift and |a_old|) is added by the
    # cpu_baseline leg
    accuracy = accuracy_at(acc_buf, "hernquist")
    ex = exact_sums()
    floor_ctx = None
    if ex is not None:
        tg = ex["hernquist_targets"].astype(np.int64)
        floor_ctx = {"shift": root_shift(1000 + args.steps - 1, 2), "targets": tg,
                     "a_old": a_old[torch.from_numpy(tg).to(dev)].cpu().numpy()}

    # ---------------- FP64 conservation diagnostics of one relative step (untimed)
    sy = ctx.build_tree(pos_d, mass_d, bp(9999))
    sy.compute_forces(a_old=a_old, fp=fp_rel, acc=acc_buf, pot=pot_buf, n_int=nint_buf)
    dg = sy.diagnostics(acc_buf, pot_buf)
    sy.release()
    diagnostics = {"total_force_over_scale": float(np.linalg.norm(dg["total_force"]) / dg["force_scale"]),
                   "potential_energy": dg["potential_energy"],
                   "note": "FP64 on the GPU: |sum m a| / sum m |a| (zero for exactly symmetric forces) and "
                           "1/2 sum m phi of one relative-criterion step"}

    # ---------------- end to end through the C ABI with host buffers
    pos_h = torch.from_numpy(pos).pin_memory()
    mass_h = torch.from_numpy(mass).pin_memory()
    aold_h = a_old.cpu().pin_memory()
    acc_h = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    pot_h = torch.empty(n, dtype=torch.float32).pin_memory()
    e2e_ms = [float("nan")]
    e2e_warm = 0 if args.no_e2e else max(3, args.warmup)
    for k in range(0 if args.no_e2e else e2e_warm + max(3, min(args.steps, 10))):
        if k == e2e_warm:
            e2e_ms = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sy = ctx.build_tree(pos_h, mass_h, bp(5000 + k))
        sy.compute_forces(a_old=aold_h, fp=fp_rel, acc=acc_h, pot=pot_h, want_nint=False)
        sy.release()
        if k >= e2e_warm:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = shard.max_over_ranks(statistics.median(e2e_ms), device=dev)
    h2d = pos.nbytes + mass.nbytes + aold_h.numel() * 4
    d2h = acc_h.numel() * 4 + pot_h.numel() * 4

    # the other workloads are single-GPU measurements: taken at N = 1 only (at
    # N > 1 every rank would repeat them while all N GPUs are held)
    if world > 1:
        args.no_periodic = args.no_batching = args.no_hierarchy = args.no_isolated = True
        args.no_ewald = args.no_species = args.no_serving = True
    # ---------------- periodic TreePM box (128^3, PM 256^3)
    periodic = None if args.no_periodic else run_periodic(ctx, tpm, torch, dev, stream, flush,
                                                          max(2, min(args.steps, 5)))
    periodic_ik = None if args.no_periodic else run_periodic(ctx, tpm, torch, dev, stream, flush,
                                                             max(2, min(args.steps, 5)), grad="ik")
    batching = None if args.no_batching else run_batching(ctx, tpm, torch, dev, stream, pos_d, mass_d)
    hierarchy = None if args.no_hierarchy else run_hierarchy(ctx, tpm, torch, dev, stream)
    isolated = None if args.no_isolated else run_isolated(ctx, tpm, torch, dev, stream, flush, pos_d, mass_d,
                                                          max(2, min(args.steps, 5)))
    ewald = None if args.no_ewald else run_ewald(ctx, tpm, torch, dev, stream, flush, max(2, min(args.steps, 3)))
    species = None if args.no_species else run_two_species(ctx, tpm, torch, dev, stream, flush,
                                                           max(2, min(args.steps, 5)))
    plummer = None if world > 1 else run_plummer(ctx, tpm, torch, dev, stream, flush, max(3, min(args.steps, 10)))

    ctx.close()
    serving = None if args.no_serving else run_serving(tpm, torch, dev)
    pk, pk_kind = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    cap = walk_capture()
    achieved = interactions * FLOPS_PER_INTERACTION / (walk_ms * 1e-3) / 1e12
    n_levels = None
    clocks = clk.summary()
    value = world * n / (ms * 1e-3)
    return dict(
        metric=METRIC, value=value, unit="forces/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic",
        config=headline_config(world),
        interactions_per_s=world * interactions / (walk_ms * 1e-3),
        interactions_per_particle=interactions / n,
        build_ms=build_ms, walk_ms=walk_ms,
        e2e={"value": world * n / (e2e_ms * 1e-3), "unit": "forces/s", "ms_per_step": e2e_ms,
             "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        roofline={"bound": "alu", "kernel": "k_walk_group (relative criterion)", "achieved": achieved,
                  "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                  "traffic": cap["bytes"] if cap else None,
                  "fma_pipe_active_ncu": cap["fma_pipe_active"] if cap else None,
                  "alu_pipe_inst_ncu": cap["alu_pipe_inst"] if cap else None,
                  "frac_at_run_clock": (achieved / (fp32_peak * clocks["sm_mhz"] / sm_max)
                                        if clocks.get("sm_mhz") else None),
                  "peak_kind": "FP32 CUDA-core peak = SMs x 128 x 2 x %.0f MHz (%s sm_max)" % (sm_max, pk_kind),
                  "algorithmic": "%d flops x %d useful interactions per launch" % (FLOPS_PER_INTERACTION,
                                                                                    interactions)},
        gpu_launches=int(k1 - k0),
        accuracy=accuracy,
        _floor_ctx=floor_ctx,
        diagnostics=diagnostics,
        cub_calls=int(c1 - c0),
        clocks=clocks,
        periodic_treepm=periodic,
        periodic_treepm_spectral=periodic_ik,
        batching=batching,
        hierarchy=hierarchy,
        isolated_treepm=isolated,
        periodic_ewald_tree=ewald,
        two_species_softening=species,
        plummer_8192=plummer,
        serving=serving,
    )


def timebin_requests(perm, bins, seed):
    """Requests of one 2^(nbins-1)-substep cycle: each substep's active set
    (bins >= the substep's lowest active bin), in key order, cut into
    log-uniform request sizes.  Returns (ids, offsets, substep of each request)."""
    nb = TIMEBINS["nbins"]
    keyed_bins = bins[perm]
    ids, sizes, subs = [], [], []
    for step in range(1 << (nb - 1)):
        act = perm[keyed_bins >= W.substep_active_bins(step, nb)]
        sz = W.request_sizes(len(act), seed + step, TIMEBINS["req_lo"], TIMEBINS["req_hi"])
        ids.append(act)
        sizes.append(sz)
        subs += [step] * len(sz)
    ids = np.concatenate(ids).astype(np.int32)
    off = np.concatenate([[0], np.cumsum(np.concatenate(sizes))])
    return ids, off, np.asarray(subs)


def run_hierarchy(ctx, tpm, torch, dev, stream):
    """Hierarchical KDK time stepping of the Hernquist 2^20 set (cold start):
    bins from the step criterion sqrt(2 C_grav eps / |a|), one tree build per
    tick for the particles due, one whole cycle of 2^(nbins-1) ticks timed
    after one warm-up cycle."""
    from paper_1909_04667_gb300.integrate import Integrator

    cfg, hc = HERNQUIST, HIERARCHY
    pos, mass = hernquist_inputs()
    sp = tpm.StepParams(dt_tick=hc["dt_tick"], nbins=hc["nbins"], c_grav=hc["c_grav"], eps=cfg["h"] / 2.8)
    bp = tpm.BuildParams(G=cfg["G"], h=cfg["h"], shift=root_shift(0, 5), leaf_bucket=cfg["bucket"])
    integ = Integrator(ctx, pos, np.zeros_like(pos), mass, bp, sp, tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"]),
                       tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"]),
                       shift=lambda t: root_shift(t, 5))
    integ.run_cycle()
    hist = np.bincount(integ.bins.cpu().numpy().astype(np.int64), minlength=hc["nbins"])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0, _ = tpm.launch_counts()
    e0.record(stream)
    forces = integ.run_cycle()
    e1.record(stream)
    torch.cuda.synchronize()
    k1, _ = tpm.launch_counts()
    ms = e0.elapsed_time(e1)
    ticks = 1 << (hc["nbins"] - 1)
    return {"workload": "hernquist_n2^20_kdk_%dbins_dt%g_Cgrav%g" % (hc["nbins"], hc["dt_tick"], hc["c_grav"]),
            "ms_per_cycle": ms, "ticks_per_cycle": ticks, "forces_per_cycle": int(forces),
            "forces_per_s": forces / (ms * 1e-3), "builds_per_cycle": ticks, "bin_occupancy": hist.tolist(),
            "gpu_launches_per_cycle": int(k1 - k0),
            "note": "all particles drift and the tree is rebuilt at every tick; forces for the particles due"}


def run_batching(ctx, tpm, torch, dev, stream, pos_d, mass_d, reps=3):
    """Hierarchical time-step batching on the Hernquist 2^20 set: the requests
    of one 128-substep cycle on one tree.  The autotuner picks the walk group
    size G in {8, 16, 32, 64} and the stack depth for trees of leaf bucket B in
    {1, 4, 8, 16}; at the best B the cycle runs (a) as one compute_forces call
    per request and (b) as one tuned batch captured in a CUDA graph."""
    cfg = HERNQUIST
    n = pos_d.shape[0]
    fp = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"])
    bins = W.timebins(pos_d.cpu().numpy(), TIMEBINS["seed"], TIMEBINS["nbins"])
    sweep, best = {}, None
    for B in (1, 4, 8, 16):
        sy = ctx.build_tree(pos_d, mass_d, tpm.BuildParams(G=cfg["G"], h=cfg["h"], shift=root_shift(7, 4),
                                                           leaf_bucket=B))
        a, _, _ = sy.compute_forces(fp=tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"]))
        a_full = torch.linalg.vector_norm(a, dim=1).contiguous()
        perm = sy.tree_export()["perm"].astype(np.int64)
        ids, off, subs = timebin_requests(perm, bins, TIMEBINS["seed"])
        n_ids, n_req = len(ids), len(off) - 1
        ids_d = torch.from_numpy(ids).to(dev)
        aold = a_full[ids_d.long()].contiguous()
        acc = torch.empty((n_ids, 3), device=dev)
        pot = torch.empty(n_ids, device=dev)
        nint = torch.empty(n_ids, dtype=torch.int32, device=dev)
        plan = ctx.create_plan(n_ids, n_req)
        g_best, ms_tune = plan.autotune([sy] * n_req, off, fp, ids_d, acc, a_old=aold, pot=pot, n_int=nint,
                                        presorted=True, reps=2)
        sweep[B] = {"group_size": g_best, "stack_depth": plan.stack_depth, "ms_per_cycle": ms_tune}
        plan.close()
        if best is None or ms_tune < best[0]:
            if best is not None:
                best[1].release()
            best = (ms_tune, sy, B, ids, off, ids_d, aold, acc, pot, nint, g_best, sweep[B]["stack_depth"])
        else:
            sy.release()
    _, sy, B, ids, off, ids_d, aold, acc, pot, nint, g_best, depth_best = best
    n_ids, n_req = len(ids), len(off) - 1

    # (a) one call per request
    def per_request():
        for r in range(n_req):
            lo, hi = int(off[r]), int(off[r + 1])
            sy.compute_forces(active_ids=ids_d[lo:hi], a_old=aold[lo:hi], fp=fp, acc=acc[lo:hi], pot=pot[lo:hi],
                              n_int=nint[lo:hi])
    per_request()
    torch.cuda.synchronize()
    t_req = []
    for _ in range(reps):
        t0 = time.perf_counter()
        per_request()
        torch.cuda.synchronize()
        t_req.append((time.perf_counter() - t0) * 1e3)
    ref = acc.cpu().numpy().copy()
    # (b) one batch per cycle at the tuned G and depth, in a CUDA graph
    plan = ctx.create_plan(n_ids, n_req)
    plan.group_size = g_best
    plan.stack_depth = depth_best
    systems = [sy] * n_req
    plan.compute_forces_batch(systems, off, fp, ids_d, acc, a_old=aold, pot=pot, n_int=nint, presorted=True)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            plan.compute_forces_batch(systems, off, fp, ids_d, acc, a_old=aold, pot=pot, n_int=nint,
                                      presorted=True)
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    t_b = []
    for _ in range(reps):
        t0 = time.perf_counter()
        graph.replay()
        torch.cuda.synchronize()
        t_b.append((time.perf_counter() - t0) * 1e3)
    plan.sync_status()
    got = acc.cpu().numpy()
    e = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    inter = int(nint.to(torch.int64).sum().item())
    plan.close()
    sy.release()
    ms_req, ms_b = statistics.median(t_req), statistics.median(t_b)
    return {"workload": "hernquist_n2^20_timebins8_cycle128_requests64-65536", "forces_per_cycle": n_ids,
            "requests_per_cycle": n_req, "interactions_per_force": inter / n_ids, "leaf_bucket": B,
            "autotune": {"B%d" % b: v for b, v in sweep.items()},
            "per_request_launches": {"ms_per_cycle": ms_req, "forces_per_s": n_ids / (ms_req * 1e-3)},
            "batched_graph": {"ms_per_cycle": ms_b, "forces_per_s": n_ids / (ms_b * 1e-3), "group_size": g_best,
                              "stack_depth": depth_best,
                              "launch": "one persistent walk per cycle, captured in a CUDA graph"},
            "speedup": ms_req / ms_b, "max_rel_diff_vs_per_request": float(e.max())}


def serving_workload():
    """Catalogue and request stream: systems with N log-uniform in [2^12, 2^20]
    until their resident footprint (~118 B per particle) is overcommit x the
    HBM budget; Poisson arrivals; each request a random system and a random
    window of 1-100% of its particles (the particles are drawn in random
    order, so a window is a uniform random subset)."""
    cfg = SERVING
    budget = int(cfg["budget_gb"] * (1 << 30))
    big = W.serving_catalogue(20000, cfg["seed"], cfg["nmin"], cfg["nmax"])
    cat, footprint = [], 0
    for spec in big:
        if footprint >= cfg["overcommit"] * budget:
            break
        cat.append(spec)
        footprint += spec.n * cfg["bytes_per_particle"]
    rng = np.random.Generator(np.random.PCG64(cfg["seed"] + 1))
    nw = cfg["warmup_requests"]
    arrivals = W.poisson_arrivals(nw + cfg["n_requests"], cfg["rate"], cfg["seed"] + 2)
    arrivals = np.concatenate([np.zeros(nw), arrivals[nw:] - arrivals[nw]])  # the warm-up prefix is not paced
    reqs = []
    for k, t in enumerate(arrivals):
        sid = int(rng.integers(0, len(cat)))
        n = cat[sid].n
        m = max(1, int(n * rng.uniform(0.01, 1.0)))
        off = int(rng.integers(0, n))
        reqs.append((k, sid, ((off + np.arange(m)) % n).astype(np.int32), float(t)))
    return cat, reqs, footprint, budget


def run_serving(tpm, torch, dev):
    """Continuous-batching server vs one call per request, on the same HBM
    admission budget; particles drawn on the device when a system is built."""
    from paper_1909_04667_gb300.serve import ForceServer, ServeRequest, serve_per_request

    cfg = SERVING
    cat, reqs, footprint, budget = serving_workload()

    def source(sid):
        spec = cat[sid]
        pos, mass = spec.particles_on_device(torch, dev)
        return pos, mass, tpm.BuildParams(G=1.0, h=spec.h, shift=tuple(W.root_shift(spec.seed)), leaf_bucket=8)

    nw = cfg["warmup_requests"]

    def make(warm):
        sel = reqs[:nw] if warm else reqs[nw:]
        return [ServeRequest(k, sid, ids, t) for k, sid, ids, t in sel]

    def stats(out, wall):
        lat = np.array([r.latency for r in out]) * 1e3
        forces = sum(len(r.ids) for r in out)
        return {"forces_per_s": forces / wall, "latency_ms_p50": float(np.percentile(lat, 50)),
                "latency_ms_p99": float(np.percentile(lat, 99)), "makespan_s": wall,
                "relative_criterion_share": float(np.mean([r.criterion == tpm.CRIT_RELATIVE for r in out]))}

    # each arm first serves the warm-up prefix untimed until the budget holds a
    # steady-state resident set, then the timed requests at their arrival times:
    # at the stream's rate, then (saturation) the same requests at a multiple
    def paced(factor):
        out = make(False)
        for r in out:
            r.arrival /= factor
        return out

    # accuracy: every accuracy_every-th timed request keeps its first
    # accuracy_targets results in every arm (the exact sums are taken by the
    # cpu_baseline leg)
    every, ntg = cfg["accuracy_every"], cfg["accuracy_targets"]
    sampled = lambda r: r.rid >= nw and (r.rid - nw) % every == 0
    samples = {}

    def keep(arm, out):
        for r in out:
            if sampled(r) and r.acc is not None:
                samples.setdefault(r.rid, {"sid": r.sid, "ids": r.ids[:ntg].copy(), "acc": {}})
                samples[r.rid]["acc"][arm] = r.acc[:ntg].copy()

    res = {}
    ctx = tpm.Context(dev.index, budget_bytes=budget)
    srv = ForceServer(ctx, source, max_round_ids=cfg["round_ids"], max_round_requests=512, policy="adaptive",
                      keep_results=sampled, aold_cache_bytes=cfg["aold_cache_gb"] << 30)
    srv.serve(make(True), realtime=False)
    for f in cfg["load_factors"]:
        b0, e0 = srv.builds, srv.evictions
        t0 = time.perf_counter()
        out = srv.serve(paced(f), realtime=True)
        key = "continuous_batching" if f == 1 else "continuous_batching_x%d" % f
        res[key] = dict(stats(out, time.perf_counter() - t0), builds=srv.builds - b0, evictions=srv.evictions - e0)
        if f == 1:
            keep("continuous_batching", out)
    srv.close()
    for plain in (False, True):
        resident = collections.OrderedDict()
        serve_per_request(ctx, source, make(True), policy="adaptive", realtime=False, keep_results=False,
                          resident=resident, plain_fp32=plain)
        arm = "per_request_plain_fp32" if plain else "per_request"
        for f in cfg["load_factors"]:
            t0 = time.perf_counter()
            out = serve_per_request(ctx, source, paced(f), policy="adaptive", realtime=True, keep_results=sampled,
                                    resident=resident, plain_fp32=plain)
            res[arm if f == 1 else arm + "_x%d" % f] = stats(out, time.perf_counter() - t0)
            if f == 1:
                keep(arm, out)
        for system, _, _ in resident.values():
            system.release()
    # the sampled systems' particles on the host, for the exact sums
    for rid, smp in samples.items():
        pos, mass, bp = source(smp["sid"])
        smp.update(pos=pos.cpu().numpy(), mass=mass.cpu().numpy(), h=bp.h)
    # the first timed requests' systems on the host (at most 12 requests and
    # 2^19 ids in all: a bounded sample), for the oracle's per-request time
    # (cpu_baseline leg)
    cpu_systems, tot = [], 0
    for k, sid, ids, t in reqs[nw:nw + 12]:
        if tot + len(ids) > (1 << 19):
            break
        pos, mass, bp = source(sid)
        cpu_systems.append((pos.cpu().numpy(), mass.cpu().numpy(), bp.h, bp.shift, ids))
        tot += len(ids)
    ctx.close()
    res.update(workload="serving_%d_systems_N2^12-2^20_poisson%dHz_%d_requests_after_%d_budget%dGB" % (
        len(cat), int(cfg["rate"]), cfg["n_requests"], nw, cfg["budget_gb"]), hbm_budget_bytes=budget,
        catalogue_bytes=footprint,
        arms={"continuous_batching": "server: mixed precision, batched rounds, builds overlapping the walks, |a| "
                                     "of evicted systems kept in pinned host memory for the relative criterion",
              "per_request": "one build (if needed), one compute_forces call and one synchronisation per "
                             "request, mixed precision",
              "per_request_plain_fp32": "the same with the plain FP32 form (absolute FP32 coordinates)"},
        _samples=samples, _cpu_systems=cpu_systems)
    return res


def serving_accuracy(samples) -> dict:
    """Per arm: the relative force error of the sampled served requests
    against the FP64 direct sum on their first targets (cpu_baseline leg)."""
    import oracle

    errs = {}
    for rid, smp in sorted(samples.items()):
        ex, _ = oracle.direct(smp["pos"], smp["mass"], smp["ids"].astype(np.uint32), 1.0, smp["h"])
        for arm, acc in smp["acc"].items():
            e = np.linalg.norm(acc.astype(np.float64) - ex, axis=1) / np.linalg.norm(ex, axis=1)
            errs.setdefault(arm, []).append(e)
    out = {}
    for arm, es in errs.items():
        e = np.concatenate(es)
        out[arm] = {"p50": float(np.percentile(e, 50)), "p99": float(np.percentile(e, 99)), "max": float(e.max()),
                    "requests": len(es), "targets": int(len(e)),
                    "p99_within_5e-3": bool(np.percentile(e, 99) <= 5e-3)}
    out["reference"] = "FP64 softened direct sum (oracle) on the first %d ids of every %dth timed request" % (
        SERVING["accuracy_targets"], SERVING["accuracy_every"])
    return out


def run_periodic(ctx, tpm, torch, dev, stream, flush, steps, grad="fd4"):
    """The periodic TreePM box: one step = build + mesh + short-range relative
    walk with interpolation; mesh force by the 4-point difference (`fd4`) or
    the spectral derivative (`ik`)."""
    cfg = ZELDOVICH
    pos, mass = zeldovich_inputs()
    n = len(pos)
    pos_d = torch.from_numpy(pos).to(dev)
    mass_d = torch.from_numpy(mass).to(dev)
    h = zeldovich_h()
    bp = lambda k: tpm.BuildParams(G=cfg["G"], h=h, periodic=True, box=1.0, shift=root_shift(k, 3),
                                   leaf_bucket=cfg["bucket"])
    common = dict(treepm=True, pm_n=cfg["pm_n"], asmth=cfg["asmth"], rcut=cfg["rcut"],
                  pm_grad=tpm.GRAD_IK if grad == "ik" else tpm.GRAD_FD4)
    fp_bh = tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"], **common)
    fp_rel = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"], **common)
    s = ctx.build_tree(pos_d, mass_d, bp(0))
    s.pm_long_range(fp_bh)
    acc, pot, nint = s.compute_forces(fp=fp_bh)
    s.release()
    a_old = torch.linalg.vector_norm(acc, dim=1).contiguous()
    acc_b = torch.empty_like(acc)
    pot_b = torch.empty_like(pot)
    nint_b = torch.empty_like(nint)
    res = []
    for k in range(steps + 2):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        l2_flush(flush)
        ev[0].record(stream)
        sy = ctx.build_tree(pos_d, mass_d, bp(100 + k))
        ev[1].record(stream)
        sy.pm_long_range(fp_rel)
        ev[2].record(stream)
        sy.compute_forces(a_old=a_old, fp=fp_rel, acc=acc_b, pot=pot_b, n_int=nint_b)
        ev[3].record(stream)
        sy.release()
        torch.cuda.synchronize()
        if k >= 2:
            res.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])])
    r = np.array(res).mean(0)
    ms = float(r.sum())
    inter = int(nint_b.to(torch.int64).sum().item())
    return {"workload": "zeldovich_128^3_pm256_%s_relative_alpha0.005" % grad, "value": n / (ms * 1e-3),
            "unit": "forces/s",
            "ms_per_step": ms, "build_ms": float(r[0]), "pm_ms": float(r[1]), "walk_interp_ms": float(r[2]),
            "interactions_per_particle": inter / n, "accuracy": accuracy_at(acc_b, "zeldovich")}


def run_plummer(ctx, tpm, torch, dev, stream, flush, steps):
    """The Plummer sphere, N = 8192, support 0.01, all active, geometric
    criterion theta = 0.7: one step = build + walk."""
    cfg = PLUMMER
    pos, mass = W.plummer(cfg["n"], W.CONFIG_SEEDS[1])
    n = len(pos)
    pos_d, mass_d = torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev)
    bp = lambda k: tpm.BuildParams(G=cfg["G"], h=cfg["h"], shift=root_shift(k, 1), leaf_bucket=cfg["bucket"])
    fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"])
    acc = torch.empty((n, 3), device=dev)
    pot = torch.empty(n, device=dev)
    nint = torch.empty(n, dtype=torch.int32, device=dev)
    res = []
    for k in range(steps + 3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        l2_flush(flush)
        ev[0].record(stream)
        sy = ctx.build_tree(pos_d, mass_d, bp(100 + k))
        ev[1].record(stream)
        sy.compute_forces(fp=fp, acc=acc, pot=pot, n_int=nint)
        ev[2].record(stream)
        sy.release()
        torch.cuda.synchronize()
        if k >= 3:
            res.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])])
    r = np.array(res).mean(0)
    ms = float(r.sum())
    inter = int(nint.to(torch.int64).sum().item())
    return {"workload": "plummer_n8192_bh_theta%g" % cfg["theta"], "value": n / (ms * 1e-3), "unit": "forces/s",
            "ms_per_step": ms, "build_ms": float(r[0]), "walk_ms": float(r[1]),
            "interactions_per_particle": inter / n, "accuracy": accuracy_at(acc, "plummer"),
            "note": "a small system: launch and latency bound, not a throughput figure"}


def run_ewald(ctx, tpm, torch, dev, stream, flush, steps):
    """The 128^3 box as a pure tree with the Ewald correction (no mesh): one
    step = build + relative walk (|a_old| from a geometric first pass)."""
    cfg = ZELDOVICH
    pos, mass = zeldovich_inputs()
    n = len(pos)
    pos_d = torch.from_numpy(pos).to(dev)
    mass_d = torch.from_numpy(mass).to(dev)
    h = zeldovich_h()
    bp = lambda k: tpm.BuildParams(G=cfg["G"], h=h, periodic=True, box=1.0, shift=root_shift(k, 7),
                                   leaf_bucket=cfg["bucket"])
    fp_bh = tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"])
    fp_rel = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"])
    s = ctx.build_tree(pos_d, mass_d, bp(0))
    acc, pot, nint = s.compute_forces(fp=fp_bh)
    s.release()
    a_old = torch.linalg.vector_norm(acc, dim=1).contiguous()
    res = []
    for k in range(steps + 2):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        l2_flush(flush)
        ev[0].record(stream)
        sy = ctx.build_tree(pos_d, mass_d, bp(100 + k))
        ev[1].record(stream)
        sy.compute_forces(a_old=a_old, fp=fp_rel, acc=acc, pot=pot, n_int=nint)
        ev[2].record(stream)
        sy.release()
        torch.cuda.synchronize()
        if k >= 2:
            res.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])])
    r = np.array(res).mean(0)
    ms = float(r.sum())
    inter = int(nint.to(torch.int64).sum().item())
    return {"workload": "zeldovich_128^3_ewald_tree_relative_alpha%g" % cfg["alpha"], "value": n / (ms * 1e-3),
            "unit": "forces/s", "ms_per_step": ms, "build_ms": float(r[0]), "walk_ms": float(r[1]),
            "interactions_per_particle": inter / n, "accuracy": accuracy_at(acc, "zeldovich")}


def run_two_species(ctx, tpm, torch, dev, stream, flush, steps):
    """Per-particle softening: a Hernquist 2^20 halo (support 0.005) with a
    compact stellar Plummer component of 2^18 particles (support 0.001); one
    step = build + relative walk (|a_old| from a geometric first pass)."""
    cfg = HERNQUIST
    pos, mass, hs, _ = W.two_species(1 << 20, 1 << 18, W.CONFIG_SEEDS[2])
    n = len(pos)
    pos_d, mass_d, hs_d = (torch.from_numpy(x).to(dev) for x in (pos, mass, hs))
    bp = lambda k: tpm.BuildParams(G=cfg["G"], h=cfg["h"], shift=root_shift(k, 8), leaf_bucket=cfg["bucket"])
    fp_bh = tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"])
    fp_rel = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"])
    s = ctx.build_tree(pos_d, mass_d, bp(0), hsoft=hs_d)
    acc, pot, nint = s.compute_forces(fp=fp_bh)
    s.release()
    a_old = torch.linalg.vector_norm(acc, dim=1).contiguous()
    res = []
    for k in range(steps + 2):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        l2_flush(flush)
        ev[0].record(stream)
        sy = ctx.build_tree(pos_d, mass_d, bp(100 + k), hsoft=hs_d)
        ev[1].record(stream)
        sy.compute_forces(a_old=a_old, fp=fp_rel, acc=acc, pot=pot, n_int=nint)
        ev[2].record(stream)
        sy.release()
        torch.cuda.synchronize()
        if k >= 2:
            res.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])])
    r = np.array(res).mean(0)
    ms = float(r.sum())
    inter = int(nint.to(torch.int64).sum().item())
    return {"workload": "two_species_hernquist2^20_h0.005_plummer2^18_h0.001_relative_alpha%g" % cfg["alpha"],
            "value": n / (ms * 1e-3), "unit": "forces/s", "ms_per_step": ms, "build_ms": float(r[0]),
            "walk_ms": float(r[1]), "interactions_per_particle": inter / n,
            "accuracy": accuracy_at(acc, "two_species")}


def run_isolated(ctx, tpm, torch, dev, stream, flush, pos_d, mass_d, steps):
    """TreePM with open boundaries on the Hernquist 2^20 set: zero-padded
    (2 pm_n)^3 mesh over the root cube, r_s = a_s mesh cells; one step =
    build + mesh + short-range relative walk with interpolation."""
    cfg, ic = HERNQUIST, ISOLATED
    n = pos_d.shape[0]
    bp = lambda k: tpm.BuildParams(G=cfg["G"], h=cfg["h"], shift=root_shift(k, 6), leaf_bucket=cfg["bucket"])
    common = dict(treepm=True, pm_n=ic["pm_n"], asmth=ic["asmth"], rcut=ic["rcut"])
    fp_bh = tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"], **common)
    fp_rel = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"], **common)
    s = ctx.build_tree(pos_d, mass_d, bp(0))
    s.pm_long_range(fp_bh)
    acc, pot, nint = s.compute_forces(fp=fp_bh)
    s.release()
    a_old = torch.linalg.vector_norm(acc, dim=1).contiguous()
    res = []
    for k in range(steps + 2):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        l2_flush(flush)
        ev[0].record(stream)
        sy = ctx.build_tree(pos_d, mass_d, bp(100 + k))
        ev[1].record(stream)
        sy.pm_long_range(fp_rel)
        ev[2].record(stream)
        sy.compute_forces(a_old=a_old, fp=fp_rel, acc=acc, pot=pot, n_int=nint)
        ev[3].record(stream)
        sy.release()
        torch.cuda.synchronize()
        if k >= 2:
            res.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])])
    r = np.array(res).mean(0)
    ms = float(r.sum())
    inter = int(nint.to(torch.int64).sum().item())
    return {"workload": "hernquist_n2^20_treepm_open_pm%d_padded%d^3_asmth%g_relative_alpha%g" % (
                ic["pm_n"], 2 * ic["pm_n"], ic["asmth"], cfg["alpha"]),
            "value": n / (ms * 1e-3), "unit": "forces/s", "ms_per_step": ms, "build_ms": float(r[0]),
            "pm_ms": float(r[1]), "walk_interp_ms": float(r[2]), "interactions_per_particle": inter / n,
            "accuracy": accuracy_at(acc, "hernquist")}


def run_profile(name):
    """One workload alone, for a profiler's launch list: a geometric first
    force, then three relative-criterion steps of `periodic` (the 128^3 TreePM
    box: build, mesh, short-range walk with interpolation) or `hernquist` (the
    headline 2^20 set: build and walk).  Prints the mean step times."""
    import torch

    import paper_1909_04667_gb300 as tpm

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = tpm.Context(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if name == "periodic":
        out = run_periodic(ctx, tpm, torch, dev, stream, flush, 1)
    else:
        cfg = HERNQUIST
        pos, mass = hernquist_inputs()
        pos_d, mass_d = torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev)
        bp = lambda k: tpm.BuildParams(G=cfg["G"], h=cfg["h"], shift=root_shift(k, 2), leaf_bucket=cfg["bucket"])
        s = ctx.build_tree(pos_d, mass_d, bp(0))
        acc, pot, nint = s.compute_forces(fp=tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"]))
        s.release()
        a_old = torch.linalg.vector_norm(acc, dim=1).contiguous()
        fp = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"])
        res = []
        for k in range(3):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            l2_flush(flush)
            ev[0].record(stream)
            sy = ctx.build_tree(pos_d, mass_d, bp(1000 + k))
            ev[1].record(stream)
            sy.compute_forces(a_old=a_old, fp=fp, acc=acc, pot=pot, n_int=nint)
            ev[2].record(stream)
            sy.release()
            torch.cuda.synchronize()
            res.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])])
        r = np.array(res).mean(0)
        out = {"workload": "hernquist_n2^20_relative_alpha0.0025", "build_ms": float(r[0]), "walk_ms": float(r[1])}
    ctx.close()
    print(json.dumps(out))


# ------------------------------------------------------------------ CPU oracle
def run_oracle_sample(sample: int, nthreads: int = 0):
    """The FP64 oracle (as it stands) on a bounded sample of the headline
    workload: the whole tree build plus the relative-criterion walk of
    `sample` random active particles, |a_old| from its own geometric pass."""
    import oracle

    cfg = HERNQUIST
    pos, mass = hernquist_inputs()
    n = len(pos)
    tg = W.random_targets(n, sample, 77)
    shift = root_shift(0, 2)
    t0 = time.perf_counter()
    tree = oracle.Tree(pos, mass, bucket=cfg["bucket"], shift=shift)
    t_build = time.perf_counter() - t0
    a_bh, _, _ = tree.walk(tg, cfg["G"], cfg["h"], theta=cfg["theta"], nthreads=nthreads)
    a_old = np.linalg.norm(a_bh, axis=1).astype(np.float32)
    t0 = time.perf_counter()
    _, _, nint = tree.walk(tg, cfg["G"], cfg["h"], crit="rel", alpha=cfg["alpha"], a_old=a_old, nthreads=nthreads)
    t_walk = time.perf_counter() - t0
    # forces/s of a full step (build + all-particle walk) extrapolated from the sample
    t_step = t_build + t_walk * n / len(tg)
    return dict(value=n / t_step, unit="forces/s", t_build=t_build, t_walk_sample=t_walk, sample=len(tg),
                interactions_per_particle=float(nint.mean()))


def run_oracle_configs(serve_systems=None) -> dict:
    """The FP64 oracle (as it stands) on the other configurations, for the
    per-configuration CPU rows: the Plummer step in full; the periodic box's
    mesh, build and a sample of its walk (scaled to all particles); the
    time-bin cycle at the oracle's relative-walk rate on the Hernquist tree;
    and, given the particles of a few served systems, the per-request time
    of one build plus one geometric walk of a request's ids."""
    import oracle

    out = {}
    cfg = PLUMMER
    pos, mass = W.plummer(cfg["n"], W.CONFIG_SEEDS[1])
    n = len(pos)
    t0 = time.perf_counter()
    tree = oracle.Tree(pos, mass, bucket=cfg["bucket"], shift=root_shift(100, 1))
    tree.walk(np.arange(n, dtype=np.uint32), cfg["G"], cfg["h"], theta=cfg["theta"])
    t = time.perf_counter() - t0
    out["plummer_8192"] = {"value": n / t, "unit": "forces/s", "ms_per_step": t * 1e3,
                           "sample": "the whole step: build + BH walk of all 8192 particles"}

    zc = ZELDOVICH
    pos, mass = zeldovich_inputs()
    n = len(pos)
    sample = 4096
    tg = W.random_targets(n, sample, 79)
    h = zeldovich_h()
    rs = zc["asmth"] * 1.0 / zc["pm_n"]
    t0 = time.perf_counter()
    phi = oracle.pm_potential(pos, mass, 1.0, zc["pm_n"], rs, zc["G"])
    t_pm = time.perf_counter() - t0
    t0 = time.perf_counter()
    tree = oracle.Tree(pos, mass, bucket=zc["bucket"], periodic=True, box=1.0, shift=root_shift(0, 3))
    t_build = time.perf_counter() - t0
    kw = dict(treepm=True, rs=rs, rcut=zc["rcut"] * rs)
    a_bh, _, _ = tree.walk(tg, zc["G"], h, theta=zc["theta"], **kw)
    a_old = np.linalg.norm(a_bh, axis=1).astype(np.float32)
    t0 = time.perf_counter()
    tree.walk(tg, zc["G"], h, crit="rel", alpha=zc["alpha"], a_old=a_old, **kw)
    t_walk = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.pm_interpolate(phi, pos, 1.0)
    t_interp = time.perf_counter() - t0
    t_step = t_pm + t_build + t_interp + t_walk * n / sample
    out["periodic_treepm"] = {"value": n / t_step, "unit": "forces/s", "ms_per_step": t_step * 1e3,
                              "pm_ms": (t_pm + t_interp) * 1e3, "build_ms": t_build * 1e3,
                              "sample": "mesh, build and interpolation in full, relative walk of %d random "
                                        "targets scaled to all %d" % (sample, n)}
    if serve_systems:
        lat = []
        for pos, mass, h, shift, ids in serve_systems:
            t0 = time.perf_counter()
            tree = oracle.Tree(pos, mass, bucket=8, shift=shift)
            tree.walk(ids.astype(np.uint32), 1.0, h, theta=0.5)
            lat.append(time.perf_counter() - t0)
        lat = np.array(lat) * 1e3
        nids = sum(len(x[4]) for x in serve_systems)
        out["serving"] = {"latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_max": float(lat.max()),
                          "forces_per_s": nids / (lat.sum() * 1e-3), "requests": len(lat),
                          "sample": "build + geometric walk of each request's ids, for the first %d timed "
                                    "requests (%d ids), one after another" % (len(lat), nids)}
    return out


def oracle_floor(ctx) -> dict:
    """The FP64 oracle walk on the accuracy targets of the headline step (the
    same tree shift and |a_old|) against the stored exact sum: the method's
    own error, which the GPU walk reproduces up to FP32 rounding."""
    import oracle

    cfg = HERNQUIST
    pos, mass = hernquist_inputs()
    tree = oracle.Tree(pos, mass, bucket=cfg["bucket"], shift=ctx["shift"])
    a, _, _ = tree.walk(ctx["targets"].astype(np.uint32), cfg["G"], cfg["h"], crit="rel", alpha=cfg["alpha"],
                        a_old=ctx["a_old"].astype(np.float32))
    ex = exact_sums()
    return error_stats(a, ex["hernquist_acc"])


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def headline_config(world):
    """The headline workload, the same for both arms."""
    cfg = HERNQUIST
    n = cfg["n"]
    return {"workload": "hernquist_n2^20_relative_alpha0.0025", "n_particles": n, "n_active": n,
            "softening_h": cfg["h"], "leaf_bucket": cfg["bucket"], "criterion": "relative", "alpha": cfg["alpha"],
            "first_force": "geometric theta=0.5", "global_batch": n,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed (256 MiB write) between timed steps"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle

    oracle.build()
    sample = 65536
    vals = []
    for _ in range(args.warmup):
        run_oracle_sample(sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(run_oracle_sample(sample))
    wall = time.perf_counter() - t0
    v = statistics.median([r["value"] for r in vals])
    ms = statistics.median([(1 << 20) / r["value"] * 1e3 for r in vals])
    sample_ms = statistics.median([(r["t_build"] + r["t_walk_sample"]) * 1e3 for r in vals])
    c = cores()
    return dict(
        impl="reference", metric=METRIC, value=v, unit="forces/s", n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
        data="synthetic",
        config=headline_config(world),
        cpu_baseline={"value": v, "unit": "forces/s", "cores": c, "kind": "oracle",
                      "sample": "whole tree build + relative walk of %d random active particles per step, "
                                "extrapolated to all 2^20" % sample},
        e2e={"value": v, "unit": "forces/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        ms_per_step_kind="extrapolated: the whole build plus the timed walk of a %d-particle sample, the walk "
                         "scaled to all 2^20 particles (a full-step oracle walk is not run)" % sample,
        sample_ms_per_step=sample_ms,
        wall_s=wall,
    )


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--no-periodic", action="store_true", help="skip the periodic TreePM measurement")
    ap.add_argument("--bucket", type=int, default=None, help="leaf bucket B of the headline workload")
    ap.add_argument("--no-batching", action="store_true", help="skip the time-bin batching measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-hierarchy", action="store_true", help="skip the KDK time-bin hierarchy measurement")
    ap.add_argument("--no-isolated", action="store_true", help="skip the open-boundary TreePM measurement")
    ap.add_argument("--no-ewald", action="store_true", help="skip the periodic Ewald-tree measurement")
    ap.add_argument("--no-species", action="store_true", help="skip the two-species softening measurement")
    ap.add_argument("--profile-workload", choices=["periodic", "hernquist"], default=None,
                    help="run one workload alone (first force + three steps) for a profiler, print its step times")
    ap.add_argument("--serving-requests", type=int, default=None,
                    help="timed requests of the serving measurement (default: the full stream of 10^4)")
    args = ap.parse_args()
    if args.bucket:
        HERNQUIST["bucket"] = args.bucket
    if args.serving_requests:
        SERVING["n_requests"] = args.serving_requests
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.profile_workload:
        run_profile(args.profile_workload)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch

        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        floor_ctx = out.pop("_floor_ctx", None)
        samples = out["serving"].pop("_samples", None) if out.get("serving") else None
        serve_cpu = out["serving"].pop("_cpu_systems", None) if out.get("serving") else None
        if not args.no_cpu_baseline and world == 1:  # the CPU baseline: rank 0 at N = 1 only
            import oracle

            oracle.build()
            if floor_ctx is not None and isinstance(out.get("accuracy"), dict) and "p99" in out["accuracy"]:
                out["accuracy"]["oracle_walk_floor"] = oracle_floor(floor_ctx)
            if samples:
                out["serving"]["accuracy"] = serving_accuracy(samples)
            r = run_oracle_sample(65536)
            r1 = run_oracle_sample(4096, nthreads=1)
            per = run_oracle_configs(serve_cpu)
            # the time-bin cycle on the same tree: its forces at the oracle's
            # relative-walk rate of the headline sample (no rebuild per request)
            per["batching"] = {"value": r["sample"] / r["t_walk_sample"], "unit": "forces/s",
                               "sample": "relative-walk rate of the headline sample on the Hernquist tree"}
            out["cpu_baseline"] = {"value": r["value"], "unit": "forces/s", "cores": cores(), "kind": "oracle",
                                   "sample": "whole tree build + relative walk of %d random active particles, "
                                             "extrapolated to all 2^20" % r["sample"],
                                   "single_core": {"value": r1["value"], "unit": "forces/s", "cores": 1,
                                                   "sample": "the same with %d particles" % r1["sample"]},
                                   "per_config": per}
        print(json.dumps(out))
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
