#!/usr/bin/env python
"""Benchmark of the short-range P3M path on GB300: SR pair interactions/s and
particle-steps/s.

Workload (default): one periodic box of 256^3 particles, side 256 grid units,
positions from Zel'dovich displacements of a Gaussian field with P(k) ~ k^-2
(sigma_delta = 1 on the grid), velocities N(0, 0.1^2), unit masses, seed 2.
One step = one full step of Eq. (tstep): long-range PM half kick, 5 short-range
SKS sub-cycles (each: stream, rebin, pair force + kick, stream), PM half kick.
Inputs stay resident in HBM; the working set (~1.5 GB) is far larger than L2,
so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  value = SR pair interactions (ordered pairs i != j
inside r_cut, summed over all sub-cycles and ranks) per second of device time.
The inside-cutoff counts come from a deterministic replay of the timed steps
with the counting kernel variant (the replay reproduces the timed trajectory
bit for bit, which is asserted).
"""
from __future__ import annotations

import argparse
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

METRIC = "SR pair interactions/s and particle-steps/s on 1 GB300 (served vs plain); p99 latency"
FLOPS_PER_PAIR = 29  # counted FP32 flops per pair (plus one rsqrt)

CONFIGS = {
    # name: (grid side, box L, seed, sub-cycles per step, dt per step)
    "zeldovich256": dict(side=256, L=256.0, seed=2, n_c=5, dt=0.5,
                         desc="256^3 Zel'dovich (P(k)~k^-2, sigma_delta=1), box 256, "
                              "PM half kicks + 5 SR sub-cycles per step"),
    "zeldovich128": dict(side=128, L=128.0, seed=2, n_c=5, dt=0.5,
                         desc="128^3 Zel'dovich (P(k)~k^-2, sigma_delta=1), box 128, "
                              "PM half kicks + 5 SR sub-cycles per step"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="zeldovich256")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU oracle sample time")
    ap.add_argument("--no-pm", action="store_true", help="short-range sub-cycles only (no PM half kicks)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched (200 boxes) segment")
    ap.add_argument("--no-served", action="store_true", help="skip the served (Poisson stream) segment")
    ap.add_argument("--served-window", type=float, default=8.0,
                    help="seconds of arrivals per served rate (the C5 stream is 60 s long; shortened to fit the run)")
    ap.add_argument("--served-cap", type=float, default=16.0, help="wall-time cap of each served rate")
    ap.add_argument("--served-rates", type=str, default="2,4,6,10,50", help="arrival rates (per s) of the served sweep")
    ap.add_argument("--no-c1", action="store_true", help="skip the plain 32^3 segment")
    ap.add_argument("--no-c3", action="store_true", help="skip the 512^3 precision segment")
    ap.add_argument("--kernel-table", type=str, default="",
                    help="write the device time of every kernel of one untimed step and of one hacc_bin call "
                         "(CUDA activity records) as JSON to this path")
    ap.add_argument("--precision", action="store_true",
                    help="precision study instead: 512^3 Zel'dovich, FP32 absolute vs cell + offset positions")
    ap.add_argument("--precision-side", type=int, default=512)
    ap.add_argument("--precision-sample", type=int, default=1 << 20)
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


def reduce_over_ranks(value: float, dist, op: str = "max", device: str = "cuda") -> float:
    """Max (the timing rule) or sum of a per-rank number over all ranks; the
    identity without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_rate(local_work: float, local_ms: float, dist, device: str = "cuda") -> dict:
    """Whole-job rate of independent replicas: work summed over ranks divided
    by the slowest rank's time (weak scaling, no data-path collective)."""
    ms = reduce_over_ranks(local_ms, dist, "max", device)
    work = reduce_over_ranks(local_work, dist, "sum", device)
    return {"ms": ms, "work": work, "rate": work / (ms / 1e3) if ms > 0 else 0.0}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def measured_traffic(n_particles: int):
    """DRAM bytes of one pair-kernel launch from the committed ncu capture,
    scaled by particles (traffic is ~63 B per particle per launch), or None
    when the kernel source changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "sr_force_traffic_zeldovich256.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, "paper_1410_2805_gb300", "csrc", "sr_force.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except Exception:
        return None
    if sha != rec.get("kernel_source_sha256_16"):
        return None
    return (rec["dram_bytes_read"] + rec["dram_bytes_write"]) * n_particles / rec["particles"]


def fp32_peak_tflops(num_sms: int, mhz: float) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return num_sms * 128 * 2 * mhz * 1e6 / 1e12


def workload_config(args, world):
    """The `config` object of the JSON line, the same for both arms."""
    cfg = CONFIGS[args.config]
    n = cfg["side"] ** 3
    return {"workload": args.config, "desc": cfg["desc"], "particles": n, "box": cfg["L"],
            "sub_cycles_per_step": cfg["n_c"], "pm": not args.no_pm, "dt": cfg["dt"],
            "l2": "inputs larger than L2 (working set ~%.1f GB)" % (n * 100 / 1e9),
            "parallelism": "replicas" if world > 1 else "single"}


def make_inputs(cfg):
    import synth
    pos = synth.zeldovich(cfg["side"], seed=cfg["seed"], L=cfg["L"])
    vel = synth.gaussian_velocities(len(pos), seed=cfg["seed"], sigma=0.1)
    return pos, vel


# ---------------------------------------------------------------------------
def cpu_oracle_rate(pos, L, split_params, target_s: float, seed: int = 99):
    """Oracle (FP64, all host cores) on a bounded random sample of particles of
    the same box: inside-cutoff pair interactions per second."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(seed)
    n = len(pos)
    # two probes fit t(m) = a + b m (a: the oracle's cell-list build over all
    # n particles, b: per sampled particle); then size the measured call
    times = []
    for m in (2048, 16384):
        sel = rng.choice(n, size=min(n, m), replace=False).astype(np.int64)
        t0 = time.perf_counter()
        oracle.force_mesh(pos, L, split_params, sel=sel)
        times.append((min(n, m), time.perf_counter() - t0))
    (m1, t1), (m2, t2) = times
    b = max((t2 - t1) / max(m2 - m1, 1), 1e-9)
    a = max(t1 - b * m1, 0.0)
    m = int(min(n, max(m2, (target_s - a) / b)))
    sel = rng.choice(n, size=m, replace=False).astype(np.int64)
    t0 = time.perf_counter()
    _, w = oracle.force_mesh(pos, L, split_params, sel=sel)
    dt = time.perf_counter() - t0
    return dict(value=w / dt, pairs=w, seconds=dt, sample_particles=m, threads=oracle.threads())


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores."""
    import numpy as np

    import oracle
    from oracle import split
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    cfg = CONFIGS[args.config]
    pos, _ = make_inputs(cfg)
    sp = split.default_split()
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    sp["eps"] = float(np.float32(sp["eps"]))
    per_step = max(1.0, 150.0 / max(1, args.steps + args.warmup) / 2)
    probe = cpu_oracle_rate(pos, cfg["L"], sp, target_s=per_step)
    m = probe["sample_particles"]
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        oracle.force_mesh(pos, cfg["L"], sp, sel=rng.choice(len(pos), size=m, replace=False).astype(np.int64))
    tot_pairs, tot_t = 0, 0.0
    for _ in range(args.steps):
        sel = rng.choice(len(pos), size=m, replace=False).astype(np.int64)
        t0 = time.perf_counter()
        _, w = oracle.force_mesh(pos, cfg["L"], sp, sel=sel)
        tot_t += time.perf_counter() - t0
        tot_pairs += w
    value = tot_pairs / tot_t
    sample = ("short-range force of %d random particles of the initial conditions of the %s box per step (all %d "
              "particles as sources, cell list rebuilt per call), FP64" % (m, cfg["desc"].split(",")[0], len(pos)))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pair interactions/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, world),
            "cpu_baseline": {"value": value, "unit": "pair interactions/s", "cores": oracle.threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pair interactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_batched(torch, hacc, ctx, split, steps=3, warmup=1, n_sub=10, seed=4):
    """200 independent blob-mixture boxes (half uniform, half in blobs of 256,
    sigma 0.5), N log-uniform in [16^3, 128^3], box side N^(1/3), step 0.1 as
    10 SR sub-cycles, one batched launch per sub-cycle, all 10 captured as
    one CUDA graph.  The launch shape (item cap x kernel variant) is picked by
    the batched autotuner on the batch itself first; FP64 diagnostics of every
    box before and after the timed steps."""
    import numpy as np

    import synth
    specs = synth.batch_boxes(200, seed=seed)
    pos, vel, boxes, off = [], [], [], 0
    for sp_ in specs:
        pos.append(synth.blob_mixture_scaled(sp_.n, sp_.L, seed=sp_.seed))
        vel.append(synth.gaussian_velocities(sp_.n, seed=sp_.seed))
        boxes.append(hacc.BatchBox(L=sp_.L, offset=off, n=sp_.n, dt=0.1))
        off += sp_.n
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        P = torch.from_numpy(np.concatenate(pos)).cuda()
        V = torch.from_numpy(np.concatenate(vel)).cuda()
        tune = ctx.batch_tune(split, boxes, P, V, reps=1, stream=stream)
        d_start = ctx.batch_diagnostics(split, boxes, P, V, stream=stream).cpu().numpy()
        for _ in range(warmup):
            ctx.batch_subcycle(split, boxes, P, V, n_sub, use_graph=True, stream=stream)
        stream.synchronize()
        snap_p, snap_v = P.clone(), V.clone()
        ctx.stats_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.batch_subcycle(split, boxes, P, V, n_sub, use_graph=True, stream=stream)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        st = ctx.stats_read(reset=True)
        fin_p, fin_v = P.clone(), V.clone()
        d_end = ctx.batch_diagnostics(split, boxes, P, V, stream=stream).cpu().numpy()
        P.copy_(snap_p)
        V.copy_(snap_v)
        ctx.stats_enable(counting=True)
        for _ in range(steps):
            ctx.batch_subcycle(split, boxes, P, V, n_sub, use_graph=True, stream=stream)
        stream.synchronize()
        cnt = ctx.stats_read(reset=True)
        ctx.stats_enable(counting=False)
        same = bool(torch.equal(P, fin_p) and torch.equal(V, fin_v))
        # the same steps once more without the graph, pair-kernel launches timed
        P.copy_(snap_p)
        V.copy_(snap_v)
        ctx.stats_enable(timing=True)
        for _ in range(steps):
            ctx.batch_subcycle(split, boxes, P, V, n_sub, use_graph=False, stream=stream)
        stream.synchronize()
        tst = ctx.stats_read(reset=True)
        ctx.stats_enable()
    ctx.sync(stream)          # raises if a coordinate left [-L, 2L)
    n = off
    peaks = measured_peaks()
    num_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = fp32_peak_tflops(num_sms, float(peaks.get("sm_max_mhz") or 2070.0))
    force_s = tst["force_ms"] / 1e3
    ach = cnt["candidate_pairs"] * FLOPS_PER_PAIR / force_s / 1e12 if force_s > 0 else None
    # per box: momentum change against the summed |m v|, and the change of
    # kinetic + short-range potential energy against KE + |PE| at the start
    # (the blobs start nearly at rest: their potential energy dominates)
    mv_scale = np.array([np.abs(v[:, :3]).sum() for v in vel])   # unit masses
    mom = np.abs(d_end[:, :3] - d_start[:, :3]).max(1) / mv_scale
    de = np.abs((d_end[:, 3] + d_end[:, 4]) - (d_start[:, 3] + d_start[:, 4]))
    energy = de / (d_start[:, 3] + np.abs(d_start[:, 4]))
    energy_ke = de / d_start[:, 3]
    default_k = 0   # cell-wide items, cell order, variant 0
    return {"workload": "200 blob-mixture boxes, N log-uniform 16^3..128^3 (total %d), 10 SR sub-cycles per "
                        "step, one batched launch per sub-cycle, CUDA graph" % n,
            "autotune": {"chosen_setting": tune["chosen"], "item_cap": tune["item_cap"], "variant": tune["variant"],
                         "heavy_first": tune["heavy_first"],
                         "tick_ms_chosen": tune["times_ms"][tune["chosen"]],
                         "tick_ms_cell_wide_cell_order_variant0": tune["times_ms"][default_k],
                         "gain_over_cell_wide_cell_order_variant0":
                             tune["times_ms"][default_k] / tune["times_ms"][tune["chosen"]],
                         "settings": "item cap in %s x queue order (cell, largest first) x %d kernel variants; "
                                     "time = one batched tick" % (list(hacc.BATCH_TUNE_CAPS), hacc.FORCE_VARIANTS),
                         "tick_ms_by_setting": tune["times_ms"]},
            "diagnostics": {"max_momentum_change_rel": float(mom.max()),
                            "max_energy_change_rel": float(energy.max()),
                            "median_energy_change_rel": float(np.median(energy)),
                            "energy_change_rel_to": "KE + |PE| of the box at the start",
                            "max_energy_change_rel_ke": float(energy_ke.max()),
                            "over": "%d steps of 10 sub-cycles (step 0.1), FP64 per-box sums" % (warmup + steps)},
            "pair_interactions_per_s": cnt["within_pairs"] / (ms / 1e3),
            "particle_steps_per_s": n * n_sub * steps / (ms / 1e3), "ms_per_step": ms / steps, "steps": steps,
            "gpu_launches": st["kernel_launches"], "replay_bitwise_equal": same,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": (ach / peak) if ach else None,
                         "evaluated_frac": (cnt["evaluated_pairs"] * FLOPS_PER_PAIR / force_s / 1e12 / peak)
                         if force_s > 0 else None,
                         "candidate_pairs_per_step": cnt["candidate_pairs"] / steps,
                         "evaluated_pairs_per_step": cnt["evaluated_pairs"] / steps,
                         "force_ms_per_step": tst["force_ms"] / steps,
                         "basis": "29 flop per 27-cell candidate pair over the pair-kernel time (events, "
                                  "a replay without the graph)"}}


def run_multilevel(torch, hacc, ctx, split, steps=3, d=2, lmax=4, seed=7, workload="blob128", dt=0.04, skin=0.05,
                   lmin=1, n_plain=None):
    """One 128^3 box: n_plain (default lmax) uniform SKS sub-cycles per step
    against the multi-level step with kick counts l = floor(floor(rho/rho0)/d) + 1
    clamped to [lmin, lmax] (Eq. (kicks)); device time per step, and the
    pair-kernel share of it."""
    n_plain = lmax if n_plain is None else n_plain
    import numpy as np

    import synth
    L = 128.0
    if workload == "blob128":
        pos0 = synth.blob_mixture_scaled(128 ** 3, L, seed=seed)
        desc = "128^3 blob mixture (blobs of 256, sigma 0.5), box 128"
    else:
        pos0 = synth.zeldovich(128, seed=seed, L=L)
        desc = "128^3 Zel'dovich (P(k)~k^-2, sigma_delta=1), box 128"
    vel0 = synth.gaussian_velocities(128 ** 3, seed=seed)
    box = hacc.Box(L=L)
    stream = torch.cuda.current_stream()
    out = {}
    for mode in ("plain", "multilevel"):
        P, V = torch.from_numpy(pos0).cuda(), torch.from_numpy(vel0).cuda()
        lev = torch.zeros(len(pos0), dtype=torch.int32, device="cuda")

        def one():
            if mode == "plain":
                ctx.subcycle(box, split, P, V, dt, n_plain)
            else:
                ctx.subcycle_ml(box, split, P, V, dt, d, lmax, skin=skin, levels=lev, lmin=lmin)
        one()
        torch.cuda.synchronize()
        ctx.stats_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            one()
        e1.record(stream)
        torch.cuda.synchronize()
        out["ms_per_step_" + mode] = e0.elapsed_time(e1) / steps
        st = ctx.stats_read(reset=True)
        out["kernel_launches_per_step_" + mode] = st["kernel_launches"] / steps
        # one more step with the pair launches timed (events around each)
        ctx.stats_enable(timing=True)
        one()
        st = ctx.stats_read(reset=True)
        ctx.stats_enable()
        out["force_ms_per_step_" + mode] = st["force_ms"]
        if mode == "multilevel":
            out["rebins_per_step"] = st["ml_rebins"]
            h = np.bincount(lev.cpu().numpy(), minlength=lmax + 1)[1:]
            out["kick_count_fractions"] = [float(x) for x in h / h.sum()]
            out["force_evaluations_per_particle"] = float((np.arange(1, lmax + 1) * h).sum() / h.sum())
    ctx.sync()
    out["speedup"] = out["ms_per_step_plain"] / out["ms_per_step_multilevel"]
    out["faster_than_uniform_sub_cycles"] = out["speedup"] > 1.0
    if out["speedup"] <= 1.0:
        out["why_slower"] = ("the particles move past half the skin between events, so the mesh is rebuilt at %.0f "
                             "events per step; the rebinnings cost more than the %.0f%% of force work the kick "
                             "counts save" % (out.get("rebins_per_step", 0), 100 * (1 - out["force_ms_per_step_multilevel"]
                                                                                 / out["force_ms_per_step_plain"])))
    out["workload"] = "%s, step %g, %d uniform sub-cycles vs d = %d, l in [%d, %d], skin %g r_cut (%d^3 cells)" % (
        desc, dt, n_plain, d, lmin, lmax, skin, hacc.ml_mesh_cells(L, split.r_cut, skin))
    return out


def run_fine_mesh(torch, hacc, ctx, split, pos, L, reps=3):
    """One force evaluation of the bench box with cells >= r_cut (27-cell
    search) and cells >= r_cut/2 (125-cell search): device time per call and
    the pair counts of each."""
    box = hacc.Box(L=L)
    stream = torch.cuda.current_stream()
    out = {}
    for R in (1, 2):
        ctx.set_stencil(R)
        try:
            ctx.sr_force(box, split, pos)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                ctx.sr_force(box, split, pos)
            e1.record(stream)
            torch.cuda.synchronize()
            ctx.stats_read(reset=True)
            ctx.stats_enable(counting=True)
            ctx.sr_force(box, split, pos)
            st = ctx.stats_read(reset=True)
            ctx.stats_enable()
        finally:
            ctx.set_stencil(1)
        out["cells_%d" % (27 if R == 1 else 125)] = {
            "ms_per_force_call": e0.elapsed_time(e1) / reps, "candidate_pairs": st["candidate_pairs"],
            "evaluated_pairs": st["evaluated_pairs"], "within_pairs": st["within_pairs"]}
    out["speedup_125_over_27"] = out["cells_27"]["ms_per_force_call"] / out["cells_125"]["ms_per_force_call"]
    out["faster_than_27_cells"] = out["speedup_125_over_27"] > 1.0
    if not out["faster_than_27_cells"]:
        out["why_slower"] = ("%.0f%% fewer evaluated pairs, but a work item of a fine cell holds ~4 particles and "
                             "pays the whole per-item staging (a 50-run table, bounds, tile set-up) for them"
                             % (100 * (1 - out["cells_125"]["evaluated_pairs"] / out["cells_27"]["evaluated_pairs"])))
    return out


def run_binning(torch, hacc, ctx, split, pos, L, reps=5):
    """hacc_bin on the bench box (wrap, exact cell key, count, scan, stable
    order): device time per call and HBM throughput on the algorithmic bytes
    (read the positions; write the cell ids, the permutation and the cell
    starts; write back the positions the wrap moves -- the timed calls repeat
    the call on positions the first call wrapped, so none)."""
    box = hacc.Box(L=L)
    work = pos.clone()
    r_cut = split.r_cut
    ctx.bin(box, r_cut, work)
    xyz = work[:, :3]
    moved = int(((xyz < 0) | (xyz >= L)).any(1).sum().item())
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.bin(box, r_cut, work)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    n = int(pos.shape[0])
    nc = hacc.mesh_cells(L, r_cut)
    alg = n * (16 + 4 + 4) + moved * 16 + (nc ** 3 + 1) * 4
    gbs = alg / (ms / 1e3) / 1e9
    peak = measured_peaks().get("hbm_gbs")
    return {"ms_per_call": ms, "algorithmic_bytes": alg, "bytes_per_particle": alg / max(n, 1),
            "moved_by_wrap": moved, "achieved_gbs": gbs,
            "peak_gbs": peak, "frac": (gbs / peak) if peak else None, "bound": "hbm",
            "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}


class RequestBoxes:
    """Each request's own seeded box: a blob mixture of its size class (one
    seeded template per class) moved by the request's own seeded periodic shift,
    with velocities of the template; built ahead of use by worker threads
    (numpy releases the GIL in these array operations)."""

    def __init__(self, seed, sides=(32, 64, 128, 256), workers=4):
        import concurrent.futures as cf

        import synth
        self.templates = {}
        for side in sides:
            self.templates[side] = (synth.blob_mixture_scaled(side ** 3, float(side), seed=seed * 7 + side),
                                    synth.gaussian_velocities(side ** 3, seed=seed * 7 + side))
        self.pool = cf.ThreadPoolExecutor(max_workers=workers)

    def build(self, req):
        import numpy as np
        side = round(req.n ** (1.0 / 3.0))
        p0, v0 = self.templates[side]
        L = np.float32(req.L)
        shift = np.random.default_rng(req.seed).uniform(0.0, float(L), 3).astype(np.float32)
        p = p0.copy()
        x = p[:, :3]
        x += shift
        x[x >= L] -= L
        x[x >= L] = 0          # a sum that rounds up to L
        return p, v0.copy()

    def submit(self, req):
        return self.pool.submit(self.build, req)

    def close(self):
        self.pool.shutdown(wait=True)


def run_served(torch, hacc, ctx, split, boxes, rate, window, cap_s, seed=5, max_active=64 << 20,
               pool_gb=40.0, budget_gb=150.0, replay=False, peak=None, variant=0):
    """Poisson arrivals (rate/s over `window` s) of runs with N in {32^3, 64^3,
    128^3, 256^3} (each its own seeded blob-mixture box, blobs of 256) and 5-50
    SR sub-cycles of step 0.01; continuous batching (admission in arrival order
    against the row pool, a cap of particles per tick and the context's HBM
    budget, one batched sub-cycle of every resident run per tick).  Arrived runs
    are handed to the server in arrival order while the server's queue holds
    fewer than two per-tick caps of particles (it cannot admit more than one
    cap per tick, so this bounds host memory without changing which run is
    admitted when).  Step latency = wall time of the tick that advanced the
    run (host, including its copies); device time of each tick from CUDA
    events on the stream.  Request latency = finish - arrival; runs unfinished
    at the cap count as finishing at the cap (censored; their number is given).
    replay: run the same tick schedule again with the counting kernel (pair
    counts; the timed session runs the plain kernel with the pair launches
    timed by events)."""
    import collections

    import numpy as np

    import synth
    reqs = synth.request_stream(rate=rate, duration=window, seed=seed)
    stream = torch.cuda.current_stream()
    sctx = hacc.Context(ctx.device, hbm_budget_bytes=int(budget_gb * 1e9))
    sctx.set_variant(variant)
    free_b = torch.cuda.mem_get_info()[0]
    pool = int(min(pool_gb * 1e9, free_b - 24e9))
    srv = hacc.Server(sctx, split, pool_bytes=pool, max_active_particles=max_active)
    pending = collections.deque(reqs)
    futures = collections.deque()          # (request, future of its buffers), arrival order
    in_queue = collections.deque()         # handed to the server, not yet admitted (FIFO)
    arrival, finished_at, keep = {}, {}, {}
    schedule = []                          # requests handed over before each tick
    lat, dev_ms = [], []
    psteps, queued_particles = 0, 0
    busy = 0.0
    lookahead = 8
    sctx.stats_read(reset=True)
    sctx.stats_enable(timing=True)
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        if now > cap_s:
            break
        while pending and len(futures) < lookahead:
            r = pending.popleft()
            futures.append((r, boxes.submit(r)))
        handed = []
        while futures and futures[0][0].t_arrival <= now and queued_particles < 2 * max_active:
            r, fut = futures.popleft()
            p, v = fut.result()
            arrival[r.rid] = r.t_arrival
            keep[r.rid] = (p, v, r)
            srv.submit(r.rid, r.L, p, v, h=0.01, steps=r.steps)
            queued_particles += r.n
            in_queue.append(r)
            handed.append(r.rid)
        if not keep:
            if not futures and not pending:
                break
            nxt = futures[0][0].t_arrival if futures else now
            time.sleep(max(0.0, min(0.01, nxt - now)))
            continue
        schedule.append(handed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ta = time.perf_counter()
        e0.record(stream)
        t = srv.tick()
        e1.record(stream)
        dt = time.perf_counter() - ta
        busy += dt
        dev_ms.append((e0, e1))
        lat += [dt] * t["active"]
        psteps += t["particles"]
        tf = time.perf_counter() - t0
        for rid in t["finished_ids"]:
            finished_at[rid] = tf
            keep.pop(rid, None)
        for _ in range(t["admitted"]):
            queued_particles -= in_queue.popleft().n
    wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    dev_total = sum(a.elapsed_time(b) for a, b in dev_ms) / 1e3
    st = sctx.stats_read(reset=True)
    sctx.stats_enable()
    sctx.sync()                # raises if a coordinate left [-L, 2L)
    srv.close()
    unfinished = [k for k in arrival if k not in finished_at]
    lat_ms = np.array(lat) * 1e3 if lat else np.zeros(1)
    resp = np.array([finished_at[k] - arrival[k] for k in finished_at] +
                    [wall - arrival[k] for k in unfinished]) if arrival else np.zeros(1)
    out = {"rate_per_s": rate, "arrival_window_s": window, "cap_s": cap_s, "wall_s": wall, "busy_s": busy,
           "device_s": dev_total, "requests_arrived": len(arrival), "requests_finished": len(finished_at),
           "requests_unfinished_censored": len(unfinished), "ticks": len(dev_ms), "run_steps": len(lat),
           "p50_step_ms": float(np.percentile(lat_ms, 50)), "p99_step_ms": float(np.percentile(lat_ms, 99)),
           "p50_request_s": float(np.percentile(resp, 50)), "p99_request_s": float(np.percentile(resp, 99)),
           "particle_steps_per_s_busy": psteps / max(busy, 1e-9),
           "particle_steps_per_s_device": psteps / max(dev_total, 1e-9),
           "force_ms": st["force_ms"], "max_active_particles": max_active, "pool_gb": pool / 1e9,
           "hbm_budget_gb": budget_gb}
    if replay:
        # the same ticks again: same hand-over schedule, so the same admissions
        # and the same batched passes, with the counting kernel
        srv = hacc.Server(sctx, split, pool_bytes=pool, max_active_particles=max_active)
        sctx.stats_read(reset=True)
        sctx.stats_enable(counting=True)
        by_id = {r.rid: r for r in reqs}
        for handed in schedule:
            for rid in handed:
                r = by_id[rid]
                p, v = boxes.build(r)
                keep[rid] = (p, v, r)
                srv.submit(rid, r.L, p, v, h=0.01, steps=r.steps)
            t = srv.tick()
            for rid in t["finished_ids"]:
                keep.pop(rid, None)
        sctx.stats_enable()
        cnt = sctx.stats_read(reset=True)
        srv.close()
        out["pair_interactions_per_s_device"] = cnt["within_pairs"] / max(dev_total, 1e-9)
        out["candidate_pairs"] = cnt["candidate_pairs"]
        out["within_pairs"] = cnt["within_pairs"]
        force_s = st["force_ms"] / 1e3
        if peak and force_s > 0:
            ach = cnt["candidate_pairs"] * FLOPS_PER_PAIR / force_s / 1e12
            ev = cnt["evaluated_pairs"] * FLOPS_PER_PAIR / force_s / 1e12
            out["roofline"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                               "frac": ach / peak, "evaluated_frac": ev / peak,
                               "basis": "29 flop per 27-cell candidate pair (counting replay of the same ticks) "
                                        "over the event-timed batched pair launches of the timed session"}
    sctx.close()
    return out


def run_served_sweep(torch, hacc, ctx, split, rates, window, cap_s, peak, seed=5, variant=0):
    """The served segment at several arrival rates (the same seeded stream
    generator, one seed per rate); the highest rate also gets the counting
    replay (pair counts, roofline).  Saturation: the particle-steps a request
    brings on average against the particle-steps per second the server
    sustained at the highest rate."""
    import synth
    boxes = RequestBoxes(seed)
    try:
        rows = []
        for k, rate in enumerate(sorted(rates)):
            last = k == len(rates) - 1
            rows.append(run_served(torch, hacc, ctx, split, boxes, rate, window, cap_s, seed=seed + 10 * k,
                                   replay=last, peak=peak, variant=variant))
    finally:
        boxes.close()
    reqs = synth.request_stream(rate=100.0, duration=60.0, seed=seed)
    per_req = sum(r.n * r.steps for r in reqs) / len(reqs)
    cap = rows[-1]["particle_steps_per_s_busy"]
    return rows, {"mean_particle_steps_per_request": per_req, "capacity_particle_steps_per_s": cap,
                  "saturation_rate_per_s": cap / per_req}


def run_c1(torch, hacc, ctx, split, peak, restore, reps=20):
    """The plain 32^3 box: 32768 particles, L = 32, half uniform and half in 64
    Gaussian blobs (sigma 0.5), seed 1.  Pair force call and its pair-kernel
    launch (CUDA events) with the setting the autotuner picks on this machine (the
    context's setting `restore` is put back afterwards), binning (hacc_bin), and
    the force error against the FP64 oracle on every particle."""
    import numpy as np

    import oracle
    import synth
    L = 32.0
    pos_np = synth.blob_mixture(32768, L, seed=1)
    pos = torch.from_numpy(pos_np).cuda()
    box = hacc.Box(L=L)
    stream = torch.cuda.current_stream()
    tune = ctx.tune(box, split, pos)
    acc = ctx.sr_force(box, split, pos)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.stats_read(reset=True)
    ctx.stats_enable(timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.sr_force(box, split, pos, acc=acc)
    e1.record(stream)
    torch.cuda.synchronize()
    call_ms = e0.elapsed_time(e1) / reps
    st = ctx.stats_read(reset=True)
    ctx.stats_enable(counting=True)
    ctx.sr_force(box, split, pos, acc=acc)
    cnt = ctx.stats_read(reset=True)
    ctx.stats_enable()
    a = acc.cpu().numpy()[:, :3].astype(np.float64)
    sp = split.as_dict()
    ref, within_o = oracle.force_mesh(pos_np, L, sp)
    rms = float(np.sqrt((ref ** 2).sum(1).mean()))
    kern_ms = st["force_ms"] / max(1, st["force_launches"])
    ach = cnt["candidate_pairs"] * FLOPS_PER_PAIR / (kern_ms / 1e3) / 1e12
    b = run_binning(torch, hacc, ctx, split, pos, L, reps=reps)
    ctx.set_item_cap(restore["item_cap"])
    ctx.set_queue_order(1 if restore["heavy_first"] else 0)
    ctx.set_variant(restore["variant"])
    return {"workload": "32^3 blob mixture (half uniform, 64 blobs sigma 0.5), box 32, seed 1",
            "autotune": {"setting": tune["chosen"], "item_cap": tune["item_cap"], "variant": tune["variant"],
                         "heavy_first": tune["heavy_first"]},
            "force_call_ms": call_ms, "pair_kernel_ms": kern_ms,
            "candidate_pairs": cnt["candidate_pairs"], "within_pairs": cnt["within_pairs"],
            "within_pairs_oracle": within_o,
            "candidate_pairs_per_s": cnt["candidate_pairs"] / (call_ms / 1e3),
            "within_pairs_per_s": cnt["within_pairs"] / (call_ms / 1e3),
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "basis": "29 flop per 27-cell candidate pair over the event-timed pair-kernel launch"},
            "binning": {"ms_per_call": b["ms_per_call"], "achieved_gbs": b["achieved_gbs"], "frac": b["frac"]},
            "max_err_rel_rms": float(np.abs(a - ref).max() / rms)}


def precision_segment(torch, hacc, side=512, sample=1 << 20, reps=3):
    """Precision study (C3): side^3 Zel'dovich particles (box side, seed 3) from
    FP64 positions, stored as FP32 absolute coordinates and as (cell id, FP32
    in-cell offset).  For each storage mode, the pair forces against the FP64
    oracle on a seeded sample of particles (all particles as sources), twice:
    on the positions the mode stores (decoded exactly in FP64: the kernel's
    arithmetic alone) and on the FP64 generator positions (storage rounding
    plus arithmetic); device times of the force and of 5 SKS sub-cycles."""
    import numpy as np

    import oracle
    import synth
    L = float(side)
    x64 = synth.zeldovich(side, seed=3, L=L, return_f64=True)
    n = len(x64)
    p32 = np.ones((n, 4), np.float32)
    p32[:, :3] = x64.astype(np.float32)
    p32[:, :3][p32[:, :3] >= np.float32(L)] = 0
    vel = synth.gaussian_velocities(n, seed=3, sigma=0.1)
    ctx = hacc.Context(torch.cuda.current_device())
    split = hacc.default_split()
    box = hacc.Box(L=L)
    stream = torch.cuda.current_stream()
    nc = hacc.mesh_cells(L, split.r_cut)

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    out = {"particles": n, "box": L, "chaining_mesh": nc}
    P = torch.from_numpy(p32).cuda()
    X = torch.from_numpy(x64).cuda()
    cell, off = ctx.ci_from_f64(box, split.r_cut, X)
    del X
    acc32 = ctx.sr_force(box, split, P)
    out["force_ms_fp32_abs"] = timed(lambda: ctx.sr_force(box, split, P, acc=acc32), reps)
    acc_ci = ctx.sr_force_ci(box, split, cell, off)
    out["force_ms_cell_offset"] = timed(lambda: ctx.sr_force_ci(box, split, cell, off), reps)
    ctx.sync()
    a32 = acc32.cpu().numpy()[:, :3].astype(np.float64)
    aci = acc_ci.cpu().numpy()[:, :3].astype(np.float64)
    c = cell.cpu().numpy().astype(np.int64)
    o = off.cpu().numpy()[:, :3].astype(np.float64)
    P2, V2 = P.clone(), torch.from_numpy(vel).cuda()
    C2, O2, V3 = cell.clone(), off.clone(), torch.from_numpy(vel).cuda()
    out["subcycle5_ms_fp32_abs"] = timed(lambda: ctx.subcycle(box, split, P2, V2, 0.5, 5), 1)
    out["subcycle5_ms_cell_offset"] = timed(lambda: ctx.subcycle_ci(box, split, C2, O2, V3, 0.5, 5), 1)
    ctx.sync()
    ctx.close()
    del P, P2, V2, C2, O2, V3, acc32, acc_ci, cell, off
    torch.cuda.empty_cache()
    # the stored cell/offset positions, decoded in FP64: (c + 1/2) W + off, W = fl32(L / nc)
    W = float(np.float32(L / nc))
    xs = np.empty((n, 4))
    xs[:, 0] = (c % nc + 0.5) * W + o[:, 0]
    xs[:, 1] = ((c // nc) % nc + 0.5) * W + o[:, 1]
    xs[:, 2] = (c // (nc * nc) + 0.5) * W + o[:, 2]
    xs[:, 3] = 1.0
    del c, o
    d = xs[:, :3] - x64
    d -= L * np.round(d / L)
    out["storage_err_cell_offset_max"] = float(np.abs(d).max())
    d = p32[:, :3].astype(np.float64) - x64
    d -= L * np.round(d / L)
    out["storage_err_fp32_abs_max"] = float(np.abs(d).max())
    del d
    sp = split.as_dict()
    sel = np.sort(np.random.default_rng(33).choice(n, size=min(n, sample), replace=False))
    t0 = time.perf_counter()
    x4 = np.concatenate([x64, np.ones((n, 1))], axis=1)
    del x64
    ref64, _ = oracle.force_mesh(x4, L, sp, sel=sel)
    del x4
    ref_ci, _ = oracle.force_mesh(xs, L, sp, sel=sel)
    del xs
    ref_32, _ = oracle.force_mesh(p32, L, sp, sel=sel)
    out["oracle_s"] = time.perf_counter() - t0
    out["oracle_threads"] = oracle.threads()
    out["sample"] = int(len(sel))

    def errs(a, ref):
        rms = float(np.sqrt((ref ** 2).sum(1).mean()))
        amag = np.sqrt((ref ** 2).sum(1))
        dd = np.sqrt(((a[sel] - ref) ** 2).sum(1))
        big = amag > 0.01 * rms
        return {"max_rel_rms": float(dd.max() / rms), "rms_rel_rms": float(np.sqrt((dd ** 2).mean()) / rms),
                "p99_own_rel": float(np.percentile(dd[big] / amag[big], 99))}

    out["cell_offset_vs_stored"] = errs(aci, ref_ci)
    out["cell_offset_vs_f64"] = errs(aci, ref64)
    out["fp32_abs_vs_stored"] = errs(a32, ref_32)
    out["fp32_abs_vs_f64"] = errs(a32, ref64)
    out["workload"] = "%d^3 Zel'dovich (P(k)~k^-2), box %d, seed 3; oracle on a %d-particle sample" % (
        side, side, len(sel))
    return out


def summary(line):
    """The headline figures of every segment, rounded, as the last key of the
    line (short enough to survive a truncated log)."""
    def r(x, d=3):
        return float("%.*g" % (d, x)) if isinstance(x, (int, float)) and x is not None else x
    out = {"c2_pairs_per_s": r(line["value"]), "c2_frac": r(line["roofline"]["frac"]),
           "c2_eval_frac": r(line["roofline"]["evaluated_frac"]), "c2_e2e": r((line.get("e2e") or {}).get("value")),
           "bin_frac": r(line["binning_roofline"]["frac"]), "bin_build_frac": r(line["binning_roofline"].get(
               "full_build_frac"))}
    b = line.get("batched")
    if b:
        out["c4_pairs_per_s"] = r(b["pair_interactions_per_s"])
        out["c4_frac"] = r(b["roofline"]["frac"])
        out["c4_eval_frac"] = r(b["roofline"].get("evaluated_frac"))
    sv = line.get("served")
    if sv:
        out["c5_sat_rate"] = r(sv["saturation"]["saturation_rate_per_s"])
        out["c5"] = [[r(x["rate_per_s"]), r(x["p50_step_ms"]), r(x["p99_step_ms"]), r(x["p50_request_s"]),
                      r(x["p99_request_s"]), x["requests_finished"], x["requests_unfinished_censored"]]
                     for x in sv["sweep"]]
        out["c5_cols"] = "rate, p50/p99 step ms, p50/p99 request s, finished, censored"
        top = sv["sweep"][-1]
        out["c5_pairs_per_s"] = r(top.get("pair_interactions_per_s_device"))
        out["c5_frac"] = r((top.get("roofline") or {}).get("frac"))
        out["c5_vs_plain"] = r(sv.get("vs_plain_pairs_per_s"))
    c1 = line.get("c1")
    if c1:
        out["c1_within_per_s"] = r(c1["within_pairs_per_s"])
        out["c1_frac"] = r(c1["roofline"]["frac"])
        out["c1_err"] = r(c1["max_err_rel_rms"])
        out["c1_bin_gbs"] = r(c1["binning"]["achieved_gbs"])
    pr = line.get("precision")
    if pr:
        out["c3_ci_vs_stored"] = r(pr["cell_offset_vs_stored"]["max_rel_rms"])
        out["c3_ci_vs_f64"] = r(pr["cell_offset_vs_f64"]["max_rel_rms"])
        out["c3_abs_vs_stored"] = r(pr["fp32_abs_vs_stored"]["max_rel_rms"])
        out["c3_abs_vs_f64"] = r(pr["fp32_abs_vs_f64"]["max_rel_rms"])
        out["c3_force_ms"] = [r(pr["force_ms_cell_offset"]), r(pr["force_ms_fp32_abs"])]
    ml = line.get("multilevel_paper")
    if ml:
        out["ml_paper_speedup"] = r(ml["speedup"])
    mv = line.get("multilevel_violent")
    if mv:
        out["ml_violent_speedup"] = r(mv["speedup"])
    fm = line.get("fine_mesh")
    if fm:
        out["fine_mesh_speedup"] = r(fm["speedup_125_over_27"])
    return out


def kernel_table(torch, fn, reps=2):
    """Device time of every kernel launched by `fn`, from the CUDA activity
    records the PyTorch profiler collects: launches, microseconds per call and
    share, largest first.  These are the kernels' own durations at the clocks
    of a normal run (no replay)."""
    import collections
    import re

    from torch.profiler import ProfilerActivity, profile
    # a first session records nothing on some builds of the profiler: run one
    # and discard it
    with profile(activities=[ProfilerActivity.CUDA]):
        fn()
        torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
    agg = collections.defaultdict(lambda: [0, 0.0])
    for ev in prof.events():
        if ev.device_type != torch.autograd.DeviceType.CUDA:
            continue
        name = re.sub(r"\(anonymous namespace\)::|hacc::|void ", "", ev.name).split("(")[0][:64]
        t = getattr(ev, "device_time_total", None)
        agg[name][0] += 1
        agg[name][1] += t if t is not None else ev.cuda_time_total
    total = sum(t for _, t in agg.values())
    rows = [{"kernel": k, "launches_per_call": c / reps, "us_per_call": t / reps, "share": t / total if total else 0.0}
            for k, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1])]
    return {"calls_profiled": reps, "device_us_per_call": total / reps, "kernels": rows}


def run_ours(args):
    import numpy as np
    import torch

    import paper_1410_2805_gb300 as hacc
    from paper_1410_2805_gb300 import build as hbuild

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hbuild.build()
    cfg = CONFIGS[args.config]
    L = cfg["L"]
    pos_np, vel_np = make_inputs(cfg)
    n = len(pos_np)
    split = hacc.default_split()
    pm = hacc.PM()
    box = hacc.Box(L=L)
    ctx = hacc.Context(local)
    stream = torch.cuda.current_stream()
    pos = torch.from_numpy(pos_np).cuda()
    vel = torch.from_numpy(vel_np).cuda()
    use_pm = not args.no_pm
    dt, n_c = cfg["dt"], cfg["n_c"]

    def step(p, v):
        if use_pm:
            ctx.step(box, split, pm, p, v, dt, n_c)
        else:
            ctx.subcycle(box, split, p, v, dt, n_c)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step(pos, vel)
    ctx.sync()
    # pick the pair-kernel variant on the warmed-up box (the state the timed
    # steps start from)
    tuning = ctx.tune(box, split, pos, reps=3)
    snap_p, snap_v = pos.clone(), vel.clone()

    # ---- timed region: device-resident inputs ----
    ctx.stats_read(reset=True)
    ctx.stats_enable(timing=True, counting=False)
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")   # lets a profiler keep to the timed steps
    e0.record(stream)
    for _ in range(args.steps):
        step(pos, vel)
    e1.record(stream)
    barrier()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ctx.sync()
    st = ctx.stats_read(reset=True)
    ctx.stats_enable(timing=False, counting=False)
    final_p, final_v = pos.clone(), vel.clone()
    ms_max = reduce_over_ranks(ms, dist, "max")

    # ---- deterministic replay with pair counting (untimed) ----
    pos.copy_(snap_p)
    vel.copy_(snap_v)
    ctx.stats_enable(timing=False, counting=True)
    for _ in range(args.steps):
        step(pos, vel)
    ctx.sync()
    cnt = ctx.stats_read(reset=True)
    ctx.stats_enable(timing=False, counting=False)
    replay_ok = bool(torch.equal(pos, final_p) and torch.equal(vel, final_v))
    within = cnt["within_pairs"]
    cand = cnt["candidate_pairs"]
    evaluated = cnt["evaluated_pairs"]

    if args.kernel_table:
        # one step from the state the timed steps start from, and one hacc_bin
        # call on those positions
        wrapped = snap_p.clone()
        ctx.bin(box, split.r_cut, wrapped)
        tables = {"workload": args.config, "pm": not args.no_pm,
                  "step": kernel_table(torch, lambda: step(snap_p.clone(), snap_v.clone())),
                  "hacc_bin": kernel_table(torch, lambda: ctx.bin(box, split.r_cut, wrapped), reps=5)}
        with open(args.kernel_table, "w") as f:
            json.dump(tables, f, indent=1)

    # ---- end to end through the host-buffer C ABI (pinned memory) ----
    e2e = None
    if not args.no_e2e:
        hp = snap_p.cpu().pin_memory()
        hv = snap_v.cpu().pin_memory()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            if use_pm:
                ctx.step_host(box, split, pm, hp, hv, dt, n_c)
            else:
                ctx.subcycle_host(box, split, hp, hv, dt, n_c)
        barrier()
        t_e2e = reduce_over_ranks(time.perf_counter() - t0, dist, "max")
        e2e_same = bool(torch.equal(hp.cuda(), final_p) and torch.equal(hv.cuda(), final_v))
        e2e = {"value": world * within / t_e2e, "unit": "pair interactions/s",
               "h2d_bytes_per_step": 2 * n * 16, "d2h_bytes_per_step": 2 * n * 16,
               "ms_per_step": 1e3 * t_e2e / args.steps, "same_result_as_device_run": e2e_same}

    # ---- numbers ----
    secs = ms_max / 1e3
    value = replica_rate(within, ms, dist)["rate"]
    psteps = world * n * n_c * args.steps / secs
    peaks = measured_peaks()
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count
    smax = float(peaks.get("sm_max_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0)
    peak = fp32_peak_tflops(num_sms, smax)
    force_s = st["force_ms"] / 1e3
    # algorithmic work: 29 flops per 27-cell candidate pair (the method's
    # chaining-mesh search); the kernel evaluates only the candidates left
    # after its per-item bounding-box cull (dropped j were outside the cutoff
    # of every i), reported beside it as the hardware efficiency
    achieved = cand * FLOPS_PER_PAIR / force_s / 1e12 if force_s > 0 else None
    evaluated_tflops = evaluated * FLOPS_PER_PAIR / force_s / 1e12 if force_s > 0 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": measured_traffic(n),
                "kernel": "k_sr_force (pair force + kick + stream)",
                "peak_basis": "FP32 FMA: %d SMs x 128 lanes x 2 flop x %.0f MHz (sm_max_mhz of measured peaks)"
                              % (num_sms, smax),
                "flops_per_pair": FLOPS_PER_PAIR, "pairs_counted": "27-cell candidate pairs",
                "candidate_pairs_per_launch": cand / max(1, st["force_launches"]),
                "evaluated_pairs_per_launch": evaluated / max(1, st["force_launches"]),
                "evaluated_tflops": evaluated_tflops,
                "evaluated_frac": (evaluated_tflops / peak) if evaluated_tflops else None,
                "force_ms_per_launch": st["force_ms"] / max(1, st["force_launches"]),
                "force_launches": st["force_launches"], "force_share_of_step": st["force_ms"] / ms if ms else None}
    binning = run_binning(torch, hacc, ctx, split, snap_p, L)
    # the chaining-mesh build inside the timed sub-cycles (binning and the
    # gather of positions, velocities and rows into cell order), event-timed:
    # 96 algorithmic bytes per particle (read positions for the key, write the
    # key, read it to count and to place, read positions and velocities and
    # write the permutation and the sorted positions and velocities)
    if st.get("builds"):
        per = st["build_ms"] / st["builds"]
        gbs = 96 * n / (per / 1e3) / 1e9
        hbm = measured_peaks().get("hbm_gbs")
        binning["full_build_ms"] = per
        binning["full_build_bytes_per_particle"] = 96
        binning["full_build_gbs"] = gbs
        binning["full_build_frac"] = gbs / hbm if hbm else None
        binning["full_build_share_of_step"] = st["build_ms"] / ms if ms else None
    line = {"metric": METRIC, "value": value, "unit": "pair interactions/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(args, world),
            "particle_steps_per_s": psteps,
            "candidate_pairs_per_s": world * cand / secs,
            "within_cutoff_pairs_per_step": within / args.steps,
            "candidate_pairs_per_step": cand / args.steps,
            "evaluated_pairs_per_step": evaluated / args.steps,
            "replay_bitwise_equal": replay_ok,
            "gpu_launches": st["kernel_launches"],
            "roofline": roofline, "binning_roofline": binning, "e2e": e2e, "clocks": clk,
            "autotune": {"setting": tuning["chosen"], "variant": tuning["variant"], "item_cap": tuning["item_cap"],
                         "heavy_first": tuning["heavy_first"], "ms_by_setting": tuning["times_ms"],
                         "settings": "item cap in %s x queue order (cell, largest first) x variants (blocks/SM, "
                                     "inner loop) = (5,indexed), (4,indexed), (5,pointer-stepped), "
                                     "(4,pointer-stepped); time = one sub-cycle's chaining-mesh build + "
                                     "kick-and-stream launch" % (list(hacc.TUNE_CAPS),)}}
    if not args.no_batch:
        line["batched"] = run_batched(torch, hacc, ctx, split)
        # Zel'dovich box at a step where most particles drift a small part of
        # a cell (the regime the paper's fixed tree assumes), and the violent
        # blob box where the mesh is rebuilt at almost every event
        line["multilevel"] = run_multilevel(torch, hacc, ctx, split, workload="zel128", d=1, lmax=4, dt=0.02,
                                            skin=0.1)
        line["multilevel_violent"] = run_multilevel(torch, hacc, ctx, split, workload="blob128", d=2, lmax=4, dt=0.04,
                                                    skin=0.1)
        # the paper's test of Sec. 3.1: 5 sub-cycles for every particle against
        # at least 2 kicks and up to two more levels, d = 20
        line["multilevel_paper"] = run_multilevel(torch, hacc, ctx, split, workload="zel128", d=20, lmin=2, lmax=4,
                                                  n_plain=5, dt=0.02, skin=0.1)
        line["fine_mesh"] = run_fine_mesh(torch, hacc, ctx, split, pos, L)
    if not args.no_served:
        rates = [float(x) for x in args.served_rates.split(",") if x]
        rows, sat = run_served_sweep(torch, hacc, ctx, split, rates, args.served_window, args.served_cap, peak,
                                     variant=tuning["variant"])
        top = rows[-1]
        line["served"] = {"sweep": rows, "saturation": sat,
                          "vs_plain_pairs_per_s": top.get("pair_interactions_per_s_device", 0.0) / (within / secs),
                          "window_note": "arrival windows of %g s per rate (C5 specifies 60 s), each rate capped at "
                                         "%g s of wall time" % (args.served_window, args.served_cap)}
    if not args.no_c1:
        line["c1"] = run_c1(torch, hacc, ctx, split, peak, tuning)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import split as osplit
        sp = osplit.default_split()
        sp["r_cut"] = float(np.float32(sp["r_cut"]))
        sp["eps"] = float(np.float32(sp["eps"]))
        # the initial conditions of the workload, the state the reference arm samples too
        host = pos_np
        cb = cpu_oracle_rate(host, L, sp, target_s=args.cpu_seconds)
        line["cpu_baseline"] = {"value": cb["value"], "unit": "pair interactions/s", "cores": cb["threads"],
                                "kind": "oracle",
                                "sample": "FP64 short-range force of %d random particles of the initial conditions "
                                          "(all %d particles as sources, %.1f s)" % (cb["sample_particles"], n,
                                                                                     cb["seconds"])}
        # the same on one core (a shorter sample)
        import oracle
        all_threads = oracle.threads()
        oracle.set_threads(1)
        try:
            c1 = cpu_oracle_rate(host, L, sp, target_s=max(2.0, args.cpu_seconds / 2))
        finally:
            oracle.set_threads(all_threads)
        line["cpu_baseline"]["single_core"] = {"value": c1["value"], "sample_particles": c1["sample_particles"],
                                               "seconds": c1["seconds"]}
    ctx.close()
    if not args.no_c3 and world == 1:
        torch.cuda.empty_cache()
        line["precision"] = precision_segment(torch, hacc)
    line["summary"] = summary(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_precision(args):
    """Precision study: the same FP64 Zel'dovich positions (side^3 particles,
    box `side`, seed 3) as FP32 absolute coordinates and as (cell id, FP32
    in-cell offset); pair forces of both against the FP64 oracle on a seeded
    random sample of particles (all particles as sources); device times of
    the force and of 5 SKS sub-cycles in both forms."""
    import numpy as np
    import torch

    import oracle
    import paper_1410_2805_gb300 as hacc
    import synth
    from oracle import split as osplit
    from paper_1410_2805_gb300 import build as hbuild

    hbuild.build()
    side = args.precision_side
    L = float(side)
    x64 = synth.zeldovich(side, seed=3, L=L, return_f64=True)
    n = len(x64)
    p32 = np.ones((n, 4), np.float32)
    p32[:, :3] = x64.astype(np.float32)
    p32[:, :3][p32[:, :3] >= np.float32(L)] = 0
    vel = synth.gaussian_velocities(n, seed=3, sigma=0.1)
    ctx = hacc.Context(0)
    split = hacc.default_split()
    box = hacc.Box(L=L)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    P = torch.from_numpy(p32).cuda()
    X = torch.from_numpy(x64).cuda()
    cell, off = ctx.ci_from_f64(box, split.r_cut, X)
    out = {}
    acc32 = ctx.sr_force(box, split, P)
    out["force_ms_fp32_abs"] = timed(lambda: ctx.sr_force(box, split, P, acc=acc32), 3)
    acc_ci = ctx.sr_force_ci(box, split, cell, off)
    out["force_ms_cell_offset"] = timed(lambda: ctx.sr_force_ci(box, split, cell, off), 3)
    ctx.sync()
    a32 = acc32.cpu().numpy()[:, :3].astype(np.float64)
    aci = acc_ci.cpu().numpy()[:, :3].astype(np.float64)
    # 5 sub-cycles of step 0.1 in both forms (copies, so the positions above stay)
    P2, V2 = P.clone(), torch.from_numpy(vel).cuda()
    C2, O2, V3 = cell.clone(), off.clone(), torch.from_numpy(vel).cuda()
    out["subcycle5_ms_fp32_abs"] = timed(lambda: ctx.subcycle(box, split, P2, V2, 0.5, 5), 1)
    out["subcycle5_ms_cell_offset"] = timed(lambda: ctx.subcycle_ci(box, split, C2, O2, V3, 0.5, 5), 1)
    ctx.sync()
    ctx.close()
    del P, X, P2, V2, C2, O2, V3, acc32, acc_ci
    sp = osplit.default_split()
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    sp["eps"] = float(np.float32(sp["eps"]))
    sel = np.sort(np.random.default_rng(33).choice(n, size=min(n, args.precision_sample), replace=False))
    t0 = time.perf_counter()
    pos64 = np.concatenate([x64, np.ones((n, 1))], axis=1)
    del x64
    ref, _ = oracle.force_mesh(pos64, L, sp, sel=sel)
    t_or = time.perf_counter() - t0
    rms = float(np.sqrt((ref ** 2).sum(1).mean()))

    amag = np.sqrt((ref ** 2).sum(1))

    def errs(a):
        d = np.sqrt(((a[sel] - ref) ** 2).sum(1))
        worst = int(np.argmax(d))
        big = amag > 0.01 * rms
        return {"max_rel_to_rms": float(d.max() / rms), "rms_rel_to_rms": float(np.sqrt((d ** 2).mean()) / rms),
                "worst_particle_abs_a_over_rms": float(amag[worst] / rms),
                "worst_particle_own_rel_err": float(d[worst] / max(amag[worst], 1e-300)),
                "max_own_rel_err_abs_a_over_1pct_rms": float((d[big] / amag[big]).max()),
                "p99_own_rel_err": float(np.percentile(d[big] / amag[big], 99))}

    out.update({"particles": n, "box": L, "sample": int(len(sel)), "oracle_s": t_or, "oracle_threads": oracle.threads(),
                "error_fp32_abs": errs(a32), "error_cell_offset": errs(aci)})
    print(json.dumps({"precision_study": out, "workload": "%d^3 Zel'dovich, box %d, seed 3" % (side, side)}),
          flush=True)
    return 0


def main():
    args = parse()
    if args.precision:
        return run_precision(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
