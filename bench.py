#!/usr/bin/env python3
"""Benchmark of the dose engine on one GB300: photon histories per second,
seconds to 1 % avg RSD, and the served form's p50/p99 latency.

A step is one complete dose calculation of the workload through the C ABI:
source sampling, Woodcock transport, interactions and tallies for every
history in N_b batches, the batch folds and the avg-RSD reduction.  Its inputs
(phantom, tables) are resident in HBM; between timed steps L2 is flushed by
writing a 256 MB buffer, outside the timed events.

Default workload: the CBCT water phantom, 256x256x128 voxels of 0.2 cm,
120 kVp, 360 projections, 1e9 histories in 10 batches.  The same JSON line
also carries, each measured in this run:
  head      the head phantom (256x256x160 x 0.1 cm, 100 kVp half fan, 2e9
            histories): histories/s, seconds to 1 % avg RSD, roofline;
  batched   64 uneven requests (64^3-256^3 water and head, 80-140 kVp, 1e7-1e9
            histories): request chains in one CUDA graph and one shared launch
            per batch, against the same requests run one after another;
  served    a Poisson stream of head requests, each stopped at 1 % avg RSD:
            p50/p99 latency and histories/s, continuous batching against one
            request at a time; GPU-filling requests (0.5 cm heads, batches of
            8e7 histories) and small ones (1 cm heads, batches of 4e6);
  error_vs_fp64_oracle  the device against the binary64 oracle on the CPU
            baseline's sample (the same histories on both sides).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--legs ...]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Prints one JSON line (rank 0).  Under torchrun the ranks share one problem of
N x 1e9 histories, each rank transporting its share of every batch, with one
binary64 sum of each batch's tally across ranks (NCCL) before the fold;
value = all histories / max-over-ranks time.
"""
import argparse
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

METRIC = "photon histories/sec and sec-to-1% avg RSD on 1 GB300; served p50/p99 latency"
UNIT = "histories/s"
SM_COUNT = 152
LANES_PER_SM_CLK = 128          # 4 schedulers x 32 lanes issue per SM clock
FLUSH_BYTES = 256 * 1024 * 1024

# Transport-kernel figures from one ncu capture (--set full, --clock-control none)
# of one launch of the same workload: lane instructions per history
# (smsp__thread_inst_executed / histories) and DRAM bytes per launch
# (dram__bytes_read + dram__bytes_write); they are not measured in this run.
KERNEL_PROFILE = {
    "cbct_water": {"lane_inst_per_history": 2088.0, "dram_bytes_per_launch": 4.345e9, "histories_per_launch": 1e8,
                   "capture": "ncu --set full --clock-control none of one transport_kernel<256,4,0,0> launch of 1e8 "
                              "CBCT-water histories (packed-voxel kernel): 8.688e9 warp instructions x 24.03 lanes; "
                              "DRAM 1.91 + 2.43 GB"},
    "head": {"lane_inst_per_history": 2450.0, "dram_bytes_per_launch": 4.465e9, "histories_per_launch": 2e8,
             "capture": "ncu --set full --clock-control none of one transport_kernel<256,4,0,0> launch of 2e8 head "
                        "histories (packed-voxel kernel): 2.656e10 warp instructions x 18.45 lanes; DRAM 2.53 + 1.94 GB"},
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(name, compton="kn", rayleigh="gauss", n_hist=None):
    """The named workload; compton "wh" switches it to the Waller-Hartree model,
    rayleigh "iaa" to the independent-atom form factor of its materials' elements."""
    import dataclasses

    from paper_1109_3266_gb300 import inputs as I
    makers = {"cbct_water": I.cbct_water, "head": I.head, "tiny_water": I.tiny_water,
              "cbct_water_bowtie": lambda: dataclasses.replace(I.cbct_water(bowtie=True), name="cbct_water_bowtie")}
    if name not in makers:
        raise SystemExit(f"unknown workload {name}")
    p = makers[name]()
    if compton != "kn" or rayleigh != "gauss":
        p = I.scaled(p, physics=dataclasses.replace(p.physics, compton=compton, rayleigh=rayleigh))
    if n_hist is not None:
        p = I.scaled(p, n_hist=n_hist)
    return p


class Clocks:
    """nvidia-smi clock and throttle sampling; summaries over marked windows."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def mark(self):
        return len(self.lines)

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.proc = None

    def summary(self, a=0, b=None):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[a:b] if b is not None else self.lines[a:]
        if not lines:   # a window shorter than one sample: the nearest sample
            lines = self.lines[max(0, a - 1):a + 1]
        for l in lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("CTD_BENCH_BACKEND", "nccl")
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# --------------------------------------------------------------------------- CPU oracle
def oracle_sample(p, seconds, threads, n_ranges=64, keep=False):
    """Histories/s of the binary64 oracle as it stands on a bounded sample of the
    workload: n_ranges equal history ranges spread evenly through the first batch,
    so that the sample covers the whole spectrum (histories run in 1 keV bin order).
    Returns (rate, histories, seconds, ranges, deposits, counts) of the last sample."""
    from oracle import oracle as O
    s = O.Setup(p, 64)
    batch = p.n_hist // p.n_batches

    def sample(n):
        per = max(1, n // n_ranges)
        ranges = [((batch * k) // n_ranges, min((batch * k) // n_ranges + per, p.n_hist)) for k in range(n_ranges)]
        t0 = time.perf_counter()
        edep, c = s.transport_ranges(ranges, threads)
        return per * n_ranges, time.perf_counter() - t0, ranges, edep, c

    n = 64 * n_ranges
    while True:
        done, dt, ranges, edep, c = sample(n)
        if dt > 0.5 or n >= batch:
            break
        n *= 4
    # size the sample from the probe's rate, then once more from the sample's own
    # rate if the first estimate (small samples pay thread start-up) fell short
    n = int(max(n_ranges, min(batch, done / max(dt, 1e-6) * seconds)))
    done, dt, ranges, edep, c = sample(n)
    if dt < 0.6 * seconds and n < batch:
        n = int(max(n_ranges, min(batch, done / max(dt, 1e-6) * seconds)))
        done, dt, ranges, edep, c = sample(n)
    return done / dt, done, dt, ranges, (edep if keep else None), c


def run_reference(args):
    rank, world = dist_init(args.gpus)
    if rank != 0:
        return
    p = workload(args.workload, args.compton, args.rayleigh)
    threads = cpu_cores()
    # each step a bounded sample, so that the whole run ends within a few minutes
    per_step = max(2.0, min(args.ref_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(p, 0.5, threads)
    rates, ns = [], []
    for _ in range(args.steps):
        r, n, dt, _, _, _ = oracle_sample(p, per_step, threads)
        rates.append(r)
        ns.append(n)
    value = float(np.mean(rates))
    sample = (f"binary64 oracle, {ns[0]} histories of {p.name} per step in 64 equal ranges spread through "
              f"batch 0 (all 1 keV bins), {threads} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * ns[0] / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": p.name, "histories_per_step": ns[0], "compton": args.compton,
                   "rayleigh": args.rayleigh},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# --------------------------------------------------------------------------- measurement pieces
def timed_runs(ctd, ctx, h, p, seed, steps, warmup, ramp_s, stream, flush, sync, clk=None):
    """An untimed clock ramp (runs for ramp_s seconds, so that an idle GPU has reached
    its clocks), exactly `warmup` warm-up runs, then `steps` runs timed with CUDA
    events on the launching stream, L2 flushed between them outside the events."""
    import torch

    def step():
        ctd.ctd_run(ctx, h, p.n_hist, seed, p.n_batches)

    t0, ramp = time.perf_counter(), 0
    while time.perf_counter() - t0 < ramp_s and ramp < 200:
        step()
        ramp += 1
    ramp_t = time.perf_counter() - t0
    for _ in range(warmup):
        step()
        flush.zero_()
    sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t_transport, launches, stats = 0.0, 0, None
    a = clk.mark() if clk else 0
    for i in range(steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        _, _, stats = ctd.ctd_get_dose_and_stddev(ctx, h, 0, want_arrays=False)
        t_transport += stats["t_transport_s"]
        launches += stats["transport_launches"]
        flush.zero_()
    torch.cuda.synchronize()
    b = clk.mark() if clk else 0
    t_dev = sum(x.elapsed_time(y) for x, y in ev) * 1e-3
    return {"t_dev": t_dev, "t_transport": t_transport, "launches": launches, "stats": stats,
            "ramp": {"seconds": ramp_t, "runs": ramp}, "clocks": clk.summary(a, b) if clk else None}


def rsd_stopped(ctd, ctx, h, p, seed, rsd, sec_run, parts=10):
    """Seconds to 1 % avg RSD, measured with the RSD-stopped served form: batches of
    1/parts of the extrapolated need N (RSD / 1 %)^2, stopped at 1 % after >= 10
    batches (the stop overshoots the need by up to one batch)."""
    import torch
    n_1 = p.n_hist * (rsd / 0.01) ** 2
    B = int(max(1e6, n_1 / parts))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rid = ctd.ctd_submit(ctx, h, B, 0.01, seed + 1, n_histories_max=int(40 * B))
    st = ctd.ctd_wait(ctx, rid, 600.0)
    return {"seconds": time.perf_counter() - t0, "histories": st["histories"], "batches": st["batches"],
            "avg_rsd": st["avg_rsd"], "batch_histories": B,
            "extrapolated_seconds": sec_run * (rsd / 0.01) ** 2}


def memory_probes(ctd, ctx, nvox):
    """Memory ceilings measured on this GPU by the library's probes over as many slots
    as the phantom has voxels: binary64 reductions into random tally slots and random
    4-byte gathers (a Woodcock step fetches its voxel's packed 4-byte word)."""
    n_ops = 1 << 31
    return {"l2_red_per_s": ctd.ctd_probe_memory(ctx, ctd.PROBE_L2_RED, nvox, n_ops),
            "gather4_per_s": ctd.ctd_probe_memory(ctx, ctd.PROBE_GATHER4, nvox, n_ops),
            "probe": f"{n_ops} operations on uniform random slots of {nvox} voxels "
                     f"({nvox * 8 / 1e6:.0f} MB binary64 tally, {nvox * 4 / 1e6:.0f} MB packed voxel words), "
                     f"mean of 3 launches after 1"}


def roofline(p, run, peaks, peak_kind, probes, prof):
    """The transport kernel against its ceilings.  frac: the algorithmic bytes of a
    history -- 5 B per Woodcock step (material byte + binary32 density, which the
    kernel reads as one packed 4-byte word) and 8 B per deposit (a binary64
    reduction) -- over one launch's histories and its average launch time, against
    the measured HBM copy bandwidth.  Beside it the L2-reduction and voxel-gather
    (4-byte gather probe) fractions of the probes' ceilings, and the SM-issue
    fraction."""
    st = run["stats"]
    n = st["histories"]
    launches = max(run["launches"], 1)
    t_launch = run["t_transport"] / launches
    hist_launch = n / st["transport_launches"]
    steps_h = st["steps"] / n
    dep_h = (st["pe"] + st["compton"]) / n
    bytes_h = 5.0 * steps_h + 8.0 * dep_h
    achieved = bytes_h * hist_launch / t_launch / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    traffic = prof.get("dram_bytes_per_launch") if prof else None
    out = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
           "traffic": traffic * hist_launch / prof["histories_per_launch"] if traffic else None,
           "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
           "kernel": "transport_kernel", "launches": run["launches"], "avg_launch_ms": 1e3 * t_launch,
           "histories_per_launch": hist_launch, "bytes_per_history": bytes_h,
           "steps_per_history": steps_h, "deposits_per_history": dep_h,
           "algorithmic_bytes_per_launch": bytes_h * hist_launch}
    hist_s = hist_launch / t_launch
    if probes:
        out["l2_reduction"] = {"achieved_per_s": hist_s * dep_h, "peak_per_s": probes["l2_red_per_s"],
                               "frac": hist_s * dep_h / probes["l2_red_per_s"]}
        out["voxel_gather"] = {"achieved_per_s": hist_s * steps_h, "peak_per_s": probes["gather4_per_s"],
                               "frac": hist_s * steps_h / probes["gather4_per_s"]}
        out["probe"] = probes["probe"]
    mhz = peaks.get("sm_max_mhz", 2070.0)
    ipeak = SM_COUNT * LANES_PER_SM_CLK * mhz * 1e6 / 1e12
    lih = prof.get("lane_inst_per_history") if prof else None
    out["issue"] = {"lane_inst_per_history": lih, "achieved_t_per_s": hist_s * lih / 1e12 if lih else None,
                    "peak_t_per_s": ipeak, "frac": hist_s * lih / 1e12 / ipeak if lih else None,
                    "peak_source": f"{SM_COUNT} SM x {LANES_PER_SM_CLK} lanes x {mhz:.0f} MHz",
                    "source": (prof or {}).get("capture")}
    return out


def error_vs_oracle(ctd, ctx, h, p, ranges, o_edep, o_counts):
    """The device over the oracle's sample (the same histories): relative error of the
    total deposit, of each voxel's deposit above 10 % of the maximum, and of the counts."""
    for i, (a, b) in enumerate(ranges):
        ctd.ctd_run_range(ctx, h, p.n_hist, p.seed, p.n_batches, a, b, clear=(i == 0))
    _, _, st = ctd.ctd_get_dose_and_stddev(ctx, h, 0, want_arrays=False)
    ed = ctd.ctd_get_edep(ctx, h, p.phantom.nvox)
    m = o_edep > 0.1 * o_edep.max()
    rel = np.abs(ed[m] - o_edep[m]) / o_edep[m]
    counts = {k: {"device": int(st[k]), "oracle": int(o_counts[k]),
                  "rel": (st[k] - o_counts[k]) / max(o_counts[k], 1)}
              for k in ("pe", "compton", "rayleigh", "fictitious", "escaped", "missed")}
    return {"histories": int(sum(b - a for a, b in ranges)), "sample": "the CPU baseline's sample, same histories",
            "total_edep_rel": float((st["e_deposited_kev"] - o_counts["e_deposited"]) / o_counts["e_deposited"]),
            "voxel_edep_rel_median": float(np.median(rel)), "voxel_edep_rel_p99": float(np.percentile(rel, 99)),
            "voxel_edep_rel_max": float(rel.max()), "voxels": int(m.sum()), "counts": counts,
            "note": "the same histories on both sides: the differences are binary32 against binary64 rounding, "
                    "and a voxel's largest difference is one history that took another path"}


def e2e_rate(ctd, ctx, p, seed, steps, world, dev):
    """The same metric end to end through the public API with host buffers: phantom
    upload from pinned memory, set-up, run, read-back of dose and stddev, release."""
    import torch
    nvox = p.phantom.nvox
    mat_h = torch.from_numpy(np.ascontiguousarray(p.phantom.mat).ravel()).pin_memory().numpy()
    rho_h = torch.from_numpy(np.ascontiguousarray(p.phantom.rho).ravel()).pin_memory().numpy()
    dose_h = torch.empty(nvox, dtype=torch.float64).pin_memory().numpy()
    sd_h = torch.empty(nvox, dtype=torch.float64).pin_memory().numpy()
    st = ctd.ctd_run_stats()
    L = ctd.lib()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        ph = p.phantom
        h2 = ctd.ctd_create_phantom(ctx, ph.nx, ph.ny, ph.nz, ph.dx, ph.dy, ph.dz, mat_h, rho_h, ph.materials)
        s = p.source
        ctd.ctd_set_source(ctx, h2, s.kind, s.sad, s.u_lo, s.u_hi, s.v_lo, s.v_hi, s.n_proj, s.arc0, s.arc1,
                           s.continuous, s.z0, s.z1)
        ctd.ctd_set_spectrum(ctx, h2, p.spectrum.e_lo, p.spectrum.e_hi, p.spectrum.w)
        if s.fluence is not None:
            ctd.ctd_set_fluence(ctx, h2, s.fluence)
        phy = p.physics
        ctd.ctd_set_physics(ctx, h2, phy.e_min, phy.e_max, phy.n_zeta, phy.majorant_scale, phy.mode, phy.max_real,
                            phy.compton)
        if phy.rayleigh == "iaa":
            for m, mat in enumerate(ph.materials):
                ctd.ctd_set_material_elements(ctx, h2, m, mat.elements)
        ctd.ctd_run(ctx, h2, p.n_hist, seed, p.n_batches)
        ctd._check(L.ctd_get_dose_and_stddev(ctx, h2, ctd._dp(dose_h), ctd._dp(sd_h), nvox, ctd.C.byref(st)))
        ctd.ctd_destroy_phantom(ctx, h2)
    t = max_over_ranks(time.perf_counter() - t0, world, dev)
    return {"value": sum_over_ranks(float(p.n_hist * steps), world, dev) / t, "unit": UNIT,
            "h2d_bytes_per_step": nvox * (1 + 4) + 3 * 8 * len(p.spectrum.w), "d2h_bytes_per_step": nvox * 16,
            "steps": steps}


# --------------------------------------------------------------------------- legs
def leg_head(ctd, args, stream, flush, peaks, peak_kind, clk):
    """The head workload: histories/s over a few timed runs, seconds to 1 %, roofline,
    error against the oracle on a short sample."""
    import torch
    p = workload("head", args.compton, args.rayleigh)
    ctx = ctd.ctd_create(device=0, stream=stream.cuda_stream, blocks_per_sm=args.blocks_per_sm,
                         threads_per_block=args.threads, chunk=args.chunk, flight_cap=args.flight_cap,
                         l2_persist=args.l2_persist, plain_overlap=args.plain_overlap)
    h = ctd.load_problem(ctx, p)
    run = timed_runs(ctd, ctx, h, p, p.seed, args.head_steps, 2, 0.0, stream, flush, torch.cuda.synchronize, clk)
    st = run["stats"]
    sec_run = run["t_dev"] / args.head_steps
    out = {"workload": "head", "voxels": [p.phantom.nx, p.phantom.ny, p.phantom.nz], "voxel_cm": p.phantom.dx,
           "histories_per_step": p.n_hist, "steps": args.head_steps, "value": p.n_hist * args.head_steps / run["t_dev"],
           "unit": UNIT, "ms_per_step": 1e3 * sec_run, "avg_rsd": st["avg_rsd"], "clocks": run["clocks"]}
    out["sec_to_1pct_avg_rsd_extrapolated"] = sec_run * (st["avg_rsd"] / 0.01) ** 2
    if args.rsd_stop:
        r = rsd_stopped(ctd, ctx, h, p, p.seed, st["avg_rsd"], sec_run, args.rsd_parts)
        out["sec_to_1pct_avg_rsd"] = r["seconds"]
        out["rsd_stopped_run"] = r
    probes = None if args.no_probe else memory_probes(ctd, ctx, p.phantom.nvox)
    out["roofline"] = roofline(p, run, peaks, peak_kind, probes, KERNEL_PROFILE.get("head"))
    if not args.no_cpu_baseline:
        _, _, _, ranges, edep, c = oracle_sample(p, 3.0, cpu_cores(), keep=True)
        out["error_vs_fp64_oracle"] = error_vs_oracle(ctd, ctx, h, p, ranges, edep, c)
    out["gpu_launches"] = run["launches"] + 17 * args.head_steps
    ctd.ctd_destroy_phantom(ctx, h)
    ctd.ctd_destroy(ctx)
    return out


def leg_batched(ctd, args, clk):
    """Uneven requests: request chains in one CUDA graph and one shared launch per
    batch (batched form) against the same requests one ctd_run after another (plain
    single-request form)."""
    import torch

    from paper_1109_3266_gb300 import inputs as I
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sides = tuple(range(64, args.max_side + 1, 32))
    reqs = I.batched_requests(args.n_requests, hist_lo=args.hist_lo, hist_hi=args.hist_hi, sides=sides)
    ctxs = [ctd.ctd_create(device=0, stream=stream.cuda_stream, blocks_per_sm=args.blocks_per_sm,
                           threads_per_block=args.threads, chunk=args.chunk, flight_cap=args.flight_cap,
                           multi_blocks_per_sm=args.multi_blocks_per_sm, shared_launch=k,
                           batch_lanes=args.batch_lanes) for k in (0, 1)]
    hss = [[ctd.load_problem(c, p) for p in reqs] for c in ctxs]
    ctx, hs = ctxs[0], hss[0]
    n_total = sum(p.n_hist for p in reqs)
    nb = 10

    def batched(k=0):
        ctd.ctd_run_batch(ctxs[k], hss[k], [p.n_hist for p in reqs], [p.seed for p in reqs], nb)

    def plain():
        for h, p in zip(hs, reqs):
            ctd.ctd_run(ctx, h, p.n_hist, p.seed, nb)

    def timed(fn, k):
        ts = []
        for _ in range(k):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) * 1e-3)
        return ts

    timed(batched, 1)
    timed(lambda: batched(1), 1)
    # the batched form's autotuner on a 5 % probe of the same requests, in a third context
    ctxs.append(ctd.ctd_create(device=0, stream=stream.cuda_stream))
    hss.append([ctd.load_problem(ctxs[2], p) for p in reqs])
    t0 = time.perf_counter()
    tune = ctd.ctd_autotune_batch(ctxs[2], hss[2], [p.n_hist for p in reqs], [p.seed for p in reqs], nb, 0.04)
    tune["seconds"] = time.perf_counter() - t0
    timed(lambda: batched(2), 1)
    a = clk.mark()
    tb = timed(batched, args.batched_reps)
    ts = timed(lambda: batched(1), args.batched_reps)
    tt = timed(lambda: batched(2), args.batched_reps)
    tp = timed(plain, args.batched_reps)
    b = clk.mark()
    rsd = [ctd.ctd_get_dose_and_stddev(ctx, h, 0, want_arrays=False)[2]["avg_rsd"] for h in hs]
    vb, vs, vt, vp = (n_total / float(np.mean(t)) for t in (tb, ts, tt, tp))
    for c, hl in zip(ctxs, hss):
        for h in hl:
            ctd.ctd_destroy_phantom(c, h)
        ctd.ctd_destroy(c)
    return {"workload": "batched", "requests": len(reqs), "histories_per_step": n_total, "batches": nb,
            "sides": sorted({p.meta["side"] for p in reqs}), "hist_range": [args.hist_lo, args.hist_hi],
            "reps": args.batched_reps, "chains_value": vb, "shared_launch_value": vs, "autotuned_value": vt,
            "plain_value": vp, "unit": UNIT, "chains_speedup_vs_plain": vb / vp,
            "shared_launch_speedup_vs_plain": vs / vp, "autotuned_speedup_vs_plain": vt / vp, "autotuner": tune,
            "chains_ms": 1e3 * float(np.mean(tb)), "shared_launch_ms": 1e3 * float(np.mean(ts)),
            "plain_ms": 1e3 * float(np.mean(tp)), "avg_rsd_range": [float(min(rsd)), float(max(rsd))],
            "launches": "chains: one chain of single-request launches per request on its own stream, one CUDA "
                        "graph; shared: one multi-request launch per batch", "clocks": clk.summary(a, b)}


def served_stream(ctd, args, clk, d, batch, rate, n_req):
    """One Poisson stream of head requests of d cm voxels, each stopped at 1 %
    avg RSD in batches of `batch` histories: continuous batching (every request
    on its own stream) against one request at a time, on the same arrivals."""
    from paper_1109_3266_gb300 import inputs as I, serve
    nx, ny, nz = int(round(25.6 / d)), int(round(25.6 / d)), int(round(16.0 / d))
    pool = [I.head_phantom(nx, ny, nz, d, seed=3 + k) for k in range(args.pool)]
    arrivals = I.served_arrivals(n_req, rate, seed=5)

    def make(seed):
        return I.head_request(pool[seed % len(pool)], seed)

    out = {}
    for label, max_active, budget in (("continuous", 0, args.round_histories), ("one_at_a_time", 1, 0.0)):
        ctx = ctd.ctd_create(device=0, multi_blocks_per_sm=args.multi_blocks_per_sm, serve_max_active=max_active,
                             shared_launch=args.shared_launch, serve_round_histories=budget)
        # warm-up: one request alone
        serve.serve(ctx, [(0.0, 4999)], make, batch, 0.01, n_histories_max=40 * batch)
        a = clk.mark()
        reqs, wall = serve.serve(ctx, arrivals, make, batch, 0.01, n_histories_max=40 * batch,
                                 time_limit_s=args.time_limit)
        b = clk.mark()
        done = [r for r in reqs if np.isfinite(r.latency)]
        hist = sum(r.histories for r in done)
        out[label] = dict(serve.latency_summary(reqs), histories_per_s=hist / wall, wall_s=wall,
                          submitted=len(reqs), mean_batches=float(np.mean([r.batches for r in done])) if done else None,
                          mean_histories=float(np.mean([r.histories for r in done])) if done else None,
                          round_histories=budget or 1e8, clocks=clk.summary(a, b))
        ctd.ctd_destroy(ctx)
    c, o = out["continuous"], out["one_at_a_time"]
    return {"phantom": [nx, ny, nz], "voxel_cm": d, "rate_per_s": rate, "requests": n_req, "batch_histories": batch,
            "rsd_target": 0.01, "min_batches": 10, "phantom_pool": args.pool, "p50_s": c["p50_s"], "p99_s": c["p99_s"],
            "value": c["histories_per_s"], "unit": UNIT,
            "launches": "shared multi-request launch" if args.shared_launch else "one stream per request",
            "continuous": c, "one_at_a_time": o,
            "throughput_vs_one_at_a_time": (c["histories_per_s"] / o["histories_per_s"]) if o["histories_per_s"]
            else None,
            "p50_vs_one_at_a_time": (c["p50_s"] / o["p50_s"]) if c["p50_s"] and o["p50_s"] else None,
            "p99_vs_one_at_a_time": (c["p99_s"] / o["p99_s"]) if c["p99_s"] and o["p99_s"] else None}


def leg_served(ctd, args, clk):
    """Poisson streams of head requests, each stopped at 1 % avg RSD: continuous
    batching against one request at a time, for requests whose batches fill the
    GPU and for small ones."""
    import torch

    torch.cuda.set_device(0)
    out = served_stream(ctd, args, clk, args.served_voxel_cm, args.batch_histories, args.rate, args.served_requests)
    out["workload"] = "served"
    out["stand_in"] = (f"heads of {args.served_voxel_cm} cm voxels instead of the 0.1 cm ones: one 0.1 cm head needs "
                       "about 1e11 histories to reach 1 % (about 15 s of this GPU), so 4 requests/s would be about 60x "
                       "over its capacity and every latency would be queueing")
    if args.served_small_requests > 0:
        out["small_requests"] = served_stream(ctd, args, clk, args.served_small_voxel_cm, args.served_small_batch,
                                              args.served_small_rate, args.served_small_requests)
    return out


# --------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch

    from paper_1109_3266_gb300 import ctd

    rank, world = dist_init(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    peaks, peak_kind = load_peaks()
    # the clock sampler starts before any GPU work, so that its start-up is not timed
    clk = Clocks(local).__enter__()

    def sync():
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()

    if world > 1:
        from paper_1109_3266_gb300 import shard
        p = workload(args.workload, args.compton, args.rayleigh, n_hist=1_000_000_000 * world)
        ctx = ctd.ctd_create(device=local, stream=stream.cuda_stream, blocks_per_sm=args.blocks_per_sm,
                             threads_per_block=args.threads, chunk=args.chunk, flight_cap=args.flight_cap)
        h = ctd.load_problem(ctx, p)
        reduce = shard.nccl_allreduce(dev)
        for _ in range(args.warmup):
            shard.run_sharded(ctd, ctx, h, p.n_hist, p.seed, p.n_batches, rank, world, reduce, dev,
                              nvox=p.phantom.nvox)
            flush.zero_()
        sync()
        a = clk.mark()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            ev[i][0].record(stream)
            st = shard.run_sharded(ctd, ctx, h, p.n_hist, p.seed, p.n_batches, rank, world, reduce, dev)
            ev[i][1].record(stream)
            flush.zero_()
        sync()
        b = clk.mark()
        t_dev = sum(x.elapsed_time(y) for x, y in ev) * 1e-3
        t_max = max_over_ranks(t_dev, world, dev)
        if rank == 0:
            print(json.dumps({
                "metric": METRIC, "value": p.n_hist * args.steps / t_max, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": p.name, "histories_per_step": p.n_hist, "batches": p.n_batches,
                           "parallelism": f"history shards x{world}, one binary64 all-reduce of each batch tally",
                           "l2": "flushed between steps (256 MB write outside timed events)"},
                "avg_rsd": st["avg_rsd"], "clocks": clk.summary(a, b),
                "gpu_launches": None,
            }), flush=True)
        clk.__exit__(None, None, None)
        ctd.ctd_destroy(ctx)
        return

    p = workload(args.workload, args.compton, args.rayleigh)
    nvox = p.phantom.nvox
    ctx = ctd.ctd_create(device=local, stream=stream.cuda_stream, blocks_per_sm=args.blocks_per_sm,
                         threads_per_block=args.threads, chunk=args.chunk, flight_cap=args.flight_cap,
                         l2_persist=args.l2_persist, plain_overlap=args.plain_overlap)
    h = ctd.load_problem(ctx, p)
    run = timed_runs(ctd, ctx, h, p, p.seed, args.steps, args.warmup, args.ramp_seconds, stream, flush, sync, clk)
    st = run["stats"]
    t_dev = run["t_dev"]
    value = p.n_hist * args.steps / t_dev
    sec_run = t_dev / args.steps
    rsd = st["avg_rsd"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sec_run, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": p.name, "voxels": [p.phantom.nx, p.phantom.ny, p.phantom.nz],
                   "voxel_cm": p.phantom.dx, "histories_per_step": p.n_hist, "batches": p.n_batches,
                   "kvp": 120 if p.name.startswith("cbct_water") else 100 if p.name == "head" else None,
                   "parallelism": "one GPU",
                   "l2": "flushed between steps (256 MB write outside timed events)",
                   "blocks_per_sm": args.blocks_per_sm, "threads": args.threads, "chunk": args.chunk,
                   "flight_cap": args.flight_cap, "compton": args.compton, "rayleigh": args.rayleigh},
        "clock_ramp": run["ramp"], "avg_rsd": rsd, "paper_sigma_bar": st["paper_sigma_bar"],
        "sec_to_1pct_avg_rsd_extrapolated": sec_run * (rsd / 0.01) ** 2,
        # Sec. 3.1's simulation efficiency 1 / (sigma_bar^2 T), T the device time of one run
        "paper_efficiency_per_s": (1.0 / (st["paper_sigma_bar"] ** 2 * sec_run) if st["paper_sigma_bar"] > 0
                                   else None),
        "clocks": run["clocks"],
    }
    if args.rsd_stop:
        r = rsd_stopped(ctd, ctx, h, p, p.seed, rsd, sec_run, args.rsd_parts)
        line["sec_to_1pct_avg_rsd"] = r["seconds"]
        line["rsd_stopped_run"] = r
    else:
        line["sec_to_1pct_avg_rsd"] = line["sec_to_1pct_avg_rsd_extrapolated"]
    line["e2e"] = e2e_rate(ctd, ctx, p, p.seed, max(1, min(args.e2e_steps, args.steps)), world, dev)
    probes = None if args.no_probe else memory_probes(ctd, ctx, nvox)
    prof = KERNEL_PROFILE.get(p.name) if args.compton == "kn" and args.rayleigh == "gauss" else None
    line["roofline"] = roofline(p, run, peaks, peak_kind, probes, prof)
    line["gpu_launches"] = run["launches"] + 17 * args.steps
    if not args.no_cpu_baseline:
        threads = cpu_cores()
        r, n, dt, ranges, edep, c = oracle_sample(p, args.ref_seconds, threads, keep=True)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"binary64 oracle, {n} histories of {p.name} in 64 equal ranges spread "
                                          f"through batch 0 (all 1 keV bins), {dt:.1f} s, {threads} threads"}
        line["error_vs_fp64_oracle"] = error_vs_oracle(ctd, ctx, h, p, ranges, edep, c)
    else:
        line["cpu_baseline"] = None
    ctd.ctd_destroy_phantom(ctx, h)
    ctd.ctd_destroy(ctx)
    legs = args.legs.split(",") if args.legs else []
    if "head" in legs:
        line["head"] = leg_head(ctd, args, stream, flush, peaks, peak_kind, clk)
    if "batched" in legs:
        line["batched"] = leg_batched(ctd, args, clk)
    if "served" in legs:
        line["served"] = leg_served(ctd, args, clk)
    clk.__exit__(None, None, None)
    print(json.dumps(line), flush=True)


def run_form(args):
    """--workload batched / served: the leg on its own, as its own JSON line."""
    from paper_1109_3266_gb300 import ctd
    with Clocks(0) as clk:
        out = leg_batched(ctd, args, clk) if args.workload == "batched" else leg_served(ctd, args, clk)
    out.update({"metric": METRIC, "n_gpus": 1, "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic"})
    if args.workload == "batched":
        out["value"] = out["chains_value"]
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cbct_water")
    ap.add_argument("--legs", default=None,
                    help="comma list of head,batched,served (default: all three for cbct_water, none otherwise; "
                         "'' for none)")
    ap.add_argument("--ramp-seconds", type=float, default=2.0, help="untimed runs before the warm-up")
    ap.add_argument("--head-steps", type=int, default=4)
    ap.add_argument("--batched-reps", type=int, default=2)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--flight-cap", type=int, default=0)
    ap.add_argument("--l2-persist", type=int, default=0, help="plain form: tally (1) or voxel words (2) persisting in L2")
    ap.add_argument("--plain-overlap", type=int, default=0, help="plain form: batches on two streams (1; 0 or -1: one stream)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-probe", action="store_true", help="skip the memory-ceiling probes")
    ap.add_argument("--rsd-stop", type=int, default=1, help="measure sec-to-1%% with the RSD-stopped form")
    ap.add_argument("--rsd-parts", type=int, default=10,
                    help="RSD-stopped form: batches of 1/parts of the extrapolated need")
    ap.add_argument("--n-requests", type=int, default=64)
    ap.add_argument("--max-side", type=int, default=256)
    ap.add_argument("--served-requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=4.0)
    ap.add_argument("--pool", type=int, default=4)
    ap.add_argument("--served-voxel-cm", type=float, default=0.5)
    ap.add_argument("--served-small-requests", type=int, default=400, help="served form, small requests (0: none)")
    ap.add_argument("--served-small-rate", type=float, default=40.0)
    ap.add_argument("--served-small-voxel-cm", type=float, default=1.0)
    ap.add_argument("--served-small-batch", type=int, default=4_000_000)
    ap.add_argument("--batch-histories", type=int, default=80_000_000)
    ap.add_argument("--time-limit", type=float, default=120.0)
    ap.add_argument("--multi-blocks-per-sm", type=int, default=0)
    ap.add_argument("--shared-launch", type=int, default=0, help="served form: one shared multi-request launch")
    ap.add_argument("--batch-lanes", type=int, default=0, help="batched form: streams the request chains share")
    ap.add_argument("--round-histories", type=float, default=1e9,
                    help="served form: histories of one batch of every running request admission keeps within")
    ap.add_argument("--compton", default="kn", choices=["kn", "wh"],
                    help="Compton model: free-electron Klein-Nishina or Waller-Hartree")
    ap.add_argument("--rayleigh", default="gauss", choices=["gauss", "iaa"],
                    help="Rayleigh form factor: analytic exp(-q^2/q0^2) or independent-atom of the elements")
    ap.add_argument("--hist-lo", type=float, default=1e7)
    ap.add_argument("--hist-hi", type=float, default=1e9)
    args = ap.parse_args()
    if args.legs is None:
        args.legs = "head,batched,served" if args.workload == "cbct_water" else ""
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("batched", "served"):
        run_form(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
