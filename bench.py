#!/usr/bin/env python3
"""Benchmark of the dose engine: photon histories per second on one GB300.

A step is one complete dose calculation of the workload through the C ABI:
source sampling, Woodcock transport, interactions and tallies for every
history in N_b batches, the batch folds and the avg-RSD reduction.  Its inputs
(phantom, tables) are resident in HBM; between timed steps L2 is flushed by
writing a 256 MB buffer, outside the timed events.

Default workload: the CBCT water phantom, 256x256x128 voxels of 0.2 cm,
120 kVp, 360 projections, 1e9 histories in 10 batches.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica (own seed); value = all histories / max-over-ranks time.
"""
import argparse
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
sys.path.insert(0, ROOT)

METRIC = "photon histories/sec (sec-to-1% avg RSD beside it)"
UNIT = "histories/s"
SM_COUNT = 152
LANES_PER_SM_CLK = 128          # 4 schedulers x 32 lanes issue per SM clock


# Transport-kernel figures from one ncu capture of one launch of the same workload
# (profiles/transport_kernel_*_full.md): lane instructions per history
# (smsp__inst_executed x thread-per-instruction ratio / histories) and DRAM
# bytes per launch (dram__bytes_read + dram__bytes_write).
KERNEL_PROFILE = {
    "cbct_water": {"lane_inst_per_history": 2603.0, "dram_bytes_per_launch": 9.16e9, "histories_per_launch": 1e8},
    "head": {"lane_inst_per_history": 3128.0, "dram_bytes_per_launch": 13.42e9, "histories_per_launch": 2e8},
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(name, compton="kn", rayleigh="gauss"):
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
    return p


class Clocks:
    """nvidia-smi clock and throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def start_window(self):
        """Samples from here on count (the sampler itself may start earlier, so that
        its own start-up does not fall into the timed region)."""
        self.window = [len(self.lines), None]

    def stop_window(self):
        if self.window is not None:
            self.window[1] = len(self.lines)

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

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if self.window is not None:
            a, b = self.window
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


# --------------------------------------------------------------------------- CPU oracle leg
def oracle_rate(p, seconds, threads, n_ranges=64):
    """Histories/s of the binary64 oracle as it stands on a bounded sample of the
    workload: n_ranges equal history ranges spread evenly through the first batch,
    so that the sample covers the whole spectrum (histories run in 1 keV bin order)."""
    from oracle import oracle as O
    s = O.Setup(p, 64)
    batch = p.n_hist // p.n_batches

    def sample(n):
        per = max(1, n // n_ranges)
        ranges = [((batch * k) // n_ranges, min((batch * k) // n_ranges + per, p.n_hist)) for k in range(n_ranges)]
        t0 = time.perf_counter()
        s.transport_ranges(ranges, threads)
        return per * n_ranges, time.perf_counter() - t0

    n = 64 * n_ranges
    while True:
        done, dt = sample(n)
        if dt > 0.5 or n >= batch:
            break
        n *= 4
    # size the sample from the probe's rate, then once more from the sample's own
    # rate if the first estimate (small samples pay thread start-up) fell short
    n = int(max(n_ranges, min(batch, done / max(dt, 1e-6) * seconds)))
    done, dt = sample(n)
    if dt < 0.6 * seconds and n < batch:
        n = int(max(n_ranges, min(batch, done / max(dt, 1e-6) * seconds)))
        done, dt = sample(n)
    return done / dt, done, dt, None


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank, world = dist_init(args.gpus)
    if rank != 0:
        return
    p = workload(args.workload, args.compton, args.rayleigh)
    threads = cpu_cores()
    for _ in range(args.warmup):
        oracle_rate(p, 0.5, threads)
    rates, ns = [], []
    for _ in range(args.steps):
        r, n, dt, _ = oracle_rate(p, args.ref_seconds, threads)
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


# --------------------------------------------------------------------------- GPU leg
def run_ours(args):
    import torch

    from paper_1109_3266_gb300 import ctd

    rank, world = dist_init(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    p = workload(args.workload, args.compton, args.rayleigh)
    seed = p.seed + 7919 * rank
    nvox = p.phantom.nvox
    ctx = ctd.ctd_create(device=local, stream=stream.cuda_stream, blocks_per_sm=args.blocks_per_sm,
                         threads_per_block=args.threads, chunk=args.chunk, flight_cap=args.flight_cap)
    h = ctd.load_problem(ctx, p)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step():
        ctd.ctd_run(ctx, h, p.n_hist, seed, p.n_batches)

    # the clock sampler starts before the warm-up, so that its start-up is not timed;
    # the warm-up runs at least its W steps and at least 2 s, so that an idle GPU has
    # ramped its clocks up before the timed region
    clk = Clocks(local).__enter__()
    t_warm = time.perf_counter()
    warmup_done = 0
    while warmup_done < args.warmup or (time.perf_counter() - t_warm < 2.0 and warmup_done < 100):
        step()
        flush.zero_()
        torch.cuda.synchronize()
        warmup_done += 1
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_transport, launches, stats = 0.0, 0, None
    clk.start_window()
    for i in range(args.steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        _, _, stats = ctd.ctd_get_dose_and_stddev(ctx, h, nvox, want_arrays=False)
        t_transport += stats["t_transport_s"]
        launches += stats["transport_launches"]
        flush.zero_()
    torch.cuda.synchronize()
    clk.stop_window()
    clk.__exit__(None, None, None)
    barrier(world)
    torch.cuda.synchronize()
    t_dev = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    t_max = max_over_ranks(t_dev, world, dev)
    hist_total = sum_over_ranks(float(p.n_hist * args.steps), world, dev)
    value = hist_total / t_max

    # sec-to-1% avg RSD: N scales as RSD^-2 at fixed variance per history (extrapolated),
    # and measured by the RSD-stopped served form: batches of a tenth of the extrapolated
    # count, stopped at 1 % after at least 10 batches
    rsd = stats["avg_rsd"]
    sec_run = t_dev / args.steps
    sec_to_1 = sec_run * (rsd / 0.01) ** 2
    measured_1 = None
    if args.rsd_stop and rank == 0:
        n_1 = p.n_hist * (rsd / 0.01) ** 2
        B = int(max(1e6, n_1 / 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rid = ctd.ctd_submit(ctx, h, B, 0.01, seed + 1, n_histories_max=int(40 * B))
        st1 = ctd.ctd_wait(ctx, rid, 600.0)
        measured_1 = {"seconds": time.perf_counter() - t0, "histories": st1["histories"], "batches": st1["batches"],
                      "avg_rsd": st1["avg_rsd"], "batch_histories": B}

    # end to end through the public API with host buffers: phantom upload, set-up,
    # run and the read-back of dose and stddev, every step
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    mat_h = torch.from_numpy(np.ascontiguousarray(p.phantom.mat).ravel()).pin_memory().numpy()
    rho_h = torch.from_numpy(np.ascontiguousarray(p.phantom.rho).ravel()).pin_memory().numpy()
    dose_h = torch.empty(nvox, dtype=torch.float64).pin_memory().numpy()
    sd_h = torch.empty(nvox, dtype=torch.float64).pin_memory().numpy()
    st = ctd.ctd_run_stats()
    L = ctd.lib()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
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
    t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_value = sum_over_ranks(float(p.n_hist * e2e_steps), world, dev) / t_e2e
    h2d = nvox * (1 + 4) + 3 * 8 * len(p.spectrum.w)
    d2h = nvox * 16

    # roofline of the transport kernel: lane-instructions per history (KERNEL_PROFILE, from
    # the ncu capture) over the SM issue ceiling 152 SM x 128 lanes x clock
    peaks, peak_kind = load_peaks()
    ck = clk.summary()
    mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = SM_COUNT * LANES_PER_SM_CLK * mhz * 1e6 / 1e12        # tera lane-instructions / s
    # the lane-instruction count was measured for the Klein-Nishina model
    prof = KERNEL_PROFILE.get(p.name, {}) if args.compton == "kn" and args.rayleigh == "gauss" else {}
    inst_per_hist = args.inst_per_history or prof.get("lane_inst_per_history")
    achieved = p.n_hist * args.steps * inst_per_hist / t_transport / 1e12 if inst_per_hist else None
    traffic = args.traffic_per_launch or prof.get("dram_bytes_per_launch")
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T lane-inst/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic,
            "lane_inst_per_history": inst_per_hist,
            "kernel": "transport_kernel", "launches": launches,
            "avg_launch_ms": 1e3 * t_transport / max(launches, 1),
            "peak_source": f"{SM_COUNT} SM x {LANES_PER_SM_CLK} lanes x {mhz:.0f} MHz ({peak_kind} max clock)"}
    # memory-side view: algorithmic bytes per history, counted live from this run's steps and deposits
    steps_per_hist = stats["steps"] / p.n_hist
    deposits_per_hist = (stats["pe"] + stats["compton"]) / p.n_hist
    bytes_per_hist = steps_per_hist * 5.0 + deposits_per_hist * 16.0
    roof["memory_side"] = {"bytes_per_history": bytes_per_hist,
                           "achieved_gbs": p.n_hist * args.steps * bytes_per_hist / t_transport / 1e9,
                           "peak_gbs": peaks.get("hbm_gbs"),
                           "atomics_per_s": p.n_hist * args.steps * deposits_per_hist / t_transport,
                           "steps_per_history": steps_per_hist, "deposits_per_history": deposits_per_hist}
    if not args.no_probe:
        # memory ceilings measured on this GPU by the library's probes, over the same
        # number of slots as the phantom: binary64 reductions into random tally slots
        # and random voxel (material + density) gathers
        n_ops = 1 << 31
        red = ctd.ctd_probe_memory(ctx, ctd.PROBE_L2_RED, nvox, n_ops)
        vox = ctd.ctd_probe_memory(ctx, ctd.PROBE_VOXEL, nvox, n_ops)
        g4 = ctd.ctd_probe_memory(ctx, ctd.PROBE_GATHER4, nvox, n_ops)
        ms = roof["memory_side"]
        steps_per_s = p.n_hist * args.steps * steps_per_hist / t_transport
        ms.update({"l2_red_peak_per_s": red, "atomic_frac": ms["atomics_per_s"] / red,
                   "voxel_gather_peak_per_s": vox, "steps_per_s": steps_per_s, "gather_frac": steps_per_s / vox,
                   "gather4_peak_per_s": g4,
                   "probe": f"{n_ops} operations on uniform random slots of {nvox} voxels "
                            f"({nvox * 8 / 1e6:.0f} MB binary64 tally, {nvox * 5 / 1e6:.0f} MB voxels), "
                            f"mean of 3 launches after 1"})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = cpu_cores()
        r, n, dt, _ = oracle_rate(p, args.ref_seconds, threads)
        cpu = {"value": r, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"binary64 oracle, {n} histories of {p.name} in 64 equal ranges spread through batch 0 "
                         f"(all 1 keV bins), {dt:.1f} s, {threads} threads"}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": warmup_done, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": p.name, "voxels": [p.phantom.nx, p.phantom.ny, p.phantom.nz],
                       "voxel_cm": p.phantom.dx, "histories_per_step": p.n_hist, "batches": p.n_batches,
                       "kvp": 120 if p.name.startswith("cbct_water") else 100 if p.name == "head" else None,
                       "parallelism": f"replicas{world}",
                       "l2": "flushed between steps (256 MB write outside timed events)",
                       "blocks_per_sm": args.blocks_per_sm, "threads": args.threads, "chunk": args.chunk,
                       "flight_cap": args.flight_cap, "compton": args.compton, "rayleigh": args.rayleigh},
            "sec_to_1pct_avg_rsd": measured_1["seconds"] if measured_1 else sec_to_1,
            "sec_to_1pct_avg_rsd_extrapolated": sec_to_1, "rsd_stopped_run": measured_1,
            "avg_rsd": rsd, "paper_sigma_bar": stats["paper_sigma_bar"],
            # Sec. 3.1's simulation efficiency 1 / (sigma_bar^2 T), T the device time of one run
            "paper_efficiency_per_s": (1.0 / (stats["paper_sigma_bar"] ** 2 * sec_run)
                                       if stats["paper_sigma_bar"] > 0 else None),
            "clocks": ck,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": launches + 17 * args.steps,
            "roofline": roof,
            "cpu_baseline": cpu,
        }), flush=True)
    ctd.ctd_destroy(ctx)


# --------------------------------------------------------------------------- batched form
def run_batched(args):
    """64 uneven requests: all in shared launches (batched form) against the same
    requests one after another (plain single-request form)."""
    import torch

    from paper_1109_3266_gb300 import ctd, inputs as I

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sides = tuple(range(64, args.max_side + 1, 32))
    reqs = I.batched_requests(args.n_requests, hist_lo=args.hist_lo, hist_hi=args.hist_hi, sides=sides)
    ctxs = [ctd.ctd_create(device=0, stream=stream.cuda_stream, blocks_per_sm=args.blocks_per_sm,
                           threads_per_block=args.threads, chunk=args.chunk, flight_cap=args.flight_cap,
                           multi_blocks_per_sm=args.multi_blocks_per_sm, shared_launch=k) for k in (0, 1)]
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
    with Clocks(0) as clk:
        tb = timed(batched, args.steps)
        ts = timed(lambda: batched(1), max(1, args.steps // 2))
        tp = timed(plain, max(1, args.steps // 2))
    rsd = [ctd.ctd_get_dose_and_stddev(ctx, h, 0, want_arrays=False)[2]["avg_rsd"] for h in hs]
    vb = n_total / float(np.mean(tb))
    vs = n_total / float(np.mean(ts))
    vp = n_total / float(np.mean(tp))
    print(json.dumps({
        "metric": "photon histories/sec, batched form vs plain single-request form", "value": vb, "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": 1e3 * float(np.mean(tb)),
        "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "batched", "requests": len(reqs), "histories_per_step": n_total, "batches": nb,
                   "sides": sorted({p.meta["side"] for p in reqs}), "hist_range": [args.hist_lo, args.hist_hi],
                   "launches": "one chain of single-request launches per request, one CUDA graph"},
        "plain_value": vp, "plain_ms_per_step": 1e3 * float(np.mean(tp)), "speedup_vs_plain": vb / vp,
        "shared_launch_value": vs, "shared_launch_speedup_vs_plain": vs / vp,
        "avg_rsd_range": [float(min(rsd)), float(max(rsd))], "clocks": clk.summary(),
    }), flush=True)
    for c, hl in zip(ctxs, hss):
        for h in hl:
            ctd.ctd_destroy_phantom(c, h)
        ctd.ctd_destroy(c)


# --------------------------------------------------------------------------- served form
def run_served(args):
    """Poisson stream of head requests, each stopped at 1 % avg RSD: continuous
    batching against one request at a time (the plain single-request form)."""
    import torch

    from paper_1109_3266_gb300 import ctd, inputs as I, serve

    torch.cuda.set_device(0)
    d = args.served_voxel_cm
    nx, ny, nz = int(round(25.6 / d)), int(round(25.6 / d)), int(round(16.0 / d))
    pool = [I.head_phantom(nx, ny, nz, d, seed=3 + k) for k in range(args.pool)]
    arrivals = I.served_arrivals(args.n_requests, args.rate, seed=5)

    def make(seed):
        return I.head_request(pool[seed % len(pool)], seed)

    out = {}
    for label, max_active in (("continuous", 0), ("one_at_a_time", 1)):
        ctx = ctd.ctd_create(device=0, multi_blocks_per_sm=args.multi_blocks_per_sm, serve_max_active=max_active,
                             shared_launch=args.shared_launch, serve_round_histories=args.round_histories)
        # warm-up: one request alone
        serve.serve(ctx, [(0.0, 4999)], make, args.batch_histories, 0.01, n_histories_max=40 * args.batch_histories)
        with Clocks(0) as clk:
            reqs, wall = serve.serve(ctx, arrivals, make, args.batch_histories, 0.01,
                                     n_histories_max=40 * args.batch_histories, time_limit_s=args.time_limit)
        done = [r for r in reqs if np.isfinite(r.latency)]
        hist = sum(r.histories for r in done)
        out[label] = dict(serve.latency_summary(reqs), histories_per_s=hist / wall, wall_s=wall,
                          submitted=len(reqs), mean_batches=float(np.mean([r.batches for r in done])) if done else None,
                          mean_histories=float(np.mean([r.histories for r in done])) if done else None,
                          clocks=clk.summary())
        ctd.ctd_destroy(ctx)
    c, o = out["continuous"], out["one_at_a_time"]
    print(json.dumps({
        "metric": "served p50/p99 latency (s) and histories/sec at 1% avg RSD", "value": c["histories_per_s"],
        "unit": UNIT, "p50_s": c["p50_s"], "p99_s": c["p99_s"], "n_gpus": 1, "higher_is_better": True,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "served", "phantom": [nx, ny, nz], "voxel_cm": d, "rate_per_s": args.rate,
                   "requests": args.n_requests, "batch_histories": args.batch_histories, "rsd_target": 0.01,
                   "min_batches": 10, "phantom_pool": args.pool, "time_limit_s": args.time_limit,
                   "launches": "shared multi-request launch" if args.shared_launch else "one stream per request",
                   "round_histories": args.round_histories or 1e8},
        "continuous": c, "one_at_a_time": o,
        "throughput_vs_one_at_a_time": (c["histories_per_s"] / o["histories_per_s"]) if o["histories_per_s"] else None,
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cbct_water")
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--flight-cap", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-probe", action="store_true", help="skip the memory-ceiling probes")
    ap.add_argument("--rsd-stop", type=int, default=1, help="measure sec-to-1%% with the RSD-stopped form")
    ap.add_argument("--inst-per-history", type=float, default=0.0)
    ap.add_argument("--n-requests", type=int, default=64)
    ap.add_argument("--max-side", type=int, default=256)
    ap.add_argument("--rate", type=float, default=4.0)
    ap.add_argument("--pool", type=int, default=4)
    ap.add_argument("--served-voxel-cm", type=float, default=0.1)
    ap.add_argument("--batch-histories", type=int, default=int(9e9))
    ap.add_argument("--time-limit", type=float, default=None)
    ap.add_argument("--multi-blocks-per-sm", type=int, default=0)
    ap.add_argument("--shared-launch", type=int, default=0, help="served form: one shared multi-request launch")
    ap.add_argument("--round-histories", type=float, default=0.0,
                    help="served form: histories one round may hold before admission stops (0: 1e8)")
    ap.add_argument("--compton", default="kn", choices=["kn", "wh"],
                    help="Compton model: free-electron Klein-Nishina or Waller-Hartree")
    ap.add_argument("--rayleigh", default="gauss", choices=["gauss", "iaa"],
                    help="Rayleigh form factor: analytic exp(-q^2/q0^2) or independent-atom of the elements")
    ap.add_argument("--hist-lo", type=float, default=1e7)
    ap.add_argument("--hist-hi", type=float, default=1e9)
    ap.add_argument("--traffic-per-launch", type=float, default=None)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
