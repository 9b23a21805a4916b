"""Request loop of the served form (continuous batching).

Requests arrive at given times; at each turn of the loop the requests that
have arrived are created on the device and submitted, and the library's
scheduler is stepped until something changes or the next request is due
(ctd_serve_wait): it takes in the batches that have finished on the GPU,
retires requests at their target avg RSD, admits queued requests by free
device memory and launches the next batches of running requests, each on its
own stream, the request with the least work left first and at high priority
(with the context's shared_launch option, one round of every running request
in one shared launch instead).  Finished requests are read back and their
phantoms released.  The scheduling and every step of the
transport run in the CUDA library; this module only drives it and keeps the
clock.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import ctd


@dataclass
class Served:
    seed: int
    t_arrival: float
    t_done: float = float("nan")
    req_id: int = -1
    handle: int = -1
    state: int = -1
    histories: int = 0
    batches: int = 0
    avg_rsd: float = float("nan")
    latency: float = float("nan")
    stats: dict = field(default_factory=dict)


def serve(ctx, arrivals, make_problem, batch_histories, rsd_target, min_batches=10, n_histories_max=0,
          keep_results=False, time_limit_s=None):
    """Run the served form over `arrivals` [(t_arrival_s, seed), ...].

    make_problem(seed) gives the inputs.Problem of a request.  Returns the
    per-request records and the wall time of the whole run.  With time_limit_s,
    requests still unfinished then are cancelled (their latency stays NaN)."""
    reqs = [Served(seed, t) for t, seed in sorted(arrivals)]
    nxt = 0
    running = {}
    t0 = time.perf_counter()
    while nxt < len(reqs) or running:
        now = time.perf_counter() - t0
        if time_limit_s is not None and now > time_limit_s:
            for r in running.values():
                ctd.ctd_cancel(ctx, r.req_id)
            ctd.ctd_serve_step(ctx)
            for r in running.values():
                r.state = ctd.REQ_CANCELLED
                ctd.ctd_destroy_phantom(ctx, r.handle)
            running.clear()
            break
        while nxt < len(reqs) and reqs[nxt].t_arrival <= now:
            r = reqs[nxt]
            p = make_problem(r.seed)
            r.handle = ctd.load_problem(ctx, p)
            r.req_id = ctd.ctd_submit(ctx, r.handle, batch_histories, rsd_target, r.seed,
                                      n_histories_max=n_histories_max, min_batches=min_batches)
            running[r.req_id] = r
            nxt += 1
        if not running:
            time.sleep(max(0.0, min(0.01, reqs[nxt].t_arrival - now)))
            continue
        # step until a batch ends or a request is admitted, at most until the next arrival
        until = 1e-3 if nxt >= len(reqs) else min(1e-3, max(0.0, reqs[nxt].t_arrival - (time.perf_counter() - t0)))
        ctd.ctd_serve_wait(ctx, until)
        t_now = time.perf_counter() - t0
        for rid in list(running):
            st = ctd.ctd_poll(ctx, rid)
            if st["state"] >= ctd.REQ_DONE:
                r = running.pop(rid)
                r.state = st["state"]
                r.t_done = t_now
                r.latency = t_now - r.t_arrival
                r.histories = st["histories"]
                r.batches = st["batches"]
                r.avg_rsd = st["avg_rsd"]
                if keep_results:
                    r.stats = ctd.ctd_get_dose_and_stddev(ctx, r.handle, 0, want_arrays=False)[2]
                ctd.ctd_destroy_phantom(ctx, r.handle)
    return reqs, time.perf_counter() - t0


def latency_summary(reqs):
    lat = np.array([r.latency for r in reqs if np.isfinite(r.latency)])
    if lat.size == 0:
        return {"p50_s": None, "p99_s": None, "done": 0}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)), "done": int(lat.size),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
