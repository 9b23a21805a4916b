"""The batched and served forms against the plain single-request form.

A request's result must be the same alone (ctd_run) and mixed with others in
shared launches (ctd_run_batch, the served scheduler): identical integer
counts, dose equal up to the order of binary64 additions.  The served form
also stops each request at its target avg RSD, admits requests that arrive
while others run, and honours cancellation, bounded waits and EBUSY."""
import numpy as np
import pytest

from paper_1109_3266_gb300 import inputs as I
from gpu_checks import histories_match_binary64

pytestmark = pytest.mark.gpu

KEYS = ("pe", "compton", "rayleigh", "fictitious", "escaped", "missed", "cutoff", "terminated", "aborted", "steps",
        "histories", "n_batches")


@pytest.fixture(scope="module")
def ctd():
    from paper_1109_3266_gb300 import build, ctd as binding
    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(ctd):
    c = ctd.ctd_create(device=0)
    yield c
    ctd.ctd_destroy(c)


@pytest.fixture(scope="module")
def shared_ctx(ctd):
    c = ctd.ctd_create(device=0, shared_launch=1)
    yield c
    ctd.ctd_destroy(c)


@pytest.fixture(params=["chains", "shared"])
def form_ctx(request, ctx, shared_ctx):
    """The batched and served forms in both launch designs."""
    return ctx if request.param == "chains" else shared_ctx


def problems():
    return [I.head(120_000, seed=31, phantom_seed=7, shape=(64, 64, 40), d=0.4),
            I.cbct_water(90_000, seed=32, shape=(48, 48, 24), d=0.8),
            I.head(60_000, seed=33, phantom_seed=8, shape=(40, 40, 24), d=0.6, kvp=80),
            I.cbct_water(7_777, seed=34, shape=(32, 32, 16), d=1.0)]


def alone(ctd, ctx, p, n=None, nb=None):
    h = ctd.load_problem(ctx, p)
    ctd.ctd_run(ctx, h, p.n_hist if n is None else n, p.seed, p.n_batches if nb is None else nb)
    dose, sd, st = ctd.ctd_get_dose_and_stddev(ctx, h, p.phantom.nvox)
    ctd.ctd_destroy_phantom(ctx, h)
    return dose, sd, st


def same(a, b):
    dose, sd, st = a
    d2, s2, st2 = b
    diff = {k: (st[k], st2[k]) for k in KEYS if st[k] != st2[k]}
    assert not diff, diff
    assert np.allclose(d2, dose, rtol=1e-9, atol=0)
    assert np.allclose(s2, sd, rtol=1e-6, atol=1e-30)
    assert st2["avg_rsd"] == pytest.approx(st["avg_rsd"], rel=1e-6)


def test_batched_equals_separate_runs(ctd, ctx, form_ctx):
    ps = problems()
    ref = [alone(ctd, ctx, p) for p in ps]
    hs = [ctd.load_problem(form_ctx, p) for p in ps]
    ctd.ctd_run_batch(form_ctx, hs, [p.n_hist for p in ps], [p.seed for p in ps], 10)
    for p, h, r in zip(ps, hs, ref):
        same(r, ctd.ctd_get_dose_and_stddev(form_ctx, h, p.phantom.nvox))
    # a second batched call on the same phantoms, in another order, gives the same again
    ctd.ctd_run_batch(form_ctx, hs[::-1], [p.n_hist for p in ps[::-1]], [p.seed for p in ps[::-1]], 10)
    for p, h, r in zip(ps, hs, ref):
        same(r, ctd.ctd_get_dose_and_stddev(form_ctx, h, p.phantom.nvox))
    for h in hs:
        ctd.ctd_destroy_phantom(form_ctx, h)


def test_batched_node_grids_and_duplicates(ctd, ctx, shared_ctx):
    tw, cw = I.tiny_water(1000), problems()[3]
    for c in (ctx, shared_ctx):
        a = ctd.load_problem(c, tw)                            # nodes 10-150 keV
        b = ctd.load_problem(c, cw)                            # nodes 1-150 keV
        with pytest.raises(ctd.CtdError):
            ctd.ctd_run_batch(c, [b, b], [1000, 1000], [1, 2], 10)
        if c is shared_ctx:
            # one shared launch holds one node grid
            with pytest.raises(ctd.CtdError):
                ctd.ctd_run_batch(c, [a, b], [1000, 1000], [1, 2], 10)
        else:
            # separate chains do not
            ctd.ctd_run_batch(c, [a, b], [tw.n_hist, cw.n_hist], [tw.seed, cw.seed], 10)
            got = [ctd.ctd_get_dose_and_stddev(c, h, p.phantom.nvox) for h, p in ((a, tw), (b, cw))]
            same(alone(ctd, c, tw, nb=10), got[0])
            same(alone(ctd, c, cw, nb=10), got[1])
        ctd.ctd_destroy_phantom(c, a)
        ctd.ctd_destroy_phantom(c, b)


def test_served_requests_equal_plain_runs(ctd, form_ctx):
    ctx = form_ctx
    ps = problems()[:3]
    B = [20_000, 15_000, 9_000]
    targets = [0.12, 0.2, 0.3]
    hs = [ctd.load_problem(ctx, p) for p in ps]
    ids = [ctd.ctd_submit(ctx, hs[i], B[i], targets[i], ps[i].seed, n_histories_max=400 * B[i])
           for i in range(2)]
    # rounds with two requests, then a third arrives while they run
    for _ in range(3):
        ctd.ctd_serve_step(ctx)
    ids.append(ctd.ctd_submit(ctx, hs[2], B[2], targets[2], ps[2].seed, n_histories_max=400 * B[2]))
    assert ctd.ctd_poll(ctx, ids[0])["state"] == ctd.REQ_RUNNING
    with pytest.raises(ctd.CtdError) as e:
        ctd.ctd_destroy_phantom(ctx, hs[0])
    assert e.value.code == 4                                   # CTD_EBUSY
    for i in ids:
        st = ctd.ctd_wait(ctx, i, 120.0)
        assert st["state"] == ctd.REQ_DONE
    for i, p in enumerate(ps):
        st = ctd.ctd_poll(ctx, ids[i])
        k = st["batches"]
        assert k >= 10 and st["histories"] == k * B[i]
        assert st["avg_rsd"] <= targets[i] or st["histories"] >= 400 * B[i]
        served = ctd.ctd_get_dose_and_stddev(ctx, hs[i], p.phantom.nvox)
        same(alone(ctd, ctx, p, n=k * B[i], nb=k), served)
        ctd.ctd_destroy_phantom(ctx, hs[i])


def test_served_cancel_timeout_and_queue(ctd, ctx):
    p = problems()[1]
    h = ctd.load_problem(ctx, p)
    rid = ctd.ctd_submit(ctx, h, 5_000, 1e-6, 1, n_histories_max=10 ** 12)
    with pytest.raises(ctd.CtdError) as e:
        ctd.ctd_wait(ctx, rid, 0.0)
    assert e.value.code == 5                                   # CTD_ETIMEOUT
    ctd.ctd_serve_step(ctx)
    assert ctd.ctd_serve_wait(ctx, 0.001) == 1                 # the request stays running
    with pytest.raises(ctd.CtdError) as e:
        ctd.ctd_serve_wait(ctx, -1.0)
    assert e.value.code == 1                                   # CTD_EINVAL
    ctd.ctd_cancel(ctx, rid)
    ctd.ctd_serve_step(ctx)
    assert ctd.ctd_poll(ctx, rid)["state"] == ctd.REQ_CANCELLED
    # a queued request cancelled before admission, then the phantom is free again
    rid2 = ctd.ctd_submit(ctx, h, 5_000, 0.5, 2)
    ctd.ctd_cancel(ctx, rid2)
    assert ctd.ctd_poll(ctx, rid2)["state"] == ctd.REQ_CANCELLED
    ctd.ctd_run(ctx, h, 10_000, 3, 10)
    ctd.ctd_destroy_phantom(ctx, h)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_poll(ctx, 10 ** 9)


def test_served_requests_join_while_others_are_on_the_gpu(ctd):
    # continuous batching: a request submitted while another's batch is on the GPU is
    # admitted and its first batch launched at the next step, without waiting for that
    # batch; the short request finishes while the long one is still running
    c = ctd.ctd_create(device=0, serve_round_histories=1e12)
    pa, pb = problems()[0], problems()[3]
    ha, hb = ctd.load_problem(c, pa), ctd.load_problem(c, pb)
    a = ctd.ctd_submit(c, ha, 200_000_000, 1e-9, 5, n_histories_max=10 ** 11)
    ctd.ctd_serve_step(c)                                      # a's first batch goes to the GPU
    b = ctd.ctd_submit(c, hb, 5_000, 0.5, pb.seed, n_histories_max=200_000)
    ctd.ctd_serve_step(c)
    sa, sb = ctd.ctd_poll(c, a), ctd.ctd_poll(c, b)
    assert sb["state"] == ctd.REQ_RUNNING and sa["batches"] == 0, (sa, sb)
    assert ctd.ctd_wait(c, b, 120.0)["state"] == ctd.REQ_DONE
    assert ctd.ctd_poll(c, a)["state"] == ctd.REQ_RUNNING
    ctd.ctd_cancel(c, a)
    ctd.ctd_serve_step(c)
    assert ctd.ctd_poll(c, a)["state"] == ctd.REQ_CANCELLED
    # b's result is the plain run of its batches
    st = ctd.ctd_poll(c, b)
    same(alone(ctd, c, pb, n=st["batches"] * 5_000, nb=st["batches"]), ctd.ctd_get_dose_and_stddev(c, hb, pb.phantom.nvox))
    ctd.ctd_destroy(c)


def test_batched_chains_on_few_streams_equal_separate_runs(ctd, ctx):
    # chains sharing two streams run the requests two at a time, each its own chain
    ps = problems()
    c = ctd.ctd_create(device=0, batch_lanes=2)
    try:
        hs = [ctd.load_problem(c, p) for p in ps]
        ctd.ctd_run_batch(c, hs, [p.n_hist for p in ps], [p.seed for p in ps], 10)
        for p, h in zip(ps, hs):
            same(alone(ctd, ctx, p), ctd.ctd_get_dose_and_stddev(c, h, p.phantom.nvox))
    finally:
        ctd.ctd_destroy(c)


def test_plain_run_on_one_or_two_streams_gives_the_same_results(ctd, ctx):
    # overlapped plain runs alternate batches between two streams and two tallies, the
    # folds in batch order; odd and even batch counts end on either stream
    c = ctd.ctd_create(device=0, plain_overlap=1)
    try:
        for p in (problems()[0], I.scaled(problems()[1], n_batches=11), I.scaled(problems()[3], n_batches=2)):
            same(alone(ctd, c, p), alone(ctd, ctx, p))
    finally:
        ctd.ctd_destroy(c)


def test_l2_persisting_tally_gives_the_same_results(ctd, ctx):
    # the access-policy window changes only what L2 keeps
    p = problems()[0]
    c = ctd.ctd_create(device=0, l2_persist=1)
    try:
        same(alone(ctd, ctx, p), alone(ctd, c, p))
    finally:
        ctd.ctd_destroy(c)


def test_served_gpu_filling_requests_equal_plain_runs(ctd):
    # batches of 1.2e7 histories fill the GPU (64 histories per resident thread): the
    # first in line runs its batches before the first stop test in one step at high
    # priority, the second fills its last batch one slice (an eighth) at a time and,
    # once first, resumes the batch it began in slices; results stay those of plain runs
    c = ctd.ctd_create(device=0, serve_round_histories=1e12)
    B = 12_000_000
    ps = [I.scaled(problems()[3], seed=41), I.scaled(problems()[3], seed=42), I.scaled(problems()[1], seed=43)]
    hs = [ctd.load_problem(c, p) for p in ps]
    ids = [ctd.ctd_submit(c, hs[i], B, 0.5, ps[i].seed, n_histories_max=6 * B, min_batches=3) for i in range(3)]
    for i in ids:
        assert ctd.ctd_wait(c, i, 120.0)["state"] == ctd.REQ_DONE
    for i, p in enumerate(ps):
        st = ctd.ctd_poll(c, ids[i])
        k = st["batches"]
        assert k >= 3 and st["histories"] == k * B
        same(alone(ctd, c, p, n=k * B, nb=k), ctd.ctd_get_dose_and_stddev(c, hs[i], p.phantom.nvox))
        ctd.ctd_destroy_phantom(c, hs[i])
    ctd.ctd_destroy(c)


def test_served_request_without_target_runs_to_its_cap(ctd):
    # rsd_target 0: the request stops at its history cap, checked from min_batches on,
    # beside another request with a target
    c = ctd.ctd_create(device=0, serve_round_histories=1e12)
    pa, pb = problems()[1], problems()[3]
    ha, hb = ctd.load_problem(c, pa), ctd.load_problem(c, pb)
    a = ctd.ctd_submit(c, ha, 30_000, 0.0, pa.seed, n_histories_max=12 * 30_000, min_batches=4)
    b = ctd.ctd_submit(c, hb, 2_000, 0.5, pb.seed, n_histories_max=100 * 2_000, min_batches=2)
    sb = ctd.ctd_wait(c, b, 120.0)
    sa = ctd.ctd_wait(c, a, 120.0)
    assert sa["state"] == sb["state"] == ctd.REQ_DONE
    assert sa["batches"] == 12 and sa["histories"] == 12 * 30_000
    same(alone(ctd, c, pa, n=12 * 30_000, nb=12), ctd.ctd_get_dose_and_stddev(c, ha, pa.phantom.nvox))
    k = sb["batches"]
    same(alone(ctd, c, pb, n=k * 2_000, nb=k), ctd.ctd_get_dose_and_stddev(c, hb, pb.phantom.nvox))
    ctd.ctd_destroy(c)


def test_serve_loop_reports_latency(ctd, ctx):
    from paper_1109_3266_gb300 import serve

    arrivals = [(0.0, 51), (0.05, 52), (0.1, 53), (0.15, 54)]

    def make(seed):
        return I.head(1, seed=seed, phantom_seed=seed, shape=(32, 32, 20), d=0.8)

    reqs, wall = serve.serve(ctx, arrivals, make, batch_histories=20_000, rsd_target=0.25, n_histories_max=4_000_000)
    summ = serve.latency_summary(reqs)
    assert summ["done"] == 4 and summ["p50_s"] > 0 and summ["p99_s"] >= summ["p50_s"]
    for r in reqs:
        assert r.state == ctd.REQ_DONE and r.batches >= 10


def test_autotune_picks_a_shape_and_results_do_not_depend_on_it(ctd, ctx):
    p = problems()[0]
    before = alone(ctd, ctx, p)
    c2 = ctd.ctd_create(device=0)
    h = ctd.load_problem(c2, p)
    r = ctd.ctd_autotune(c2, h, 200_000, seed=5)
    assert (r["threads_per_block"], r["blocks_per_sm"]) in ((256, 3), (256, 4), (128, 7), (128, 8))
    assert r["chunk"] in (64, 256, 1024) and r["flight_cap"] in (1, 2, 4, 8)
    assert r["n_tried"] in (48, 49) and r["histories_per_s"] >= r["baseline_per_s"] * 0.999
    ctd.ctd_run(c2, h, p.n_hist, p.seed, p.n_batches)
    same(before, ctd.ctd_get_dose_and_stddev(c2, h, p.phantom.nvox))
    ctd.ctd_destroy_phantom(c2, h)
    ctd.ctd_destroy(c2)


def test_batched_full_size_requests(ctd, oracle):
    # the specified 64 requests (cubes of 64^3 to 256^3 voxels, water and head, 80-140 kVp)
    # in the launch configuration the benchmark times, with histories scaled down: batched
    # results equal separate runs, and sampled history ranges of two requests equal the
    # binary32 oracle bit for bit
    from test_gpu_parity import COUNT_KEYS as CK
    reqs = [I.scaled(p, n_hist=max(20_000, p.n_hist // 2000)) for p in I.batched_requests(64)]
    c = ctd.ctd_create(device=0)
    hs = [ctd.load_problem(c, p) for p in reqs]
    ctd.ctd_run_batch(c, hs, [p.n_hist for p in reqs], [p.seed for p in reqs], 10)
    got = [ctd.ctd_get_dose_and_stddev(c, h, 0, want_arrays=False)[2] for h in hs]
    picks = [0, 13, 38, 63]
    doses = {r: ctd.ctd_get_dose_and_stddev(c, hs[r], reqs[r].phantom.nvox)[0] for r in picks}
    for r, p in enumerate(reqs):
        ctd.ctd_run(c, hs[r], p.n_hist, p.seed, 10)
        st = ctd.ctd_get_dose_and_stddev(c, hs[r], 0, want_arrays=False)[2]
        diff = {k: (got[r][k], st[k]) for k in CK if got[r][k] != st[k]}
        assert not diff, (r, diff)
        if r in picks:
            assert np.allclose(ctd.ctd_get_dose_and_stddev(c, hs[r], p.phantom.nvox)[0], doses[r], rtol=1e-9, atol=0)
    for r in (1, 62):
        p = reqs[r]
        histories_match_binary64(ctd, c, hs[r], p, oracle, ranges=[(0, 3000), (p.n_hist - 3000, p.n_hist)])
    ctd.ctd_destroy(c)


def test_batched_autotuner_picks_a_shape_and_results_do_not_depend_on_it(ctd, ctx):
    ps = problems()
    ref = [alone(ctd, ctx, p) for p in ps]
    c = ctd.ctd_create(device=0)
    hs = [ctd.load_problem(c, p) for p in ps]
    r = ctd.ctd_autotune_batch(c, hs, [p.n_hist for p in ps], [p.seed for p in ps], 10, probe_fraction=0.2)
    assert r["n_tried"] == 29 and r["histories_per_s"] > 0 and r["baseline_per_s"] > 0
    assert r["shared_launch"] in (0, 1) and r["chunk"] in (256, 1024) and r["flight_cap"] in (2, 4)
    assert r["batch_lanes"] in (2, 4, 8, 16, 64)
    # the context keeps the choice; the full requests give what they give alone
    ctd.ctd_run_batch(c, hs, [p.n_hist for p in ps], [p.seed for p in ps], 10)
    for p, h, rr in zip(ps, hs, ref):
        same(rr, ctd.ctd_get_dose_and_stddev(c, h, p.phantom.nvox))
    with pytest.raises(ctd.CtdError):
        ctd.ctd_autotune_batch(c, hs, [p.n_hist for p in ps], [p.seed for p in ps], 10, probe_fraction=0.0)
    ctd.ctd_destroy(c)


def test_served_admission_by_free_device_memory(ctd):
    # a reserve larger than any GPU's memory keeps a request queued: waiting on it is
    # refused with CTD_ENOMEM instead of spinning, and it can still be cancelled
    p = problems()[3]
    tight = ctd.ctd_create(device=0, serve_reserve_bytes=1e15)
    h = ctd.load_problem(tight, p)
    rid = ctd.ctd_submit(tight, h, 5_000, 0.5, 1)
    with pytest.raises(ctd.CtdError) as e:
        ctd.ctd_wait(tight, rid, 30.0)
    assert e.value.code == 2                                   # CTD_ENOMEM
    assert ctd.ctd_poll(tight, rid)["state"] == ctd.REQ_QUEUED
    ctd.ctd_cancel(tight, rid)
    assert ctd.ctd_poll(tight, rid)["state"] == ctd.REQ_CANCELLED
    ctd.ctd_destroy(tight)
    # the same request under the default reserve is admitted and finishes
    c = ctd.ctd_create(device=0)
    h = ctd.load_problem(c, p)
    rid = ctd.ctd_submit(c, h, 5_000, 0.5, 1)
    assert ctd.ctd_wait(c, rid, 60.0)["state"] == ctd.REQ_DONE
    ctd.ctd_destroy(c)


@pytest.mark.parametrize("shape", [dict(threads_per_block=128, blocks_per_sm=7, chunk=64, flight_cap=1),
                                   dict(threads_per_block=256, blocks_per_sm=3, chunk=1024, flight_cap=8),
                                   dict(threads_per_block=128, blocks_per_sm=8, chunk=256, flight_cap=2),
                                   dict(threads_per_block=64, blocks_per_sm=5, chunk=96, flight_cap=3)])
def test_results_do_not_depend_on_the_launch_shape(ctd, ctx, shape):
    # every history's random numbers depend only on (seed, history): block shape,
    # residency, claim size and flight cap change only the order of the tally's additions
    p = problems()[1]
    before = alone(ctd, ctx, p)
    c2 = ctd.ctd_create(device=0, **shape)
    same(before, alone(ctd, c2, p))
    ctd.ctd_destroy(c2)
