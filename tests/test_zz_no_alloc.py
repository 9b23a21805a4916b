"""ctd_avg_rsd_noalloc: the avg-RSD reduction for callers that cannot allocate
device memory when they need it (such as hosts whose own pool allocator owns
all device memory).  It keeps its partial sums in
a fixed device array inside the library instead of allocating scratch.  Its
results must equal those ctd_run reports through the allocating path, on two
calls in a row and for two different inputs, and sizes beyond the array's
reach must be refused.  This file sorts last so that a run stopping at the
first failure has already run every other test."""
import numpy as np
import pytest

from paper_1109_3266_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_avg_rsd_matches_allocating_path():
    import torch

    from paper_1109_3266_gb300 import build, ctd

    build.build()
    ctx = ctd.ctd_create(device=0)
    stream = torch.cuda.current_stream()
    problems = (I.head(200_000, shape=(48, 48, 30), d=0.5), I.tiny_water(50_000))
    for p in problems:
        dose, sd, st, h = ctd.run_problem(ctx, p)
        d_dose = torch.from_numpy(dose).cuda()
        d_sd = torch.from_numpy(sd).cuda()
        d_rho = torch.from_numpy(np.ascontiguousarray(p.phantom.rho).ravel().copy()).cuda()
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        for _ in range(2):
            out.fill_(float("nan"))
            ctd.ctd_avg_rsd_noalloc(d_dose.data_ptr(), d_sd.data_ptr(), d_rho.data_ptr(), dose.size,
                                    out.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize()
            r = out.cpu().numpy()
            assert r[0] == pytest.approx(st["avg_rsd"], rel=1e-9)
            assert r[1] == pytest.approx(st["paper_sigma_bar"], rel=1e-9)
            assert r[2] == pytest.approx(st["d_max"], rel=1e-12)
        ctd.ctd_destroy_phantom(ctx, h)
    ctd.ctd_destroy(ctx)


def test_noalloc_refuses_sizes_beyond_its_scratch():
    import torch

    from paper_1109_3266_gb300 import ctd

    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ctd.CtdError) as e:
        ctd.ctd_avg_rsd_noalloc(t.data_ptr(), t.data_ptr(), t.data_ptr(), 67_108_865, t.data_ptr())
    assert e.value.code == 1 and "67,108,864" in str(e.value)
