"""Source trajectories on the GPU (Sec. 2.2.6): discrete and continuous
circles, the partial 200-degree arc of the paper's head-and-neck case, and
helical CT trajectories, each following the binary64 oracle history by
history and giving its dose within 3 sigma."""
import math

import numpy as np
import pytest

from paper_1109_3266_gb300 import inputs as I
from gpu_checks import histories_match_binary64
from test_gpu_parity import dose_parity

pytestmark = pytest.mark.gpu


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


def with_source(p, src):
    import dataclasses
    return dataclasses.replace(p, source=src)


SOURCES = {
    "circle_continuous": I.arc_source(100.0, -8.0, 8.0, -6.0, 6.0, continuous=True),
    "arc_200": I.arc_source(100.0, -8.0, 8.0, -6.0, 6.0, n_proj=200, arc0=0.0, arc1=math.radians(200.0)),
    "helical": I.helical_source(100.0, -8.0, 8.0, -2.0, 2.0, turns=3.0, z0=-6.0, z1=6.0, n_proj_per_turn=120),
    "helical_continuous": I.helical_source(100.0, -8.0, 8.0, -2.0, 2.0, turns=2.5, z0=-5.0, z1=4.0,
                                           continuous=True),
}


@pytest.mark.parametrize("name", sorted(SOURCES))
def test_trajectory_matches_oracles(ctd, ctx, oracle, name):
    p = with_source(I.head(200_000, seed=21, phantom_seed=5, shape=(48, 48, 40), d=0.5), SOURCES[name])
    dose, sd, st, h = ctd.run_problem(ctx, p)
    r64 = oracle.run(p, precision=64)
    frac, nmask = dose_parity(dose, sd, r64.dose, r64.std)
    assert nmask > 50 and frac >= 0.99, (frac, nmask)
    histories_match_binary64(ctd, ctx, h, p, oracle)
    ctd.ctd_destroy_phantom(ctx, h)
