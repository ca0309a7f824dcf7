"""Ragged serving (models of different n and m served together through rom_serve):
per-group results equal the standalone solve, admission by memory footprint defers
groups to a later wave, and the latency percentiles follow the waves."""
import numpy as np
import pytest

from paper_2307_16894_gb300 import binding, serving
from gpu_helpers import GpuRun, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_serving_matches_standalone():
    groups = serving.make_groups(120, share_2d=0.75, steps=3)
    srv = serving.Server(groups, precision="fp32", autotune=False)
    outs = []
    for k in range(3):
        wall, lat, info = srv.step(k)
        assert (info["status"] == 0).all()
        outs.append([g["P"].cpu().numpy().copy() for g in groups])
    srv.close()
    for gi, g in enumerate(groups):
        r = GpuRun(g["rom"], g["coef"])
        for k in range(3):
            P, A, inf = r.step(g["paths"][:, k], tol_rel=1e-9, tol_abs=g["rom"]["tol_abs"], max_iter=50,
                               max_ls=6, precision="fp32", start="prev")
            assert np.array_equal(P, outs[k][gi]), (g["name"], k)
        r.close()


def test_serving_autotune_and_admission():
    groups = serving.make_groups(90, share_2d=1.0, steps=3)
    # a budget that admits only the first group in the first wave
    srv0 = serving.Server(groups, precision="fp32", autotune=True, budget_bytes=1)
    waves = [g["wave"] for g in groups]
    assert waves.count(1) >= 1
    lats = []
    for k in range(3):
        wall, lat, info = srv0.step(k)
        assert (info["status"] == 0).all()
        lats.append(lat)
    srv0.close()
    lat = np.concatenate(lats)
    p50, p99 = np.percentile(lat, [50, 99])
    assert 0 < p50 <= p99
