"""Ragged serving (models of different n and m served together by rom_serve, one CUDA-graph
launch per wave): per-group results equal the standalone solve; a memory budget that forces
several waves gives the same answers (to the Newton tolerance) with states only for one wave
at a time; every model of the family (2D n 16/24/32, 3D n 48/64/95) matches the FP64 oracle."""
import numpy as np
import pytest

from paper_2307_16894_gb300 import serving
from gpu_helpers import GpuRun, OracleRun, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run(groups, steps, **kw):
    srv = serving.Server(groups, precision="fp32", **kw)
    outs, lats = [], []
    for k in range(steps):
        wall, lat, info = srv.step(k)
        assert (info["status"] == 0).all()
        outs.append([srv.pbar(gi) for gi in range(len(groups))])
        lats.append(lat)
    waves = len(srv.waves)
    srv.close()
    return outs, lats, waves


def test_serving_matches_standalone():
    groups = serving.make_groups(120, share_2d=0.75, steps=3)
    outs, _, waves = run(groups, 3, autotune=False)
    assert waves == 1
    for gi, g in enumerate(groups):
        r = GpuRun(g["rom"], g["coef"])
        for k in range(3):
            P, A, inf = r.step(g["paths"][:, k], tol_rel=1e-9, tol_abs=g["rom"]["tol_abs"], max_iter=50,
                               max_ls=6, precision="fp32", start="prev")
            assert np.array_equal(P, outs[k][gi]), (g["name"], k)
        r.close()


def test_serving_waves_under_budget():
    """A budget of about a third of the total state footprint: at least three waves, groups split
    across waves, the same converged Pbar as the single-wave run, latencies growing by wave."""
    groups = serving.make_groups(120, share_2d=0.75, steps=3)
    ref, _, _ = run(groups, 3, autotune=False)
    per = serving.state_bytes_per_instance(groups)
    total = sum(g["B"] * p for g, p in zip(groups, per))
    srv = serving.Server(groups, precision="fp32", autotune=True, budget_bytes=int(total / 3.2))
    assert len(srv.waves) >= 3
    live = []
    for k in range(3):
        wall, lat, info = srv.step(k)
        assert (info["status"] == 0).all()
        live.append(sum(c["state"] is not None for c in srv.chunks))
        for gi in range(len(groups)):
            assert rel(srv.pbar(gi), ref[k][gi]) <= 1e-7, (gi, k)
        p50, p99 = np.percentile(lat, [50, 99])
        assert 0 < p50 <= p99 <= wall + 1e-6
    assert max(live) == 0          # states exist only while their wave runs
    srv.close()


def test_family_members_vs_oracle():
    """Two instances of every model of the ragged family, three load steps, against the oracle."""
    groups = serving.make_groups(len(serving.FAMILY_2D + serving.FAMILY_3D) * 2, share_2d=0.5, steps=3)
    outs, _, _ = run(groups, 3, autotune=False)
    names = set()
    for gi, g in enumerate(groups):
        names.add(g["name"])
        o = OracleRun(g["rom"], g["coef"])
        for k in range(3):
            ref = o.step(g["paths"][:, k], tol_rel=1e-10, tol_abs=g["rom"]["tol_abs"], start="prev")
            assert (ref["status"] == 0).all()
            assert rel(outs[k][gi], ref["Pbar"]) <= 1e-7, (g["name"], k, rel(outs[k][gi], ref["Pbar"]))
    assert names == set(serving.available(serving.FAMILY_2D + serving.FAMILY_3D))
