"""CUDA path vs the FP64 oracle through the C ABI (needs a GB300)."""
import numpy as np
import pytest

from paper_2307_16894_gb300 import binding, workload
from gpu_helpers import GpuRun, OracleRun, cpinv_from_fp, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run_pair(rom, coef, paths, check_every=1, tol_P=1e-11, tol_q=1e-11, **kw):
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef)
    kw.setdefault("tol_abs", rom["tol_abs"])
    worst = dict(P=0.0, A=0.0, q=0.0)
    for k in range(paths.shape[1]):
        P, A, info = g.step(paths[:, k], **kw)
        ref = o.step(paths[:, k], **kw)
        assert np.array_equal(info["status"], ref["status"]), (k, info["status"], ref["status"])
        assert np.array_equal(info["iters"], ref["iters"]), (k, info["iters"], ref["iters"])
        assert np.array_equal(info["evals"], ref["evals"]), (k, info["evals"], ref["evals"])
        ok = ref["status"] == 0
        assert np.array_equal(info["n_yield"][ok], ref["n_yield"][ok]), k
        if ok.any():
            worst["P"] = max(worst["P"], rel(P[ok], ref["Pbar"][ok]))
            worst["A"] = max(worst["A"], rel(A[ok], ref["Abar"][ok]))
        a, cp, xi = g.st.export()
        worst["q"] = max(worst["q"], rel(a, o.q))
        if k % check_every == 0 or k == paths.shape[1] - 1:
            assert rel(cp, cpinv_from_fp(o.Fp, rom["d"])) <= 1e-11, k
            assert np.abs(xi - o.xi).max() <= 1e-11 * max(o.xi.max(), 1e-3), k
    g.close()
    assert worst["P"] <= tol_P, worst
    assert worst["q"] <= tol_q, worst
    assert worst["A"] <= 1e-9, worst
    return worst


def test_c1_full_path_fp64():
    rom, mu, coef, paths = workload.batch("c1")
    w = run_pair(rom, coef, paths, tol_rel=1e-10, max_iter=25, max_ls=6, precision="fp64")
    print("c1 worst", w)


def test_c1_prev_start():
    rom, mu, coef, paths = workload.batch("c1")
    run_pair(rom, coef, paths[:, :8], tol_rel=1e-10, max_iter=25, max_ls=6, start="prev")


def test_c1_zero_load():
    rom, mu, coef, paths = workload.batch("c1")
    g = GpuRun(rom, coef)
    P, A, info = g.step(np.eye(2)[None], tol_rel=1e-10, tol_abs=rom["tol_abs"])
    assert info["iters"][0] == 0 and info["status"][0] == 0
    assert np.all(P == 0.0)
    a, cp, xi = g.st.export()
    assert np.all(a == 0) and np.all(xi == 0)
    g.close()


def test_c1_objectivity_polar():
    rom, mu, coef, paths = workload.batch("c1")
    th = 0.6
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    g1, g2 = GpuRun(rom, coef), GpuRun(rom, coef)
    for k in range(3):
        P1, A1, _ = g1.step(paths[:, k], tol_abs=rom["tol_abs"])
        P2, A2, _ = g2.step(R[None] @ paths[:, k], tol_abs=rom["tol_abs"])
        assert rel(P2[0], R @ P1[0]) <= 1e-12
        At = np.einsum("ia,ajbl,kb->ijkl", R, A1[0].reshape(2, 2, 2, 2), R).reshape(4, 4)
        assert rel(A2[0], At) <= 1e-10
    g1.close(); g2.close()


def test_c1_ragged_batch_fp64():
    """Several instances with different geometry and load, mixed batch (non-multiple of tile sizes)."""
    rom, _, _, _ = workload.batch("c1")
    rng = np.random.default_rng(3)
    B = 13
    mu = rng.uniform(0.2, 0.35, (B, 1))
    from paper_2307_16894_gb300 import inputs
    paths = np.stack([inputs.stretch_path(2, 500 + b, 6, 0.95, 1.05) for b in range(B)])
    run_pair(rom, mu, paths, tol_rel=1e-10, max_iter=25, max_ls=6)


def test_not_converged_is_not_committed():
    rom, mu, coef, paths = workload.batch("c1")
    g = GpuRun(rom, coef)
    P, A, info = g.step(paths[:, 3], tol_abs=rom["tol_abs"], max_iter=1)
    assert info["status"][0] == binding.ROM_E_NOT_CONVERGED
    assert np.isnan(P).all()
    a, cp, xi = g.st.export()
    assert np.all(a == 0) and np.all(xi == 0)
    P, A, info = g.step(paths[:, 0], tol_abs=rom["tol_abs"])
    assert info["status"][0] == 0
    g.close()


def test_state_export_import_resume():
    rom, mu, coef, paths = workload.batch("c1")
    g = GpuRun(rom, coef)
    for k in range(4):
        g.step(paths[:, k], tol_abs=rom["tol_abs"])
    a, cp, xi = g.st.export()
    P1, _, i1 = g.step(paths[:, 4], tol_abs=rom["tol_abs"])
    h = GpuRun(rom, coef)
    h.st.import_(a, cp, xi)
    P2, _, i2 = h.step(paths[:, 4], tol_abs=rom["tol_abs"])
    assert np.array_equal(P1, P2) and np.array_equal(i1, i2)
    g.close(); h.close()


def test_bad_geometry_rejected():
    rom, mu, coef, paths = workload.batch("c1")
    ctx = binding.Context(2, 0)
    ctx.load_basis(rom["G"])
    ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
    with pytest.raises(binding.RomError, match="det F_mu"):
        ctx.set_geometry(rom["Gmu"], np.array([[-40.0]]))
    ctx.close()


def test_fp32_tangent_matches_fp64_answer():
    rom, mu, coef, paths = workload.batch("c1")
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef)
    for k in range(6):
        P, A, info = g.step(paths[:, k], tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=50, precision="fp32")
        ref = o.step(paths[:, k], tol_rel=1e-10, tol_abs=rom["tol_abs"])
        assert info["status"][0] == 0
        assert rel(P, ref["Pbar"]) <= 1e-7
        assert rel(A, ref["Abar"]) <= 1e-4
    g.close()
