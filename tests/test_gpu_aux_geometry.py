"""The reduced auxiliary geometry problem on the device (rom_set_geometry_aux; Sec. 3.4, Eqs.
auxiliary_problem and reduced_aux_problem) against the oracle, whose map comes from the
full-order auxiliary solution: the reduced step on the device-solved geometry equals the
oracle's reduced step on the full-order geometry (FP64: Pbar 1e-11, Abar 1e-9, equal iteration
counts; TF32 tensor-core path: Pbar 1e-7).  Families: 2D porous cell (16x16 Q4, void radius mu)
and 3D inclusion cell (12^3 hex8, semi-axes mu) at B = 16384 with sampled instances; a shape that
inverts the mapped elements is refused."""
import os
import time

import numpy as np
import pytest

from oracle import aux
from paper_2307_16894_gb300 import binding, workload
from gpu_helpers import OracleRun, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def have(name):
    return os.path.exists(os.path.join(workload.DATA, "rom_%s.npz" % name))


def make_ctx(rom, mu):
    ctx = binding.Context(rom["d"], 0)
    ctx.load_basis(rom["G"])
    ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
    t0 = time.perf_counter()
    ctx.set_geometry_aux(rom, mu)
    return ctx, time.perf_counter() - t0


@pytest.mark.skipif(not have("a1"), reason="model file absent")
def test_aux_geometry_2d_fp64_full_path():
    rom, mu, _, paths = workload.batch("a1", B=32)
    ctx, _ = make_ctx(rom, mu)
    st = ctx.state_create(len(mu))
    o = OracleRun(rom, aux.theta_of_mu(mu, rom["aux_mu_ref"]))
    kw = dict(tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, max_ls=6, start="prev")
    for k in range(paths.shape[1]):
        P, A, info = ctx.step(st, binding.make_opts(**kw), paths[:, k])
        ref = o.step(paths[:, k], **kw)
        assert np.array_equal(info["status"], ref["status"]), k
        assert np.array_equal(info["iters"], ref["iters"]), (k, info["iters"], ref["iters"])
        ok = ref["status"] == 0
        assert rel(P[ok], ref["Pbar"][ok]) <= 1e-11, k
        assert rel(A[ok], ref["Abar"][ok]) <= 1e-9, k
    st.close()
    ctx.close()


@pytest.mark.skipif(not have("a3"), reason="model file absent")
@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_aux_geometry_3d_full_batch_sampled(prec):
    rom, mu, _, paths = workload.batch("a3")
    paths = paths[:, :6]                         # the first 6 steps of the 20-step paths
    B = len(mu)
    ctx, t_geo = make_ctx(rom, mu)
    print("rom_set_geometry_aux B=%d m=%d: %.2f ms (host copies, device solve, det check)" % (B, rom["m"], 1e3 * t_geo))
    sample = np.unique(np.linspace(0, B - 1, 6).round().astype(np.int64))
    st = ctx.state_create(B)
    o = OracleRun(rom, aux.theta_of_mu(mu[sample], rom["aux_mu_ref"]))
    fp64 = prec == "fp64"
    kw = dict(tol_rel=1e-10 if fp64 else 1e-9, tol_abs=rom["tol_abs"], max_iter=25 if fp64 else 50, max_ls=6,
              start="prev", precision=prec)
    for k in range(paths.shape[1]):
        P, A, info = ctx.step(st, binding.make_opts(**kw), paths[:, k])
        ref = o.step(paths[sample, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, max_ls=6, start="prev")
        assert (info["status"] == 0).mean() >= 0.999
        assert np.array_equal(info["status"][sample], ref["status"])
        if fp64:
            assert np.array_equal(info["iters"][sample], ref["iters"]), k
        assert rel(P[sample], ref["Pbar"]) <= (1e-11 if fp64 else 1e-7), (k, rel(P[sample], ref["Pbar"]))
        assert rel(A[sample], ref["Abar"]) <= (1e-9 if fp64 else 1e-4), k
    st.close()
    ctx.close()


@pytest.mark.skipif(not have("a1"), reason="model file absent")
def test_aux_geometry_refuses_inverted_shape():
    rom = workload.load_model("rom_a1")
    ctx = binding.Context(2, 0)
    ctx.load_basis(rom["G"])
    ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
    # theta = mu / r_p - 1 = -2.5: the void boundary moves through its centre
    with pytest.raises(binding.RomError, match="det F_mu"):
        ctx.set_geometry_aux(rom, np.array([[0.3], [-1.5 * rom["aux_mu_ref"][0]]]))
    ctx.set_geometry_aux(rom, np.array([[0.3]]))          # a valid shape afterwards
    ctx.close()
