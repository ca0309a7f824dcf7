"""rom_step_noalloc, the allocation-free step for callers that cannot call
cudaMalloc (a solver inside a pre-sized pool or arena, or a host application that
must not grow its device footprint after start-up).
Its work space is a static device array; the test checks its outputs and
updated state against rom_step (the allocating entry point) on two calls in a
row, in FP64 and on the mixed FP32 path (FP32 tangent and stiffness, FP32 LU
with FP64 refinement), and that an oversized batch is refused.  Kept in a file of its own that
pytest collects last."""
import numpy as np
import pytest

from paper_2307_16894_gb300 import binding, inputs, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_rom_step_two_calls(prec):
    import torch
    rom = workload.load_model("rom_c1")
    d, n, m = rom["d"], rom["n"], rom["m"]
    B = 13
    rng = np.random.default_rng(21)
    mu = rng.uniform(0.2, 0.35, (B, 1))
    paths = np.stack([inputs.stretch_path(2, 900 + b, 4, 0.95, 1.06) for b in range(B)])
    fp64 = prec == "fp64"
    kw = dict(tol_rel=1e-10 if fp64 else 1e-9, tol_abs=rom["tol_abs"], max_iter=25 if fp64 else 50, max_ls=6,
              precision=prec, start="prev")
    # FP64: the same arithmetic as rom_step; FP32: both sides converge to the relative residual
    # 1e-9 through their own FP32 stiffness, so they agree to well inside the 1e-7 bound on Pbar
    tp, ta, tq = (1e-11, 1e-9, 1e-11) if fp64 else (1e-8, 1e-5, 1e-8)
    opts = binding.make_opts(**kw)

    # reference: the allocating context path
    ctx = binding.Context(d, 0)
    ctx.load_basis(rom["G"])
    ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
    ctx.set_geometry(rom["Gmu"], mu)
    st = ctx.state_create(B)
    ref = [ctx.step(st, opts, paths[:, k]) for k in range(2)]
    a_ref, cp_ref, xi_ref = st.export()
    st.close()
    ctx.close()

    # allocation-free path: the caller owns every device array
    dev = torch.device("cuda", 0)
    t = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    G_d, w_d, ph_d, Gmu_d, mu_d = t(rom["G"]), t(rom["w"]), t(rom["phase"], torch.int32), t(rom["Gmu"]), t(mu)
    a_d = torch.zeros((B, n), dtype=torch.float64, device=dev)
    da_d = torch.zeros((B, n), dtype=torch.float64, device=dev)
    cp0 = np.zeros((B, 4, m))
    cp0[:, 0] = 1.0
    cp0[:, 2] = 1.0
    cp0[:, 3] = 1.0
    cp_d = t(cp0)
    xi_d = torch.zeros((B, m), dtype=torch.float64, device=dev)
    P_d = torch.empty((B, d, d), dtype=torch.float64, device=dev)
    A_d = torch.empty((B, d * d, d * d), dtype=torch.float64, device=dev)
    I_d = torch.zeros((B, binding.INFO_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    for k in range(2):
        F_d = t(paths[:, k])
        binding.step_noalloc(d, G_d, w_d, ph_d, Gmu_d, rom["phases"], rom["omega"], mu_d, a_d, da_d, cp_d, xi_d,
                             opts, F_d, P_d, A_d, I_d)
        torch.cuda.synchronize()
        P, A, info = ref[k]
        info2 = np.frombuffer(I_d.cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE)
        assert np.array_equal(info2["status"], info["status"])
        if fp64:
            assert np.array_equal(info2["iters"], info["iters"])
        else:
            assert np.abs(info2["iters"] - info["iters"]).max() <= 1
        ok = info["status"] == 0
        assert ok.all()
        assert rel(P_d.cpu().numpy(), P) <= tp
        assert rel(A_d.cpu().numpy(), A) <= ta
    assert rel(a_d.cpu().numpy(), a_ref) <= tq
    assert rel(np.swapaxes(cp_d.cpu().numpy(), 1, 2), cp_ref) <= tq
    assert np.abs(xi_d.cpu().numpy() - xi_ref).max() <= tq * max(xi_ref.max(), 1e-3)


def test_noalloc_rejects_oversized_batch():
    import torch
    rom = workload.load_model("rom_c1")
    d, n, m = rom["d"], rom["n"], rom["m"]
    B = 100_000
    dev = torch.device("cuda", 0)
    t = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device=dev)
    opts = binding.make_opts(1e-10, rom["tol_abs"])
    with pytest.raises(binding.RomError, match="static"):
        binding.step_noalloc(d, t(rom["G"]), t(rom["w"]), t(rom["phase"], torch.int32), t(rom["Gmu"]),
                             rom["phases"], rom["omega"], z(B, 1), z(B, n), z(B, n), z(B, 4, m), z(B, m), opts,
                             z(B, d, d), z(B, d, d), z(B, d * d, d * d), None)
