"""Graph mode (one CUDA-graph launch per load step, Newton passes in a device-driven
conditional WHILE node) gives the same results as the host-driven loop."""
import numpy as np
import pytest

from paper_2307_16894_gb300 import binding, workload
from gpu_helpers import torch_stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run(rom, coef, paths, graphs, **kw):
    import torch
    d = rom["d"]
    ctx = binding.Context(d, 0, torch_stream())
    ctx.load_basis(rom["G"])
    ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
    ctx.set_geometry(rom["Gmu"], coef)
    ctx.use_graphs(graphs)
    st = ctx.state_create(len(coef))
    opts = binding.make_opts(**kw)
    B = len(coef)
    Fd = torch.from_numpy(np.ascontiguousarray(paths.transpose(1, 0, 2, 3))).cuda()
    Pd = torch.empty((B, d, d), dtype=torch.float64, device="cuda")
    Ad = torch.empty((B, d * d, d * d), dtype=torch.float64, device="cuda")
    Id = torch.empty((B, binding.INFO_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    out = []
    for k in range(paths.shape[1]):
        ctx.step_device(st, opts, Fd[k], Pd, Ad, Id)
        torch.cuda.synchronize()
        out.append((Pd.cpu().numpy().copy(), Ad.cpu().numpy().copy(),
                    np.frombuffer(Id.cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE).copy()))
    a, cp, xi = st.export()
    st.close()
    ctx.close()
    return out, (a, cp, xi)


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_graph_equals_host_loop(prec):
    rom, mu, coef, paths = workload.batch("c2", B=41, steps=8)
    kw = dict(tol_rel=1e-10 if prec == "fp64" else 1e-9, tol_abs=rom["tol_abs"], max_iter=50, max_ls=6,
              precision=prec, start="prev")
    o1, s1 = run(rom, coef, paths, False, **kw)
    o2, s2 = run(rom, coef, paths, True, **kw)
    for (P1, A1, i1), (P2, A2, i2) in zip(o1, o2):
        assert np.array_equal(i1, i2)
        assert np.array_equal(P1, P2) and np.array_equal(A1, A2)
    for x, y in zip(s1, s2):
        assert np.array_equal(x, y)
