"""Host-side pieces of the device offline stage (no GPU): the package's structured grid and
V^p Gram matrix equal the oracle's mesh and Gram matrix (the dof numbering must agree so that
device and oracle snapshots can be compared entry by entry)."""
import numpy as np
import pytest

from oracle import build_roms, fe
from paper_2307_16894_gb300 import mesh, offline


@pytest.mark.parametrize("d,N", [(2, 16), (3, 6)])
def test_grid_and_vp_gram_equal_oracle(d, N):
    pf = build_roms.phase_2d if d == 2 else build_roms.phase_3d
    a, b = fe.Mesh(d, N, pf), mesh.Grid(d, N, pf)
    assert np.array_equal(a.edof, b.edof) and a.ndof == b.ndof
    assert np.array_equal(a.el_phase, b.el_phase)
    assert np.abs(a.dN - b.dN).max() == 0.0 and np.array_equal(a.gw, b.gw)
    assert np.abs(a.X - b.X).max() < 1e-15
    Ma, Mb = a.mass_and_laplace().tocsr(), offline.vp_gram(b).tocsr()
    assert abs(Ma - Mb).max() < 1e-15
