"""Pin of the oracle's shape sensitivities dPbar/dmu (Eq. eff_sensitivities_full with the
reduced fluctuation sensitivity from K dq = -df/dmu) against central finite differences of
the oracle's own converged load step in mu, from the same committed history.  The sensitivity
is taken with respect to the coefficients of the affine map F_mu = I + sum_k mu_k Gmu_k (the
geometry parameters of the library's interface)."""
import os

import numpy as np
import pytest

import oracle
from paper_2307_16894_gb300 import workload


def geometry(rom, coef):
    d, m = rom["d"], rom["m"]
    Gmu = rom["Gmu"].reshape(m, d, d, -1)
    Fm = np.eye(d)[None, None] + np.einsum("iack,bk->biac", Gmu, np.atleast_2d(coef))
    return np.ascontiguousarray(np.linalg.inv(Fm)), np.ascontiguousarray(np.abs(np.linalg.det(Fm)))


def history(rom, coef, paths, nsteps):
    """(q, Fp, xi) after the first nsteps load steps of the paths"""
    d, n, m = rom["d"], rom["n"], rom["m"]
    B = len(coef)
    Finv, J = geometry(rom, coef)
    q = np.zeros((B, n))
    Fp = np.tile(np.eye(3), (B, m, 1, 1)).copy()
    xi = np.zeros((B, m))
    for k in range(nsteps):
        o = oracle.rom_batch(rom, Finv, J, paths[:, k], q, Fp, xi, 1e-13, 1e-14, 40, want_A=False)
        assert (o["status"] == 0).all()
    return q, Fp, xi


def check(name, B, nhist, h, tol):
    rom, mu, coef, paths = workload.batch(name, B=B)
    q, Fp, xi = history(rom, coef, paths, nhist)
    F = paths[:, nhist]

    def step(c, sens=False):
        Finv, J = geometry(rom, c)
        kw = {}
        if sens:
            kw["dFinv"], kw["dJ"] = oracle.geometry_derivatives(rom, Finv, J)
        o = oracle.rom_batch(rom, Finv, J, F, q.copy(), Fp.copy(), xi.copy(), 1e-12, 1e-15, 40, want_A=False, **kw)
        assert (o["status"] == 0).all()
        return o

    o = step(coef, sens=True)
    S = o["dPdmu"]                                   # [B, d, d, n_par]
    npar = coef.shape[1]
    for k in range(npar):
        e = np.zeros_like(coef)
        e[:, k] = h
        fd = (step(coef + e)["Pbar"] - step(coef - e)["Pbar"]) / (2 * h)
        err = np.abs(S[..., k] - fd).max() / np.abs(fd).max()
        print(name, "k=%d" % k, "max |analytic - FD| / max |FD| = %.2e" % err,
              "plastic points:", o["n_yield"])
        assert err <= tol, (k, err)
    return o


def test_sensitivity_fd_2d():
    """2D porous RVE (c2 model, n = 24, m = 160), after 12 load steps (plastic)."""
    o = check("c2", 3, 12, 1e-5, 1e-6)
    assert (o["n_yield"] > 0).all()


@pytest.mark.skipif(not os.path.exists(os.path.join(workload.DATA, "rom_c3.npz")), reason="3D model file not generated")
def test_sensitivity_fd_3d():
    """3D inclusion RVE (c3 model, n = 64, m = 600, three map coefficients), after 6 load steps."""
    check("c3", 1, 6, 1e-5, 1e-6)


def test_sensitivity_objectivity_2d():
    """With the polar split the step is objective, so dPbar/dmu(R Fbar) = R dPbar/dmu(Fbar): a
    pin of the rotation handling of the sensitivities that does not use finite differences."""
    rom, mu, coef, paths = workload.batch("c2", B=2)
    q, Fp, xi = history(rom, coef, paths, 6)
    F = paths[:, 6]
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    Finv, J = geometry(rom, coef)
    dFinv, dJ = oracle.geometry_derivatives(rom, Finv, J)
    outs = []
    for FF in (F, np.einsum("ij,bjk->bik", R, F)):
        o = oracle.rom_batch(rom, Finv, J, np.ascontiguousarray(FF), q.copy(), Fp.copy(), xi.copy(), 1e-12, 1e-15, 40,
                             want_A=False, dFinv=dFinv, dJ=dJ)
        assert (o["status"] == 0).all()
        outs.append(o["dPdmu"])
    rot = np.einsum("ij,bjkp->bikp", R, outs[0])
    err = np.abs(outs[1] - rot).max() / np.abs(rot).max()
    print("objectivity of dPbar/dmu: %.2e" % err)
    assert err <= 1e-8


def test_geometry_derivatives_fd():
    """dF_mu^-1/dmu and d|det F_mu|/dmu of the affine map vs central differences in mu."""
    rom, mu, coef, paths = workload.batch("c3" if os.path.exists(os.path.join(workload.DATA, "rom_c3.npz")) else "c2",
                                          B=2)
    Finv, J = geometry(rom, coef)
    dFinv, dJ = oracle.geometry_derivatives(rom, Finv, J)
    h = 1e-6
    for k in range(coef.shape[1]):
        e = np.zeros_like(coef)
        e[:, k] = h
        Fp_, Jp = geometry(rom, coef + e)
        Fm_, Jm = geometry(rom, coef - e)
        assert np.abs((Fp_ - Fm_) / (2 * h) - dFinv[:, :, k]).max() <= 1e-7 * np.abs(dFinv).max()
        assert np.abs((Jp - Jm) / (2 * h) - dJ[:, :, k]).max() <= 1e-7 * np.abs(dJ).max()
