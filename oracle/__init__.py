"""ORACLE — test infrastructure only.

Plain FP64 CPU reference of the paper's method (arXiv 2307.16894): the
finite-strain J2 material point (Appendix A), the full-order FE model on the
parent domain (Sec. 2), POD and ECM (Sec. 3.1-3.2, Algorithm 1 offline) and
the online hyper-reduced Newton solve with effective stress and stiffness
(Sec. 3.2-3.3, Algorithm 1 online).  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path of ``paper_2307_16894_gb300``.

The compute-heavy loops are plain C (``orc_material.c``, ``orc_rom.c``)
loaded through ctypes; this module is the marshalling layer.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_SRC = ["orc_material.c", "orc_rom.c"]

HARD_LINEAR = 0
HARD_POWER = 1


class Phase(ctypes.Structure):
    """Material phase: linear sigma_y = s0 + H xi, power sigma_y = s0 (1 + k xi)^p;
    s0 = inf means purely elastic (Appendix A, Eq. j2_2)."""
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("hard_law", ctypes.c_int),
                ("s0", ctypes.c_double), ("H_or_k", ctypes.c_double), ("p", ctypes.c_double)]


def build(force=False):
    """Compile the C oracle with gcc into oracle/_build/liborc.so."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "orc.h")])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB names a prebuilt copy of this library to load instead; the planted-mistake
        # tests point it at deliberately broken builds of these sources
        _lib = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
        d = ctypes.c_double
        i = ctypes.c_int
        p = ctypes.c_void_p
        _lib.orc_material_batch.argtypes = [i, i, p, p, p, p, p, p, p, p, p, p, p]
        _lib.orc_rom_step.restype = i
        _lib.orc_rom_batch.argtypes = [i, i, i, i, i, i, p, p, p, p, p, p, d, p, p, p, p, d, d, i, i,
                                       p, p, p, p, p, p, p, p, p, i, p, p, p]
        _lib.orc_fe_elements.argtypes = [i, i, i, i, p, p, p, p, p, p, p, p, p, p, p, p,
                                         p, p, p, p, p, p, p, p, i, i]
        _lib.orc_polar.argtypes = [i, p, p, p]
        _lib.orc_sigma_y.restype = d
        _lib.orc_sigma_y.argtypes = [p, d, p]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def phases_array(phases):
    """list of dicts (E, nu, law, s0, k, p) -> ctypes array of Phase"""
    arr = (Phase * len(phases))()
    for j, ph in enumerate(phases):
        law = HARD_POWER if ph.get("law", "power") == "power" else HARD_LINEAR
        arr[j] = Phase(ph["E"], ph["nu"], law, ph["s0"], ph["k"], ph.get("p", 1.0))
    return arr


def sigma_y(phase, xi):
    arr = phases_array([phase])
    return lib().orc_sigma_y(ctypes.cast(arr, ctypes.c_void_p), float(xi), None)


def material(d, F3, Fp, xi, phase_idx, phases, tangent=True):
    """Material update at npt independent points (Appendix A).

    F3, Fp: [npt, 3, 3]; xi: [npt]; returns P [npt,d,d], A [npt,d*d,d*d] (or None),
    P33 [npt], Fp_new [npt,3,3], xi_new [npt], plastic [npt] (bool)."""
    F3 = _f64(F3).reshape(-1, 9)
    npt = F3.shape[0]
    Fp = _f64(Fp).reshape(npt, 9)
    xi = _f64(xi).reshape(npt)
    ph = _i32(np.broadcast_to(np.asarray(phase_idx), (npt,)))
    P = np.zeros((npt, d * d))
    A = np.zeros((npt, d ** 4)) if tangent else None
    P33 = np.zeros(npt)
    Fpn = np.zeros((npt, 9))
    xin = np.zeros(npt)
    pl = np.zeros(npt, dtype=np.int32)
    parr = phases_array(phases)
    lib().orc_material_batch(d, npt, _ptr(F3), _ptr(Fp), _ptr(xi), _ptr(ph), ctypes.cast(parr, ctypes.c_void_p),
                             _ptr(P), _ptr(A), _ptr(P33), _ptr(Fpn), _ptr(xin), _ptr(pl))
    return (P.reshape(npt, d, d), None if A is None else A.reshape(npt, d * d, d * d), P33,
            Fpn.reshape(npt, 3, 3), xin, pl.astype(bool))


def polar(F):
    F = _f64(F)
    d = F.shape[-1]
    R = np.zeros_like(F)
    U = np.zeros_like(F)
    lib().orc_polar(d, _ptr(F), _ptr(R), _ptr(U))
    return R, U


def geometry_derivatives(rom, Finv, J):
    """dF_mu^-1/dmu_k = -F_mu^-1 Gmu_k F_mu^-1 and d|det F_mu|/dmu_k = |det F_mu| tr(F_mu^-1 Gmu_k)
    at every point, for the affine map F_mu = I + sum_k mu_k Gmu_k (the derivative of the inverse
    and of the determinant that Eq. eff_sensitivities_full needs).  Finv [B, m, d, d], J [B, m]
    -> dFinv [B, m, n_par, d, d], dJ [B, m, n_par]."""
    d, m = rom["d"], rom["m"]
    Gmu = rom["Gmu"].reshape(m, d, d, -1)                         # [m, d, d, n_par]
    FG = np.einsum("bmac,mcdk->bmkad", Finv, Gmu)                 # F_mu^-1 Gmu_k
    dFinv = -np.einsum("bmkac,bmcd->bmkad", FG, Finv)
    dJ = J[:, :, None] * np.einsum("bmkaa->bmk", FG)
    return np.ascontiguousarray(dFinv), np.ascontiguousarray(dJ)


def rom_batch(rom, Finv, J, Fbar, q, Fp, xi, tol_rel, tol_abs, max_iter, max_ls=6, polar_split=True,
              nthreads=None, want_A=True, dFinv=None, dJ=None):
    """One load step of the online reduced solve for B instances (in place on q, Fp, xi).

    rom: dict with d, n, m, G [m, d*d, n], w [m], phase [m], phases (list), omega.
    Finv [B, m, d, d], J [B, m], Fbar [B, d, d], q [B, n] (start iterate on entry,
    solution on exit), Fp [B, m, 3, 3], xi [B, m].  With dFinv, dJ (geometry_derivatives)
    the outputs include the shape sensitivities dPdmu [B, d, d, n_par].  Returns a dict."""
    d, n, m = rom["d"], rom["n"], rom["m"]
    B = Fbar.shape[0]
    for name, arr in (("q", q), ("Fp", Fp), ("xi", xi)):
        assert arr.dtype == np.float64 and arr.flags.c_contiguous, name
    G = _f64(rom["G"])
    w = _f64(rom["w"])
    ph = _i32(rom["phase"])
    Finv = _f64(Finv)
    J = _f64(J)
    Fbar = _f64(Fbar)
    out = {
        "Pbar": np.zeros((B, d, d)), "Abar": np.zeros((B, d * d, d * d)) if want_A else None,
        "P33bar": np.zeros(B), "iters": np.zeros(B, np.int32), "evals": np.zeros(B, np.int32),
        "n_yield": np.zeros(B, np.int32),
        "status": np.zeros(B, np.int32), "res0": np.zeros(B), "res": np.zeros(B)}
    npar = 0
    if dFinv is not None:
        npar = dFinv.shape[2]
        dFinv, dJ = _f64(dFinv), _f64(dJ)
        out["dPdmu"] = np.zeros((B, d, d, npar))
    parr = phases_array(rom["phases"])
    nthreads = nthreads or min(os.cpu_count() or 1, max(B, 1))
    lib().orc_rom_batch(B, nthreads, 1 if polar_split else 0, d, n, m, _ptr(G), _ptr(w), _ptr(ph),
                        ctypes.cast(parr, ctypes.c_void_p), _ptr(Finv), _ptr(J), float(rom.get("omega", 1.0)),
                        _ptr(Fbar), _ptr(q), _ptr(Fp), _ptr(xi), float(tol_rel), float(tol_abs), int(max_iter),
                        int(max_ls), _ptr(out["Pbar"]), _ptr(out["Abar"]), _ptr(out["P33bar"]), _ptr(out["iters"]),
                        _ptr(out["evals"]), _ptr(out["n_yield"]), _ptr(out["status"]), _ptr(out["res0"]), _ptr(out["res"]),
                        npar, _ptr(dFinv) if npar else None, _ptr(dJ) if npar else None,
                        _ptr(out["dPdmu"]) if npar else None)
    return out


def fe_elements(mesh, phases, Finv, J, Fbar, wdofs, Fp, xi, want_K=True, nthreads=None):
    """Element loops of the mapped full-order weak form (Sec. 2.1)."""
    d, ne, nen, ngp = mesh.d, mesh.ne, mesh.nen, mesh.ngp
    ned = nen * d
    fe = np.zeros((ne, ned))
    Ke = np.zeros((ne, ned, ned)) if want_K else None
    nq = ne * ngp
    Fp_tr = np.zeros((nq, 9))
    xi_tr = np.zeros(nq)
    Pq = np.zeros((nq, d * d))
    Aq = np.zeros((nq, d ** 4))
    P33q = np.zeros(nq)
    plq = np.zeros(nq, np.int32)
    parr = phases_array(phases)
    lib().orc_fe_elements(d, ne, nen, ngp, _ptr(_i32(mesh.conn)), _ptr(_i32(mesh.dofmap)), _ptr(_i32(mesh.el_phase)),
                          ctypes.cast(parr, ctypes.c_void_p), _ptr(_f64(mesh.dN)), _ptr(_f64(mesh.gw)),
                          _ptr(_f64(Finv)), _ptr(_f64(J)), _ptr(_f64(Fbar)), _ptr(_f64(wdofs)),
                          _ptr(_f64(Fp)), _ptr(_f64(xi)), _ptr(fe), _ptr(Ke), _ptr(Fp_tr), _ptr(xi_tr),
                          _ptr(Pq), _ptr(Aq), _ptr(P33q), _ptr(plq), 1 if want_K else 0,
                          nthreads or (os.cpu_count() or 1))
    return dict(fe=fe, Ke=Ke, Fp_tr=Fp_tr, xi_tr=xi_tr, Pq=Pq, Aq=Aq, P33q=P33q, plastic=plq.astype(bool))
