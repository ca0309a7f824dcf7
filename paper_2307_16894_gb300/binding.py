"""Thin ctypes binding of the C ABI in include/podecm.h (argument marshalling only).

Every step of the hyper-reduced solve runs in libpodecm.so's CUDA kernels;
there is no CPU fallback: loading fails loudly if the library is missing.
Names follow the C calls (rom_create -> Context, rom_load_basis ->
Context.load_basis, ...).  Device buffers are torch CUDA tensors (plumbing
only); host buffers are numpy arrays.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpodecm.so")

ROM_OK, ROM_E_ARG, ROM_E_STATE, ROM_E_CUDA, ROM_E_NOMEM, ROM_E_NOT_CONVERGED, ROM_E_NONFINITE = range(7)
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
START = {"plain": 0, "prev": 1, "mlp": 2}

INFO_DTYPE = np.dtype([("iters", "<i4"), ("evals", "<i4"), ("status", "<i4"), ("n_yield", "<i4"),
                       ("res0", "<f8"), ("res", "<f8")])

EXPORTED = ["rom_create", "rom_destroy", "rom_load_basis", "rom_load_cubature", "rom_set_geometry",
            "rom_state_create", "rom_state_destroy", "rom_state_export", "rom_state_import", "rom_step",
            "rom_step_device", "rom_sync", "rom_last_error", "rom_profile", "rom_profile_read",
            "rom_step_noalloc", "rom_mlp_init", "rom_mlp_nparams", "rom_mlp_params", "rom_mlp_norm",
            "rom_mlp_train_step", "rom_mlp_loss_grad", "rom_mlp_predict", "rom_features", "rom_debug_stiffness",
            "rom_debug_tangent", "rom_debug_residual", "rom_use_graphs", "rom_sensitivity", "rom_sensitivity_device",
            "rom_state_bytes", "rom_autotune", "rom_serve", "rom_set_geometry_aux", "rom_pod", "rom_ecm",
            "rom_fe_train", "rom_ecm_integrands"]

KERNEL_GROUPS = ["start", "constitutive", "assemble", "solve", "finalize", "bookkeeping", "learned_start", "force",
                 "sensitivity"]


class RomPhase(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("hard_law", ctypes.c_int32),
                ("s0", ctypes.c_double), ("H_or_k", ctypes.c_double), ("p", ctypes.c_double)]


class RomOpts(ctypes.Structure):
    _fields_ = [("tol_rel", ctypes.c_double), ("tol_abs", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("max_ls", ctypes.c_int32), ("precision", ctypes.c_int32), ("start", ctypes.c_int32),
                ("polar_split", ctypes.c_int32), ("want_abar", ctypes.c_int32), ("fp64_residual", ctypes.c_int32)]


class RomNoallocModel(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int32), ("m", ctypes.c_int32), ("n_par", ctypes.c_int32),
                ("n_phase", ctypes.c_int32), ("G", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("phase", ctypes.c_void_p), ("Gmu", ctypes.c_void_p), ("phases", ctypes.c_void_p),
                ("omega_vol", ctypes.c_double)]


class RomAuxModel(ctypes.Structure):
    _fields_ = [("n_p", ctypes.c_int32), ("n_rb", ctypes.c_int32), ("n_deim", ctypes.c_int32),
                ("mu_ref", ctypes.c_void_p), ("Ahat", ctypes.c_void_p), ("Mdeim", ctypes.c_void_p),
                ("S", ctypes.c_void_p), ("GL", ctypes.c_void_p), ("Gpsi", ctypes.c_void_p)]


class RomFeMesh(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("ne", ctypes.c_int32), ("nen", ctypes.c_int32), ("ngp", ctypes.c_int32),
                ("ndof", ctypes.c_int32), ("edof", ctypes.c_void_p), ("dN", ctypes.c_void_p), ("gw", ctypes.c_void_p),
                ("el_phase", ctypes.c_void_p)]


class RomError(RuntimeError):
    pass


_lib = None


def lib(path=None):
    """Load libpodecm.so (built by __graft_entry__.build()); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RomError("CUDA library %s not built (run __graft_entry__.build())" % path)
    L = ctypes.CDLL(path)
    p, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.rom_create.argtypes = [pp, i, i, p]
    L.rom_destroy.argtypes = [p]
    L.rom_load_basis.argtypes = [p, i, i, p]
    L.rom_load_cubature.argtypes = [p, i, p, p, i, p, d]
    L.rom_set_geometry.argtypes = [p, i64, i, p, p]
    L.rom_set_geometry_aux.argtypes = [p, i64, p, p]
    L.rom_pod.argtypes = [p, i64, i, p, p, p, p, p, i, p, p, p, p, ctypes.c_size_t]
    L.rom_fe_train.argtypes = [p, i, p, i, i, p, p, i, p, d, d, i, i, p, p, p, p, p, p, ctypes.c_size_t]
    L.rom_ecm_integrands.argtypes = [p, p, i, p, i, p, p, p, p, ctypes.c_size_t]
    L.rom_ecm.argtypes = [p, i, i64, p, p, i, d, d, i, p, p, p, p, p, p, ctypes.c_size_t]
    L.rom_state_create.argtypes = [p, i64, pp]
    L.rom_state_destroy.argtypes = [p]
    L.rom_state_export.argtypes = [p, p, p, p, p]
    L.rom_state_import.argtypes = [p, p, p, p, p]
    L.rom_step.argtypes = [p, p, p, p, p, p, p]
    L.rom_step_device.argtypes = [p, p, p, p, p, p, p]
    L.rom_sync.argtypes = [p]
    L.rom_profile.argtypes = [p, i]
    L.rom_profile_read.argtypes = [p, i, p, p, p]
    L.rom_step_noalloc.argtypes = [p, i64, p, p, p, p, p, p, p, p, p, p, p, p, ctypes.c_size_t]
    L.rom_mlp_init.argtypes = [p, i, i, i, i, i64]
    L.rom_mlp_nparams.argtypes = [p, p]
    L.rom_mlp_params.argtypes = [p, p, p]
    L.rom_mlp_norm.argtypes = [p, p]
    L.rom_mlp_train_step.argtypes = [p, p, p, i64, ctypes.c_float, i, p]
    L.rom_mlp_loss_grad.argtypes = [p, p, p, i64, i, p, p]
    L.rom_mlp_predict.argtypes = [p, p, i64, i, p]
    L.rom_features.argtypes = [p, p, p, p]
    L.rom_debug_stiffness.argtypes = [p, p, p]
    L.rom_debug_tangent.argtypes = [p, p, p, i64]
    L.rom_use_graphs.argtypes = [p, i]
    L.rom_state_bytes.argtypes = [p, i64, p]
    L.rom_autotune.argtypes = [p, p, p, p, p, p]
    L.rom_serve.argtypes = [i, p, p, p, p, p, p, p, p]
    L.rom_last_error.argtypes = [p]
    L.rom_last_error.restype = ctypes.c_char_p
    for f in EXPORTED:
        if f != "rom_last_error":
            getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _p(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_opts(tol_rel=1e-10, tol_abs=0.0, max_iter=25, max_ls=6, precision="fp64", start="plain",
              polar_split=True, want_abar=True, fp64_residual=False):
    return RomOpts(float(tol_rel), float(tol_abs), int(max_iter), int(max_ls), PREC[precision], START[start],
                   int(bool(polar_split)), int(bool(want_abar)), int(bool(fp64_residual)))


class Context:
    """rom_ctx: one model (basis, cubature, geometry) on one device and stream.

    stream: a cudaStream_t (int) or None (the context creates its own); 0 (torch's
    default stream) is passed as cudaStreamLegacy.  A context that receives torch
    tensors must run on the stream those tensors are used on
    (torch.cuda.current_stream().cuda_stream)."""

    def __init__(self, dim, device=0, stream=None):
        self.L = lib()
        self.dim = dim
        h = ctypes.c_void_p()
        if stream is None:
            st = None                       # the library creates its own stream
        elif int(stream) == 0:
            st = ctypes.c_void_p(1)         # handle 0 = legacy default stream -> cudaStreamLegacy
        else:
            st = ctypes.c_void_p(int(stream))
        self._check(self.L.rom_create(ctypes.byref(h), int(dim), int(device), st), "rom_create", ctx=None)
        self.h = h
        self.n = self.m = self.n_par = 0

    def _check(self, status, what, ctx="self"):
        if status != ROM_OK:
            msg = ""
            if ctx == "self" and getattr(self, "h", None):
                msg = self.L.rom_last_error(self.h).decode()
            raise RomError("%s failed with status %d: %s" % (what, status, msg))

    def close(self):
        if getattr(self, "h", None):
            self.L.rom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_basis(self, G):
        G = _f64(G)
        m, d2, n = G.shape
        self._check(self.L.rom_load_basis(self.h, n, m, _p(G)), "rom_load_basis")
        self.n, self.m = n, m

    def load_cubature(self, w, phase, phases, omega=1.0):
        w = _f64(w)
        phase = np.ascontiguousarray(phase, dtype=np.int32)
        arr = (RomPhase * len(phases))()
        for k, ph in enumerate(phases):
            arr[k] = RomPhase(ph["E"], ph["nu"], 1 if ph.get("law", "power") == "power" else 0, ph["s0"], ph["k"],
                              ph.get("p", 1.0))
        self._check(self.L.rom_load_cubature(self.h, len(w), _p(w), _p(phase), len(phases),
                                             ctypes.cast(arr, ctypes.c_void_p), float(omega)), "rom_load_cubature")

    def set_geometry(self, Gmu, mu):
        Gmu = _f64(Gmu)
        mu = _f64(mu)
        B, n_par = mu.shape
        self._check(self.L.rom_set_geometry(self.h, B, n_par, _p(Gmu), _p(mu)), "rom_set_geometry")
        self.n_par = n_par

    def set_geometry_aux(self, rom, mu):
        """rom_set_geometry_aux: the reduced auxiliary problem (Sec. 3.4) of a model file with
        map = "aux" (aux_mu_ref, aux_Ahat, aux_Mdeim, aux_S, aux_GL, aux_Gpsi), solved on the
        device for the shape parameters mu [B, n_p]."""
        keep = [_f64(rom[k]) for k in ("aux_mu_ref", "aux_Ahat", "aux_Mdeim", "aux_S", "aux_GL", "aux_Gpsi")]
        mu = _f64(np.atleast_2d(mu))
        n_p, n_rb, n_deim = keep[0].size, keep[1].shape[0], keep[2].shape[1]
        a = RomAuxModel(n_p, n_rb, n_deim, *[k.ctypes.data for k in keep])
        self._check(self.L.rom_set_geometry_aux(self.h, mu.shape[0], ctypes.byref(a), _p(mu)), "rom_set_geometry_aux")
        self.n_par = n_p + n_rb

    def state_create(self, B):
        h = ctypes.c_void_p()
        self._check(self.L.rom_state_create(self.h, int(B), ctypes.byref(h)), "rom_state_create")
        return State(self, h, B)

    def step(self, state, opts, Fbar, want_abar=True):
        """Host-buffer step: returns (Pbar [B,d,d], Abar [B,d2,d2] or None, info [B] structured)."""
        d = self.dim
        Fbar = _f64(Fbar)
        B = Fbar.shape[0]
        Pbar = np.empty((B, d, d))
        Abar = np.empty((B, d * d, d * d)) if want_abar else None
        info = np.zeros(B, INFO_DTYPE)
        self._check(self.L.rom_step(self.h, state.h, ctypes.byref(opts), _p(Fbar), _p(Pbar), _p(Abar), _p(info)),
                    "rom_step")
        return Pbar, Abar, info

    def step_device(self, state, opts, Fbar_d, Pbar_d, Abar_d, info_d):
        """Device-buffer step (torch CUDA tensors), asynchronous on the context stream."""
        self._check(self.L.rom_step_device(self.h, state.h, ctypes.byref(opts), _p(Fbar_d), _p(Pbar_d),
                                           _p(Abar_d), _p(info_d)), "rom_step_device")

    def sensitivity(self, state):
        """dPbar/dmu [B, d, d, n_par] of the last step (Eq. eff_sensitivities_full); NaN where the
        step did not converge."""
        out = np.empty((state.B, self.dim, self.dim, self.n_par))
        self._check(self.L.rom_sensitivity(self.h, state.h, _p(out)), "rom_sensitivity")
        return out

    def sensitivity_device(self, state, out_d):
        """Same into a device buffer of B * d * d * n_par doubles, asynchronous on the stream."""
        self._check(self.L.rom_sensitivity_device(self.h, state.h, _p(out_d)), "rom_sensitivity_device")

    def sync(self):
        self._check(self.L.rom_sync(self.h), "rom_sync")

    def state_bytes(self, B):
        v = ctypes.c_int64()
        self._check(self.L.rom_state_bytes(self.h, int(B), ctypes.byref(v)), "rom_state_bytes")
        return v.value

    def autotune(self, state, opts):
        t, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        self._check(self.L.rom_autotune(self.h, state.h, ctypes.byref(opts), ctypes.byref(t), ctypes.byref(c),
                                        ctypes.byref(ms)), "rom_autotune")
        return t.value, c.value, ms.value

    def use_graphs(self, enable=True):
        self._check(self.L.rom_use_graphs(self.h, int(enable)), "rom_use_graphs")

    # ---- learned Newton start
    def mlp_init(self, n_in, width, depth, n_out, max_rows):
        self._check(self.L.rom_mlp_init(self.h, n_in, width, depth, n_out, int(max_rows)), "rom_mlp_init")
        n = ctypes.c_int64()
        self._check(self.L.rom_mlp_nparams(self.h, ctypes.byref(n)), "rom_mlp_nparams")
        self.mlp_shape = (n_in, width, depth, n_out)
        return n.value

    def mlp_params(self, set_params=None):
        n = ctypes.c_int64()
        self._check(self.L.rom_mlp_nparams(self.h, ctypes.byref(n)), "rom_mlp_nparams")
        out = np.empty(n.value, np.float32)
        sp = None if set_params is None else np.ascontiguousarray(set_params, np.float32)
        self._check(self.L.rom_mlp_params(self.h, _p(out), _p(sp)), "rom_mlp_params")
        return out

    def mlp_norm(self, x_mean, x_std, y_mean, y_std):
        v = np.ascontiguousarray(np.concatenate([x_mean, x_std, y_mean, y_std]), np.float32)
        self._check(self.L.rom_mlp_norm(self.h, _p(v)), "rom_mlp_norm")

    def mlp_train_step(self, X_d, Y_d, lr, t, loss_d=None):
        self._check(self.L.rom_mlp_train_step(self.h, _p(X_d), _p(Y_d), X_d.shape[0], float(lr), int(t), _p(loss_d)),
                    "rom_mlp_train_step")

    def mlp_loss_grad(self, X_d, Y_d, bf16, grad_d, loss_d):
        self._check(self.L.rom_mlp_loss_grad(self.h, _p(X_d), _p(Y_d), X_d.shape[0], int(bf16), _p(grad_d),
                                             _p(loss_d)), "rom_mlp_loss_grad")

    def mlp_predict(self, X_d, bf16, out_d):
        self._check(self.L.rom_mlp_predict(self.h, _p(X_d), X_d.shape[0], int(bf16), _p(out_d)), "rom_mlp_predict")

    def features(self, state, Fbar_d, X_d):
        self._check(self.L.rom_features(self.h, state.h, _p(Fbar_d), _p(X_d)), "rom_features")

    def profile(self, enable):
        self._check(self.L.rom_profile(self.h, int(enable)), "rom_profile")

    def profile_read(self):
        """{group: (ms, launches, flops)} of the kernels timed since profile(1)."""
        out = {}
        for k, name in enumerate(KERNEL_GROUPS):
            ms, ln, fl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
            self._check(self.L.rom_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(ln), ctypes.byref(fl)),
                        "rom_profile_read")
            out[name] = (ms.value, ln.value, fl.value)
        return out


class State:
    """rom_state: reduced coordinates and history of B instances."""

    def __init__(self, ctx, h, B):
        self.ctx, self.h, self.B = ctx, h, B

    def stiffness(self):
        """K [B, n, n] of the last evaluated iterate (diagnostics)."""
        c = self.ctx
        K = np.empty((self.B, c.n, c.n))
        c._check(c.L.rom_debug_stiffness(c.h, self.h, _p(K)), "rom_debug_stiffness")
        return K

    def tangent(self, fp64):
        """At [B, d^4, m] of the last pass (diagnostics); fp64: the step ran with precision fp64."""
        c = self.ctx
        d4 = c.dim ** 4
        mA = (c.m + 3) & ~3
        At = np.empty((self.B, d4, mA), dtype=np.float64 if fp64 else np.float32)
        c._check(c.L.rom_debug_tangent(c.h, self.h, _p(At), At.nbytes), "rom_debug_tangent")
        return At[:, :, :c.m]

    def residual(self):
        """(r [B, n], v [B, d*d, m]) of the last pass (diagnostics)."""
        c = self.ctx
        r = np.empty((self.B, c.n))
        v = np.empty((self.B, c.dim * c.dim, c.m))
        c._check(c.L.rom_debug_residual(c.h, self.h, _p(r), _p(v)), "rom_debug_residual")
        return r, v

    def export(self, history=True):
        """(a [B, n], C^p^-1 [B, m, nc], xi [B, m]); history=False skips the last two (None)."""
        c = self.ctx
        nc = 4 if c.dim == 2 else 6
        a = np.empty((self.B, c.n))
        cp = np.empty((self.B, c.m, nc)) if history else None
        xi = np.empty((self.B, c.m)) if history else None
        c._check(c.L.rom_state_export(c.h, self.h, _p(a), _p(cp), _p(xi)), "rom_state_export")
        return a, cp, xi

    def import_(self, a=None, Cpinv=None, xi=None):
        c = self.ctx
        c._check(c.L.rom_state_import(c.h, self.h, _p(None if a is None else _f64(a)),
                                      _p(None if Cpinv is None else _f64(Cpinv)),
                                      _p(None if xi is None else _f64(xi))), "rom_state_import")

    def close(self):
        if self.h:
            self.ctx.L.rom_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def phase_array(phases):
    arr = (RomPhase * len(phases))()
    for k, ph in enumerate(phases):
        arr[k] = RomPhase(ph["E"], ph["nu"], 1 if ph.get("law", "power") == "power" else 0, ph["s0"], ph["k"],
                          ph.get("p", 1.0))
    return arr


def step_noalloc(dim, G_d, w_d, phase_d, Gmu_d, phases, omega, mu_d, a_d, da_prev_d, Cpinv_d, xi_d, opts,
                 Fbar_d, Pbar_d, Abar_d, info_d, stream=None):
    """rom_step_noalloc: one load step with every array supplied by the caller (torch CUDA
    tensors) and the work space in the library's static device array."""
    L = lib()
    m, d2, n = G_d.shape
    arr = phase_array(phases)
    model = RomNoallocModel(dim, n, m, Gmu_d.shape[-1], len(phases), G_d.data_ptr(), w_d.data_ptr(),
                            phase_d.data_ptr(), Gmu_d.data_ptr(), ctypes.cast(arr, ctypes.c_void_p), float(omega))
    buf = ctypes.create_string_buffer(512)
    st = L.rom_step_noalloc(ctypes.byref(model), int(mu_d.shape[0]), _p(mu_d), _p(a_d), _p(da_prev_d), _p(Cpinv_d),
                            _p(xi_d), ctypes.byref(opts), _p(Fbar_d), _p(Pbar_d), _p(Abar_d), _p(info_d),
                            ctypes.c_void_p(stream) if stream else None, buf, 512)
    if st != ROM_OK:
        raise RomError("rom_step_noalloc failed with status %d: %s" % (st, buf.value.decode()))


def serve(ctxs, states, opts, F, P, A=None, I=None):
    """rom_serve: one load step for G groups (torch device buffers); returns group_ms [G]."""
    L = lib()
    G = len(ctxs)
    VP = ctypes.c_void_p * G
    o = (RomOpts * G)(*opts)
    ms = (ctypes.c_float * G)()
    arr = lambda xs: VP(*[x.data_ptr() for x in xs]) if xs is not None else None
    st = L.rom_serve(G, VP(*[c.h.value for c in ctxs]), VP(*[s.h.value for s in states]), o, arr(F), arr(P),
                     arr(A), arr(I), ms)
    if st != ROM_OK:
        raise RomError("rom_serve failed with status %d: %s" % (st, L.rom_last_error(ctxs[0].h).decode()))
    return np.array(ms[:])


# ---- offline stage on the device (context-free calls)
def pod(S_d, n_modes, M=None, wdiag_d=None, stream=None):
    """rom_pod on torch CUDA tensors: S_d [ns, N] (float64); M a scipy CSR matrix (copied to the
    device) or None; wdiag_d [N] or None.  Returns (Phi [n_modes, N] tensor, lam [ns] tensor, sweeps)."""
    import torch
    L = lib()
    ns, N = S_d.shape
    dev = S_d.device
    Phi = torch.empty((n_modes, N), dtype=torch.float64, device=dev)
    lam = torch.empty(ns, dtype=torch.float64, device=dev)
    keep = []
    rp = cl = vl = None
    if M is not None:
        rp = torch.as_tensor(np.ascontiguousarray(M.indptr, dtype=np.int32), device=dev)
        cl = torch.as_tensor(np.ascontiguousarray(M.indices, dtype=np.int32), device=dev)
        vl = torch.as_tensor(np.ascontiguousarray(M.data, dtype=np.float64), device=dev)
        keep += [rp, cl, vl]
    sw = ctypes.c_int()
    err = ctypes.create_string_buffer(512)
    st = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    s = L.rom_pod(st, N, ns, _p(S_d.contiguous()), _p(rp), _p(cl), _p(vl), _p(wdiag_d), int(n_modes), _p(Phi),
                  _p(lam), ctypes.byref(sw), err, len(err))
    if s != ROM_OK:
        raise RomError("rom_pod failed with status %d: %s" % (s, err.value.decode()))
    return Phi, lam, sw.value


def ecm(F_d, wq_d, m=None, tol=None, volume_weight=10.0, cap=None, stream=None):
    """rom_ecm on torch CUDA tensors F_d [P, M], wq_d [M] (float64).  Returns (idx, w, err, rank)."""
    import torch
    L = lib()
    P, Mq = F_d.shape
    mm = int(m) if m is not None else 0
    cap = int(cap or (mm if mm > 0 else min(Mq, 4096)))
    idx = np.zeros(cap, np.int64)
    w = np.zeros(cap)
    mo, rk, er = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    err = ctypes.create_string_buffer(512)
    st = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    s = L.rom_ecm(st, P, Mq, _p(F_d.contiguous()), _p(wq_d.contiguous()), mm, float(tol or 0.0), float(volume_weight),
                  cap, _p(idx), _p(w), ctypes.byref(mo), ctypes.byref(er), ctypes.byref(rk), err, len(err))
    if s != ROM_OK:
        raise RomError("rom_ecm failed with status %d: %s" % (s, err.value.decode()))
    return idx[:mo.value], w[:mo.value], er.value, rk.value


def _phase_array(phases):
    arr = (RomPhase * len(phases))()
    for k, ph in enumerate(phases):
        arr[k] = RomPhase(ph["E"], ph["nu"], 1 if ph.get("law", "power") == "power" else 0, ph["s0"], ph["k"],
                          ph.get("p", 1.0))
    return arr


def fe_mesh(grid):
    """rom_fe_mesh of a mesh.Grid (the arrays are kept alive on the returned structure)"""
    keep = [np.ascontiguousarray(grid.edof, np.int32), _f64(grid.dN), _f64(grid.gw),
            np.ascontiguousarray(grid.el_phase, np.int32)]
    m = RomFeMesh(grid.d, grid.ne, grid.nen, grid.ngp, grid.ndof, *[k.ctypes.data for k in keep])
    m._keep = keep
    return m


def fe_train(grid, phases, Gq, coef, paths, tol_rel=1e-10, tol_abs=1e-9, max_iter=40, max_split=8, want_W=True):
    """rom_fe_train: full-order training solves of S samples.  Gq [nq, d, d, n_par], coef [S, n_par],
    paths [S, steps, d, d] (host).  Returns dict(w [S, steps, ndof], W [S, steps, nq, d*d] or None,
    Pbar [S, steps, d, d], iters, substeps)."""
    L = lib()
    d = grid.d
    coef = _f64(np.atleast_2d(coef))
    paths = _f64(paths)
    S, steps = paths.shape[:2]
    n_par = coef.shape[1]
    Gq = _f64(Gq).reshape(grid.nq, d * d, n_par)
    w = np.zeros((S, steps, grid.ndof))
    W = np.zeros((S, steps, grid.nq, d * d)) if want_W else None
    Pbar = np.zeros((S, steps, d, d))
    its = np.zeros((S, steps), np.int32)
    sub = np.zeros((S, steps), np.int32)
    m = fe_mesh(grid)
    arr = _phase_array(phases)
    err = ctypes.create_string_buffer(512)
    st = L.rom_fe_train(ctypes.byref(m), len(phases), ctypes.cast(arr, ctypes.c_void_p), S, n_par, _p(Gq), _p(coef),
                        steps, _p(paths), float(tol_rel), float(tol_abs), int(max_iter), int(max_split), _p(w), _p(W),
                        _p(Pbar), _p(its), _p(sub), err, len(err))
    if st != ROM_OK:
        raise RomError("rom_fe_train failed with status %d: %s" % (st, err.value.decode()))
    return dict(w=w, W=W, Pbar=Pbar, iters=its, substeps=sub)


def ecm_integrands(grid, Phi_d, B_d, stream=None):
    """rom_ecm_integrands on torch CUDA tensors Phi_d [n, ndof], B_d [L, nq, d*d]; returns
    (gradPhi [nq, d*d, n], F [n*L, nq]) tensors."""
    import torch
    L = lib()
    n, Lm = Phi_d.shape[0], B_d.shape[0]
    gradPhi = torch.empty((grid.nq, grid.d * grid.d, n), dtype=torch.float64, device=Phi_d.device)
    F = torch.empty((n * Lm, grid.nq), dtype=torch.float64, device=Phi_d.device)
    m = fe_mesh(grid)
    err = ctypes.create_string_buffer(512)
    st = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    s = L.rom_ecm_integrands(st, ctypes.byref(m), n, _p(Phi_d.contiguous()), Lm, _p(B_d.contiguous()), _p(gradPhi),
                             _p(F), err, len(err))
    if s != ROM_OK:
        raise RomError("rom_ecm_integrands failed with status %d: %s" % (s, err.value.decode()))
    return gradPhi, F
