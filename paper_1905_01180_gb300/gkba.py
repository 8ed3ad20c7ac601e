"""Thin Python binding of libgkba (include/gkba.h): argument marshalling only.

Every step of the GKBA second-Born path runs in the library's CUDA kernels;
this module converts numpy arrays (host buffers) or torch CUDA tensors
(device buffers) into the C ABI's pointers and sizes.  It fails loudly when
the shared library is missing: there is no CPU fallback.

Complex arrays are complex128 (interleaved re, im), N x N row-major; v is
float64 with shape (N, N, N, N) (general interaction), (N,) (U_i of the
diagonal basis) or (N, N) (V_ij of the symmetric basis).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgkba.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT, ENUMERIC, EUNSUPPORTED = range(8)
FP64, SPLIT_TF32, SPLIT_TF32_ACC = 0, 1, 2
V_GENERAL, V_DIAGONAL, V_SYMMETRIC = 0, 1, 2
HISTORY_SUM, HISTORY_TIME_LINEAR = 0, 1
_HISTORY = {"sum": HISTORY_SUM, "time_linear": HISTORY_TIME_LINEAR,
            HISTORY_SUM: HISTORY_SUM, HISTORY_TIME_LINEAR: HISTORY_TIME_LINEAR}
_INTERACTION = {"general": V_GENERAL, "diagonal": V_DIAGONAL, "symmetric": V_SYMMETRIC,
                V_GENERAL: V_GENERAL, V_DIAGONAL: V_DIAGONAL, V_SYMMETRIC: V_SYMMETRIC}
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESTATE", 5: "ETIMEOUT",
           6: "ENUMERIC", 7: "EUNSUPPORTED"}

EXPORTED = ["gkba_init", "gkba_sigma", "gkba_collision", "gkba_step", "gkba_set_history",
            "gkba_get_history", "gkba_get_state", "gkba_mean_field", "gkba_adjoint",
            "gkba_get_stats", "gkba_last_error", "gkba_destroy", "gkba_sigma_noalloc",
            "gkba_batch_create", "gkba_batch_step", "gkba_batch_last_error", "gkba_batch_destroy",
            "gkba_selftest_timeout", "gkba_sigma3", "gkba_collision_vjp",
            "gkba_measure_tf32_mma", "gkba_batch_set_options", "gkba_batch_autotune"]


class GKBAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("dt", ctypes.c_double), ("max_steps", ctypes.c_int),
                ("precision", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("device", ctypes.c_int),
                ("timing", ctypes.c_int), ("acc_window", ctypes.c_int),
                ("interaction", ctypes.c_int), ("history", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong),
                ("ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


_lib = None


def load():
    """Load libgkba.so (built by ``paper_1905_01180_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.gkba_init.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Config), P, P, P, P, I]
    L.gkba_sigma.argtypes = [P, I, P, P, P, I]
    L.gkba_collision.argtypes = [P, I, P, P, P, P, I]
    L.gkba_step.argtypes = [P, D, D, P, P, P]
    L.gkba_set_history.argtypes = [P, I, P, P, I]
    L.gkba_get_history.argtypes = [P, ctypes.POINTER(I), P, P]
    L.gkba_get_state.argtypes = [P, ctypes.POINTER(I), P]
    L.gkba_mean_field.argtypes = [P, P, P, I]
    L.gkba_adjoint.argtypes = [P, P, P, P, P]
    L.gkba_get_stats.argtypes = [P, ctypes.POINTER(KernelStat), I, ctypes.POINTER(I),
                                 ctypes.POINTER(ctypes.c_longlong), I]
    L.gkba_last_error.argtypes = [P]
    L.gkba_last_error.restype = ctypes.c_char_p
    L.gkba_destroy.argtypes = [P]
    L.gkba_destroy.restype = None
    L.gkba_sigma_noalloc.argtypes = [I, I, P, P, P, P, P, ctypes.c_char_p, ctypes.c_size_t]
    L.gkba_batch_create.argtypes = [ctypes.POINTER(P), P, I, ctypes.c_size_t]
    L.gkba_selftest_timeout.argtypes = [P, D, P]
    L.gkba_measure_tf32_mma.argtypes = [P, I, P]
    L.gkba_sigma3.argtypes = [P, I, P, P, P, P, I]
    L.gkba_collision_vjp.argtypes = [P, I, P, P, P, P, P, P, P, I]
    L.gkba_batch_step.argtypes = [P, P, P, P, P]
    L.gkba_batch_set_options.argtypes = [P, I]
    L.gkba_batch_autotune.argtypes = [P, P, P, P, P, P, P]
    L.gkba_batch_last_error.argtypes = [P]
    L.gkba_batch_last_error.restype = ctypes.c_char_p
    L.gkba_batch_destroy.argtypes = [P]
    L.gkba_batch_destroy.restype = None
    for name in EXPORTED:
        if name not in ("gkba_last_error", "gkba_destroy", "gkba_batch_last_error",
                        "gkba_batch_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _host(x, dtype):
    a = np.ascontiguousarray(x, dtype=dtype)
    return a, a.ctypes.data


def _dev(x, dtype_name):
    import torch
    want = {"c16": torch.complex128, "f64": torch.float64}[dtype_name]
    if not x.is_cuda:
        raise ValueError("torch tensors passed to libgkba must live on a CUDA device")
    t = x.contiguous()
    if t.dtype != want:
        t = t.to(want)
    return t, t.data_ptr()


class Context:
    """One GKBA system on one GPU (wraps a gkba_ctx).

    precision: "fp64", "tf32" (split-TF32 on the tensor cores) or "tf32acc";
    interaction: "general" (v_ijkl), "diagonal" (U_i) or "symmetric" (V_ij);
    history: "sum" (each step sums the whole history) or "time_linear" (the
    history sum kept as one N^4 accumulator; FP64 and a general v only).
    """

    def __init__(self, h, v, d, rho0, dt, max_steps=0, precision="fp64", stream=None,
                 workspace_bytes=0, device=-1, timing=False, acc_window=0, interaction="general",
                 history="sum"):
        L = load()
        on_dev = _is_torch(h)
        N = int(h.shape[0])
        kind = _INTERACTION[interaction]
        want = {V_GENERAL: (N, N, N, N), V_DIAGONAL: (N,), V_SYMMETRIC: (N, N)}[kind]
        if tuple(v.shape) != want:
            raise ValueError(f"v has shape {tuple(v.shape)}, the {interaction} interaction takes {want}")
        keep = []
        if on_dev:
            ph = _dev(h, "c16"); pv = _dev(v, "f64"); pd = _dev(d, "c16"); pr = _dev(rho0, "c16")
        else:
            ph = _host(h, np.complex128); pv = _host(v, np.float64)
            pd = _host(d, np.complex128); pr = _host(rho0, np.complex128)
        keep += [ph, pv, pd, pr]
        prec = {"fp64": FP64, "tf32": SPLIT_TF32, "tf32acc": SPLIT_TF32_ACC, FP64: FP64,
                SPLIT_TF32: SPLIT_TF32, SPLIT_TF32_ACC: SPLIT_TF32_ACC}[precision]
        cfg = Config(N=N, dt=float(dt), max_steps=int(max_steps), precision=prec,
                     cuda_stream=stream, workspace_bytes=int(workspace_bytes), device=int(device),
                     timing=1 if timing else 0, acc_window=int(acc_window), interaction=kind,
                     history=_HISTORY[history])
        handle = ctypes.c_void_p()
        st = L.gkba_init(ctypes.byref(handle), ctypes.byref(cfg), ph[1], pv[1], pd[1], pr[1],
                         1 if on_dev else 0)
        if st != OK:
            raise GKBAError(st, L.gkba_last_error(None).decode())
        self._h = handle
        self.N = N
        self.dt = float(dt)
        self.max_steps = int(max_steps)
        self.precision = prec
        self.interaction = kind
        self.history = _HISTORY[history]

    # -- helpers -------------------------------------------------------
    def _check(self, st):
        if st != OK:
            raise GKBAError(st, load().gkba_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().gkba_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls ---------------------------------------------------------
    def sigma(self, G, Gbar):
        """Eq. (2bse) for a batch (U, N, N) or a single (N, N) pair."""
        single = G.ndim == 2
        n = 1 if single else int(G.shape[0])
        if _is_torch(G):
            import torch
            g, gp = _dev(G, "c16"); gb, gbp = _dev(Gbar, "c16")
            out = torch.empty_like(g)
            self._check(load().gkba_sigma(self._h, n, gp, gbp, out.data_ptr(), 1))
            return out
        g, gp = _host(G, np.complex128); gb, gbp = _host(Gbar, np.complex128)
        out = np.empty_like(g)
        self._check(load().gkba_sigma(self._h, n, gp, gbp, out.ctypes.data, 0))
        return out

    def collision(self, rho_hist, T_hist, weights=None):
        """First line of Eq. (collint) over the L points of the history."""
        Lh = int(rho_hist.shape[0])
        if _is_torch(rho_hist):
            import torch
            r, rp = _dev(rho_hist, "c16"); t, tp = _dev(T_hist, "c16")
            wp = None
            if weights is not None:
                w, wp = _dev(weights, "f64")
            out = torch.empty((self.N, self.N), dtype=torch.complex128, device=r.device)
            self._check(load().gkba_collision(self._h, Lh, rp, tp, wp, out.data_ptr(), 1))
            return out
        r, rp = _host(rho_hist, np.complex128); t, tp = _host(T_hist, np.complex128)
        wp = None
        if weights is not None:
            w, wp = _host(weights, np.float64)
        out = np.empty((self.N, self.N), np.complex128)
        self._check(load().gkba_collision(self._h, Lh, rp, tp, wp, out.ctypes.data, 0))
        return out

    def sigma3(self, A, B, C):
        """S3(A, B, C)_ij = sum v_irpn w_mqsj A_nm B_sr C_pq for (U, N, N) batches."""
        a, ap = _host(A, np.complex128); b, bp = _host(B, np.complex128)
        c, cp = _host(C, np.complex128)
        n = 1 if a.ndim == 2 else int(a.shape[0])
        out = np.empty_like(a)
        self._check(load().gkba_sigma3(self._h, n, ap, bp, cp, out.ctypes.data, 0))
        return out

    def collision_vjp(self, rho_hist, T_hist, I_bar, weights=None, want_v=False):
        """Adjoint of ``collision``: (rho_bar, T_bar[, v_bar]) for
        I_bar = dL/dRe I + i dL/dIm I (v_bar: FP64 contexts, host arrays)."""
        Lh = int(rho_hist.shape[0])
        if _is_torch(rho_hist):
            import torch
            r, rp = _dev(rho_hist, "c16"); t, tp = _dev(T_hist, "c16")
            ib, ibp = _dev(I_bar, "c16")
            wp = None
            if weights is not None:
                w, wp = _dev(weights, "f64")
            rb = torch.empty_like(r)
            tb = torch.empty_like(t)
            self._check(load().gkba_collision_vjp(self._h, Lh, rp, tp, wp, ibp, rb.data_ptr(),
                                                  tb.data_ptr(), None, 1))
            return rb, tb
        r, rp = _host(rho_hist, np.complex128); t, tp = _host(T_hist, np.complex128)
        ib, ibp = _host(I_bar, np.complex128)
        wp = None
        if weights is not None:
            w, wp = _host(weights, np.float64)
        rb = np.empty_like(r)
        tb = np.empty_like(t)
        vb = np.empty((self.N,) * 4, np.float64) if want_v else None
        self._check(load().gkba_collision_vjp(self._h, Lh, rp, tp, wp, ibp, rb.ctypes.data,
                                              tb.ctypes.data, vb.ctypes.data if want_v else None, 0))
        return (rb, tb, vb) if want_v else (rb, tb)

    def step(self, E_n, E_np1):
        """One Heun step; returns (rho_{n+1}, I(t_n), diag(t_n))."""
        rho = np.empty((self.N, self.N), np.complex128)
        I = np.empty((self.N, self.N), np.complex128)
        diag = np.empty(4, np.float64)
        self._check(load().gkba_step(self._h, float(E_n), float(E_np1), rho.ctypes.data,
                                     I.ctypes.data, diag.ctypes.data))
        return rho, I, diag

    def mean_field(self, rho):
        r, rp = _host(rho, np.complex128)
        out = np.empty_like(r)
        self._check(load().gkba_mean_field(self._h, rp, out.ctypes.data, 0))
        return out

    def set_history(self, n, rho_hist, T_hist):
        if _is_torch(rho_hist):
            r, rp = _dev(rho_hist, "c16"); t, tp = _dev(T_hist, "c16")
            self._check(load().gkba_set_history(self._h, int(n), rp, tp, 1))
        else:
            r, rp = _host(rho_hist, np.complex128); t, tp = _host(T_hist, np.complex128)
            self._check(load().gkba_set_history(self._h, int(n), rp, tp, 0))

    def get_history(self):
        n = ctypes.c_int()
        self._check(load().gkba_get_history(self._h, ctypes.byref(n), None, None))
        rho = np.empty((n.value + 1, self.N, self.N), np.complex128)
        T = np.empty_like(rho)
        self._check(load().gkba_get_history(self._h, ctypes.byref(n), rho.ctypes.data, T.ctypes.data))
        return n.value, rho, T

    def get_state(self):
        n = ctypes.c_int()
        rho = np.empty((self.N, self.N), np.complex128)
        self._check(load().gkba_get_state(self._h, ctypes.byref(n), rho.ctypes.data))
        return n.value, rho

    def stats(self, reset=False):
        arr = (KernelStat * 16)()
        n = ctypes.c_int()
        tot = ctypes.c_longlong()
        self._check(load().gkba_get_stats(self._h, arr, 16, ctypes.byref(n), ctypes.byref(tot),
                                          1 if reset else 0))
        out = {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms,
                                          flops=arr[i].flops, bytes=arr[i].bytes)
               for i in range(n.value)}
        return out, tot.value

    def selftest_timeout(self, limit_ms=50.0):
        """Run the bounded-wait self-test; returns (status, elapsed_ms of both CTAs)."""
        el = np.zeros(2, np.float64)
        st = load().gkba_selftest_timeout(self._h, float(limit_ms), el.ctypes.data)
        return st, el

    def measure_tf32_mma(self, iters=100000):
        """Tensor-pipe rate (TFLOP/s) of back-to-back kind::tf32 MMAs of the
        stage kernels' shape on every SM pair (gkba_measure_tf32_mma)."""
        out = np.zeros(1, np.float64)
        self._check(load().gkba_measure_tf32_mma(self._h, int(iters), out.ctypes.data))
        return float(out[0])

    def adjoint(self, rho_bar_final, want_v=False):
        """Gradients of L(rho(t_n)) w.r.t. the field samples E(t_0 .. t_n),
        rho(t_0) [and v] through the steps taken since
        gkba_init; rho_bar_final = dL/dRe rho(t_n) + i dL/dIm rho(t_n).
        Returns (E_bar, rho0_bar[, v_bar])."""
        rb, rbp = _host(rho_bar_final, np.complex128)
        n = ctypes.c_int()
        self._check(load().gkba_get_state(self._h, ctypes.byref(n), None))
        E_bar = np.zeros(n.value + 1, np.float64)
        r0 = np.empty((self.N, self.N), np.complex128)
        vb = np.empty((self.N,) * 4, np.float64) if want_v else None
        self._check(load().gkba_adjoint(self._h, rbp, E_bar.ctypes.data, r0.ctypes.data,
                                        vb.ctypes.data if want_v else None))
        return (E_bar, r0, vb) if want_v else (E_bar, r0)


class Batch:
    """Several Contexts (split-TF32, general interaction) advanced together:
    the history contractions of all systems share each stage launch, split
    by basis-size group (gkba_batch_*).  The contexts stay usable on their own
    afterwards."""

    def __init__(self, contexts, workspace_bytes=0):
        L = load()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        handle = ctypes.c_void_p()
        st = L.gkba_batch_create(ctypes.byref(handle), ctypes.cast(arr, ctypes.c_void_p),
                                 len(self.contexts), int(workspace_bytes))
        if st != OK:
            raise GKBAError(st, L.gkba_batch_last_error(None).decode())
        self._h = handle

    def step(self, E_n, E_np1):
        """One Heun step of every member; returns (list of rho, list of diagnostics)."""
        n = len(self.contexts)
        En = np.ascontiguousarray(np.broadcast_to(np.asarray(E_n, np.float64), (n,)))
        Enp = np.ascontiguousarray(np.broadcast_to(np.asarray(E_np1, np.float64), (n,)))
        rhos = [np.empty((c.N, c.N), np.complex128) for c in self.contexts]
        diags = [np.empty(4, np.float64) for _ in self.contexts]
        rp = (ctypes.c_void_p * n)(*[r.ctypes.data for r in rhos])
        dp = (ctypes.c_void_p * n)(*[d.ctypes.data for d in diags])
        L = load()
        st = L.gkba_batch_step(self._h, En.ctypes.data, Enp.ctypes.data,
                               ctypes.cast(rp, ctypes.c_void_p), ctypes.cast(dp, ctypes.c_void_p))
        if st != OK:
            raise GKBAError(st, L.gkba_batch_last_error(self._h).decode())
        return rhos, diags

    def set_options(self, use_graph=False):
        """use_graph: capture each step's device work and launch it as one CUDA graph."""
        L = load()
        st = L.gkba_batch_set_options(self._h, 1 if use_graph else 0)
        if st != OK:
            raise GKBAError(st, L.gkba_batch_last_error(self._h).decode())

    def autotune(self):
        """Choose the launch parameters per basis-size group by timing them on
        the device (gkba_batch_autotune); returns one dict per group."""
        L = load()
        n = ctypes.c_int()
        Ns, units, aw, kw = (np.zeros(8, np.int32) for _ in range(4))
        us = np.zeros(8, np.float64)
        st = L.gkba_batch_autotune(self._h, ctypes.byref(n), Ns.ctypes.data, units.ctypes.data,
                                   aw.ctypes.data, kw.ctypes.data, us.ctypes.data)
        if st != OK:
            raise GKBAError(st, L.gkba_batch_last_error(self._h).decode())
        return [dict(N=int(Ns[g]), units_per_round=int(units[g]), acc_window=int(aw[g]),
                     s4_item_k=int(kw[g]), us_per_unit=float(us[g])) for g in range(min(n.value, 8))]

    def close(self):
        if getattr(self, "_h", None):
            load().gkba_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def collision_autograd(ctx, rho_hist, T_hist, weights=None):
    """I = ctx.collision(rho_hist, T_hist) as a differentiable torch op on CUDA
    complex128 tensors: the backward pass is gkba_collision_vjp (PyTorch's
    complex gradient convention, dL/dRe + i dL/dIm, is the library's)."""
    import torch

    class _Collision(torch.autograd.Function):
        @staticmethod
        def forward(fctx, rho, T):
            fctx.save_for_backward(rho, T)
            return ctx.collision(rho, T, weights)

        @staticmethod
        def backward(fctx, I_bar):
            rho, T = fctx.saved_tensors
            rb, tb = ctx.collision_vjp(rho, T, I_bar.contiguous(), weights)
            return rb, tb

    return _Collision.apply(rho_hist, T_hist)


def dipole_autograd(make_context, E, d=None):
    """L = Re Tr[d rho(t_n)] after len(E) - 1 Heun steps of a fresh context
    (``make_context()`` returns a Context at step 0; d defaults to the dipole
    the context was built with, passed explicitly here) as a torch op of the
    field samples E (float64 tensor): the backward pass is gkba_adjoint."""
    import torch

    class _Dipole(torch.autograd.Function):
        @staticmethod
        def forward(fctx, Ev):
            e = Ev.detach().cpu().numpy().astype(np.float64)
            ctx = make_context()
            rho = None
            for k in range(len(e) - 1):
                rho, _, _ = ctx.step(e[k], e[k + 1])
            fctx.gkba = ctx
            return torch.tensor(float(np.real(np.trace(d @ rho))), dtype=torch.float64,
                                device=Ev.device)

        @staticmethod
        def backward(fctx, gL):
            ctx = fctx.gkba
            E_bar, _ = ctx.adjoint(np.asarray(d, np.complex128).conj().T)
            ctx.close()
            return gL * torch.as_tensor(E_bar, dtype=torch.float64, device=gL.device)

    if d is None:
        raise ValueError("pass the dipole matrix d of the loss")
    return _Dipole.apply(E)


def coulomb_factor_grad(B, v_bar):
    """dL/dB^P for Coulomb integrals built from factors, v_ijkl = sum_P
    B^P_il B^P_jk (B real, shape (n_P, N, N)), given dL/dv (every entry of v
    an independent variable, as gkba_adjoint / gkba_collision_vjp return it):
    dL/dB^P_ab = sum_jk vbar_ajkb B^P_jk + sum_il vbar_iabl B^P_il."""
    B = np.asarray(B, np.float64)
    vb = np.asarray(v_bar, np.float64)
    return (np.einsum("ajkb,pjk->pab", vb, B, optimize=True)
            + np.einsum("iabl,pil->pab", vb, B, optimize=True))
