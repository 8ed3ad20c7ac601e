"""Gradients of the Heun propagation by reverse-mode automatic differentiation.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; the product path never
imports it).  The forward below is the stepper of ``oracle.propagate`` written
once more with PyTorch CPU tensors in complex128, so that ``torch.autograd``
gives the exact derivatives of the discrete trajectory:

* Sigma by the paper's N^5 path, Eq. (2b-opt) (as ``oracle.sigma_paper``);
* the GKBA Green's functions of Eqs. (gkba), (prop) (as ``oracle.gkba_greens``);
* the collision integral, first line of Eq. (collint), with trapezoid weights;
* the mean field Sigma_HF of Sec. II and h_HF = h + E(t) d + Sigma_HF;
* Heun's method on Eq. (equalt) with U_n = exp(-i dt (h_HF(t_n, rho_n) +
  h_HF(t_{n+1}, rho~)) / 2) and T(t_{n+1}, t_k) = U_n T(t_n, t_k).

The exponential is ``torch.linalg.matrix_exp`` (whose derivative PyTorch
provides) instead of the eigendecomposition of ``oracle.expm_hermitian``;
the tests pin this forward to ``oracle.propagate`` and its gradients to
central finite differences of ``oracle.propagate``.

Gradient convention: for a real loss and a complex input z the returned
gradient is dL/dRe z + i dL/dIm z (PyTorch's convention).
"""
from __future__ import annotations

import numpy as np
import torch

__all__ = ["propagate_torch", "dipole_gradients"]


def _sigma_paper(v, G, Gb):
    """Eq. (2b-opt) batched over a leading axis (v complex-typed, real values)."""
    T1 = torch.einsum("mqsj,bnm->bnqsj", v, G)
    T2 = torch.einsum("irpn,bsr->bispn", v, Gb)
    T3 = torch.einsum("bpq,bispn->bisqn", G, T2)
    return (2.0 * torch.einsum("bnqsj,bisqn->bij", T1, T3)
            - torch.einsum("bqnjs,bisnq->bij", T1, T3))


def _adj(X):
    return X.conj().transpose(-1, -2)


def _collision(v, rho, T, c):
    """I = sum_k c_k [Sigma^>(t,t_k) G^<(t_k,t) - Sigma^<(t,t_k) G^>(t_k,t)]
    with G^<(t,t_k) = i T rho_k, G^>(t,t_k) = -i T (1 - rho_k) and
    G(t_k, t) = -G(t, t_k)^dag; Sigma^{<>} = S(G^{<>}(t,t_k), G^{><}(t_k,t))."""
    N = rho.shape[-1]
    eye = torch.eye(N, dtype=rho.dtype)
    Gl_tk = 1j * (T @ rho)
    Gg_tk = -1j * (T @ (eye - rho))
    Gl_kt = -_adj(Gl_tk)
    Gg_kt = -_adj(Gg_tk)
    Sl = _sigma_paper(v, Gl_tk, Gg_kt)
    Sg = _sigma_paper(v, Gg_tk, Gl_kt)
    terms = Sg @ Gl_kt - Sl @ Gg_kt
    return torch.einsum("k,kij->ij", c.to(terms.dtype), terms)


def _trapezoid(L, dt):
    w = torch.full((L,), dt, dtype=torch.float64)
    if L == 1:
        return torch.zeros(1, dtype=torch.float64)
    w[0] = w[-1] = 0.5 * dt
    return w


def _hf(v, rho):
    """(Sigma_HF)_ij = sum_kl (2 v_iklj - v_ikjl) rho_lk."""
    return 2.0 * torch.einsum("iklj,lk->ij", v, rho) - torch.einsum("ikjl,lk->ij", v, rho)


def _rhs(h_hf, rho, I):
    """d rho/dt = -i [h_HF, rho] - (I + I^dag), Eq. (equalt) with G^<(t,t) = i rho."""
    return -1j * (h_hf @ rho - rho @ h_hf) - (I + _adj(I))


def propagate_torch(h, v, d, rho0, dt, n_steps, E):
    """Heun propagation from rho(t_0) = rho0 over n_steps with E[n] = E(t_n)
    (n = 0 .. n_steps).  All arguments are torch tensors (h, d, rho0 complex
    N x N; v real or complex N^4; E real).  Returns the list rho(t_0 ..
    t_{n_steps})."""
    N = rho0.shape[0]
    vc = v.to(torch.complex128)
    eye = torch.eye(N, dtype=torch.complex128)
    rhos = [rho0]
    Ts = [eye]  # T(t_n, t_k), k = 0 .. n
    for n in range(n_steps):
        rho_n = rhos[-1]
        hA = h + E[n] * d + _hf(vc, rho_n)
        L = n + 1
        I_n = _collision(vc, torch.stack(rhos), torch.stack(Ts), _trapezoid(L, dt)) if L >= 2 \
            else torch.zeros((N, N), dtype=torch.complex128)
        k1 = _rhs(hA, rho_n, I_n)
        rho_t = rho_n + dt * k1
        hB = h + E[n + 1] * d + _hf(vc, rho_t)
        U = torch.linalg.matrix_exp(-1j * dt * 0.5 * (hA + hB))
        Ts = [U @ T for T in Ts] + [eye]
        I_t = _collision(vc, torch.stack(rhos + [rho_t]), torch.stack(Ts), _trapezoid(L + 1, dt))
        k2 = _rhs(hB, rho_t, I_t)
        rhos.append(rho_n + 0.5 * dt * (k1 + k2))
    return rhos


def dipole_gradients(h, B, d, rho0, dt, n_steps, E):
    """Gradients of the final dipole L = Re Tr[d rho(t_n)] (n = n_steps) for
    Coulomb integrals v_ijkl = sum_P B^P_il B^P_jk (Eq. (coulomb) with real
    factors): returns dict(L, E_bar, rho0_bar, B_bar, v_bar) as numpy arrays,
    E_bar[k] = dL/dE(t_k), B_bar[P] = dL/dB^P (every entry of B^P an
    independent variable), v_bar = dL/dv at fixed B (every entry of v an
    independent variable, through the formulas above), rho0_bar in the
    complex convention of the module docstring."""
    tc = lambda x: torch.tensor(np.asarray(x), dtype=torch.complex128)
    Et = torch.tensor(np.asarray(E, np.float64), requires_grad=True)
    Bt = torch.tensor(np.asarray(B, np.float64), requires_grad=True)
    r0 = tc(rho0).requires_grad_(True)
    v = torch.einsum("pil,pjk->ijkl", Bt, Bt)
    v.retain_grad()
    dt_d = tc(d)
    rhos = propagate_torch(tc(h), v, dt_d, r0, dt, n_steps, Et)
    L = torch.real(torch.trace(dt_d @ rhos[-1]))
    L.backward()
    return dict(L=float(L.detach()), E_bar=Et.grad.numpy().copy(), rho0_bar=r0.grad.numpy().copy(),
                B_bar=Bt.grad.numpy().copy(), v_bar=v.grad.numpy().copy())
