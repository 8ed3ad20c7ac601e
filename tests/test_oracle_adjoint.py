"""Pins of the oracle's collision-integral adjoint (``collision_vjp``) and of
the trilinear form ``sigma3``: finite differences of ``collision``, the
reduction S3(G, Gb, G) = S(G, Gb), and the slot identities that express each
derivative of Eq. (2bse) as another S3 evaluation."""
import numpy as np
import pytest

import gkba_inputs as gi
import oracle as O


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def cplx(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def test_sigma3_reduces_to_sigma_and_matches_bruteforce():
    N = 4
    v = gi.random_symmetric_v(N, seed=1)
    rng = np.random.default_rng(2)
    A, B, C = cplx(rng, N, N), cplx(rng, N, N), cplx(rng, N, N)
    w = O.exchange_folded(v)
    brute = np.einsum("irpn,mqsj,nm,sr,pq->ij", v, w, A, B, C, optimize=False)
    assert rel(O.sigma3(v, A, B, C), brute) < 1e-13
    assert rel(O.sigma3(v, A, B, A), O.sigma_bruteforce(v, A, B)) < 1e-13
    # the two G slots differ when A != C (a transposed slot would not be caught otherwise)
    assert rel(O.sigma3(v, A, B, C), O.sigma3(v, C, B, A)) > 1e-3


@pytest.mark.parametrize("which", ["rho", "T"])
def test_collision_vjp_matches_finite_differences(which):
    # L(rho, T) = Re sum conj(Ibar) I(rho, T); dL along a random complex
    # direction by central differences against Re sum conj(xbar) dx
    N, L = 4, 3
    v = gi.random_symmetric_v(N, seed=3)
    rng = np.random.default_rng(4)
    rho = cplx(rng, L, N, N) * 0.3
    T = cplx(rng, L, N, N) * 0.3
    w = np.array([0.01, 0.02, 0.01])
    Ibar = cplx(rng, N, N)
    rho_bar, T_bar = O.collision_vjp(v, rho, T, w, Ibar)
    d = cplx(rng, L, N, N)

    def loss(eps):
        r, t = (rho + eps * d, T) if which == "rho" else (rho, T + eps * d)
        return np.real(np.sum(np.conj(Ibar) * O.collision(v, r, t, w)))

    eps = 1e-5
    fd = (loss(eps) - loss(-eps)) / (2 * eps)
    xbar = rho_bar if which == "rho" else T_bar
    ad = np.real(np.sum(np.conj(xbar) * d))
    assert abs(fd - ad) < 1e-7 * max(abs(fd), 1.0), (fd, ad)


def test_collision_vjp_catches_planted_mistakes():
    # the FD pin above rejects a dropped slot, a missing conjugate or a sign
    N, L = 3, 2
    v = gi.random_symmetric_v(N, seed=5)
    rng = np.random.default_rng(6)
    rho, T = cplx(rng, L, N, N) * 0.3, cplx(rng, L, N, N) * 0.3
    w = np.array([0.02, 0.02])
    Ibar = cplx(rng, N, N)
    rb, Tb = O.collision_vjp(v, rho, T, w, Ibar)
    d = cplx(rng, L, N, N)
    eps = 1e-5
    f = lambda e: np.real(np.sum(np.conj(Ibar) * O.collision(v, rho + e * d, T, w)))
    fd = (f(eps) - f(-eps)) / (2 * eps)
    good = np.real(np.sum(np.conj(rb) * d))
    assert abs(fd - good) < 1e-7 * abs(fd)
    for bad in (rb.conj(), -rb, 0.5 * rb):
        assert abs(fd - np.real(np.sum(np.conj(bad) * d))) > 1e-3 * abs(fd)


def test_slot_derivatives_are_sigma3_evaluations():
    # The identities the CUDA path uses (w_abcd = w_badc = w_dcba = w_cdab for
    # 8-fold symmetric v): with Sbar the adjoint of S(G, Gb),
    #   dL/dGb* = S3(G*, Sbar^T, G*)^T
    #   dL/dG*  = S3(Sbar, G*^T, Gb*^T) + S3(Gb*^T, G*^T, Sbar)
    N = 4
    v = gi.random_symmetric_v(N, seed=7)
    w = O.exchange_folded(v)
    rng = np.random.default_rng(8)
    G, Gb, Sbar = cplx(rng, N, N), cplx(rng, N, N), cplx(rng, N, N)
    Gc, Gbc = G.conj(), Gb.conj()
    gb_direct = np.einsum("irpn,mqsj,nm,pq,ij->sr", v, w, Gc, Gc, Sbar, optimize=True)
    g_direct = (np.einsum("irpn,mqsj,sr,pq,ij->nm", v, w, Gbc, Gc, Sbar, optimize=True)
                + np.einsum("irpn,mqsj,nm,sr,ij->pq", v, w, Gc, Gbc, Sbar, optimize=True))
    assert rel(O.sigma3(v, Gc, Sbar.T, Gc).T, gb_direct) < 1e-13
    assert rel(O.sigma3(v, Sbar, Gc.T, Gbc.T) + O.sigma3(v, Gbc.T, Gc.T, Sbar), g_direct) < 1e-13


def symmetrize8(x):
    """Average over the 8-fold permutation group of Eq. (symmetries)."""
    perms = [(0, 1, 2, 3), (1, 0, 3, 2), (3, 2, 1, 0), (2, 3, 0, 1),
             (3, 1, 2, 0), (1, 3, 0, 2), (0, 2, 1, 3), (2, 0, 3, 1)]
    return sum(x.transpose(p) for p in perms) / 8.0


def test_collision_vjp_v_matches_finite_differences():
    # L(v) = Re sum conj(Ibar) I(v) along an 8-fold symmetric direction
    N, L = 4, 3
    v = gi.random_symmetric_v(N, seed=11)
    rng = np.random.default_rng(12)
    rho, T = cplx(rng, L, N, N) * 0.3, cplx(rng, L, N, N) * 0.3
    w = np.array([0.01, 0.02, 0.01])
    Ibar = cplx(rng, N, N)
    dv = symmetrize8(rng.normal(size=(N,) * 4))
    assert np.allclose(dv, dv.transpose(1, 0, 3, 2)) and np.allclose(dv, dv.transpose(3, 2, 1, 0))
    vbar = O.collision_vjp_v(v, rho, T, w, Ibar)
    f = lambda e: np.real(np.sum(np.conj(Ibar) * O.collision(v + e * dv, rho, T, w)))
    eps = 1e-5
    fd = (f(eps) - f(-eps)) / (2 * eps)
    ad = float(np.sum(vbar * dv))
    assert abs(fd - ad) < 1e-7 * max(abs(fd), 1.0), (fd, ad)
    # planted mistake: the v slot alone (the w = 2v - v_exch slot dropped)
    wf = O.exchange_folded(v)
    vslot = np.zeros((N,) * 4)
    for k in range(L):
        P = T[k] @ rho[k]
        Q = T[k] - P
        for G, Gb, coef in ((P, Q.conj().T, -w[k]), (Q, P.conj().T, w[k])):
            Sc = ((coef * Ibar) @ Gb.conj().T).conj()
            vslot += np.real(np.einsum("ij,mqsj,nm,sr,pq->irpn", Sc, wf, G, Gb, G, optimize=True))
    assert abs(float(np.sum(vslot * dv)) - fd) > 1e-3 * abs(fd)
