"""Pins for the oracle's GKBA reconstruction, collision integral, mean field and
time stepper (Sec. II of arXiv:1905.01180).

The paper prints no trajectory values, so the stepper is pinned by conservation
laws of Eq. (equalt), by the non-interacting closed form, and by the second
order of the Heun scheme.
"""
import numpy as np
import pytest
import scipy.linalg

import gkba_inputs as gi
import oracle as O


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_gkba_equal_time_and_adjoint_relations():
    # At t_k = t (T = 1): G^>(t,t) - G^<(t,t) = -i (Sec. II) and rho = -i G^<(t,t).
    N = 5
    rho, T = gi.history(N, 3, 0.05, seed=1)
    Gl, Gg, Glk, Ggk = O.gkba_greens(T[-1:], rho[-1:])
    assert np.abs(Gg[0] - Gl[0] + 1j * np.eye(N)).max() < 1e-14
    assert np.abs(-1j * Gl[0] - rho[-1]).max() < 1e-14
    # G^{<>}(t_k, t) = -[G^{<>}(t, t_k)]^dag
    Gl, Gg, Glk, Ggk = O.gkba_greens(T, rho)
    assert np.abs(Glk + np.conj(np.swapaxes(Gl, 1, 2))).max() < 1e-14
    assert np.abs(Ggk + np.conj(np.swapaxes(Gg, 1, 2))).max() < 1e-14


def test_history_propagators_are_unitary():
    rho, T = gi.history(6, 5, 0.05, seed=2)
    for k in range(5):
        assert np.abs(T[k] @ T[k].conj().T - np.eye(6)).max() < 1e-13
        assert np.abs(rho[k] - rho[k].conj().T).max() < 1e-14
        ev = np.linalg.eigvalsh(rho[k])
        assert ev.min() > -1e-12 and ev.max() < 1 + 1e-12


def test_self_energy_time_reversal():
    # Sigma^<(t_k, t) = -Sigma^<(t, t_k)^dag, with Sigma^<(t_k,t) =
    # S(G^<(t_k,t), G^>(t,t_k)).
    N = 4
    v = gi.random_symmetric_v(N, seed=3)
    rho, T = gi.history(N, 2, 0.1, seed=4)
    Gl, Gg, Glk, Ggk = O.gkba_greens(T, rho)
    fwd = O.sigma_independent(v, Gl, Ggk)
    bwd = O.sigma_independent(v, Glk, Gg)
    assert rel(bwd, -np.conj(np.swapaxes(fwd, 1, 2))) < 1e-12


def test_collision_phase_free_form():
    # With P = T rho, Q = T - P the phases in Eq. (collint) cancel:
    # I = sum_k c_k [S(Q, P^dag) P^dag - S(P, Q^dag) Q^dag].
    N, L = 4, 5
    v = gi.random_symmetric_v(N, seed=5)
    rho, T = gi.history(N, L, 0.05, seed=6)
    c = np.linspace(0.3, 1.1, L)
    I = O.collision(v, rho, T, c)
    P = T @ rho
    Q = T - P
    Pd = np.conj(np.swapaxes(P, 1, 2))
    Qd = np.conj(np.swapaxes(Q, 1, 2))
    want = sum(c[k] * (O.sigma_bruteforce(v, Q[k], Pd[k]) @ Pd[k]
                       - O.sigma_bruteforce(v, P[k], Qd[k]) @ Qd[k]) for k in range(L))
    assert rel(I, want) < 1e-12
    # the three contraction routes give the same I
    assert rel(O.collision(v, rho, T, c, route="paper"), I) < 1e-12
    assert rel(O.collision(v, rho, T, c, route="bruteforce"), I) < 1e-12


def test_collision_particle_conservation_and_linearity():
    N, L = 5, 6
    v = gi.random_symmetric_v(N, seed=7)
    rho, T = gi.history(N, L, 0.05, seed=8)
    w = O.trapezoid_weights(L, 0.05)
    I = O.collision(v, rho, T, w)
    # Tr[I + I^dag] = 0: particle number is conserved by Eq. (equalt)
    assert abs(np.trace(I).real) < 1e-13 * np.abs(I).max() * N
    assert np.abs(I).max() > 1e-6
    # v = 0 => I = 0
    assert np.abs(O.collision(0 * v, rho, T, w)).max() == 0.0
    # linear in the weights: unit weights pick single history points
    parts = [O.collision(v, rho, T, np.eye(L)[k]) for k in range(L)]
    assert rel(sum(w[k] * parts[k] for k in range(L)), I) < 1e-13


def test_trapezoid_weights():
    dt = 0.05
    for L in (2, 3, 10):
        w = O.trapezoid_weights(L, dt)
        t = dt * np.arange(L)
        assert abs(w.sum() - dt * (L - 1)) < 1e-15
        assert abs((w * (3 * t + 1)).sum() - (1.5 * t[-1] ** 2 + t[-1])) < 1e-13
    assert O.trapezoid_weights(1, dt).tolist() == [0.0]


def test_hf_self_energy_closed_forms():
    # Hubbard v: Sigma_HF = diag(U_i rho_ii); density-density v_ijkl =
    # V_ij d_il d_jk: Sigma_HF = 2 diag(V diag(rho)) - V o rho (Hartree + Fock).
    N = 5
    rho, _ = gi.history(N, 1, 0.1, seed=9)
    rho = rho[0]
    U = np.array([1.0, 0.5, 2.0, 0.3, 1.1])
    vh = np.zeros((N,) * 4)
    for i in range(N):
        vh[i, i, i, i] = U[i]
    assert np.abs(O.hf_self_energy(vh, rho) - np.diag(U * np.diag(rho))).max() < 1e-15
    idx = np.arange(N)
    V = 1.0 / np.sqrt(1.0 + (idx[:, None] - idx[None, :]) ** 2)
    vo = np.zeros((N,) * 4)
    for i in range(N):
        for j in range(N):
            vo[i, j, j, i] = V[i, j]
    want = 2 * np.diag(V @ np.diag(rho)) - V * rho
    assert np.abs(O.hf_self_energy(vo, rho) - want).max() < 1e-14


def test_expm_hermitian():
    rng = np.random.default_rng(10)
    A = rng.normal(size=(7, 7)) + 1j * rng.normal(size=(7, 7))
    H = A + A.conj().T
    assert np.abs(O.expm_hermitian(H, 0.07) - scipy.linalg.expm(-0.07j * H)).max() < 1e-13


def test_free_propagation_closed_form():
    # v = 0, E = 0: rho(t) = e^{-iht} rho0 e^{iht} exactly (the Heun step with
    # the averaged propagator is exact when h_HF does not depend on rho).
    s = gi.system(6, 4, seed=0)
    dt, n = 0.05, 40
    p = O.propagate(s["h"], 0 * s["v"], s["d"], s["rho0"], dt, n, np.zeros(n + 1))
    for k in (1, 17, 40):
        U = scipy.linalg.expm(-1j * s["h"] * dt * k)
        assert np.abs(p.rho[k] - U @ s["rho0"] @ U.conj().T).max() < 1e-12
    assert np.abs(p.I).max() == 0.0


@pytest.fixture(scope="module")
def config0():
    s = gi.system(4, 8, seed=0)
    dt, n = 0.05, 200
    E = gi.field(dt * np.arange(n + 1))
    return s, O.propagate(s["h"], s["v"], s["d"], s["rho0"], dt, n, E)


def test_config0_invariants(config0):
    s, p = config0
    tr = np.trace(p.rho, axis1=1, axis2=2)
    assert np.abs(tr - tr[0]).max() < 1e-12
    assert abs(tr[0] - s["n_occ"]) < 1e-12
    assert np.abs(p.rho - np.conj(np.swapaxes(p.rho, 1, 2))).max() < 1e-13
    assert np.abs(np.trace(p.I, axis1=1, axis2=2).real).max() < 1e-12
    # the quench from the non-interacting ground state lowers the correlation
    # energy below zero (MP2-like, Sec. III)
    assert p.energy_corr[-1] < 0.0


def test_energy_conservation_second_order():
    # Field-free: E = Tr[h rho] + 1/2 Tr[Sigma_HF rho] + 1/2 Im Tr I is
    # conserved up to the Heun step error, which is O(dt^2).
    s = gi.system(4, 8, seed=0)
    drifts = []
    for dt in (0.1, 0.05):
        n = int(round(6.0 / dt))
        p = O.propagate(s["h"], s["v"], s["d"], s["rho0"], dt, n, np.zeros(n + 1))
        drifts.append(np.abs(p.energy_total - p.energy_total[0]).max())
    ratio = drifts[0] / drifts[1]
    assert 3.5 < ratio < 4.5, drifts
    assert drifts[1] < 1e-3


def test_flipped_sigma_sign_breaks_energy_conservation(monkeypatch):
    # Planted mistake (Sigma -> -Sigma, i.e. an extra i^2): the energy is no
    # longer conserved, which is how the sign of Eq. (2bse) is pinned.
    s = gi.system(4, 8, seed=0)
    dt, n = 0.1, 60
    good = O.propagate(s["h"], s["v"], s["d"], s["rho0"], dt, n, np.zeros(n + 1))
    # the propagation's default route is the paper's Eq. (2b-opt)
    orig = O.sigma_paper
    monkeypatch.setattr(O, "sigma_paper", lambda v, G, Gb: -orig(v, G, Gb))
    with np.errstate(all="ignore"):
        try:
            bad = O.propagate(s["h"], s["v"], s["d"], s["rho0"], dt, n, np.zeros(n + 1))
            d_bad = np.abs(bad.energy_total - bad.energy_total[0]).max()
        except np.linalg.LinAlgError:
            d_bad = np.inf  # the run diverged to non-finite values
    d_good = np.abs(good.energy_total - good.energy_total[0]).max()
    assert not (d_bad <= 20 * d_good)
