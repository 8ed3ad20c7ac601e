"""Pins of the oracle's time-linear form of the history sum.

The time-linear collision integral rewrites the first line of Eq. (collint)
for propagators of the form T(t_n, t_k) = Ucal_n Ucal_k^dag (Eq. prop as a
product of one-step unitaries), so it must reproduce the history sum of
``oracle.collision`` on any such history; that sum is itself pinned by the
brute-force Eq. (2bse) and the closed forms (test_oracle_sigma.py,
test_oracle_gkba.py).  Random complex unitaries and random densities make a
dropped conjugate, a transposed factor or a wrong sign in any of the three
back-transformed indices fail.
"""
import numpy as np
import pytest

import gkba_inputs as gi
import oracle as O


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def haar(rng, n):
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def unitary_history(N, L, seed):
    rng = np.random.default_rng(seed)
    Uc = np.array([haar(rng, N) for _ in range(L)])
    Un = haar(rng, N)
    T = np.array([Un @ Uc[k].conj().T for k in range(L)])
    return Uc, Un, T


@pytest.mark.parametrize("N,L", [(2, 3), (3, 5), (5, 4), (6, 7)])
def test_collision_time_linear_equals_history_sum(N, L):
    s = gi.system(N, 4, seed=N)
    rho, _ = gi.history(N, L, 0.02, seed=L)
    Uc, Un, T = unitary_history(N, L, seed=10 * N + L)
    w = O.trapezoid_weights(L, 0.02)
    ref = O.collision(s["v"], rho, T, w)
    got = O.collision_time_linear(s["v"], rho, Uc, Un, w)
    assert rel(got, ref) < 1e-12


def test_caller_weights_and_single_points():
    # arbitrary weights (signs included), and each history point alone
    N, L = 4, 5
    s = gi.system(N, 4, seed=2)
    rho, _ = gi.history(N, L, 0.02, seed=3)
    Uc, Un, T = unitary_history(N, L, seed=4)
    w = np.random.default_rng(5).normal(size=L)
    assert rel(O.collision_time_linear(s["v"], rho, Uc, Un, w),
               O.collision(s["v"], rho, T, w)) < 1e-12
    for k in range(L):
        e = np.zeros(L)
        e[k] = 1.0
        assert rel(O.collision_time_linear(s["v"], rho, Uc, Un, e),
                   O.collision(s["v"], rho, T, e)) < 1e-12


def test_identity_propagators_reduce_to_plain_factors():
    # Ucal = 1: X = rho, Xb = 1 - rho, and T = 1 for every point
    N, L = 3, 4
    s = gi.system(N, 4, seed=6)
    rho, _ = gi.history(N, L, 0.05, seed=7)
    eye = np.eye(N, dtype=complex)
    X, Xb = O.time_linear_factors(eye, rho[1])
    assert np.allclose(X, rho[1]) and np.allclose(Xb, eye - rho[1])
    w = O.trapezoid_weights(L, 0.05)
    got = O.collision_time_linear(s["v"], rho, np.array([eye] * L), eye, w)
    assert rel(got, O.collision(s["v"], rho, np.array([eye] * L), w)) < 1e-12


def test_dropped_conjugate_is_caught():
    # the back-transform of the r index needs conj(Ucal); without it the
    # result is O(1) off, so the history-sum pin above would fail
    N, L = 4, 3
    s = gi.system(N, 4, seed=8)
    rho, _ = gi.history(N, L, 0.02, seed=9)
    Uc, Un, T = unitary_history(N, L, seed=11)
    w = O.trapezoid_weights(L, 0.02)
    Lam = sum(w[k] * O.time_linear_term(s["v"], *O.time_linear_factors(Uc[k], rho[k]))
              for k in range(L))
    l1 = np.einsum("na,abcd->nbcd", Un, Lam)
    l2 = np.einsum("pb,nbcd->npcd", Un, l1)
    l3 = np.einsum("rc,npcd->nprd", Un, l2)  # planted: conj dropped
    wrong = np.einsum("irpn,nprd->id", s["v"], l3) @ Un.conj().T
    ref = O.collision(s["v"], rho, T, w)
    assert rel(O.time_linear_apply(s["v"], Lam, Un), ref) < 1e-12
    assert rel(wrong, ref) > 1e-2


@pytest.mark.parametrize("N,n,dt", [(4, 12, 0.05), (6, 8, 0.02)])
def test_time_linear_stepper_equals_history_sum_stepper(N, n, dt):
    s = gi.system(N, 8, seed=N)
    E = np.array([0.1 * np.sin(0.3 * k) for k in range(n + 1)])
    a = O.propagate(s["h"], s["v"], s["d"], s["rho0"], dt, n, E)
    b = O.propagate_time_linear(s["h"], s["v"], s["d"], s["rho0"], dt, n, E)
    for k in range(n + 1):
        assert rel(b.rho[k], a.rho[k]) < 1e-12
        if k > 0:
            assert rel(b.I[k], a.I[k]) < 1e-11
    assert np.abs(b.energy_total - a.energy_total).max() < 1e-12
    assert np.abs(b.I[0]).max() == 0.0


def test_time_linear_stepper_against_config1_golden():
    # the N = 24 propagation (32 factors, dt = 0.02, the pulse) stored by the
    # history-sum oracle (tests/golden/make_config1_oracle.py): the first 20
    # steps of the time-linear stepper reproduce it
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "config1_oracle_100steps.npz"))
    s = gi.system(24, 32, seed=0)
    dt = float(g["dt"])
    E = gi.field(dt * np.arange(1001))
    n = 20
    r = O.propagate_time_linear(s["h"], s["v"], s["d"], s["rho0"], dt, n, E)
    for i, m in enumerate(g["steps"]):
        if m <= n:
            assert rel(r.rho[m], g["rho"][i]) < 1e-12
    assert np.abs(r.energy_total - g["energy_total"][: n + 1]).max() < 1e-12
