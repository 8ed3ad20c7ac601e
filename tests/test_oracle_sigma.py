"""Pins for the oracle's second-Born self-energy (Sec. III of arXiv:1905.01180).

Each check compares the oracle with something other than itself: a closed form
the paper derives (Eqs. 2b-diag, 2b-symm, bubble-contract, x-contract), the
literal N^8 definition (Eq. 2bse), scaling laws of the cubic form, and the
adjoint symmetry of real, symmetric interactions.  ``test_pins_catch_mistakes``
plants plausible errors in a copy of the formula and shows a pin fails.
"""
import numpy as np
import pytest

import gkba_inputs as gi
import oracle as O


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_loops_match_bruteforce(N):
    v = gi.random_symmetric_v(N, seed=10 + N)
    G, Gb = gi.random_pair(N, seed=20 + N)
    assert rel(O.sigma_loops(v, G, Gb), O.sigma_bruteforce(v, G, Gb)) < 1e-13


def test_single_orbital_closed_form():
    # N = 1: Sigma = 2 v^2 G Gb G - v^2 G Gb G = v^2 G^2 Gb  (Eq. 2bse)
    v = np.full((1, 1, 1, 1), 0.7)
    G = np.array([[0.3 - 1.1j]])
    Gb = np.array([[-0.8 + 0.25j]])
    want = 0.49 * G[0, 0] ** 2 * Gb[0, 0]
    for fn in (O.sigma_loops, O.sigma_bruteforce, O.sigma_paper, O.sigma_independent):
        assert abs(fn(v, G, Gb)[0, 0] - want) < 1e-15


@pytest.mark.parametrize("N", [4, 5])
def test_three_routes_agree(N):
    v = gi.random_symmetric_v(N, seed=N)
    G, Gb = gi.random_pair(N, seed=100 + N)
    a = O.sigma_bruteforce(v, G, Gb)
    assert rel(O.sigma_paper(v, G, Gb), a) < 1e-12
    assert rel(O.sigma_independent(v, G, Gb), a) < 1e-12


def test_independent_route_needs_no_symmetry():
    # For a real v without the permutation symmetry, Eq. (2bse) still defines
    # Sigma; the independent route (w = 2v - v_qmsj) matches it, while the
    # paper's Eq. (2b-opt) re-uses T1 via Eq. (symmetries) and does not.
    N = 4
    rng = np.random.default_rng(7)
    v = rng.normal(size=(N, N, N, N))
    G, Gb = gi.random_pair(N, seed=8)
    a = O.sigma_bruteforce(v, G, Gb)
    assert rel(O.sigma_independent(v, G, Gb), a) < 1e-12
    assert rel(O.sigma_paper(v, G, Gb), a) > 1e-3


def _hubbard_v(U):
    N = len(U)
    v = np.zeros((N,) * 4)
    for i in range(N):
        v[i, i, i, i] = U[i]
    return v


def _ohno_v(V):
    N = V.shape[0]
    v = np.zeros((N,) * 4)
    for i in range(N):
        for j in range(N):
            v[i, j, j, i] = V[i, j]
    return v


def _ohno_V(N, U=1.0):
    idx = np.arange(N)
    return U / np.sqrt(1.0 + (idx[:, None] - idx[None, :]) ** 2)


@pytest.mark.parametrize("route", ["bruteforce", "paper", "independent"])
def test_hubbard_closed_form(route):
    # Eq. (2b-diag): Sigma_ij = U_i U_j G_ij Gb_ji G_ij, and its matrix form
    # Eq. (2b-diag-opt) diag(V) o diag(V) o G o Gb^T o G.
    U = np.array([1.0, 0.4, 2.0, 1.3, 0.7])
    G, Gb = gi.random_pair(5, seed=3)
    fn = {"bruteforce": O.sigma_bruteforce, "paper": O.sigma_paper,
          "independent": O.sigma_independent}[route]
    got = fn(_hubbard_v(U), G, Gb)
    want = np.array([[U[i] * U[j] * G[i, j] * Gb[j, i] * G[i, j] for j in range(5)]
                     for i in range(5)])
    assert rel(got, want) < 1e-13
    assert rel(O.sigma_hubbard(U, G, Gb), want) < 1e-15


@pytest.mark.parametrize("route", ["bruteforce", "paper", "independent"])
def test_ohno_symmetric_closed_form(route):
    # Eq. (2b-symm) for v_ijkl = V_ij delta_il delta_jk with the Ohno V.
    N = 5
    V = _ohno_V(N)
    G, Gb = gi.random_pair(N, seed=4)
    fn = {"bruteforce": O.sigma_bruteforce, "paper": O.sigma_paper,
          "independent": O.sigma_independent}[route]
    got = fn(_ohno_v(V), G, Gb)
    want = np.zeros((N, N), complex)
    for i in range(N):
        for j in range(N):
            for k in range(N):
                for l in range(N):
                    want[i, j] += V[i, k] * V[j, l] * (2 * G[i, j] * Gb[l, k] * G[k, l]
                                                       - G[i, l] * Gb[l, k] * G[k, j])
    assert rel(got, want) < 1e-13
    assert rel(O.sigma_symmetric(V, G, Gb), want) < 1e-13


def test_bubble_one_liner_and_exchange_diagonal():
    # Eq. (bubble-contract) equals the bubble (first) term of Eq. (2b-symm);
    # Eq. (x-contract) equals the diagonal of the exchange (second) term.
    N = 6
    V = _ohno_V(N, U=0.8)
    G, Gb = gi.random_pair(N, seed=5)
    bub = np.zeros((N, N), complex)
    exc = np.zeros((N, N), complex)
    for i in range(N):
        for j in range(N):
            for k in range(N):
                for l in range(N):
                    bub[i, j] += 2 * V[i, k] * V[j, l] * G[i, j] * Gb[l, k] * G[k, l]
                    exc[i, j] -= V[i, k] * V[j, l] * G[i, l] * Gb[l, k] * G[k, j]
    assert rel(O.sigma_bubble(V, G, Gb), bub) < 1e-13
    assert rel(O.sigma_exchange_diag(V, G, Gb), np.diag(exc)) < 1e-13


@pytest.mark.parametrize("fn", [O.sigma_paper, O.sigma_independent])
def test_scaling_laws(fn):
    N = 5
    v = gi.random_symmetric_v(N, seed=11)
    G, Gb = gi.random_pair(N, seed=12)
    S = fn(v, G, Gb)
    assert np.abs(fn(0 * v, G, Gb)).max() == 0.0
    lam = 1.7
    assert rel(fn(lam * v, G, Gb), lam ** 2 * S) < 1e-13
    a, b = 0.3 - 0.8j, -1.2 + 0.4j
    assert rel(fn(v, a * G, b * Gb), a ** 2 * b * S) < 1e-13


@pytest.mark.parametrize("fn", [O.sigma_bruteforce, O.sigma_paper, O.sigma_independent])
def test_adjoint_symmetry(fn):
    # Real, symmetric v: S(G^dag, Gb^dag) = S(G, Gb)^dag, which gives
    # Sigma(t', t) = -Sigma(t, t')^dag for the GKBA Green's functions.
    N = 4
    v = gi.random_symmetric_v(N, seed=13)
    G, Gb = gi.random_pair(N, seed=14)
    assert rel(fn(v, G.conj().T, Gb.conj().T), fn(v, G, Gb).conj().T) < 1e-12


def test_batched_equals_single():
    N = 4
    v = gi.random_symmetric_v(N, seed=15)
    Gs = np.stack([gi.random_pair(N, seed=s)[0] for s in range(3)])
    Gbs = np.stack([gi.random_pair(N, seed=s)[1] for s in range(3)])
    for fn in (O.sigma_paper, O.sigma_independent):
        got = fn(v, Gs, Gbs)
        for b in range(3):
            assert rel(got[b], fn(v, Gs[b], Gbs[b])) < 1e-14


def test_pins_catch_mistakes():
    """Plausible mistakes in Eq. (2bse) each break one of the pins above."""
    N = 4
    U = np.array([1.0, 0.4, 2.0, 1.3])
    V = _ohno_V(N)
    G, Gb = gi.random_pair(N, seed=21)

    def s(v, G, Gb, wd=2.0, wx=1.0, gb_t=False, sign=1.0, vperm="irpn"):
        Gb2 = Gb.T if gb_t else Gb
        d = np.einsum(f"{vperm},mqsj,nm,sr,pq->ij", v, v, G, Gb2, G)
        x = np.einsum(f"{vperm},mqsj,nq,sr,pm->ij", v, v, G, Gb2, G)
        return sign * (wd * d - wx * x)

    hub_want = O.sigma_hubbard(U, G, Gb)
    ohno_want = O.sigma_symmetric(V, G, Gb)
    vh, vo = _hubbard_v(U), _ohno_v(V)
    assert rel(s(vh, G, Gb), hub_want) < 1e-13 and rel(s(vo, G, Gb), ohno_want) < 1e-13
    mistakes = [dict(wx=0.0), dict(sign=-1.0), dict(gb_t=True), dict(wd=1.0),
                dict(vperm="irnp"), dict(vperm="ripn")]
    for mk in mistakes:
        caught = rel(s(vh, G, Gb, **mk), hub_want) > 1e-3 or rel(s(vo, G, Gb, **mk), ohno_want) > 1e-3
        assert caught, mk
