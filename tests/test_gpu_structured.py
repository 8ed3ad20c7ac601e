"""GPU parity of the diagonal- and symmetric-basis paths (Sec. III A, B).

The library evaluates the self-energy of these interactions with dedicated
FP64 kernels (Eq. 2b-diag, Eq. 2b-symm) instead of the N^5 contraction chain.
They are checked against the oracle's closed forms (pinned against the
brute-force Eq. (2bse) in tests/test_oracle_sigma.py), against the oracle's
general route on the expanded v_ijkl, and against the library's own general
FP64 path on the same expanded v.  Tolerance 1e-12 / 1e-10 (FP64 throughout).
"""
import time

import numpy as np
import pytest

import gkba_inputs as gi
import oracle as O
from _check import check, rel

pytestmark = pytest.mark.gpu




@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_01180_gb300 import build as b
    b.build()
    import paper_1905_01180_gb300 as p
    return p


def expand(kind, v):
    """v_ijkl of Sec. III A (v_iiii = U_i) or Sec. III B (v_ijji = V_ij)."""
    N = v.shape[0]
    full = np.zeros((N,) * 4)
    for i in range(N):
        if kind == "diagonal":
            full[i, i, i, i] = v[i]
        else:
            for j in range(N):
                full[i, j, j, i] = v[i, j]
    return full


def closed_form(kind, v, G, Gb):
    return O.sigma_hubbard(v, G, Gb) if kind == "diagonal" else O.sigma_symmetric(v, G, Gb)


@pytest.mark.parametrize("kind", ["diagonal", "symmetric"])
@pytest.mark.parametrize("N", [1, 4, 10, 13, 33])
def test_structured_sigma_vs_closed_forms(P, kind, N):
    c = gi.chain(N, kind, U=0.8)
    pairs = [gi.random_pair(N, seed=10 + u) for u in range(3)]
    G = np.array([p[0] for p in pairs])
    Gb = np.array([p[1] for p in pairs])
    ctx = P.Context(c["h"], c["v"], c["d"], c["rho0"], 0.05, interaction=kind)
    S = ctx.sigma(G, Gb)
    ctx.close()
    for u in range(3):
        check(S[u], closed_form(kind, c["v"], G[u], Gb[u]), 1e-12)


@pytest.mark.parametrize("kind", ["diagonal", "symmetric"])
def test_structured_collision_vs_oracle(P, kind):
    # the collision integral (Eq. collint) over a synthetic history, against
    # the oracle's general route on the expanded v_ijkl
    N, L, dt = 10, 6, 0.025
    c = gi.chain(N, kind)
    rho, T = gi.history(N, L, dt, seed=3)
    ctx = P.Context(c["h"], c["v"], c["d"], c["rho0"], dt, interaction=kind)
    I = ctx.collision(rho, T)
    ctx.close()
    ref = O.collision(expand(kind, c["v"]), rho, T, O.trapezoid_weights(L, dt), route="paper")
    e = check(I, ref, 1e-12, f"{kind} collision")
    print(f"{kind} N={N} L={L} collision rel err {e:.3e}")


@pytest.mark.parametrize("kind,dt", [("diagonal", 0.01), ("symmetric", 0.025)])
def test_structured_propagation_vs_oracle(P, kind, dt):
    # 20 Heun steps of the chain workload from the confined state (field-free)
    N, n = 10, 20
    c = gi.chain(N, kind)
    E = np.zeros(n + 1)
    ref = O.propagate(c["h"], expand(kind, c["v"]), c["d"], c["rho0"], dt, n, E, route="paper")
    ctx = P.Context(c["h"], c["v"], c["d"], c["rho0"], dt, max_steps=n, interaction=kind)
    worst = 0.0
    for k in range(n):
        rho, I, diag = ctx.step(0.0, 0.0)
        worst = max(worst, check(rho, ref.rho[k + 1], 1e-10, f"rho step {k + 1}"))
        assert abs(diag[1] - ref.energy_total[k]) < 1e-10
    ctx.close()
    print(f"{kind} chain, {n} steps: max rel err of rho vs oracle {worst:.3e}")
    assert worst < 1e-10


@pytest.mark.parametrize("kind,dt", [("diagonal", 0.01), ("symmetric", 0.025)])
def test_structured_matches_general_path(P, kind, dt):
    # the same model through the N^5 contraction chain (FP64) on the expanded v
    N, n = 10, 200
    c = gi.chain(N, kind)
    a = P.Context(c["h"], c["v"], c["d"], c["rho0"], dt, max_steps=n, interaction=kind)
    b = P.Context(c["h"], expand(kind, c["v"]), c["d"], c["rho0"], dt, max_steps=n)
    worst = 0.0
    for _ in range(n):
        ra, _, _ = a.step(0.0, 0.0)
        rb, _, _ = b.step(0.0, 0.0)
        worst = max(worst, rel(ra, rb))
    a.close()
    b.close()
    print(f"{kind} chain, {n} steps: structured vs general FP64 path {worst:.3e}")
    assert worst < 1e-11


@pytest.mark.slow
@pytest.mark.parametrize("kind,dt,n", [("diagonal", 0.01, 5000), ("symmetric", 0.025, 2000)])
def test_paper_chain_workloads(P, kind, dt, n):
    # Sec. IV cases (1) and (2): N_b = 10 chain, N_t steps of length delta,
    # released from the confined state.  Particle number is conserved, rho
    # stays Hermitian, and without a field the energy is conserved up to the
    # O(dt^2) Heun error.
    N = 10
    c = gi.chain(N, kind)
    ctx = P.Context(c["h"], c["v"], c["d"], c["rho0"], dt, max_steps=n, interaction=kind)
    t0 = time.perf_counter()
    tr, en = [], []
    for _ in range(n):
        rho, I, diag = ctx.step(0.0, 0.0)
        tr.append(diag[0])
        en.append(diag[1])
    wall = time.perf_counter() - t0
    ctx.close()
    tr, en = np.array(tr), np.array(en)
    drift = np.abs(en - en[0]).max()
    print(f"{kind} chain N={N}, {n} steps of {dt}: {wall:.2f} s, |Tr rho - {N // 2}| "
          f"{np.abs(tr - N // 2).max():.2e}, energy drift {drift:.2e} (E = {en[0]:.4f})")
    assert np.abs(tr - N // 2).max() < 1e-9
    assert np.abs(rho - rho.conj().T).max() < 1e-12
    assert drift < 1e-3 * abs(en[0])
