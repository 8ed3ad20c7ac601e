"""Stacked batches of systems (gkba_batch_*): many systems of uneven N and
history length advanced together, the history contractions of all systems of
the same N sharing each kernel launch.

Per unit the arithmetic of a stacked launch is the one of a single-system
launch (the per-system w and v layouts are selected per unit and per 256-row
group; padding units are zero with weight 0), so a batch step must reproduce
the members' own gkba_step to rounding of the history sum's grouping.
"""
import numpy as np
import pytest

import gkba_inputs as gi

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_01180_gb300 import build as b
    b.build()
    import paper_1905_01180_gb300 as p
    return p


def make(P, N, L, seed, steps, precision="tf32"):
    # a system with a synthetic history of L points (the last L points of a
    # longer one are a valid history as well)
    s = gi.system(N, 8, seed=seed)
    rho, T = gi.history(N, L, 0.02, seed=seed)
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.02, max_steps=L + steps,
                    precision=precision)
    ctx.set_history(L - 1, rho, T)
    return ctx


@pytest.mark.parametrize("precision", ["tf32", "tf32acc"])
def test_batch_matches_individual_steps(P, precision):
    # three groups (N = 12 twice, 16, 24) with uneven histories
    spec = [(12, 30, 1), (12, 45, 2), (16, 10, 3), (24, 20, 4)]
    steps = 3
    batched = [make(P, N, L, sd, steps, precision) for N, L, sd in spec]
    alone = [make(P, N, L, sd, steps, precision) for N, L, sd in spec]
    E = [0.01 * k for k in range(steps + 1)]
    with P.Batch(batched) as b:
        for k in range(steps):
            rhos, diags = b.step(E[k], E[k + 1])
            for i, c in enumerate(alone):
                rho, _, diag = c.step(E[k], E[k + 1])
                assert rel(rhos[i], rho) < 1e-12, (k, spec[i])
                assert np.abs(diags[i] - diag).max() < 1e-10, (k, spec[i])
    # the members stay usable on their own
    rho_b, _, _ = batched[0].step(E[-1], E[-1])
    rho_a, _, _ = alone[0].step(E[-1], E[-1])
    assert rel(rho_b, rho_a) < 1e-12
    for c in batched + alone:
        c.close()


def test_batch_of_uneven_sizes(P):
    # one system per basis size of the batched workload (N = 8 ... 48, padded
    # bases 16, 16, 16, 32, 32, 48) and histories of 12 ... 70 points
    spec = [(8, 70, 11), (12, 40, 12), (16, 25, 13), (24, 12, 14), (32, 30, 15), (48, 16, 16)]
    batched = [make(P, N, L, sd, 1) for N, L, sd in spec]
    alone = [make(P, N, L, sd, 1) for N, L, sd in spec]
    with P.Batch(batched) as b:
        rhos, _ = b.step(0.0, 0.0)
    for i, c in enumerate(alone):
        rho, _, _ = c.step(0.0, 0.0)
        e = rel(rhos[i], rho)
        print(f"batch N={spec[i][0]} L={spec[i][1]}: rel diff to own step {e:.2e}")
        assert e < 1e-12
    for c in batched + alone:
        c.close()


def test_batch_rejects_bad_members(P):
    s = gi.system(8, 4, seed=0)
    a = P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.02, max_steps=2, precision="tf32")
    f = P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.02, max_steps=2, precision="fp64")
    with pytest.raises(P.GKBAError) as ei:
        P.Batch([a, f])
    assert ei.value.status == 1
    with pytest.raises(P.GKBAError) as ei:
        P.Batch([a, a])
    assert ei.value.status == 1
    with P.Batch([a]) as b:
        b.step(0.0, 0.0)
        b.step(0.0, 0.0)
        with pytest.raises(P.GKBAError) as ei:
            b.step(0.0, 0.0)  # history full
        assert ei.value.status == 4
    a.close()
    f.close()
