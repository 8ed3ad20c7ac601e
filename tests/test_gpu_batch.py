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


def member(N, L, seed):
    # a system with a synthetic history of L points (the last L points of a
    # longer one are a valid history as well)
    s = gi.system(N, 8, seed=seed)
    rho, T = gi.history(N, L, 0.02, seed=seed)
    return s, rho, T


def make(P, N, L, seed, steps, precision="tf32"):
    s, rho, T = member(N, L, seed)
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


@pytest.mark.parametrize("precision", ["tf32", "tf32acc"])
def test_batch_step_vs_oracle(P, precision):
    # One stacked step of members of every basis-size group of the batched
    # workload (N = 8 ... 48), each checked against the oracle's Heun step
    # (Eq. equalt) from that member's own history with the paper's Eq.
    # (2b-opt) contraction: rho(t_{n+1}) and, through the step's diagnostics,
    # E_c = 1/2 Im Tr I(t_n) and Re Tr I(t_n).
    spec = [(8, 40, 21), (12, 25, 22), (16, 18, 23), (24, 12, 24), (32, 9, 25), (48, 6, 26),
            (16, 7, 27)]
    dt, E_n, E_np1 = 0.02, 0.03, -0.02
    batched = [make(P, N, L, sd, 1, precision) for N, L, sd in spec]
    with P.Batch(batched) as b:
        rhos, diags = b.step(E_n, E_np1)
    for i, (N, L, sd) in enumerate(spec):
        s, rho, T = member(N, L, sd)
        r_ref, I_ref, _ = O.heun_step(s["h"], s["v"], s["d"], list(rho), list(T), dt, E_n, E_np1,
                                      route="paper")
        # the step's increment rho(t_{n+1}) - rho(t_n) is linear in the two
        # collision integrals (plus FP64 commutators), so it carries their
        # relative error: the split-TF32 collision tolerance applies to it
        e = check(rhos[i] - rho[-1], r_ref - rho[-1], 2e-5, f"member N={N} L={L} increment")
        check(rhos[i], r_ref, 1e-5, f"member N={N} L={L} rho")
        ec_ref = 0.5 * np.trace(I_ref).imag
        # |Tr X| <= sqrt(N) ||X||_F bounds the trace's error by the matrix's
        assert abs(diags[i][2] - ec_ref) < 2e-5 * 0.5 * np.sqrt(N) * np.linalg.norm(I_ref), \
            (N, L, diags[i][2], ec_ref)
        assert abs(diags[i][3]) < 1e-5 * np.abs(I_ref).max() * N
        print(f"batch member N={N} L={L} {precision}: rho vs oracle {e:.2e}, "
              f"E_c {diags[i][2]:.6e} vs {ec_ref:.6e}")
    for c in batched:
        c.close()


def test_batch_graph_steps_match_eager_steps(P):
    # the same kernels in the same order, launched as one captured graph per
    # step (the executable graph updated in place as the histories grow)
    spec = [(8, 20, 31), (12, 14, 32), (24, 9, 33), (48, 5, 34)]
    steps = 3
    eager = [make(P, N, L, sd, steps) for N, L, sd in spec]
    graph = [make(P, N, L, sd, steps) for N, L, sd in spec]
    E = [0.02 * k for k in range(steps + 1)]
    with P.Batch(eager) as a, P.Batch(graph) as g:
        g.set_options(use_graph=True)
        for k in range(steps):
            ra, da = a.step(E[k], E[k + 1])
            rg, dg = g.step(E[k], E[k + 1])
            for i in range(len(spec)):
                assert np.array_equal(ra[i], rg[i]), (k, spec[i])
                assert np.array_equal(da[i], dg[i]), (k, spec[i])
    for c in eager + graph:
        c.close()


def test_batch_autotune_records_choices_and_keeps_accuracy(P):
    # the autotuner's choices per basis-size group, then a tuned (graph) step
    # against the oracle's Heun step
    spec = [(8, 30, 41), (16, 22, 42), (32, 12, 43), (48, 6, 44)]
    dt, E_n, E_np1 = 0.02, 0.01, -0.03
    ctxs = [make(P, N, L, sd, 1) for N, L, sd in spec]
    with P.Batch(ctxs) as b:
        tuned = b.autotune()
        b.set_options(use_graph=True)
        rhos, diags = b.step(E_n, E_np1)
    print("autotuned:", tuned)
    assert [t["N"] for t in tuned] == [8, 16, 32, 48]
    for t in tuned:
        assert t["units_per_round"] >= 1 and t["acc_window"] in (8, 16, 32)
        assert t["s4_item_k"] in (4096, 8192, 16384) and t["us_per_unit"] > 0
    for i, (N, L, sd) in enumerate(spec):
        s, rho, T = member(N, L, sd)
        r_ref, _, _ = O.heun_step(s["h"], s["v"], s["d"], list(rho), list(T), dt, E_n, E_np1,
                                  route="paper")
        check(rhos[i] - rho[-1], r_ref - rho[-1], 2e-5, f"tuned member N={N} increment")
        check(rhos[i], r_ref, 1e-5, f"tuned member N={N} rho")
    for c in ctxs:
        c.close()
