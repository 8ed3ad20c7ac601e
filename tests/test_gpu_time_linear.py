"""The time-linear history (gkba_config.history = GKBA_HISTORY_TIME_LINEAR):
gkba_step with the history sum of Eq. (collint) kept as one N^4 accumulator.

It is an exact rewrite of the history sum for T(t_n, t_k) = Ucal_n Ucal_k^+,
so every step must reproduce the history-sum stepper (FP64 GPU path) and the
oracle's propagation to rounding.  Tolerances: 1e-11 on rho and the energies
against the history-sum stepper, 1e-10 against the oracle, 1e-9 on the
collision integral (it carries the cancellation of Sigma^> G^< - Sigma^< G^>).
On a split-TF32 context the same steps run their contractions on the tensor
cores: 1e-5 on rho and 2e-5 on I against the oracle and the FP64 path.
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


def field(n, dt):
    return 0.2 * np.sin(0.7 * np.arange(n + 1) * dt * 10)


@pytest.mark.parametrize("N,n,dt", [(8, 40, 0.05), (13, 25, 0.02), (1, 6, 0.1)])
def test_time_linear_matches_history_sum_stepper(P, N, n, dt):
    s = gi.system(N, 8, seed=N)
    E = field(n, dt)
    a = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n)
    b = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, history="time_linear")
    worst_rho = worst_I = worst_E = 0.0
    for k in range(n):
        ra, Ia, da = a.step(E[k], E[k + 1])
        rb, Ib, db = b.step(E[k], E[k + 1])
        worst_rho = max(worst_rho, rel(rb, ra))
        if k > 0:
            worst_I = max(worst_I, rel(Ib, Ia))
        else:
            assert np.abs(Ib).max() == 0.0
        worst_E = max(worst_E, abs(db[1] - da[1]))
    print(f"N={N}, {n} steps: time-linear vs history sum rho {worst_rho:.2e} "
          f"I {worst_I:.2e} energy {worst_E:.2e}")
    assert worst_rho < 1e-11 and worst_I < 1e-9 and worst_E < 1e-11
    # the propagator history stays available in this mode
    na, rha, Ta = a.get_history()
    nb, rhb, Tb = b.get_history()
    assert na == nb == n and rel(Tb, Ta) < 1e-13
    a.close()
    b.close()


def test_time_linear_matches_oracle(P):
    N, n, dt = 6, 15, 0.05
    s = gi.system(N, 8, seed=2)
    E = field(n, dt)
    ref = O.propagate(s["h"], s["v"], s["d"], s["rho0"], dt, n, E, route="paper")
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, history="time_linear")
    for k in range(n):
        rho, I, diag = ctx.step(E[k], E[k + 1])
        check(rho, ref.rho[k + 1], 1e-10)
        if k > 0:
            check(I, ref.I[k], 1e-9)
        assert abs(diag[1] - ref.energy_total[k]) < 1e-10
    ctx.close()


def test_work_per_step_does_not_grow_with_history(P):
    # two accumulator chains per step (t_n and the predicted t_{n+1}) at any n
    N, n, dt = 8, 12, 0.05
    s = gi.system(N, 8, seed=5)
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, history="time_linear")
    per_step = []
    for k in range(n):
        ctx.stats(reset=True)
        ctx.step(0.0, 0.0)
        st, _ = ctx.stats()
        per_step.append((st["S1_w_x_Gbar"]["launches"], st["S1_w_x_Gbar"]["flops"],
                         st["time_linear"]["launches"]))
    assert all(p[0] == 2 for p in per_step)
    assert len(set(per_step[1:])) == 1
    ctx.close()


@pytest.mark.parametrize("ws_units", [0, 4])
def test_set_history_rebuilds_the_accumulator(P, ws_units):
    # restore a checkpoint of a history-sum run into a time-linear context
    # (rebuild over 9 points, in chunks of 2 when the workspace holds 4 units)
    N, n0, n1, dt = 8, 9, 6, 0.05
    s = gi.system(N, 8, seed=7)
    E = field(n0 + n1, dt)
    a = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n0 + n1)
    for k in range(n0):
        a.step(E[k], E[k + 1])
    n, rho_hist, T_hist = a.get_history()
    N2 = N * N
    per_unit = 2 * (2 * N2 * N2 * 8) + 6 * N2 * 8 + N * 2 * N * 8 + 20 * N2 * 16 + 8
    ws = int(4.5 * per_unit) if ws_units else 0
    b = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n0 + n1,
                  workspace_bytes=ws, history="time_linear")
    b.set_history(n, rho_hist, T_hist)
    for k in range(n0, n0 + n1):
        ra, Ia, _ = a.step(E[k], E[k + 1])
        rb, Ib, _ = b.step(E[k], E[k + 1])
        check(rb, ra, 1e-11)
        check(Ib, Ia, 1e-9)
    a.close()
    b.close()


def test_set_history_needs_identity_at_t_n(P):
    N, dt = 5, 0.05
    s = gi.system(N, 8, seed=1)
    rho, T = gi.history(N, 4, dt, seed=2)
    T = T.copy()
    T[-1] = T[0]  # not the identity
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=6, history="time_linear")
    with pytest.raises(P.GKBAError) as ei:
        ctx.set_history(3, rho, T)
    assert ei.value.status == P.gkba.EINVAL
    ctx.close()


def test_adjoint_of_a_time_linear_run(P):
    # the trajectory is the history-sum one up to rounding, and so are the
    # gradients gkba_adjoint takes through it
    N, n, dt = 5, 8, 0.05
    s = gi.system(N, 8, seed=3)
    E = field(n, dt)
    out = []
    for mode in ("sum", "time_linear"):
        ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, history=mode)
        for k in range(n):
            ctx.step(E[k], E[k + 1])
        out.append(ctx.adjoint(s["d"]))
        ctx.close()
    (Ea, ra), (Eb, rb) = out
    assert rel(Eb, Ea) < 1e-10 and rel(rb, ra) < 1e-10


def test_time_linear_runs_are_bitwise_reproducible(P):
    # fixed-order FP64 GEMMs and reductions: two runs agree bit for bit
    N, n, dt = 9, 6, 0.05
    s = gi.system(N, 8, seed=4)
    E = field(n, dt)
    outs = []
    for _ in range(2):
        ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, history="time_linear")
        outs.append([ctx.step(E[k], E[k + 1]) for k in range(n)])
        ctx.close()
    for (ra, Ia, da), (rb, Ib, db) in zip(*outs):
        assert np.array_equal(ra, rb) and np.array_equal(Ia, Ib) and np.array_equal(da, db)


def test_config1_time_linear_full_run(P):
    # N = 24, 32 factors, dt = 0.02, the pulse on [0, 10], 1000 Heun steps:
    # the first 100 against the oracle (tests/golden, written by the oracle
    # only), then the whole run's invariants (particle number, Hermiticity,
    # E_c < 0) with the time-linear history in FP64
    import os
    import time
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "config1_oracle_100steps.npz"))
    s = gi.system(24, 32, seed=0)
    dt = float(g["dt"])
    E = gi.field(dt * np.arange(1001))
    n = 1000
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, history="time_linear")
    rho_at, tr, herm, ec = {}, [], 0.0, []
    t0 = time.perf_counter()
    for k in range(n):
        rho, I, diag = ctx.step(E[k], E[k + 1])
        if k < 100:
            rho_at[k + 1] = rho
            assert abs(diag[1] - g["energy_total"][k]) < 1e-10 * max(1.0, abs(g["energy_total"][k]))
        tr.append(diag[0])
        ec.append(diag[2])
        herm = max(herm, np.abs(rho - rho.conj().T).max())
    wall = time.perf_counter() - t0
    ctx.close()
    w_rho = max(check(rho_at[m], r, 1e-10, f"rho step {m}") for m, r in zip(g["steps"][1:], g["rho"][1:]))
    tr = np.array(tr)
    print(f"config1 time-linear FP64: 1000 steps in {wall:.2f} s, rho vs oracle (100 steps) "
          f"{w_rho:.2e}, |Tr rho - 6| {np.abs(tr - 6).max():.2e}, herm {herm:.2e}, "
          f"E_c end {ec[-1]:.4e}")
    assert w_rho < 1e-10
    assert np.abs(tr - 6.0).max() < 1e-11
    assert herm < 1e-12
    assert ec[-1] < 0.0


@pytest.mark.parametrize("precision", ["tf32", "tf32acc"])
def test_time_linear_split_tf32_matches_oracle(P, precision):
    # terms, their accumulation over j, the three back-transforms and stage S4
    # on the tensor cores; Lambda_acc in FP64.  Against the oracle's history-sum
    # propagation (Eq. (2b-opt) contraction) step by step.
    N, n, dt = 6, 15, 0.05
    s = gi.system(N, 8, seed=2)
    E = field(n, dt)
    ref = O.propagate(s["h"], s["v"], s["d"], s["rho0"], dt, n, E, route="paper")
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, history="time_linear",
                    precision=precision)
    wr = wi = 0.0
    for k in range(n):
        rho, I, diag = ctx.step(E[k], E[k + 1])
        wr = max(wr, check(rho, ref.rho[k + 1], 1e-5, f"rho step {k + 1}"))
        if k > 0:
            wi = max(wi, check(I, ref.I[k], 2e-5, f"I step {k}"))
    print(f"time-linear {precision} N={N}: rho vs oracle {wr:.2e}, I {wi:.2e}")
    ctx.close()


@pytest.mark.parametrize("N,n", [(13, 12), (32, 8), (34, 6)])
def test_time_linear_split_tf32_matches_fp64(P, N, n):
    # Np = 16, 32 (K-blocked X3) and 48: the split-TF32 time-linear steps
    # against the FP64 history-sum stepper (dt = 0.02: with dt = 0.05 the
    # seeded systems from N = 40 on leave Heun's stability region in FP64 too)
    dt = 0.02
    s = gi.system(N, 8, seed=N)
    E = field(n, dt)
    a = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n)
    b = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, history="time_linear",
                  precision="tf32")
    wr = wi = 0.0
    for k in range(n):
        ra, Ia, da = a.step(E[k], E[k + 1])
        rb, Ib, db = b.step(E[k], E[k + 1])
        wr = max(wr, check(rb, ra, 1e-5, f"rho step {k + 1}"))
        if k > 0:
            wi = max(wi, check(Ib, Ia, 2e-5, f"I step {k}"))
        assert abs(db[0] - da[0]) < 1e-6  # particle number (split-TF32 Re Tr I)
    print(f"time-linear split-TF32 N={N}: rho vs FP64 history sum {wr:.2e}, I {wi:.2e}")
    a.close()
    b.close()


def test_time_linear_split_tf32_set_history(P):
    # the accumulator rebuilt over 9 history points in one batch, then steps,
    # against the FP64 history-sum stepper
    N, n0, n1, dt = 16, 9, 4, 0.05
    s = gi.system(N, 8, seed=7)
    E = field(n0 + n1, dt)
    a = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n0 + n1)
    for k in range(n0):
        a.step(E[k], E[k + 1])
    n, rho_hist, T_hist = a.get_history()
    b = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n0 + n1, history="time_linear",
                  precision="tf32")
    b.set_history(n, rho_hist, T_hist)
    for k in range(n0, n0 + n1):
        ra, Ia, _ = a.step(E[k], E[k + 1])
        rb, Ib, _ = b.step(E[k], E[k + 1])
        check(rb, ra, 1e-5, f"rho step {k + 1}")
        check(Ib, Ia, 2e-5, f"I step {k}")
    a.close()
    b.close()
