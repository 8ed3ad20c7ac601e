"""Adjoint of the Heun stepper (gkba_adjoint): gradients of the final dipole
L = Re Tr[d rho(t_n)] with respect to the field samples E(t_k) and the
initial state rho(t_0), through every collision integral of the trajectory.

Pins: central finite differences of the library's own forward propagation
(FP64), and finite differences of the oracle's propagation (an independent
forward), at small N.
"""
import numpy as np
import pytest

import gkba_inputs as gi
import oracle as O
from _check import check

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


def run(P, s, dt, E, rho0=None, precision="fp64"):
    n = len(E) - 1
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"] if rho0 is None else rho0, dt,
                    max_steps=n, precision=precision)
    for k in range(n):
        rho, _, _ = ctx.step(E[k], E[k + 1])
    return ctx, float(np.real(np.trace(s["d"] @ rho)))


def setup(N=6, n=12, dt=0.05):
    s = gi.system(N, 8, seed=3)
    E = 0.2 * np.sin(0.7 * np.arange(n + 1) * dt * 10)
    return s, dt, E


def test_field_gradient_matches_library_finite_differences(P):
    s, dt, E = setup()
    ctx, L0 = run(P, s, dt, E)
    E_bar, rho0_bar = ctx.adjoint(s["d"])
    ctx.close()
    eps = 1e-5
    for k in (0, 3, 7, len(E) - 1):
        Ep, Em = E.copy(), E.copy()
        Ep[k] += eps
        Em[k] -= eps
        cp, Lp = run(P, s, dt, Ep)
        cm, Lm = run(P, s, dt, Em)
        cp.close()
        cm.close()
        fd = (Lp - Lm) / (2 * eps)
        print(f"dL/dE_{k}: adjoint {E_bar[k]:+.10e}  finite differences {fd:+.10e}")
        assert abs(E_bar[k] - fd) < 1e-6 * max(abs(fd), 1e-3)


def test_initial_state_gradient_matches_finite_differences(P):
    s, dt, E = setup()
    ctx, L0 = run(P, s, dt, E)
    _, rho0_bar = ctx.adjoint(s["d"])
    ctx.close()
    rng = np.random.default_rng(9)
    X = rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6))
    D = 0.5 * (X + X.conj().T)  # Hermitian direction (gkba_init checks rho0)
    eps = 1e-5
    cp, Lp = run(P, s, dt, E, s["rho0"] + eps * D)
    cm, Lm = run(P, s, dt, E, s["rho0"] - eps * D)
    cp.close()
    cm.close()
    fd = (Lp - Lm) / (2 * eps)
    ad = float(np.real(np.sum(np.conj(rho0_bar) * D)))
    print(f"dL/drho0 along D: adjoint {ad:+.10e}  finite differences {fd:+.10e}")
    assert abs(ad - fd) < 1e-6 * max(abs(fd), 1e-3)


def test_field_gradient_matches_oracle_finite_differences(P):
    # the independent forward: the oracle's Heun propagation
    N, n, dt = 4, 8, 0.05
    s = gi.system(N, 4, seed=5)
    E = 0.3 * np.cos(np.arange(n + 1) * 0.4)
    ctx, _ = run(P, s, dt, E)
    E_bar, _ = ctx.adjoint(s["d"])
    ctx.close()

    def loss(Ev):
        pr = O.propagate(s["h"], s["v"], s["d"], s["rho0"], dt, n, Ev)
        return float(np.real(np.trace(s["d"] @ pr.rho[n])))

    eps = 1e-5
    for k in range(n + 1):
        Ep, Em = E.copy(), E.copy()
        Ep[k] += eps
        Em[k] -= eps
        fd = (loss(Ep) - loss(Em)) / (2 * eps)
        assert abs(E_bar[k] - fd) < 1e-6 * max(abs(fd), 1e-3), (k, E_bar[k], fd)


def test_split_tf32_gradient_close_to_fp64(P):
    s, dt, E = setup(N=16, n=10)
    c64, _ = run(P, s, dt, E)
    g64, _ = c64.adjoint(s["d"])
    c64.close()
    ctf, _ = run(P, s, dt, E, precision="tf32acc")
    gtf, _ = ctf.adjoint(s["d"])
    ctf.close()
    e = np.linalg.norm(gtf - g64) / np.linalg.norm(g64)
    print(f"split-TF32 (accurate) field gradient vs FP64: rel {e:.2e}")
    assert e < 1e-3


def test_dipole_autograd(P):
    # torch autograd of the final dipole w.r.t. the pulse samples
    import torch
    from paper_1905_01180_gb300 import gkba
    s, dt, E = setup(N=6, n=8)
    make = lambda: P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=len(E) - 1)
    Et = torch.tensor(E, dtype=torch.float64, requires_grad=True)
    L = gkba.dipole_autograd(make, Et, s["d"])
    L.backward()
    ctx, L0 = run(P, s, dt, E)
    E_bar, _ = ctx.adjoint(s["d"])
    ctx.close()
    assert abs(L.item() - L0) < 1e-12
    assert np.allclose(Et.grad.numpy(), E_bar, rtol=1e-12, atol=1e-15)


def test_adjoint_after_batched_steps(P):
    # gkba_batch_step records the trajectory like gkba_step: the adjoint of a
    # member equals the adjoint of the same system stepped on its own
    s, dt, E = setup(N=8, n=6)
    n = len(E) - 1
    make = lambda: P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, precision="tf32")
    other = gi.system(12, 8, seed=7)
    a, b = make(), make()
    c = P.Context(other["h"], other["v"], other["d"], other["rho0"], dt, max_steps=n, precision="tf32")
    with P.Batch([a, c]) as bt:
        for k in range(n):
            bt.step([E[k], 0.0], [E[k + 1], 0.0])
    for k in range(n):
        b.step(E[k], E[k + 1])
    ga, ra = a.adjoint(s["d"])
    gb, rb = b.adjoint(s["d"])
    for x in (a, b, c):
        x.close()
    assert np.array_equal(ga, gb) and np.array_equal(ra, rb)


def symmetrize8(x):
    perms = [(0, 1, 2, 3), (1, 0, 3, 2), (3, 2, 1, 0), (2, 3, 0, 1),
             (3, 1, 2, 0), (1, 3, 0, 2), (0, 2, 1, 3), (2, 0, 3, 1)]
    return sum(x.transpose(p) for p in perms) / 8.0


def test_coulomb_gradient_matches_finite_differences(P):
    # dL/dv through every collision integral and mean field of the trajectory,
    # along an 8-fold symmetric direction (gkba_init accepts v +- eps dv)
    N, n, dt = 5, 8, 0.05
    s = gi.system(N, 6, seed=8)
    E = 0.2 * np.sin(np.arange(n + 1) * 0.5)
    ctx, _ = run(P, s, dt, E)
    _, _, vbar = ctx.adjoint(s["d"], want_v=True)
    ctx.close()
    dv = symmetrize8(np.random.default_rng(10).normal(size=(N,) * 4))
    eps = 1e-6

    def loss(vv):
        s2 = dict(s)
        s2["v"] = vv
        c, L = run(P, s2, dt, E)
        c.close()
        return L

    fd = (loss(s["v"] + eps * dv) - loss(s["v"] - eps * dv)) / (2 * eps)
    ad = float(np.sum(vbar * dv))
    print(f"dL/dv along dv: adjoint {ad:+.10e}  finite differences {fd:+.10e}")
    assert abs(ad - fd) < 1e-6 * max(abs(fd), 1e-3)


def test_coulomb_factor_gradient(P):
    # gradients of the final dipole w.r.t. the Coulomb factors B^P of
    # v = sum_P B^P (x) B^P, along a direction that keeps every B^P symmetric
    from paper_1905_01180_gb300 import gkba
    N, nP, n, dt = 4, 3, 6, 0.05
    s = gi.system(N, 4, seed=12)
    rng = np.random.default_rng(13)
    B = rng.normal(size=(nP, N, N)) * 0.4
    B = 0.5 * (B + B.transpose(0, 2, 1))
    vofB = lambda b: np.einsum("pil,pjk->ijkl", b, b)
    E = 0.2 * np.cos(np.arange(n + 1) * 0.3)

    def forward(b):
        s2 = dict(s)
        s2["v"] = vofB(b)
        return run(P, s2, dt, E)

    ctx, _ = forward(B)
    _, _, vbar = ctx.adjoint(s["d"], want_v=True)
    ctx.close()
    gB = gkba.coulomb_factor_grad(B, vbar)
    dB = rng.normal(size=B.shape)
    dB = 0.5 * (dB + dB.transpose(0, 2, 1))
    eps = 1e-6
    cp, Lp = forward(B + eps * dB)
    cm, Lm = forward(B - eps * dB)
    cp.close()
    cm.close()
    fd = (Lp - Lm) / (2 * eps)
    ad = float(np.sum(gB * dB))
    print(f"dL/dB along dB: adjoint {ad:+.10e}  finite differences {fd:+.10e}")
    assert abs(ad - fd) < 1e-6 * max(abs(fd), 1e-3)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("tf32acc", 1e-5), ("tf32", 1e-5)])
def test_gradients_vs_oracle_autograd(P, precision, tol):
    # The oracle's FP64 gradient of the whole trajectory (reverse-mode autograd
    # of its Heun propagation, Eq. (equalt)) at N = 6: dL/dE(t_k), dL/drho(t_0)
    # and dL/dB^P for L = Re Tr[d rho(t_n)].  The library's v_bar is chained to
    # the factors (coulomb_factor_grad).  Directions that break the symmetry of
    # rho0 (Hermitian) or of B^P (symmetric) leave the model's domain, so the
    # Hermitian / symmetric parts are compared.
    from oracle import stepper_grad as SG
    from paper_1905_01180_gb300 import gkba
    N, n, dt = 6, 10, 0.05
    s = gi.system(N, 6, seed=21)
    E = 0.2 * np.sin(0.9 * np.arange(n + 1) * dt * 10)
    ref = SG.dipole_gradients(s["h"], s["B"], s["d"], s["rho0"], dt, n, E)
    ctx, L = run(P, s, dt, E, precision=precision)
    E_bar, r0, vb = ctx.adjoint(s["d"], want_v=True)
    ctx.close()
    assert abs(L - ref["L"]) < max(tol, 1e-12) * abs(ref["L"])
    herm = lambda X: 0.5 * (X + X.conj().T)
    symm = lambda B: 0.5 * (B + B.transpose(0, 2, 1))
    eE = check(E_bar, ref["E_bar"], tol, "dL/dE")
    er = check(herm(r0), herm(ref["rho0_bar"]), tol, "dL/drho0")
    eB = check(symm(gkba.coulomb_factor_grad(s["B"], vb)), symm(ref["B_bar"]), tol, "dL/dB")
    print(f"{precision}: vs oracle autograd dL/dE {eE:.2e} dL/drho0 {er:.2e} dL/dB {eB:.2e}")


def test_adjoint_refusals(P):
    # a trajectory that did not start at step 0 and a structured interaction
    # are refused (no partial results)
    N, dt = 6, 0.05
    s = gi.system(N, 4, seed=2)
    rho, T = gi.history(N, 3, dt, seed=3)
    c = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=4)
    c.set_history(2, rho, T)
    c.step(0.0, 0.0)
    with pytest.raises(P.GKBAError) as ei:
        c.adjoint(s["d"])
    assert ei.value.status == P.gkba.EUNSUPPORTED
    c.close()
    ch = gi.chain(6, "diagonal")
    c = P.Context(ch["h"], ch["v"], ch["d"], ch["rho0"], dt, max_steps=2, interaction="diagonal")
    c.step(0.0, 0.0)
    with pytest.raises(P.GKBAError) as ei:
        c.adjoint(ch["d"])
    assert ei.value.status == P.gkba.EUNSUPPORTED
    c.close()
    c = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=2, precision="tf32")
    c.step(0.0, 0.0)
    E_bar, _, vb = c.adjoint(s["d"], want_v=True)  # all gradients on the split-TF32 path
    assert np.isfinite(E_bar).all() and np.isfinite(vb).all()
    c.close()
