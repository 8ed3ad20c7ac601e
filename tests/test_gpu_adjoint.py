"""GPU parity of the collision integral's adjoint (gkba_collision_vjp) and of
the trilinear form it is built from (gkba_sigma3), against the oracle.

The oracle's collision_vjp differentiates the einsum of Eq. (2bse) slot by
slot and is pinned by finite differences (tests/test_oracle_adjoint.py); the
CUDA path evaluates each slot derivative as an S3 value on the tensor-core (or
FP64) contraction chain.  Tolerances: FP64 path 1e-10; split-TF32 path 1e-4
(each of the four S3 evaluations carries the 2e-5 gate of the forward path,
and the gradient sums terms of different sign).
"""
import numpy as np
import pytest

import gkba_inputs as gi
import oracle as O
from _check import check, rel

pytestmark = pytest.mark.gpu




def cplx(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


TOL = {"fp64": 1e-10, "tf32": 1e-4}


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_01180_gb300 import build as b
    b.build()
    import paper_1905_01180_gb300 as p
    return p


@pytest.mark.parametrize("precision", ["fp64", "tf32"])
@pytest.mark.parametrize("N", [4, 13, 24])
def test_sigma3_vs_oracle(P, precision, N):
    s = gi.system(N, 8, seed=N)
    rng = np.random.default_rng(N)
    A, B, C = (cplx(rng, 3, N, N) for _ in range(3))
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.02, precision=precision)
    S = ctx.sigma3(A, B, C)
    ctx.close()
    e = check(S, O.sigma3(s["v"], A, B, C), 1e-10 if precision == "fp64" else 2e-5, "S3")
    print(f"N={N} {precision} sigma3 rel err {e:.2e}")


@pytest.mark.parametrize("precision", ["fp64", "tf32"])
@pytest.mark.parametrize("N,L", [(8, 4), (16, 3), (13, 3), (40, 2)])
def test_collision_vjp_vs_oracle(P, precision, N, L):
    s = gi.system(N, 8, seed=1)
    rho, T = gi.history(N, L, 0.02, seed=2)
    rng = np.random.default_rng(3)
    Ibar = cplx(rng, N, N)
    w = O.trapezoid_weights(L, 0.02)
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.02, precision=precision)
    rb, tb = ctx.collision_vjp(rho, T, Ibar)
    ctx.close()
    rr, tr = O.collision_vjp(s["v"], rho, T, w, Ibar)
    er = check(rb, rr, TOL[precision], "rho_bar")
    et = check(tb, tr, TOL[precision], "T_bar")
    print(f"N={N} L={L} {precision} collision VJP rel err rho_bar {er:.2e} T_bar {et:.2e}")


def test_collision_autograd(P):
    # torch autograd through the library: I = collision(rho, T) on the GPU,
    # loss = Re sum conj(a) I; the gradients equal the oracle's adjoint
    import torch
    from paper_1905_01180_gb300 import gkba
    N, L = 8, 3
    s = gi.system(N, 8, seed=4)
    rho, T = gi.history(N, L, 0.02, seed=5)
    a = cplx(np.random.default_rng(6), N, N)
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.02)
    r = torch.tensor(rho, device="cuda", requires_grad=True)
    t = torch.tensor(T, device="cuda", requires_grad=True)
    I = gkba.collision_autograd(ctx, r, t)
    loss = torch.real(torch.sum(torch.conj(torch.tensor(a, device="cuda")) * I))
    loss.backward()
    rr, tr = O.collision_vjp(s["v"], rho, T, O.trapezoid_weights(L, 0.02), a)
    check(r.grad.cpu().numpy(), rr, 1e-10)
    check(t.grad.cpu().numpy(), tr, 1e-10)
    ref = O.collision(s["v"], rho, T, O.trapezoid_weights(L, 0.02), route="paper")
    check(I.detach().cpu().numpy(), ref, 1e-10)
    ctx.close()


def test_collision_vjp_v_vs_oracle(P):
    # dL/dv through the collision integral (FP64 path) against the oracle's
    # slot-by-slot einsum derivative (pinned by finite differences)
    N, L = 5, 3
    s = gi.system(N, 8, seed=6)
    rho, T = gi.history(N, L, 0.02, seed=7)
    Ibar = cplx(np.random.default_rng(8), N, N)
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.02)
    rb, tb, vb = ctx.collision_vjp(rho, T, Ibar, want_v=True)
    ctx.close()
    ref = O.collision_vjp_v(s["v"], rho, T, O.trapezoid_weights(L, 0.02), Ibar)
    e = check(vb, ref, 1e-10, "v_bar")
    print(f"N={N} L={L} collision dL/dv rel err {e:.2e}")
    rr, tr = O.collision_vjp(s["v"], rho, T, O.trapezoid_weights(L, 0.02), Ibar)
    check(rb, rr, 1e-10, "rho_bar")
    check(tb, tr, 1e-10, "T_bar")


@pytest.mark.parametrize("N", [5, 32, 40])
@pytest.mark.parametrize("precision", ["tf32", "tf32acc"])
def test_collision_vjp_v_split_tf32_vs_oracle(P, N, precision):
    # dL/dv on the tensor-core path: the v slot reads the chain's FP32 X3, the
    # w slot runs the chain on the omega layout of v.  N = 5 and 40 pad to
    # Np = 16 and 48 (row-major X3), N = 32 is the K-blocked X3 layout.
    L = 3
    s = gi.system(N, 8, seed=16)
    rho, T = gi.history(N, L, 0.02, seed=17)
    Ibar = cplx(np.random.default_rng(18), N, N)
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.02, precision=precision)
    rb, tb, vb = ctx.collision_vjp(rho, T, Ibar, want_v=True)
    ctx.close()
    ref = O.collision_vjp_v(s["v"], rho, T, O.trapezoid_weights(L, 0.02), Ibar)
    e = check(vb, ref, 2e-5, f"v_bar N={N} {precision}")
    print(f"N={N} L={L} {precision} collision dL/dv rel err {e:.2e}")
    rr, tr = O.collision_vjp(s["v"], rho, T, O.trapezoid_weights(L, 0.02), Ibar)
    check(rb, rr, 2e-5, "rho_bar")
    check(tb, tr, 2e-5, "T_bar")
