"""Failure detection and race detection on the GPU without a fault.

* Every device-side wait of the tcgen05 kernels is bounded; an expired wait
  records a code in the context's error word, raises the abort flags of both
  CTAs of a pair and returns, and the host reports GKBA_ETIMEOUT.  The
  self-test makes such a wait run out on a barrier that nothing arrives at,
  then checks that the context keeps working.
* Run-to-run bitwise reproducibility of the FP64 and split-TF32 paths (fixed
  reduction orders) serves as a race detector.
"""
import numpy as np
import pytest

import gkba_inputs as gi
import oracle as O

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


def test_bounded_wait_timeout_reports_and_recovers(P):
    N = 16
    s = gi.system(N, 4, seed=1)
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.02, precision="tf32")
    st, el = ctx.selftest_timeout(50.0)
    print(f"self-test: status {st}, waits ended after {el[0]:.1f} ms (expired) and {el[1]:.1f} ms (peer)")
    assert st == P.gkba.ETIMEOUT
    assert 50.0 <= el[0] < 1000.0          # the expired wait ran to its limit
    assert el[1] < el[0] + 100.0           # the peer left on the abort flag, not its 5 s limit
    assert "timed out" in P.load().gkba_last_error(ctx._h).decode()
    # the error word was consumed; the context still computes correctly
    rho, T = gi.history(N, 3, 0.02, seed=2)
    I = ctx.collision(rho, T)
    ref = O.collision(s["v"], rho, T, O.trapezoid_weights(3, 0.02))
    assert rel(I, ref) < 2e-5
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "tf32"])
def test_runs_are_bitwise_reproducible(P, precision):
    N, L = 24, 9
    s = gi.system(N, 8, seed=4)
    rho, T = gi.history(N, L, 0.02, seed=5)
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.02, precision=precision)
    I1 = ctx.collision(rho, T)
    I2 = ctx.collision(rho, T)
    ctx.close()
    assert np.array_equal(I1, I2)
