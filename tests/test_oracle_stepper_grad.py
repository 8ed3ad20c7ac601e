"""Pins of the oracle's stepper gradients (``oracle.stepper_grad``).

The autograd forward is pinned to ``oracle.propagate`` (the NumPy stepper,
itself pinned in ``test_oracle_gkba.py``), and every gradient to central
finite differences of ``oracle.propagate``: along the field samples E(t_k),
along a Hermitian direction of rho(t_0) and along a symmetric direction of
each Coulomb factor B^P (v_ijkl = sum_P B^P_il B^P_jk).
"""
import numpy as np
import pytest

import gkba_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
from oracle import stepper_grad as SG  # noqa: E402


def setup(N=3, n_P=3, n=5, dt=0.05, seed=11):
    s = gi.system(N, n_P, seed=seed)
    E = 0.3 * np.cos(np.arange(n + 1) * 0.4)
    return s, dt, n, E


def dipole(s, dt, n, E, rho0=None, B=None):
    v = s["v"] if B is None else np.einsum("pil,pjk->ijkl", B, B)
    pr = O.propagate(s["h"], v, s["d"], s["rho0"] if rho0 is None else rho0, dt, n, E)
    return float(np.real(np.trace(s["d"] @ pr.rho[n])))


def test_autograd_forward_matches_numpy_propagation():
    s, dt, n, E = setup(N=4, n_P=4, n=6)
    t = lambda x: torch.tensor(x)
    rhos = SG.propagate_torch(t(s["h"]), t(s["v"]), t(s["d"]), t(s["rho0"]), dt, n,
                              torch.tensor(E))
    ref = O.propagate(s["h"], s["v"], s["d"], s["rho0"], dt, n, E)
    err = max(np.abs(r.numpy() - ref.rho[k]).max() for k, r in enumerate(rhos))
    assert err < 1e-13, err


def test_field_gradient_matches_finite_differences():
    s, dt, n, E = setup()
    g = SG.dipole_gradients(s["h"], s["B"], s["d"], s["rho0"], dt, n, E)
    assert abs(g["L"] - dipole(s, dt, n, E)) < 1e-13
    eps = 1e-5
    for k in range(n + 1):
        Ep, Em = E.copy(), E.copy()
        Ep[k] += eps
        Em[k] -= eps
        fd = (dipole(s, dt, n, Ep) - dipole(s, dt, n, Em)) / (2 * eps)
        assert abs(g["E_bar"][k] - fd) < 1e-8 * max(abs(fd), 1e-2), (k, g["E_bar"][k], fd)
    # the last sample enters only through the last step's predictor field
    assert abs(g["E_bar"][n]) > 0


def test_initial_state_gradient_matches_finite_differences():
    s, dt, n, E = setup()
    g = SG.dipole_gradients(s["h"], s["B"], s["d"], s["rho0"], dt, n, E)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    D = 0.5 * (X + X.conj().T)
    eps = 1e-5
    fd = (dipole(s, dt, n, E, rho0=s["rho0"] + eps * D)
          - dipole(s, dt, n, E, rho0=s["rho0"] - eps * D)) / (2 * eps)
    ad = float(np.real(np.sum(np.conj(g["rho0_bar"]) * D)))
    assert abs(ad - fd) < 1e-8 * max(abs(fd), 1e-2), (ad, fd)


def test_coulomb_factor_gradient_matches_finite_differences():
    s, dt, n, E = setup()
    g = SG.dipole_gradients(s["h"], s["B"], s["d"], s["rho0"], dt, n, E)
    rng = np.random.default_rng(5)
    for P in range(s["B"].shape[0]):
        X = rng.normal(size=(3, 3))
        D = np.zeros_like(s["B"])
        D[P] = 0.5 * (X + X.T)
        eps = 1e-5
        fd = (dipole(s, dt, n, E, B=s["B"] + eps * D) - dipole(s, dt, n, E, B=s["B"] - eps * D)) \
            / (2 * eps)
        ad = float(np.sum(g["B_bar"] * D))
        assert abs(ad - fd) < 1e-8 * max(abs(fd), 1e-2), (P, ad, fd)
    # dL/dv at fixed B chains to dL/dB through v = sum_P B^P_il B^P_jk
    chained = (np.einsum("ajkb,pjk->pab", g["v_bar"], s["B"])
               + np.einsum("iabl,pil->pab", g["v_bar"], s["B"]))
    assert np.abs(chained - g["B_bar"]).max() < 1e-12 * np.abs(g["B_bar"]).max()
