"""Seeded synthetic inputs for the GKBA second-Born workloads.

This module only *draws* inputs; it holds none of the method's arithmetic
(no self-energy, no collision integral, no mean field, no time stepping).
Both the CPU oracle (``oracle/``) and the CUDA path (``paper_1905_01180_gb300``)
take their inputs from here, so the two sides see bit-identical arrays.

Model inputs follow Sec. II of Tuovinen, Covito & Sentef (arXiv:1905.01180):
a one-body matrix h_ij (Eq. onebody), real Coulomb integrals v_ijkl with the
8-fold permutation symmetry of Eq. (symmetries), a dipole matrix d and an
initial one-particle density matrix rho0.  The paper's own integrals (CH4 in an
Octopus Kohn-Sham basis) are not available, so a seeded generator stands in:

* v_ijkl = sum_P B^P_il B^P_jk with symmetric Gaussian B^P
  (sigma_P = 0.3 exp(-P/4)), which is real and 8-fold symmetric because the
  pairs (i,l) and (j,k) sit at the same space point in Eq. (coulomb);
* h = diag(concat(linspace(-1,-0.5,N/2), linspace(0.5,1,N/2))) plus a symmetric
  off-diagonal part drawn from U(-0.1, 0.1);
* d symmetric with entries U(-1, 1);
* rho0 = projector on the n_occ = max(1, N//4) lowest eigenvectors of h
  (per spin; spin-restricted, Sec. II);
* E(t) = 0.1 sin^2(pi t/10) sin(t) on [0, 10], zero elsewhere.

Draw order from ``numpy.random.default_rng(seed)`` (PCG64): the upper triangle
of h's off-diagonal part (row-major), then each B^P's upper triangle including
the diagonal (row-major), then d's upper triangle including the diagonal.

For a single collision-integral evaluation with a long history, ``history``
draws random Hermitian rho_k with eigenvalues in [0, 1] and random unitary
propagators T(t, t_k) = U_{L-2} ... U_k, U_j = exp(-i H_j dt), H_j random
Hermitian with N(0, 0.5^2) real and imaginary parts; T(t, t_{L-1}) = 1.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

__all__ = [
    "field",
    "system",
    "history",
    "random_pair",
    "random_symmetric_v",
    "chain",
]


def field(t):
    """Pulse E(t) = 0.1 sin^2(pi t / 10) sin(t) for 0 <= t <= 10, else 0."""
    t = np.asarray(t, dtype=np.float64)
    e = 0.1 * np.sin(np.pi * t / 10.0) ** 2 * np.sin(t)
    return np.where((t >= 0.0) & (t <= 10.0), e, 0.0)


def _h_diagonal(N):
    if N == 1:
        return np.array([-1.0])
    lo = N // 2
    hi = N - lo
    return np.concatenate([np.linspace(-1.0, -0.5, lo), np.linspace(0.5, 1.0, hi)])


def system(N, n_P, seed=0, n_occ=None):
    """Seeded model system: returns dict(h, v, d, rho0, B, n_occ).

    h, d, rho0 are complex128 (N, N); v is float64 (N, N, N, N) indexed
    v[i, j, k, l] as in Eq. (coulomb); B is float64 (n_P, N, N).
    """
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(N, k=1)
    iu0 = np.triu_indices(N, k=0)

    h = np.diag(_h_diagonal(N)).astype(np.float64)
    off = rng.uniform(-0.1, 0.1, size=len(iu[0]))
    h[iu] = off
    h[(iu[1], iu[0])] = off

    B = np.zeros((n_P, N, N))
    for P in range(n_P):
        sig = 0.3 * np.exp(-P / 4.0)
        vals = rng.normal(0.0, sig, size=len(iu0[0]))
        B[P][iu0] = vals
        B[P][(iu0[1], iu0[0])] = vals

    d = np.zeros((N, N))
    dv = rng.uniform(-1.0, 1.0, size=len(iu0[0]))
    d[iu0] = dv
    d[(iu0[1], iu0[0])] = dv

    # v_ijkl = sum_P B^P_il B^P_jk  (pairs (i,l) and (j,k))
    v = np.einsum("pil,pjk->ijkl", B, B, optimize=True)

    if n_occ is None:
        n_occ = max(1, N // 4)
    _, vecs = np.linalg.eigh(h)
    occ = vecs[:, :n_occ]
    rho0 = occ @ occ.conj().T

    return dict(
        h=h.astype(np.complex128),
        v=np.ascontiguousarray(v),
        d=d.astype(np.complex128),
        rho0=rho0.astype(np.complex128),
        B=B,
        n_occ=n_occ,
    )


def _haar_unitary(rng, N):
    z = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def history(N, L, dt, seed=0):
    """Synthetic two-time history for one collision-integral evaluation.

    Returns (rho_hist, T_hist), complex128 arrays of shape (L, N, N):
    rho_hist[k] = V_k diag(lambda_k) V_k^dagger with V_k Haar and
    lambda_k ~ U[0, 1]; T_hist[k] = U_{L-2} ... U_k with
    U_j = expm(-i H_j dt), and T_hist[L-1] = identity.
    """
    rng = np.random.default_rng(seed)
    rho = np.empty((L, N, N), np.complex128)
    for k in range(L):
        V = _haar_unitary(rng, N)
        lam = rng.uniform(0.0, 1.0, size=N)
        rho[k] = (V * lam[None, :]) @ V.conj().T
    T = np.empty((L, N, N), np.complex128)
    T[L - 1] = np.eye(N)
    Hs = []
    for _ in range(L - 1):
        A = rng.normal(0.0, 0.5, size=(N, N)) + 1j * rng.normal(0.0, 0.5, size=(N, N))
        Hs.append(0.5 * (A + A.conj().T))
    for k in range(L - 2, -1, -1):
        U = scipy.linalg.expm(-1j * dt * Hs[k])
        T[k] = T[k + 1] @ U
    return rho, T


def random_pair(N, seed=0, scale=1.0):
    """A random complex pair (G, Gbar) of N x N matrices (standard normal)."""
    rng = np.random.default_rng(seed)
    G = scale * (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)))
    Gb = scale * (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)))
    return G, Gb


def random_symmetric_v(N, n_P=None, seed=0):
    """Random real 8-fold symmetric v = sum_P B^P_il B^P_jk (Gaussian B^P)."""
    rng = np.random.default_rng(seed)
    if n_P is None:
        n_P = N
    B = rng.normal(size=(n_P, N, N))
    B = 0.5 * (B + B.transpose(0, 2, 1))
    return np.ascontiguousarray(np.einsum("pil,pjk->ijkl", B, B, optimize=True))


def chain(N, interaction="diagonal", J=-1.0, U=1.0, W=100.0):
    """Polymer-chain workloads of Sec. IV: a 1D chain of N sites with
    nearest-neighbour hopping J (open ends) and either

    * interaction="diagonal":  on-site U_i = U (Hubbard-like, Sec. III A), or
    * interaction="symmetric": Ohno V_ij = U / sqrt(1 + |i - j|^2) (Sec. III B).

    Initial state: N//2 particles per spin confined to the N//2 leftmost sites,
    rho0 = projector on the N//2 lowest eigenvectors of h + W sum_{i >= N//2}
    |i><i| (W = 100, a strong confinement); the propagation uses h alone (the
    confinement is released at t = 0).  d = diag(i - (N-1)/2), the site
    position, for a field if one is applied.  Deterministic (no draws).

    Returns dict(h, v, d, rho0) with v = the vector U (diagonal) or the matrix
    V (symmetric), the form gkba_init takes for those interactions.
    """
    h = np.zeros((N, N), np.complex128)
    for i in range(N - 1):
        h[i, i + 1] = h[i + 1, i] = J
    idx = np.arange(N)
    if interaction == "diagonal":
        v = np.full(N, float(U))
    elif interaction == "symmetric":
        v = U / np.sqrt(1.0 + (idx[:, None] - idx[None, :]) ** 2.0)
    else:
        raise ValueError(f"unknown interaction {interaction!r}")
    n_occ = max(1, N // 2)
    hc = h + np.diag(np.where(idx >= N // 2, W, 0.0))
    _, vec = np.linalg.eigh(hc)
    occ = vec[:, :n_occ]
    rho0 = occ @ occ.conj().T
    rho0 = 0.5 * (rho0 + rho0.conj().T)
    d = np.diag(idx - 0.5 * (N - 1)).astype(np.complex128)
    return dict(h=h, v=np.ascontiguousarray(v), d=d, rho0=rho0)
