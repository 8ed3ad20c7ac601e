"""CPU oracle for the GKBA + second-Born hot path (FP64 / complex128).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call
this package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg (``cpu_baseline`` / ``--impl reference``) use it.  It shares
no code with the CUDA path; both sides take their inputs from ``gkba_inputs``.

Every function restates one passage of Tuovinen, Covito & Sentef,
"Efficient computation of the second-Born self-energy using tensor-contraction
operations" (arXiv:1905.01180).  Plain definitions are written out as such;
a library primitive (``numpy.einsum`` on two operands, ``numpy.linalg.eigh``)
serves as one step where the paper itself names that step.  Units of the
same formula are batched along a leading axis, nothing else is reordered.

Notation (Sec. III): for the self-energy S(G, Gbar) the first argument is
G = G^{<>}(t, t') and the second Gbar = G^{><}(t', t).

Readings of the paper that the oracle fixes (each is pinned by a test in
``tests/test_oracle_*.py``):

* Sigma is Eq. (2bse) with prefactors 2 and -1 and no extra factor i^2;
  Eq. (2bse) reduces to the Hubbard form Eq. (2b-diag) with exactly these.
* The lower limit t0 of the HF propagator in Eq. (prop) is read as t'
  (otherwise G^R(t, t) != -i); T(t_n, t_k) = U_{n-1} ... U_k.
* The collision integral I(t) is the first line of Eq. (collint); the second
  line is its adjoint, so the equation of motion uses I + I^dagger.
* The time integral in Eq. (collint) is the trapezoid rule over t_0 .. t_n.
* The time stepper is Heun's method with the propagator built from the
  average of h_HF at both ends of the step (the paper used no
  predictor-corrector; a second-order scheme is required here).
* Spin-restricted: rho, I and Sigma are per spin (Sec. II).

Beyond the paper: ``collision_vjp`` / ``collision_vjp_v`` (reverse-mode
derivatives of the collision integral) and the time-linear form of the
history sum (``collision_time_linear``, ``propagate_time_linear``), each
pinned against the plain definitions above (finite differences, the history
sum).  ``oracle.stepper_grad`` (a submodule, imported on demand because it
needs PyTorch) gives the gradients of the whole Heun trajectory by automatic
differentiation of the same stepper, pinned by finite differences.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "sigma_loops",
    "sigma_bruteforce",
    "sigma_paper",
    "sigma_independent",
    "sigma3",
    "sigma_hubbard",
    "sigma_symmetric",
    "sigma_bubble",
    "sigma_exchange_diag",
    "gkba_greens",
    "self_energies",
    "trapezoid_weights",
    "collision",
    "collision_vjp",
    "collision_vjp_v",
    "hf_self_energy",
    "expm_hermitian",
    "Propagation",
    "heun_step",
    "propagate",
    "energy",
    "time_linear_factors",
    "time_linear_term",
    "time_linear_apply",
    "collision_time_linear",
    "propagate_time_linear",
]

# --------------------------------------------------------------------------
# Second-Born self-energy, Sec. III
# --------------------------------------------------------------------------


def sigma_loops(v, G, Gb):
    """Eq. (2bse) as eight explicit Python loops (use at N <= 3 only).

    Sigma_ij = 2 sum v_irpn v_mqsj G_nm Gb_sr G_pq
             -   sum v_irpn v_mqsj G_nq Gb_sr G_pm
    """
    N = G.shape[0]
    S = np.zeros((N, N), np.complex128)
    for i in range(N):
        for j in range(N):
            acc = 0.0 + 0.0j
            for m in range(N):
                for n in range(N):
                    for p in range(N):
                        for q in range(N):
                            for r in range(N):
                                for s in range(N):
                                    vv = v[i, r, p, n] * v[m, q, s, j]
                                    acc += vv * (2.0 * G[n, m] * Gb[s, r] * G[p, q]
                                                 - G[n, q] * Gb[s, r] * G[p, m])
            S[i, j] = acc
    return S


def sigma_bruteforce(v, G, Gb):
    """Eq. (2bse) summed over all eight indices at once (N^8; N <= 6).

    ``optimize=False`` makes numpy iterate the full index space directly.
    G, Gb may carry a leading batch axis.
    """
    if G.ndim == 3:
        return np.stack([sigma_bruteforce(v, g, gb) for g, gb in zip(G, Gb)])
    d = np.einsum("irpn,mqsj,nm,sr,pq->ij", v, v, G, Gb, G, optimize=False)
    x = np.einsum("irpn,mqsj,nq,sr,pm->ij", v, v, G, Gb, G, optimize=False)
    return 2.0 * d - x


def sigma_paper(v, G, Gb):
    """The paper's N^5 contraction path, Eq. (2b-opt) / Fig. 2.

    T1_nqsj = sum_m v_mqsj G_nm
    T2_ispn = sum_r v_irpn Gb_sr
    T3_isqn = sum_p G_pq T2_ispn
    Sigma_ij = sum_nqs (2 T1_nqsj T3_isqn - T1_qnjs T3_isnq)
    The exchange term re-uses T1 with permuted indices, which relies on the
    permutation symmetry of Eq. (symmetries).  Batched over a leading axis.
    """
    batched = G.ndim == 3
    if not batched:
        G, Gb = G[None], Gb[None]
    T1 = np.einsum("mqsj,bnm->bnqsj", v, G, optimize=True)
    T2 = np.einsum("irpn,bsr->bispn", v, Gb, optimize=True)
    T3 = np.einsum("bpq,bispn->bisqn", G, T2, optimize=True)
    S = (2.0 * np.einsum("bnqsj,bisqn->bij", T1, T3, optimize=True)
         - np.einsum("bqnjs,bisnq->bij", T1, T3, optimize=True))
    return S if batched else S[0]


def exchange_folded(v):
    """w_mqsj = 2 v_mqsj - v_qmsj: the direct (weight 2) and exchange
    (weight -1) terms of Eq. (2bse) after relabelling m <-> q in the second
    term.  For v with the symmetry v_ijkl = v_jilk this equals
    2 v_mqsj - v_mqjs ("w = 2v - v_exch")."""
    return 2.0 * v - v.transpose(1, 0, 2, 3)


def sigma_independent(v, G, Gb):
    """An N^5 ordering that shares no intermediate with Eq. (2b-opt).

    W1_mqrj = sum_s w_mqsj Gb_sr
    W2_mprj = sum_q G_pq W1_mqrj
    W3_nprj = sum_m G_nm W2_mprj
    Sigma_ij = sum_rpn v_irpn W3_nprj
    with w from ``exchange_folded`` (no symmetry of v is assumed).
    Batched over a leading axis.
    """
    batched = G.ndim == 3
    if not batched:
        G, Gb = G[None], Gb[None]
    w = exchange_folded(v)
    W1 = np.einsum("mqsj,bsr->bmqrj", w, Gb, optimize=True)
    W2 = np.einsum("bpq,bmqrj->bmprj", G, W1, optimize=True)
    W3 = np.einsum("bnm,bmprj->bnprj", G, W2, optimize=True)
    S = np.einsum("irpn,bnprj->bij", v, W3, optimize=True)
    return S if batched else S[0]


def sigma3(v, A, B, C):
    """Eq. (2bse) with its two G slots given separate matrices:

    S3(A, B, C)_ij = sum_{mnpqrs} v_irpn w_mqsj A_nm B_sr C_pq,

    so that S(G, Gbar) = S3(G, Gbar, G).  The same four-step ordering as
    ``sigma_independent``.  Batched over a leading axis.
    """
    batched = A.ndim == 3
    if not batched:
        A, B, C = A[None], B[None], C[None]
    w = exchange_folded(v)
    W1 = np.einsum("mqsj,bsr->bmqrj", w, B, optimize=True)
    W2 = np.einsum("bpq,bmqrj->bmprj", C, W1, optimize=True)
    W3 = np.einsum("bnm,bmprj->bnprj", A, W2, optimize=True)
    S = np.einsum("irpn,bnprj->bij", v, W3, optimize=True)
    return S if batched else S[0]


def sigma_hubbard(U, G, Gb):
    """Diagonal basis, Eq. (2b-diag): Sigma_ij = U_i U_j G_ij Gb_ji G_ij
    for v_ijkl = U_i delta_ij delta_ik delta_il."""
    return np.outer(U, U) * G * Gb.T * G


def sigma_symmetric(V, G, Gb):
    """Symmetric basis, Eq. (2b-symm), for v_ijkl = V_ij delta_il delta_jk:
    Sigma_ij = 2 sum_kl V_ik V_jl G_ij Gb_lk G_kl - sum_kl V_ik V_jl G_il Gb_lk G_kj."""
    b = 2.0 * np.einsum("ik,jl,ij,lk,kl->ij", V, V, G, Gb, G, optimize=False)
    x = np.einsum("ik,jl,il,lk,kj->ij", V, V, G, Gb, G, optimize=False)
    return b - x


def sigma_bubble(V, G, Gb):
    """Bubble one-liner, Eq. (bubble-contract):
    Sigma^b = 2 G o [(V x {[V x (Gb^T o G)]^T})^T]."""
    inner = V @ (Gb.T * G)
    return 2.0 * G * (V @ inner.T).T


def sigma_exchange_diag(V, G, Gb):
    """Diagonal of the exchange term, Eq. (x-contract):
    Sigma^x_ii = -{(V o G) x [Gb x (V^T o G)]}_ii."""
    return -np.diag((V * G) @ (Gb @ (V.T * G)))


# --------------------------------------------------------------------------
# GKBA reconstruction and collision integral, Sec. II
# --------------------------------------------------------------------------


def gkba_greens(T, rho):
    """Eqs. (gkba), (prop) and G^>(t,t) = -i + G^<(t,t), for t >= t_k:

    G^<(t, t_k) =  i T rho_k          G^>(t, t_k) = -i T (1 - rho_k)
    G^<(t_k, t) = -[G^<(t, t_k)]^dag  G^>(t_k, t) = -[G^>(t, t_k)]^dag
    with T = T(t, t_k) and G^<(t, t) = i rho (rho = -i G^<(t, t), Sec. II).
    Returns (Gl_tk, Gg_tk, Gl_kt, Gg_kt) batched over k.
    """
    N = rho.shape[-1]
    eye = np.eye(N)
    Gl_tk = 1j * (T @ rho)
    Gg_tk = -1j * (T @ (eye - rho))
    Gl_kt = -np.conj(np.swapaxes(Gl_tk, -1, -2))
    Gg_kt = -np.conj(np.swapaxes(Gg_tk, -1, -2))
    return Gl_tk, Gg_tk, Gl_kt, Gg_kt


def self_energies(v, T, rho, route="paper"):
    """Sigma^<(t, t_k) and Sigma^>(t, t_k) from Eq. (2bse) with the GKBA
    Green's functions (explicit i phases).  Sigma^{<>} = S(G^{<>}(t,t_k),
    G^{><}(t_k,t)).  ``route`` picks the contraction order."""
    fn = {"independent": sigma_independent, "paper": sigma_paper,
          "bruteforce": sigma_bruteforce}[route]
    Gl_tk, Gg_tk, Gl_kt, Gg_kt = gkba_greens(T, rho)
    Sl = fn(v, Gl_tk, Gg_kt)
    Sg = fn(v, Gg_tk, Gl_kt)
    return Sl, Sg


def trapezoid_weights(L, dt):
    """Trapezoid rule over t_0 .. t_{L-1}: dt/2 at both ends, dt inside;
    one point spans a zero-length interval and gets weight 0."""
    w = np.full(L, dt, dtype=np.float64)
    if L == 1:
        return np.zeros(1)
    w[0] = w[-1] = 0.5 * dt
    return w


def collision(v, rho_hist, T_hist, weights, route="paper", chunk=256):
    """First line of Eq. (collint) with the time integral as a weighted sum:

    I(t) = sum_k c_k [Sigma^>(t,t_k) G^<(t_k,t) - Sigma^<(t,t_k) G^>(t_k,t)]

    rho_hist[k] = rho(t_k), T_hist[k] = T(t, t_k), weights[k] = c_k.
    """
    L, N, _ = rho_hist.shape
    I = np.zeros((N, N), np.complex128)
    for a in range(0, L, chunk):
        b = min(L, a + chunk)
        T, rho, c = T_hist[a:b], rho_hist[a:b], weights[a:b]
        Gl_tk, Gg_tk, Gl_kt, Gg_kt = gkba_greens(T, rho)
        fn = {"independent": sigma_independent, "paper": sigma_paper,
              "bruteforce": sigma_bruteforce}[route]
        Sl = fn(v, Gl_tk, Gg_kt)
        Sg = fn(v, Gg_tk, Gl_kt)
        terms = Sg @ Gl_kt - Sl @ Gg_kt
        I += np.einsum("k,kij->ij", c, terms)
    return I


def collision_vjp(v, rho_hist, T_hist, weights, Ibar):
    """Reverse-mode derivative of ``collision`` (first line of Eq. collint).

    For a real loss L(I) and gradients written as real pairs (Xbar =
    dL/dRe X + i dL/dIm X, so that dL = Re sum conj(Xbar) dX), returns
    (rho_bar, T_bar), each L x N x N, for a given Ibar.  It is the chain rule
    through
        I   = sum_k c_k [S(Q_k, P_k^+) P_k^+ - S(P_k, Q_k^+) Q_k^+],
        P_k = T_k rho_k,  Q_k = T_k - P_k,
    where Y = S Gbar gives Sbar = Ybar Gbar^+ and Gbar-bar = S^+ Ybar, a
    conjugate transpose Gbar = X^+ gives Xbar = (Gbar-bar)^+, and each slot of
    Eq. (2bse), S_ij = sum v_irpn w_mqsj G_nm Gb_sr G_pq (holomorphic in G and
    Gb, v and w real), is differentiated by writing out its sum with the
    differentiated factor left open and the others conjugated.
    """
    L, N, _ = rho_hist.shape
    w = exchange_folded(v)
    eye = np.eye(N)
    rho_bar = np.zeros((L, N, N), np.complex128)
    T_bar = np.zeros((L, N, N), np.complex128)
    for k in range(L):
        T, rho, c = T_hist[k], rho_hist[k], weights[k]
        P = T @ rho
        Q = T - P
        Pbar = np.zeros((N, N), np.complex128)
        Qbar = np.zeros((N, N), np.complex128)
        # unit 0: -c S(P, Q^+) Q^+ ; unit 1: +c S(Q, P^+) P^+
        for G, Gb, coef, first in ((P, Q.conj().T, -c, True), (Q, P.conj().T, c, False)):
            S = sigma_independent(v, G, Gb)
            Ybar = coef * Ibar
            Sbar = Ybar @ Gb.conj().T
            Gb_bar = S.conj().T @ Ybar
            Gc, Gbc = G.conj(), Gb.conj()
            Gb_bar = Gb_bar + np.einsum("irpn,mqsj,nm,pq,ij->sr", v, w, Gc, Gc, Sbar, optimize=True)
            G_bar = (np.einsum("irpn,mqsj,sr,pq,ij->nm", v, w, Gbc, Gc, Sbar, optimize=True)
                     + np.einsum("irpn,mqsj,nm,sr,ij->pq", v, w, Gc, Gbc, Sbar, optimize=True))
            if first:
                Pbar += G_bar
                Qbar += Gb_bar.conj().T
            else:
                Qbar += G_bar
                Pbar += Gb_bar.conj().T
        rho_bar[k] = T.conj().T @ (Pbar - Qbar)
        T_bar[k] = Pbar @ rho.conj().T + Qbar @ (eye - rho).conj().T
    return rho_bar, T_bar


def collision_vjp_v(v, rho_hist, T_hist, weights, Ibar):
    """Derivative of Re sum conj(Ibar) I with respect to the Coulomb
    integrals v_abcd (each entry an independent real variable) through the
    collision integral (first line of Eq. collint).  Per unit (G, Gb) with
    adjoint Sbar of S (as in ``collision_vjp``), v enters Eq. (2bse) twice:
      v-slot:  vbar_irpn += Re sum_j conj(Sbar_ij) sum_mqs w_mqsj G_nm Gb_sr G_pq
      w-slot:  wbar_mqsj += Re sum_i conj(Sbar_ij) sum_rpn v_irpn G_nm Gb_sr G_pq
    and w_mqsj = 2 v_mqsj - v_qmsj gives vbar_abcd += 2 wbar_abcd - wbar_bacd.
    """
    L, N, _ = rho_hist.shape
    w = exchange_folded(v)
    vbar = np.zeros((N,) * 4)
    wbar = np.zeros((N,) * 4)
    for k in range(L):
        T, rho, c = T_hist[k], rho_hist[k], weights[k]
        P = T @ rho
        Q = T - P
        for G, Gb, coef in ((P, Q.conj().T, -c), (Q, P.conj().T, c)):
            Sbar = (coef * Ibar) @ Gb.conj().T
            Sc = Sbar.conj()
            vbar += np.real(np.einsum("ij,mqsj,nm,sr,pq->irpn", Sc, w, G, Gb, G, optimize=True))
            wbar += np.real(np.einsum("ij,irpn,nm,sr,pq->mqsj", Sc, v, G, Gb, G, optimize=True))
    return vbar + 2.0 * wbar - wbar.transpose(1, 0, 2, 3)



# --------------------------------------------------------------------------
# Time-linear form of the history sum (an extension; not in the paper)
#
# With the HF propagator of Eq. (prop) as a product of one-step unitaries,
# T(t_n, t_k) = Ucal_n Ucal_k^dag (Ucal_0 = 1, Ucal_{k+1} = U_k Ucal_k), the
# GKBA pieces of history point k factor as
#   P_k = T rho_k = Ucal_n X_k,          X_k    = Ucal_k^dag rho_k
#   Q_k = T - P_k = Ucal_n Xb_k,         Xb_k   = Ucal_k^dag (1 - rho_k)
#   P_k^dag = X_k^dag Ucal_n^dag,        Q_k^dag = Xb_k^dag Ucal_n^dag.
# Substituting into Eq. (2bse) moves every Ucal_n onto the indices that v
# carries (n, p with Ucal, r with conj(Ucal)) and onto the right factor of the
# first line of Eq. (collint), so that
#   I(t_n) = [sum_{npr} v_irpn (Ucal x_n Ucal x_p conj(Ucal) x_r Lambda_n)] Ucal_n^dag,
#   Lambda_n = sum_k c_k [Z(Xb_k, X_k) x_j X_k^dag - Z(X_k, Xb_k) x_j Xb_k^dag],
#   Z(A, B)_{a b c j} = sum_{mqs} w_mqsj A_am A_bq conj(B)_cs.
# Lambda_n is an N^4 tensor that changes only by the terms of new history
# points (and the trapezoid end weights), so a step costs O(N^5) whatever the
# history length.  The result equals ``collision`` up to rounding.
# --------------------------------------------------------------------------


def time_linear_factors(Ucal_k, rho_k):
    """X_k = Ucal_k^dag rho_k and Xb_k = Ucal_k^dag (1 - rho_k) (batched)."""
    Uh = np.conj(np.swapaxes(Ucal_k, -1, -2))
    X = Uh @ rho_k
    return X, Uh - X


def _z_tensor(w, A, B):
    """Z(A, B)_{abcj} = sum_{mqs} w_mqsj A_am A_bq conj(B)_cs, one index at a time."""
    y1 = np.einsum("mqsj,cs->mqcj", w, np.conj(B))
    y2 = np.einsum("bq,mqcj->mbcj", A, y1)
    return np.einsum("am,mbcj->abcj", A, y2)


def time_linear_term(v, X, Xb):
    """The t-independent contribution of one history point (weight 1):
    Z(Xb, X) x_j X^dag - Z(X, Xb) x_j Xb^dag, as Lambda[a][b][c][j']."""
    w = exchange_folded(v)
    Xh, Xbh = np.conj(X.T), np.conj(Xb.T)
    greater = np.einsum("abcj,jk->abck", _z_tensor(w, Xb, X), Xh)
    lesser = np.einsum("abcj,jk->abck", _z_tensor(w, X, Xb), Xbh)
    return greater - lesser


def time_linear_apply(v, Lam, Ucal_n):
    """I(t_n) from the accumulated tensor: move Ucal_n back onto the three v
    indices, contract with v as in Eq. (2bse), multiply by Ucal_n^dag."""
    l1 = np.einsum("na,abcd->nbcd", Ucal_n, Lam)
    l2 = np.einsum("pb,nbcd->npcd", Ucal_n, l1)
    l3 = np.einsum("rc,npcd->nprd", np.conj(Ucal_n), l2)
    S = np.einsum("irpn,nprd->id", v, l3)
    return S @ np.conj(Ucal_n.T)


def collision_time_linear(v, rho_hist, Ucal_hist, Ucal_n, weights):
    """First line of Eq. (collint) for T(t_n, t_k) = Ucal_n Ucal_k^dag via the
    accumulated tensor: Lambda = sum_k c_k term_k, I = apply(Lambda, Ucal_n)."""
    N = rho_hist.shape[-1]
    Lam = np.zeros((N,) * 4, np.complex128)
    for k in range(rho_hist.shape[0]):
        if weights[k] == 0.0:
            continue
        X, Xb = time_linear_factors(Ucal_hist[k], rho_hist[k])
        Lam += weights[k] * time_linear_term(v, X, Xb)
    return time_linear_apply(v, Lam, Ucal_n)


def hf_self_energy(v, rho):
    """(Sigma_HF)_ij = sum_kl (2 v_iklj - v_ikjl) rho_lk (Sec. II)."""
    return 2.0 * np.einsum("iklj,lk->ij", v, rho) - np.einsum("ikjl,lk->ij", v, rho)


def expm_hermitian(H, dt):
    """exp(-i dt H) for Hermitian H via its eigendecomposition."""
    lam, V = np.linalg.eigh(H)
    return (V * np.exp(-1j * dt * lam)[None, :]) @ V.conj().T


# --------------------------------------------------------------------------
# Time stepping of Eq. (equalt)
# --------------------------------------------------------------------------


class Propagation:
    """Result of ``propagate``: rho[n], I[n] (k1's collision integral at t_n),
    E_field[n], and per-step diagnostics."""

    def __init__(self, rho, I, E, energy_total, energy_corr):
        self.rho = rho
        self.I = I
        self.E = E
        self.energy_total = energy_total
        self.energy_corr = energy_corr


def _rhs(h_hf, rho, I):
    """d rho / dt from Eq. (equalt) with G^<(t,t) = i rho:
    i d(i rho)/dt = [h_HF, i rho] + (I + I^dag)  =>
    d rho/dt = -i [h_HF, rho] - (I + I^dag)."""
    return -1j * (h_hf @ rho - rho @ h_hf) - (I + I.conj().T)


def energy(h, d, E, v, rho, I):
    """E(t) = Tr[(h + E d) rho] + 1/2 Tr[Sigma_HF rho] + 1/2 Im Tr I (per spin).
    Returns (total, correlation part)."""
    one = np.trace((h + E * d) @ rho).real
    hf = 0.5 * np.trace(hf_self_energy(v, rho) @ rho).real
    ec = 0.5 * np.trace(I).imag
    return one + hf + ec, ec


def heun_step(h, v, d, rho_hist, T_row, dt, E_n, E_np1, route="paper"):
    """One Heun step t_n -> t_{n+1} of Eq. (equalt) from an explicit history.

    rho_hist[k] = rho(t_k) and T_row[k] = T(t_n, t_k) for k = 0 .. n
    (T_row[n] = 1).  With F = -i[h_HF, rho] - (I + I^dag),
    h_HF(t, rho) = h + E(t) d + Sigma_HF(rho):
      k1 = F(t_n, rho_n) over the history t_0..t_n with T(t_n, .)
      rho~ = rho_n + dt k1
      U_n = exp(-i dt (h_HF(t_n, rho_n) + h_HF(t_{n+1}, rho~)) / 2)
      T(t_{n+1}, t_k) = U_n T(t_n, t_k), T(t_{n+1}, t_{n+1}) = 1
      k2 = F(t_{n+1}, rho~) over t_0..t_n, t_{n+1} (rho~ in the last slot)
      rho_{n+1} = rho_n + dt/2 (k1 + k2)
    Returns (rho_{n+1}, I(t_n) of k1, T(t_{n+1}, .) as a list).
    """
    N = rho_hist[0].shape[0]

    def coll(rhos, Ts):
        L = len(rhos)
        if L < 2:
            return np.zeros((N, N), np.complex128)
        return collision(v, np.array(rhos), np.array(Ts), trapezoid_weights(L, dt), route)

    rho_n = rho_hist[-1]
    hhf_n = h + E_n * d + hf_self_energy(v, rho_n)
    I_n = coll(list(rho_hist), list(T_row))
    k1 = _rhs(hhf_n, rho_n, I_n)
    rho_t = rho_n + dt * k1
    hhf_t = h + E_np1 * d + hf_self_energy(v, rho_t)
    U = expm_hermitian(0.5 * (hhf_n + hhf_t), dt)
    T_next = [U @ T for T in T_row] + [np.eye(N, dtype=np.complex128)]
    I_t = coll(list(rho_hist) + [rho_t], T_next)
    k2 = _rhs(hhf_t, rho_t, I_t)
    return rho_n + 0.5 * dt * (k1 + k2), I_n, T_next


def propagate(h, v, d, rho0, dt, n_steps, E_samples, route="paper"):
    """Heun stepping of Eq. (equalt) with the GKBA collision integral: n_steps
    calls of ``heun_step`` from rho(t_0) = rho0 with E_samples[n] = E(t_n),
    n = 0 .. n_steps.  Returns a ``Propagation`` with rho[0..n_steps] and
    I[0..n_steps] (I[n] is k1's collision integral at t_n; the last one is
    evaluated without a step) and the energy of every t_n.
    """
    N = rho0.shape[0]
    rho_hist = [rho0.copy()]
    T_row = [np.eye(N, dtype=np.complex128)]
    Is, energies, ecs = [], [], []
    for n in range(n_steps + 1):
        if n == n_steps:
            I_n = np.zeros((N, N), np.complex128) if n == 0 else collision(
                v, np.array(rho_hist), np.array(T_row), trapezoid_weights(n + 1, dt), route)
        else:
            rho_next, I_n, T_row = heun_step(h, v, d, rho_hist, T_row, dt, E_samples[n],
                                             E_samples[n + 1], route)
        Is.append(I_n)
        et, ec = energy(h, d, E_samples[n], v, rho_hist[n], I_n)
        energies.append(et)
        ecs.append(ec)
        if n < n_steps:
            rho_hist.append(rho_next)

    return Propagation(np.array(rho_hist), np.array(Is), np.asarray(E_samples[: n_steps + 1]),
                       np.array(energies), np.array(ecs))


def propagate_time_linear(h, v, d, rho0, dt, n_steps, E_samples):
    """``propagate`` with the collision integrals taken from the accumulated
    tensor of ``collision_time_linear`` instead of the history sum.

    Ucal_0 = 1 and Ucal_{n+1} = U_n Ucal_n with the same U_n as ``propagate``.
    Lambda_acc holds the history points t_0 .. t_{n-1} with the weights they
    keep from then on (dt/2 for t_0, dt after it); the point t_n (k1) or the
    predicted point t_{n+1} (k2, rho~) enters with the trapezoid end weight
    dt/2, and rho_n is added to Lambda_acc once it is final.
    """
    N = rho0.shape[0]
    eye = np.eye(N, dtype=np.complex128)
    rho_hist = [rho0.copy()]
    Ucal = eye.copy()
    lam_acc = np.zeros((N,) * 4, np.complex128)
    Is, energies, ecs = [], [], []

    def term(rho, Uc):
        X, Xb = time_linear_factors(Uc, rho)
        return time_linear_term(v, X, Xb)

    for n in range(n_steps + 1):
        rho_n = rho_hist[n]
        hhf_n = h + E_samples[n] * d + hf_self_energy(v, rho_n)
        t_n = term(rho_n, Ucal)
        I_n = np.zeros((N, N), np.complex128) if n == 0 else \
            time_linear_apply(v, lam_acc + 0.5 * dt * t_n, Ucal)
        Is.append(I_n)
        et, ec = energy(h, d, E_samples[n], v, rho_n, I_n)
        energies.append(et)
        ecs.append(ec)
        if n == n_steps:
            break
        k1 = _rhs(hhf_n, rho_n, I_n)
        rho_t = rho_n + dt * k1
        hhf_t = h + E_samples[n + 1] * d + hf_self_energy(v, rho_t)
        U = expm_hermitian(0.5 * (hhf_n + hhf_t), dt)
        lam_acc = lam_acc + (0.5 * dt if n == 0 else dt) * t_n
        Ucal = U @ Ucal
        I_t = time_linear_apply(v, lam_acc + 0.5 * dt * term(rho_t, Ucal), Ucal)
        k2 = _rhs(hhf_t, rho_t, I_t)
        rho_hist.append(rho_n + 0.5 * dt * (k1 + k2))

    return Propagation(np.array(rho_hist), np.array(Is), np.asarray(E_samples[: n_steps + 1]),
                       np.array(energies), np.array(ecs))
