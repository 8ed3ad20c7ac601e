/*
 * gkba.h - C ABI of the GKBA second-Born collision-integral library (sm_103a).
 *
 * The library evaluates, on one GPU, the hot path of Tuovinen, Covito and
 * Sentef, "Efficient computation of the second-Born self-energy using
 * tensor-contraction operations" (arXiv:1905.01180):
 *
 *   Sec. III, Eq. (2bse)   second-Born self-energy
 *        Sigma_ij = 2 sum v_irpn v_mqsj G_nm Gb_sr G_pq - sum v_irpn v_mqsj G_nq Gb_sr G_pm
 *     computed as four chained N^5 contractions (one index each) with the
 *     direct and exchange terms folded into w_mqsj = 2 v_mqsj - v_qmsj;
 *   Sec. II, Eqs. (gkba), (prop)   G^<(t,t_k) = i T(t,t_k) rho_k,
 *        G^>(t,t_k) = -i T(t,t_k)(1 - rho_k), with the Hartree-Fock propagator
 *        T(t_n,t_k) = U_{n-1} ... U_k (lower limit of Eq. (prop) read as t');
 *   Sec. II, Eq. (collint) first line, time integral as a weighted sum over
 *        the history t_0 .. t_n:
 *        I(t) = sum_k c_k [Sigma^>(t,t_k) G^<(t_k,t) - Sigma^<(t,t_k) G^>(t_k,t)]
 *             = sum_k c_k [S(Q_k,P_k^+) P_k^+ - S(P_k,Q_k^+) Q_k^+],
 *        P_k = T(t,t_k) rho_k, Q_k = T(t,t_k) - P_k;
 *   Sec. II, Eq. (equalt)   d rho/dt = -i [h + E(t) d + Sigma_HF(rho), rho] - (I + I^+),
 *        (Sigma_HF)_ij = sum_kl (2 v_iklj - v_ikjl) rho_lk, advanced by Heun's
 *        method with U_n = exp(-i dt (h_HF(t_n) + h_HF(t_{n+1}))/2).
 * Also (each documented at its declaration): the diagonal and symmetric
 * interactions of Sec. III A-B (gkba_config.interaction); beyond the paper,
 * stacked batches of systems (gkba_batch_*), gradients (gkba_sigma3,
 * gkba_collision_vjp, gkba_adjoint) and the time-linear history of
 * gkba_step (gkba_config.history).
 *
 * Conventions shared by every call
 *  - Complex matrices are N x N, row-major, interleaved (re, im) doubles
 *    (the memory layout of C99 double complex / numpy complex128).
 *  - v is N^4 real doubles, v[((i*N + j)*N + k)*N + l] = v_ijkl (Eq. coulomb).
 *  - rho, I, Sigma are per spin (spin-restricted, Sec. II).
 *  - The caller owns every buffer it passes; the library copies what it keeps.
 *    "on_device" arguments say whether the caller's pointers are device
 *    pointers (nonzero) or host pointers (zero, pinned or pageable).
 *  - Calls are stream-ordered on the context's stream and synchronous at
 *    return: host outputs are written when the call returns.
 *  - Nothing aborts: every call returns a gkba_status, and gkba_last_error()
 *    gives a message.  Device-side waits are bounded and report
 *    GKBA_ETIMEOUT.  Calls on one context are not thread-safe.
 */
#ifndef GKBA_H
#define GKBA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gkba_ctx gkba_ctx; /* opaque; created by gkba_init, freed by gkba_destroy */

typedef enum {
    GKBA_OK = 0,
    GKBA_EINVAL = 1,      /* bad argument: size, NULL, non-Hermitian input, asymmetric v, non-finite data */
    GKBA_ENOMEM = 2,      /* device or host allocation failed */
    GKBA_ECUDA = 3,       /* a CUDA runtime/driver call failed (message has the CUDA error) */
    GKBA_ESTATE = 4,      /* call not valid in the current state (e.g. history full) */
    GKBA_ETIMEOUT = 5,    /* a device-side wait ran past its limit; results are invalid */
    GKBA_ENUMERIC = 6,    /* non-finite values produced */
    GKBA_EUNSUPPORTED = 7 /* valid request that the library does not implement */
} gkba_status;

typedef enum {
    GKBA_FP64 = 0,       /* every contraction in FP64 on the CUDA cores */
    GKBA_SPLIT_TF32 = 1, /* contractions on tcgen05 tensor cores: FP32 data,
                            3 TF32 products (hi*hi + hi*lo + lo*hi), FP32
                            accumulation in short tensor-memory windows (see
                            gkba_config.acc_window), added on the CUDA cores and
                            across the last contraction's K ranges in FP64;
                            P/Q, T recursion, I history sum and rho update stay FP64 */
    GKBA_SPLIT_TF32_ACC = 2 /* as GKBA_SPLIT_TF32; for N > 48, where the first three
                            contractions accumulate a whole tile in one tensor-memory
                            accumulator, the correction products go to a second
                            accumulator so that only hi*hi truncates at the scale of
                            the result (about 15 % slower there; identical to
                            GKBA_SPLIT_TF32 for N <= 48) */
} gkba_precision;

typedef enum {
    GKBA_V_GENERAL = 0,   /* v: N^4 real Coulomb integrals v_ijkl (Sec. III C) */
    GKBA_V_DIAGONAL = 1,  /* v: N reals U_i, v_ijkl = U_i d_ij d_ik d_il (Sec. III A,
                             Hubbard-like on-site interaction); Sigma by Eq. (2b-diag) */
    GKBA_V_SYMMETRIC = 2  /* v: N*N real symmetric V_ij, v_ijkl = V_ij d_il d_jk
                             (Sec. III B, density-density interaction); Sigma by
                             Eq. (2b-symm), bubble and exchange */
} gkba_interaction;

typedef enum {
    GKBA_HISTORY_SUM = 0,        /* each collision integral of gkba_step sums Eq. (collint)
                                    over the whole history: O(L N^5) per step */
    GKBA_HISTORY_TIME_LINEAR = 1 /* gkba_step keeps the history sum as one N^4 accumulator
                                    (T(t_n,t_k) = Ucal_n Ucal_k^+ factored out; an extension,
                                    not in the paper): O(N^5) per step at any history
                                    length, the same result up to rounding.  General v
                                    only; 2 x 16 N^4 bytes more device memory.  On a
                                    split-TF32 context the contractions (terms, their
                                    accumulation over j, the three back-transforms and
                                    stage S4) run on the tensor cores and the
                                    accumulator stays FP64 */
} gkba_history;

typedef struct {
    int N;             /* basis size, 1 <= N <= 128 (tensor-core modes: N <= 96) */
    double dt;         /* time step delta (> 0) */
    int max_steps;     /* history capacity: t_0 .. t_{max_steps} (>= 0) */
    int precision;     /* gkba_precision */
    void* cuda_stream; /* cudaStream_t to run on; NULL = the library creates one */
    size_t workspace_bytes; /* cap on the contraction workspace (0 = default 64 GiB, at most
                               85 % of the free device memory);
                               the batch of (t_k, component) units is sized to fit */
    int device;        /* CUDA device ordinal (-1 = current device) */
    int timing;        /* nonzero: time every contraction kernel with CUDA events
                          (see gkba_get_stats) */
    int acc_window;    /* split-TF32 modes: K length (8 or 16; 32 behaves as 16;
                          0 = 32) of one tensor-memory accumulation window of the
                          first three contractions for N <= 48.  The tensor core
                          truncates its FP32 accumulator additions toward zero, a
                          coherent bias that grows with the accumulation length,
                          so those contractions (for N <= 48) and the last one
                          (K = N^3, always 32-wide windows) accumulate only a
                          window of K in tensor memory before the epilogue adds it
                          in FP32 registers (Kahan-compensated in the last one);
                          inside a window the correction products come first and
                          hi*hi last, so only the hi*hi MMAs truncate at the scale
                          of the result.  For N > 48 the first three
                          contractions accumulate a tile's whole K (96 or 192). */
    int interaction;   /* gkba_interaction: form of the v argument of gkba_init;
                          GKBA_V_DIAGONAL / GKBA_V_SYMMETRIC need precision GKBA_FP64 */
    int history;       /* gkba_history: how gkba_step evaluates the history sum
                          (GKBA_HISTORY_TIME_LINEAR needs GKBA_V_GENERAL, else
                          GKBA_EUNSUPPORTED) */
} gkba_config;

/* Per-kernel-class counters (see gkba_get_stats). */
typedef struct {
    const char* name;       /* kernel class name */
    long long launches;     /* launches since the last reset */
    double ms;              /* summed CUDA-event time (only when cfg.timing) */
    double flops;           /* summed algorithmic flops of those launches */
    double bytes;           /* summed algorithmic (compulsory) DRAM bytes */
} gkba_kernel_stat;

/*
 * gkba_init - create a context for the model of Sec. II, Eq. (hamiltonian).
 *   h    N*N complex Hermitian one-body matrix h_ij (Eq. onebody), no field
 *   v    the interaction, by cfg->interaction:
 *          GKBA_V_GENERAL   N^4 real Coulomb integrals with the 8-fold symmetry
 *                           of Eq. (symmetries)
 *          GKBA_V_DIAGONAL  N reals U_i (v_ijkl = U_i d_ij d_ik d_il)
 *          GKBA_V_SYMMETRIC N*N real symmetric V_ij (v_ijkl = V_ij d_il d_jk)
 *   d    N*N complex Hermitian dipole matrix; the field enters as h + E(t) d
 *   rho0 N*N complex Hermitian initial density matrix rho(t_0) (per spin)
 * Builds the contraction layouts of v and w = 2v - v_exch on the device (the
 * diagonal and symmetric forms are expanded to v_ijkl for the mean field;
 * their self-energy uses Eq. (2b-diag) / Eq. (2b-symm) directly), and the
 * history store (rho_0 = rho0, T(t_0,t_0) = 1).  Returns GKBA_EINVAL for
 * non-Hermitian h/d/rho0, a v that breaks Eq. (symmetries) (tolerance 1e-10
 * relative), an asymmetric V, a structured interaction with a split-TF32
 * precision, non-finite data or bad sizes; *out is NULL on failure.
 */
gkba_status gkba_init(gkba_ctx** out, const gkba_config* cfg, const double* h, const double* v,
                      const double* d, const double* rho0, int inputs_on_device);

/*
 * gkba_sigma - second-Born self-energy S(G, Gb) of Eq. (2bse) for n_units
 * independent pairs (G = G^{<>}(t,t'), Gb = G^{><}(t',t), Sec. III notation).
 *   G, Gbar  n_units * N*N complex each
 *   S_out    n_units * N*N complex: S_u = Eq. (2bse) evaluated on (G_u, Gbar_u)
 * Runs on the context's precision path.
 */
gkba_status gkba_sigma(gkba_ctx* ctx, int n_units, const double* G, const double* Gbar,
                       double* S_out, int on_device);

/*
 * gkba_collision - collision integral I(t) of Eq. (collint), first line, for
 * an explicit history of L >= 1 points t_0 .. t_{L-1} = t:
 *   rho_hist  L*N*N complex: rho(t_k)
 *   T_hist    L*N*N complex: HF propagator T(t, t_k) of Eq. (prop)
 *             (T_hist[L-1] is normally the identity)
 *   weights   L doubles c_k, or NULL for the trapezoid rule with cfg.dt
 *             (dt/2 at both ends, dt inside; L == 1 gives I = 0)
 *   I_out     N*N complex: I(t) = sum_k c_k [S(Q_k,P_k^+) P_k^+ - S(P_k,Q_k^+) Q_k^+]
 * All of P/Q reconstruction, the contractions, the products with P^+/Q^+ and
 * the FP64 history sum run on the device.  The equation of motion uses
 * I + I^+ (the second line of Eq. (collint) is the adjoint of the first).
 */
gkba_status gkba_collision(gkba_ctx* ctx, int L, const double* rho_hist, const double* T_hist,
                           const double* weights, double* I_out, int on_device);

/*
 * gkba_step - one Heun step t_n -> t_{n+1} of Eq. (equalt) with the field
 * samples E_n = E(t_n), E_np1 = E(t_{n+1}):
 *   k1 = F(t_n, rho_n) over the history t_0..t_n, rho~ = rho_n + dt k1,
 *   U_n = exp(-i dt (h_HF(t_n,rho_n) + h_HF(t_{n+1},rho~))/2),
 *   T(t_{n+1},t_k) = U_n T(t_n,t_k), k2 = F(t_{n+1}, rho~) over t_0..t_{n+1},
 *   rho_{n+1} = rho_n + dt/2 (k1 + k2),  F = -i[h_HF, rho] - (I + I^+).
 * Outputs (host pointers, each may be NULL):
 *   rho_out   N*N complex: rho_{n+1}
 *   I_out     N*N complex: I(t_n) of k1
 *   diag_out  4 doubles at t_n: {Tr rho_n, E_total, E_corr, Re Tr I_n} with
 *             E_total = Tr[(h+E_n d) rho_n] + 1/2 Tr[Sigma_HF rho_n] + E_corr,
 *             E_corr = 1/2 Im Tr I_n (per spin).
 * With cfg.history = GKBA_HISTORY_TIME_LINEAR both collision integrals come
 * from the accumulator (time_linear.cu): k1's adds rho_n's term with weight
 * dt/2 to the points t_0..t_{n-1}, k2's rho~'s term; rho_n's term then joins
 * the accumulator with its final weight.
 * GKBA_ESTATE when the history is full (n == cfg.max_steps), or in the
 * time-linear mode after a failed step (gkba_set_history restores a state).
 */
gkba_status gkba_step(gkba_ctx* ctx, double E_n, double E_np1, double* rho_out, double* I_out,
                      double* diag_out);

/*
 * gkba_set_history - replace the stepper state (checkpoint restore): the
 * history t_0 .. t_n with rho_hist[k] = rho(t_k) and T_hist[k] = T(t_n, t_k),
 * k = 0..n (n + 1 points; T_hist[n] should be the identity).
 * GKBA_EINVAL when n > cfg.max_steps.  In the time-linear mode T_hist[n]
 * must be the identity (max deviation 1e-12, else GKBA_EINVAL) and the
 * accumulator is rebuilt from the n points before t_n with Ucal_k^+ =
 * T_hist[k] (O(n N^5) once).
 */
gkba_status gkba_set_history(gkba_ctx* ctx, int n, const double* rho_hist, const double* T_hist,
                             int on_device);

/*
 * gkba_get_history - copy the stepper state out (checkpoint save): n and,
 * when the pointers are non-NULL, rho_hist / T_hist with (n+1)*N*N complex
 * each (host pointers).
 */
gkba_status gkba_get_history(const gkba_ctx* ctx, int* n, double* rho_hist, double* T_hist);

/* gkba_get_state - current step index n and rho(t_n) (host, may be NULL). */
gkba_status gkba_get_state(const gkba_ctx* ctx, int* n, double* rho);

/*
 * gkba_mean_field - (Sigma_HF)_ij = sum_kl (2 v_iklj - v_ikjl) rho_lk (Sec. II)
 * for one N*N complex rho; output N*N complex.
 */
gkba_status gkba_mean_field(gkba_ctx* ctx, const double* rho, double* sigma_hf, int on_device);

/*
 * gkba_adjoint - reverse-mode gradient through the Heun stepper and the
 * collision integrals of the n steps taken since gkba_init (or
 * gkba_set_history(0, ...)): the discrete adjoint of gkba_step as
 * implemented, for a loss L(rho(t_n)) of the final state.
 *   rho_bar_final N*N complex (host): dL/dRe rho(t_n) + i dL/dIm rho(t_n)
 *                 (for L = Tr[d rho(t_n)], d Hermitian: rho_bar_final = d)
 *   E_bar         n+1 doubles (host): dL/dE_k for the field samples of the
 *                 steps (E(t_k) as passed to step k and to step k-1 as E_np1)
 *   rho0_bar      N*N complex (host, may be NULL): dL/drho(t_0), same convention
 * gkba_step records the predictor state and the propagator of every step;
 * the backward pass un-propagates the T(t, t_k) rows with U_n^+ (U_n unitary),
 * so no checkpoints are needed.  Each step costs two collision-integral
 * adjoints (about eight collision integrals) plus N^3 work, including the
 * Frechet derivative of the exponential (a 2N x 2N exponential).
 *   v_bar         N^4 doubles (host, may be NULL): dL/dv_abcd through every
 *                 collision integral and mean field of the trajectory (each
 *                 entry an independent real variable).  On a split-TF32
 *                 context the two slot contractions read the FP32 X3 of the
 *                 tensor-core chain (the w slot runs the chain once more on
 *                 the omega layout of v) and sum in FP64.
 * GKBA_EUNSUPPORTED for a structured interaction or a trajectory started by
 * gkba_set_history(n > 0).
 */
gkba_status gkba_adjoint(gkba_ctx* ctx, const double* rho_bar_final, double* E_bar, double* rho0_bar,
                         double* v_bar);

/*
 * gkba_get_stats - kernel counters since the last reset: fills up to
 * max_stats entries and returns their number in *n_stats; *total_launches is
 * the number of library kernel launches.  reset != 0 clears the counters
 * after reading.
 */
gkba_status gkba_get_stats(gkba_ctx* ctx, gkba_kernel_stat* stats, int max_stats, int* n_stats,
                           long long* total_launches, int reset);

/*
 * gkba_sigma_noalloc - the FP64 self-energy of gkba_sigma (Eq. (2bse) for
 * n_units pairs G, Gbar) without a context and without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory, such as code that runs while a CUDA graph is
 * being captured, a host framework that owns every allocation on the device,
 * or a service that runs under a fixed memory budget.
 *   N        basis size, 1 <= N <= 24 (larger N is rejected with GKBA_EINVAL)
 *   v        device pointer, N^4 real doubles v_ijkl (Eq. coulomb layout)
 *   G, Gbar  device pointers, n_units * N*N complex each
 *   S_out    device pointer, n_units * N*N complex
 *   cuda_stream  cudaStream_t to enqueue on (NULL = the legacy default stream)
 *   err, err_len optional caller buffer for a message on failure
 * Scratch is a 32 MiB file-scope __device__ array that every GPU which loads
 * the library holds until the process exits; no cudaMalloc, cudaFree or other
 * allocating routine is called.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress, with the device current);
 * make that first call before any stream capture.  All calls share the
 * array, so calls that overlap on the GPU (other streams, other threads)
 * race with each other: serialise them.  Every scratch element a call reads
 * is written earlier in the same call, so nothing left by a previous call
 * leaks into the result.  The call only enqueues work: S_out is valid after
 * the stream is synchronised.  Launch errors return GKBA_ECUDA (checked after
 * every chunk of units, so a failed launch stops the rest); a CUDA error that
 * is already pending from earlier work on the calling thread is reported as
 * GKBA_ECUDA before anything is launched and left in place.
 */
gkba_status gkba_sigma_noalloc(int N, int n_units, const double* v, const double* G,
                               const double* Gbar, double* S_out, void* cuda_stream, char* err,
                               size_t err_len);

/*
 * gkba_sigma3 - the trilinear form behind Eq. (2bse) with its two G slots
 * separated: S3(A, B, C)_ij = sum v_irpn w_mqsj A_nm B_sr C_pq, so that
 * S(G, Gb) = S3(G, Gb, G).  n_units triples of N*N complex matrices; runs on
 * the context's precision path (general interaction only: GKBA_EUNSUPPORTED
 * otherwise).  Used by the adjoint: every derivative of S is an S3 value.
 */
gkba_status gkba_sigma3(gkba_ctx* ctx, int n_units, const double* A, const double* B,
                        const double* C, double* S_out, int on_device);

/*
 * gkba_collision_vjp - adjoint (vector-Jacobian product) of gkba_collision:
 * for a real loss L(I) and I_bar = dL/dRe I + i dL/dIm I (N*N complex),
 * returns rho_bar and T_bar (L*N*N complex each, same convention) for the
 * same history and weights (NULL: trapezoid).  The derivative of each slot of
 * Eq. (2bse) is evaluated as an S3 value on the context's precision path,
 * chained through P_k = T_k rho_k, Q_k = T_k - P_k and the products with
 * P_k^+ / Q_k^+ in FP64.  General interaction only (GKBA_EUNSUPPORTED
 * otherwise).  Costs about four collision integrals.
 *   v_bar  N^4 doubles or NULL: dL/dv_abcd, every entry an independent real
 *          variable (chain it to a parametrization of v, e.g. Coulomb
 *          factors, on the caller's side); one more chain (S1-S3) and
 *          two slot contractions per unit, on either precision path.
 */
gkba_status gkba_collision_vjp(gkba_ctx* ctx, int L, const double* rho_hist, const double* T_hist,
                               const double* weights, const double* I_bar, double* rho_bar,
                               double* T_bar, double* v_bar, int on_device);

/*
 * Stacked batches of systems: many systems of uneven basis size and history
 * length advanced together.  The (t_k, component) units of all systems of the
 * same N are stacked (per system only the w and v layouts differ, and the
 * kernels select them per unit), and the groups of different N share each
 * stage launch; the per-system N^2 / N^3 work (mean field, propagator, Heun
 * update) runs per system.
 *
 * gkba_batch_create - ctxs: n_ctx distinct contexts made by gkba_init with
 *   the same split-TF32 precision and acc_window, the general interaction and
 *   the same device.  They stay owned by the caller and must outlive the
 *   batch; during gkba_batch_step every member runs on the batch's stream.
 *   workspace_bytes caps the stacked workspaces of all groups together (0 =
 *   64 GiB, each group at most 85 % of the free device memory).  Returns
 *   GKBA_EINVAL for other contexts, GKBA_ENOMEM when a group's workspace does
 *   not fit.
 * gkba_batch_step - one Heun step (as gkba_step) of every member; E_n and
 *   E_np1 hold n_ctx field samples; rho_out and diag_out are arrays of n_ctx
 *   host pointers (the arrays or their entries may be NULL).  A member whose
 *   history is full fails the whole call with GKBA_ESTATE before any work.
 * gkba_batch_last_error - message of the last failing batch call (NULL batch:
 *   the last failed gkba_batch_create).
 */
typedef struct gkba_batch gkba_batch;
gkba_status gkba_batch_create(gkba_batch** out, gkba_ctx* const* ctxs, int n_ctx,
                              size_t workspace_bytes);
gkba_status gkba_batch_step(gkba_batch* batch, const double* E_n, const double* E_np1,
                            double* const* rho_out, double* const* diag_out);
const char* gkba_batch_last_error(const gkba_batch* batch);
void gkba_batch_destroy(gkba_batch* batch);

/*
 * How a stacked batch runs (the paper has no counterpart; properties of this
 * implementation).
 *
 * Every round of gkba_batch_step's collision integrals puts the batches of
 * all basis-size groups into one launch per contraction stage: the launch's
 * CTA pairs are split between the groups in proportion to their estimated
 * cost, each group with its own tensor maps and parameters.
 *
 * gkba_batch_set_options - use_graph = 1: each gkba_batch_step captures its
 *   device work (all members, both collision integrals) on the batch's stream
 *   and launches it as one CUDA graph; the previous step's executable graph is
 *   updated in place when the step's launch sequence kept its shape, else
 *   instantiated anew.  use_graph = 0 (default): launched one by one.  The
 *   results are the same either way (same kernels, same order).
 * gkba_batch_autotune - chooses per group, by timing contraction rounds on
 *   the device over units built from the members' current histories (it reads
 *   them, changes no member state): the K length of a stage-S4 work item
 *   (4096, 8192 or 16384), the accumulation window of the windowed stage
 *   kernel (acc_window 8 or 16; both keep the split-TF32 tolerance) and the
 *   units per round (from the workspace's down by halves while each stage
 *   launch keeps two 256-row tiles per CTA pair), coordinate by coordinate,
 *   fastest per unit.  The choices stay with the batch and are returned per
 *   group (arrays of at least 8 entries, NULL to skip): N, units per round,
 *   acc_window, S4 item K and the measured microseconds per unit.
 */
gkba_status gkba_batch_set_options(gkba_batch* batch, int use_graph);
gkba_status gkba_batch_autotune(gkba_batch* batch, int* n_groups, int* N, int* units,
                                int* acc_window, int* s4_item_k, double* us_per_unit);

/*
 * gkba_selftest_timeout - failure detection without a GPU fault: runs a
 * 2-CTA kernel whose even CTA waits, with the bounded wait of the contraction
 * kernels and a limit of limit_ms (0 < limit_ms <= 1000), on a barrier that
 * nothing arrives at; the odd CTA must leave early on its peer's abort flag.
 * Returns GKBA_ETIMEOUT (the error word the expired wait wrote, read as after
 * every call), elapsed_ms[0..1] (may be NULL) = each CTA's time in its wait.
 * The context stays usable.
 */
gkba_status gkba_selftest_timeout(gkba_ctx* ctx, double limit_ms, double* elapsed_ms);

/*
 * gkba_measure_tf32_mma - measures the tensor-pipe rate that bounds the
 * split-TF32 contraction (the roofline denominator; the paper has no
 * counterpart): every pair of SMs issues `iters` x 4 back-to-back
 * tcgen05.mma.cta_group::2.kind::tf32 instructions of the stage kernels'
 * shape (M = 256, N = 192, K = 8, A in tensor memory, B in shared memory,
 * zero operands) with nothing else running on the SM; the launch is timed
 * with CUDA events on the context's stream after a shorter warm-up launch.
 *   iters   16 ... 1e8 (1e5 takes about 20 ms on a GB300)
 *   tflops  out: 2 x 256 x 192 x 8 flops per MMA over the measured time
 */
gkba_status gkba_measure_tf32_mma(gkba_ctx* ctx, int iters, double* tflops);

/* Message for the last failing call on ctx (or the last failed gkba_init when ctx is NULL). */
const char* gkba_last_error(const gkba_ctx* ctx);

/* Free every device and host resource of ctx (NULL is a no-op). */
void gkba_destroy(gkba_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GKBA_H */
