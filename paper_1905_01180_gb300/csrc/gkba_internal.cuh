// gkba_internal.cuh - context, kernel classes and launch helpers shared by the
// translation units of libgkba (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gkba.h"

namespace gkba {

// z-ranges of the two-pass split-K reduction of the last contraction
constexpr int kReduceSplit = 16;

// Kernel classes counted by gkba_get_stats.  The algorithmic flops and bytes
// of each launch are added at launch time (see the per-class comments in
// gkba_api.cu).
enum KernelClass : int {
    K_W1 = 0,    // S1: X1 = w x_s Gbar          (real x complex, 4 N^5 / unit)
    K_W2,        // S2: X2 = G x_q X1            (complex x complex, 8 N^5 / unit)
    K_W3,        // S3: X3 = G x_m X2            (complex x complex, 8 N^5 / unit)
    K_FIN,       // S4: S = v . X3 over (n,r,p)  (real x complex, 4 N^5 / unit, split-K)
    K_PREP,      // P/Q reconstruction and per-unit operand forms
    K_RED,       // split-K reduction, S.Gbar products, weighted history sum
    K_STEP,      // mean field, commutators, expm, T recursion, Heun update
    K_TL,        // time-linear history: accumulator GEMM and update, back-transforms
    K_COUNT
};

extern const char* kKernelClassNames[K_COUNT];

// NVTX range for profilers (a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct TimedLaunch {
    int cls;
    cudaEvent_t a, b;
};

}  // namespace gkba

struct gkba_ctx {
    // configuration
    int N = 0;          // basis size
    int Np = 0;         // padded basis for the tensor-core path (multiple of 16)
    double dt = 0.0;
    int max_steps = 0;
    int prec = GKBA_FP64;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t ws_cap = 0;
    bool timing = false;
    int num_sms = 0;
    int pair_clusters = 0;  // co-resident 2-CTA clusters of the stage kernel
    int fin_pair_clusters = 0;  // same for the S4 kernel
    int kind = GKBA_V_GENERAL;  // gkba_interaction
    // Stacked batches of several systems (gkba_batch): wS32 / vKhi / vKlo hold
    // nsys systems' layouts and unit_sys (device) maps each unit to its system.
    const int* unit_sys = nullptr;
    int nsys = 1;
    double* vm = nullptr;       // U (N) or V (N*N) of a structured interaction
    int history = GKBA_HISTORY_SUM;  // gkba_history
    int acc_window = 32;

    // model on the device
    double2* h = nullptr;   // N*N
    double2* d = nullptr;   // N*N
    double* v = nullptr;    // N^4, v[i][j][k][l]
    double* hfK = nullptr;  // N^4, hfK[(i*N+j)*N*N + l*N + k] = 2 v_iklj - v_ikjl

    // FP64 contraction operands (natural N)
    double* wS64 = nullptr;  // [j][m][q][s] = w_mqsj
    double* vK64 = nullptr;  // [i][n][r][p] = v_irpn

    // split-TF32 contraction operands (padded Np, zero padding)
    float* wS32 = nullptr;    // raw FP32 [j][m][q][s]
    float* vO32 = nullptr;    // omega layout of v, FP32 [i][n][p][r] (dL/dv, made on demand)
    float* xsw = nullptr;     // row weights of the slot contractions (dL/dv, time-linear)
    size_t xsw_bytes = 0;
    float* vKhi = nullptr;    // TF32-rounded [i][(n,r,p)]
    float* vKlo = nullptr;    // TF32-rounded remainder

    // history store: slot k holds rho(t_k) and T(t_n, t_k)
    int n = 0;
    double2* rho_hist = nullptr;  // (max_steps + 2) * N*N
    double2* T_a = nullptr;       // current T row
    double2* T_b = nullptr;       // next T row (double buffer)

    // stepper scratch (N*N complex each unless noted)
    double2* hhf_n = nullptr;
    double2* hhf_t = nullptr;
    double2* k1 = nullptr;
    double2* k2 = nullptr;
    double2* Ia = nullptr;       // I(t_n)
    double2* Ib = nullptr;       // I(t_{n+1}) of the corrector
    double2* U = nullptr;
    double2* ex0 = nullptr;      // expm work
    double2* ex1 = nullptr;
    double2* ex2 = nullptr;
    double2* tmp0 = nullptr;
    double2* tmp1 = nullptr;
    double* dscal = nullptr;     // device scalars: [0..7] diagnostics, [8] expm norm
    int* dint = nullptr;         // device ints: [0] expm squarings, [1] error word
    double* hdiag = nullptr;     // pinned host copy of diagnostics

    // contraction workspace (lazily sized)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int ub = 0;                  // units per batch
    int ub_cap = 0;              // units the workspace was sized for
    int ub_limit = 0;            // stacked batches: units per round chosen by the autotuner (0: ub)
    int fin_kw = 4096;           // K length of an S4 work item (a multiple of 4096)
    // sub-buffers inside ws
    void* X13 = nullptr;
    size_t x13_bytes = 0;
    void* X2 = nullptr;
    void* part = nullptr;
    size_t part_bytes = 0;
    double2* PQ = nullptr;       // P and Q for ub/2 history points: 2 * (ub/2) * N*N
    void* formsB1 = nullptr;     // per-unit B operand of S1
    void* formsG = nullptr;      // per-unit B operand of S2/S3
    void* formsG3 = nullptr;     // per-unit B operand of S3 when its slot differs (sep_A)
    double2* vjp = nullptr;      // adjoint scratch: 10 blocks of vjp_units N*N units
    int vjp_units = 0;
    // trajectory record of gkba_step for the adjoint (steps adj_from .. n-1)
    double2* rhot_hist = nullptr;  // rho~ (predictor) of each step
    double2* U_hist = nullptr;     // U_n of each step
    std::vector<double> E_a, E_b;  // E(t_n), E(t_{n+1}) passed to each step
    int adj_from = 0;              // first recorded step (0 after gkba_init)
    double2* adj_ws = nullptr;     // backward-pass buffers
    size_t adj_ws_bytes = 0;
    double* vomega = nullptr;      // v in the [i][n][p][r] layout (w-slot chain of dL/dv)
    double* vgrad = nullptr;       // dL/dv accumulators: vslot, wslot (N x N^3 each), natural N^4
    bool sep_A = false;          // contraction of S3(A, B, C): S3 reads formsG3
    double2* Mb = nullptr;       // per-unit Gbar (= the right factor of S.Gbar), ub * N*N
    double* coef = nullptr;      // per-unit weight (+-c_k), ub
    double2* Su = nullptr;       // per-unit S, ub * N*N
    double2* Yu = nullptr;       // per-unit coef * S . Gbar, ub * N*N
    double2* red_tmp = nullptr;  // split-K reduction scratch: kReduceSplit * ub * N*N

    // time-linear history (GKBA_HISTORY_TIME_LINEAR): T(t_n, t_k) = Ucal_n Ucal_k^+
    double* tl_acc = nullptr;    // Lambda_acc, 2 N^4 doubles, [j][n][r][c][p]
    double* tl_s = nullptr;      // Lambda of one collision / back-transform scratch, same size
    double2* tl_W = nullptr;     // W_n = Ucal_n^+ (N*N)
    double2* tl_Wn = nullptr;    // W_{n+1} during a step
    double* tl_uf = nullptr;     // real forms of Ucal and conj(Ucal), 2 x (2N)^2
    bool tl_broken = false;      // a step failed after Lambda_acc changed

    // caller-buffer staging for host-pointer calls
    void* stage = nullptr;
    size_t stage_bytes = 0;

    // statistics
    long long launches = 0;
    long long cls_launches[gkba::K_COUNT] = {};
    double cls_ms[gkba::K_COUNT] = {};
    double cls_flops[gkba::K_COUNT] = {};
    double cls_bytes[gkba::K_COUNT] = {};
    std::vector<gkba::TimedLaunch> pending;
    std::vector<cudaEvent_t> event_pool;

    std::string err;
};

namespace gkba {

// Record an error message on the context and return the status.
gkba_status fail(gkba_ctx* c, gkba_status st, const char* fmt, ...);

// The contraction runs on the tensor cores (split-TF32 modes) or in FP64.
inline bool tensor_core_path(const gkba_ctx* c) { return c->prec != GKBA_FP64; }

// Check a CUDA runtime call; on failure record it and return GKBA_ECUDA.
#define GKBA_CUDA(ctx, call)                                                              \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return ::gkba::fail((ctx), GKBA_ECUDA, "%s failed: %s (%s:%d)", #call,        \
                                cudaGetErrorString(e_), __FILE__, __LINE__);              \
    } while (0)

#define GKBA_TRY(expr)                 \
    do {                               \
        gkba_status s_ = (expr);       \
        if (s_ != GKBA_OK) return s_;  \
    } while (0)

// Launch bookkeeping: count a launch of class cls with its algorithmic flops and
// bytes, and (when timing) bracket it with events.  Usage:
//   auto t = launch_begin(ctx, K_W2, flops, bytes); kernel<<<...>>>(...); launch_end(ctx, t);
struct LaunchToken {
    int cls;
    cudaEvent_t a;
};
LaunchToken launch_begin(gkba_ctx* c, int cls, double flops, double bytes);
gkba_status launch_end(gkba_ctx* c, LaunchToken t);
// Fold finished event pairs into the per-class times (synchronises the stream).
gkba_status harvest_timing(gkba_ctx* c);

// ---- FP64 kernels (fp64_kernels.cu) ---------------------------------------

// Output scatter of a stage GEMM: row = (a*Db + b)*Dx + x, col = c*Dy + y,
// offset = a*SA + b*SB + x*SX + c*SC + y*SY.
struct StageMap {
    long long SA, SB, SX, SC, SY;
    int Dx, Db, Dy;
    long long XB = 0;  // nonzero: x enters as (x / 32) * XB + x % 32 (K-blocked layout)
};

// D[z][row][col] = sum_k A[z][row*lda + k] * B[z][col*ldb + k] (FP64, K-major).
// Mode 0: z indexes units (per-z strides sAz, sBz, sOz; K = Ktot).
// Mode 1: z indexes K-chunks of length Kc (split-K; out += z*sOz).
gkba_status gemm64_stage(gkba_ctx* c, int cls, const double* A, long long lda, long long sAz,
                         const double* B, long long ldb, long long sBz, double* out,
                         long long sOz, int M, int Nc, long long Ktot, int nz, int splitk,
                         long long Kc, StageMap map, double flops, double bytes);

// Complex batched GEMM: C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b] (+ I if add_identity),
// op = 'N' or 'C' (conjugate transpose); square n x n matrices, per-batch strides in elements.
// K chunk (a multiple of the stage GEMM's K slice) of a split-K stage GEMM of
// M x Nc outputs so that its launch fills about one wave of resident blocks,
// with at most max_chunks chunks.
long long gemm64_splitk_chunk(gkba_ctx* c, int M, int Nc, long long K, long long max_chunks);
gkba_status zgemm_batched(gkba_ctx* c, int cls, int n, char opA, char opB, double2 alpha,
                          const double2* A, long long sA, const double2* B, long long sB,
                          double2 beta, double2* C, long long sC, int batch, int add_identity);

// Stepper helpers.
gkba_status mean_field(gkba_ctx* c, const double2* rho, double2* out);
gkba_status h_hf(gkba_ctx* c, double E, const double2* rho, double2* out);  // h + E d + Sigma_HF
gkba_status rhs(gkba_ctx* c, const double2* hhf, const double2* rho, const double2* I,
                double2* out);  // -i[hhf, rho] - (I + I^+)
gkba_status expm_step(gkba_ctx* c, const double2* hA, const double2* hB,
                      double2* U);  // U = exp(-i dt (hA + hB)/2)
gkba_status axpy_c(gkba_ctx* c, double2* y, const double2* x, const double2* z, double a,
                   double b, int n);  // y = a*x + b*z (elementwise, n complex)
gkba_status set_identity(gkba_ctx* c, double2* A, int count);  // count N*N identities
gkba_status diagnostics(gkba_ctx* c, double E_n, const double2* rho, const double2* I,
                        double* out4);  // device out4 = {Tr rho, E_tot, E_c, ReTrI}

// Contraction driver: I_out (device, N*N) = collision over L history points.
gkba_status collision_dev(gkba_ctx* c, int L, const double2* rho, const double2* T,
                          const double* weights_dev, double2* I_out);
// S_out (device) for n_units (G, Gbar) pairs (device).
gkba_status sigma_dev(gkba_ctx* c, int n_units, const double2* G, const double2* Gb,
                      double2* S_out);

// Contraction backends (one batch of units whose forms are already built).
gkba_status contract_batch_fp64(gkba_ctx* c, int nb);
gkba_status contract_batch_tf32(gkba_ctx* c, int nb);
// Structured interaction (GKBA_V_DIAGONAL / GKBA_V_SYMMETRIC): S(G_u, Gb_u) into Su.
gkba_status contract_structured(gkba_ctx* c, int nb, const double2* G, const double2* Gb);
gkba_status tf32_prepare_model(gkba_ctx* c);  // build wS32, vKhi, vKlo
gkba_status tf32_prepare_vgrad(gkba_ctx* c);  // build vO32
gkba_status tf32_chain_omega(gkba_ctx* c, int nb);
gkba_status vbar_slot_tf32(gkba_ctx* c, int nb, const double2* Sbar, int transposeS, double* out);
gkba_status tl_terms_tf32(gkba_ctx* c, int nb, const double2* Gb, int k0, double w_first,
                          double w_rest, double* D);
gkba_status tl_apply_tf32(gkba_ctx* c, const double2* W, const double* lam);
// Several contexts' batches in one launch per stage (forms built; shared stream).
gkba_status contract_batch_tf32_multi(gkba_ctx* const* cs, const int* nbs, int n);
gkba_status fp64_prepare_model(gkba_ctx* c);  // build wS64, vK64, hfK

// Per-unit operand forms for a batch: units u = 0..nb-1 given (G_u, Gb_u) pointers
// laid out as G = base_G + u*N*N etc.  Writes formsB1/formsG (precision-specific),
// Mb (= Gb) and coef.
gkba_status build_forms(gkba_ctx* c, int nb, const double2* G, long long sG,
                        const double2* Gb, long long sGb, int gb_conj_of_other);
gkba_status build_forms_gkba(gkba_ctx* c, int k0, int nk, int L, const double2* rho,
                             const double2* T, const double* w);
gkba_status reduce_batch(gkba_ctx* c, int nb, double2* I_acc, double2* S_out);
gkba_status units_from_history(gkba_ctx* c, int N, int k0, int nk, int L, double dt,
                               const double2* rho, const double2* T, const double* w, double2* G,
                               double2* Gb, double* coef);
gkba_status weighted_sum_units(gkba_ctx* c, int N, int nb, const double* coef, const double2* Y,
                               double2* I);
gkba_status build_forms_fp64(gkba_ctx* c, int nb, const double2* G, const double2* Gb);
gkba_status build_forms_tf32(gkba_ctx* c, int nb, const double2* G, const double2* Gb);
gkba_status build_forms3_fp64(gkba_ctx* c, int nb, const double2* A);
// adjoint of the collision integral: per-unit elementwise steps (N x N units)
gkba_status unit_xform(gkba_ctx* c, int nb, const double2* in, double2* out, int conj, int transpose);
gkba_status unit_acc(gkba_ctx* c, int nb, double2* y, const double2* x, int transpose);
gkba_status scale_units(gkba_ctx* c, int nb, const double* coef, const double2* Ibar, double2* Y);
gkba_status vjp_points(gkba_ctx* c, int nk, const double2* Gbar, const double2* Gbbar, double2* Pbar,
                       double2* Qbar);
// adjoint of the Heun step (N x N helpers)
gkba_status add_i_diff(gkba_ctx* c, double2* y, const double2* a, const double2* b, double s);
gkba_status ibar_from_kbar(gkba_ctx* c, const double2* kb, double2* Ib);
gkba_status mean_field_adj(gkba_ctx* c, const double2* hb, double2* rb);
gkba_status field_grad(gkba_ctx* c, const double2* hb, double* out);
gkba_status expm_adj(gkba_ctx* c, const double2* hA, const double2* hB, const double2* Ubar,
                     double2* hA_bar, double2* hB_bar, double2* scratch);
gkba_status sum_units(gkba_ctx* c, int nb, const double2* src, double2* dst);
// gradient with respect to v (FP64 path)
gkba_status fp64_chain_x3(gkba_ctx* c, int nb, const double* A1, const StageMap* m3 = nullptr,
                          long long sOz3 = 0);
gkba_status vbar_slot(gkba_ctx* c, int nb, const double2* Sbar, int transposeS, const double* X,
                      double* out);
gkba_status fold_vbar(gkba_ctx* c, const double* vslot, const double* wslot, double* vbar);
gkba_status vbar_mean_field(gkba_ctx* c, const double2* hb, const double2* rho, double* vbar);
gkba_status build_vomega64(gkba_ctx* c, double* out);
gkba_status collision_vjp_dev(gkba_ctx* c, int L, const double2* rho, const double2* T,
                              const double* w, const double2* Ibar, double2* rho_bar,
                              double2* T_bar, double* vslot = nullptr, double* wslot = nullptr);
gkba_status build_forms3_tf32(gkba_ctx* c, int nb, const double2* A);
gkba_status reduce_partials_launch(gkba_ctx* c, int nb, int nz, long long zstride, long long Rld,
                                   const void* part, bool fp32, double2* S);
// K length of one work item of the tensor-core S4 stage (one FP32 partial per
// item and output row).
constexpr int kTcItemK = 4096;
// Default K length of one tensor-memory accumulation window of that stage.
constexpr int kTcWindowK = 32;
size_t tf32_part_bytes(int Np, int ub, int kchunk);
// Launch the bounded-wait self-test (a wait that must run out); elapsed_ms[2].
gkba_status wait_selftest(gkba_ctx* c, double limit_ms, double* elapsed_ms);
gkba_status measure_tf32_mma(gkba_ctx* c, int iters, double* tflops);

// ---- time-linear history (time_linear.cu) ---------------------------------
// Terms of nk history points (rho_k, W_k = Ucal_k^+ at stride sW) summed into
// c->X2 as D[j][n][r][c][p], point k0 + i weighted (k0 + i == 0 ? w_first : w_rest).
gkba_status tl_terms(gkba_ctx* c, int nk, const double2* rho, const double2* W, long long sW,
                     int k0, double w_first, double w_rest);
// tl_s = tl_acc + a D (when write_s) and tl_acc += b D (when add_acc), D = c->X2.
gkba_status tl_update(gkba_ctx* c, double a, double b, bool write_s, bool add_acc);
// I = [v . (Ucal x_n Ucal x_p conj(Ucal) x_r tl_s)] Ucal^+ with Ucal = W^+;
// overwrites tl_s, X2 and X13.
gkba_status tl_apply(gkba_ctx* c, const double2* W, double2* I_out);

// Workspace sizing: make sure the workspace holds ub units (returns actual ub).
gkba_status ensure_workspace(gkba_ctx* c, int want_units);
gkba_status ensure_stage(gkba_ctx* c, size_t bytes);

}  // namespace gkba
