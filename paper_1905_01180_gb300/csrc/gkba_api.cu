// gkba_api.cu - C ABI entry points of libgkba: context life cycle, input
// validation, the history store, the contraction driver (collision integral
// of Eq. (collint) over a batched list of (t_k, component) units) and the
// Heun stepper of Eq. (equalt).  See include/gkba.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "gkba_internal.cuh"

namespace gkba {

const char* kKernelClassNames[K_COUNT] = {"S1_w_x_Gbar", "S2_G_x_X1", "S3_G_x_X2", "S4_v_dot_X3",
                                          "prep",        "reduce",    "stepper",   "time_linear"};

static std::mutex g_err_mu;
static std::string g_last_init_error;

gkba_status fail(gkba_ctx* c, gkba_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else {
        std::lock_guard<std::mutex> g(g_err_mu);
        g_last_init_error = buf;
    }
    return st;
}

LaunchToken launch_begin(gkba_ctx* c, int cls, double flops, double bytes) {
    LaunchToken t{cls, nullptr};
    c->launches++;
    c->cls_launches[cls]++;
    c->cls_flops[cls] += flops;
    c->cls_bytes[cls] += bytes;
    if (c->timing && (cls == K_W1 || cls == K_W2 || cls == K_W3 || cls == K_FIN)) {
        cudaEvent_t a;
        if (!c->event_pool.empty()) {
            a = c->event_pool.back();
            c->event_pool.pop_back();
        } else if (cudaEventCreate(&a) != cudaSuccess) {
            return t;
        }
        cudaEventRecord(a, c->stream);
        t.a = a;
    }
    return t;
}

gkba_status launch_end(gkba_ctx* c, LaunchToken t) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(c, GKBA_ECUDA, "kernel launch (%s) failed: %s", kKernelClassNames[t.cls],
                    cudaGetErrorString(e));
    if (t.a) {
        cudaEvent_t b;
        if (!c->event_pool.empty()) {
            b = c->event_pool.back();
            c->event_pool.pop_back();
        } else if (cudaEventCreate(&b) != cudaSuccess) {
            c->event_pool.push_back(t.a);
            return GKBA_OK;
        }
        cudaEventRecord(b, c->stream);
        c->pending.push_back(TimedLaunch{t.cls, t.a, b});
    }
    return GKBA_OK;
}

gkba_status harvest_timing(gkba_ctx* c) {
    if (c->pending.empty()) return GKBA_OK;
    GKBA_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto& p : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->cls_ms[p.cls] += ms;
        c->event_pool.push_back(p.a);
        c->event_pool.push_back(p.b);
    }
    c->pending.clear();
    return GKBA_OK;
}

// Allocation helper: carve aligned sub-buffers out of one block.
struct Carver {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    }
};

gkba_status ensure_workspace(gkba_ctx* c, int want_units) {
    const long long N = c->N, NN = N * N;
    want_units = std::max(2, want_units + (want_units & 1));
    const bool tc = tensor_core_path(c);
    const bool gen = c->kind == GKBA_V_GENERAL;  // structured kinds need no stage buffers
    const long long Np = c->Np;
    const double x_bytes = !gen ? 0.0 : tc ? 2.0 * Np * Np * Np * Np * 4 : 2.0 * NN * NN * 8;
    const double form_bytes = !gen ? 0.0 : tc ? 4.0 * 2 * Np * Np * 4 : (2.0 * NN + 4.0 * NN) * 8;
    const double N3 = (double)NN * N;
    const double part_per_unit = !gen ? 0.0
                                 : tc ? (std::ceil((double)Np * Np * Np / kTcItemK) * Np * 2.0 * Np * 4)
                                      : (std::ceil(N3 / 8192.0) * N * 2.0 * N * 8);
    const double per_unit = 2 * x_bytes + form_bytes + part_per_unit + (4.0 + kReduceSplit) * NN * 16 + 8;
    size_t cap = c->ws_cap;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const size_t usable = (size_t)((double)(free_b + c->ws_bytes) * 0.85);
        cap = std::min(cap, usable);
    }
    long long fit = (long long)((double)cap / per_unit);
    fit -= fit & 1;
    if (fit < 2)
        return fail(c, GKBA_ENOMEM, "workspace cap %.3g GB holds fewer than 2 units (%.3g GB each)",
                    cap / 1e9, per_unit / 1e9);
    int ub = (int)std::min<long long>(fit, want_units);
    if (c->ws && ub <= c->ub_cap) {
        c->ub = ub;
        return GKBA_OK;
    }
    if (c->ws) {
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    Carver cv;
    // the last stage's K-blocked X3 pads the batch's 2 Np ub rows to 256
    const double x3_blocked = tc && gen ? (double)Np * Np * Np * (((2.0 * Np * ub + 255) / 256) * 256) * 4 : 0.0;
    const size_t x13_bytes = (size_t)std::max(x_bytes * ub, std::floor(x3_blocked));
    const size_t oX13 = cv.take(x13_bytes);
    const size_t oX2 = cv.take((size_t)(x_bytes * ub));
    size_t part_bytes;
    if (!gen) part_bytes = 0;
    else if (tc) part_bytes = tf32_part_bytes((int)Np, ub, c->acc_window);
    else {
        const long long nz = (long long)std::ceil(N3 / 8192.0);
        part_bytes = (size_t)(nz * N * 2LL * N * ub * 8);
        // the time-linear collision splits one unit's K into up to 1024 chunks
        if (c->history == GKBA_HISTORY_TIME_LINEAR)
            part_bytes = std::max(part_bytes, (size_t)(1024LL * N * 2LL * N * 8));
    }
    const size_t oPart = cv.take(part_bytes);
    const size_t oB1 = cv.take(!gen ? 0 : tc ? (size_t)(2LL * 2 * Np * Np * ub * 4) : (size_t)(2LL * NN * ub * 8));
    const size_t oG = cv.take(!gen ? 0 : tc ? (size_t)(2LL * 4 * Np * Np * ub * 4) : (size_t)(4LL * NN * ub * 8));
    const size_t oG3 = cv.take(!gen ? 0 : tc ? (size_t)(2LL * 4 * Np * Np * ub * 4) : (size_t)(4LL * NN * ub * 8));
    const size_t oPQ = cv.take((size_t)(ub * NN * 16));
    const size_t oMb = cv.take((size_t)(ub * NN * 16));
    const size_t oCoef = cv.take((size_t)ub * 8);
    const size_t oSu = cv.take((size_t)(ub * NN * 16));
    const size_t oYu = cv.take((size_t)(ub * NN * 16));
    const size_t oRed = cv.take((size_t)(kReduceSplit * ub * NN * 16));
    void* ws = nullptr;
    if (cudaMalloc(&ws, cv.off) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GKBA_ENOMEM, "cudaMalloc(%zu) for the contraction workspace failed", cv.off);
    }
    char* b = (char*)ws;
    c->ws = ws;
    c->ws_bytes = cv.off;
    c->ub = ub;
    c->ub_cap = ub;
    c->X13 = b + oX13;
    c->x13_bytes = x13_bytes;
    c->X2 = b + oX2;
    c->part = b + oPart;
    c->part_bytes = part_bytes;
    c->formsB1 = b + oB1;
    c->formsG = b + oG;
    c->formsG3 = b + oG3;
    c->PQ = (double2*)(b + oPQ);
    c->Mb = (double2*)(b + oMb);
    c->coef = (double*)(b + oCoef);
    c->Su = (double2*)(b + oSu);
    c->Yu = (double2*)(b + oYu);
    c->red_tmp = (double2*)(b + oRed);
    return GKBA_OK;
}

gkba_status ensure_stage(gkba_ctx* c, size_t bytes) {
    if (bytes <= c->stage_bytes) return GKBA_OK;
    if (c->stage) cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    if (cudaMalloc(&c->stage, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GKBA_ENOMEM, "cudaMalloc(%zu) for staging failed", bytes);
    }
    c->stage_bytes = bytes;
    return GKBA_OK;
}

// One batch of nb units: (G_u, Gb_u) at G, Gb (stride N*N; the general paths
// read the forms built from them) -> S_u in c->Su.
static gkba_status contract(gkba_ctx* c, int nb, const double2* G, const double2* Gb) {
    NvtxRange r("gkba contraction batch");
    if (c->kind != GKBA_V_GENERAL) return contract_structured(c, nb, G, Gb);
    if (tensor_core_path(c)) return contract_batch_tf32(c, nb);
    return contract_batch_fp64(c, nb);
}

gkba_status collision_dev(gkba_ctx* c, int L, const double2* rho, const double2* T,
                          const double* weights_dev, double2* I_out) {
    NvtxRange r("gkba collision");
    const long long NN = (long long)c->N * c->N;
    GKBA_CUDA(c, cudaMemsetAsync(I_out, 0, NN * sizeof(double2), c->stream));
    if (L <= 1 && weights_dev == nullptr) return GKBA_OK;  // zero-length time interval
    GKBA_TRY(ensure_workspace(c, 2 * L));
    const int nk_per = c->ub / 2;
    for (int k0 = 0; k0 < L; k0 += nk_per) {
        const int nk = std::min(nk_per, L - k0);
        GKBA_TRY(build_forms_gkba(c, k0, nk, L, rho, T, weights_dev));
        GKBA_TRY(contract(c, 2 * nk, c->Su, c->Mb));
        GKBA_TRY(reduce_batch(c, 2 * nk, I_out, nullptr));
    }
    return GKBA_OK;
}

gkba_status sigma_dev(gkba_ctx* c, int n_units, const double2* G, const double2* Gb, double2* S_out) {
    const long long NN = (long long)c->N * c->N;
    GKBA_TRY(ensure_workspace(c, n_units));
    for (int u0 = 0; u0 < n_units; u0 += c->ub) {
        const int nb = std::min(c->ub, n_units - u0);
        GKBA_TRY(build_forms(c, nb, G + u0 * NN, NN, Gb + u0 * NN, NN, 0));
        GKBA_TRY(contract(c, nb, G + u0 * NN, Gb + u0 * NN));
        GKBA_TRY(reduce_batch(c, nb, nullptr, S_out + u0 * NN));
    }
    return GKBA_OK;
}

// S3(A_u, B_u, C_u) of nb units (device, stride N*N) into c->Su: the
// contraction chain with B in stage S1's slot, C in S2's and A in S3's.
static gkba_status contract3(gkba_ctx* c, int nb, const double2* A, const double2* B,
                             const double2* C) {
    const long long NN = (long long)c->N * c->N;
    GKBA_TRY(build_forms(c, nb, C, NN, B, NN, 0));
    if (A != C) {
        GKBA_TRY(tensor_core_path(c) ? build_forms3_tf32(c, nb, A) : build_forms3_fp64(c, nb, A));
        c->sep_A = true;
    }
    const gkba_status st = contract(c, nb, C, B);
    c->sep_A = false;
    return st;
}

gkba_status sigma3_dev(gkba_ctx* c, int n_units, const double2* A, const double2* B,
                       const double2* C, double2* S_out) {
    const long long NN = (long long)c->N * c->N;
    GKBA_TRY(ensure_workspace(c, n_units));
    for (int u0 = 0; u0 < n_units; u0 += c->ub) {
        const int nb = std::min(c->ub, n_units - u0);
        GKBA_TRY(contract3(c, nb, A + u0 * NN, B + u0 * NN, C + u0 * NN));
        GKBA_CUDA(c, cudaMemcpyAsync(S_out + u0 * NN, c->Su, nb * NN * sizeof(double2),
                                     cudaMemcpyDeviceToDevice, c->stream));
    }
    return GKBA_OK;
}

// Reverse mode of collision_dev: given Ibar (device, N*N), rho_bar and
// T_bar (device, L*N*N) for the L history points.  Gradients are real pairs
// (dL/dRe + i dL/dIm).  Per batch of units (G_u, Gb_u) with coefficient c_u:
//   Ybar = c_u Ibar;  Sbar = Ybar Gb^+;  Gbbar = S^+ Ybar (from Y = S Gb)
//   Gbbar += S3(G*, Sbar^T, G*)^T                      (S's Gb slot)
//   Gbar   = S3(Sbar, G*^T, Gb*^T) + S3(Gb*^T, G*^T, Sbar)  (its two G slots)
// (the slot derivatives of Eq. (2bse) written as S3 evaluations, valid for
// w = 2v - v_exch with v 8-fold symmetric); then
//   Pbar = Gbar(P slot) + Gbbar(P^+ slot)^+,  Qbar likewise,
//   rho_bar = T^+ (Pbar - Qbar),  T_bar = (Pbar - Qbar) rho^+ + Qbar.
gkba_status collision_vjp_dev(gkba_ctx* c, int L, const double2* rho, const double2* T,
                              const double* w, const double2* Ibar, double2* rho_bar,
                              double2* T_bar, double* vslot, double* wslot) {
    const int N = c->N;
    const long long NN = (long long)N * N;
    GKBA_TRY(ensure_workspace(c, 2 * L));
    if (c->vjp_units < c->ub) {
        if (c->vjp) cudaFree(c->vjp);
        c->vjp = nullptr;
        c->vjp_units = 0;
        if (cudaMalloc(&c->vjp, 10ull * c->ub * NN * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, GKBA_ENOMEM, "adjoint scratch of %d units does not fit", c->ub);
        }
        c->vjp_units = c->ub;
    }
    const long long blk = (long long)c->vjp_units * NN;
    double2 *Gv = c->vjp, *Gbv = Gv + blk, *Sv = Gv + 2 * blk, *Sbv = Gv + 3 * blk,
            *Gbb = Gv + 4 * blk, *Gbr = Gv + 5 * blk, *tA = Gv + 6 * blk, *tB = Gv + 7 * blk,
            *tC = Gv + 8 * blk, *D = Gv + 9 * blk;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    const int nk_per = c->ub / 2;
    for (int k0 = 0; k0 < L; k0 += nk_per) {
        const int nk = std::min(nk_per, L - k0), nb = 2 * nk;
        GKBA_TRY(units_from_history(c, N, k0, nk, L, c->dt, rho, T, w, Gv, Gbv, c->coef));
        GKBA_TRY(contract3(c, nb, Gv, Gbv, Gv));  // S_u
        GKBA_CUDA(c, cudaMemcpyAsync(Sv, c->Su, nb * NN * sizeof(double2), cudaMemcpyDeviceToDevice,
                                     c->stream));
        GKBA_TRY(scale_units(c, nb, c->coef, Ibar, tC));  // Ybar
        GKBA_TRY(zgemm_batched(c, K_RED, N, 'N', 'C', one, tC, NN, Gbv, NN, zero, Sbv, NN, nb, 0));
        GKBA_TRY(zgemm_batched(c, K_RED, N, 'C', 'N', one, Sv, NN, tC, NN, zero, Gbb, NN, nb, 0));
        if (vslot && tensor_core_path(c)) {
            // dL/dv (tensor cores): the v slot against the X3 of S above, still in
            // X13; the w slot against the chain run on the omega layout of v
            GKBA_TRY(vbar_slot_tf32(c, nb, Sbv, 0, vslot));
            GKBA_TRY(unit_xform(c, nb, Gv, tA, 0, 1));
            GKBA_TRY(unit_xform(c, nb, Gbv, tB, 0, 1));
            GKBA_TRY(build_forms(c, nb, tA, NN, tB, NN, 0));
            GKBA_TRY(tf32_chain_omega(c, nb));
            GKBA_TRY(vbar_slot_tf32(c, nb, Sbv, 1, wslot));
        } else if (vslot) {
            // dL/dv (FP64 path): the v slot against X3 = W3 still in X13 from S above
            GKBA_TRY(vbar_slot(c, nb, Sbv, 0, (const double*)c->X13, vslot));
            // the w slot against the same chain run on v in the omega layout with G^T, Gb^T
            GKBA_TRY(unit_xform(c, nb, Gv, tA, 0, 1));
            GKBA_TRY(unit_xform(c, nb, Gbv, tB, 0, 1));
            GKBA_TRY(build_forms(c, nb, tA, NN, tB, NN, 0));
            GKBA_TRY(fp64_chain_x3(c, nb, c->vomega));
            GKBA_TRY(vbar_slot(c, nb, Sbv, 1, (const double*)c->X13, wslot));
        }
        GKBA_TRY(unit_xform(c, nb, Gv, tA, 1, 0));   // G*
        GKBA_TRY(unit_xform(c, nb, Sbv, tB, 0, 1));  // Sbar^T
        GKBA_TRY(contract3(c, nb, tA, tB, tA));
        GKBA_TRY(unit_acc(c, nb, Gbb, c->Su, 1));
        GKBA_TRY(unit_xform(c, nb, Gv, tB, 1, 1));   // G*^T
        GKBA_TRY(unit_xform(c, nb, Gbv, tC, 1, 1));  // Gb*^T
        GKBA_TRY(contract3(c, nb, Sbv, tB, tC));
        GKBA_CUDA(c, cudaMemcpyAsync(Gbr, c->Su, nb * NN * sizeof(double2), cudaMemcpyDeviceToDevice,
                                     c->stream));
        GKBA_TRY(contract3(c, nb, tC, tB, Sbv));
        GKBA_TRY(unit_acc(c, nb, Gbr, c->Su, 0));
        GKBA_TRY(vjp_points(c, nk, Gbr, Gbb, tA, tB));  // Pbar, Qbar
        GKBA_TRY(axpy_c(c, D, tA, tB, 1.0, -1.0, (int)(nk * NN)));
        GKBA_TRY(zgemm_batched(c, K_RED, N, 'C', 'N', one, T + k0 * NN, NN, D, NN, zero,
                               rho_bar + k0 * NN, NN, nk, 0));
        GKBA_TRY(zgemm_batched(c, K_RED, N, 'N', 'C', one, D, NN, rho + k0 * NN, NN, zero,
                               T_bar + k0 * NN, NN, nk, 0));
        GKBA_TRY(axpy_c(c, T_bar + k0 * NN, T_bar + k0 * NN, tB, 1.0, 1.0, (int)(nk * NN)));
    }
    return GKBA_OK;
}

// After a public call: wait for the stream, fold timings, check the device
// error word written by bounded waits.
static gkba_status finish(gkba_ctx* c) {
    GKBA_CUDA(c, cudaStreamSynchronize(c->stream));
    GKBA_TRY(harvest_timing(c));
    int errw = 0;
    GKBA_CUDA(c, cudaMemcpy(&errw, c->dint + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (errw != 0) {
        cudaMemset(c->dint + 1, 0, sizeof(int));
        return fail(c, GKBA_ETIMEOUT, "device-side wait timed out (code %d); results invalid", errw);
    }
    return GKBA_OK;
}

}  // namespace gkba

using namespace gkba;

namespace {

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Max |A - A^+| relative to max |A| for an interleaved complex N x N matrix.
bool hermitian(const double* a, int N, double tol) {
    double mx = 0.0, dev = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            const double re = a[2 * (i * N + j)], im = a[2 * (i * N + j) + 1];
            const double tre = a[2 * (j * N + i)], tim = a[2 * (j * N + i) + 1];
            mx = std::max(mx, std::hypot(re, im));
            dev = std::max(dev, std::hypot(re - tre, im + tim));
        }
    return dev <= tol * std::max(mx, 1e-300);
}

// Eq. (symmetries): v_ijkl = v_jilk = v_klij = v_lkji = v_ikjl = v_ljki = v_kilj = v_jlik.
bool eightfold(const double* v, int N, double tol) {
    const long long n = N;
    double mx = 0.0;
    for (long long e = 0; e < n * n * n * n; ++e) mx = std::max(mx, std::fabs(v[e]));
    const double lim = tol * std::max(mx, 1e-300);
    auto at = [&](long long i, long long j, long long k, long long l) { return v[((i * n + j) * n + k) * n + l]; };
    for (long long i = 0; i < n; ++i)
        for (long long j = 0; j < n; ++j)
            for (long long k = 0; k < n; ++k)
                for (long long l = 0; l < n; ++l) {
                    const double x = at(i, j, k, l);
                    if (std::fabs(x - at(j, i, l, k)) > lim || std::fabs(x - at(k, l, i, j)) > lim ||
                        std::fabs(x - at(l, k, j, i)) > lim || std::fabs(x - at(i, k, j, l)) > lim ||
                        std::fabs(x - at(l, j, k, i)) > lim || std::fabs(x - at(k, i, l, j)) > lim ||
                        std::fabs(x - at(j, l, i, k)) > lim)
                        return false;
                }
    return true;
}

gkba_status copy_in(gkba_ctx* c, void* dst, const void* src, size_t bytes, int on_device) {
    GKBA_CUDA(c, cudaMemcpyAsync(dst, src, bytes,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 c->stream));
    return GKBA_OK;
}

gkba_status alloc(gkba_ctx* c, void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, GKBA_ENOMEM, "cudaMalloc(%zu) failed", bytes);
    }
    return GKBA_OK;
}

void free_ctx(gkba_ctx* c) {
    if (!c) return;
    if (c->device >= 0) cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    void* ptrs[] = {c->tl_acc, c->tl_s, c->tl_W, c->tl_Wn, c->tl_uf,
                    c->h, c->d, c->v, c->vm, c->vjp, c->rhot_hist, c->U_hist, c->adj_ws, c->vomega,
                    c->vgrad, c->hfK, c->wS64, c->vK64, c->wS32, c->vO32, c->xsw, c->vKhi, c->vKlo,
                    c->rho_hist, c->T_a, c->T_b, c->hhf_n, c->hhf_t, c->k1, c->k2, c->Ia, c->Ib,
                    c->U, c->ex0, c->ex1, c->ex2, c->tmp0, c->tmp1, c->dscal, c->dint, c->ws,
                    c->stage};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->hdiag) cudaFreeHost(c->hdiag);
    for (auto& p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // namespace

namespace gkba {
gkba_status fp64_prepare_model(gkba_ctx* c);
}

extern "C" {

gkba_status gkba_init(gkba_ctx** out, const gkba_config* cfg, const double* h, const double* v,
                      const double* d, const double* rho0, int inputs_on_device) {
    if (out) *out = nullptr;
    if (!out || !cfg) return fail(nullptr, GKBA_EINVAL, "gkba_init: out and cfg must be non-NULL");
    if (!h || !v || !d || !rho0) return fail(nullptr, GKBA_EINVAL, "gkba_init: NULL model input");
    const int N = cfg->N;
    if (N < 1 || N > 128) return fail(nullptr, GKBA_EINVAL, "gkba_init: N=%d outside [1, 128]", N);
    if (!(cfg->dt > 0.0) || !std::isfinite(cfg->dt))
        return fail(nullptr, GKBA_EINVAL, "gkba_init: dt must be positive and finite");
    if (cfg->max_steps < 0 || cfg->max_steps > 100000000)
        return fail(nullptr, GKBA_EINVAL, "gkba_init: max_steps=%d invalid", cfg->max_steps);
    if (cfg->acc_window != 0 && cfg->acc_window != 8 && cfg->acc_window != 16 && cfg->acc_window != 32)
        return fail(nullptr, GKBA_EINVAL, "gkba_init: acc_window=%d must be 0, 8, 16 or 32",
                    cfg->acc_window);
    if (cfg->precision != GKBA_FP64 && cfg->precision != GKBA_SPLIT_TF32 &&
        cfg->precision != GKBA_SPLIT_TF32_ACC)
        return fail(nullptr, GKBA_EINVAL, "gkba_init: unknown precision %d", cfg->precision);
    const int kind = cfg->interaction;
    if (kind != GKBA_V_GENERAL && kind != GKBA_V_DIAGONAL && kind != GKBA_V_SYMMETRIC)
        return fail(nullptr, GKBA_EINVAL, "gkba_init: unknown interaction %d", kind);
    if (kind != GKBA_V_GENERAL && cfg->precision != GKBA_FP64)
        return fail(nullptr, GKBA_EINVAL,
                    "gkba_init: diagonal and symmetric interactions run in FP64 (precision %d)",
                    cfg->precision);
    if (cfg->history != GKBA_HISTORY_SUM && cfg->history != GKBA_HISTORY_TIME_LINEAR)
        return fail(nullptr, GKBA_EINVAL, "gkba_init: unknown history mode %d", cfg->history);
    if (cfg->history == GKBA_HISTORY_TIME_LINEAR && kind != GKBA_V_GENERAL)
        return fail(nullptr, GKBA_EUNSUPPORTED,
                    "gkba_init: the time-linear history needs a general v");
    const int Np = ((N + 15) / 16) * 16;
    if (cfg->precision != GKBA_FP64 && Np > 96)
        return fail(nullptr, GKBA_EINVAL,
                    "gkba_init: the split-TF32 path supports N <= 96 (N=%d)", N);
    const size_t NN = (size_t)N * N, N4 = NN * NN;

    // Host copies for validation (device inputs are copied back first).
    // v as given (N^4, N or N*N values) and expanded to v_ijkl
    const size_t nv = kind == GKBA_V_GENERAL ? N4 : kind == GKBA_V_DIAGONAL ? (size_t)N : NN;
    std::vector<double> hh(2 * NN), dh(2 * NN), rh(2 * NN), vm(nv), vh;
    if (inputs_on_device) {
        if (cudaMemcpy(hh.data(), h, 2 * NN * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(dh.data(), d, 2 * NN * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(rh.data(), rho0, 2 * NN * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(vm.data(), v, nv * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return fail(nullptr, GKBA_EINVAL, "gkba_init: inputs_on_device but a pointer is not readable device memory");
        }
    } else {
        memcpy(hh.data(), h, 2 * NN * 8);
        memcpy(dh.data(), d, 2 * NN * 8);
        memcpy(rh.data(), rho0, 2 * NN * 8);
        memcpy(vm.data(), v, nv * 8);
    }
    if (!finite_all(hh.data(), 2 * NN) || !finite_all(dh.data(), 2 * NN) ||
        !finite_all(rh.data(), 2 * NN) || !finite_all(vm.data(), nv))
        return fail(nullptr, GKBA_EINVAL, "gkba_init: non-finite values in h, v, d or rho0");
    if (kind == GKBA_V_GENERAL) {
        vh.swap(vm);
    } else {
        // Sec. III A: v_iiii = U_i;  Sec. III B: v_ijji = V_ij (l = i, k = j)
        vh.assign(N4, 0.0);
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                if (kind == GKBA_V_DIAGONAL && i != j) continue;
                const double x = kind == GKBA_V_DIAGONAL ? vm[i] : vm[(size_t)i * N + j];
                vh[(((size_t)i * N + j) * N + j) * N + i] = x;
            }
        if (kind == GKBA_V_SYMMETRIC) {
            double mx = 0.0, dev = 0.0;
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    mx = std::max(mx, std::fabs(vm[(size_t)i * N + j]));
                    dev = std::max(dev, std::fabs(vm[(size_t)i * N + j] - vm[(size_t)j * N + i]));
                }
            if (dev > 1e-12 * std::max(mx, 1e-300))
                return fail(nullptr, GKBA_EINVAL, "gkba_init: V of a symmetric interaction is not symmetric");
        }
    }
    if (!hermitian(hh.data(), N, 1e-10)) return fail(nullptr, GKBA_EINVAL, "gkba_init: h is not Hermitian");
    if (!hermitian(dh.data(), N, 1e-10)) return fail(nullptr, GKBA_EINVAL, "gkba_init: d is not Hermitian");
    if (!hermitian(rh.data(), N, 1e-10)) return fail(nullptr, GKBA_EINVAL, "gkba_init: rho0 is not Hermitian");
    if (!eightfold(vh.data(), N, 1e-10))
        return fail(nullptr, GKBA_EINVAL, "gkba_init: v breaks the 8-fold permutation symmetry");

    gkba_ctx* c = new gkba_ctx();
    c->N = N;
    c->Np = Np;
    c->dt = cfg->dt;
    c->max_steps = cfg->max_steps;
    c->prec = cfg->precision;
    c->kind = kind;
    c->history = cfg->history;
    c->ws_cap = cfg->workspace_bytes ? cfg->workspace_bytes : ((size_t)64 << 30);
    c->timing = cfg->timing != 0;
    c->acc_window = cfg->acc_window > 0 ? cfg->acc_window : kTcWindowK;
    c->device = -1;
    auto bail = [&](gkba_status st) {
        {
            std::lock_guard<std::mutex> g(g_err_mu);
            g_last_init_error = c->err;
        }
        free_ctx(c);
        return st;
    };
    int dev = cfg->device;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            fail(c, GKBA_ECUDA, "gkba_init: no CUDA device");
            return bail(GKBA_ECUDA);
        }
    }
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        fail(c, GKBA_ECUDA, "gkba_init: cudaSetDevice(%d) failed", dev);
        return bail(GKBA_ECUDA);
    }
    c->device = dev;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        fail(c, GKBA_ECUDA, "gkba_init: cudaGetDeviceProperties failed");
        return bail(GKBA_ECUDA);
    }
    c->num_sms = prop.multiProcessorCount;
    if (tensor_core_path(c) && !(prop.major == 10 && prop.minor == 3)) {
        fail(c, GKBA_EUNSUPPORTED, "gkba_init: split-TF32 path needs an sm_103 GPU (found sm_%d%d)",
             prop.major, prop.minor);
        return bail(GKBA_EUNSUPPORTED);
    }
    if (cfg->cuda_stream) {
        c->stream = (cudaStream_t)cfg->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            fail(c, GKBA_ECUDA, "gkba_init: stream creation failed");
            return bail(GKBA_ECUDA);
        }
        c->own_stream = true;
    }
    const size_t cap = (size_t)c->max_steps + 1;
    gkba_status st = GKBA_OK;
#define ALLOC(ptr, bytes)                                                  \
    do {                                                                   \
        void* p_ = nullptr;                                                \
        st = alloc(c, &p_, (bytes));                                       \
        if (st != GKBA_OK) return bail(st);                                \
        ptr = (decltype(ptr))p_;                                           \
    } while (0)
    ALLOC(c->h, NN * 16);
    ALLOC(c->d, NN * 16);
    ALLOC(c->v, N4 * 8);
    ALLOC(c->hfK, N4 * 8);
    ALLOC(c->rho_hist, cap * NN * 16);
    ALLOC(c->T_a, cap * NN * 16);
    ALLOC(c->T_b, cap * NN * 16);
    ALLOC(c->rhot_hist, cap * NN * 16);
    ALLOC(c->U_hist, cap * NN * 16);
    ALLOC(c->hhf_n, NN * 16);
    ALLOC(c->hhf_t, NN * 16);
    ALLOC(c->k1, NN * 16);
    ALLOC(c->k2, NN * 16);
    ALLOC(c->Ia, NN * 16);
    ALLOC(c->Ib, NN * 16);
    ALLOC(c->U, NN * 16);
    ALLOC(c->ex0, NN * 16);
    ALLOC(c->ex1, NN * 16);
    ALLOC(c->ex2, NN * 16);
    ALLOC(c->tmp0, NN * 16);
    ALLOC(c->tmp1, NN * 16);
    ALLOC(c->dscal, 16 * 8);
    ALLOC(c->dint, 4 * 4);
    if (kind != GKBA_V_GENERAL) {
        ALLOC(c->vm, nv * 8);
    } else if (c->prec == GKBA_FP64) {
        ALLOC(c->wS64, N4 * 8);
        ALLOC(c->vK64, N4 * 8);
        if (c->history == GKBA_HISTORY_TIME_LINEAR) {
            ALLOC(c->tl_acc, 2 * N4 * 8);
            ALLOC(c->tl_s, 2 * N4 * 8);
            ALLOC(c->tl_W, NN * 16);
            ALLOC(c->tl_Wn, NN * 16);
            ALLOC(c->tl_uf, 8 * NN * 8);
        }
    } else {
        const size_t Np4 = (size_t)Np * Np * Np * Np;
        ALLOC(c->wS32, Np4 * 4);
        ALLOC(c->vKhi, Np4 * 4);
        ALLOC(c->vKlo, Np4 * 4);
        if (c->history == GKBA_HISTORY_TIME_LINEAR) {
            ALLOC(c->tl_acc, 2 * N4 * 8);
            ALLOC(c->tl_s, 2 * N4 * 8);
            ALLOC(c->tl_W, NN * 16);
            ALLOC(c->tl_Wn, NN * 16);
        }
    }
#undef ALLOC
    if (cudaMallocHost((void**)&c->hdiag, 16 * 8) != cudaSuccess) {
        fail(c, GKBA_ENOMEM, "cudaMallocHost failed");
        return bail(GKBA_ENOMEM);
    }
    if ((st = copy_in(c, c->h, hh.data(), NN * 16, 0)) != GKBA_OK) return bail(st);
    if ((st = copy_in(c, c->d, dh.data(), NN * 16, 0)) != GKBA_OK) return bail(st);
    if ((st = copy_in(c, c->v, vh.data(), N4 * 8, 0)) != GKBA_OK) return bail(st);
    if (c->vm && (st = copy_in(c, c->vm, vm.data(), nv * 8, 0)) != GKBA_OK) return bail(st);
    if ((st = copy_in(c, c->rho_hist, rh.data(), NN * 16, 0)) != GKBA_OK) return bail(st);
    if (cudaMemsetAsync(c->dint, 0, 16, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->dscal, 0, 128, c->stream) != cudaSuccess) {
        fail(c, GKBA_ECUDA, "gkba_init: memset failed");
        return bail(GKBA_ECUDA);
    }
    if ((st = set_identity(c, c->T_a, 1)) != GKBA_OK) return bail(st);
    if (c->tl_acc) {
        if (cudaMemsetAsync(c->tl_acc, 0, 2 * N4 * 8, c->stream) != cudaSuccess) {
            fail(c, GKBA_ECUDA, "gkba_init: memset failed");
            return bail(GKBA_ECUDA);
        }
        if ((st = set_identity(c, c->tl_W, 1)) != GKBA_OK) return bail(st);
    }
    if ((st = fp64_prepare_model(c)) != GKBA_OK) return bail(st);
    if (tensor_core_path(c) && (st = tf32_prepare_model(c)) != GKBA_OK) return bail(st);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        fail(c, GKBA_ECUDA, "gkba_init: %s", cudaGetErrorString(cudaGetLastError()));
        return bail(GKBA_ECUDA);
    }
    c->n = 0;
    c->adj_from = 0;
    c->E_a.assign(cap, 0.0);
    c->E_b.assign(cap, 0.0);
    *out = c;
    return GKBA_OK;
}

gkba_status gkba_sigma(gkba_ctx* c, int n_units, const double* G, const double* Gbar, double* S_out,
                       int on_device) {
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_sigma: NULL context");
    if (n_units < 0 || (n_units > 0 && (!G || !Gbar || !S_out)))
        return fail(c, GKBA_EINVAL, "gkba_sigma: bad arguments");
    if (n_units == 0) return GKBA_OK;
    GKBA_CUDA(c, cudaSetDevice(c->device));
    const size_t NN = (size_t)c->N * c->N, bytes = NN * 16 * (size_t)n_units;
    const double2 *dG, *dGb;
    double2* dS;
    if (on_device) {
        dG = (const double2*)G;
        dGb = (const double2*)Gbar;
        dS = (double2*)S_out;
    } else {
        GKBA_TRY(ensure_stage(c, 3 * bytes));
        dG = (double2*)c->stage;
        dGb = (double2*)((char*)c->stage + bytes);
        dS = (double2*)((char*)c->stage + 2 * bytes);
        GKBA_TRY(copy_in(c, (void*)dG, G, bytes, 0));
        GKBA_TRY(copy_in(c, (void*)dGb, Gbar, bytes, 0));
    }
    GKBA_TRY(sigma_dev(c, n_units, dG, dGb, dS));
    if (!on_device)
        GKBA_CUDA(c, cudaMemcpyAsync(S_out, dS, bytes, cudaMemcpyDeviceToHost, c->stream));
    return finish(c);
}

gkba_status gkba_collision(gkba_ctx* c, int L, const double* rho_hist, const double* T_hist,
                           const double* weights, double* I_out, int on_device) {
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_collision: NULL context");
    if (L < 1 || !rho_hist || !T_hist || !I_out)
        return fail(c, GKBA_EINVAL, "gkba_collision: need L >= 1 and non-NULL history and output");
    GKBA_CUDA(c, cudaSetDevice(c->device));
    const size_t NN = (size_t)c->N * c->N, hb = NN * 16 * (size_t)L;
    if (weights && !on_device) {
        for (int k = 0; k < L; ++k)
            if (!std::isfinite(weights[k])) return fail(c, GKBA_EINVAL, "gkba_collision: non-finite weight");
    }
    const double2 *dR, *dT;
    const double* dW = nullptr;
    double2* dI;
    const size_t wb = ((size_t)L * 8 + 255) & ~(size_t)255;
    if (on_device) {
        dR = (const double2*)rho_hist;
        dT = (const double2*)T_hist;
        dW = weights;
        dI = (double2*)I_out;
    } else {
        GKBA_TRY(ensure_stage(c, 2 * hb + wb + NN * 16));
        char* s = (char*)c->stage;
        dR = (double2*)s;
        dT = (double2*)(s + hb);
        double* w = (double*)(s + 2 * hb);
        dI = (double2*)(s + 2 * hb + wb);
        GKBA_TRY(copy_in(c, (void*)dR, rho_hist, hb, 0));
        GKBA_TRY(copy_in(c, (void*)dT, T_hist, hb, 0));
        if (weights) {
            GKBA_TRY(copy_in(c, w, weights, (size_t)L * 8, 0));
            dW = w;
        }
    }
    GKBA_TRY(collision_dev(c, L, dR, dT, dW, dI));
    if (!on_device)
        GKBA_CUDA(c, cudaMemcpyAsync(I_out, dI, NN * 16, cudaMemcpyDeviceToHost, c->stream));
    return finish(c);
}

// Buffers of dL/dv: the omega layout of v (FP64, or FP32 padded to Np on the
// tensor-core path) and three FP64 accumulators (v slot N x N^3, w slot
// N x N^3, natural N^4), zeroed.
static gkba_status prepare_vgrad(gkba_ctx* c) {
    const size_t N4 = (size_t)c->N * c->N * c->N * c->N;
    if (tensor_core_path(c)) {
        GKBA_TRY(tf32_prepare_vgrad(c));
    } else if (!c->vomega) {
        GKBA_TRY(alloc(c, (void**)&c->vomega, N4 * 8));
        GKBA_TRY(build_vomega64(c, c->vomega));
    }
    if (!c->vgrad) GKBA_TRY(alloc(c, (void**)&c->vgrad, 3 * N4 * 8));
    GKBA_CUDA(c, cudaMemsetAsync(c->vgrad, 0, 3 * N4 * 8, c->stream));
    return GKBA_OK;
}

gkba_status gkba_sigma3(gkba_ctx* c, int n_units, const double* A, const double* B,
                        const double* C, double* S_out, int on_device) {
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_sigma3: NULL context");
    if (n_units < 0 || (n_units > 0 && (!A || !B || !C || !S_out)))
        return fail(c, GKBA_EINVAL, "gkba_sigma3: bad arguments");
    if (c->kind != GKBA_V_GENERAL)
        return fail(c, GKBA_EUNSUPPORTED, "gkba_sigma3: general interaction only");
    if (n_units == 0) return GKBA_OK;
    GKBA_CUDA(c, cudaSetDevice(c->device));
    const size_t NN = (size_t)c->N * c->N, bytes = NN * 16 * (size_t)n_units;
    const double2 *dA, *dB, *dC;
    double2* dS;
    if (on_device) {
        dA = (const double2*)A;
        dB = (const double2*)B;
        dC = (const double2*)C;
        dS = (double2*)S_out;
    } else {
        GKBA_TRY(ensure_stage(c, 4 * bytes));
        char* st = (char*)c->stage;
        dA = (double2*)st;
        dB = (double2*)(st + bytes);
        dC = (double2*)(st + 2 * bytes);
        dS = (double2*)(st + 3 * bytes);
        GKBA_TRY(copy_in(c, (void*)dA, A, bytes, 0));
        GKBA_TRY(copy_in(c, (void*)dB, B, bytes, 0));
        GKBA_TRY(copy_in(c, (void*)dC, C, bytes, 0));
    }
    GKBA_TRY(sigma3_dev(c, n_units, dA, dB, dC, dS));
    if (!on_device)
        GKBA_CUDA(c, cudaMemcpyAsync(S_out, dS, bytes, cudaMemcpyDeviceToHost, c->stream));
    return finish(c);
}

gkba_status gkba_collision_vjp(gkba_ctx* c, int L, const double* rho_hist, const double* T_hist,
                               const double* weights, const double* I_bar, double* rho_bar,
                               double* T_bar, double* v_bar, int on_device) {
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_collision_vjp: NULL context");
    if (L < 1 || !rho_hist || !T_hist || !I_bar || !rho_bar || !T_bar)
        return fail(c, GKBA_EINVAL, "gkba_collision_vjp: need L >= 1 and non-NULL arrays");
    if (c->kind != GKBA_V_GENERAL)
        return fail(c, GKBA_EUNSUPPORTED, "gkba_collision_vjp: general interaction only");
    GKBA_CUDA(c, cudaSetDevice(c->device));
    const size_t NN = (size_t)c->N * c->N, hb = NN * 16 * (size_t)L;
    const size_t wb = ((size_t)L * 8 + 255) & ~(size_t)255;
    const double2 *dR, *dT, *dIb;
    const double* dW = nullptr;
    double2 *dRb, *dTb;
    if (on_device) {
        dR = (const double2*)rho_hist;
        dT = (const double2*)T_hist;
        dW = weights;
        dIb = (const double2*)I_bar;
        dRb = (double2*)rho_bar;
        dTb = (double2*)T_bar;
    } else {
        if (weights)
            for (int k = 0; k < L; ++k)
                if (!std::isfinite(weights[k]))
                    return fail(c, GKBA_EINVAL, "gkba_collision_vjp: non-finite weight");
        GKBA_TRY(ensure_stage(c, 4 * hb + wb + NN * 16));
        char* s = (char*)c->stage;
        dR = (double2*)s;
        dT = (double2*)(s + hb);
        dRb = (double2*)(s + 2 * hb);
        dTb = (double2*)(s + 3 * hb);
        double* w = (double*)(s + 4 * hb);
        dIb = (double2*)(s + 4 * hb + wb);
        GKBA_TRY(copy_in(c, (void*)dR, rho_hist, hb, 0));
        GKBA_TRY(copy_in(c, (void*)dT, T_hist, hb, 0));
        GKBA_TRY(copy_in(c, (void*)dIb, I_bar, NN * 16, 0));
        if (weights) {
            GKBA_TRY(copy_in(c, w, weights, (size_t)L * 8, 0));
            dW = w;
        }
    }
    const size_t N4 = NN * NN;
    double *vs = nullptr, *ws = nullptr;
    if (v_bar) {
        GKBA_TRY(prepare_vgrad(c));
        vs = c->vgrad;
        ws = c->vgrad + N4;
    }
    GKBA_TRY(collision_vjp_dev(c, L, dR, dT, dW, dIb, dRb, dTb, vs, ws));
    if (v_bar) {
        GKBA_TRY(fold_vbar(c, vs, ws, c->vgrad + 2 * N4));
        GKBA_CUDA(c, cudaMemcpyAsync(v_bar, c->vgrad + 2 * N4, N4 * 8,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                     c->stream));
    }
    if (!on_device) {
        GKBA_CUDA(c, cudaMemcpyAsync(rho_bar, dRb, hb, cudaMemcpyDeviceToHost, c->stream));
        GKBA_CUDA(c, cudaMemcpyAsync(T_bar, dTb, hb, cudaMemcpyDeviceToHost, c->stream));
    }
    return finish(c);
}

gkba_status gkba_mean_field(gkba_ctx* c, const double* rho, double* sigma_hf, int on_device) {
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_mean_field: NULL context");
    if (!rho || !sigma_hf) return fail(c, GKBA_EINVAL, "gkba_mean_field: NULL argument");
    GKBA_CUDA(c, cudaSetDevice(c->device));
    const size_t NN = (size_t)c->N * c->N;
    const double2* dR;
    double2* dO;
    if (on_device) {
        dR = (const double2*)rho;
        dO = (double2*)sigma_hf;
    } else {
        GKBA_TRY(ensure_stage(c, 2 * NN * 16));
        dR = (double2*)c->stage;
        dO = (double2*)((char*)c->stage + NN * 16);
        GKBA_TRY(copy_in(c, (void*)dR, rho, NN * 16, 0));
    }
    GKBA_TRY(mean_field(c, dR, dO));
    if (!on_device) GKBA_CUDA(c, cudaMemcpyAsync(sigma_hf, dO, NN * 16, cudaMemcpyDeviceToHost, c->stream));
    return finish(c);
}

gkba_status gkba_step(gkba_ctx* c, double E_n, double E_np1, double* rho_out, double* I_out,
                      double* diag_out) {
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_step: NULL context");
    if (!std::isfinite(E_n) || !std::isfinite(E_np1))
        return fail(c, GKBA_EINVAL, "gkba_step: non-finite field sample");
    if (c->n >= c->max_steps)
        return fail(c, GKBA_ESTATE, "gkba_step: history full (n=%d, max_steps=%d)", c->n, c->max_steps);
    const bool tl = c->history == GKBA_HISTORY_TIME_LINEAR;
    if (tl && c->tl_broken)
        return fail(c, GKBA_ESTATE,
                    "gkba_step: the time-linear accumulator was left inconsistent by a failed step; "
                    "gkba_set_history rebuilds it");
    GKBA_CUDA(c, cudaSetDevice(c->device));
    NvtxRange r("gkba_step");
    const int n = c->n;
    const long long NN = (long long)c->N * c->N;
    double2* rho_n = c->rho_hist + n * NN;
    double2* rho_t = c->rho_hist + (n + 1) * NN;
    // predictor
    GKBA_TRY(h_hf(c, E_n, rho_n, c->hhf_n));
    if (tl) {
        // Lambda of t_n = Lambda_acc + dt/2 term_n; then term_n joins Lambda_acc
        // with its final weight (dt/2 for t_0, dt after)
        c->tl_broken = true;  // until the step completes
        GKBA_TRY(ensure_workspace(c, 2));
        GKBA_TRY(tl_terms(c, 1, rho_n, c->tl_W, 0, 0, 1.0, 1.0));
        GKBA_TRY(tl_update(c, 0.5 * c->dt, n == 0 ? 0.5 * c->dt : c->dt, n > 0, true));
        if (n == 0)
            GKBA_CUDA(c, cudaMemsetAsync(c->Ia, 0, NN * sizeof(double2), c->stream));
        else
            GKBA_TRY(tl_apply(c, c->tl_W, c->Ia));
    } else {
        GKBA_TRY(collision_dev(c, n + 1, c->rho_hist, c->T_a, nullptr, c->Ia));
    }
    GKBA_TRY(diagnostics(c, E_n, rho_n, c->Ia, c->dscal));
    GKBA_TRY(rhs(c, c->hhf_n, rho_n, c->Ia, c->k1));
    GKBA_TRY(axpy_c(c, rho_t, rho_n, c->k1, 1.0, c->dt, (int)NN));
    GKBA_CUDA(c, cudaMemcpyAsync(c->rhot_hist + n * NN, rho_t, NN * 16, cudaMemcpyDeviceToDevice, c->stream));
    GKBA_TRY(h_hf(c, E_np1, rho_t, c->hhf_t));
    // propagator recursion T(t_{n+1}, t_k) = U_n T(t_n, t_k); T(t_{n+1}, t_{n+1}) = 1
    GKBA_TRY(expm_step(c, c->hhf_n, c->hhf_t, c->U));
    GKBA_CUDA(c, cudaMemcpyAsync(c->U_hist + n * NN, c->U, NN * 16, cudaMemcpyDeviceToDevice, c->stream));
    c->E_a[n] = E_n;
    c->E_b[n] = E_np1;
    GKBA_TRY(zgemm_batched(c, K_STEP, c->N, 'N', 'N', make_double2(1.0, 0.0), c->U, 0, c->T_a, NN,
                           make_double2(0.0, 0.0), c->T_b, NN, n + 1, 0));
    GKBA_TRY(set_identity(c, c->T_b + (n + 1) * NN, 1));
    // corrector
    if (tl) {
        // W_{n+1} = Ucal_{n+1}^+ = W_n U_n^+; Lambda = Lambda_acc + dt/2 term(rho~)
        GKBA_TRY(zgemm_batched(c, K_STEP, c->N, 'N', 'C', make_double2(1.0, 0.0), c->tl_W, 0, c->U,
                               0, make_double2(0.0, 0.0), c->tl_Wn, 0, 1, 0));
        GKBA_TRY(tl_terms(c, 1, rho_t, c->tl_Wn, 0, 0, 1.0, 1.0));
        GKBA_TRY(tl_update(c, 0.5 * c->dt, 0.0, true, false));
        GKBA_TRY(tl_apply(c, c->tl_Wn, c->Ib));
    } else {
        GKBA_TRY(collision_dev(c, n + 2, c->rho_hist, c->T_b, nullptr, c->Ib));
    }
    GKBA_TRY(rhs(c, c->hhf_t, rho_t, c->Ib, c->k2));
    GKBA_TRY(axpy_c(c, c->k2, c->k1, c->k2, 1.0, 1.0, (int)NN));
    GKBA_TRY(axpy_c(c, rho_t, rho_n, c->k2, 1.0, 0.5 * c->dt, (int)NN));
    std::swap(c->T_a, c->T_b);
    if (tl) std::swap(c->tl_W, c->tl_Wn);
    c->n = n + 1;
    if (rho_out)
        GKBA_CUDA(c, cudaMemcpyAsync(rho_out, rho_t, NN * 16, cudaMemcpyDeviceToHost, c->stream));
    if (I_out) GKBA_CUDA(c, cudaMemcpyAsync(I_out, c->Ia, NN * 16, cudaMemcpyDeviceToHost, c->stream));
    if (diag_out) GKBA_CUDA(c, cudaMemcpyAsync(c->hdiag, c->dscal, 4 * 8, cudaMemcpyDeviceToHost, c->stream));
    GKBA_TRY(finish(c));
    if (diag_out) memcpy(diag_out, c->hdiag, 4 * 8);
    c->tl_broken = false;
    return GKBA_OK;
}

gkba_status gkba_set_history(gkba_ctx* c, int n, const double* rho_hist, const double* T_hist,
                             int on_device) {
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_set_history: NULL context");
    if (n < 0 || n > c->max_steps || !rho_hist || !T_hist)
        return fail(c, GKBA_EINVAL, "gkba_set_history: n=%d outside [0, max_steps=%d] or NULL", n,
                    c->max_steps);
    GKBA_CUDA(c, cudaSetDevice(c->device));
    const long long NN = (long long)c->N * c->N;
    const size_t bytes = (size_t)(n + 1) * NN * 16;
    GKBA_TRY(copy_in(c, c->rho_hist, rho_hist, bytes, on_device));
    GKBA_TRY(copy_in(c, c->T_a, T_hist, bytes, on_device));
    if (c->history == GKBA_HISTORY_TIME_LINEAR) {
        // Ucal_n = 1 and Ucal_k^+ = T(t_n, t_k): needs T(t_n, t_n) = 1
        std::vector<double> Tn(2 * NN);
        GKBA_CUDA(c, cudaMemcpyAsync(Tn.data(), c->T_a + (size_t)n * NN, NN * 16,
                                     cudaMemcpyDeviceToHost, c->stream));
        GKBA_CUDA(c, cudaStreamSynchronize(c->stream));
        double dev = 0.0;
        for (long long e = 0; e < NN; ++e) {
            const double re = Tn[2 * e] - ((e / c->N == e % c->N) ? 1.0 : 0.0);
            dev = std::max(dev, std::hypot(re, Tn[2 * e + 1]));
        }
        if (!(dev <= 1e-12))
            return fail(c, GKBA_EINVAL,
                        "gkba_set_history: T(t_n, t_n) must be the identity (max deviation %.3g)", dev);
        c->tl_broken = true;
        GKBA_CUDA(c, cudaMemsetAsync(c->tl_acc, 0, 2 * (size_t)NN * NN * 8, c->stream));
        GKBA_TRY(set_identity(c, c->tl_W, 1));
        if (n > 0) {
            // Lambda_acc = sum_{k < n} c_k term_k, c_0 = dt/2, c_k = dt
            GKBA_TRY(ensure_workspace(c, 2 * n));
            const int nk_per = c->ub / 2;
            for (int k0 = 0; k0 < n; k0 += nk_per) {
                const int nk = std::min(nk_per, n - k0);
                GKBA_TRY(tl_terms(c, nk, c->rho_hist + (size_t)k0 * NN, c->T_a + (size_t)k0 * NN, NN,
                                  k0, 0.5 * c->dt, c->dt));
                GKBA_TRY(tl_update(c, 0.0, 1.0, false, true));
            }
        }
    }
    c->n = n;
    c->adj_from = n;  // steps before n were not recorded
    GKBA_TRY(finish(c));
    c->tl_broken = false;
    return GKBA_OK;
}

gkba_status gkba_get_history(const gkba_ctx* cc, int* n, double* rho_hist, double* T_hist) {
    gkba_ctx* c = const_cast<gkba_ctx*>(cc);
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_get_history: NULL context");
    GKBA_CUDA(c, cudaSetDevice(c->device));
    if (n) *n = c->n;
    const size_t bytes = (size_t)(c->n + 1) * c->N * c->N * 16;
    if (rho_hist) GKBA_CUDA(c, cudaMemcpyAsync(rho_hist, c->rho_hist, bytes, cudaMemcpyDeviceToHost, c->stream));
    if (T_hist) GKBA_CUDA(c, cudaMemcpyAsync(T_hist, c->T_a, bytes, cudaMemcpyDeviceToHost, c->stream));
    GKBA_CUDA(c, cudaStreamSynchronize(c->stream));
    return GKBA_OK;
}

gkba_status gkba_get_state(const gkba_ctx* cc, int* n, double* rho) {
    gkba_ctx* c = const_cast<gkba_ctx*>(cc);
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_get_state: NULL context");
    GKBA_CUDA(c, cudaSetDevice(c->device));
    if (n) *n = c->n;
    if (rho) {
        const size_t NN = (size_t)c->N * c->N;
        GKBA_CUDA(c, cudaMemcpyAsync(rho, c->rho_hist + c->n * NN, NN * 16, cudaMemcpyDeviceToHost, c->stream));
        GKBA_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return GKBA_OK;
}

gkba_status gkba_adjoint(gkba_ctx* c, const double* rho_bar_final, double* E_bar, double* rho0_bar,
                         double* v_bar) {
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_adjoint: NULL context");
    if (!rho_bar_final || !E_bar) return fail(c, GKBA_EINVAL, "gkba_adjoint: NULL argument");
    if (c->kind != GKBA_V_GENERAL)
        return fail(c, GKBA_EUNSUPPORTED, "gkba_adjoint: general interaction only");
    if (c->adj_from != 0)
        return fail(c, GKBA_EUNSUPPORTED,
                    "gkba_adjoint: the trajectory must start at gkba_init or gkba_set_history(0, ...)");
    GKBA_CUDA(c, cudaSetDevice(c->device));
    NvtxRange nr("gkba_adjoint");
    const int M = c->n, N = c->N;
    const long long NN = (long long)N * N;
    const size_t H = (size_t)(M + 2) * NN;  // one history-sized block
    const size_t need = (7 * H + 12 * NN + 16 * NN) * sizeof(double2) + (size_t)(M + 1) * 8 + 256;
    if (c->adj_ws_bytes < need) {
        if (c->adj_ws) cudaFree(c->adj_ws);
        c->adj_ws = nullptr;
        c->adj_ws_bytes = 0;
        if (cudaMalloc(&c->adj_ws, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, GKBA_ENOMEM, "gkba_adjoint: %zu bytes of backward buffers do not fit", need);
        }
        c->adj_ws_bytes = need;
    }
    double2* base = c->adj_ws;
    double2 *Rb = base, *Tcur = base + H, *Tprv = base + 2 * H, *Tb = base + 3 * H,
            *srho = base + 4 * H, *sT = base + 5 * H, *prod = base + 6 * H;
    double2* sm = base + 7 * H;
    double2 *kb = sm, *kb1 = sm + NN, *hA = sm + 2 * NN, *hB = sm + 3 * NN, *hAb = sm + 4 * NN,
            *hBb = sm + 5 * NN, *rtb = sm + 6 * NN, *Ib = sm + 7 * NN, *P1 = sm + 8 * NN,
            *P2 = sm + 9 * NN, *Ub = sm + 10 * NN, *save = sm + 11 * NN;
    double2* fre = sm + 12 * NN;  // 4 (2N)^2 blocks = 16 NN
    double* Eb = (double*)(fre + 16 * NN);
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    const double dt = c->dt;
    GKBA_CUDA(c, cudaMemsetAsync(Rb, 0, H * sizeof(double2), c->stream));
    GKBA_CUDA(c, cudaMemsetAsync(Tb, 0, H * sizeof(double2), c->stream));
    GKBA_CUDA(c, cudaMemsetAsync(Eb, 0, (size_t)(M + 1) * 8, c->stream));
    GKBA_TRY(copy_in(c, Rb + (size_t)M * NN, rho_bar_final, NN * 16, 0));
    const size_t N4 = (size_t)NN * NN;
    double *vs = nullptr, *ws = nullptr, *vn = nullptr;
    if (v_bar) {
        GKBA_TRY(prepare_vgrad(c));
        vs = c->vgrad;
        ws = c->vgrad + N4;
        vn = c->vgrad + 2 * N4;
    }
    GKBA_CUDA(c, cudaMemcpyAsync(Tcur, c->T_a, (size_t)(M + 1) * NN * 16, cudaMemcpyDeviceToDevice,
                                 c->stream));
    for (int n = M - 1; n >= 0; --n) {
        const double2* rho_n = c->rho_hist + (size_t)n * NN;
        const double2* rho_t = c->rhot_hist + (size_t)n * NN;
        const double2* U = c->U_hist + (size_t)n * NN;
        double2* Rn = Rb + (size_t)n * NN;
        double2* Rn1 = Rb + (size_t)(n + 1) * NN;
        GKBA_TRY(h_hf(c, c->E_a[n], rho_n, hA));
        GKBA_TRY(h_hf(c, c->E_b[n], rho_t, hB));
        // T(t_n, t_k) = U^+ T(t_{n+1}, t_k), k <= n (U unitary)
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'C', 'N', one, U, 0, Tcur, NN, zero, Tprv, NN, n + 1, 0));
        // rho_{n+1} = rho_n + dt/2 (k1 + k2)
        GKBA_TRY(axpy_c(c, kb, Rn1, Rn1, 0.5 * dt, 0.0, (int)NN));
        GKBA_TRY(axpy_c(c, Rn, Rn, Rn1, 1.0, 1.0, (int)NN));
        // k2 = -i[hB, rho~] - (I~ + I~^+)
        GKBA_CUDA(c, cudaMemsetAsync(hAb, 0, 4 * NN * sizeof(double2), c->stream));  // hAb hBb rtb Ib
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'C', one, kb, 0, rho_t, 0, zero, P1, 0, 1, 0));
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'C', 'N', one, rho_t, 0, kb, 0, zero, P2, 0, 1, 0));
        GKBA_TRY(add_i_diff(c, hBb, P1, P2, 1.0));
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'N', one, hB, 0, kb, 0, zero, P1, 0, 1, 0));
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'N', one, kb, 0, hB, 0, zero, P2, 0, 1, 0));
        GKBA_TRY(add_i_diff(c, rtb, P1, P2, 1.0));
        GKBA_TRY(ibar_from_kbar(c, kb, Ib));
        // corrector collision over rho_0 .. rho_n, rho~ with T(t_{n+1}, .)
        double2* slot = c->rho_hist + (size_t)(n + 1) * NN;
        GKBA_CUDA(c, cudaMemcpyAsync(save, slot, NN * 16, cudaMemcpyDeviceToDevice, c->stream));
        GKBA_CUDA(c, cudaMemcpyAsync(slot, rho_t, NN * 16, cudaMemcpyDeviceToDevice, c->stream));
        gkba_status st = collision_vjp_dev(c, n + 2, c->rho_hist, Tcur, nullptr, Ib, srho, sT, vs, ws);
        GKBA_CUDA(c, cudaMemcpyAsync(slot, save, NN * 16, cudaMemcpyDeviceToDevice, c->stream));
        GKBA_TRY(st);
        GKBA_TRY(axpy_c(c, Rb, Rb, srho, 1.0, 1.0, (int)((n + 1) * NN)));
        GKBA_TRY(axpy_c(c, rtb, rtb, srho + (size_t)(n + 1) * NN, 1.0, 1.0, (int)NN));
        GKBA_TRY(axpy_c(c, Tb, Tb, sT, 1.0, 1.0, (int)((n + 2) * NN)));
        // T(t_{n+1}, t_k) = U T(t_n, t_k): Ubar = sum_k Tbar_k T(t_n, t_k)^+, Tbar_k <- U^+ Tbar_k
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'C', one, Tb, NN, Tprv, NN, zero, prod, NN, n + 1, 0));
        GKBA_TRY(sum_units(c, n + 1, prod, Ub));
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'C', 'N', one, U, 0, Tb, NN, zero, prod, NN, n + 1, 0));
        GKBA_CUDA(c, cudaMemcpyAsync(Tb, prod, (size_t)(n + 1) * NN * 16, cudaMemcpyDeviceToDevice, c->stream));
        GKBA_CUDA(c, cudaMemsetAsync(Tb + (size_t)(n + 1) * NN, 0, NN * 16, c->stream));
        // U = exp(-i dt (hA + hB)/2)
        GKBA_TRY(expm_adj(c, hA, hB, Ub, hAb, hBb, fre));
        // hB = h + E_{n+1} d + Sigma_HF(rho~)
        GKBA_TRY(field_grad(c, hBb, Eb + n + 1));
        if (vn) GKBA_TRY(vbar_mean_field(c, hBb, rho_t, vn));
        GKBA_TRY(mean_field_adj(c, hBb, rtb));
        // rho~ = rho_n + dt k1
        GKBA_TRY(axpy_c(c, Rn, Rn, rtb, 1.0, 1.0, (int)NN));
        GKBA_TRY(axpy_c(c, kb1, kb, rtb, 1.0, dt, (int)NN));
        // k1 = -i[hA, rho_n] - (I_n + I_n^+)
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'C', one, kb1, 0, rho_n, 0, zero, P1, 0, 1, 0));
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'C', 'N', one, rho_n, 0, kb1, 0, zero, P2, 0, 1, 0));
        GKBA_TRY(add_i_diff(c, hAb, P1, P2, 1.0));
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'N', one, hA, 0, kb1, 0, zero, P1, 0, 1, 0));
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'N', one, kb1, 0, hA, 0, zero, P2, 0, 1, 0));
        GKBA_TRY(add_i_diff(c, Rn, P1, P2, 1.0));
        GKBA_TRY(ibar_from_kbar(c, kb1, Ib));
        // collision over rho_0 .. rho_n with T(t_n, .)
        GKBA_TRY(collision_vjp_dev(c, n + 1, c->rho_hist, Tprv, nullptr, Ib, srho, sT, vs, ws));
        GKBA_TRY(axpy_c(c, Rb, Rb, srho, 1.0, 1.0, (int)((n + 1) * NN)));
        GKBA_TRY(axpy_c(c, Tb, Tb, sT, 1.0, 1.0, (int)((n + 1) * NN)));
        // hA = h + E_n d + Sigma_HF(rho_n)
        GKBA_TRY(field_grad(c, hAb, Eb + n));
        if (vn) GKBA_TRY(vbar_mean_field(c, hAb, rho_n, vn));
        GKBA_TRY(mean_field_adj(c, hAb, Rn));
        std::swap(Tcur, Tprv);
    }
    GKBA_CUDA(c, cudaMemcpyAsync(E_bar, Eb, (size_t)(M + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    if (v_bar) {
        GKBA_TRY(fold_vbar(c, vs, ws, vn));
        GKBA_CUDA(c, cudaMemcpyAsync(v_bar, vn, N4 * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    if (rho0_bar)
        GKBA_CUDA(c, cudaMemcpyAsync(rho0_bar, Rb, NN * 16, cudaMemcpyDeviceToHost, c->stream));
    return finish(c);
}

gkba_status gkba_get_stats(gkba_ctx* c, gkba_kernel_stat* stats, int max_stats, int* n_stats,
                           long long* total_launches, int reset) {
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_get_stats: NULL context");
    GKBA_TRY(harvest_timing(c));
    const int n = std::min(max_stats, (int)K_COUNT);
    for (int i = 0; stats && i < n; ++i) {
        stats[i].name = kKernelClassNames[i];
        stats[i].launches = c->cls_launches[i];
        stats[i].ms = c->cls_ms[i];
        stats[i].flops = c->cls_flops[i];
        stats[i].bytes = c->cls_bytes[i];
    }
    if (n_stats) *n_stats = stats ? n : 0;
    if (total_launches) *total_launches = c->launches;
    if (reset) {
        c->launches = 0;
        for (int i = 0; i < K_COUNT; ++i) {
            c->cls_launches[i] = 0;
            c->cls_ms[i] = c->cls_flops[i] = c->cls_bytes[i] = 0.0;
        }
    }
    return GKBA_OK;
}

gkba_status gkba_selftest_timeout(gkba_ctx* c, double limit_ms, double* elapsed_ms) {
    if (!c) return fail(nullptr, GKBA_EINVAL, "gkba_selftest_timeout: NULL context");
    if (!(limit_ms > 0.0) || limit_ms > 1000.0)
        return fail(c, GKBA_EINVAL, "gkba_selftest_timeout: limit_ms must be in (0, 1000]");
    GKBA_CUDA(c, cudaSetDevice(c->device));
    GKBA_TRY(wait_selftest(c, limit_ms, elapsed_ms));
    return finish(c);  // reads the error word the expired wait wrote: GKBA_ETIMEOUT
}

gkba_status gkba_measure_tf32_mma(gkba_ctx* c, int iters, double* tflops) {
    if (!c || !tflops) return fail(c, GKBA_EINVAL, "gkba_measure_tf32_mma: NULL argument");
    if (iters < 16 || iters > 100000000)
        return fail(c, GKBA_EINVAL, "gkba_measure_tf32_mma: iters=%d must be in [16, 1e8]", iters);
    GKBA_CUDA(c, cudaSetDevice(c->device));
    GKBA_TRY(measure_tf32_mma(c, iters, tflops));
    return finish(c);
}

const char* gkba_last_error(const gkba_ctx* c) {
    if (c) return c->err.c_str();
    std::lock_guard<std::mutex> g(g_err_mu);
    return g_last_init_error.c_str();
}

void gkba_destroy(gkba_ctx* c) { free_ctx(c); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Stacked batches of systems (many systems of uneven N and history length).
// Systems of the same N form a group; the (t_k, component) units of all
// systems of a group are stacked into shared launches of the contraction
// kernels.  Per system only the w layout (S1's A) and the v layout (S4's B)
// differ; both sit in group buffers [system][...] that the kernels index with
// a per-unit system table.  Each system's units are padded with zero units
// (G = Gbar = 0, coefficient 0) to a multiple of 256 / gcd(256, 2 Np) so that
// no 256-row group of S4 straddles two systems.
// ---------------------------------------------------------------------------
constexpr int kMaxBatchLaunchGroups = 8;  // groups per stage launch (the kernels' limit)

struct gkba_batch {
    int device = -1;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<gkba_ctx*> ctx;  // members (owned by the caller)
    struct Group {
        int N = 0;
        std::vector<int> members;  // indices into ctx
        gkba_ctx* sh = nullptr;    // workspace, group layouts and stream of the group
        int pu = 1;                // unit padding quantum
        int* sys_dev = nullptr;    // unit -> system (group-local index), per collision
        int* sys_host[2] = {nullptr, nullptr};  // pinned staging, one per collision of a step
        long long sys_cap = 0;
        // autotuner record (gkba_batch_autotune)
        double us_per_unit = 0.0;
    };
    std::vector<Group> groups;
    bool use_graph = false;          // gkba_batch_set_options
    cudaGraphExec_t gexec = nullptr; // the last step's executable graph (updated in place)
    long long graph_steps = 0, graph_rebuilds = 0;
};

namespace {

gkba_status batch_fail(gkba_batch* b, gkba_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    std::lock_guard<std::mutex> g(g_err_mu);
    g_last_init_error = buf;
    return st;
}

void free_batch(gkba_batch* b) {
    if (!b) return;
    if (b->device >= 0) cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto& g : b->groups) {
        if (g.sys_dev) cudaFree(g.sys_dev);
        for (int i = 0; i < 2; ++i)
            if (g.sys_host[i]) cudaFreeHost(g.sys_host[i]);
        if (g.sh) {
            g.sh->stream = nullptr;  // the batch's stream, destroyed below
            free_ctx(g.sh);
        }
    }
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// The stacked (t_k, component) units of one collision of every member, per
// group: each member's units padded to the group's quantum, a unit -> system
// table on the device.
struct CollisionPlan {
    struct Seg {
        gkba_ctx* c;
        int L;
        const double2* T;
        double2* I;
        long long u0;   // first unit in the group's stacked list
        long long nu;   // real units 2 L
        long long np;   // padded units
    };
    std::vector<std::vector<Seg>> segs;
    std::vector<long long> total;
    std::vector<int*> dev;
};

// Collision `which` of a step: L = n + 1 points with T = T_a (into Ia), or
// n + 2 points with T = T_b (into Ib).  Zeroes the members' I.
gkba_status plan_collision(gkba_batch* b, int which, CollisionPlan& P, bool zero_I = true) {
    const int G = (int)b->groups.size();
    P.segs.assign(G, {});
    P.total.assign(G, 0);
    P.dev.assign(G, nullptr);
    for (int gi = 0; gi < G; ++gi) {
        gkba_batch::Group& g = b->groups[gi];
        gkba_ctx* sh = g.sh;
        const long long NN = (long long)g.N * g.N;
        for (int m : g.members) {
            gkba_ctx* c = b->ctx[m];
            CollisionPlan::Seg sg;
            sg.c = c;
            sg.L = which == 0 ? c->n + 1 : c->n + 2;
            sg.T = which == 0 ? c->T_a : c->T_b;
            sg.I = which == 0 ? c->Ia : c->Ib;
            sg.u0 = P.total[gi];
            sg.nu = 2LL * sg.L;
            sg.np = ((sg.nu + g.pu - 1) / g.pu) * g.pu;
            P.total[gi] += sg.np;
            if (zero_I) GKBA_CUDA(sh, cudaMemsetAsync(sg.I, 0, NN * sizeof(double2), sh->stream));
            P.segs[gi].push_back(sg);
        }
        const long long total = P.total[gi];
        if (total > g.sys_cap) {
            if (g.sys_dev) cudaFree(g.sys_dev);
            for (int i = 0; i < 2; ++i)
                if (g.sys_host[i]) cudaFreeHost(g.sys_host[i]);
            g.sys_dev = nullptr;
            g.sys_host[0] = g.sys_host[1] = nullptr;
            g.sys_cap = 0;
            // one device table per collision of a step (the first may still be read)
            if (cudaMalloc(&g.sys_dev, 2 * total * sizeof(int)) != cudaSuccess ||
                cudaMallocHost(&g.sys_host[0], total * sizeof(int)) != cudaSuccess ||
                cudaMallocHost(&g.sys_host[1], total * sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                return fail(sh, GKBA_ENOMEM, "batch: unit table allocation failed");
            }
            g.sys_cap = total;
        }
        int* host = g.sys_host[which];
        P.dev[gi] = g.sys_dev + (long long)which * g.sys_cap;
        for (size_t i = 0; i < P.segs[gi].size(); ++i)
            for (long long u = 0; u < P.segs[gi][i].np; ++u) host[P.segs[gi][i].u0 + u] = (int)i;
        GKBA_CUDA(sh, cudaMemcpyAsync(P.dev[gi], host, total * sizeof(int), cudaMemcpyHostToDevice,
                                      sh->stream));
    }
    return GKBA_OK;
}

// Grow every group's unit tables to the larger collision of the coming step
// (n + 2 points per member) before a graph capture, so that none is
// allocated while the stream is captured.
gkba_status ensure_tables(gkba_batch* b) {
    for (auto& g : b->groups) {
        long long total = 0;
        for (int m : g.members)
            total += ((2LL * (b->ctx[m]->n + 2) + g.pu - 1) / g.pu) * g.pu;
        if (total <= g.sys_cap) continue;
        if (g.sys_dev) cudaFree(g.sys_dev);
        for (int i = 0; i < 2; ++i)
            if (g.sys_host[i]) cudaFreeHost(g.sys_host[i]);
        g.sys_dev = nullptr;
        g.sys_host[0] = g.sys_host[1] = nullptr;
        g.sys_cap = 0;
        if (cudaMalloc(&g.sys_dev, 2 * total * sizeof(int)) != cudaSuccess ||
            cudaMallocHost(&g.sys_host[0], total * sizeof(int)) != cudaSuccess ||
            cudaMallocHost(&g.sys_host[1], total * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return fail(g.sh, GKBA_ENOMEM, "batch: unit table allocation failed");
        }
        g.sys_cap = total;
    }
    return GKBA_OK;
}

// Units per round of group g: the workspace's, or the autotuner's choice.
long long round_units(const gkba_batch::Group& g) {
    const gkba_ctx* sh = g.sh;
    return sh->ub_limit > 0 ? std::min(sh->ub, sh->ub_limit) : sh->ub;
}

// Stage units [U0, U0 + nb) of group gi in its workspace (G, Gbar, weights,
// forms) and point its unit table at them.
gkba_status stage_round(gkba_batch* b, int gi, const CollisionPlan& P, long long U0, long long nb) {
    gkba_batch::Group& g = b->groups[gi];
    gkba_ctx* sh = g.sh;
    const int N = g.N;
    const long long NN = (long long)N * N;
    for (const auto& sg : P.segs[gi]) {
        const long long a = std::max(U0, sg.u0), e = std::min(U0 + nb, sg.u0 + sg.np);
        if (a >= e) continue;
        const long long ra = a - sg.u0, re = e - sg.u0;  // units of this system in the batch
        const long long off = a - U0;                    // their offset in the batch
        const long long real_end = std::min(re, sg.nu);
        if (ra < real_end) {
            const int k0 = (int)(ra / 2), nk = (int)((real_end - ra) / 2);
            GKBA_TRY(units_from_history(sh, N, k0, nk, sg.L, sg.c->dt, sg.c->rho_hist, sg.T, nullptr,
                                        sh->Su + off * NN, sh->Mb + off * NN, sh->coef + off));
        }
        const long long pad0 = std::max(ra, sg.nu);
        if (pad0 < re) {
            const long long po = off + (pad0 - ra), pn = re - pad0;
            GKBA_CUDA(sh, cudaMemsetAsync(sh->Su + po * NN, 0, pn * NN * sizeof(double2), sh->stream));
            GKBA_CUDA(sh, cudaMemsetAsync(sh->Mb + po * NN, 0, pn * NN * sizeof(double2), sh->stream));
            GKBA_CUDA(sh, cudaMemsetAsync(sh->coef + po, 0, pn * sizeof(double), sh->stream));
        }
    }
    GKBA_TRY(build_forms_tf32(sh, (int)nb, sh->Su, sh->Mb));
    sh->unit_sys = P.dev[gi] + U0;
    return GKBA_OK;
}

// Collision integrals of every member of every group over its own history.
// The groups advance together in rounds: in each round every group with
// units left stages its next batch, and one launch per stage covers the
// batches of all of them (contract_batch_tf32_multi).
gkba_status batch_collision(gkba_batch* b, int which) {
    NvtxRange nr("gkba batch collision");
    CollisionPlan P;
    GKBA_TRY(plan_collision(b, which, P));
    const int G = (int)b->groups.size();
    std::vector<long long> U0(G, 0);
    for (;;) {
        std::vector<int> act;
        for (int gi = 0; gi < G; ++gi)
            if (U0[gi] < P.total[gi]) act.push_back(gi);
        if (act.empty()) break;
        for (size_t a0 = 0; a0 < act.size(); a0 += kMaxBatchLaunchGroups) {
            const int na = (int)std::min<size_t>(kMaxBatchLaunchGroups, act.size() - a0);
            gkba_ctx* cs[kMaxBatchLaunchGroups];
            int nbs[kMaxBatchLaunchGroups];
            for (int k = 0; k < na; ++k) {
                const int gi = act[a0 + k];
                const long long nb = std::min(round_units(b->groups[gi]), P.total[gi] - U0[gi]);
                GKBA_TRY(stage_round(b, gi, P, U0[gi], nb));
                cs[k] = b->groups[gi].sh;
                nbs[k] = (int)nb;
            }
            const gkba_status st = contract_batch_tf32_multi(cs, nbs, na);
            for (int k = 0; k < na; ++k) cs[k]->unit_sys = nullptr;
            GKBA_TRY(st);
            for (int k = 0; k < na; ++k) {
                const int gi = act[a0 + k];
                gkba_ctx* sh = cs[k];
                const int N = b->groups[gi].N;
                const long long NN = (long long)N * N;
                const long long nb = nbs[k];
                GKBA_TRY(zgemm_batched(sh, K_RED, N, 'N', 'N', make_double2(1.0, 0.0), sh->Su, NN, sh->Mb,
                                       NN, make_double2(0.0, 0.0), sh->Yu, NN, (int)nb, 0));
                for (const auto& sg : P.segs[gi]) {
                    const long long a = std::max(U0[gi], sg.u0), e = std::min(U0[gi] + nb, sg.u0 + sg.nu);
                    if (a >= e) continue;
                    GKBA_TRY(weighted_sum_units(sh, N, (int)(e - a), sh->coef + (a - U0[gi]),
                                                sh->Yu + (a - U0[gi]) * NN, sg.I));
                }
                U0[gi] += nb;
            }
        }
    }
    return GKBA_OK;
}

// Device time per unit of one contraction round of group gi at the group's
// current parameters: nb units of the plan, staged once, contracted twice
// (the second run timed with events on the batch stream).
gkba_status tune_round(gkba_batch* b, int gi, const CollisionPlan& P, long long nb, double* us_per_unit) {
    gkba_ctx* sh = b->groups[gi].sh;
    GKBA_TRY(stage_round(b, gi, P, 0, nb));
    gkba_status st = contract_batch_tf32(sh, (int)nb);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == GKBA_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        cudaGetLastError();
        st = fail(sh, GKBA_ECUDA, "autotune: event creation failed");
    }
    if (st == GKBA_OK) {
        cudaEventRecord(e0, sh->stream);
        st = contract_batch_tf32(sh, (int)nb);
        cudaEventRecord(e1, sh->stream);
    }
    sh->unit_sys = nullptr;
    float ms = 0.0f;
    if (st == GKBA_OK) {
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            st = fail(sh, GKBA_ECUDA, "autotune: timing failed");
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    GKBA_TRY(st);
    *us_per_unit = 1e3 * ms / (double)nb;
    return GKBA_OK;
}

// Per group, a coordinate search over the launch parameters that change
// neither the result beyond the split-TF32 tolerance nor the memory held:
// the S4 work-item length (4096, 8192, 16384 K; fewer partial sums, fewer
// and longer items), the accumulation window of the windowed stage kernel
// (8 or 16 K, both within the tolerance), then the units per round (from
// the workspace's down by halves while the stage launches keep two 256-row
// tiles per cluster; smaller rounds keep the intermediates in L2).  A
// candidate replaces the incumbent only when it is at least kTuneGain faster
// per unit (timing noise does not move the choice).
constexpr double kTuneGain = 0.03;

gkba_status autotune(gkba_batch* b) {
    CollisionPlan P;
    GKBA_TRY(plan_collision(b, 0, P, false));
    for (int gi = 0; gi < (int)b->groups.size(); ++gi) {
        gkba_batch::Group& g = b->groups[gi];
        gkba_ctx* sh = g.sh;
        const long long Np = sh->Np, N3 = Np * Np * Np;
        const long long n0 = std::min<long long>(sh->ub, (P.total[gi] / g.pu) * g.pu);
        if (n0 < g.pu) continue;
        sh->ub_limit = 0;
        double best = 0.0;
        GKBA_TRY(tune_round(b, gi, P, n0, &best));
        // S4 work-item length
        if (N3 > kTcItemK) {
            int best_kw = sh->fin_kw;
            for (int kw : {kTcItemK, 2 * kTcItemK, 4 * kTcItemK}) {
                if (kw == best_kw || kw > 2 * N3) continue;
                const int keep = sh->fin_kw;
                sh->fin_kw = kw;
                double t = 0.0;
                GKBA_TRY(tune_round(b, gi, P, n0, &t));
                if (t < best * (1.0 - kTuneGain)) {
                    best = t;
                    best_kw = kw;
                } else {
                    sh->fin_kw = keep;
                }
            }
            sh->fin_kw = best_kw;
        }
        // accumulation window of the windowed stage kernel (2 Np <= 96)
        if (2 * Np <= 96) {
            const int keep = sh->acc_window;
            const int other = keep == 8 ? 16 : 8;
            sh->acc_window = other;
            double t = 0.0;
            GKBA_TRY(tune_round(b, gi, P, n0, &t));
            if (t < best * (1.0 - kTuneGain)) best = t;
            else sh->acc_window = keep;
        }
        // units per round
        // two 256-row tiles per cluster at least: nb Np^3 / 256 >= 2 clusters
        const long long need = (2LL * sh->pair_clusters * 256 + N3 - 1) / N3;
        const long long min_units = std::max<long long>(g.pu, (need + g.pu - 1) / g.pu * g.pu);
        long long best_nb = n0;
        for (long long nb = ((n0 / 2) / g.pu) * g.pu; nb >= min_units; nb = ((nb / 2) / g.pu) * g.pu) {
            double t = 0.0;
            GKBA_TRY(tune_round(b, gi, P, nb, &t));
            if (t < best * (1.0 - kTuneGain)) {
                best = t;
                best_nb = nb;
            }
            if (nb == g.pu) break;
        }
        sh->ub_limit = best_nb < sh->ub ? (int)best_nb : 0;
        g.us_per_unit = best;
    }
    return GKBA_OK;
}

// One Heun step of every member (the sequence of gkba_step, with both
// collision integrals of all members evaluated in stacked launches).
gkba_status batch_step(gkba_batch* b, const double* E_n, const double* E_np1,
                       double* const* rho_out, double* const* diag_out) {
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        gkba_ctx* c = b->ctx[i];
        const long long NN = (long long)c->N * c->N;
        GKBA_TRY(h_hf(c, E_n[i], c->rho_hist + c->n * NN, c->hhf_n));
    }
    GKBA_TRY(batch_collision(b, 0));
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        gkba_ctx* c = b->ctx[i];
        const int n = c->n;
        const long long NN = (long long)c->N * c->N;
        double2* rho_n = c->rho_hist + n * NN;
        double2* rho_t = c->rho_hist + (n + 1) * NN;
        GKBA_TRY(diagnostics(c, E_n[i], rho_n, c->Ia, c->dscal));
        GKBA_TRY(rhs(c, c->hhf_n, rho_n, c->Ia, c->k1));
        GKBA_TRY(axpy_c(c, rho_t, rho_n, c->k1, 1.0, c->dt, (int)NN));
        GKBA_CUDA(c, cudaMemcpyAsync(c->rhot_hist + n * NN, rho_t, NN * 16, cudaMemcpyDeviceToDevice,
                                     c->stream));
        GKBA_TRY(h_hf(c, E_np1[i], rho_t, c->hhf_t));
        GKBA_TRY(expm_step(c, c->hhf_n, c->hhf_t, c->U));
        GKBA_CUDA(c, cudaMemcpyAsync(c->U_hist + n * NN, c->U, NN * 16, cudaMemcpyDeviceToDevice,
                                     c->stream));
        c->E_a[n] = E_n[i];
        c->E_b[n] = E_np1[i];
        GKBA_TRY(zgemm_batched(c, K_STEP, c->N, 'N', 'N', make_double2(1.0, 0.0), c->U, 0, c->T_a,
                               NN, make_double2(0.0, 0.0), c->T_b, NN, n + 1, 0));
        GKBA_TRY(set_identity(c, c->T_b + (n + 1) * NN, 1));
    }
    GKBA_TRY(batch_collision(b, 1));
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        gkba_ctx* c = b->ctx[i];
        const int n = c->n;
        const long long NN = (long long)c->N * c->N;
        double2* rho_n = c->rho_hist + n * NN;
        double2* rho_t = c->rho_hist + (n + 1) * NN;
        GKBA_TRY(rhs(c, c->hhf_t, rho_t, c->Ib, c->k2));
        GKBA_TRY(axpy_c(c, c->k2, c->k1, c->k2, 1.0, 1.0, (int)NN));
        GKBA_TRY(axpy_c(c, rho_t, rho_n, c->k2, 1.0, 0.5 * c->dt, (int)NN));
        std::swap(c->T_a, c->T_b);
        c->n = n + 1;
        if (rho_out && rho_out[i])
            GKBA_CUDA(c, cudaMemcpyAsync(rho_out[i], rho_t, NN * 16, cudaMemcpyDeviceToHost, c->stream));
        if (diag_out && diag_out[i])
            GKBA_CUDA(c, cudaMemcpyAsync(c->hdiag, c->dscal, 4 * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    return GKBA_OK;
}

}  // namespace

extern "C" {

gkba_status gkba_batch_create(gkba_batch** out, gkba_ctx* const* ctxs, int n_ctx,
                              size_t workspace_bytes) {
    if (out) *out = nullptr;
    if (!out || !ctxs || n_ctx < 1)
        return batch_fail(nullptr, GKBA_EINVAL, "gkba_batch_create: out, ctxs and n_ctx >= 1 required");
    for (int i = 0; i < n_ctx; ++i) {
        gkba_ctx* c = ctxs[i];
        if (!c) return batch_fail(nullptr, GKBA_EINVAL, "gkba_batch_create: context %d is NULL", i);
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c)
                return batch_fail(nullptr, GKBA_EINVAL, "gkba_batch_create: context %d listed twice", i);
        if (!tensor_core_path(c) || c->kind != GKBA_V_GENERAL)
            return batch_fail(nullptr, GKBA_EINVAL,
                              "gkba_batch_create: context %d is not a split-TF32 general-basis context", i);
        if (c->prec != ctxs[0]->prec || c->device != ctxs[0]->device || c->acc_window != ctxs[0]->acc_window)
            return batch_fail(nullptr, GKBA_EINVAL,
                              "gkba_batch_create: contexts differ in precision, device or acc_window");
    }
    gkba_batch* b = new gkba_batch();
    b->device = ctxs[0]->device;
    b->ctx.assign(ctxs, ctxs + n_ctx);
    auto bail = [&](gkba_status st) {
        free_batch(b);
        return st;
    };
    if (cudaSetDevice(b->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return bail(batch_fail(nullptr, GKBA_ECUDA, "gkba_batch_create: stream creation failed"));
    }
    for (int i = 0; i < n_ctx; ++i) {
        int gi = -1;
        for (size_t k = 0; k < b->groups.size(); ++k)
            if (b->groups[k].N == ctxs[i]->N) gi = (int)k;
        if (gi < 0) {
            b->groups.emplace_back();
            b->groups.back().N = ctxs[i]->N;
            gi = (int)b->groups.size() - 1;
        }
        b->groups[gi].members.push_back(i);
    }
    const size_t cap_total = workspace_bytes ? workspace_bytes : ((size_t)64 << 30);
    for (auto& g : b->groups) {
        gkba_ctx* c0 = ctxs[g.members[0]];
        gkba_ctx* sh = new gkba_ctx();
        g.sh = sh;
        sh->N = g.N;
        sh->Np = c0->Np;
        sh->prec = c0->prec;
        sh->dt = c0->dt;
        sh->device = b->device;
        sh->stream = b->stream;
        sh->num_sms = c0->num_sms;
        sh->pair_clusters = c0->pair_clusters;
        sh->fin_pair_clusters = c0->fin_pair_clusters;
        sh->acc_window = c0->acc_window;
        sh->ws_cap = cap_total / b->groups.size();
        sh->nsys = (int)g.members.size();
        const long long Np = sh->Np, Np4 = Np * Np * Np * Np;
        const size_t lay = (size_t)sh->nsys * Np4 * 4;
        if (cudaMalloc(&sh->dint, 16) != cudaSuccess || cudaMalloc(&sh->wS32, lay) != cudaSuccess ||
            cudaMalloc(&sh->vKhi, lay) != cudaSuccess || cudaMalloc(&sh->vKlo, lay) != cudaSuccess) {
            cudaGetLastError();
            return bail(batch_fail(nullptr, GKBA_ENOMEM, "gkba_batch_create: layout allocation failed"));
        }
        cudaMemsetAsync(sh->dint, 0, 16, b->stream);
        for (size_t k = 0; k < g.members.size(); ++k) {
            gkba_ctx* c = ctxs[g.members[k]];
            cudaStreamSynchronize(c->stream);
            cudaMemcpyAsync(sh->wS32 + k * Np4, c->wS32, Np4 * 4, cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(sh->vKhi + k * Np4, c->vKhi, Np4 * 4, cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(sh->vKlo + k * Np4, c->vKlo, Np4 * 4, cudaMemcpyDeviceToDevice, b->stream);
        }
        const long long rows = 2 * Np;
        long long gcd = 256, r = rows;
        while (r) {
            const long long t = gcd % r;
            gcd = r;
            r = t;
        }
        g.pu = (int)(256 / gcd);
        // the largest collision of the group: every member at a full history
        long long want = 0;
        for (int m : g.members)
            want += ((2LL * (ctxs[m]->max_steps + 1) + g.pu - 1) / g.pu) * g.pu;
        gkba_status st = ensure_workspace(sh, (int)std::min<long long>(want, 1 << 30));
        if (st != GKBA_OK) {
            batch_fail(nullptr, st, "gkba_batch_create: %s", sh->err.c_str());
            return bail(st);
        }
        sh->ub = (sh->ub / g.pu) * g.pu;
        if (sh->ub < g.pu)
            return bail(batch_fail(nullptr, GKBA_ENOMEM,
                                   "gkba_batch_create: workspace holds fewer than %d units at N=%d", g.pu, g.N));
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(batch_fail(nullptr, GKBA_ECUDA, "gkba_batch_create: device copies failed"));
    }
    *out = b;
    return GKBA_OK;
}

gkba_status gkba_batch_step(gkba_batch* b, const double* E_n, const double* E_np1,
                            double* const* rho_out, double* const* diag_out) {
    if (!b) return batch_fail(nullptr, GKBA_EINVAL, "gkba_batch_step: NULL batch");
    if (!E_n || !E_np1) return batch_fail(b, GKBA_EINVAL, "gkba_batch_step: NULL field samples");
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        if (!std::isfinite(E_n[i]) || !std::isfinite(E_np1[i]))
            return batch_fail(b, GKBA_EINVAL, "gkba_batch_step: non-finite field sample for system %zu", i);
        if (b->ctx[i]->n >= b->ctx[i]->max_steps)
            return batch_fail(b, GKBA_ESTATE, "gkba_batch_step: history of system %zu is full", i);
    }
    if (cudaSetDevice(b->device) != cudaSuccess) {
        cudaGetLastError();
        return batch_fail(b, GKBA_ECUDA, "gkba_batch_step: cudaSetDevice failed");
    }
    // members run on the batch's stream for the duration of the step
    std::vector<cudaStream_t> saved(b->ctx.size());
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        cudaStreamSynchronize(b->ctx[i]->stream);
        saved[i] = b->ctx[i]->stream;
        b->ctx[i]->stream = b->stream;
    }
    gkba_status st;
    {
        NvtxRange nr("gkba_batch_step");
        if (b->use_graph) {
            // capture the step's device work and launch it as one graph; the
            // previous step's executable graph is updated in place when the
            // launch sequence kept its shape, else instantiated anew
            st = ensure_tables(b);
            if (st == GKBA_OK) {
                if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                    cudaGetLastError();
                    st = batch_fail(b, GKBA_ECUDA, "gkba_batch_step: stream capture could not begin");
                } else {
                    st = batch_step(b, E_n, E_np1, rho_out, diag_out);
                    cudaGraph_t graph = nullptr;
                    const cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
                    if (st == GKBA_OK && ce != cudaSuccess) {
                        cudaGetLastError();
                        st = batch_fail(b, GKBA_ECUDA, "gkba_batch_step: stream capture failed: %s",
                                        cudaGetErrorString(ce));
                    }
                    if (st == GKBA_OK) {
                        bool ok = false;
                        if (b->gexec) {
                            cudaGraphExecUpdateResultInfo info;
                            ok = cudaGraphExecUpdate(b->gexec, graph, &info) == cudaSuccess;
                            if (!ok) {
                                cudaGetLastError();
                                cudaGraphExecDestroy(b->gexec);
                                b->gexec = nullptr;
                            }
                        }
                        if (!ok) {
                            ++b->graph_rebuilds;
                            if (cudaGraphInstantiate(&b->gexec, graph, 0) != cudaSuccess) {
                                cudaGetLastError();
                                b->gexec = nullptr;
                                st = batch_fail(b, GKBA_ECUDA, "gkba_batch_step: graph instantiation failed");
                            }
                        }
                        if (st == GKBA_OK) {
                            if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess) {
                                cudaGetLastError();
                                st = batch_fail(b, GKBA_ECUDA, "gkba_batch_step: graph launch failed");
                            }
                            ++b->graph_steps;
                        }
                    }
                    if (graph) cudaGraphDestroy(graph);
                }
            }
        } else {
            st = batch_step(b, E_n, E_np1, rho_out, diag_out);
        }
    }
    const cudaError_t se = cudaStreamSynchronize(b->stream);
    for (size_t i = 0; i < b->ctx.size(); ++i) b->ctx[i]->stream = saved[i];
    if (st != GKBA_OK) {
        for (gkba_ctx* c : b->ctx)
            if (!c->err.empty()) b->err = c->err;
        for (auto& g : b->groups)
            if (!g.sh->err.empty()) b->err = g.sh->err;
        return st;
    }
    if (se != cudaSuccess) return batch_fail(b, GKBA_ECUDA, "gkba_batch_step: %s", cudaGetErrorString(se));
    for (auto& g : b->groups) {
        int errw = 0;
        if (cudaMemcpy(&errw, g.sh->dint + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return batch_fail(b, GKBA_ECUDA, "gkba_batch_step: error word read failed");
        if (errw != 0) {
            cudaMemset(g.sh->dint + 1, 0, sizeof(int));
            return batch_fail(b, GKBA_ETIMEOUT, "gkba_batch_step: device-side wait timed out (code %d)", errw);
        }
    }
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (diag_out && diag_out[i]) memcpy(diag_out[i], b->ctx[i]->hdiag, 4 * 8);
    return GKBA_OK;
}

const char* gkba_batch_last_error(const gkba_batch* b) {
    if (b) return b->err.c_str();
    std::lock_guard<std::mutex> g(g_err_mu);
    return g_last_init_error.c_str();
}

void gkba_batch_destroy(gkba_batch* b) { free_batch(b); }

gkba_status gkba_batch_set_options(gkba_batch* b, int use_graph) {
    if (!b) return batch_fail(nullptr, GKBA_EINVAL, "gkba_batch_set_options: NULL batch");
    if (use_graph != 0 && use_graph != 1)
        return batch_fail(b, GKBA_EINVAL, "gkba_batch_set_options: use_graph must be 0 or 1");
    b->use_graph = use_graph != 0;
    return GKBA_OK;
}

gkba_status gkba_batch_autotune(gkba_batch* b, int* n_groups, int* N_out, int* units, int* acc_window,
                                int* s4_item_k, double* us_per_unit) {
    if (!b) return batch_fail(nullptr, GKBA_EINVAL, "gkba_batch_autotune: NULL batch");
    if (cudaSetDevice(b->device) != cudaSuccess) {
        cudaGetLastError();
        return batch_fail(b, GKBA_ECUDA, "gkba_batch_autotune: cudaSetDevice failed");
    }
    std::vector<cudaStream_t> saved(b->ctx.size());
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        cudaStreamSynchronize(b->ctx[i]->stream);
        saved[i] = b->ctx[i]->stream;
        b->ctx[i]->stream = b->stream;
    }
    gkba_status st = autotune(b);
    const cudaError_t se = cudaStreamSynchronize(b->stream);
    for (size_t i = 0; i < b->ctx.size(); ++i) b->ctx[i]->stream = saved[i];
    if (st != GKBA_OK) {
        for (auto& g : b->groups)
            if (!g.sh->err.empty()) b->err = g.sh->err;
        return st;
    }
    if (se != cudaSuccess) return batch_fail(b, GKBA_ECUDA, "gkba_batch_autotune: %s", cudaGetErrorString(se));
    for (auto& g : b->groups) {
        int errw = 0;
        if (cudaMemcpy(&errw, g.sh->dint + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return batch_fail(b, GKBA_ECUDA, "gkba_batch_autotune: error word read failed");
        if (errw != 0) {
            cudaMemset(g.sh->dint + 1, 0, sizeof(int));
            return batch_fail(b, GKBA_ETIMEOUT, "gkba_batch_autotune: device-side wait timed out (code %d)", errw);
        }
    }
    if (n_groups) *n_groups = (int)b->groups.size();
    for (size_t gi = 0; gi < b->groups.size() && gi < (size_t)kMaxBatchLaunchGroups; ++gi) {
        const auto& g = b->groups[gi];
        if (N_out) N_out[gi] = g.N;
        if (units) units[gi] = (int)round_units(g);
        if (acc_window) acc_window[gi] = g.sh->acc_window;
        if (s4_item_k) s4_item_k[gi] = g.sh->fin_kw;
        if (us_per_unit) us_per_unit[gi] = g.us_per_unit;
    }
    return GKBA_OK;
}

}  // extern "C"
