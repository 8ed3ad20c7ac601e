// time_linear.cu - the history sum of Eq. (collint) in time-linear form (an
// extension of the method): FP64 on the CUDA cores, or its contractions on the
// tensor cores (split-TF32 contexts; Lambda_acc stays FP64).
//
// With the HF propagator of Eq. (prop) written as a product of the step
// unitaries, T(t_n, t_k) = Ucal_n Ucal_k^+ (Ucal_{k+1} = U_k Ucal_k), the GKBA
// factors of Eq. (gkba) split into a part fixed at t_k and Ucal_n:
//   P_k = Ucal_n X_k,  Q_k = Ucal_n Xb_k,  X_k = W_k rho_k,  Xb_k = W_k - X_k,
// with W_k = Ucal_k^+.  In Eq. (2bse) every Ucal_n then sits on an index that
// v carries (n and p with Ucal, r with conj(Ucal)) or on the right factor of
// the first line of Eq. (collint), so
//   I(t_n) = [sum_{npr} v_irpn (Ucal x_n Ucal x_p conj(Ucal) x_r Lambda)] Ucal^+,
//   Lambda = sum_k c_k [Z(Xb_k, X_k) x_j X_k^+ - Z(X_k, Xb_k) x_j Xb_k^+],
//   Z(A, B)_{n p r j} = sum_{mqs} w_mqsj A_nm A_pq conj(B)_rs,
// where Z(A, B) is stage S3's output of the FP64 chain run on (G, Gbar) =
// (A, B^+).  The stepper keeps Lambda_acc (points t_0 .. t_{n-1} with their
// final weights) and adds each point once, so a step costs O(N^5) whatever
// the history length.
//
// Layouts (planar complex, c = re/im):
//   X3T  [(n,r,p)][u][c][j]   stage S3 output, one row per (n,r,p)
//   D, Lambda_acc, tl_s  [j][n][r][c][p]
//   back-transforms: [j][n][r][(c,p)] -x_p-> [j][r][p][(c,n)] -x_n->
//                    [j][p][n][(c,r)] -x_r-> X3 [c][j][n][r][p] -> stage S4.
#include <algorithm>
#include <cmath>

#include "gkba_internal.cuh"

namespace gkba {

namespace {

inline unsigned grid1(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// History points i = 0..nk-1: G[2i] holds X = W_i rho_i on entry.  Writes
//   G[2i+1] = Xb = W_i - X,  Gb[2i] = Xb^+,  Gb[2i+1] = X^+,
// i.e. unit 2i is (G, Gbar) = (X, Xb^+) (Sigma^< part) and unit 2i+1 is
// (Xb, X^+) (Sigma^> part).
__global__ void k_tl_points(int N, int nk, const double2* __restrict__ W, long long sW,
                            double2* __restrict__ G, double2* __restrict__ Gb) {
    const long long NN = (long long)N * N;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NN * nk) return;
    const long long i = e / NN, rr = e % NN;
    const int a = (int)(rr / N), b = (int)(rr % N);
    const double2 x = G[2 * i * NN + rr];
    const double2 w = W[i * sW + rr];
    const double2 xb = make_double2(w.x - x.x, w.y - x.y);
    G[(2 * i + 1) * NN + rr] = xb;
    Gb[2 * i * NN + (long long)b * N + a] = make_double2(xb.x, -xb.y);
    Gb[(2 * i + 1) * NN + (long long)b * N + a] = make_double2(x.x, -x.y);
}

// Right factors of the accumulator GEMM, K = 2N nb columns:
//   M[(c2, j2)][(u, c, j)] = real form of coef_u Gb_u^T,
// coef_u = -wt (u even) or +wt (u odd), wt the weight of point k0 + u/2.
__global__ void k_tl_mcat(int N, int nb, const double2* __restrict__ Gb, int k0, double w_first,
                          double w_rest, double* __restrict__ M) {
    const long long NN = (long long)N * N;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NN * nb) return;
    const int u = (int)(e / NN);
    const long long rr = e % NN;
    const int j = (int)(rr / N), j2 = (int)(rr % N);
    const double wt = (k0 + u / 2 == 0) ? w_first : w_rest;
    const double coef = (u & 1) ? wt : -wt;
    const double2 g = Gb[(long long)u * NN + rr];  // Gb_u[j][j2]
    const double re = coef * g.x, im = coef * g.y;
    const long long K = 2LL * N * nb, col = 2LL * N * u;
    M[(long long)j2 * K + col + j] = re;
    M[(long long)j2 * K + col + N + j] = -im;
    M[(long long)(N + j2) * K + col + j] = im;
    M[(long long)(N + j2) * K + col + N + j] = re;
}

// Real forms (2N x 2N, rows (c', p), columns (c, q)) of Ucal = W^+ and of
// conj(Ucal) = W^T: blocks [[Re, -Im], [Im, Re]].
__global__ void k_tl_uforms(int N, const double2* __restrict__ W, double* __restrict__ Ur,
                            double* __restrict__ Urc) {
    const long long NN = (long long)N * N;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NN) return;
    const int p = (int)(e / N), q = (int)(e % N);
    const double2 w = W[(long long)q * N + p];  // Ucal_pq = conj(w), conj(Ucal)_pq = w
    const long long ld = 2LL * N;
    const double ur = w.x, ui = -w.y;
    Ur[(long long)p * ld + q] = ur;
    Ur[(long long)p * ld + N + q] = -ui;
    Ur[(long long)(N + p) * ld + q] = ui;
    Ur[(long long)(N + p) * ld + N + q] = ur;
    Urc[(long long)p * ld + q] = ur;
    Urc[(long long)p * ld + N + q] = ui;
    Urc[(long long)(N + p) * ld + q] = -ui;
    Urc[(long long)(N + p) * ld + N + q] = ur;
}

// S = acc + a D (write_s), acc += b D (add_acc); n doubles, read once each.
__global__ void k_tl_update(long long n, double* __restrict__ acc, const double* __restrict__ D,
                            double* __restrict__ S, double a, double b, int write_s, int add_acc) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const double x = acc[e], d = D[e];
        if (write_s) S[e] = fma(a, d, x);
        if (add_acc) acc[e] = fma(b, d, x);
    }
}

}  // namespace

gkba_status tl_terms(gkba_ctx* c, int nk, const double2* rho, const double2* W, long long sW,
                     int k0, double w_first, double w_rest) {
    NvtxRange r("gkba time-linear terms");
    const int N = c->N;
    const int nb = 2 * nk;
    if (nk < 1 || nb > c->ub) return fail(c, GKBA_EINVAL, "tl_terms: %d points for %d units", nk, c->ub);
    const long long NN = (long long)N * N, N2 = NN, N3 = N2 * N, N4 = N3 * N;
    double2* G = c->PQ;   // ub units
    double2* Gb = c->Mb;  // ub units
    GKBA_TRY(zgemm_batched(c, K_PREP, N, 'N', 'N', make_double2(1.0, 0.0), W, sW, rho, NN,
                           make_double2(0.0, 0.0), G, 2 * NN, nk, 0));
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_tl_points<<<grid1(nk * NN, 256), 256, 0, c->stream>>>(N, nk, W, sW, G, Gb);
    GKBA_TRY(launch_end(c, t));
    if (tensor_core_path(c)) {
        // split-TF32 chain on the tensor cores, FP64 accumulation of D
        GKBA_TRY(build_forms_tf32(c, nb, G, Gb));
        c->sep_A = false;
        return tl_terms_tf32(c, nb, Gb, k0, w_first, w_rest, (double*)c->X2);
    }
    GKBA_TRY(build_forms_fp64(c, nb, G, Gb));
    double* M = (double*)c->formsG3;  // 4 N^2 nb doubles; unused by this chain (sep_A off)
    t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_tl_mcat<<<grid1(nb * NN, 256), 256, 0, c->stream>>>(N, nb, Gb, k0, w_first, w_rest, M);
    GKBA_TRY(launch_end(c, t));
    // S1-S3 with the S3 output as X3T[(n,r,p)][u][c][j] (row length K = 2N nb)
    const long long K = 2LL * N * nb;
    const StageMap m3{1, N * K, K, N, N2 * K, N, N, N};
    c->sep_A = false;
    GKBA_TRY(fp64_chain_x3(c, nb, c->wS64, &m3, 2LL * N));
    // D[(n,r,p)][(c2,j2)] = sum_(u,c,j) X3T[(n,r,p)][(u,c,j)] M[(c2,j2)][(u,c,j)],
    // stored as [j2][n][r][c2][p]
    const StageMap md{2 * N2, 2 * N, 1, N, 2 * N3, N, N, N};
    return gemm64_stage(c, K_TL, (const double*)c->X13, K, 0, M, K, 0, (double*)c->X2, 0,
                        (int)N3, 2 * N, K, 1, 0, 0, md, 2.0 * N3 * 2 * N * K,
                        8.0 * (N3 * K + 2 * N4));
}

gkba_status tl_update(gkba_ctx* c, double a, double b, bool write_s, bool add_acc) {
    const long long N = c->N, n = 2 * N * N * N * N;
    const unsigned blocks = (unsigned)std::min<long long>(grid1(n, 256), 8LL * c->num_sms);
    auto t = launch_begin(c, K_TL, 2.0 * n, 8.0 * n * (2 + (write_s ? 1 : 0) + (add_acc ? 1 : 0)));
    k_tl_update<<<blocks, 256, 0, c->stream>>>(n, c->tl_acc, (const double*)c->X2, c->tl_s, a, b,
                                               write_s ? 1 : 0, add_acc ? 1 : 0);
    return launch_end(c, t);
}

gkba_status tl_apply(gkba_ctx* c, const double2* W, double2* I_out) {
    NvtxRange r("gkba time-linear collision");
    const int N = c->N;
    const long long NN = (long long)N * N, N2 = NN, N3 = N2 * N, N4 = N3 * N;
    GKBA_TRY(ensure_workspace(c, 2));
    if (tensor_core_path(c)) {
        GKBA_TRY(tl_apply_tf32(c, W, c->tl_s));
        return zgemm_batched(c, K_RED, N, 'N', 'N', make_double2(1.0, 0.0), c->Su, 0, W, 0,
                             make_double2(0.0, 0.0), I_out, 0, 1, 0);
    }
    double* Ur = c->tl_uf;
    double* Urc = c->tl_uf + 4 * NN;
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_tl_uforms<<<grid1(NN, 256), 256, 0, c->stream>>>(N, W, Ur, Urc);
    GKBA_TRY(launch_end(c, t));
    const double fl = 8.0 * (double)N4 * N, by = 8.0 * 4 * N4;
    double* X2 = (double*)c->X2;
    double* X13 = (double*)c->X13;
    // x_p with Ucal: rows (j, n, r) of tl_s -> X2 [j][r][p][(c, n)];
    // x_n with Ucal: rows (j, r, p) of X2 -> tl_s [j][p][n][(c, r)] (same scatter)
    const StageMap mrot{2 * N3, 1, 2 * N2, N, 2 * N, N, N, N};
    GKBA_TRY(gemm64_stage(c, K_TL, c->tl_s, 2 * N, 0, Ur, 2 * N, 0, X2, 0, (int)N3, 2 * N, 2 * N,
                          1, 0, 0, mrot, fl, by));
    GKBA_TRY(gemm64_stage(c, K_TL, X2, 2 * N, 0, Ur, 2 * N, 0, c->tl_s, 0, (int)N3, 2 * N, 2 * N,
                          1, 0, 0, mrot, fl, by));
    // x_r with conj(Ucal): rows (j, p, n) of tl_s -> X13 as X3 [c][j][n][r][p]
    const StageMap mx3{N3, 1, N2, N4, N, N, N, N};
    GKBA_TRY(gemm64_stage(c, K_TL, c->tl_s, 2 * N, 0, Urc, 2 * N, 0, X13, 0, (int)N3, 2 * N, 2 * N,
                          1, 0, 0, mx3, fl, by));
    // stage S4 on one unit: D[(c, j)][i] = sum_(n,r,p) X3[c][j][(n,r,p)] vK[i][(n,r,p)],
    // split-K into chunks that fill one wave of blocks (one unit has few output tiles)
    const long long R = 2LL * N;
    const long long Kc = gemm64_splitk_chunk(c, (int)R, N, N3, (long long)(c->part_bytes / (N * R * 8)));
    const int nz = (int)((N3 + Kc - 1) / Kc);
    const StageMap m4{0, 0, 1, 0, R, (int)R, 1, N};
    GKBA_TRY(gemm64_stage(c, K_FIN, X13, N3, 0, c->vK64, N3, 0, (double*)c->part, N * R, (int)R, N,
                          N3, nz, 1, Kc, m4, 4.0 * (double)N4 * N, 8.0 * 3 * N4));
    GKBA_TRY(reduce_partials_launch(c, 1, nz, N * R, R, c->part, false, c->Su));
    // I = S Ucal^+ = S W
    return zgemm_batched(c, K_RED, N, 'N', 'N', make_double2(1.0, 0.0), c->Su, 0, W, 0,
                         make_double2(0.0, 0.0), I_out, 0, 1, 0);
}

}  // namespace gkba
