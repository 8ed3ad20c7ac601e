// fp64_kernels.cu - FP64 kernels of the GKBA second-Born path:
//  * the chained-contraction stage GEMM for the FP64 path (Eq. 2bse evaluated
//    as four one-index contractions, see gkba_api.cu for the stage list),
//  * GKBA reconstruction P_k = T(t,t_k) rho_k, Q_k = T(t,t_k) - P_k (Eq. gkba),
//  * split-K reduction and the weighted history sum of Eq. (collint),
//  * the time-local pieces of Eq. (equalt): Sigma_HF, h_HF, commutator,
//    U_n = exp(-i dt h) by scaling and squaring with a Taylor polynomial,
//    the propagator recursion T(t_{n+1},t_k) = U_n T(t_n,t_k), Heun updates.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <mutex>

#include "gkba_internal.cuh"

namespace gkba {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// ---------------------------------------------------------------------------
// Stage GEMM (FP64): D[row][col] = sum_k A[row*lda+k] * B[col*ldb+k]; the
// result is scattered by the stage's index map.  64x64 output tile, 16-wide
// K slices staged in shared memory, 4x4 outputs per thread.
// ---------------------------------------------------------------------------
constexpr int G64_BM = 64, G64_BN = 64, G64_BK = 16;

__global__ void __launch_bounds__(256) k_gemm64_stage(const double* __restrict__ A, long long lda,
                                                      long long sAz, const double* __restrict__ B,
                                                      long long ldb, long long sBz,
                                                      double* __restrict__ out, long long sOz, int M,
                                                      int Nc, long long Ktot, int splitk,
                                                      long long Kc, StageMap map) {
    const int z = blockIdx.z;
    long long K = Ktot;
    if (splitk) {
        const long long k0 = (long long)z * Kc;
        K = Ktot - k0 < Kc ? Ktot - k0 : Kc;
        A += k0;
        B += k0;
        out += (long long)z * sOz;
    } else {
        A += (long long)z * sAz;
        B += (long long)z * sBz;
        out += (long long)z * sOz;
    }
    const long long m0 = (long long)blockIdx.y * G64_BM;
    const int n0 = blockIdx.x * G64_BN;
    __shared__ double As[G64_BK][G64_BM + 1];
    __shared__ double Bs[G64_BK][G64_BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (long long kb = 0; kb < K; kb += G64_BK) {
        for (int e = tid; e < G64_BM * G64_BK; e += 256) {
            const int r = e / G64_BK, kk = e % G64_BK;
            const long long gr = m0 + r, gk = kb + kk;
            As[kk][r] = (gr < M && gk < K) ? A[gr * lda + gk] : 0.0;
        }
        for (int e = tid; e < G64_BN * G64_BK; e += 256) {
            const int cidx = e / G64_BK, kk = e % G64_BK;
            const long long gc = n0 + cidx, gk = kb + kk;
            Bs[kk][cidx] = (gc < Nc && gk < K) ? B[gc * ldb + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < G64_BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long row = m0 + ty + 16 * i;
        if (row >= M) continue;
        const long long x = row % map.Dx;
        const long long rb = row / map.Dx;
        const long long b = rb % map.Db;
        const long long a = rb / map.Db;
        const long long roff = a * map.SA + b * map.SB + x * map.SX;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = n0 + tx + 16 * j;
            if (col >= Nc) continue;
            const int cc = col / map.Dy, y = col % map.Dy;
            out[roff + cc * map.SC + (long long)y * map.SY] = acc[i][j];
        }
    }
}

// ---------------------------------------------------------------------------
// Complex batched GEMM for N x N matrices (FP64):
//   C = alpha op(A) op(B) + beta C (+ identity), op in {N, C = conj-transpose}.
// When skip_ge != nullptr and idx >= *skip_ge the block copies op(A) into C
// instead (used for the data-dependent number of squarings in expm).
// ---------------------------------------------------------------------------
constexpr int ZT = 16;

__global__ void __launch_bounds__(256) k_zgemm(int n, int opA, int opB, double2 alpha,
                                               const double2* __restrict__ A, long long sA,
                                               const double2* __restrict__ B, long long sB,
                                               double2 beta, double2* __restrict__ C, long long sC,
                                               int add_identity, const int* skip_ge, int idx) {
    const int b = blockIdx.z;
    A += (long long)b * sA;
    B += (long long)b * sB;
    C += (long long)b * sC;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row = blockIdx.y * ZT + ty, col = blockIdx.x * ZT + tx;
    if (skip_ge != nullptr && idx >= *skip_ge) {
        if (row < n && col < n) {
            double2 a = opA ? cconj(A[(long long)col * n + row]) : A[(long long)row * n + col];
            C[(long long)row * n + col] = a;
        }
        return;
    }
    __shared__ double2 As[ZT][ZT + 1], Bs[ZT][ZT + 1];
    double2 acc = make_double2(0.0, 0.0);
    for (int kb = 0; kb < n; kb += ZT) {
        // As[ty][tx] = op(A)[row][kb+tx]
        {
            const int r = blockIdx.y * ZT + ty, k = kb + tx;
            double2 v = make_double2(0.0, 0.0);
            if (r < n && k < n) v = opA ? cconj(A[(long long)k * n + r]) : A[(long long)r * n + k];
            As[ty][tx] = v;
        }
        // Bs[ty][tx] = op(B)[kb+ty][col]
        {
            const int k = kb + ty, cidx = blockIdx.x * ZT + tx;
            double2 v = make_double2(0.0, 0.0);
            if (k < n && cidx < n) v = opB ? cconj(B[(long long)cidx * n + k]) : B[(long long)k * n + cidx];
            Bs[ty][tx] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < ZT; ++kk) acc = cadd(acc, cmul(As[ty][kk], Bs[kk][tx]));
        __syncthreads();
    }
    if (row < n && col < n) {
        double2 r = cmul(alpha, acc);
        if (beta.x != 0.0 || beta.y != 0.0) r = cadd(r, cmul(beta, C[(long long)row * n + col]));
        if (add_identity && row == col) r.x += 1.0;
        C[(long long)row * n + col] = r;
    }
}

// Sigma_HF(rho)_ij = sum_{l,k} hfK[(i,j),(l,k)] rho_lk, plus h + E d when add_h.
// One warp per (i, j); lanes stride over (l, k).
__global__ void k_mean_field(int N, const double* __restrict__ hfK, const double2* __restrict__ rho,
                             const double2* __restrict__ h, const double2* __restrict__ d, double E,
                             int add_h, double2* __restrict__ out) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int NN = N * N;
    if (warp >= NN) return;
    const double* row = hfK + (long long)warp * NN;
    double re = 0.0, im = 0.0;
    for (int e = lane; e < NN; e += 32) {
        const double kv = row[e];
        const double2 r = rho[e];
        re = fma(kv, r.x, re);
        im = fma(kv, r.y, im);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        if (add_h) {
            re += h[warp].x + E * d[warp].x;
            im += h[warp].y + E * d[warp].y;
        }
        out[warp] = make_double2(re, im);
    }
}

// out = -i (HR - RH) - (I + I^+), where HR = H rho and RH = rho H.
__global__ void k_rhs(int N, const double2* __restrict__ HR, const double2* __restrict__ RH,
                      const double2* __restrict__ I, double2* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * N) return;
    const int i = e / N, j = e % N;
    const double2 c = make_double2(HR[e].x - RH[e].x, HR[e].y - RH[e].y);
    const double2 a = I[e], bt = I[j * N + i];
    // -i c = (c.y, -c.x); I + I^+ at (i,j) = I_ij + conj(I_ji)
    out[e] = make_double2(c.y - (a.x + bt.x), -c.x - (a.y - bt.y));
}

// y = a x + b z (elementwise complex, real a and b).
__global__ void k_lincomb(long long n, double2* __restrict__ y, const double2* __restrict__ x,
                          const double2* __restrict__ z, double a, double b) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double2 xv = x[e];
    const double2 zv = z ? z[e] : make_double2(0.0, 0.0);
    y[e] = make_double2(a * xv.x + b * zv.x, a * xv.y + b * zv.y);
}

__global__ void k_set_identity(int N, int count, double2* __restrict__ A) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long NN = (long long)N * N;
    if (e >= NN * count) return;
    const long long r = e % NN;
    A[e] = make_double2((r / N) == (r % N) ? 1.0 : 0.0, 0.0);
}

// expm set-up: A = -i dt (hA + hB)/2; writes A into X, its 1-norm (max column
// sum of |A_ij|) and the number of squarings s so that ||A||/2^s <= 1/2, then
// scales X by 2^-s.  One block.
__global__ void k_expm_setup(int N, double dt, const double2* __restrict__ hA,
                             const double2* __restrict__ hB, double2* __restrict__ X,
                             double* __restrict__ norm_out, int* __restrict__ s_out) {
    __shared__ double colmax[1024];
    const int tid = threadIdx.x;
    double best = 0.0;
    for (int j = tid; j < N; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < N; ++i) {
            const long long e = (long long)i * N + j;
            const double hr = 0.5 * (hA[e].x + hB[e].x), hi = 0.5 * (hA[e].y + hB[e].y);
            s += dt * sqrt(hr * hr + hi * hi);
        }
        best = fmax(best, s);
    }
    colmax[tid] = best;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) colmax[tid] = fmax(colmax[tid], colmax[tid + o]);
        __syncthreads();
    }
    const double nrm = colmax[0];
    int s = 0;
    while (s < 30 && ldexp(nrm, -s) > 0.5) ++s;
    const double scale = ldexp(1.0, -s);
    for (int e = tid; e < N * N; e += blockDim.x) {
        const double hr = 0.5 * (hA[e].x + hB[e].x), hi = 0.5 * (hA[e].y + hB[e].y);
        // -i dt h = (dt*hi, -dt*hr)
        X[e] = make_double2(scale * dt * hi, -scale * dt * hr);
    }
    if (tid == 0) {
        *norm_out = nrm;
        *s_out = s;
    }
}

// The whole exponential for N <= 24 in one block, matrices in shared memory
// (the same algorithm as k_expm_setup followed by the Horner and squaring
// products: A = -i dt (hA + hB)/2 scaled by 2^-s so that ||A||_1 / 2^s <= 1/2,
// the degree-18 Taylor polynomial by Horner, Y = I + X Y / k for k = 18 .. 1,
// then min(s, 16) squarings).  One launch instead of 37 for small bases.
constexpr int kExpmSmallN = 24;
__device__ void smem_zgemm(int N, const double2* A, const double2* B, double2* C, double alpha,
                           int add_identity) {
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i = e / N, j = e % N;
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < N; ++k) acc = cadd(acc, cmul(A[i * N + k], B[k * N + j]));
        double2 r = make_double2(alpha * acc.x, alpha * acc.y);
        if (add_identity && i == j) r.x += 1.0;
        C[e] = r;
    }
}
__global__ void __launch_bounds__(256) k_expm_small(int N, double dt, const double2* __restrict__ hA,
                                                     const double2* __restrict__ hB,
                                                     double2* __restrict__ U,
                                                     double* __restrict__ norm_out,
                                                     int* __restrict__ s_out) {
    __shared__ double2 X[kExpmSmallN * kExpmSmallN], Y[kExpmSmallN * kExpmSmallN],
        Z[kExpmSmallN * kExpmSmallN];
    __shared__ double colsum[kExpmSmallN];
    const int tid = threadIdx.x, NN = N * N;
    for (int j = tid; j < N; j += blockDim.x) {
        double sum = 0.0;
        for (int i = 0; i < N; ++i) {
            const int e = i * N + j;
            const double hr = 0.5 * (hA[e].x + hB[e].x), hi = 0.5 * (hA[e].y + hB[e].y);
            sum += dt * sqrt(hr * hr + hi * hi);
        }
        colsum[j] = sum;
    }
    __syncthreads();
    double nrm = 0.0;
    for (int j = 0; j < N; ++j) nrm = fmax(nrm, colsum[j]);
    int s = 0;
    while (s < 30 && ldexp(nrm, -s) > 0.5) ++s;
    const double scale = ldexp(1.0, -s);
    for (int e = tid; e < NN; e += blockDim.x) {
        const double hr = 0.5 * (hA[e].x + hB[e].x), hi = 0.5 * (hA[e].y + hB[e].y);
        X[e] = make_double2(scale * dt * hi, -scale * dt * hr);  // -i dt h / 2^s
        Y[e] = make_double2((e / N == e % N) ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    double2 *y = Y, *z = Z;
    for (int k = 18; k >= 1; --k) {
        smem_zgemm(N, X, y, z, 1.0 / k, 1);
        __syncthreads();
        double2* t = y; y = z; z = t;
    }
    const int nsq = s < 16 ? s : 16;
    for (int q = 0; q < nsq; ++q) {
        smem_zgemm(N, y, y, z, 1.0, 0);
        __syncthreads();
        double2* t = y; y = z; z = t;
    }
    for (int e = tid; e < NN; e += blockDim.x) U[e] = y[e];
    if (tid == 0) {
        *norm_out = nrm;
        *s_out = s;
    }
}

// Diagnostics at t_n: {Tr rho, E_total, E_corr, Re Tr I}.
// E_total = 1/2 (Tr[(h+E d) rho] + Tr[h_HF rho]) + 1/2 Im Tr I.
__global__ void k_diagnostics(int N, double E, const double2* __restrict__ h,
                              const double2* __restrict__ d, const double2* __restrict__ hhf,
                              const double2* __restrict__ rho, const double2* __restrict__ I,
                              double* __restrict__ out) {
    __shared__ double s0[256], s1[256], s2[256];
    const int tid = threadIdx.x;
    double t1 = 0.0, t2 = 0.0, tr = 0.0;
    for (int e = tid; e < N * N; e += blockDim.x) {
        const int i = e / N, j = e % N;
        const double2 r = rho[j * N + i];
        const double2 a = make_double2(h[e].x + E * d[e].x, h[e].y + E * d[e].y);
        t1 += a.x * r.x - a.y * r.y;
        t2 += hhf[e].x * r.x - hhf[e].y * r.y;
        if (i == j) tr += rho[e].x;
    }
    s0[tid] = t1;
    s1[tid] = t2;
    s2[tid] = tr;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) {
            s0[tid] += s0[tid + o];
            s1[tid] += s1[tid + o];
            s2[tid] += s2[tid + o];
        }
        __syncthreads();
    }
    if (tid == 0) {
        double trI_re = 0.0, trI_im = 0.0;
        for (int i = 0; i < N; ++i) {
            trI_re += I[i * N + i].x;
            trI_im += I[i * N + i].y;
        }
        const double ec = 0.5 * trI_im;
        out[0] = s2[0];
        out[1] = 0.5 * (s0[0] + s1[0]) + ec;
        out[2] = ec;
        out[3] = trI_re;
    }
}

// ---------------------------------------------------------------------------
// GKBA unit forms (FP64 path).  Unit u of a batch holds (G_u, Gb_u); the
// stage-1 operand is B1[u][(c,r)][s] = Gb_c[s][r] (2N x N), the stage-2/3
// operand is the real form of G: Gr[u][(c',p)][(c,q)] with blocks
// [[Re G, -Im G], [Im G, Re G]] (2N x 2N).
// ---------------------------------------------------------------------------
__global__ void k_forms64(int N, int nb, const double2* __restrict__ G, const double2* __restrict__ Gb,
                          double* __restrict__ B1, double* __restrict__ Gr) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long NN = (long long)N * N;
    if (e >= NN * nb) return;
    const int u = (int)(e / NN);
    const int rr = (int)(e % NN);
    const int a = rr / N, b = rr % N;
    // stage-1 operand: entry (s = a, r = b); skipped when only the G forms are wanted
    if (B1 != nullptr) {
        const double2 gb = Gb[u * NN + rr];  // Gb[s][r]
        double* b1 = B1 + (long long)u * 2 * NN;
        b1[(long long)(0 * N + b) * N + a] = gb.x;
        b1[(long long)(1 * N + b) * N + a] = gb.y;
    }
    // stage-2/3 operand: entry (p = a, q = b)
    const double2 g = G[u * NN + rr];
    double* gr = Gr + (long long)u * 4 * NN;
    const long long ld = 2 * N;
    gr[(long long)(0 * N + a) * ld + 0 * N + b] = g.x;
    gr[(long long)(0 * N + a) * ld + 1 * N + b] = -g.y;
    gr[(long long)(1 * N + a) * ld + 0 * N + b] = g.y;
    gr[(long long)(1 * N + a) * ld + 1 * N + b] = g.x;
}

// Units of history point k (batch-local kk = k - k0): u = 2 kk + comp,
//   comp 0 (Sigma^<): G = P_k, Gb = Q_k^+, coefficient -c_k,
//   comp 1 (Sigma^>): G = Q_k, Gb = P_k^+, coefficient +c_k,
// so that I = sum_u coef_u S(G_u, Gb_u) Gb_u (first line of Eq. collint).
// Writes G_u into Gout, Gb_u into Mb and the coefficients.
__global__ void k_gkba_units(int N, int nk, int k0, int L, double dt, const double2* __restrict__ P,
                             const double2* __restrict__ Q, const double* __restrict__ w,
                             double2* __restrict__ Gout, double2* __restrict__ Mb,
                             double* __restrict__ coef) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long NN = (long long)N * N;
    if (e >= NN * nk) return;
    const int kk = (int)(e / NN);
    const int rr = (int)(e % NN);
    const int i = rr / N, j = rr % N;
    const long long base = (long long)kk * NN;
    const double2 p = P[base + rr], q = Q[base + rr];
    const double2 pt = P[base + (long long)j * N + i], qt = Q[base + (long long)j * N + i];
    Gout[(2 * kk + 0) * NN + rr] = p;
    Gout[(2 * kk + 1) * NN + rr] = q;
    Mb[(2 * kk + 0) * NN + rr] = make_double2(qt.x, -qt.y);  // (Q^+)_ij = conj(Q_ji)
    Mb[(2 * kk + 1) * NN + rr] = make_double2(pt.x, -pt.y);
    if (rr == 0) {
        const int k = k0 + kk;
        double c;
        if (w != nullptr) c = w[k];
        else if (L <= 1) c = 0.0;
        else c = (k == 0 || k == L - 1) ? 0.5 * dt : dt;
        coef[2 * kk + 0] = -c;
        coef[2 * kk + 1] = c;
    }
}

// S_u[i][j] = sum_z part[z][i][u*2N + j] + i part[z][i][u*2N + N + j]
// (split-K partials of the last contraction, rows (u, c, j)).  Two passes with
// a fixed summation order (deterministic): pass 1 sums z-range zc of each
// element into tmp[zc], pass 2 adds the z-ranges in order.  Partials are FP64
// (FP64 path) or FP32 (tensor-core path); all sums are FP64.
// Compensated (Kahan) running sum in the partials' own precision: the error
// stays at a few ulps of the sum whatever the number of terms, and FP32 adds
// run at full rate (GB300's FP64 rate is low).
template <typename TP>
struct KahanSum {
    TP s = 0, c = 0;
    __device__ __forceinline__ void add(TP x) {
        const TP y = x - c;
        const TP t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <typename TP>
__global__ void k_reduce_partials_p1(int N, int Np, int nb, int nz, int zper, long long zstride,
                                     long long Rld, const TP* __restrict__ part,
                                     double2* __restrict__ tmp) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long NN = (long long)N * N;
    if (e >= NN * nb) return;
    const int zc = blockIdx.y;
    const int u = (int)(e / NN);
    const int rr = (int)(e % NN);
    const int i = rr / N, j = rr % N;
    const long long r_re = (long long)u * 2 * Np + j, r_im = r_re + Np;
    const int z0 = zc * zper, z1 = min(nz, z0 + zper);
    KahanSum<TP> re[2], im[2];
    const TP* base = part + (long long)i * Rld;
    int z = z0;
    for (; z + 2 <= z1; z += 2) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const TP* pz = base + (long long)(z + q) * zstride;
            re[q].add(pz[r_re]);
            im[q].add(pz[r_im]);
        }
    }
    if (z < z1) {
        const TP* pz = base + (long long)z * zstride;
        re[0].add(pz[r_re]);
        im[0].add(pz[r_im]);
    }
    const double sre = ((double)re[0].s - (double)re[0].c) + ((double)re[1].s - (double)re[1].c);
    const double sim = ((double)im[0].s - (double)im[0].c) + ((double)im[1].s - (double)im[1].c);
    tmp[(long long)zc * NN * nb + e] = make_double2(sre, sim);
}

__global__ void k_reduce_partials_p2(long long n, int nzc, const double2* __restrict__ tmp,
                                     double2* __restrict__ S) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double re = 0.0, im = 0.0;
    for (int zc = 0; zc < nzc; ++zc) {
        const double2 t = tmp[(long long)zc * n + e];
        re += t.x;
        im += t.y;
    }
    S[e] = make_double2(re, im);
}

// I_acc[e] += sum_u coef[u] * Y[u][e] in two passes with a fixed order
// (deterministic): pass 1 sums the contiguous unit range z of every element
// into tmp[z][e] (blockIdx.y = z), pass 2 adds the ranges in order.  Small
// bases have few elements and many units (N = 10: 100 elements, up to 10^4
// units per batch), so the units are spread over the grid, not looped by one
// thread per element.
constexpr int kWsumRanges = 256;
__global__ void k_weighted_sum_p1(int NN, int nb, int per, const double* __restrict__ coef,
                                  const double2* __restrict__ Y, double2* __restrict__ tmp) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NN) return;
    const int u0 = blockIdx.y * per;
    const int u1 = min(nb, u0 + per);
    double re = 0.0, im = 0.0;
    for (int u = u0; u < u1; ++u) {
        const double c = coef[u];
        const double2 y = Y[(long long)u * NN + e];
        re = fma(c, y.x, re);
        im = fma(c, y.y, im);
    }
    tmp[(long long)blockIdx.y * NN + e] = make_double2(re, im);
}
__global__ void k_weighted_sum_p2(int NN, int nz, const double2* __restrict__ tmp,
                                  double2* __restrict__ I_acc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NN) return;
    double re = 0.0, im = 0.0;
    for (int z = 0; z < nz; ++z) {
        const double2 t = tmp[(long long)z * NN + e];
        re += t.x;
        im += t.y;
    }
    I_acc[e].x += re;
    I_acc[e].y += im;
}

// hfK[(i*N + j)*N*N + l*N + k] = 2 v_iklj - v_ikjl  (Sigma_HF as a matrix-vector product)
__global__ void k_build_hfK(int N, const double* __restrict__ v, double* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = N, N4 = n * n * n * n;
    if (e >= N4) return;
    const long long k = e % n, l = (e / n) % n, j = (e / n / n) % n, i = e / n / n / n;
    out[e] = 2.0 * v[((i * n + k) * n + l) * n + j] - v[((i * n + k) * n + j) * n + l];
}

// wS[j][m][q][s] = w_mqsj = 2 v_mqsj - v_qmsj (the direct and exchange terms of
// Eq. (2bse) after relabelling m <-> q in the exchange term).
__global__ void k_build_wS64(int N, const double* __restrict__ v, double* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = N, N4 = n * n * n * n;
    if (e >= N4) return;
    const long long s = e % n, q = (e / n) % n, m = (e / n / n) % n, j = e / n / n / n;
    out[e] = 2.0 * v[((m * n + q) * n + s) * n + j] - v[((q * n + m) * n + s) * n + j];
}

// vK[i][n][r][p] = v_irpn (K index (n, r, p) of the last contraction).
__global__ void k_build_vK64(int N, const double* __restrict__ v, double* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = N, N4 = n * n * n * n;
    if (e >= N4) return;
    const long long p = e % n, r = (e / n) % n, nn = (e / n / n) % n, i = e / n / n / n;
    out[e] = v[((i * n + r) * n + p) * n + nn];
}

inline unsigned grid1(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---------------------------------------------------------------------------
// Structured interactions (Sec. III A, B): the self-energy without the N^5
// contraction chain.
// ---------------------------------------------------------------------------
// Diagonal basis, Eq. (2b-diag): S_ij = U_i U_j G_ij Gb_ji G_ij
// (the entrywise form diag(V) o diag(V) o G o Gb^T o G of Eq. (2b-diag-opt)).
__global__ void k_sigma_diag(int N, int nb, const double* __restrict__ U,
                             const double2* __restrict__ G, const double2* __restrict__ Gb,
                             double2* __restrict__ S) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long NN = (long long)N * N;
    if (e >= NN * nb) return;
    const long long u = e / NN;
    const int rr = (int)(e % NN);
    const int i = rr / N, j = rr % N;
    const double2 g = G[e];
    const double2 x = cmul(cmul(g, g), Gb[u * NN + (long long)j * N + i]);
    const double s = U[i] * U[j];
    S[e] = make_double2(s * x.x, s * x.y);
}

// Symmetric basis, Eq. (2b-symm), bubble and exchange together:
//   S_ij = sum_kl V_ik V_jl (2 G_ij Gb_lk G_kl - G_il Gb_lk G_kj)
//        = sum_l V_jl (2 G_ij r_l - G_il W_lj)
// with, for the row i of the block,
//   r_l  = sum_k V_ik Gb_lk G_kl   (the bubble's [V x (Gb^T o G)]_il, Eq. bubble-contract)
//   W_lj = sum_k V_ik Gb_lk G_kj   (N^3 per row: the exchange term has no
//                                   matrix-product form for the full matrix).
// One block per (row i, unit u); r_l in shared memory; a thread per column j
// (the Gb_lk loads are the same for all threads of a warp, the G_kj loads are
// consecutive in j).  N^4 per unit.
__global__ void k_sigma_symm(int N, const double* __restrict__ V, const double2* __restrict__ G,
                             const double2* __restrict__ Gb, double2* __restrict__ S) {
    extern __shared__ double2 r_sh[];
    const int i = blockIdx.x;
    const long long NN = (long long)N * N;
    const double2* g = G + (long long)blockIdx.y * NN;
    const double2* gb = Gb + (long long)blockIdx.y * NN;
    const double* vi = V + (long long)i * N;
    for (int l = threadIdx.x; l < N; l += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < N; ++k) {
            const double2 a = gb[(long long)l * N + k];
            acc = cadd(acc, cmul(make_double2(vi[k] * a.x, vi[k] * a.y), g[(long long)k * N + l]));
        }
        r_sh[l] = acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double2 gij = g[(long long)i * N + j];
        double2 s = make_double2(0.0, 0.0);
        for (int l = 0; l < N; ++l) {
            double2 w = make_double2(0.0, 0.0);
            for (int k = 0; k < N; ++k) {
                const double2 a = gb[(long long)l * N + k];
                w = cadd(w, cmul(make_double2(vi[k] * a.x, vi[k] * a.y), g[(long long)k * N + j]));
            }
            const double2 b = cmul(gij, r_sh[l]);
            const double2 x = cmul(g[(long long)i * N + l], w);
            const double vjl = V[(long long)j * N + l];
            s = cadd(s, make_double2(vjl * (2.0 * b.x - x.x), vjl * (2.0 * b.y - x.y)));
        }
        S[(long long)blockIdx.y * NN + (long long)i * N + j] = s;
    }
}

// Same for N <= 24, one block per unit with G, Gb, V and r in shared memory:
//   r[i][l] = sum_k V_ik Gb_lk G_kl = [V x (Gb^T o G)]_il   (N^3)
//   S_ij    = sum_l V_jl (2 G_ij r[i][l] - G_il sum_k V_ik Gb_lk G_kj)   (N^2 per (i, j))
constexpr int kSymmSmallN = 24;  // 32 KB of static shared memory
__global__ void __launch_bounds__(256) k_sigma_symm_small(int N, const double* __restrict__ V,
                                                           const double2* __restrict__ G,
                                                           const double2* __restrict__ Gb,
                                                           double2* __restrict__ S) {
    __shared__ double2 g[kSymmSmallN * kSymmSmallN], gb[kSymmSmallN * kSymmSmallN],
        r[kSymmSmallN * kSymmSmallN];
    __shared__ double vs[kSymmSmallN * kSymmSmallN];
    const int NN = N * N;
    const long long base = (long long)blockIdx.x * NN;
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
        g[e] = G[base + e];
        gb[e] = Gb[base + e];
        vs[e] = V[e];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
        const int i = e / N, l = e % N;
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < N; ++k) {
            const double2 a = cmul(gb[l * N + k], g[k * N + l]);
            acc = make_double2(fma(vs[i * N + k], a.x, acc.x), fma(vs[i * N + k], a.y, acc.y));
        }
        r[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
        const int i = e / N, j = e % N;
        const double2 gij = g[e];
        double2 s = make_double2(0.0, 0.0);
        for (int l = 0; l < N; ++l) {
            double2 w = make_double2(0.0, 0.0);
            for (int k = 0; k < N; ++k) {
                const double2 a = gb[l * N + k];
                w = cadd(w, cmul(make_double2(vs[i * N + k] * a.x, vs[i * N + k] * a.y), g[k * N + j]));
            }
            const double2 b = cmul(gij, r[i * N + l]);
            const double2 x = cmul(g[i * N + l], w);
            const double vjl = vs[j * N + l];
            s = cadd(s, make_double2(vjl * (2.0 * b.x - x.x), vjl * (2.0 * b.y - x.y)));
        }
        S[base + e] = s;
    }
}

// ---------------------------------------------------------------------------
// Adjoint of the collision integral: per-unit elementwise steps.
// ---------------------------------------------------------------------------
// out_u = op(in_u) for N x N units: conjugate and/or transpose.
__global__ void k_unit_xform(int N, long long n_el, const double2* __restrict__ in,
                             double2* __restrict__ out, int conj, int transpose) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const long long NN = (long long)N * N, u = e / NN;
    const int rr = (int)(e % NN), i = rr / N, j = rr % N;
    double2 x = in[u * NN + (transpose ? (long long)j * N + i : rr)];
    if (conj) x.y = -x.y;
    out[e] = x;
}
// y_u += x_u (or x_u^T)
__global__ void k_unit_acc(int N, long long n_el, double2* __restrict__ y,
                           const double2* __restrict__ x, int transpose) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const long long NN = (long long)N * N, u = e / NN;
    const int rr = (int)(e % NN), i = rr / N, j = rr % N;
    const double2 a = x[u * NN + (transpose ? (long long)j * N + i : rr)];
    y[e].x += a.x;
    y[e].y += a.y;
}
// Ybar_u = coef_u Ibar (I = sum_u coef_u Y_u with real coefficients)
__global__ void k_scale_units(int N, int nb, const double* __restrict__ coef,
                              const double2* __restrict__ Ibar, double2* __restrict__ Y) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long NN = (long long)N * N;
    if (e >= NN * nb) return;
    const double c = coef[e / NN];
    const double2 b = Ibar[e % NN];
    Y[e] = make_double2(c * b.x, c * b.y);
}
// Per history point k (units 2k: G = P, Gb = Q^+; 2k+1: G = Q, Gb = P^+):
//   Pbar = Gbar_(2k) + (Gbbar_(2k+1))^+,  Qbar = Gbar_(2k+1) + (Gbbar_(2k))^+
__global__ void k_vjp_points(int N, int nk, const double2* __restrict__ Gbar,
                             const double2* __restrict__ Gbbar, double2* __restrict__ Pbar,
                             double2* __restrict__ Qbar) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long NN = (long long)N * N;
    if (e >= NN * nk) return;
    const long long k = e / NN;
    const int rr = (int)(e % NN), i = rr / N, j = rr % N;
    const long long tr = (long long)j * N + i;
    const double2 g0 = Gbar[(2 * k) * NN + rr], g1 = Gbar[(2 * k + 1) * NN + rr];
    const double2 b0 = Gbbar[(2 * k) * NN + tr], b1 = Gbbar[(2 * k + 1) * NN + tr];
    Pbar[e] = make_double2(g0.x + b1.x, g0.y - b1.y);
    Qbar[e] = make_double2(g1.x + b0.x, g1.y - b0.y);
}

// ---------------------------------------------------------------------------
// Adjoint of the Heun step: small N x N helpers.
// ---------------------------------------------------------------------------
// y += i s (a - b)
__global__ void k_add_i_diff(long long n, double2* __restrict__ y, const double2* __restrict__ a,
                             const double2* __restrict__ b, double s) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double re = a[e].x - b[e].x, im = a[e].y - b[e].y;
    y[e].x += -s * im;
    y[e].y += s * re;
}
// Ibar = -(kbar + kbar^+)   (k = ... - (I + I^+))
__global__ void k_ibar_from_kbar(int N, const double2* __restrict__ kb, double2* __restrict__ Ib) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * N) return;
    const int i = e / N, j = e % N;
    const double2 a = kb[e], b = kb[j * N + i];
    Ib[e] = make_double2(-(a.x + b.x), -(a.y - b.y));
}
// rho_bar[l][k] += sum_ij hfK[(i,j)][(l,k)] hbar[i][j]  (adjoint of the mean field, hfK real)
__global__ void k_mean_field_adj(int N, const double* __restrict__ hfK, const double2* __restrict__ hb,
                                 double2* __restrict__ rb) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int NN = N * N;
    if (warp >= NN) return;
    double re = 0.0, im = 0.0;
    for (int e = lane; e < NN; e += 32) {
        const double kv = hfK[(long long)e * NN + warp];
        re = fma(kv, hb[e].x, re);
        im = fma(kv, hb[e].y, im);
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        rb[warp].x += re;
        rb[warp].y += im;
    }
}
// out += Re sum_ij conj(hbar_ij) d_ij   (dL/dE for h = ... + E d, E real); one block
__global__ void k_field_grad(int N, const double2* __restrict__ hb, const double2* __restrict__ d,
                             double* __restrict__ out) {
    __shared__ double part[256];
    double acc = 0.0;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) acc += hb[e].x * d[e].x + hb[e].y * d[e].y;
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out += part[0];
}
// Fréchet block for the adjoint of U = exp(X), X = -i dt (hA + hB)/2:
//   Z = [[X^+, Ubar / nu], [0, X^+]] (2N x 2N), nu = max(1, ||Ubar||_1) so that
// the scaling of the exponential stays small; the top-right block of exp(Z)
// times nu is L_exp(X^+, Ubar) = Xbar.  One block.
__global__ void k_frechet_block(int N, double dt, const double2* __restrict__ hA,
                                const double2* __restrict__ hB, const double2* __restrict__ Ub,
                                double2* __restrict__ Z, double* __restrict__ nu_out) {
    __shared__ double colmax[256];
    double best = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double sum = 0.0;
        for (int i = 0; i < N; ++i) sum += hypot(Ub[i * N + j].x, Ub[i * N + j].y);
        best = fmax(best, sum);
    }
    colmax[threadIdx.x] = best;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) colmax[threadIdx.x] = fmax(colmax[threadIdx.x], colmax[threadIdx.x + o]);
        __syncthreads();
    }
    const double nu = fmax(1.0, colmax[0]);
    const int M = 2 * N;
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        const int r = e / M, c = e % M;
        double2 z = make_double2(0.0, 0.0);
        if ((r < N && c < N) || (r >= N && c >= N)) {
            // X^+ with X = -i dt h, h = (hA + hB)/2 Hermitian: X^+ = i dt h
            const int i = r % N, j = c % N;
            const double hr = 0.5 * (hA[i * N + j].x + hB[i * N + j].x);
            const double hi = 0.5 * (hA[i * N + j].y + hB[i * N + j].y);
            z = make_double2(-dt * hi, dt * hr);
        } else if (r < N && c >= N) {
            const double2 u = Ub[r * N + (c - N)];
            z = make_double2(u.x / nu, u.y / nu);
        }
        Z[e] = z;
    }
    if (threadIdx.x == 0) *nu_out = nu;
}
// hbar_A += (i dt / 2) nu W[0:N, N:2N];  hbar_B += same  (X = -i dt (hA + hB)/2)
__global__ void k_frechet_apply(int N, double dt, const double2* __restrict__ W,
                                const double* __restrict__ nu, double2* __restrict__ hA_b,
                                double2* __restrict__ hB_b) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * N) return;
    const int i = e / N, j = e % N;
    const double2 w = W[i * (2 * N) + N + j];
    const double s = 0.5 * dt * (*nu);
    const double2 a = make_double2(-s * w.y, s * w.x);  // i s w
    hA_b[e].x += a.x;
    hA_b[e].y += a.y;
    hB_b[e].x += a.x;
    hB_b[e].y += a.y;
}
// exp(Z) for a general complex n x n matrix: scaling set-up (1-norm, number of
// squarings s with ||Z||_1 / 2^s <= 1/2, Z scaled by 2^-s into X).  One block.
__global__ void k_expm_setup_general(int n, const double2* __restrict__ Z, double2* __restrict__ X,
                                     int* __restrict__ s_out) {
    __shared__ double colmax[256];
    double best = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double sum = 0.0;
        for (int i = 0; i < n; ++i) sum += hypot(Z[i * n + j].x, Z[i * n + j].y);
        best = fmax(best, sum);
    }
    colmax[threadIdx.x] = best;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) colmax[threadIdx.x] = fmax(colmax[threadIdx.x], colmax[threadIdx.x + o]);
        __syncthreads();
    }
    const double nrm = colmax[0];
    int s = 0;
    while (s < 16 && ldexp(nrm, -s) > 0.5) ++s;
    const double scale = ldexp(1.0, -s);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        X[e] = make_double2(scale * Z[e].x, scale * Z[e].y);
    if (threadIdx.x == 0) *s_out = s;
}

// dst = sum_u src_u over nb N x N units (fixed order)
__global__ void k_sum_units(long long NN, int nb, const double2* __restrict__ src,
                            double2* __restrict__ dst) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NN) return;
    double re = 0.0, im = 0.0;
    for (int u = 0; u < nb; ++u) {
        re += src[u * NN + e].x;
        im += src[u * NN + e].y;
    }
    dst[e] = make_double2(re, im);
}

// ---------------------------------------------------------------------------
// Gradient with respect to the Coulomb integrals (FP64 path).
// ---------------------------------------------------------------------------
// out[a][K] += sum_{u, c, b} S_c(u, a, b) X[u][c][b][K]   (K < N^3)
// with S_c the real (c = 0) / imaginary (c = 1) part of Sbar_u[a][b], or of
// Sbar_u[b][a] when transposeS; X planar complex [u][c][N][N^3] (unit stride
// 2 N^4), i.e. out = Re sum conj(Sbar) X over the contracted index.
__global__ void k_vbar_slot(int N, int nb, const double2* __restrict__ Sbar, int transposeS,
                            const double* __restrict__ X, double* __restrict__ out) {
    const long long N3 = (long long)N * N * N;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N3 * N) return;
    const int a = (int)(e / N3);
    const long long K = e % N3;
    const long long NN = (long long)N * N;
    double acc = 0.0;
    for (int u = 0; u < nb; ++u) {
        const double* xu = X + (long long)u * 2 * N * N3;
        const double2* su = Sbar + (long long)u * NN;
        for (int b = 0; b < N; ++b) {
            const double2 sv = transposeS ? su[(long long)b * N + a] : su[(long long)a * N + b];
            acc = fma(sv.x, xu[(long long)b * N3 + K], acc);
            acc = fma(sv.y, xu[N3 * N + (long long)b * N3 + K], acc);
        }
    }
    out[e] += acc;
}
// vbar[a][b][c][d] += vslot[a][(d, b, c)] + 2 wslot[d][(a, c, b)] - wslot[d][(b, c, a)]
// (vslot[i][(n,r,p)] = dL/dv_irpn; wslot[j][(m,s,q)] = dL/dw_mqsj, w_mqsj = 2 v_mqsj - v_qmsj)
__global__ void k_fold_vbar(int N, const double* __restrict__ vslot, const double* __restrict__ wslot,
                            double* __restrict__ vbar) {
    const long long n = N;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n * n * n) return;
    const long long d = e % n, c = (e / n) % n, b = (e / n / n) % n, a = e / n / n / n;
    const long long N3 = n * n * n;
    double x = vslot[a * N3 + (d * n + b) * n + c];
    x += 2.0 * wslot[d * N3 + (a * n + c) * n + b];
    x -= wslot[d * N3 + (b * n + c) * n + a];
    vbar[e] += x;
}
// Mean-field part, for h = ... + Sigma_HF(rho), Sigma_HF_ij = sum_kl (2 v_iklj - v_ikjl) rho_lk:
// vbar[a][b][c][d] += 2 Re(conj(hbar_ad) rho_cb) - Re(conj(hbar_ac) rho_db)
__global__ void k_vbar_mean_field(int N, const double2* __restrict__ hb, const double2* __restrict__ rho,
                                  double* __restrict__ vbar) {
    const long long n = N;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n * n * n) return;
    const long long d = e % n, c = (e / n) % n, b = (e / n / n) % n, a = e / n / n / n;
    const double2 h1 = hb[a * n + d], r1 = rho[c * n + b];
    const double2 h2 = hb[a * n + c], r2 = rho[d * n + b];
    vbar[e] += 2.0 * (h1.x * r1.x + h1.y * r1.y) - (h2.x * r2.x + h2.y * r2.y);
}
// omega layout for the w-slot chain: wO[i][n][p][r] = v_irpn
__global__ void k_build_vomega64(int N, const double* __restrict__ v, double* __restrict__ out) {
    const long long n = N;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n * n * n) return;
    const long long r = e % n, p = (e / n) % n, nn = (e / n / n) % n, i = e / n / n / n;
    out[e] = v[((i * n + r) * n + p) * n + nn];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host wrappers
// ---------------------------------------------------------------------------

gkba_status fp64_prepare_model(gkba_ctx* c) {
    const long long n = c->N, N4 = n * n * n * n;
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_build_hfK<<<grid1(N4, 256), 256, 0, c->stream>>>(c->N, c->v, c->hfK);
    GKBA_TRY(launch_end(c, t));
    if (c->prec != GKBA_FP64 || c->kind != GKBA_V_GENERAL) return GKBA_OK;
    t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_build_wS64<<<grid1(N4, 256), 256, 0, c->stream>>>(c->N, c->v, c->wS64);
    GKBA_TRY(launch_end(c, t));
    t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_build_vK64<<<grid1(N4, 256), 256, 0, c->stream>>>(c->N, c->v, c->vK64);
    return launch_end(c, t);
}

gkba_status gemm64_stage(gkba_ctx* c, int cls, const double* A, long long lda, long long sAz,
                         const double* B, long long ldb, long long sBz, double* out,
                         long long sOz, int M, int Nc, long long Ktot, int nz, int splitk,
                         long long Kc, StageMap map, double flops, double bytes) {
    dim3 grid((Nc + G64_BN - 1) / G64_BN, (M + G64_BM - 1) / G64_BM, nz);
    if (grid.y > 65535u) return fail(c, GKBA_EINVAL, "stage GEMM: M=%d too large", M);
    auto t = launch_begin(c, cls, flops, bytes);
    k_gemm64_stage<<<grid, 256, 0, c->stream>>>(A, lda, sAz, B, ldb, sBz, out, sOz, M, Nc, Ktot,
                                                splitk, Kc, map);
    return launch_end(c, t);
}

long long gemm64_splitk_chunk(gkba_ctx* c, int M, int Nc, long long K, long long max_chunks) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemm64_stage, 256, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long bpz = (long long)((Nc + G64_BN - 1) / G64_BN) * ((M + G64_BM - 1) / G64_BM);
    long long nz = std::max(1LL, (long long)per_sm * c->num_sms / bpz);
    nz = std::min(nz, std::max(1LL, max_chunks));
    const long long Kc = (K + nz - 1) / nz;
    return (Kc + G64_BK - 1) / G64_BK * G64_BK;
}

static gkba_status zgemm_impl(gkba_ctx* c, int cls, int n, char opA, char opB, double2 alpha,
                              const double2* A, long long sA, const double2* B, long long sB,
                              double2 beta, double2* C, long long sC, int batch, int add_identity,
                              const int* skip_ge, int idx) {
    if (batch <= 0) return GKBA_OK;
    dim3 grid((n + ZT - 1) / ZT, (n + ZT - 1) / ZT, 1);
    const double flops = 8.0 * n * (double)n * n;
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nbat = batch - b0 < 65535 ? batch - b0 : 65535;
        grid.z = nbat;
        auto t = launch_begin(c, cls, flops * nbat, 0.0);
        k_zgemm<<<grid, 256, 0, c->stream>>>(n, opA == 'C', opB == 'C', alpha, A + b0 * sA, sA,
                                             B + b0 * sB, sB, beta, C + b0 * sC, sC, add_identity,
                                             skip_ge, idx);
        GKBA_TRY(launch_end(c, t));
    }
    return GKBA_OK;
}

gkba_status zgemm_batched(gkba_ctx* c, int cls, int n, char opA, char opB, double2 alpha,
                          const double2* A, long long sA, const double2* B, long long sB,
                          double2 beta, double2* C, long long sC, int batch, int add_identity) {
    return zgemm_impl(c, cls, n, opA, opB, alpha, A, sA, B, sB, beta, C, sC, batch, add_identity,
                      nullptr, 0);
}

gkba_status mean_field(gkba_ctx* c, const double2* rho, double2* out) {
    const int NN = c->N * c->N;
    auto t = launch_begin(c, K_STEP, 8.0 * NN * (double)NN, 8.0 * NN * (double)NN);
    k_mean_field<<<grid1((long long)NN * 32, 256), 256, 0, c->stream>>>(c->N, c->hfK, rho, c->h,
                                                                         c->d, 0.0, 0, out);
    return launch_end(c, t);
}

gkba_status h_hf(gkba_ctx* c, double E, const double2* rho, double2* out) {
    const int NN = c->N * c->N;
    auto t = launch_begin(c, K_STEP, 8.0 * NN * (double)NN, 8.0 * NN * (double)NN);
    k_mean_field<<<grid1((long long)NN * 32, 256), 256, 0, c->stream>>>(c->N, c->hfK, rho, c->h,
                                                                         c->d, E, 1, out);
    return launch_end(c, t);
}

gkba_status rhs(gkba_ctx* c, const double2* hhf, const double2* rho, const double2* I, double2* out) {
    const int N = c->N;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'N', one, hhf, 0, rho, 0, zero, c->tmp0, 0, 1, 0));
    GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'N', one, rho, 0, hhf, 0, zero, c->tmp1, 0, 1, 0));
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_rhs<<<grid1((long long)N * N, 256), 256, 0, c->stream>>>(N, c->tmp0, c->tmp1, I, out);
    return launch_end(c, t);
}

gkba_status expm_step(gkba_ctx* c, const double2* hA, const double2* hB, double2* U) {
    // Scaling and squaring with a degree-18 Taylor polynomial (Moler & Van Loan,
    // "Nineteen dubious ways to compute the exponential of a matrix"): with
    // ||A/2^s||_1 <= 1/2 the truncation error is below 0.5^19/19! ~ 1e-23.
    const int N = c->N;
    const long long NN = (long long)N * N;
    double2* X = c->ex0;  // scaled argument B = A / 2^s
    double2* Y = c->ex1;
    double2* Z = c->ex2;
    if (N <= kExpmSmallN) {
        auto t = launch_begin(c, K_STEP, 0.0, 0.0);
        k_expm_small<<<1, 256, 0, c->stream>>>(N, c->dt, hA, hB, U, c->dscal + 8, c->dint + 0);
        return launch_end(c, t);
    }
    {
        auto t = launch_begin(c, K_STEP, 0.0, 0.0);
        k_expm_setup<<<1, 256, 0, c->stream>>>(N, c->dt, hA, hB, X, c->dscal + 8, c->dint + 0);
        GKBA_TRY(launch_end(c, t));
    }
    const int deg = 18;
    // Y = I + X / deg
    {
        auto t = launch_begin(c, K_STEP, 0.0, 0.0);
        k_set_identity<<<grid1(NN, 256), 256, 0, c->stream>>>(N, 1, Y);
        GKBA_TRY(launch_end(c, t));
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'N', make_double2(1.0 / deg, 0.0), X, 0, Y, 0,
                               make_double2(0.0, 0.0), Z, 0, 1, 1));
        std::swap(Y, Z);
    }
    for (int k = deg - 1; k >= 1; --k) {
        GKBA_TRY(zgemm_batched(c, K_STEP, N, 'N', 'N', make_double2(1.0 / k, 0.0), X, 0, Y, 0,
                               make_double2(0.0, 0.0), Z, 0, 1, 1));
        std::swap(Y, Z);
    }
    // up to kMaxSq squarings; step i is a copy when i >= s (device-side count)
    const int kMaxSq = 16;
    for (int i = 0; i < kMaxSq; ++i) {
        GKBA_TRY(zgemm_impl(c, K_STEP, N, 'N', 'N', make_double2(1.0, 0.0), Y, 0, Y, 0,
                            make_double2(0.0, 0.0), Z, 0, 1, 0, c->dint + 0, i));
        std::swap(Y, Z);
    }
    GKBA_CUDA(c, cudaMemcpyAsync(U, Y, NN * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    return GKBA_OK;
}

gkba_status axpy_c(gkba_ctx* c, double2* y, const double2* x, const double2* z, double a, double b,
                   int n) {
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_lincomb<<<grid1(n, 256), 256, 0, c->stream>>>(n, y, x, z, a, b);
    return launch_end(c, t);
}

gkba_status set_identity(gkba_ctx* c, double2* A, int count) {
    const long long n = (long long)c->N * c->N * count;
    if (n == 0) return GKBA_OK;
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_set_identity<<<grid1(n, 256), 256, 0, c->stream>>>(c->N, count, A);
    return launch_end(c, t);
}

gkba_status diagnostics(gkba_ctx* c, double E_n, const double2* rho, const double2* I, double* out4) {
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_diagnostics<<<1, 256, 0, c->stream>>>(c->N, E_n, c->h, c->d, c->hhf_n, rho, I, out4);
    return launch_end(c, t);
}

// P_k = T_k rho_k, Q_k = T_k - P_k for k in [k0, k0+nk), then the unit list.
// The G_u are staged in Su (free until the reduction of this batch).
gkba_status build_forms_gkba(gkba_ctx* c, int k0, int nk, int L, const double2* rho,
                             const double2* T, const double* w) {
    const int N = c->N;
    const long long NN = (long long)N * N;
    double2* P = c->PQ;
    double2* Q = c->PQ + (long long)nk * NN;
    GKBA_TRY(zgemm_batched(c, K_PREP, N, 'N', 'N', make_double2(1.0, 0.0), T + k0 * NN, NN,
                           rho + k0 * NN, NN, make_double2(0.0, 0.0), P, NN, nk, 0));
    {
        auto t = launch_begin(c, K_PREP, 0.0, 0.0);
        k_lincomb<<<grid1(nk * NN, 256), 256, 0, c->stream>>>(nk * NN, Q, T + k0 * NN, P, 1.0, -1.0);
        GKBA_TRY(launch_end(c, t));
    }
    {
        auto t = launch_begin(c, K_PREP, 0.0, 0.0);
        k_gkba_units<<<grid1(nk * NN, 256), 256, 0, c->stream>>>(N, nk, k0, L, c->dt, P, Q, w,
                                                                  c->Su, c->Mb, c->coef);
        GKBA_TRY(launch_end(c, t));
    }
    return build_forms(c, 2 * nk, c->Su, NN, c->Mb, NN, 0);
}

// Units of history points k0 .. k0+nk-1 of one system (history of L points,
// trapezoid weights with dt when w is null) written to G / Gb / coef (unit
// stride N*N), with c->PQ as scratch.  Used by stacked batches of systems.
gkba_status units_from_history(gkba_ctx* c, int N, int k0, int nk, int L, double dt,
                               const double2* rho, const double2* T, const double* w, double2* G,
                               double2* Gb, double* coef) {
    const long long NN = (long long)N * N;
    double2* P = c->PQ;
    double2* Q = c->PQ + (long long)nk * NN;
    GKBA_TRY(zgemm_batched(c, K_PREP, N, 'N', 'N', make_double2(1.0, 0.0), T + k0 * NN, NN,
                           rho + k0 * NN, NN, make_double2(0.0, 0.0), P, NN, nk, 0));
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_lincomb<<<grid1(nk * NN, 256), 256, 0, c->stream>>>(nk * NN, Q, T + k0 * NN, P, 1.0, -1.0);
    GKBA_TRY(launch_end(c, t));
    t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_gkba_units<<<grid1(nk * NN, 256), 256, 0, c->stream>>>(N, nk, k0, L, dt, P, Q, w, G, Gb, coef);
    return launch_end(c, t);
}

// I += sum_u coef[u] Y[u] over nb units of one system (N x N), two passes.
gkba_status weighted_sum_units(gkba_ctx* c, int N, int nb, const double* coef, const double2* Y,
                               double2* I) {
    const long long NN = (long long)N * N;
    const int nz = nb < kWsumRanges ? nb : kWsumRanges;
    const int per = (nb + nz - 1) / nz;
    auto t = launch_begin(c, K_RED, 0.0, 0.0);
    k_weighted_sum_p1<<<dim3(grid1(NN, 128), nz), 128, 0, c->stream>>>((int)NN, nb, per, coef, Y,
                                                                       c->red_tmp);
    GKBA_TRY(launch_end(c, t));
    t = launch_begin(c, K_RED, 0.0, 0.0);
    k_weighted_sum_p2<<<grid1(NN, 256), 256, 0, c->stream>>>((int)NN, nz, c->red_tmp, I);
    return launch_end(c, t);
}

gkba_status unit_xform(gkba_ctx* c, int nb, const double2* in, double2* out, int conj, int transpose) {
    const long long n = (long long)nb * c->N * c->N;
    auto t = launch_begin(c, K_RED, 0.0, 0.0);
    k_unit_xform<<<grid1(n, 256), 256, 0, c->stream>>>(c->N, n, in, out, conj, transpose);
    return launch_end(c, t);
}
gkba_status unit_acc(gkba_ctx* c, int nb, double2* y, const double2* x, int transpose) {
    const long long n = (long long)nb * c->N * c->N;
    auto t = launch_begin(c, K_RED, 0.0, 0.0);
    k_unit_acc<<<grid1(n, 256), 256, 0, c->stream>>>(c->N, n, y, x, transpose);
    return launch_end(c, t);
}
gkba_status scale_units(gkba_ctx* c, int nb, const double* coef, const double2* Ibar, double2* Y) {
    const long long n = (long long)nb * c->N * c->N;
    auto t = launch_begin(c, K_RED, 0.0, 0.0);
    k_scale_units<<<grid1(n, 256), 256, 0, c->stream>>>(c->N, nb, coef, Ibar, Y);
    return launch_end(c, t);
}
gkba_status vjp_points(gkba_ctx* c, int nk, const double2* Gbar, const double2* Gbbar, double2* Pbar,
                       double2* Qbar) {
    const long long n = (long long)nk * c->N * c->N;
    auto t = launch_begin(c, K_RED, 0.0, 0.0);
    k_vjp_points<<<grid1(n, 256), 256, 0, c->stream>>>(c->N, nk, Gbar, Gbbar, Pbar, Qbar);
    return launch_end(c, t);
}

gkba_status add_i_diff(gkba_ctx* c, double2* y, const double2* a, const double2* b, double s) {
    const long long n = (long long)c->N * c->N;
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_add_i_diff<<<grid1(n, 256), 256, 0, c->stream>>>(n, y, a, b, s);
    return launch_end(c, t);
}
gkba_status ibar_from_kbar(gkba_ctx* c, const double2* kb, double2* Ib) {
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_ibar_from_kbar<<<grid1((long long)c->N * c->N, 256), 256, 0, c->stream>>>(c->N, kb, Ib);
    return launch_end(c, t);
}
gkba_status mean_field_adj(gkba_ctx* c, const double2* hb, double2* rb) {
    const int NN = c->N * c->N;
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_mean_field_adj<<<grid1((long long)NN * 32, 256), 256, 0, c->stream>>>(c->N, c->hfK, hb, rb);
    return launch_end(c, t);
}
gkba_status field_grad(gkba_ctx* c, const double2* hb, double* out) {
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_field_grad<<<1, 256, 0, c->stream>>>(c->N, hb, c->d, out);
    return launch_end(c, t);
}
// exp(Z) of a general complex n x n matrix (Taylor degree 18 by Horner after
// scaling, then the squarings); X, Y, W: n x n scratch, result in W.
static gkba_status expm_general(gkba_ctx* c, int n, const double2* Z, double2* X, double2* Y,
                                double2* W) {
    {
        auto t = launch_begin(c, K_STEP, 0.0, 0.0);
        k_expm_setup_general<<<1, 256, 0, c->stream>>>(n, Z, X, c->dint + 0);
        GKBA_TRY(launch_end(c, t));
        t = launch_begin(c, K_STEP, 0.0, 0.0);
        k_set_identity<<<grid1((long long)n * n, 256), 256, 0, c->stream>>>(n, 1, Y);
        GKBA_TRY(launch_end(c, t));
    }
    double2 *y = Y, *z = W;
    for (int k = 18; k >= 1; --k) {
        GKBA_TRY(zgemm_batched(c, K_STEP, n, 'N', 'N', make_double2(1.0 / k, 0.0), X, 0, y, 0,
                               make_double2(0.0, 0.0), z, 0, 1, 1));
        std::swap(y, z);
    }
    for (int i = 0; i < 16; ++i) {
        GKBA_TRY(zgemm_impl(c, K_STEP, n, 'N', 'N', make_double2(1.0, 0.0), y, 0, y, 0,
                            make_double2(0.0, 0.0), z, 0, 1, 0, c->dint + 0, i));
        std::swap(y, z);
    }
    if (y != W)
        GKBA_CUDA(c, cudaMemcpyAsync(W, y, (size_t)n * n * sizeof(double2), cudaMemcpyDeviceToDevice,
                                     c->stream));
    return GKBA_OK;
}
// Adjoint of U = exp(-i dt (hA + hB)/2): hA_bar, hB_bar += (i dt / 2) L_exp(X^+, Ubar).
// scratch: 4 blocks of (2N)^2 entries.
gkba_status expm_adj(gkba_ctx* c, const double2* hA, const double2* hB, const double2* Ubar,
                     double2* hA_bar, double2* hB_bar, double2* scratch) {
    const int N = c->N, M = 2 * N;
    const long long MM = (long long)M * M;
    double2 *Z = scratch, *X = scratch + MM, *Y = scratch + 2 * MM, *W = scratch + 3 * MM;
    {
        auto t = launch_begin(c, K_STEP, 0.0, 0.0);
        k_frechet_block<<<1, 256, 0, c->stream>>>(N, c->dt, hA, hB, Ubar, Z, c->dscal + 12);
        GKBA_TRY(launch_end(c, t));
    }
    GKBA_TRY(expm_general(c, M, Z, X, Y, W));
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_frechet_apply<<<grid1((long long)N * N, 256), 256, 0, c->stream>>>(N, c->dt, W, c->dscal + 12,
                                                                         hA_bar, hB_bar);
    return launch_end(c, t);
}

gkba_status sum_units(gkba_ctx* c, int nb, const double2* src, double2* dst) {
    const long long NN = (long long)c->N * c->N;
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_sum_units<<<grid1(NN, 256), 256, 0, c->stream>>>(NN, nb, src, dst);
    return launch_end(c, t);
}

gkba_status vbar_slot(gkba_ctx* c, int nb, const double2* Sbar, int transposeS, const double* X,
                      double* out) {
    const long long n = (long long)c->N * c->N * c->N * c->N;
    auto t = launch_begin(c, K_RED, 0.0, 0.0);
    k_vbar_slot<<<grid1(n, 256), 256, 0, c->stream>>>(c->N, nb, Sbar, transposeS, X, out);
    return launch_end(c, t);
}
gkba_status fold_vbar(gkba_ctx* c, const double* vslot, const double* wslot, double* vbar) {
    const long long n = (long long)c->N * c->N * c->N * c->N;
    auto t = launch_begin(c, K_RED, 0.0, 0.0);
    k_fold_vbar<<<grid1(n, 256), 256, 0, c->stream>>>(c->N, vslot, wslot, vbar);
    return launch_end(c, t);
}
gkba_status vbar_mean_field(gkba_ctx* c, const double2* hb, const double2* rho, double* vbar) {
    const long long n = (long long)c->N * c->N * c->N * c->N;
    auto t = launch_begin(c, K_STEP, 0.0, 0.0);
    k_vbar_mean_field<<<grid1(n, 256), 256, 0, c->stream>>>(c->N, hb, rho, vbar);
    return launch_end(c, t);
}
gkba_status build_vomega64(gkba_ctx* c, double* out) {
    const long long n = (long long)c->N * c->N * c->N * c->N;
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_build_vomega64<<<grid1(n, 256), 256, 0, c->stream>>>(c->N, c->v, out);
    return launch_end(c, t);
}

gkba_status build_forms_fp64(gkba_ctx* c, int nb, const double2* G, const double2* Gb) {
    const long long NN = (long long)c->N * c->N;
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_forms64<<<grid1(nb * NN, 256), 256, 0, c->stream>>>(c->N, nb, G, Gb, (double*)c->formsB1,
                                                          (double*)c->formsG);
    return launch_end(c, t);
}

// G forms of stage S3 from a separate matrix A (trilinear S3(A, B, C)).
gkba_status build_forms3_fp64(gkba_ctx* c, int nb, const double2* A) {
    const long long NN = (long long)c->N * c->N;
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_forms64<<<grid1(nb * NN, 256), 256, 0, c->stream>>>(c->N, nb, A, nullptr, nullptr,
                                                          (double*)c->formsG3);
    return launch_end(c, t);
}

gkba_status reduce_partials_launch(gkba_ctx* c, int nb, int nz, long long zstride, long long Rld,
                                   const void* part, bool fp32, double2* S) {
    const long long NN = (long long)c->N * c->N;
    const int nzc = nz < kReduceSplit ? nz : kReduceSplit;
    const int zper = (nz + nzc - 1) / nzc;
    const int Np = tensor_core_path(c) ? c->Np : c->N;
    dim3 g1(grid1(nb * NN, 256), nzc);
    auto t = launch_begin(c, K_RED, 0.0, 0.0);
    if (fp32)
        k_reduce_partials_p1<float><<<g1, 256, 0, c->stream>>>(c->N, Np, nb, nz, zper, zstride, Rld,
                                                               (const float*)part, c->red_tmp);
    else
        k_reduce_partials_p1<double><<<g1, 256, 0, c->stream>>>(c->N, Np, nb, nz, zper, zstride,
                                                                Rld, (const double*)part, c->red_tmp);
    GKBA_TRY(launch_end(c, t));
    t = launch_begin(c, K_RED, 0.0, 0.0);
    k_reduce_partials_p2<<<grid1(nb * NN, 256), 256, 0, c->stream>>>(nb * NN, nzc, c->red_tmp, S);
    return launch_end(c, t);
}

// Y_u = S_u Gb_u, I_acc += sum_u coef_u Y_u (fixed order).  When S_out is
// non-null the S_u are copied out instead (gkba_sigma).
gkba_status reduce_batch(gkba_ctx* c, int nb, double2* I_acc, double2* S_out) {
    const int N = c->N;
    const long long NN = (long long)N * N;
    if (S_out != nullptr) {
        GKBA_CUDA(c, cudaMemcpyAsync(S_out, c->Su, nb * NN * sizeof(double2),
                                     cudaMemcpyDeviceToDevice, c->stream));
        return GKBA_OK;
    }
    GKBA_TRY(zgemm_batched(c, K_RED, N, 'N', 'N', make_double2(1.0, 0.0), c->Su, NN, c->Mb, NN,
                           make_double2(0.0, 0.0), c->Yu, NN, nb, 0));
    // nz <= nb <= ub ranges of N*N entries: red_tmp holds 16 ub of them
    const int nz = nb < kWsumRanges ? nb : kWsumRanges;
    const int per = (nb + nz - 1) / nz;
    auto t = launch_begin(c, K_RED, 0.0, 0.0);
    k_weighted_sum_p1<<<dim3(grid1(NN, 128), nz), 128, 0, c->stream>>>((int)NN, nb, per, c->coef,
                                                                       c->Yu, c->red_tmp);
    GKBA_TRY(launch_end(c, t));
    t = launch_begin(c, K_RED, 0.0, 0.0);
    k_weighted_sum_p2<<<grid1(NN, 256), 256, 0, c->stream>>>((int)NN, nz, c->red_tmp, I_acc);
    return launch_end(c, t);
}

// FP64 contraction of one batch (units 0..nb-1 with forms built):
//   S1  X1[j][r][m][c][q] = sum_s wS[j][m][q][s] B1[(c,r)][s]
//   S2  X2[j][r][p][c'][m] = sum_(c,q) X1[(j,r,m)][(c,q)] Gr[(c',p)][(c,q)]
//   S3  X3[c'][j][n][r][p] = sum_(c,m) X2[(j,r,p)][(c,m)] Gr[(c',n)][(c,m)]
//   S4  D[(u,c,j)][i] = sum_(n,r,p) X3[u][(c,j)][(n,r,p)] vK[i][(n,r,p)], split-K
// i.e. W1 = w x_s Gb, W2 = G x_q W1, W3 = G x_m W2, Sigma = v . W3.
// Stages S1-S3 of the FP64 chain into X13 = X3[u][c'][j][n][r][p], with A1
// the stage-S1 operand (w in the [j][m][q][s] layout, or any tensor in it).
// m3 / sOz3, when given, replace the output scatter of S3 (rows (j, r, p),
// columns (c', n), unit offset sOz3).
gkba_status fp64_chain_x3(gkba_ctx* c, int nb, const double* A1, const StageMap* m3,
                          long long sOz3) {
    const int N = c->N;
    const long long N2 = (long long)N * N, N3 = N2 * N, N4 = N3 * N;
    double* X13 = (double*)c->X13;
    double* X2 = (double*)c->X2;
    const double fl_cr = 4.0 * (double)N4 * N;   // complex x real stage, per unit
    const double fl_cc = 8.0 * (double)N4 * N;   // complex x complex stage, per unit
    {
        StageMap m{2 * N3, 2 * N, 1, N, 2 * N2, N, N, N};
        GKBA_TRY(gemm64_stage(c, K_W1, A1, N, 0, (const double*)c->formsB1, N, 2 * N2, X13,
                              2 * N4, (int)N3, 2 * N, N, nb, 0, 0, m, fl_cr * nb,
                              8.0 * (N4 + 2 * N4 * nb)));
    }
    {
        StageMap m{2 * N3, 2 * N2, 1, N, 2 * N, N, N, N};
        GKBA_TRY(gemm64_stage(c, K_W2, X13, 2 * N, 2 * N4, (const double*)c->formsG, 2 * N, 4 * N2,
                              X2, 2 * N4, (int)N3, 2 * N, 2 * N, nb, 0, 0, m, fl_cc * nb,
                              8.0 * 4 * N4 * nb));
    }
    {
        const StageMap m = m3 ? *m3 : StageMap{N3, N, 1, N4, N2, N, N, N};
        GKBA_TRY(gemm64_stage(c, K_W3, X2, 2 * N, 2 * N4,
                              (const double*)(c->sep_A ? c->formsG3 : c->formsG), 2 * N, 4 * N2,
                              X13, m3 ? sOz3 : 2 * N4, (int)N3, 2 * N, 2 * N, nb, 0, 0, m,
                              fl_cc * nb, 8.0 * 4 * N4 * nb));
    }
    return GKBA_OK;
}

gkba_status contract_batch_fp64(gkba_ctx* c, int nb) {
    const int N = c->N;
    const long long N2 = (long long)N * N, N3 = N2 * N, N4 = N3 * N;
    double* X13 = (double*)c->X13;
    const double fl_cr = 4.0 * (double)N4 * N;
    GKBA_TRY(fp64_chain_x3(c, nb, c->wS64));
    const long long R = 2LL * N * nb;
    const long long Kc = 8192;
    const int nz = (int)((N3 + Kc - 1) / Kc);
    {
        StageMap m{0, 0, 1, 0, R, (int)R, 1, N};
        GKBA_TRY(gemm64_stage(c, K_FIN, X13, N3, 0, c->vK64, N3, 0, (double*)c->part, N * R,
                              (int)R, N, N3, nz, 1, Kc, m, fl_cr * nb,
                              8.0 * (2 * N4 * nb + N4)));
    }
    return reduce_partials_launch(c, nb, nz, N * R, R, c->part, false, c->Su);
}

// Self-energy of a structured interaction for nb units (G_u, Gb_u device
// pointers with stride N*N) into c->Su; the kernels write c->PQ (free at this
// point of a batch) because G may alias c->Su.
gkba_status contract_structured(gkba_ctx* c, int nb, const double2* G, const double2* Gb) {
    const int N = c->N;
    const long long NN = (long long)N * N;
    const double n = N;
    if (c->kind == GKBA_V_DIAGONAL) {
        auto t = launch_begin(c, K_W1, 6.0 * n * n * nb, 48.0 * n * n * nb);
        k_sigma_diag<<<grid1(nb * NN, 256), 256, 0, c->stream>>>(N, nb, c->vm, G, Gb, c->PQ);
        GKBA_TRY(launch_end(c, t));
    } else if (N <= kSymmSmallN) {
        const int bs = N * N >= 256 ? 256 : ((N * N + 31) / 32) * 32;
        auto t = launch_begin(c, K_W1, 8.0 * n * n * n * n * nb, 48.0 * n * n * nb);
        k_sigma_symm_small<<<nb, bs, 0, c->stream>>>(N, c->vm, G, Gb, c->PQ);
        GKBA_TRY(launch_end(c, t));
    } else {
        const int bs = N >= 128 ? 128 : ((N + 31) / 32) * 32;
        auto t = launch_begin(c, K_W1, 8.0 * n * n * n * n * nb, 48.0 * n * n * nb);
        k_sigma_symm<<<dim3(N, nb), bs, N * sizeof(double2), c->stream>>>(N, c->vm, G, Gb, c->PQ);
        GKBA_TRY(launch_end(c, t));
    }
    GKBA_CUDA(c, cudaMemcpyAsync(c->Su, c->PQ, nb * NN * sizeof(double2), cudaMemcpyDeviceToDevice,
                                 c->stream));
    return GKBA_OK;
}

}  // namespace gkba

namespace gkba {

// ---------------------------------------------------------------------------
// Allocation-free FP64 self-energy (gkba_sigma_noalloc, include/gkba.h).
//
// For callers that cannot allocate device memory (code that runs while a
// CUDA graph is being captured, inside a host framework that owns every
// allocation, or under a fixed memory budget), this entry point evaluates the
// same FP64 contraction as gkba_sigma without a context and without any
// allocation: its scratch is the file-scope array below, which every GPU that
// loads the library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB per device
constexpr int kNoAllocMaxN = 24;
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device ordinal (null until set up).
void* g_noalloc_addr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mu;

gkba_status noalloc_fail(char* err, size_t err_len, gkba_status st, const char* fmt, ...) {
    if (err != nullptr && err_len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, err_len, fmt, ap);
        va_end(ap);
    }
    return st;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

}  // namespace gkba

extern "C" gkba_status gkba_sigma_noalloc(int N, int n_units, const double* v, const double* G,
                                          const double* Gbar, double* S_out, void* cuda_stream,
                                          char* err, size_t err_len) {
    using namespace gkba;
    if (err != nullptr && err_len > 0) err[0] = '\0';
    if (N < 1 || N > kNoAllocMaxN)
        return noalloc_fail(err, err_len, GKBA_EINVAL,
                            "gkba_sigma_noalloc: N=%d outside [1, %d] (static scratch of %zu bytes)", N,
                            kNoAllocMaxN, kNoAllocScratchBytes);
    if (n_units < 0) return noalloc_fail(err, err_len, GKBA_EINVAL, "gkba_sigma_noalloc: n_units < 0");
    if (n_units == 0) return GKBA_OK;
    if (!v || !G || !Gbar || !S_out)
        return noalloc_fail(err, err_len, GKBA_EINVAL, "gkba_sigma_noalloc: NULL pointer argument");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess)
        return noalloc_fail(err, err_len, GKBA_ECUDA, "gkba_sigma_noalloc: cudaGetDevice: %s",
                            cudaGetErrorString(ce));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return noalloc_fail(err, err_len, GKBA_EUNSUPPORTED, "gkba_sigma_noalloc: device %d", dev);
    void* base = nullptr;
    {
        // Set-up once per device (with that device current): the host-side
        // symbol is a stand-in, so the kernels get the device address.
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (g_noalloc_addr[dev] == nullptr) {
            void* p = nullptr;
            ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (ce != cudaSuccess || p == nullptr)
                return noalloc_fail(err, err_len, GKBA_ECUDA,
                                    "gkba_sigma_noalloc: cudaGetSymbolAddress: %s",
                                    cudaGetErrorString(ce));
            g_noalloc_addr[dev] = p;
        }
        base = g_noalloc_addr[dev];
    }
    const long long n = N, NN = n * n, N3 = NN * n, N4 = N3 * n;
    const long long Kc = 8192;
    const int nz = (int)((N3 + Kc - 1) / Kc);
    // scratch layout: wS | vK | per-batch: B1 | Gr | X13 | X2 | part | red
    const size_t model_b = 2 * round256((size_t)N4 * 8);
    const size_t unit_b = round256((size_t)2 * NN * 8) + round256((size_t)4 * NN * 8) +
                          2 * round256((size_t)2 * N4 * 8) + round256((size_t)nz * n * 2 * n * 8) +
                          round256((size_t)kReduceSplit * NN * 16);
    if (model_b + unit_b > kNoAllocScratchBytes)
        return noalloc_fail(err, err_len, GKBA_EINVAL, "gkba_sigma_noalloc: N=%d does not fit", N);
    const int ub = (int)std::min<size_t>((kNoAllocScratchBytes - model_b) / unit_b, (size_t)n_units);
    char* s = (char*)base;
    double* wS = (double*)s;
    double* vK = (double*)(s + round256((size_t)N4 * 8));
    char* q = s + model_b;
    double* B1 = (double*)q;
    q += round256((size_t)2 * NN * 8 * ub);
    double* Gr = (double*)q;
    q += round256((size_t)4 * NN * 8 * ub);
    double* X13 = (double*)q;
    q += round256((size_t)2 * N4 * 8 * ub);
    double* X2 = (double*)q;
    q += round256((size_t)2 * N4 * 8 * ub);
    double* part = (double*)q;
    q += round256((size_t)nz * n * 2 * n * 8 * ub);
    double2* red = (double2*)q;
    q += round256((size_t)kReduceSplit * NN * 16 * ub);
    if ((size_t)(q - s) > kNoAllocScratchBytes)
        return noalloc_fail(err, err_len, GKBA_EINVAL, "gkba_sigma_noalloc: scratch layout overflow");

    // An error pending from earlier, unrelated work is reported as such and
    // left in place for its owner; launch errors of this call are checked
    // after every group of launches, so a failed launch stops the rest.
    ce = cudaPeekAtLastError();
    if (ce != cudaSuccess)
        return noalloc_fail(err, err_len, GKBA_ECUDA,
                            "gkba_sigma_noalloc: a CUDA error is pending from earlier work: %s",
                            cudaGetErrorString(ce));
    // model operands (rebuilt on every call; every element is written)
    k_build_wS64<<<grid1(N4, 256), 256, 0, stream>>>(N, v, wS);
    k_build_vK64<<<grid1(N4, 256), 256, 0, stream>>>(N, v, vK);
    ce = cudaGetLastError();
    if (ce != cudaSuccess)
        return noalloc_fail(err, err_len, GKBA_ECUDA, "gkba_sigma_noalloc: launch failed: %s",
                            cudaGetErrorString(ce));
    const double2* Gd = (const double2*)G;
    const double2* Gbd = (const double2*)Gbar;
    double2* Sd = (double2*)S_out;
    for (int u0 = 0; u0 < n_units; u0 += ub) {
        const int nb = std::min(ub, n_units - u0);
        k_forms64<<<grid1(nb * NN, 256), 256, 0, stream>>>(N, nb, Gd + u0 * NN, Gbd + u0 * NN, B1, Gr);
        {
            StageMap m{2 * N3, 2 * n, 1, n, 2 * NN, N, N, N};
            dim3 g((2 * N + G64_BN - 1) / G64_BN, (unsigned)((N3 + G64_BM - 1) / G64_BM), nb);
            k_gemm64_stage<<<g, 256, 0, stream>>>(wS, n, 0, B1, n, 2 * NN, X13, 2 * N4, (int)N3,
                                                  2 * N, n, 0, 0, m);
        }
        {
            StageMap m{2 * N3, 2 * NN, 1, n, 2 * n, N, N, N};
            dim3 g((2 * N + G64_BN - 1) / G64_BN, (unsigned)((N3 + G64_BM - 1) / G64_BM), nb);
            k_gemm64_stage<<<g, 256, 0, stream>>>(X13, 2 * n, 2 * N4, Gr, 2 * n, 4 * NN, X2, 2 * N4,
                                                  (int)N3, 2 * N, 2 * n, 0, 0, m);
        }
        {
            StageMap m{N3, n, 1, N4, NN, N, N, N};
            dim3 g((2 * N + G64_BN - 1) / G64_BN, (unsigned)((N3 + G64_BM - 1) / G64_BM), nb);
            k_gemm64_stage<<<g, 256, 0, stream>>>(X2, 2 * n, 2 * N4, Gr, 2 * n, 4 * NN, X13, 2 * N4,
                                                  (int)N3, 2 * N, 2 * n, 0, 0, m);
        }
        const long long R = 2LL * n * nb;
        {
            StageMap m{0, 0, 1, 0, R, (int)R, 1, N};
            dim3 g((N + G64_BN - 1) / G64_BN, (unsigned)((R + G64_BM - 1) / G64_BM), nz);
            k_gemm64_stage<<<g, 256, 0, stream>>>(X13, N3, 0, vK, N3, 0, part, n * R, (int)R, N, N3,
                                                  1, Kc, m);
        }
        const int nzc = nz < kReduceSplit ? nz : kReduceSplit;
        const int zper = (nz + nzc - 1) / nzc;
        dim3 g1(grid1(nb * NN, 256), nzc);
        k_reduce_partials_p1<double><<<g1, 256, 0, stream>>>(N, N, nb, nz, zper, n * R, R, part, red);
        k_reduce_partials_p2<<<grid1(nb * NN, 256), 256, 0, stream>>>(nb * NN, nzc, red, Sd + u0 * NN);
        ce = cudaGetLastError();
        if (ce != cudaSuccess)
            return noalloc_fail(err, err_len, GKBA_ECUDA, "gkba_sigma_noalloc: launch failed: %s",
                                cudaGetErrorString(ce));
    }
    return GKBA_OK;
}

