// tc_kernels.cu - split-TF32 contraction of the second-Born self-energy on
// the sm_103a tensor cores (tcgen05 + TMA + TMEM).
//
// Eq. (2bse) of arXiv:1905.01180 is evaluated as four one-index contractions
// (Sec. III, "general basis"; the ordering contracts w's s index first):
//   S1  X1[j][r][m][c][q]  = sum_s  w_mqsj Gb_c[s][r]                 (w real)
//   S2  X2[j][r][p][c'][m] = sum_q  G[p][q] X1[..][q]                 (complex)
//   S3  X3[c'][j][n][r][p] = sum_m  G[n][m] X2[..][m]                 (complex)
//   S4  Sigma[i][j]        = sum_(n,r,p) v_irpn X3[j][n][r][p]         (v real)
// with w_mqsj = 2 v_mqsj - v_qmsj (direct minus exchange).  Each stage is a
// real GEMM D[M][Nc] = sum_K A[M][K] B[Nc][K]:
//   * A (the large, streamed operand) is FP32 in HBM; TMA stages 128 x 32
//     tiles (128-byte swizzle) in shared memory, a converter warpgroup splits
//     every element into TF32 hi and lo (x = hi + lo, see split_tf32 and, for
//     S4, split_tf32_exact_lo) and writes both into tensor memory
//     (tcgen05.st), where the MMA reads A;
//   * B (the small per-unit matrix, or v for S4) is stored pre-split hi/lo;
//   * each K-step issues hi*hi + hi*lo + lo*hi (3xTF32) into an FP32 TMEM
//     accumulator; S4 accumulates every 32-wide K chunk in its own window,
//     adds the windows of a work item (4096 K by default) with Kahan in FP32
//     registers, and the reduction kernel adds the items' partial sums.
// S1-S3 run on CTA pairs (cta_group::2, M = 256): B's rows are split between
// the two CTAs' shared memory, which leaves room for the complex B' that
// turns the planar (Re, Im) halves of A into one real K range:
// [[Re G | -Im G]; [Im G | Re G]].
//
// Every mbarrier wait is bounded (globaltimer); on timeout the kernel raises
// an abort flag, records an error word, drains its in-flight TMA loads and
// MMAs, frees its tensor memory and returns.
#include <cuda.h>

#include <algorithm>
#include <cstdlib>

#include "gkba_internal.cuh"
#include "tf32_round.h"

namespace gkba {

namespace {

constexpr unsigned long long kWaitLimitNs = 4000000000ull;  // 4 s per wait
constexpr int kBM = 128;                                   // rows per tile (TMEM lanes)
constexpr int kKC = 32;                                    // K floats per chunk (128 B rows)
constexpr int kTileBytes = kBM * kKC * 4;                  // 16 KiB

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* m) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)m) : "memory");
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* m, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4}], [%2];" ::"r"(dst),
        "l"((unsigned long long)m), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap* m, uint32_t bar, int x, int y,
                                       int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4, %5}], [%2];" ::"r"(dst),
        "l"((unsigned long long)m), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap* m, uint32_t bar, int x, int y,
                                       int z, int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4, %5, %6}], [%2];" ::"r"(dst),
        "l"((unsigned long long)m), "r"(bar), "r"(x), "r"(y), "r"(z), "r"(w)
        : "memory");
}
// --- CTA-pair (cta_group::2) forms ---
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
// Shared::cluster address of the same shared variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
// Arrive on an mbarrier of another CTA of the cluster (default .release.cta
// semantics: what the peer consumes is tensor memory written and completed
// with tcgen05.wait::st / read with tcgen05.wait::ld before the arrive, or
// shared memory filled by TMA, so the arrive itself orders the hand-off; a
// cluster-scope release here made every arrive of the converter a fence that
// doubled its time per chunk).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}
// Bounded wait of the CTA-pair kernel; on timeout it raises this CTA's and the
// peer CTA's abort flags (peer_abort: shared::cluster address).
__device__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                             uint32_t peer_abort, int* err, int code,
                             unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63u) == 0) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > limit_ns) {
                *abort_flag = 1;
                st_cluster_u32(peer_abort, 1u);
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}
__device__ __forceinline__ bool warp_wait_cl(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                             uint32_t peer_abort, int* err, int code) {
    const bool r = mbar_wait_cl(bar, parity, abort_flag, peer_abort, err, code);
    return __all_sync(0xffffffffu, r);
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc_pair(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
// D[tmem] (+)= A[tmem] * B[smem desc] over the CTA pair: M = 256 (128 rows per
// CTA's TMEM), B's N rows split in halves across the two CTAs' shared memory.
// Called by all 32 lanes of a converged warp with warp-uniform operands: one
// elected lane issues the instruction.  Issuing from a single divergent lane
// instead halved the MMA rate at N = 96 (measured with gkba_measure_tf32_mma's
// kernel): the operands then are per-thread values.
__device__ __forceinline__ void mma_tf32_pair(uint32_t d, uint32_t a, unsigned long long bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::2.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive (once the earlier MMAs issued by this warp are done) on the mbarrier
// at this shared offset in every CTA of `mask`; warp-collective like
// mma_tf32_pair.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar, uint16_t mask) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
        "[%0], %1;\n\t}" ::"r"(bar),
        "h"(mask)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

#define R8(a, o) "r"(a[o + 0]), "r"(a[o + 1]), "r"(a[o + 2]), "r"(a[o + 3]), "r"(a[o + 4]), "r"(a[o + 5]), "r"(a[o + 6]), "r"(a[o + 7])
#define W8(a, o) "=r"(a[o + 0]), "=r"(a[o + 1]), "=r"(a[o + 2]), "=r"(a[o + 3]), "=r"(a[o + 4]), "=r"(a[o + 5]), "=r"(a[o + 6]), "=r"(a[o + 7])

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
        "%29, %30, %31, %32};" ::"r"(taddr),
        R8(v, 0), R8(v, 8), R8(v, 16), R8(v, 24)
        : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : W8(v, 0), W8(v, 8), W8(v, 16), W8(v, 24)
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : W8(v, 0), W8(v, 8)
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes grouped by 8 (stride-byte-offset 1024), sm_100-family version bit.
__device__ __forceinline__ unsigned long long desc_sw128(uint32_t saddr) {
    unsigned long long d = (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= 1ull << 16;                              // leading byte offset (unused when swizzled)
    d |= (unsigned long long)(1024 >> 4) << 32;   // stride byte offset
    d |= 1ull << 46;                              // descriptor version
    d |= 2ull << 61;                              // SWIZZLE_128B
    return d;
}

// Instruction descriptor of the CTA-pair MMA: kind::tf32, FP32 accumulator,
// A and B TF32, K-major, M = 256 (two 128-row halves), N = n.
__host__ __device__ constexpr uint32_t idesc_tf32_pair(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)((2 * kBM) >> 4) << 24);
}

// TF32 split of the streamed A operand, selected at compile time:
//   0: hi = rna(x), lo = rna(x - hi)           (|error| <= 2^-23 |x| per element,
//      unbiased: lo is exact in TF32, so no truncation toward zero remains)
//   1: hi = x truncated to TF32, lo = rna(x - hi)
//   2: hi = x truncated to TF32, lo = x - hi    (the MMA keeps lo's leading
//      11 bits: |error| <= 2^-21 |x|), two full-rate integer/FP ops per element
#ifndef GKBA_SPLIT_MODE
#define GKBA_SPLIT_MODE 0
#endif

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
#if GKBA_SPLIT_MODE == 0
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
#elif GKBA_SPLIT_MODE == 1
    hi = __float_as_uint(x) & 0xFFFFE000u;
    lo = tf32_rna(x - __uint_as_float(hi));
#else
    hi = __float_as_uint(x) & 0xFFFFE000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
#endif
}

// Load row r (0..127) of a 128 x 32 FP32 tile written by TMA with the 128-byte
// swizzle (16-byte chunk j of row r sits at chunk j ^ (r & 7)) and split it
// into TF32 hi / lo registers.
__device__ __forceinline__ void load_split_row(const uint8_t* tile, int r, uint32_t (&hi)[32],
                                               uint32_t (&lo)[32]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 v = *reinterpret_cast<const float4*>(tile + r * 128 + ((j ^ (r & 7)) << 4));
        split_tf32(v.x, hi[4 * j + 0], lo[4 * j + 0]);
        split_tf32(v.y, hi[4 * j + 1], lo[4 * j + 1]);
        split_tf32(v.z, hi[4 * j + 2], lo[4 * j + 2]);
        split_tf32(v.w, hi[4 * j + 3], lo[4 * j + 3]);
    }
}

// The split of the last contraction's streamed operand, on full-rate integer
// and FP32 instructions only (the conversion instruction issues at a fraction
// of that rate, and this split bounded the S4 converter):
//   hi = x rounded to TF32, to nearest with ties away from zero, on integer
//        instructions (tf32_rna_bits, tf32_round.h); bit-identical to
//        cvt.rna.tf32.f32 for every finite x;
//   lo = x - hi, exact in FP32 (x and hi are within a factor of two), passed
//        unrounded: the MMA reads its leading 11 bits.  lo is a multiple of
//        x's ulp no larger than half a TF32 ulp of x, so it has at most 12
//        significant bits and the MMA drops at most the last one, the bit a
//        rounding of lo would round away: |x - hi - lo_mma| <= 2^-23 |x|, as
//        with a rounded lo.  The sign of lo is that of the rounding of hi,
//        not of x, so this truncation adds no coherent bias to the product.
// A non-finite x gives a NaN lo (inf - inf, NaN - anything), so it reaches the
// sum as a NaN, as with the rounded split.
__device__ __forceinline__ void split_tf32_exact_lo(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_rna_bits(__float_as_uint(x));
    lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ void load_split_row_exact_lo(const uint8_t* tile, int r, uint32_t (&hi)[32],
                                                        uint32_t (&lo)[32]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 v = *reinterpret_cast<const float4*>(tile + r * 128 + ((j ^ (r & 7)) << 4));
        split_tf32_exact_lo(v.x, hi[4 * j + 0], lo[4 * j + 0]);
        split_tf32_exact_lo(v.y, hi[4 * j + 1], lo[4 * j + 1]);
        split_tf32_exact_lo(v.z, hi[4 * j + 2], lo[4 * j + 2]);
        split_tf32_exact_lo(v.w, hi[4 * j + 3], lo[4 * j + 3]);
    }
}

// ---------------------------------------------------------------------------
// Stages S1-S3: resident per-unit B operand, persistent CTAs over (unit, tile).
// ---------------------------------------------------------------------------
// Position and phase bit of a ring of n barriers, advanced one entry at a
// time: keeps divisions by ring sizes that are not powers of two (64-bit
// integer division is a long software routine) out of the issue loops.
struct Ring {
    int i;
    uint32_t ph;
    int n;
    __device__ explicit Ring(int n_) : i(0), ph(0u), n(n_) {}
    __device__ __forceinline__ void next() {
        if (++i == n) {
            i = 0;
            ph ^= 1u;
        }
    }
};

struct StageParams {
    int Np;
    int planes;        // 1 for S1 (real A), 2 for S2/S3 (planar complex A)
    int kch;           // K-chunks per plane: ceil(Np / 32)
    int mtiles;        // Np^3 / 128
    long long M;       // rows = Np^3
    int units;         // units in the batch
    int a_unit;        // A has a unit coordinate (S2/S3) or is shared (S1)
    const int* unit_sys;  // batches of several systems: unit -> system (3-D S1 map), else null
    float* out;
    long long out_unit;
    StageMap map;
    int* err;
    int wsteps;        // 0: one accumulator per tile; 1 or 2: windows of that many K steps
    int nring;         // windowed: accumulators in the ring (<= kStageRing)
    int as2;           // windowed: ring stride in columns (2 Np rounded up to 32)
    int astages;       // A pipeline stages (4 .. kStageAStagesMax, set with the shared memory)
};

static_assert(sizeof(StageParams) % 4 == 0 && sizeof(StageParams) / 4 <= 384, "StageParams copy");
// One launch of the stage kernel: up to kMaxLaunchGroups groups (problems of
// different Np or operands), each with its own parameters and tensor maps; the
// clusters [cl_begin[g], cl_begin[g + 1]) of the grid work on group g.
constexpr int kMaxLaunchGroups = 8;
struct StageLaunch {
    CUtensorMap tmA[kMaxLaunchGroups];
    CUtensorMap tmBhi[kMaxLaunchGroups];
    CUtensorMap tmBlo[kMaxLaunchGroups];
    StageParams p[kMaxLaunchGroups];
    int cl_begin[kMaxLaunchGroups + 1];
    int ngroups;
};

// Output address of row `row` of unit u through the stage's map (rows below
// 2^31: 32-bit unsigned division).
__device__ __forceinline__ float* stage_out_row(const StageParams& p, int u, uint32_t row) {
    const uint32_t Dx = (uint32_t)p.map.Dx, Db = (uint32_t)p.map.Db;
    const uint32_t x = row % Dx, rb = row / Dx;
    const long long xo = p.map.XB ? (long long)(x >> 5) * p.map.XB + (x & 31) : (long long)x * p.map.SX;
    return p.out + (long long)u * p.out_unit + (long long)(rb / Db) * p.map.SA +
           (long long)(rb % Db) * p.map.SB + xo;
}

// A pipeline stages (16 KB each): as many as shared memory holds next to the
// resident B operand, up to kStageAStagesMax.  The loads of a stage kernel
// are latency-bound: at a few microseconds of load latency under load, an
// SM streams about (stages x 16 KB) per latency, so every stage counts.
constexpr int kStageAStagesMax = 8;
// dynamic shared memory of one CTA
constexpr size_t kStageSmemMax = 227 * 1024;
constexpr int kStageRing = 8;
constexpr int kStageThreads = 384;  // warp 0 TMA, warp 1 MMA, 4-7 converter, 8-11 epilogue

// ---------------------------------------------------------------------------
// Stages S1-S3 on CTA pairs (cta_group::2).  A cluster of two CTAs on two SMs
// computes 256-row tiles: each CTA stages, splits and holds its own 128 rows
// of A in its tensor memory and its own half of the B rows in shared memory;
// the even CTA issues every MMA for the pair (M = 256, N = 2 Np), and each
// CTA's TMEM receives the full 2 Np columns of its 128 rows.
//
// With B split by rows the complex stages need no half-width MMAs: B' holds
//   even CTA (Re output columns):  [ Re G | -Im G ]   over K = (plane, q)
//   odd CTA  (Im output columns):  [ Im G |  Re G ]
// so the Re and Im planes of A are two K ranges of one real GEMM of
// N = 2 Np.  S1 (real A) uses the Re / Im halves of [Re Gb^T; Im Gb^T].
//
// Barriers: A pipeline (AFULL/AEMPTY) and B loads (BFULL) are per CTA; the
// converters and epilogues of both CTAs arrive on the even CTA's TFULL / ACCE
// (count 8: four warps per CTA); MMA completion is multicast to both CTAs'
// TEMPTY / ACCF / BEMPTY.  The odd CTA forwards its B completion to the even
// CTA's BPEER.  Every wait is bounded and a timeout raises both CTAs' abort
// flags.
//
// Tensor memory (512 columns, same address in both CTAs): accumulators at
// columns 0 and 256 (2 Np <= 192 each, double-buffered over tiles), A slots
// (TF32 hi in 32 columns, lo in the next 32) at 192 and 448.  SPLIT_ACC:
// hi*hi accumulates at column 0 and the two correction products at 256 (a
// single, not double-buffered, pair), summed in the epilogue; the main
// accumulator then sees a third of the truncating accumulator additions.
// ---------------------------------------------------------------------------
template <bool SPLIT_ACC, bool GROUPED>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kStageThreads, 1)
    k_tc_pair(const __grid_constant__ StageLaunch L) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // the group this cluster works on: the launch's clusters are split between
    // its groups (problems of different Np or operands), each runs the
    // pipeline below with its own parameters and tensor maps
    // GROUPED = false: a one-group launch, whose parameters the loops read
    // from the parameter block at constant offsets; a grouped launch indexes
    // them by the cluster's group (generic loads).  Shared-memory copies of
    // the parameters measured slower than either.
    const int cid_all = (int)cluster_id_x();
    int grp = 0;
    if (GROUPED)
        while (grp + 1 < L.ngroups && cid_all >= L.cl_begin[grp + 1]) ++grp;
    const StageParams& p = GROUPED ? L.p[grp] : L.p[0];
    const CUtensorMap* tmA = GROUPED ? &L.tmA[grp] : &L.tmA[0];
    const CUtensorMap* tmBhi = GROUPED ? &L.tmBhi[grp] : &L.tmBhi[0];
    const CUtensorMap* tmBlo = GROUPED ? &L.tmBlo[grp] : &L.tmBlo[0];
    const int Np = p.Np;
    const int nchunk = p.planes * p.kch;                // K-chunks per tile
    const uint32_t chunkB = (uint32_t)(Np * 128);       // one K-chunk of this CTA's Np B rows
    uint8_t* sBhi = smem;
    uint8_t* sBlo = sBhi + nchunk * chunkB;
    uint8_t* sA = sBlo + nchunk * chunkB;
    const int nas = p.astages;  // A stages of this launch (<= kStageAStagesMax)
    uint64_t* bars = (uint64_t*)(sA + nas * kTileBytes);
    constexpr int BFULL = 0, BPEER = 1, BEMPTY = 2, AFULL = 3, AEMPTY = AFULL + kStageAStagesMax,
                  TFULL = AEMPTY + kStageAStagesMax, TEMPTY = TFULL + 2, ACCF = TEMPTY + 2,
                  ACCE = ACCF + 2, DRAIN = ACCE + 2, WF = DRAIN + 1, WE = WF + kStageRing,
                  NBARS = WE + kStageRing;
    uint32_t* tmem_slot = (uint32_t*)(bars + NBARS);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    // a 32 x 32 FP32 staging block per epilogue warp (after the 512-byte
    // barrier area) through which the epilogue turns its per-row results into
    // 16-byte stores
    float* stage_out = (float*)(sA + nas * kTileBytes + 512);
    auto bar = [&](int i) { return smem_u32(bars + i); };

    const uint32_t rank = cluster_rank();
    const uint32_t peer_abort = mapa_rank(smem_u32((const void*)abort_flag), rank ^ 1u);
    auto bar0 = [&](int i) { return mapa_rank(bar(i), 0); };  // the even CTA's barrier
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(bar(BFULL), 1);
        mbar_init(bar(BPEER), 1);
        mbar_init(bar(BEMPTY), 1);
        for (int s = 0; s < nas; ++s) {
            mbar_init(bar(AFULL + s), 1);
            mbar_init(bar(AEMPTY + s), 4);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(bar(TFULL + s), 8);
            mbar_init(bar(TEMPTY + s), 1);
            mbar_init(bar(ACCF + s), 1);
            mbar_init(bar(ACCE + s), 8);
        }
        for (int b = 0; b < kStageRing; ++b) {
            mbar_init(bar(WF + b), 1);
            mbar_init(bar(WE + b), 8);
        }
        mbar_init(bar(DRAIN), 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        prefetch_tmap(tmA);
        prefetch_tmap(tmBhi);
        prefetch_tmap(tmBlo);
    }
    if (warp == 1) {
        tmem_alloc_pair(smem_u32(tmem_slot), 512);
        tmem_relinquish_pair();
        tc_fence_before();
    }
    __syncthreads();
    cluster_sync_all();  // barriers of both CTAs initialised, TMEM allocated
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // A slot columns: windowed mode 0 / 64 (the ring follows at 128), else 192 / 448
    const bool win = p.wsteps > 0;
    const uint32_t slot_col0 = win ? 0u : 192u, slot_col1 = win ? 64u : 448u;
    const int ktail = (Np & (kKC - 1)) ? (Np & (kKC - 1)) / 8 : 4;  // K steps of a plane's last chunk
    // K steps of chunk c (a plane's last chunk holds Np % 32 = 16 valid K when Np is an odd
    // multiple of 16) and windows per tile in the windowed mode
    int win_per_tile = 0;
    if (win)
        for (int c = 0; c < nchunk; ++c) win_per_tile += ((c % p.kch) == p.kch - 1 ? ktail : 4) / p.wsteps;

    const long long ipu = p.mtiles / 2;  // 256-row tiles per unit
    // tile and row indices stay below 2^31 (checked on the host): 32-bit
    // unsigned division, a short instruction sequence, in the per-tile paths
    const uint32_t ipu32 = (uint32_t)ipu;
    const long long total = (long long)p.units * ipu;
    const long long ncl = L.cl_begin[grp + 1] - L.cl_begin[grp], cid = cid_all - L.cl_begin[grp];
    const long long t0 = total * cid / ncl;
    const long long t1 = total * (cid + 1) / ncl;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both CTAs) ----------------
            int cur_u = -1;
            uint32_t bph = 0;
            long long it = 0;
            Ring ar(nas);  // A stage and its phase
            bool ok = true, loaded_b = false;
            for (long long t = t0; t < t1 && ok; ++t) {
                const int u = (int)((uint32_t)t / ipu32);
                const long long row0 = (long long)((uint32_t)t % ipu32) * (2 * kBM) + (long long)rank * kBM;
                if (u != cur_u) {
                    if (cur_u >= 0) {
                        if (!mbar_wait_cl(bar(BEMPTY), bph, abort_flag, peer_abort, p.err, 1)) { ok = false; break; }
                        bph ^= 1;
                    }
                    mbar_expect_tx(bar(BFULL), 2u * nchunk * chunkB);
                    for (int c = 0; c < nchunk; ++c) {
                        const int pl = c / p.kch, kc = c % p.kch;
                        const int y = (pl * 2 + (int)rank) * Np;
                        tma_3d(smem_u32(sBhi + c * chunkB), tmBhi, bar(BFULL), kc * kKC, y, u);
                        tma_3d(smem_u32(sBlo + c * chunkB), tmBlo, bar(BFULL), kc * kKC, y, u);
                    }
                    loaded_b = true;
                    cur_u = u;
                }
                for (int c = 0; c < nchunk && ok; ++c, ++it) {
                    const int pl = c / p.kch, kc = c % p.kch;
                    const int s = ar.i;
                    const uint32_t ph = ar.ph;
                    ar.next();
                    if (!mbar_wait_cl(bar(AEMPTY + s), ph ^ 1, abort_flag, peer_abort, p.err, 2)) { ok = false; break; }
                    mbar_expect_tx(bar(AFULL + s), kTileBytes);
                    const uint32_t dst = smem_u32(sA + s * kTileBytes);
                    if (p.a_unit) tma_4d(dst, tmA, bar(AFULL + s), kc * kKC, pl, (int)row0, u);
                    else if (p.unit_sys) tma_3d(dst, tmA, bar(AFULL + s), kc * kKC, (int)row0, p.unit_sys[u]);
                    else tma_2d(dst, tmA, bar(AFULL + s), kc * kKC, (int)row0);
                }
            }
            if (*abort_flag) {
                for (int s = 0; s < nas; ++s) {
                    if (it > s) {
                        const long long last = it - 1 - ((it - 1 - s) % nas);
                        const uint32_t ph = (uint32_t)((last / nas) & 1);
                        const unsigned long long g0 = gtimer();
                        while (!mbar_try(bar(AFULL + s), ph) && gtimer() - g0 < kWaitLimitNs) {}
                    }
                }
                if (loaded_b) {
                    const unsigned long long g0 = gtimer();
                    while (!mbar_try(bar(BFULL), bph) && gtimer() - g0 < kWaitLimitNs) {}
                }
            }
        }
    } else if (warp == 1) {
        if (rank == 0) {
            // ---------------- MMA issuer (even CTA, for the pair) ----------------
            const uint32_t id = idesc_tf32_pair(2 * Np);
            const unsigned long long dBhi0 = desc_sw128(smem_u32(sBhi));
            const unsigned long long dBlo0 = desc_sw128(smem_u32(sBlo));
            int cur_u = -1;
            uint32_t bfph = 0;
            long long it = 0, tile_i = 0;
            Ring wr(p.nring > 0 ? p.nring : 1);
            bool ok = true, issued = false;
            for (long long t = t0; t < t1 && ok; ++t, ++tile_i) {
                const int u = (int)((uint32_t)t / ipu32);
                if (u != cur_u) {
                    if (!warp_wait_cl(bar(BFULL), bfph, abort_flag, peer_abort, p.err, 3)) { ok = false; break; }
                    if (!warp_wait_cl(bar(BPEER), bfph, abort_flag, peer_abort, p.err, 3)) { ok = false; break; }
                    bfph ^= 1;
                    cur_u = u;
                    tc_fence_after();
                }
                if (win) {
                    // Windowed accumulation: every wsteps K steps go to the next
                    // accumulator of a ring that the epilogue drains into FP32
                    // register sums; inside a window the correction products come
                    // first, while the accumulator is still small, then hi*hi.
                    int kc = 0;
                    for (int c = 0; c < nchunk && ok; ++c, ++it) {
                        const int slot = (int)(it & 1);
                        const uint32_t sph = (uint32_t)((it >> 1) & 1);
                        if (!warp_wait_cl(bar(TFULL + slot), sph, abort_flag, peer_abort, p.err, 5)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t ahi = tmem + (slot ? slot_col1 : slot_col0);
                        const unsigned long long dh = dBhi0 + ((unsigned long long)(c * chunkB) >> 4);
                        const unsigned long long dl = dBlo0 + ((unsigned long long)(c * chunkB) >> 4);
                        const int ksteps = kc == p.kch - 1 ? ktail : 4;
                        if (++kc == p.kch) kc = 0;
                        for (int kw = 0; kw < ksteps; kw += p.wsteps, wr.next()) {
                            const int b = wr.i;
                            if (!warp_wait_cl(bar(WE + b), wr.ph ^ 1u, abort_flag, peer_abort, p.err, 19)) { ok = false; break; }
                            tc_fence_after();
                            const uint32_t dw = tmem + 128u + (uint32_t)(b * p.as2);
#pragma unroll 1
                            for (int kk = kw; kk < kw + p.wsteps; ++kk) {
                                mma_tf32_pair(dw, ahi + kk * 8, dl + 2ull * kk, id, kk == kw ? 0u : 1u);
                                mma_tf32_pair(dw, ahi + kk * 8 + 32, dh + 2ull * kk, id, 1u);
                            }
#pragma unroll 1
                            for (int kk = kw; kk < kw + p.wsteps; ++kk)
                                mma_tf32_pair(dw, ahi + kk * 8, dh + 2ull * kk, id, 1u);
                            mma_commit_pair(bar(WF + b), (uint16_t)3);
                        }
                        if (!ok) break;
                        issued = true;
                        mma_commit_pair(bar(TEMPTY + slot), (uint16_t)3);
                    }
                    if (!ok) break;
                    if (t + 1 < t1 && (int)((uint32_t)(t + 1) / ipu32) != u) mma_commit_pair(bar(BEMPTY), (uint16_t)3);
                    continue;
                }
                const int ab = SPLIT_ACC ? 0 : (int)(tile_i & 1);
                const uint32_t abph = SPLIT_ACC ? (uint32_t)(tile_i & 1) : (uint32_t)((tile_i >> 1) & 1);
                if (!warp_wait_cl(bar(ACCE + ab), abph ^ 1, abort_flag, peer_abort, p.err, 4)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dacc = tmem + (uint32_t)(ab * 256);
                const uint32_t dcor = SPLIT_ACC ? tmem + 256u : dacc;
                // the last chunk of a plane holds Np % 32 = 16 valid K when Np is an odd
                // multiple of 16 (the rest is the TMA's zero fill): its zero K steps are
                // skipped.  kc counts chunks within the plane (no division in this loop:
                // this thread's issue rate bounds the kernel).
                if (!SPLIT_ACC && nchunk <= 2) {
                    // The tile's whole K fits the two A slots: issue every correction
                    // product first, while the accumulator is still small, then hi*hi,
                    // so the only truncating additions at the scale of the result are
                    // those of the hi*hi MMAs (as with separate accumulators, but
                    // keeping the double-buffered accumulator).
                    int ksteps[2];
                    for (int c = 0; c < nchunk; ++c) {
                        const long long ic = it + c;
                        if (!warp_wait_cl(bar(TFULL + (int)(ic & 1)), (uint32_t)((ic >> 1) & 1), abort_flag, peer_abort, p.err, 5)) { ok = false; break; }
                        ksteps[c] = (c % p.kch) == p.kch - 1 ? ktail : 4;
                    }
                    if (!ok) break;
                    tc_fence_after();
                    bool first = true;
                    for (int c = 0; c < nchunk; ++c) {
                        const uint32_t ahi = tmem + (((it + c) & 1) ? slot_col1 : slot_col0);
                        const unsigned long long dh = dBhi0 + ((unsigned long long)(c * chunkB) >> 4);
                        const unsigned long long dl = dBlo0 + ((unsigned long long)(c * chunkB) >> 4);
#pragma unroll 1
                        for (int kk = 0; kk < ksteps[c]; ++kk) {
                            mma_tf32_pair(dacc, ahi + kk * 8, dl + 2ull * kk, id, first ? 0u : 1u);
                            mma_tf32_pair(dacc, ahi + kk * 8 + 32, dh + 2ull * kk, id, 1u);
                            first = false;
                        }
                    }
                    for (int c = 0; c < nchunk; ++c) {
                        const uint32_t ahi = tmem + (((it + c) & 1) ? slot_col1 : slot_col0);
                        const unsigned long long dh = dBhi0 + ((unsigned long long)(c * chunkB) >> 4);
#pragma unroll 1
                        for (int kk = 0; kk < ksteps[c]; ++kk)
                            mma_tf32_pair(dacc, ahi + kk * 8, dh + 2ull * kk, id, 1u);
                        mma_commit_pair(bar(TEMPTY + (int)((it + c) & 1)), (uint16_t)3);
                    }
                    it += nchunk;
                    issued = true;
                    mma_commit_pair(bar(ACCF + ab), (uint16_t)3);
                    if (t + 1 < t1 && (int)((uint32_t)(t + 1) / ipu32) != u) mma_commit_pair(bar(BEMPTY), (uint16_t)3);
                    continue;
                }
                int kc = 0;
                for (int c = 0; c < nchunk; ++c, ++it) {
                    const int slot = (int)(it & 1);
                    const uint32_t sph = (uint32_t)((it >> 1) & 1);
                    if (!warp_wait_cl(bar(TFULL + slot), sph, abort_flag, peer_abort, p.err, 5)) { ok = false; break; }
                    tc_fence_after();
                    // descriptor start field = address >> 4: a 32-byte K step adds 2
                    const uint32_t ahi = tmem + (slot ? slot_col1 : slot_col0);
                    const unsigned long long dh = dBhi0 + ((unsigned long long)(c * chunkB) >> 4);
                    const unsigned long long dl = dBlo0 + ((unsigned long long)(c * chunkB) >> 4);
                    const int ksteps = kc == p.kch - 1 ? ktail : 4;
                    if (++kc == p.kch) kc = 0;
#pragma unroll 1
                    for (int kk = 0; kk < ksteps; ++kk) {
                        const uint32_t ah = ahi + kk * 8, al = ah + 32;
                        const unsigned long long o = 2ull * kk;
                        mma_tf32_pair(dacc, ah, dh + o, id, (c | kk) ? 1u : 0u);
                        mma_tf32_pair(dcor, ah, dl + o, id, (SPLIT_ACC && !(c | kk)) ? 0u : 1u);
                        mma_tf32_pair(dcor, al, dh + o, id, 1u);
                    }
                    issued = true;
                    mma_commit_pair(bar(TEMPTY + slot), (uint16_t)3);
                }
                if (!ok) break;
                mma_commit_pair(bar(ACCF + ab), (uint16_t)3);
                if (t + 1 < t1 && (int)((uint32_t)(t + 1) / ipu32) != u) mma_commit_pair(bar(BEMPTY), (uint16_t)3);
            }
            (void)issued;
            // Closing commit to both CTAs: it completes once every MMA this
            // thread issued is done, so neither CTA leaves (or frees its TMEM)
            // while an MMA still reads its shared memory or tensor memory,
            // also when a wait gave up.
            mma_commit_pair(bar(DRAIN), (uint16_t)3);
            const unsigned long long g0 = gtimer();
            while (!mbar_try(bar(DRAIN), 0) && gtimer() - g0 < kWaitLimitNs) {}
        } else if (lane == 0) {
            const unsigned long long g0 = gtimer();
            while (!mbar_try(bar(DRAIN), 0) && gtimer() - g0 < kWaitLimitNs) {}
        }
    } else if (warp == 2) {
        if (lane == 0 && rank == 1) {
            // ---------------- B relay (odd CTA): its B half landed -> even CTA ----------------
            int cur_u = -1;
            uint32_t bph = 0;
            for (long long t = t0; t < t1; ++t) {
                const int u = (int)((uint32_t)t / ipu32);
                if (u == cur_u) continue;
                cur_u = u;
                if (!mbar_wait_cl(bar(BFULL), bph, abort_flag, peer_abort, p.err, 9)) break;
                bph ^= 1;
                mbar_arrive_cluster(bar0(BPEER));
            }
        }
    } else if (warp >= 4 && warp < 8) {
        // ---------------- converter: FP32 A tile -> TF32 hi/lo in this CTA's TMEM ----------------
        const int wq = warp & 3;
        const int r = wq * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16);
        long long it = 0;
        Ring ar(nas);  // A stage and its phase
        bool ok = true;
        for (long long t = t0; t < t1 && ok; ++t) {
            for (int c = 0; c < nchunk; ++c, ++it) {
                const int s = ar.i;
                const uint32_t ph = ar.ph;
                ar.next();
                if (!warp_wait_cl(bar(AFULL + s), ph, abort_flag, peer_abort, p.err, 6)) { ok = false; break; }
                uint32_t hi[32], lo[32];
                load_split_row(sA + s * kTileBytes, r, hi, lo);
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(AEMPTY + s));
                const int slot = (int)(it & 1);
                const uint32_t sph = (uint32_t)((it >> 1) & 1);
                if (!warp_wait_cl(bar(TEMPTY + slot), sph ^ 1, abort_flag, peer_abort, p.err, 7)) { ok = false; break; }
                tc_fence_after();
                const uint32_t ta = lane_base + (slot ? slot_col1 : slot_col0);
                tmem_st32(ta, hi);
                tmem_st32(ta + 32, lo);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(bar0(TFULL + slot));
            }
        }
    } else if (warp >= 8) {
        // ---------------- epilogue: this CTA's 128 rows, TMEM -> HBM ----------------
        const int wq = warp & 3;
        const int rloc = wq * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16);
        const int ncc = (2 * Np) / 32;
        long long tile_i = 0;
        Ring wr(p.nring > 0 ? p.nring : 1);
        bool ok = true;
        // 16-byte stores need rows that run contiguously in memory, 16-byte
        // aligned column offsets and a 16-byte aligned output
        const bool vec_out = (p.map.XB != 0 || p.map.SX == 1) && (p.map.XB % 4) == 0 &&
                             (p.map.SA % 4) == 0 && (p.map.SB % 4) == 0 && (p.map.SC % 4) == 0 &&
                             (p.map.SY % 4) == 0 && (p.out_unit % 4) == 0 && (p.map.Dx % 4) == 0 &&
                             (((uintptr_t)p.out) & 15) == 0;
        for (long long t = t0; t < t1 && ok && win; ++t) {
            // windowed mode (2 Np <= 96): add the tile's windows in FP32 registers
            const int u = (int)((uint32_t)t / ipu32);
            float acc[96];
#pragma unroll
            for (int j = 0; j < 96; ++j) acc[j] = 0.0f;
            for (int i = 0; i < win_per_tile; ++i, wr.next()) {
                const int b = wr.i;
                if (!warp_wait_cl(bar(WF + b), wr.ph, abort_flag, peer_abort, p.err, 20)) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    if (cc < ncc) {
                        uint32_t v[32];
                        tmem_ld32(lane_base + 128u + (uint32_t)(b * p.as2 + cc * 32), v);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[cc * 32 + j] += __uint_as_float(v[j]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(bar0(WE + b));
            }
            if (!ok) break;
            if (vec_out) {
                // 16-byte stores: four consecutive rows of one column are contiguous
                // (x runs along the rows with unit stride or inside a 32-wide block);
                // lane l stores rows 4 (l % 8) .. + 3 of columns l / 8 + 4 i.  Tiles
                // never cross the M rows of a unit (M = Np^3 is a multiple of 256).
                const uint32_t row = ((uint32_t)t % ipu32) * (2 * kBM) + rank * kBM + wq * 32 + 4 * (lane & 7);
                float* o = stage_out_row(p, u, row);
                float* stg = stage_out + wq * 1024;
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    if (cc < ncc) {
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < 32; ++j) stg[j * 32 + lane] = acc[cc * 32 + j];
                        __syncwarp();
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int cl = 4 * i + (lane >> 3);
                            const int col = cc * 32 + cl;
                            const int hc = col >= Np ? 1 : 0;
                            const int y = col - hc * Np;
                            const float4 v4 = *reinterpret_cast<const float4*>(stg + cl * 32 + 4 * (lane & 7));
                            if (col < 2 * Np && (long long)row + 3 < p.M)
                                *reinterpret_cast<float4*>(o + hc * p.map.SC + (long long)y * p.map.SY) = v4;
                        }
                    }
                }
            } else {
                const uint32_t row = ((uint32_t)t % ipu32) * (2 * kBM) + rank * kBM + rloc;
                float* o = stage_out_row(p, u, row);
#pragma unroll
                for (int col = 0; col < 96; ++col) {
                    if (col < 2 * Np && (long long)row < p.M) {
                        const int hc = col >= Np ? 1 : 0;
                        const int y = col - hc * Np;
                        o[hc * p.map.SC + (long long)y * p.map.SY] = acc[col];
                    }
                }
            }
        }
        for (long long t = t0; t < t1 && ok && !win; ++t, ++tile_i) {
            const int u = (int)((uint32_t)t / ipu32);
            const int ab = SPLIT_ACC ? 0 : (int)(tile_i & 1);
            const uint32_t abph = SPLIT_ACC ? (uint32_t)(tile_i & 1) : (uint32_t)((tile_i >> 1) & 1);
            if (!warp_wait_cl(bar(ACCF + ab), abph, abort_flag, peer_abort, p.err, 8)) { ok = false; break; }
            tc_fence_after();
            const uint32_t row = ((uint32_t)t % ipu32) * (2 * kBM) + rank * kBM + rloc;
            const bool valid = (long long)row < p.M;
            float* o = stage_out_row(p, u, row);
            // 16-byte stores through the warp's staging block (see the windowed path)
            const uint32_t row4 = ((uint32_t)t % ipu32) * (2 * kBM) + rank * kBM + wq * 32 + 4 * (lane & 7);
            float* o4 = vec_out ? stage_out_row(p, u, row4) : nullptr;
            float* stg = stage_out + wq * 1024;
            for (int cc = 0; cc < ncc; ++cc) {
                uint32_t v[32];
                tmem_ld32(lane_base + (uint32_t)(ab * 256 + cc * 32), v);
                if (SPLIT_ACC) {
                    uint32_t w[32];
                    tmem_ld32(lane_base + (uint32_t)(256 + cc * 32), w);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(w[j]));
                } else {
                    tmem_wait_ld();
                }
                if (vec_out) {
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 32; ++j) stg[j * 32 + lane] = __uint_as_float(v[j]);
                    __syncwarp();
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int cl = 4 * i + (lane >> 3);
                        const int col = cc * 32 + cl;
                        const int hc = col >= Np ? 1 : 0;
                        const int y = col - hc * Np;
                        const float4 v4 = *reinterpret_cast<const float4*>(stg + cl * 32 + 4 * (lane & 7));
                        if ((long long)row4 + 3 < p.M)
                            *reinterpret_cast<float4*>(o4 + hc * p.map.SC + (long long)y * p.map.SY) = v4;
                    }
                } else if (valid) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = cc * 32 + j;
                        const int hc = col >= Np ? 1 : 0;
                        const int y = col - hc * Np;
                        o[hc * p.map.SC + (long long)y * p.map.SY] = __uint_as_float(v[j]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(bar0(ACCE + ab));
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // no MMA, remote arrive or peer read of this CTA's memory remains
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// Stage S4: D[(u,c,j)][i] = sum_K X3[(u,c,j)][K] vK[i][K], K = Np^3, split-K.
// ---------------------------------------------------------------------------
struct FinalParams {
    int Np;
    long long K;
    int KW;        // K length of a work item (one FP32 partial per item and row)
    int nks;
    long long rows;
    int ngroups;
    float* part;   // [ks][i][Rld]
    long long Rld;
    int* err;
    int blocked;   // A is K-blocked: [K/32][Rld rows][32] (3-D map) instead of [rows][K]
    int KS;        // unused (the windows are the 32-wide chunks)
    const int* unit_sys;  // batches of several systems: unit -> system (3-D vK maps), else null
};

constexpr int kFinThreads = 448;  // 14 warps: see the S4 kernel

static_assert(sizeof(FinalParams) % 4 == 0 && sizeof(FinalParams) / 4 <= 448, "FinalParams copy");
// One launch of the S4 kernel over up to kMaxLaunchGroups groups (see StageLaunch).
struct FinalLaunch {
    CUtensorMap tmA[kMaxLaunchGroups];
    CUtensorMap tmBhi[kMaxLaunchGroups];
    CUtensorMap tmBlo[kMaxLaunchGroups];
    FinalParams p[kMaxLaunchGroups];
    int cl_begin[kMaxLaunchGroups + 1];
    int ngroups;
};

// ---------------------------------------------------------------------------
// Stage S4 on CTA pairs: D[(u,c,j)][i] = sum_K X3[(u,c,j)][K] vK[i][K].
//
// Work item = (256-row group g: one 128-row tile per CTA, a K range of KW).
// Per 32-wide K chunk each CTA stages its A box and its Np/2 rows of vK (hi
// and lo) in one of eight pipeline stages; a converter warpgroup splits the A
// box into TF32 hi and lo in the CTA's tensor memory (split_tf32_exact_lo:
// full-rate instructions only, the split with the conversion instruction
// bounded this stage); the MMA warp of the even CTA issues M = 256, N = Np
// MMAs for the pair.
//
// Accuracy: the tensor core truncates its FP32 accumulator additions toward
// zero.  Over the N^3-long sum of this stage that bias is not uniform: it
// depends on how much a unit's partial sums cancel, so it differs between the
// Sigma^< and Sigma^> units and breaks the exact cancellation behind
// particle-number conservation (Re Tr I = 0); measured against the FP64
// path it grows with the accumulation length roughly as its 1.8th power.
// This stage therefore accumulates each 32-wide chunk in its own tensor-
// memory window, drained by the epilogue into FP32 register sums with Kahan
// compensation (so the number of windows adds no rounding error).  Inside a
// window the two correction products hi*lo + lo*hi (about 2^-11 of the
// result) are issued first, while the accumulator is still small, and the
// hi*hi products after them, so the only truncations at the scale of the
// result are those of the four hi*hi MMAs.
//
// Tensor memory (512 columns, same address in both CTAs): two A slots (hi
// in 32 columns, lo in the next 32) at 0 and 64, so the converter works one
// chunk ahead of the MMAs; four window accumulators of AS = Np rounded up to
// 32 columns at 128 + w AS, so the MMAs run up to three windows ahead of the
// epilogue.  Chunk c uses A slot c mod 2 and window c mod 4.  (Three slots
// sharing one index with three windows coupled the converter and the
// epilogue more tightly: per-role clock counters showed the MMA warp waiting
// on both.)
//
// Warps: 0 TMA producer, 1 MMA issuer (even CTA; the whole warp, one elected
// lane issues), 4-7 converter, and eight epilogue warps, two per tensor-
// memory lane quarter (a warp reads only the lanes of quarter warp % 4), each
// draining half of a window's Np columns: 8-11 the first half, 12, 13, 2, 3
// the second.  The epilogue adds a window into its Kahan sums with scalar FP32
// instructions (PACKED = false) or on packed FP32 pairs (PACKED = true, two
// columns per add.f32x2 / sub.f32x2); both give the same bits, the launch
// takes the faster one for its column width.
//
// Barriers (every wait is bounded):
//   FULL[stage]  TMA bytes landed;
//   EMPTY[stage] the stage may be refilled: the 4 converter warps arrive once
//                the chunk's MMAs are done (they read A, the MMAs read B);
//   TFULL[slot]  the slot's hi / lo are in tensor memory (4 converter warps of
//                each CTA arrive on the even CTA's barrier);
//   DONE[win]    one multicast commit per chunk once its MMAs are done: the
//                window is full (epilogue); for chunk c the converter of chunk
//                c + 2 reads it as "A slot and stage B of chunk c are free";
//   WE[win]      the window was drained (8 epilogue warps of each CTA).
// One commit per chunk: each tcgen05.commit costs the tensor pipe about 130
// clocks (measured), a quarter of the chunk's MMA time.
// ---------------------------------------------------------------------------
constexpr int kFinPairStages = 8;
constexpr int kFinKC = kKC;      // K per pipeline chunk and window: one 32-wide TMA box
constexpr int kFinMaxNp = 96;
constexpr int kFinSlots = 2;     // A (hi, lo) slots in tensor memory
constexpr int kFinWins = 4;      // window accumulators in tensor memory
constexpr uint32_t kFinWinCol = 64u * kFinSlots;  // first window accumulator column
constexpr int kFinEpiWarps = 8;

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : W8(v, 0)
                 : "r"(taddr)
                 : "memory");
}

// Packed FP32 pairs (sm_100 family): one add.f32x2 / sub.f32x2 performs two
// independent round-to-nearest FP32 operations, so the Kahan update of two
// columns takes the issue slots of one (bitwise the scalar update on each).
__device__ __forceinline__ unsigned long long f2_pack(uint32_t a, uint32_t b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long x, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// Kahan: sum + cmp carries the exact running sum to about 2 ulp
__device__ __forceinline__ void kahan2(unsigned long long& sum, unsigned long long& cmp, unsigned long long v) {
    const unsigned long long y = f2_sub(v, cmp);
    const unsigned long long t = f2_add(sum, y);
    cmp = f2_sub(f2_sub(t, sum), y);
    sum = t;
}

template <bool GROUPED, bool PACKED>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kFinThreads, 1)
    k_tc_final_pair(const __grid_constant__ FinalLaunch L) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // the group this cluster works on (see StageLaunch)
    const int cid_all = (int)cluster_id_x();
    int grp = 0;
    if (GROUPED)  // as in the stage kernel
        while (grp + 1 < L.ngroups && cid_all >= L.cl_begin[grp + 1]) ++grp;
    const FinalParams& p = GROUPED ? L.p[grp] : L.p[0];
    const CUtensorMap* tmA = GROUPED ? &L.tmA[grp] : &L.tmA[0];
    const CUtensorMap* tmBhi = GROUPED ? &L.tmBhi[grp] : &L.tmBhi[0];
    const CUtensorMap* tmBlo = GROUPED ? &L.tmBlo[grp] : &L.tmBlo[0];
    const int Np = p.Np, Nh = Np / 2;
    const uint32_t AS = (uint32_t)((Np + 31) & ~31);  // window accumulator stride in columns
    const uint32_t bbytes = (uint32_t)(Nh * 128);     // this CTA's B rows, one 32-wide box
    const uint32_t stage_bytes = kTileBytes + 2 * bbytes;  // A, Bhi, Blo
    uint64_t* bars = (uint64_t*)(smem + kFinPairStages * stage_bytes);
    constexpr int FULL = 0, EMPTY = FULL + kFinPairStages, TFULL = EMPTY + kFinPairStages,
                  DONE = TFULL + kFinSlots, WE = DONE + kFinWins, DRAIN = WE + kFinWins,
                  NBARS = DRAIN + 1;
    uint32_t* tmem_slot = (uint32_t*)(bars + NBARS);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    auto bar = [&](int i) { return smem_u32(bars + i); };
    auto stA = [&](int s) { return smem + s * stage_bytes; };
    auto stBhi = [&](int s) { return smem + s * stage_bytes + kTileBytes; };
    auto stBlo = [&](int s) { return smem + s * stage_bytes + kTileBytes + bbytes; };

    const uint32_t rank = cluster_rank();
    const uint32_t peer_abort = mapa_rank(smem_u32((const void*)abort_flag), rank ^ 1u);
    auto bar0 = [&](int i) { return mapa_rank(bar(i), 0); };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kFinPairStages; ++s) {
            mbar_init(bar(FULL + s), 1);
            mbar_init(bar(EMPTY + s), 4);  // the 4 converter warps
        }
        for (int s = 0; s < kFinSlots; ++s) mbar_init(bar(TFULL + s), 8);
        for (int w = 0; w < kFinWins; ++w) {
            mbar_init(bar(DONE + w), 1);
            mbar_init(bar(WE + w), 2 * kFinEpiWarps);
        }
        mbar_init(bar(DRAIN), 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        prefetch_tmap(tmA);
        prefetch_tmap(tmBhi);
        prefetch_tmap(tmBlo);
    }
    if (warp == 1) {
        tmem_alloc_pair(smem_u32(tmem_slot), 512);
        tmem_relinquish_pair();
        tc_fence_before();
    }
    __syncthreads();
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long items = (long long)p.ngroups * p.nks;
    const long long ncl = L.cl_begin[grp + 1] - L.cl_begin[grp], cid = cid_all - L.cl_begin[grp];
    // epilogue role e = 4 h + quarter: warps 8-11 (h = 0), 12, 13, 2, 3 (h = 1)
    const int epi = warp >= 8 ? warp - 8 : (warp == 2 || warp == 3) ? warp + 4 : -1;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both CTAs) ----------------
            long long it = 0;
            Ring st(kFinPairStages);
            bool ok = true;
            for (long long item = cid; item < items && ok; item += ncl) {
                const int g = (int)(item % p.ngroups), ks = (int)(item / p.ngroups);
                const long long k0 = (long long)ks * p.KW;
                const long long k1 = k0 + p.KW < p.K ? k0 + p.KW : p.K;
                const int row0 = g * 2 * kBM + (int)rank * kBM;
                // a 256-row group never straddles two systems (their units are padded)
                const int sys = p.unit_sys ? p.unit_sys[(g * 2 * kBM) / (2 * Np)] : 0;
                for (long long k = k0; k < k1; k += kFinKC, ++it, st.next()) {
                    const int s = st.i;
                    if (!mbar_wait_cl(bar(EMPTY + s), st.ph ^ 1, abort_flag, peer_abort, p.err, 11)) { ok = false; break; }
                    mbar_expect_tx(bar(FULL + s), stage_bytes);
                    const int kh = (int)k;
                    if (p.blocked) tma_3d(smem_u32(stA(s)), tmA, bar(FULL + s), 0, row0, kh >> 5);
                    else tma_2d(smem_u32(stA(s)), tmA, bar(FULL + s), kh, row0);
                    if (p.unit_sys) {
                        tma_3d(smem_u32(stBhi(s)), tmBhi, bar(FULL + s), kh, (int)rank * Nh, sys);
                        tma_3d(smem_u32(stBlo(s)), tmBlo, bar(FULL + s), kh, (int)rank * Nh, sys);
                    } else {
                        tma_2d(smem_u32(stBhi(s)), tmBhi, bar(FULL + s), kh, (int)rank * Nh);
                        tma_2d(smem_u32(stBlo(s)), tmBlo, bar(FULL + s), kh, (int)rank * Nh);
                    }
                }
            }
            if (*abort_flag) {
                for (int s = 0; s < kFinPairStages; ++s) {
                    if (it > s) {
                        const long long last = it - 1 - ((it - 1 - s) % kFinPairStages);
                        const uint32_t ph = (uint32_t)((last / kFinPairStages) & 1);
                        const unsigned long long g0 = gtimer();
                        while (!mbar_try(bar(FULL + s), ph) && gtimer() - g0 < kWaitLimitNs) {}
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (rank == 0) {
            // ---------------- MMA issuer (even CTA, for the pair; warp-collective) ----------------
            const uint32_t id = idesc_tf32_pair(Np);
            Ring st(kFinPairStages), sl(kFinSlots), sw(kFinWins);
            bool ok = true;
            for (long long item = cid; item < items && ok; item += ncl) {
                const int ks = (int)(item / p.ngroups);
                const long long k0 = (long long)ks * p.KW;
                const long long k1 = k0 + p.KW < p.K ? k0 + p.KW : p.K;
                for (long long k = k0; k < k1 && ok; k += kFinKC, st.next(), sl.next(), sw.next()) {
                    const int s = st.i, j = sl.i, w = sw.i;
                    if (!warp_wait_cl(bar(TFULL + j), sl.ph, abort_flag, peer_abort, p.err, 13)) { ok = false; break; }
                    if (!warp_wait_cl(bar(WE + w), sw.ph ^ 1u, abort_flag, peer_abort, p.err, 12)) { ok = false; break; }
                    tc_fence_after();
                    // a 32-byte K step adds 2 to the descriptor's start field
                    const unsigned long long dh = desc_sw128(smem_u32(stBhi(s)));
                    const unsigned long long dl = desc_sw128(smem_u32(stBlo(s)));
                    const uint32_t ahi = tmem + (uint32_t)(j * 64), alo = ahi + 32u;
                    const uint32_t dw = tmem + kFinWinCol + (uint32_t)w * AS;
                    // correction products first (the window starts from zero), then hi*hi
                    mma_tf32_pair(dw, ahi, dl, id, 0u);
                    mma_tf32_pair(dw, alo, dh, id, 1u);
                    mma_tf32_pair(dw, ahi + 8, dl + 2, id, 1u);
                    mma_tf32_pair(dw, alo + 8, dh + 2, id, 1u);
                    mma_tf32_pair(dw, ahi + 16, dl + 4, id, 1u);
                    mma_tf32_pair(dw, alo + 16, dh + 4, id, 1u);
                    mma_tf32_pair(dw, ahi + 24, dl + 6, id, 1u);
                    mma_tf32_pair(dw, alo + 24, dh + 6, id, 1u);
                    mma_tf32_pair(dw, ahi, dh, id, 1u);
                    mma_tf32_pair(dw, ahi + 8, dh + 2, id, 1u);
                    mma_tf32_pair(dw, ahi + 16, dh + 4, id, 1u);
                    mma_tf32_pair(dw, ahi + 24, dh + 6, id, 1u);
                    mma_commit_pair(bar(DONE + w), (uint16_t)3);
                }
            }
            // closing commit: no CTA leaves while an MMA reads its memory
            mma_commit_pair(bar(DRAIN), (uint16_t)3);
            const unsigned long long g0 = gtimer();
            while (!mbar_try(bar(DRAIN), 0) && gtimer() - g0 < kWaitLimitNs) {}
        } else if (lane == 0) {
            const unsigned long long g0 = gtimer();
            while (!mbar_try(bar(DRAIN), 0) && gtimer() - g0 < kWaitLimitNs) {}
        }
    } else if (warp >= 4 && warp < 8) {
        // ---------------- converter: A box -> TF32 hi / lo in this CTA's TMEM ----------------
        // Software-pipelined: the tensor-memory stores of chunk c complete
        // (tcgen05.wait::st, then TFULL) while chunk c + 1 is read and split,
        // unless chunk c + 1 has not landed yet.  A chunk's stage is released
        // (EMPTY) once its MMAs are done, observed when its A slot is reused
        // two chunks later (DONE of its window).
        const int wq = warp & 3;
        const int r = wq * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16);
        Ring st(kFinPairStages), sl(kFinSlots), rel(kFinPairStages), dn(kFinWins);
        long long it = 0;
        bool ok = true;
        int pend = -1;  // slot whose stores were issued but not yet waited for
        auto finish_pending = [&]() {
            if (pend >= 0) {
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(bar0(TFULL + pend));
                pend = -1;
            }
        };
        for (long long item = cid; item < items && ok; item += ncl) {
            const int ks = (int)(item / p.ngroups);
            const long long k0 = (long long)ks * p.KW;
            const long long k1 = k0 + p.KW < p.K ? k0 + p.KW : p.K;
            for (long long k = k0; k < k1; k += kFinKC, ++it, st.next(), sl.next()) {
                const int s = st.i;
                if (pend >= 0 && !__all_sync(0xffffffffu, mbar_try(bar(FULL + s), st.ph))) finish_pending();
                if (!warp_wait_cl(bar(FULL + s), st.ph, abort_flag, peer_abort, p.err, 14)) { ok = false; break; }
                uint32_t hi[32], lo[32];
                load_split_row_exact_lo(stA(s), r, hi, lo);
                finish_pending();
                const int j = sl.i;
                // the slot (and chunk c - 2's stage) is free once chunk c - 2's MMAs
                // are done: the DONE of chunk c - 2's window (dn trails by two chunks)
                if (it >= kFinSlots) {
                    if (!warp_wait_cl(bar(DONE + dn.i), dn.ph, abort_flag, peer_abort, p.err, 15)) { ok = false; break; }
                    dn.next();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar(EMPTY + rel.i));
                    rel.next();
                }
                tc_fence_after();
                const uint32_t ta = lane_base + (uint32_t)(j * 64);
                tmem_st32(ta, hi);
                tmem_st32(ta + 32, lo);
                pend = j;
            }
        }
        if (ok) finish_pending();
        else tmem_wait_st();  // no store may be in flight when the CTA frees its tensor memory
    } else if (epi >= 0) {
        // ---------------- epilogue: Kahan sums of the drained windows, one partial per item ----------------
        const int wq = warp & 3;  // == epi & 3
        const int rloc = wq * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16);
        const int cw = Np / 2;                 // columns of this warp: [c0, c0 + cw)
        const int c0 = (epi >> 2) * cw;
        constexpr int kMaxC = kFinMaxNp / 2;   // 48
        Ring sl(kFinWins);
        bool ok = true;
        for (long long item = cid; item < items && ok; item += ncl) {
            const int g = (int)(item % p.ngroups), ks = (int)(item / p.ngroups);
            const long long k0 = (long long)ks * p.KW;
            const long long k1 = k0 + p.KW < p.K ? k0 + p.KW : p.K;
            if (!PACKED) {
                // scalar Kahan updates (same bits as the packed pairs below; the
                // faster form at 48 columns per warp, Np = 96)
                float sum[kMaxC], cmp[kMaxC];
#pragma unroll
                for (int j = 0; j < kMaxC; ++j) sum[j] = cmp[j] = 0.0f;
                for (long long kw = k0; kw < k1; kw += kFinKC, sl.next()) {
                    const int b = sl.i;
                    if (!warp_wait_cl(bar(DONE + b), sl.ph, abort_flag, peer_abort, p.err, 16)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t col = lane_base + kFinWinCol + (uint32_t)b * AS + (uint32_t)c0;
                    // 16 columns per load while they last, then an 8-column tail
#pragma unroll
                    for (int q = 0; q < kMaxC / 16; ++q) {
                        if (q * 16 + 16 <= cw) {
                            uint32_t v[16];
                            tmem_ld16(col + (uint32_t)(q * 16), v);
                            tmem_wait_ld();
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                // Kahan: sum + cmp carries the exact running sum to ~2 ulp
                                const float y = __uint_as_float(v[j]) - cmp[q * 16 + j];
                                const float t = sum[q * 16 + j] + y;
                                cmp[q * 16 + j] = (t - sum[q * 16 + j]) - y;
                                sum[q * 16 + j] = t;
                            }
                        }
                    }
                    if (cw & 8) {
                        uint32_t v[8];
                        tmem_ld8(col + (uint32_t)(cw - 8), v);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
#pragma unroll
                            for (int q = 0; q < kMaxC / 8; ++q) {
                                if (q * 8 == cw - 8) {
                                    const float y = __uint_as_float(v[j]) - cmp[q * 8 + j];
                                    const float t = sum[q * 8 + j] + y;
                                    cmp[q * 8 + j] = (t - sum[q * 8 + j]) - y;
                                    sum[q * 8 + j] = t;
                                }
                            }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_cluster(bar0(WE + b));
                }
                if (!ok) break;
                float* base = p.part + (long long)ks * Np * p.Rld;
                const long long row = (long long)g * 2 * kBM + (long long)rank * kBM + rloc;
#pragma unroll
                for (int j = 0; j < kMaxC; ++j)
                    if (j < cw) base[(long long)(c0 + j) * p.Rld + row] = sum[j];
                continue;
            }
            // column pairs (2 i, 2 i + 1) packed in one 64-bit register each
            unsigned long long sum[kMaxC / 2], cmp[kMaxC / 2];
#pragma unroll
            for (int j = 0; j < kMaxC / 2; ++j) sum[j] = cmp[j] = 0ull;
            for (long long kw = k0; kw < k1; kw += kFinKC, sl.next()) {
                const int b = sl.i;
                if (!warp_wait_cl(bar(DONE + b), sl.ph, abort_flag, peer_abort, p.err, 16)) { ok = false; break; }
                tc_fence_after();
                const uint32_t col = lane_base + kFinWinCol + (uint32_t)b * AS + (uint32_t)c0;
                // 16 columns per load while they last, then an 8-column tail
#pragma unroll
                for (int q = 0; q < kMaxC / 16; ++q) {
                    if (q * 16 + 16 <= cw) {
                        uint32_t v[16];
                        tmem_ld16(col + (uint32_t)(q * 16), v);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            kahan2(sum[q * 8 + j], cmp[q * 8 + j], f2_pack(v[2 * j], v[2 * j + 1]));
                    }
                }
                if (cw & 8) {
                    uint32_t v[8];
                    tmem_ld8(col + (uint32_t)(cw - 8), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
#pragma unroll
                        for (int q = 0; q < kMaxC / 8; ++q) {
                            if (q * 8 == cw - 8)
                                kahan2(sum[q * 4 + j], cmp[q * 4 + j], f2_pack(v[2 * j], v[2 * j + 1]));
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(bar0(WE + b));
            }
            if (!ok) break;
            float* base = p.part + (long long)ks * Np * p.Rld;
            const long long row = (long long)g * 2 * kBM + (long long)rank * kBM + rloc;
#pragma unroll
            for (int j = 0; j < kMaxC / 2; ++j) {
                if (2 * j < cw) {
                    float a, b;
                    f2_unpack(sum[j], a, b);
                    base[(long long)(c0 + 2 * j) * p.Rld + row] = a;
                    base[(long long)(c0 + 2 * j + 1) * p.Rld + row] = b;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// Self-test of the bounded waits (failure detection without a GPU fault): a
// 2-CTA cluster whose even CTA waits, with the waits of the contraction
// kernels (mbar_wait_cl) and a short limit, on an mbarrier that nothing
// arrives at.  Its wait runs out, records `code` in the error word and
// raises both CTAs' abort flags; the odd CTA, waiting on its own barrier with
// a 100x longer limit, must leave on its peer's flag.  No TMA, no tensor
// memory; every loop is bounded.
// ---------------------------------------------------------------------------
__global__ void __cluster_dims__(2, 1, 1) k_wait_selftest(int* err, unsigned long long limit_ns,
                                                          unsigned long long* elapsed_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_s;
    volatile int* abort_flag = &abort_s;
    const uint32_t rank = cluster_rank();
    const uint32_t peer_abort = mapa_rank(smem_u32((const void*)abort_flag), rank ^ 1u);
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    cluster_sync_all();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = gtimer();
        const unsigned long long lim = rank == 0 ? limit_ns : 100ull * limit_ns;
        (void)mbar_wait_cl(smem_u32(&bar), 0, abort_flag, peer_abort, err, 90 + (int)rank, lim);
        elapsed_ns[rank] = gtimer() - t0;
    }
    __syncthreads();
    cluster_sync_all();  // no remote store is in flight when either CTA leaves
}

// ---------------------------------------------------------------------------
// Tensor-pipe rate probe (measurement of the roofline denominator): every
// CTA pair runs a stream of back-to-back M = 256, N = 192, K = 8 kind::tf32
// MMAs (A in tensor memory, B in shared memory, both zero), the shape and
// operand placement of the stage kernels, with nothing else on the SM.  The
// host times the launch with CUDA events; flops = pairs x iters x 4 x
// 2 x 256 x 192 x 8.  One commit per 64 MMAs bounds the issue queue; the
// closing commit keeps both CTAs resident until the last MMA is done.
// ---------------------------------------------------------------------------
constexpr int kRateN = 192;
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(128, 1)
    k_mma_rate(int iters, int* err) {
    __shared__ __align__(1024) uint8_t sB[(kRateN / 2) * 128];
    __shared__ __align__(8) uint64_t bars[3];  // two alternating periodic commits, the closing one
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_s;
    volatile int* abort_flag = &abort_s;
    const uint32_t rank = cluster_rank();
    const uint32_t peer_abort = mapa_rank(smem_u32((const void*)abort_flag), rank ^ 1u);
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kRateN / 2) * 32; i += blockDim.x)
        reinterpret_cast<float*>(sB)[i] = 0.0f;
    if (threadIdx.x == 0) {
        for (int b = 0; b < 3; ++b) mbar_init(smem_u32(&bars[b]), 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    // zero B (generic writes) must be visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) {
        tmem_alloc_pair(smem_u32(&tmem_slot), 512);
        tmem_relinquish_pair();
        tc_fence_before();
    }
    __syncthreads();
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    {   // A (32 columns at 256) = 0 in this CTA's 128 lanes
        uint32_t z[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) z[j] = 0u;
        tmem_st32(tmem + ((uint32_t)(warp * 32) << 16) + 256u, z);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
    tc_fence_after();
    if (rank == 0 && warp == 0) {
        // one period = 16 iterations (64 MMAs), committed to bars[period & 1];
        // before issuing period q + 1 wait for period q - 1, so one period is
        // always queued behind the running one
        const uint32_t id = idesc_tf32_pair(kRateN);
        const unsigned long long db = desc_sw128(smem_u32(sB));
        bool ok = true;
        for (int i = 0; i < iters && ok; ++i) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_tf32_pair(tmem, tmem + 256u + kk * 8, db + 2ull * kk, id, (i | kk) ? 1u : 0u);
            if ((i & 15) == 15) {
                const int q = i >> 4;
                mma_commit_pair(smem_u32(&bars[q & 1]), (uint16_t)3);
                if (q >= 1)
                    ok = warp_wait_cl(smem_u32(&bars[(q - 1) & 1]), (uint32_t)(((q - 1) >> 1) & 1),
                                      abort_flag, peer_abort, err, 95);
            }
        }
        mma_commit_pair(smem_u32(&bars[2]), (uint16_t)3);
        const unsigned long long g0 = gtimer();
        while (!mbar_try(smem_u32(&bars[2]), 0) && gtimer() - g0 < kWaitLimitNs) {}
    } else if (rank == 1 && threadIdx.x == 0) {
        // the odd CTA receives the multicast commits too; it only waits for the closing one
        const unsigned long long g0 = gtimer();
        while (!mbar_try(smem_u32(&bars[2]), 0) && gtimer() - g0 < kWaitLimitNs) {}
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// Operand preparation kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
    const uint32_t h = tf32_rna((float)x);
    hi = __uint_as_float(h);
    lo = __uint_as_float(tf32_rna((float)(x - (double)hi)));
}

// wS32[j][m][q][s] = w_mqsj = 2 v_mqsj - v_qmsj (zero in the padding).
__global__ void k_build_wS32(int N, int Np, const double* __restrict__ v, float* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long Np4 = (long long)Np * Np * Np * Np;
    if (e >= Np4) return;
    const int s = (int)(e % Np), q = (int)((e / Np) % Np), m = (int)((e / Np / Np) % Np),
              j = (int)(e / Np / Np / Np);
    float w = 0.0f;
    if (s < N && q < N && m < N && j < N) {
        const long long NN = N;
        const double a = v[((m * NN + q) * NN + s) * NN + j];
        const double b = v[((q * NN + m) * NN + s) * NN + j];
        w = (float)(2.0 * a - b);
    }
    out[e] = w;
}

// vK[i][n][r][p] = v_irpn split into TF32 hi / lo (zero in the padding).
__global__ void k_build_vK32(int N, int Np, const double* __restrict__ v, float* __restrict__ hi,
                             float* __restrict__ lo) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long Np4 = (long long)Np * Np * Np * Np;
    if (e >= Np4) return;
    const int pp = (int)(e % Np), r = (int)((e / Np) % Np), n = (int)((e / Np / Np) % Np),
              i = (int)(e / Np / Np / Np);
    float h = 0.0f, l = 0.0f;
    if (pp < N && r < N && n < N && i < N) {
        const long long NN = N;
        split_f64(v[((i * NN + r) * NN + pp) * NN + n], h, l);
    }
    hi[e] = h;
    lo[e] = l;
}

// Omega layout of v for the w-slot chain of dL/dv: vO[i][n][p][r] = v_irpn
// (zero in the padding); it takes wS32's place as stage S1's A operand.
__global__ void k_build_vO32(int N, int Np, const double* __restrict__ v, float* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long Np4 = (long long)Np * Np * Np * Np;
    if (e >= Np4) return;
    const int r = (int)(e % Np), pp = (int)((e / Np) % Np), n = (int)((e / Np / Np) % Np),
              i = (int)(e / Np / Np / Np);
    float x = 0.0f;
    if (r < N && pp < N && n < N && i < N) {
        const long long NN = N;
        x = (float)v[((i * NN + r) * NN + pp) * NN + n];
    }
    out[e] = x;
}

// Contraction of the X3 that stages S1-S3 left in X13 (rows (u, c, b) =
// (2u + c) Np + b, K = (n, r, p)) over its rows, against per-row weights:
//   out[(a % N) SJ + (a / N) SC + n SN + r SR + p] += sum_{u, c, b < N} w(u, c, b, a) X3[(u,c,b)][(n,r,p)]
// for a < A.  Two uses:
//   mode 0 (one slot of dL/dv, A = N): w = Re / Im (c = 0 / 1) of Sbar_u[a][b]
//     (Sbar_u[b][a] when transposeS), i.e. out = Re sum conj(Sbar) X3 over b;
//   mode 1 (the time-linear accumulator, A = 2N, a = (c2, j2)): w = the real
//     form of coef_u Gb_u^T, coef_u = -wt (u even) / +wt (u odd), wt the
//     trapezoid weight of history point k0 + u / 2:
//       (c2, c) = (0, 0): Re, (0, 1): -Im, (1, 0): Im, (1, 1): Re of coef_u Gb_u[b][j2].
// A thread owns one K (in the N basis) and kXsA consecutive a; the rows are
// split over blockIdx.z.  Products and the runs of one staged round (64 rows)
// are FP32 (X3 is FP32), each round is added into an FP64 sum, and the
// block's sums go to out (FP64 atomics when several blocks along z share an
// output).
struct XSlotParams {
    int N, Np, nb;
    long long Rld;         // rows of the K-blocked X3 layout
    int blocked;           // X3 K-blocked (Np % 32 == 0) or row-major [row][Np^3]
    long long rows_per_z;  // compact rows (u, c, b < N) per blockIdx.z
    int A;                 // output columns a
    int mode;              // 0: dL/dv slot, 1: time-linear accumulator
    const double2* S;      // Sbar_u (mode 0) or Gb_u (mode 1), N x N per unit
    int transposeS;
    int k0;
    double w_first, w_rest;
    const float* X;
    double* out;
    long long SJ, SC, SN, SR;
};
constexpr int kXsA = 32;       // a per thread (blockIdx.y picks the range)
constexpr int kXsRows = 64;    // rows of weights staged in shared memory at a time
constexpr int kXsThreads = 128;
// The per-row weights of k_xslot_tc, once per launch: W[R][a] (R the compact
// row (u, c, b), a < A), FP32.
__global__ void k_xslot_weights(const XSlotParams p, float* __restrict__ W) {
    const int N = p.N;
    const long long NN = (long long)N * N;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long Rtot = 2LL * N * p.nb;
    if (e >= Rtot * p.A) return;
    const uint32_t Rc = (uint32_t)(e / p.A);
    const int a = (int)(e - (long long)Rc * p.A);
    const uint32_t uc = Rc / (uint32_t)N;
    const int b = (int)(Rc - uc * (uint32_t)N), u = (int)(uc >> 1), cc = (int)(uc & 1);
    float val;
    if (p.mode == 0) {
        const double2 sv = p.transposeS ? p.S[u * NN + (long long)b * N + a] : p.S[u * NN + (long long)a * N + b];
        val = (float)(cc ? sv.y : sv.x);
    } else {
        const int c2 = a / N, j2 = a % N;
        const double2 g = p.S[u * NN + (long long)b * N + j2];
        const double wt = (p.k0 + u / 2 == 0) ? p.w_first : p.w_rest;
        const double coef = (u & 1) ? wt : -wt;
        const double re = coef * g.x, im = coef * g.y;
        val = (float)(c2 == 0 ? (cc == 0 ? re : -im) : (cc == 0 ? im : re));
    }
    W[e] = val;
}

__global__ void __launch_bounds__(kXsThreads, 2) k_xslot_tc(const XSlotParams p, const float* __restrict__ W) {
    __shared__ float sW[kXsRows][kXsA];
    __shared__ long long sOff[kXsRows];  // X3 offset of each staged row
    const int N = p.N, Np = p.Np;
    const long long NN = (long long)N * N, N3 = NN * N;
    const long long Np3 = (long long)Np * Np * Np;
    const long long KN = (long long)blockIdx.x * kXsThreads + threadIdx.x;
    const bool kok = KN < N3;
    const long long n = KN / NN, r = (KN / N) % N, pp = KN % N;
    const long long K = (n * Np + r) * Np + pp;
    const float* xk = p.blocked ? p.X + (K >> 5) * p.Rld * 32 + (K & 31) : p.X + K;
    const long long xstride = p.blocked ? 32 : Np3;  // per X3 row
    const int a0 = blockIdx.y * kXsA;
    const long long Rtot = 2LL * N * p.nb;  // compact rows (u, c, b < N)
    const long long R0 = (long long)blockIdx.z * p.rows_per_z;
    const long long R1 = R0 + p.rows_per_z < Rtot ? R0 + p.rows_per_z : Rtot;
    float acc[kXsA];
    double sum[kXsA];
#pragma unroll
    for (int t = 0; t < kXsA; ++t) sum[t] = 0.0;
    for (long long rs = R0; rs < R1; rs += kXsRows) {
        const int nrow = (int)(R1 - rs < kXsRows ? R1 - rs : kXsRows);
        __syncthreads();
        for (int e = threadIdx.x; e < kXsRows * kXsA; e += kXsThreads) {
            const int rr = e / kXsA, aa = e % kXsA, a = a0 + aa;
            float val = 0.0f;
            if (rr < nrow) {
                const long long R = rs + rr;
                if (aa == 0) {
                    // compact row (u, c, b) of X3; rows stay below 2^31 (host-checked)
                    const uint32_t Rc = (uint32_t)R, uc = Rc / (uint32_t)N;
                    sOff[rr] = ((long long)uc * Np + (int)(Rc - uc * (uint32_t)N)) * xstride;
                }
                if (a < p.A) val = W[R * p.A + a];
            } else if (aa == 0) {
                sOff[rr] = 0;
            }
            sW[rr][aa] = val;
        }
        __syncthreads();
        if (kok) {
            // one staged round (<= 64 rows) in FP32, then into the FP64 sums;
            // the loads of four rows are issued together
#pragma unroll
            for (int t = 0; t < kXsA; ++t) acc[t] = 0.0f;
            int rr = 0;
            for (; rr + 4 <= nrow; rr += 4) {
                const float x0 = xk[sOff[rr]], x1 = xk[sOff[rr + 1]], x2 = xk[sOff[rr + 2]],
                            x3 = xk[sOff[rr + 3]];
#pragma unroll
                for (int t = 0; t < kXsA; ++t) {
                    float v = fmaf(sW[rr][t], x0, acc[t]);
                    v = fmaf(sW[rr + 1][t], x1, v);
                    v = fmaf(sW[rr + 2][t], x2, v);
                    acc[t] = fmaf(sW[rr + 3][t], x3, v);
                }
            }
            for (; rr < nrow; ++rr) {
                const float x = xk[sOff[rr]];
#pragma unroll
                for (int t = 0; t < kXsA; ++t) acc[t] = fmaf(sW[rr][t], x, acc[t]);
            }
#pragma unroll
            for (int t = 0; t < kXsA; ++t) sum[t] += (double)acc[t];
        }
    }
    if (!kok) return;
    const long long ko = n * p.SN + r * p.SR + pp;
    // one block along z: this thread owns its outputs (plain adds); else the
    // blocks of a column share them (FP64 atomics)
    const bool own = gridDim.z == 1;
#pragma unroll
    for (int t = 0; t < kXsA; ++t) {
        const int a = a0 + t;
        if (a >= p.A) continue;
        double* o = p.out + (a % N) * p.SJ + (a / N) * p.SC + ko;
        if (own) *o += sum[t];
        else atomicAdd(o, sum[t]);
    }
}

// Time-linear back-transforms: Ucal = W^+ and conj(Ucal) = W^T as two units.
__global__ void k_tl_ucal2(int N, const double2* __restrict__ W, double2* __restrict__ out) {
    const long long NN = (long long)N * N;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NN) return;
    const int pr = (int)(e / N), q = (int)(e % N);
    const double2 w = W[(long long)q * N + pr];
    out[e] = make_double2(w.x, -w.y);
    out[NN + e] = w;
}

// Lambda (FP64, N basis, [j][n][r][c][p]) to FP32 in the Np basis, zero
// padded: one warp per row (j, n, r, c), its lanes over p (one index
// decomposition per row instead of per element).
__global__ void k_tl_lam32(int N, int Np, const double* __restrict__ lam, float* __restrict__ out) {
    const long long rows = 2LL * Np * Np * Np;
    const long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const int lane = threadIdx.x & 31;
    const int cc = (int)(row & 1);
    long long q = row >> 1;
    const int r = (int)(q % Np);
    q /= Np;
    const int n = (int)(q % Np);
    const int j = (int)(q / Np);
    float* o = out + row * Np;
    const bool in = j < N && n < N && r < N;
    const double* l = lam + ((((long long)j * N + n) * N + r) * 2 + cc) * N;
    for (int pp = lane; pp < Np; pp += 32) o[pp] = (in && pp < N) ? (float)l[pp] : 0.0f;
}

// Per-unit B operands of the tensor-core path (padded to Np, zero padding),
// stored as TF32 hi then lo blocks of ub units:
//   B1[u][(c,r)][s] = Gb_c[s][r]                                   (S1)
//   Gs[u][b][p][q]  = (Re G, Im G, -Im G, Re G)[b] [p][q]           (S2, S3)
// Block 2 pl + h is the K-plane pl of output half h (the rows held by CTA h
// of a pair) of B' = [[Re G | -Im G]; [Im G | Re G]].
__global__ void k_forms_tf32(int N, int Np, int nb, int ub, const double2* __restrict__ G,
                             const double2* __restrict__ Gb, float* __restrict__ B1,
                             float* __restrict__ Gs) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per = 2LL * Np * Np;
    if (e >= per * nb) return;
    const int u = (int)(e / per);
    const int rr = (int)(e % per);
    const int row = rr / Np, k = rr % Np;  // row = (c, idx), k = K index
    const int comp = row / Np, idx = row % Np;
    const long long NN = (long long)N * N;
    float bh = 0.f, bl = 0.f, gh = 0.f, gl = 0.f;
    if (idx < N && k < N) {
        if (B1 != nullptr) {
            const double2 gb = Gb[u * NN + (long long)k * N + idx];  // Gb[s = k][r = idx]
            split_f64(comp ? gb.y : gb.x, bh, bl);
        }
        const double2 g = G[u * NN + (long long)idx * N + k];    // G[p = idx][q = k]
        split_f64(comp ? g.y : g.x, gh, gl);
    }
    if (B1 != nullptr) {  // null: only the G forms (stage S3's slot of S3(A, B, C))
        B1[e] = bh;
        B1[per * ub + e] = bl;
    }
    // Gs: Re G -> blocks 0 and 3, Im G -> block 1 and (negated) block 2
    const long long pg = 2 * per;
    const long long g0 = (long long)u * pg + rr;
    const long long g1 = (long long)u * pg + per + (comp ? 0 : Np * (long long)Np) + (long long)idx * Np + k;
    Gs[g0] = gh;
    Gs[pg * ub + g0] = gl;
    Gs[g1] = comp ? -gh : gh;
    Gs[pg * ub + g1] = comp ? -gl : gl;
}

inline unsigned grid1(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---------------------------------------------------------------------------
// Host side: tensor maps
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode(gkba_ctx* c, gkba_status* st) {
    static EncodeTiledFn fn = nullptr;
    if (fn) return fn;
    cudaDriverEntryPointQueryResult q;
    void* ptr = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || ptr == nullptr) {
        *st = fail(c, GKBA_ECUDA, "cuTensorMapEncodeTiled not available (%s)", cudaGetErrorString(e));
        return nullptr;
    }
    fn = (EncodeTiledFn)ptr;
    return fn;
}

gkba_status make_map(gkba_ctx* c, CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims,
                     const cuuint64_t* strides_bytes, const cuuint32_t* box) {
    gkba_status st = GKBA_OK;
    EncodeTiledFn enc = get_encode(c, &st);
    if (!enc) return st;
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base),
                     dims, strides_bytes, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(c, GKBA_ECUDA, "cuTensorMapEncodeTiled failed (%d), rank %d", (int)r, rank);
    return GKBA_OK;
}

constexpr int kMaxTcNp = 96;  // largest padded basis of the tensor-core path
// Shared memory of a stage launch with `astages` A stages.
size_t stage_smem_bytes(int Np, int astages) {
    const int kch = (Np + kKC - 1) / kKC;
    // plus the epilogue's 4 x 4 KB staging blocks
    return 1024 + 2ull * kch * (2 * Np * 128) + (size_t)astages * kTileBytes + 512 + 4 * 32 * 32 * 4;
}
// The most A stages that fit next to the B operand (at least 4).
int stage_astages(int Np) {
    int a = kStageAStagesMax;
    while (a > 4 && stage_smem_bytes(Np, a) > kStageSmemMax) --a;
    return a;
}
size_t stage_smem_bytes(int Np) { return stage_smem_bytes(Np, stage_astages(Np)); }
size_t final_pair_smem_bytes(int Np) {
    return 1024 + (size_t)kFinPairStages * (kTileBytes + 2 * (Np / 2) * 128) + 512;
}
// K length of one S4 work item (one FP32 partial per item and row); a
// multiple of every hi*hi window length and of Np^3 for Np a multiple of 16.

}  // namespace

// Model operands of the tensor-core path (once per context).
gkba_status tf32_prepare_model(gkba_ctx* c) {
    const long long Np4 = (long long)c->Np * c->Np * c->Np * c->Np;
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_build_wS32<<<grid1(Np4, 256), 256, 0, c->stream>>>(c->N, c->Np, c->v, c->wS32);
    GKBA_TRY(launch_end(c, t));
    t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_build_vK32<<<grid1(Np4, 256), 256, 0, c->stream>>>(c->N, c->Np, c->v, c->vKhi, c->vKlo);
    GKBA_TRY(launch_end(c, t));
    // The shared-memory limit is a property of the kernel, not of a context:
    // set it for the largest basis so that contexts of different N coexist.
    for (auto kfn : {k_tc_pair<false, false>, k_tc_pair<true, false>, k_tc_pair<false, true>,
                     k_tc_pair<true, true>})
        GKBA_CUDA(c, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kStageSmemMax));
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(c->num_sms & ~1));
        cfg.blockDim = dim3(kStageThreads);
        cfg.dynamicSmemBytes = stage_smem_bytes(c->Np);
        cfg.stream = c->stream;
        int ncl = 0;
        GKBA_CUDA(c, cudaOccupancyMaxActiveClusters(&ncl, k_tc_pair<false, false>, &cfg));
        if (ncl < 1) return fail(c, GKBA_ECUDA, "no 2-CTA cluster of the stage kernel fits on an SM pair");
        c->pair_clusters = ncl;
    }
    for (auto kfn : {k_tc_final_pair<false, false>, k_tc_final_pair<true, false>, k_tc_final_pair<false, true>,
                     k_tc_final_pair<true, true>})
        GKBA_CUDA(c, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)final_pair_smem_bytes(kMaxTcNp)));
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(c->num_sms & ~1));
        cfg.blockDim = dim3(kFinThreads);
        cfg.dynamicSmemBytes = final_pair_smem_bytes(c->Np);
        cfg.stream = c->stream;
        int ncl = 0;
        GKBA_CUDA(c, cudaOccupancyMaxActiveClusters(&ncl, k_tc_final_pair<false, true>, &cfg));
        if (ncl < 1) return fail(c, GKBA_ECUDA, "no 2-CTA cluster of the S4 kernel fits on an SM pair");
        c->fin_pair_clusters = ncl;
    }
    return GKBA_OK;
}

gkba_status build_forms_tf32(gkba_ctx* c, int nb, const double2* G, const double2* Gb) {
    const long long per = 2LL * c->Np * c->Np;
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_forms_tf32<<<grid1(per * nb, 256), 256, 0, c->stream>>>(c->N, c->Np, nb, c->ub_cap, G, Gb,
                                                              (float*)c->formsB1, (float*)c->formsG);
    return launch_end(c, t);
}

gkba_status build_forms3_tf32(gkba_ctx* c, int nb, const double2* A) {
    const long long per = 2LL * c->Np * c->Np;
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_forms_tf32<<<grid1(per * nb, 256), 256, 0, c->stream>>>(c->N, c->Np, nb, c->ub_cap, A, nullptr,
                                                              nullptr, (float*)c->formsG3);
    return launch_end(c, t);
}

gkba_status build_forms(gkba_ctx* c, int nb, const double2* G, long long sG, const double2* Gb,
                        long long sGb, int) {
    (void)sG;
    (void)sGb;
    if (c->kind != GKBA_V_GENERAL) return GKBA_OK;  // structured: no contraction forms
    if (tensor_core_path(c)) return build_forms_tf32(c, nb, G, Gb);
    return build_forms_fp64(c, nb, G, Gb);
}

// Parameters shared by every stage launch of nb units (S1-S3 and the
// time-linear back-transforms); the caller sets planes, a_unit, out and map.
static StageParams stage_base(gkba_ctx* c, int nb) {
    const int Np = c->Np;
    const long long N3 = (long long)Np * Np * Np;
    StageParams sp{};
    sp.Np = Np;
    sp.kch = (Np + kKC - 1) / kKC;
    sp.mtiles = (int)(N3 / kBM);
    sp.M = N3;
    sp.units = nb;
    sp.out_unit = 2 * N3 * Np;
    sp.unit_sys = nullptr;
    sp.err = c->dint + 1;
    // windowed accumulation where the ring fits next to the A slots (2 Np <= 96)
    sp.as2 = ((2 * Np + 31) / 32) * 32;
    sp.wsteps = 2 * Np <= 96 ? std::max(1, std::min(2, c->acc_window / 8)) : 0;
    sp.nring = std::min(kStageRing, (512 - 128) / sp.as2);
    sp.astages = stage_astages(Np);
    return sp;
}

// ---------------------------------------------------------------------------
// Launch plans: the tensor maps and parameters of one stage of one problem.
// A launch takes up to kMaxLaunchGroups plans (problems of different Np or
// operands, e.g. the basis-size groups of a stacked batch) and splits its
// clusters between them by their estimated cost.
// ---------------------------------------------------------------------------
struct StagePlan {
    CUtensorMap mA, mBh, mBl;
    StageParams sp;
    long long pair_tiles;  // 256-row tiles (an upper bound for the group's clusters)
    double weight;         // relative cost for the cluster split
    double flops, bytes;   // algorithmic counts for the statistics
    int cls;
};
struct FinalPlan {
    CUtensorMap mA, mBh, mBl;
    FinalParams fp;
    long long items;
    double weight, flops, bytes;
};

// Relative cost of a stage: the pair's MMA issue sets the pace, three MMAs per
// K step at about 85 clocks each up to N = 128 columns and proportionally
// more beyond (measured with the rate probe), plus a per-tile epilogue share.
static double stage_weight(const StageParams& sp, long long pair_tiles) {
    const int ksteps = sp.planes * ((sp.Np + 7) / 8);
    const double per_mma = std::max(1.0, 2.0 * sp.Np / 128.0);
    return (double)pair_tiles * (3.0 * ksteps * per_mma + 8.0);
}

// Split `avail` clusters between n groups in proportion to w (at least one
// each, at most cap[g] useful): cl_begin[0..n]; returns the clusters used.
static int split_clusters(int avail, const double* w, const long long* cap, int n, int* cl_begin) {
    int cl[kMaxLaunchGroups];
    double W = 0.0;
    for (int g = 0; g < n; ++g) W += w[g];
    int used = 0;
    for (int g = 0; g < n; ++g) {
        const long long want = W > 0.0 ? (long long)(avail * w[g] / W) : 1;
        cl[g] = (int)std::max(1LL, std::min(cap[g], want));
        used += cl[g];
    }
    // hand out what rounding left, to the groups with the most work per cluster
    while (used < avail) {
        int best = -1;
        double bw = 0.0;
        for (int g = 0; g < n; ++g)
            if (cl[g] < cap[g] && w[g] / cl[g] > bw) {
                bw = w[g] / cl[g];
                best = g;
            }
        if (best < 0) break;
        ++cl[best];
        ++used;
    }
    // more groups than clusters can hold cannot occur (n <= 8 < clusters); trim otherwise
    while (used > avail) {
        int best = 0;
        for (int g = 1; g < n; ++g)
            if (cl[g] > cl[best]) best = g;
        if (cl[best] == 1) break;
        --cl[best];
        --used;
    }
    cl_begin[0] = 0;
    for (int g = 0; g < n; ++g) cl_begin[g + 1] = cl_begin[g] + cl[g];
    return cl_begin[n];
}

// One launch of the stage kernel over n plans (same precision mode).
static gkba_status launch_stage_group(gkba_ctx* c, const StagePlan* const* plans, int n, int cls) {
    if (n < 1 || n > kMaxLaunchGroups) return fail(c, GKBA_EINVAL, "stage launch of %d groups", n);
    StageLaunch L{};
    double w[kMaxLaunchGroups];
    long long cap[kMaxLaunchGroups];
    size_t smem = 0;
    double fl = 0.0, by = 0.0;
    for (int g = 0; g < n; ++g) {
        L.tmA[g] = plans[g]->mA;
        L.tmBhi[g] = plans[g]->mBh;
        L.tmBlo[g] = plans[g]->mBl;
        L.p[g] = plans[g]->sp;
        w[g] = plans[g]->weight;
        cap[g] = std::max(1LL, plans[g]->pair_tiles);
        smem = std::max(smem, stage_smem_bytes(plans[g]->sp.Np, plans[g]->sp.astages));
        fl += plans[g]->flops;
        by += plans[g]->bytes;
    }
    L.ngroups = n;
    const int ncl = split_clusters(c->pair_clusters, w, cap, n, L.cl_begin);
    const bool acc = c->prec == GKBA_SPLIT_TF32_ACC;
    auto stage_kernel = n > 1 ? (acc ? k_tc_pair<true, true> : k_tc_pair<false, true>)
                              : (acc ? k_tc_pair<true, false> : k_tc_pair<false, false>);
    auto t = launch_begin(c, cls, fl, by);
    stage_kernel<<<2 * ncl, kStageThreads, smem, c->stream>>>(L);
    return launch_end(c, t);
}

static gkba_status launch_final_group(gkba_ctx* c, const FinalPlan* const* plans, int n) {
    if (n < 1 || n > kMaxLaunchGroups) return fail(c, GKBA_EINVAL, "S4 launch of %d groups", n);
    FinalLaunch L{};
    double w[kMaxLaunchGroups];
    long long cap[kMaxLaunchGroups];
    size_t smem = 0;
    double fl = 0.0, by = 0.0;
    for (int g = 0; g < n; ++g) {
        L.tmA[g] = plans[g]->mA;
        L.tmBhi[g] = plans[g]->mBh;
        L.tmBlo[g] = plans[g]->mBl;
        L.p[g] = plans[g]->fp;
        w[g] = plans[g]->weight;
        cap[g] = std::max(1LL, plans[g]->items);
        smem = std::max(smem, final_pair_smem_bytes(plans[g]->fp.Np));
        fl += plans[g]->flops;
        by += plans[g]->bytes;
    }
    L.ngroups = n;
    const int ncl = split_clusters(c->fin_pair_clusters, w, cap, n, L.cl_begin);
    // Kahan updates of the epilogue: scalar when every group has Np = 96 (48
    // columns per epilogue warp), packed FP32 pairs otherwise (measured: the
    // pairs are 9-10 % faster at 16 and 24 columns, 5 % slower at 48)
    bool all96 = true;
    for (int g = 0; g < n; ++g) all96 = all96 && plans[g]->fp.Np == kFinMaxNp;
    auto fin_kernel = n > 1 ? (all96 ? k_tc_final_pair<true, false> : k_tc_final_pair<true, true>)
                            : (all96 ? k_tc_final_pair<false, false> : k_tc_final_pair<false, true>);
    auto t = launch_begin(c, K_FIN, fl, by);
    fin_kernel<<<2 * ncl, kFinThreads, smem, c->stream>>>(L);
    return launch_end(c, t);
}

// Plan of stage S4 for nb units whose X3 stages S1-S3 (or the time-linear
// back-transforms) left in X13.
static gkba_status plan_final(gkba_ctx* c, int nb, FinalPlan& F) {
    const int Np = c->Np;
    const long long N2 = (long long)Np * Np, N3 = N2 * Np, N4 = N3 * Np;
    float* X13 = (float*)c->X13;
    const double Nr = c->N;
    const double fl_cr = 4.0 * Nr * Nr * Nr * Nr * Nr;
    const double N4r = Nr * Nr * Nr * Nr;
    const bool multi = c->unit_sys != nullptr;
    const long long rows = 2LL * Np * nb;
    const bool blocked = (Np % 32) == 0;
    if (blocked) {
        const long long Rl = ((2LL * Np * nb + 2 * kBM - 1) / (2 * kBM)) * (2 * kBM);
        cuuint64_t d[3] = {32, (cuuint64_t)Rl, (cuuint64_t)(N3 / 32)};
        cuuint64_t s[2] = {32 * 4, (cuuint64_t)(Rl * 32 * 4)};
        cuuint32_t b[3] = {kKC, kBM, 1};
        GKBA_TRY(make_map(c, &F.mA, X13, 3, d, s, b));
    } else {
        cuuint64_t d[2] = {(cuuint64_t)N3, (cuuint64_t)(2LL * Np * nb)};
        cuuint64_t s[1] = {(cuuint64_t)N3 * 4};
        cuuint32_t b[2] = {kKC, kBM};
        GKBA_TRY(make_map(c, &F.mA, X13, 2, d, s, b));
    }
    if (multi) {
        cuuint64_t d[3] = {(cuuint64_t)N3, (cuuint64_t)Np, (cuuint64_t)c->nsys};
        cuuint64_t s[2] = {(cuuint64_t)N3 * 4, (cuuint64_t)(N4 * 4)};
        cuuint32_t b[3] = {kKC, (cuuint32_t)(Np / 2), 1};
        GKBA_TRY(make_map(c, &F.mBh, c->vKhi, 3, d, s, b));
        GKBA_TRY(make_map(c, &F.mBl, c->vKlo, 3, d, s, b));
    } else {
        // each CTA of an S4 pair loads Np/2 rows of vK
        cuuint64_t d[2] = {(cuuint64_t)N3, (cuuint64_t)Np};
        cuuint64_t s[1] = {(cuuint64_t)N3 * 4};
        cuuint32_t b[2] = {kKC, (cuuint32_t)(Np / 2)};
        GKBA_TRY(make_map(c, &F.mBh, c->vKhi, 2, d, s, b));
        GKBA_TRY(make_map(c, &F.mBl, c->vKlo, 2, d, s, b));
    }
    // split-K over (n,r,p)
    FinalParams& fp = F.fp;
    fp = FinalParams{};
    fp.Np = Np;
    fp.K = N3;
    fp.KS = c->acc_window;
    fp.KW = c->fin_kw >= kTcItemK ? c->fin_kw : kTcItemK;
    fp.nks = (int)((N3 + fp.KW - 1) / fp.KW);
    fp.rows = rows;
    fp.ngroups = (int)((rows + 2 * kBM - 1) / (2 * kBM));
    fp.Rld = (long long)fp.ngroups * 2 * kBM;
    fp.blocked = blocked ? 1 : 0;
    fp.part = (float*)c->part;
    fp.err = c->dint + 1;
    fp.unit_sys = c->unit_sys;
    if ((size_t)fp.nks * Np * fp.Rld * 4 > c->part_bytes)
        return fail(c, GKBA_ESTATE, "partial buffer too small");
    F.items = (long long)fp.ngroups * fp.nks;
    F.weight = (double)F.items * (Np + 32);
    F.flops = fl_cr * nb;
    F.bytes = 4.0 * (2 * N4r * nb + 2 * N4r);
    return GKBA_OK;
}

// Stage S4 and the reduction of nb units whose X3 stages S1-S3 (or the
// time-linear back-transforms) left in X13: S_u -> c->Su.
static gkba_status tf32_final(gkba_ctx* c, int nb) {
    FinalPlan F;
    GKBA_TRY(plan_final(c, nb, F));
    const FinalPlan* fpl = &F;
    GKBA_TRY(launch_final_group(c, &fpl, 1));
    return reduce_partials_launch(c, nb, F.fp.nks, (long long)c->Np * F.fp.Rld, F.fp.Rld, c->part, true,
                                  c->Su);
}

// Plans of stages S1-S3 of one batch (forms built) with A1 as S1's A operand
// (wS32, or the omega layout of v for dL/dv): X3 lands in X13, K-blocked when
// Np % 32 == 0.
static gkba_status plan_chain(gkba_ctx* c, int nb, const float* A1, StagePlan (&P)[3]) {
    const int Np = c->Np;
    const long long N2 = (long long)Np * Np, N3 = N2 * Np, N4 = N3 * Np;
    if ((long long)nb * (N3 / kBM) >= (1LL << 31))
        return fail(c, GKBA_EINVAL, "%d units exceed the stage kernel's 32-bit tile index", nb);
    float* X13 = (float*)c->X13;
    float* X2 = (float*)c->X2;
    const long long per = 2LL * Np * Np;
    float* B1hi = (float*)c->formsB1;
    float* B1lo = B1hi + per * c->ub_cap;
    float* Gshi = (float*)c->formsG;
    float* Gslo = Gshi + 2 * per * c->ub_cap;
    float* G3hi = (float*)(c->sep_A ? c->formsG3 : c->formsG);  // stage S3's slot
    float* G3lo = G3hi + 2 * per * c->ub_cap;
    // Flops below are the algorithmic counts of the N-basis problem (padding excluded).
    const double Nr = c->N;
    const double fl_cr = 4.0 * Nr * Nr * Nr * Nr * Nr, fl_cc = 2.0 * fl_cr;
    const double N4r = Nr * Nr * Nr * Nr;

    const bool multi = c->unit_sys != nullptr;  // several systems: w and v per system
    if (multi) {
        cuuint64_t d[3] = {(cuuint64_t)Np, (cuuint64_t)N3, (cuuint64_t)c->nsys};
        cuuint64_t s[2] = {(cuuint64_t)Np * 4, (cuuint64_t)(N4 * 4)};
        cuuint32_t b[3] = {kKC, kBM, 1};
        GKBA_TRY(make_map(c, &P[0].mA, A1, 3, d, s, b));
    } else {
        cuuint64_t d[2] = {(cuuint64_t)Np, (cuuint64_t)N3};
        cuuint64_t s[1] = {(cuuint64_t)Np * 4};
        cuuint32_t b[2] = {kKC, kBM};
        GKBA_TRY(make_map(c, &P[0].mA, A1, 2, d, s, b));
    }
    {
        cuuint64_t d[4] = {(cuuint64_t)Np, 2, (cuuint64_t)N3, (cuuint64_t)nb};
        cuuint64_t s[3] = {(cuuint64_t)Np * 4, (cuuint64_t)2 * Np * 4, (cuuint64_t)(2 * N4 * 4)};
        cuuint32_t b[4] = {kKC, 1, kBM, 1};
        GKBA_TRY(make_map(c, &P[1].mA, X13, 4, d, s, b));
        GKBA_TRY(make_map(c, &P[2].mA, X2, 4, d, s, b));
    }
    {
        // B1[u][(c,r)][s]; Gs[u][4 blocks][p][q]; each CTA of a pair loads Np rows
        cuuint64_t d[3] = {(cuuint64_t)Np, (cuuint64_t)2 * Np, (cuuint64_t)nb};
        cuuint64_t s[2] = {(cuuint64_t)Np * 4, (cuuint64_t)per * 4};
        cuuint32_t b[3] = {kKC, (cuuint32_t)Np, 1};
        GKBA_TRY(make_map(c, &P[0].mBh, B1hi, 3, d, s, b));
        GKBA_TRY(make_map(c, &P[0].mBl, B1lo, 3, d, s, b));
        cuuint64_t dg[3] = {(cuuint64_t)Np, (cuuint64_t)4 * Np, (cuuint64_t)nb};
        cuuint64_t sg[2] = {(cuuint64_t)Np * 4, (cuuint64_t)2 * per * 4};
        GKBA_TRY(make_map(c, &P[1].mBh, Gshi, 3, dg, sg, b));
        GKBA_TRY(make_map(c, &P[1].mBl, Gslo, 3, dg, sg, b));
        GKBA_TRY(make_map(c, &P[2].mBh, G3hi, 3, dg, sg, b));
        GKBA_TRY(make_map(c, &P[2].mBl, G3lo, 3, dg, sg, b));
    }
    const long long pair_tiles = (long long)nb * (N3 / kBM) / 2;
    StageParams sp = stage_base(c, nb);
    // S1: rows (j,m,q), cols (c,r) -> X1[j][r][m][c][q]
    sp.planes = 1;
    sp.a_unit = 0;
    sp.unit_sys = c->unit_sys;
    sp.out = X13;
    sp.map = StageMap{2 * N3, 2 * Np, 1, Np, 2 * N2, Np, Np, Np};
    P[0].sp = sp;
    P[0].flops = fl_cr * nb;
    P[0].bytes = 4.0 * (N4r + 2 * N4r * nb);
    P[0].cls = K_W1;
    // S2: rows (j,r,m), K (c,q), cols (c',p) -> X2[j][r][p][c'][m]
    sp.planes = 2;
    sp.a_unit = 1;
    sp.unit_sys = nullptr;
    sp.out = X2;
    sp.map = StageMap{2 * N3, 2 * N2, 1, Np, 2 * Np, Np, Np, Np};
    P[1].sp = sp;
    P[1].flops = fl_cc * nb;
    P[1].bytes = 4.0 * 4 * N4r * nb;
    P[1].cls = K_W2;
    // S3: rows (j,r,p), K (c,m), cols (c',n) -> X3 with rows (u,c',j) and K (n,r,p):
    // K-blocked X3[K/32][Rld][32] when Np % 32 == 0 (one contiguous 16 KB block
    // per 128 x 32 tile of the last stage), else X3[u][c'][j][n][r][p].
    const long long rows = 2LL * Np * nb;
    const long long Rld = ((rows + 2 * kBM - 1) / (2 * kBM)) * (2 * kBM);
    const bool blocked = (Np % 32) == 0;
    if (blocked && (size_t)(N3 * Rld * 4) > c->x13_bytes)
        return fail(c, GKBA_ESTATE, "X3 buffer too small for the K-blocked layout");
    sp.out = X13;
    if (blocked) {
        sp.map = StageMap{32, Np * Rld, 0, 32 * Np, N2 * Rld, Np, Np, Np, 32 * Rld};
        sp.out_unit = 2LL * Np * 32;
    } else {
        sp.map = StageMap{N3, Np, 1, N4, N2, Np, Np, Np};
    }
    P[2].sp = sp;
    P[2].flops = fl_cc * nb;
    P[2].bytes = 4.0 * 4 * N4r * nb;
    P[2].cls = K_W3;
    for (int k = 0; k < 3; ++k) {
        P[k].pair_tiles = pair_tiles;
        P[k].weight = stage_weight(P[k].sp, pair_tiles);
    }
    return GKBA_OK;
}

// Stages S1-S3 of one batch; with do_final, stage S4 and the reduction follow:
// S_u -> c->Su.
static gkba_status tf32_chain(gkba_ctx* c, int nb, const float* A1, bool do_final) {
    StagePlan P[3];
    GKBA_TRY(plan_chain(c, nb, A1, P));
    for (int k = 0; k < 3; ++k) {
        const StagePlan* pk = &P[k];
        GKBA_TRY(launch_stage_group(c, &pk, 1, P[k].cls));
    }
    if (!do_final) return GKBA_OK;
    return tf32_final(c, nb);
}

// Tensor-core contraction of one batch (forms built): S_u -> c->Su.
gkba_status contract_batch_tf32(gkba_ctx* c, int nb) { return tf32_chain(c, nb, c->wS32, true); }

// Several problems at once (each context's forms built, its batch of nbs[i]
// units): one launch per stage for all of them, the clusters split by cost;
// then each context's reduction: S_u -> cs[i]->Su.  The contexts share c0's
// stream and precision mode.
gkba_status contract_batch_tf32_multi(gkba_ctx* const* cs, const int* nbs, int n) {
    if (n < 1 || n > kMaxLaunchGroups) return fail(cs[0], GKBA_EINVAL, "%d problems in one launch", n);
    gkba_ctx* c0 = cs[0];
    StagePlan P[kMaxLaunchGroups][3];
    for (int i = 0; i < n; ++i) GKBA_TRY(plan_chain(cs[i], nbs[i], cs[i]->wS32, P[i]));
    for (int k = 0; k < 3; ++k) {
        const StagePlan* pk[kMaxLaunchGroups];
        for (int i = 0; i < n; ++i) pk[i] = &P[i][k];
        GKBA_TRY(launch_stage_group(c0, pk, n, P[0][k].cls));
    }
    FinalPlan F[kMaxLaunchGroups];
    const FinalPlan* fk[kMaxLaunchGroups];
    for (int i = 0; i < n; ++i) {
        GKBA_TRY(plan_final(cs[i], nbs[i], F[i]));
        fk[i] = &F[i];
    }
    GKBA_TRY(launch_final_group(c0, fk, n));
    for (int i = 0; i < n; ++i)
        GKBA_TRY(reduce_partials_launch(cs[i], nbs[i], F[i].fp.nks, (long long)cs[i]->Np * F[i].fp.Rld,
                                        F[i].fp.Rld, cs[i]->part, true, cs[i]->Su));
    return GKBA_OK;
}

// dL/dv on the tensor-core path: the omega layout of v (once per context).
gkba_status tf32_prepare_vgrad(gkba_ctx* c) {
    if (c->vO32) return GKBA_OK;
    const long long Np4 = (long long)c->Np * c->Np * c->Np * c->Np;
    if (cudaMalloc(&c->vO32, Np4 * 4) != cudaSuccess) {
        cudaGetLastError();
        c->vO32 = nullptr;
        return fail(c, GKBA_ENOMEM, "omega layout of v (%lld floats) does not fit", Np4);
    }
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_build_vO32<<<grid1(Np4, 256), 256, 0, c->stream>>>(c->N, c->Np, c->v, c->vO32);
    return launch_end(c, t);
}

// X3 of the w-slot chain: stages S1-S3 with the omega layout of v (forms built).
gkba_status tf32_chain_omega(gkba_ctx* c, int nb) { return tf32_chain(c, nb, c->vO32, false); }

// Launch of k_xslot_tc over the X3 of nb units in X13.
static gkba_status xslot_launch(gkba_ctx* c, int nb, XSlotParams xp, int cls, double bytes) {
    const int N = c->N, Np = c->Np;
    const long long N3 = (long long)N * N * N;
    const long long rows = 2LL * Np * nb;
    xp.N = N;
    xp.Np = Np;
    xp.nb = nb;
    xp.Rld = ((rows + 2 * kBM - 1) / (2 * kBM)) * (2 * kBM);
    xp.blocked = (Np % 32) == 0 ? 1 : 0;
    xp.X = (const float*)c->X13;
    const long long Rtot = 2LL * N * nb;
    if (Rtot >= (1LL << 31)) return fail(c, GKBA_EINVAL, "slot contraction of %d units: too many rows", nb);
    const unsigned gx = grid1(N3, kXsThreads), gy = (unsigned)((xp.A + kXsA - 1) / kXsA);
    // enough blocks for about eight per SM, each over at least 1024 rows
    long long gz = std::max(1LL, std::min((Rtot + 1023) / 1024,
                                          (8LL * c->num_sms + gx * gy - 1) / ((long long)gx * gy)));
    const long long per = ((Rtot + gz - 1) / gz + kXsRows - 1) / kXsRows * kXsRows;
    gz = (Rtot + per - 1) / per;
    xp.rows_per_z = per;
    const size_t wbytes = (size_t)Rtot * xp.A * sizeof(float);
    if (wbytes > c->xsw_bytes) {
        if (c->xsw) cudaFree(c->xsw);
        c->xsw = nullptr;
        c->xsw_bytes = 0;
        if (cudaMalloc(&c->xsw, wbytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, GKBA_ENOMEM, "slot contraction weights (%zu bytes) do not fit", wbytes);
        }
        c->xsw_bytes = wbytes;
    }
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_xslot_weights<<<grid1(Rtot * xp.A, 256), 256, 0, c->stream>>>(xp, c->xsw);
    GKBA_TRY(launch_end(c, t));
    t = launch_begin(c, cls, 2.0 * (double)N3 * xp.A * Rtot, bytes);
    k_xslot_tc<<<dim3(gx, gy, (unsigned)gz), kXsThreads, 0, c->stream>>>(xp, c->xsw);
    return launch_end(c, t);
}

gkba_status vbar_slot_tf32(gkba_ctx* c, int nb, const double2* Sbar, int transposeS, double* out) {
    const long long N = c->N;
    XSlotParams xp{};
    xp.A = (int)N;
    xp.mode = 0;
    xp.S = Sbar;
    xp.transposeS = transposeS;
    xp.out = out;
    xp.SJ = N * N * N;
    xp.SC = 0;
    xp.SN = N * N;
    xp.SR = N;
    return xslot_launch(c, nb, xp, K_RED, 4.0 * 2.0 * N * nb * N * N * N);
}

// One complex one-index transform of a single unit on the stage kernel (S2 /
// S3 form): A planar [rows][c][Np] FP32 at `in`, B the TF32 forms of unit
// `bunit` in formsG3, output through `map` into `out`.
static gkba_status tl_stage(gkba_ctx* c, const float* in, int bunit, float* out, StageMap map,
                            long long out_unit) {
    const int Np = c->Np;
    const long long N3 = (long long)Np * Np * Np, N4 = N3 * Np;
    const long long per = 2LL * Np * Np;
    const float* Bhi = (const float*)c->formsG3 + 2 * per * bunit;
    const float* Blo = (const float*)c->formsG3 + 2 * per * c->ub_cap + 2 * per * bunit;
    StagePlan P;
    {
        cuuint64_t d[4] = {(cuuint64_t)Np, 2, (cuuint64_t)N3, 1};
        cuuint64_t s[3] = {(cuuint64_t)Np * 4, (cuuint64_t)2 * Np * 4, (cuuint64_t)(2 * N4 * 4)};
        cuuint32_t b[4] = {kKC, 1, kBM, 1};
        GKBA_TRY(make_map(c, &P.mA, in, 4, d, s, b));
    }
    {
        cuuint64_t d[3] = {(cuuint64_t)Np, (cuuint64_t)4 * Np, 1};
        cuuint64_t s[2] = {(cuuint64_t)Np * 4, (cuuint64_t)2 * per * 4};
        cuuint32_t b[3] = {kKC, (cuuint32_t)Np, 1};
        GKBA_TRY(make_map(c, &P.mBh, Bhi, 3, d, s, b));
        GKBA_TRY(make_map(c, &P.mBl, Blo, 3, d, s, b));
    }
    P.sp = stage_base(c, 1);
    P.sp.planes = 2;
    P.sp.a_unit = 1;
    P.sp.out = out;
    P.sp.out_unit = out_unit;
    P.sp.map = map;
    P.pair_tiles = N3 / kBM / 2;
    P.weight = stage_weight(P.sp, P.pair_tiles);
    const double Nr = c->N;
    P.flops = 8.0 * Nr * Nr * Nr * Nr * Nr;
    P.bytes = 4.0 * 4 * Nr * Nr * Nr * Nr;
    P.cls = K_TL;
    const StagePlan* pp = &P;
    return launch_stage_group(c, &pp, 1, K_TL);
}

// The time-linear collision's tensor contractions on the tensor cores:
//   S = sum_{npr} v_irpn (Ucal x_n Ucal x_p conj(Ucal) x_r Lambda)_{j n r p} -> c->Su
// with Ucal = W^+ and Lambda FP64 [j][n][r][c][p] (N basis).  Lambda is
// rounded to FP32 (it is a sum that is already final), the three one-index
// transforms run on the stage kernel and the last writes X3 in stage S4's
// layout:
//   x_p, Ucal:       rows (j, n, r)  -> [j][n][p'][c'][r]
//   x_r, conj(Ucal): rows (j, n, p') -> [j][r'][p'][c'][n]
//   x_n, Ucal:       rows (j, r', p') -> X3 (rows (c', j), K (n', r', p'))
gkba_status tl_apply_tf32(gkba_ctx* c, const double2* W, const double* lam) {
    const int N = c->N, Np = c->Np;
    const long long NN = (long long)N * N;
    const long long N2 = (long long)Np * Np, N3 = N2 * Np, N4 = N3 * Np;
    double2* UU = c->Yu;  // Ucal, conj(Ucal)
    auto t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_tl_ucal2<<<grid1(NN, 256), 256, 0, c->stream>>>(N, W, UU);
    GKBA_TRY(launch_end(c, t));
    t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_forms_tf32<<<grid1(2LL * Np * Np * 2, 256), 256, 0, c->stream>>>(N, Np, 2, c->ub_cap, UU, nullptr,
                                                                        nullptr, (float*)c->formsG3);
    GKBA_TRY(launch_end(c, t));
    float* X2 = (float*)c->X2;
    float* X13 = (float*)c->X13;
    t = launch_begin(c, K_PREP, 0.0, 0.0);
    k_tl_lam32<<<grid1(2 * N3, 8), 256, 0, c->stream>>>(N, Np, lam, X2);  // 8 rows per block
    GKBA_TRY(launch_end(c, t));
    GKBA_TRY(tl_stage(c, X2, 0, X13, StageMap{2 * N3, 2 * N2, 1, Np, 2 * Np, Np, Np, Np}, 2 * N4));
    GKBA_TRY(tl_stage(c, X13, 1, X2, StageMap{2 * N3, 1, 2 * Np, Np, 2 * N2, Np, Np, Np}, 2 * N4));
    const long long Rld = 2 * kBM;  // one unit: 2 Np <= 256 rows
    const bool blocked = (Np % 32) == 0;
    if (blocked && (size_t)(N3 * Rld * 4) > c->x13_bytes)
        return fail(c, GKBA_ESTATE, "X3 buffer too small for the K-blocked layout");
    if (blocked)
        GKBA_TRY(tl_stage(c, X2, 0, X13, StageMap{32, Np * Rld, 0, 32 * Np, N2 * Rld, Np, Np, Np, 32 * Rld},
                          2LL * Np * 32));
    else
        GKBA_TRY(tl_stage(c, X2, 0, X13, StageMap{N3, Np, 1, N4, N2, Np, Np, Np}, 2 * N4));
    return tf32_final(c, 1);
}

// Time-linear terms on the tensor cores (forms of the nb = 2 nk units built):
// stages S1-S3 give Z(X_k, Xb_k) and Z(Xb_k, X_k) as X3; the accumulator
// contraction over j writes D = sum_k c_k [Z(Xb_k, X_k) x_j X_k^+ - Z(X_k, Xb_k) x_j Xb_k^+]
// as FP64 [j2][n][r][c2][p] (planar complex).
gkba_status tl_terms_tf32(gkba_ctx* c, int nb, const double2* Gb, int k0, double w_first,
                          double w_rest, double* D) {
    const long long N = c->N;
    GKBA_TRY(tf32_chain(c, nb, c->wS32, false));
    GKBA_CUDA(c, cudaMemsetAsync(D, 0, 2 * N * N * N * N * 8, c->stream));
    XSlotParams xp{};
    xp.A = (int)(2 * N);
    xp.mode = 1;
    xp.S = Gb;
    xp.k0 = k0;
    xp.w_first = w_first;
    xp.w_rest = w_rest;
    xp.out = D;
    xp.SJ = 2 * N * N * N;
    xp.SC = N;
    xp.SN = 2 * N * N;
    xp.SR = 2 * N;
    return xslot_launch(c, nb, xp, K_TL, 4.0 * 2.0 * N * nb * N * N * N + 8.0 * 2 * N * N * N * N);
}


gkba_status wait_selftest(gkba_ctx* c, double limit_ms, double* elapsed_ms) {
    unsigned long long* el = nullptr;
    GKBA_CUDA(c, cudaMalloc(&el, 2 * sizeof(unsigned long long)));
    GKBA_CUDA(c, cudaMemsetAsync(el, 0, 2 * sizeof(unsigned long long), c->stream));
    k_wait_selftest<<<2, 32, 0, c->stream>>>(c->dint + 1, (unsigned long long)(limit_ms * 1e6), el);
    const cudaError_t le = cudaGetLastError();
    unsigned long long h[2] = {0, 0};
    const cudaError_t ce = cudaMemcpyAsync(h, el, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    cudaFree(el);
    if (le != cudaSuccess || ce != cudaSuccess)
        return fail(c, GKBA_ECUDA, "wait self-test: %s", cudaGetErrorString(le != cudaSuccess ? le : ce));
    if (elapsed_ms) {
        elapsed_ms[0] = h[0] * 1e-6;
        elapsed_ms[1] = h[1] * 1e-6;
    }
    return GKBA_OK;
}

gkba_status measure_tf32_mma(gkba_ctx* c, int iters, double* tflops) {
    // unused dynamic shared memory keeps one CTA (and one tensor-memory
    // allocation) per SM, as in the stage kernels
    const int pad = 150 * 1024;
    GKBA_CUDA(c, cudaFuncSetAttribute(k_mma_rate, cudaFuncAttributeMaxDynamicSharedMemorySize, pad));
    int ncl = 0;
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(c->num_sms & ~1));
        cfg.blockDim = dim3(128);
        cfg.dynamicSmemBytes = pad;
        cfg.stream = c->stream;
        GKBA_CUDA(c, cudaOccupancyMaxActiveClusters(&ncl, k_mma_rate, &cfg));
    }
    if (ncl < 1) return fail(c, GKBA_ECUDA, "no 2-CTA cluster of the rate probe fits");
    const int pairs = std::min(ncl, c->num_sms / 2);
    cudaEvent_t e0, e1;
    GKBA_CUDA(c, cudaEventCreate(&e0));
    GKBA_CUDA(c, cudaEventCreate(&e1));
    k_mma_rate<<<2 * pairs, 128, pad, c->stream>>>(std::max(16, iters / 8), c->dint + 1);  // warm-up
    cudaEventRecord(e0, c->stream);
    k_mma_rate<<<2 * pairs, 128, pad, c->stream>>>(iters, c->dint + 1);
    cudaEventRecord(e1, c->stream);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t se = cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (le != cudaSuccess || se != cudaSuccess)
        return fail(c, GKBA_ECUDA, "rate probe: %s", cudaGetErrorString(le != cudaSuccess ? le : se));
    const double flops = (double)pairs * iters * 4.0 * 2.0 * 256.0 * kRateN * 8.0;
    *tflops = ms > 0.0f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return GKBA_OK;
}

size_t tf32_part_bytes(int Np, int ub, int kchunk) {
    const long long N3 = (long long)Np * Np * Np;
    (void)kchunk;
    const long long kw = kTcItemK;
    const long long nks = (N3 + kw - 1) / kw;
    const long long rows = 2LL * Np * ub;
    const long long Rld = ((rows + 255) / 256) * 256;
    return (size_t)(nks * Np * Rld * 4);
}

}  // namespace gkba
