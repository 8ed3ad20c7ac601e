// Exhaustive host check of gkba::tf32_rna_bits (csrc/tf32_round.h), the
// integer rounding of FP32 to TF32 used by the last contraction's split, and
// of the split's exactness, over all 2^32 FP32 bit patterns.
//
// The reference is the definition of the rounding, computed in double: TF32
// keeps 10 stored mantissa bits, so in the binade [2^E, 2^(E+1)) of a normal
// x (E = -126 for subnormals, whose spacing is fixed) the representable
// magnitudes are the multiples of 2^(E-10); round to nearest with ties away
// from zero picks floor(|x| / 2^(E-10) + 1/2) of them (exact in double), and a
// result of 2^128 or more is infinity.
//
// Printed: "finite_mismatch <n> first <pattern>", "split_inexact <n>",
// "nonfinite_lo_finite <n>" and "overflow_to_inf <n>"; exit status 0.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "tf32_round.h"

static float as_float(uint32_t u) {
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
static uint32_t as_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

static uint32_t reference_rna(uint32_t u) {
    const uint32_t sign = u & 0x80000000u;
    const double ax = std::fabs((double)as_float(u));
    if (ax == 0.0) return sign;
    int e = 0;
    std::frexp(ax, &e);  // ax = f 2^e, f in [1/2, 1): binade exponent e - 1
    const int E = e - 1 < -126 ? -126 : e - 1;
    const double q = std::ldexp(1.0, E - 10);
    const double r = std::floor(ax / q + 0.5) * q;
    const float y = r >= std::ldexp(1.0, 128) ? INFINITY : (float)r;
    return as_bits(y) | sign;
}

int main() {
    unsigned nt = std::thread::hardware_concurrency();
    if (nt < 1) nt = 1;
    if (nt > 64) nt = 64;
    std::atomic<unsigned long long> mismatch{0}, inexact{0}, nonfinite_bad{0}, overflow{0};
    std::atomic<unsigned long long> first{~0ull};
    std::vector<std::thread> th;
    const unsigned long long total = 1ull << 32;
    for (unsigned t = 0; t < nt; ++t) {
        th.emplace_back([&, t]() {
            unsigned long long mm = 0, ie = 0, nb = 0, ov = 0, f0 = ~0ull;
            const unsigned long long b = total * t / nt, e = total * (t + 1) / nt;
            for (unsigned long long i = b; i < e; ++i) {
                const uint32_t u = (uint32_t)i;
                const float x = as_float(u);
                const uint32_t hb = gkba::tf32_rna_bits(u);
                const float hi = as_float(hb);
                const float lo = x - hi;  // the split's lo, as the kernel forms it
                if ((u & 0x7F800000u) == 0x7F800000u) {
                    // infinity or NaN: lo must come out NaN so that it reaches the sum
                    if (!std::isnan(lo)) ++nb;
                    continue;
                }
                if (hb != reference_rna(u)) {
                    ++mm;
                    if (i < f0) f0 = i;
                }
                if (std::isinf(hi)) {
                    ++ov;  // |x| beyond the largest TF32 value: hi = inf, lo = -inf
                    continue;
                }
                if ((double)hi + (double)lo != (double)x) ++ie;
            }
            mismatch += mm;
            inexact += ie;
            nonfinite_bad += nb;
            overflow += ov;
            unsigned long long cur = first.load();
            while (f0 < cur && !first.compare_exchange_weak(cur, f0)) {
            }
        });
    }
    for (auto& x : th) x.join();
    std::printf("finite_mismatch %llu first %llx\n", mismatch.load(), first.load());
    std::printf("split_inexact %llu\n", inexact.load());
    std::printf("nonfinite_lo_finite %llu\n", nonfinite_bad.load());
    std::printf("overflow_to_inf %llu\n", overflow.load());
    return 0;
}
