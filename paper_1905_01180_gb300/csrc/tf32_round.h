// tf32_round.h - rounding of an FP32 bit pattern to TF32 on integer
// instructions, shared by the device code and a host-side test.
//
// TF32 keeps FP32's sign and 8-bit exponent and the top 10 of its 23 stored
// mantissa bits.  Adding half a TF32 ulp (bit 12) to the sign-magnitude bit
// pattern and clearing the 13 dropped bits rounds the magnitude to nearest,
// ties away from zero; a carry out of the mantissa moves into the exponent,
// which is the rounded value at a binade boundary (and infinity past the
// largest finite TF32 value).  For every finite x this equals the
// conversion instruction cvt.rna.tf32.f32; NaN and infinity inputs are not
// handled (the caller keeps them non-finite, see split_tf32_exact_lo).
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define GKBA_TF32_HD __host__ __device__ __forceinline__
#else
#define GKBA_TF32_HD inline
#endif

namespace gkba {

GKBA_TF32_HD uint32_t tf32_rna_bits(uint32_t u) { return (u + 0x1000u) & 0xFFFFE000u; }

}  // namespace gkba
