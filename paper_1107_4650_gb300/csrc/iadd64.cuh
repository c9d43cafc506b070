// IEEE 754 binary64 addition, rounded to nearest (ties to even), computed on the integer units.
//
// GB300 issues FP64 instructions at about 1.7 per SM per clock but 32-bit integer instructions at about 64
// times that rate, so an addition restated on the integer units can take load off the FP64 pipe, which bounds
// the FP64 sweeps.  The result is the same bits as the hardware addition (the correctly rounded sum is unique).
//
// Method (the textbook alignment-and-round procedure for binary floating-point addition): order the operands
// by magnitude; widen both significands (53 bits with the hidden one) by 10 zero bits; shift the smaller one
// right by the exponent difference, folding every bit shifted out into its lowest bit (the sticky bit); add or
// subtract the aligned significands; normalise so that the leading one lands in bit 63; round the 53 upper bits
// to nearest, ties to even, on the 11 bits below them; repack, letting a carry out of the rounded significand
// step the exponent.  With at least two bits below the rounding bit, folding the lost bits into one sticky bit
// cannot move the sum across a rounding boundary: the folded and the exact sum lie strictly between the same two
// even multiples of the lowest kept bit.
//
// Operands outside the fast domain take the hardware addition: a smaller operand that is zero or subnormal, a
// larger operand with biased exponent below 64 (the result might be subnormal) or above 0x7fd (inf, NaN, or
// a sum that needs the overflow path).  Exact cancellation gives +0, as round-to-nearest prescribes.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define DIRAC_IADD_HD __host__ __device__ __forceinline__
#else
#define DIRAC_IADD_HD static inline
#endif

namespace dirac {

DIRAC_IADD_HD uint64_t iadd_bits(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    return u;
#endif
}

DIRAC_IADD_HD double iadd_double(uint64_t u) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, sizeof x);
    return x;
#endif
}

DIRAC_IADD_HD double iadd_hw(double a, double b) {
#if defined(__CUDA_ARCH__)
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}

DIRAC_IADD_HD int iadd_clz(uint64_t r) {  // r != 0
#if defined(__CUDA_ARCH__)
    return __clzll((long long)r);
#else
    return __builtin_clzll(r);
#endif
}

// a + b, the same bits as the hardware binary64 addition in round-to-nearest mode.
DIRAC_IADD_HD double iadd_rn(double a, double b) {
    const uint64_t ua = iadd_bits(a), ub = iadd_bits(b);
    const bool swp = (ua << 1) < (ub << 1);  // order by magnitude (exponent, then significand)
    const uint64_t hi = swp ? ub : ua, lo = swp ? ua : ub;
    const int eh = (int)(hi >> 52) & 0x7ff, el = (int)(lo >> 52) & 0x7ff;
    if (el == 0 || eh < 64 || eh > 0x7fd) return iadd_hw(a, b);
    const uint64_t frac = (1ull << 52) - 1;
    const uint64_t mh = ((hi & frac) | (1ull << 52)) << 10;  // leading one in bit 62
    const uint64_t ml = ((lo & frac) | (1ull << 52)) << 10;
    const int d = eh - el < 63 ? eh - el : 63;  // ml < 2^63, so a shift by 63 leaves nothing
    uint64_t sh = ml >> d;
    sh |= (uint64_t)((sh << d) != ml);  // sticky
    const uint64_t r = ((ua ^ ub) >> 63) ? mh - sh : mh + sh;
    if (r == 0) return 0.0;
    const int lz = iadd_clz(r);  // 0 after a carry, 1 without, more after cancellation (then no sticky)
    const uint64_t n = r << lz;
    const uint64_t mant = n >> 11;  // 53 bits, the hidden one in bit 52
    const uint32_t rem = (uint32_t)n & 0x7ffu;
    const uint64_t up = (rem + (uint32_t)(mant & 1u)) > 0x400u ? 1u : 0u;  // nearest, ties to even
    // exponent eh + 1 - lz >= 2; the hidden bit adds one to the field, a carry out of the rounding another
    const uint64_t res = ((uint64_t)(eh - lz) << 52) + mant + up;
    return iadd_double(res | (hi & (1ull << 63)));
}

DIRAC_IADD_HD double isub_rn(double a, double b) { return iadd_rn(a, -b); }

}  // namespace dirac
