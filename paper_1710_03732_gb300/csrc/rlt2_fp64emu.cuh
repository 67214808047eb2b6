// IEEE 754 binary64 addition and subtraction, round to nearest with ties to
// even, computed with integer operations only.
//
// GB300 retires FP64 additions at about 1.6 lanes per clock per SM and 32-bit
// integer operations at about 128, so a kernel whose FP64 pipe is saturated
// (the z move) can move some of its exactly rounded additions onto the integer
// pipes.  The result must be the FP64 pipe's bit for bit (the moves are held
// to the oracle exactly), so this is a full implementation of the IEEE
// definition for finite operands:
//   - the operands are ordered by magnitude; the smaller one's significand is
//     aligned to the larger one's exponent with 10 extra low bits, the bits
//     shifted out beyond them folded into the lowest bit (sticky);
//   - the significands are added or subtracted (exact in 64 bits);
//   - the sum is normalised: one right shift on a carry (sticky kept), or a
//     left shift by the leading-zero count, limited so that the exponent stays
//     >= 1 (gradual underflow: the result is then subnormal);
//   - it is rounded to 53 bits by the 10 low bits (above half, or exactly half
//     with an odd last bit, rounds up); adding the significand to the biased
//     exponent field minus one carries a rounding overflow into the exponent
//     and leaves subnormals with field 0;
//   - an exact zero from operands of opposite sign is +0 (round to nearest);
//     equal-sign zeros keep their sign; an exponent that reaches 2047 gives
//     infinity with the larger operand's sign.
// Infinite or NaN operands are not handled (the kernels' values are finite).
// Written from the IEEE 754 definition of correctly rounded addition.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define RLT2_HD __host__ __device__ __forceinline__
#else
#define RLT2_HD inline
#endif

namespace rlt2 {

RLT2_HD int emu_clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

RLT2_HD uint64_t emu_add_bits(uint64_t ua, uint64_t ub) {
  constexpr uint64_t kSign = 0x8000000000000000ull, kFrac = 0x000FFFFFFFFFFFFFull, kHidden = 1ull << 52;
  uint64_t ma = ua & ~kSign, mb = ub & ~kSign;
  if (ma < mb) {  // |a| >= |b| from here on
    const uint64_t t = ua;
    ua = ub;
    ub = t;
    const uint64_t m = ma;
    ma = mb;
    mb = m;
  }
  const uint64_t sign = ua & kSign;
  const bool subtract = ((ua ^ ub) & kSign) != 0;
  const int ea_f = (int)(ma >> 52), eb_f = (int)(mb >> 52);
  const uint64_t fa = (ma & kFrac) | (ea_f ? kHidden : 0), fb = (mb & kFrac) | (eb_f ? kHidden : 0);
  const int ea = ea_f ? ea_f : 1, eb = eb_f ? eb_f : 1;  // subnormals: exponent 1, no hidden bit
  const uint64_t A = fa << 10;                            // hidden bit at 62
  uint64_t B = fb << 10;
  const int d = ea - eb;  // >= 0
  if (d >= 63) {
    B = B != 0 ? 1ull : 0ull;
  } else if (d > 0) {
    const uint64_t lost = B & ((1ull << d) - 1);
    B = (B >> d) | (lost != 0 ? 1ull : 0ull);
  }
  uint64_t R = subtract ? A - B : A + B;
  if (R == 0) return subtract ? 0ull : sign;  // x - x = +0; -0 + -0 = -0
  int e = ea;
  if (R >> 63) {
    R = (R >> 1) | (R & 1ull);
    e += 1;
  } else {
    int sh = emu_clz64(R) - 1;  // shifts that bring the leading bit to 62
    if (sh > e - 1) sh = e - 1;  // no lower than exponent 1: subnormal
    R <<= sh;
    e -= sh;
  }
  uint64_t mant = R >> 10;
  const unsigned rb = (unsigned)(R & 0x3FFull);
  if (rb > 0x200u || (rb == 0x200u && (mant & 1ull))) mant += 1;
  if (e >= 2047 || (e == 2046 && (mant >> 53))) return sign | 0x7FF0000000000000ull;  // overflow: infinity
  return sign | (((uint64_t)(e - 1) << 52) + mant);
}

#if defined(__CUDACC__)
// a + b and a - b on doubles, rounded as __dadd_rn / __dsub_rn
__device__ __forceinline__ double emu_dadd(double a, double b) {
  return __longlong_as_double((long long)emu_add_bits((uint64_t)__double_as_longlong(a),
                                                     (uint64_t)__double_as_longlong(b)));
}
__device__ __forceinline__ double emu_dsub(double a, double b) {
  return __longlong_as_double((long long)emu_add_bits((uint64_t)__double_as_longlong(a),
                                                     (uint64_t)__double_as_longlong(b) ^ 0x8000000000000000ull));
}
#endif

}  // namespace rlt2
