// Double -> float and double -> float-float conversions on the integer pipes.
//
// On GB300 a double -> float conversion issues on the FP64 pipe, which runs about 1/64 of
// the FP32 rate; kernels that stream FP64 data into FP32 or float-float arithmetic were
// bound by it. These helpers round from the bit pattern instead (IEEE 754 round to nearest,
// ties to even) and give, on their fast path, exactly what the conversion instruction gives:
//   d2f(x)        = RN_float(x)
//   d2ff(x, h, l) : h = RN_float(x), l = RN_float(x - h)   (x - h is exact in double)
//   f2d(x)        = x widened to double (exact)
// Fast path: 2^-74 <= |x| < 2^127 for d2ff, 2^-126 <= |x| < 2^127 for d2f (both words then
// normal floats); every other value (zero, subnormals, overflow, inf, nan) takes the
// conversion instructions. The host build (plain C++) runs the same integer logic and serves
// the exhaustive-by-class check of the test suite.
#pragma once
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define GW_HD __host__ __device__ __forceinline__
#else
#define GW_HD inline
#endif

namespace gwi {
namespace cvt {

GW_HD uint64_t dbits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}

GW_HD float fbits(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof f);
  return f;
#endif
}

GW_HD uint32_t ubits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}

GW_HD double dfrom(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double d;
  std::memcpy(&d, &u, sizeof d);
  return d;
#endif
}

GW_HD double f2d_hw(float x) { return (double)x; }

GW_HD float i2f_rn(int32_t r) {
#if defined(__CUDA_ARCH__)
  return __int2float_rn(r);
#else
  return (float)r;  // the default rounding mode: to nearest, ties to even
#endif
}

GW_HD float d2f_hw(double x) {
#if defined(__CUDA_ARCH__)
  return __double2float_rn(x);
#else
  return (float)x;
#endif
}

// Rounds the 53-bit significand of x (biased exponent E, 949 <= E <= 1149 or, for the high
// word alone, 897 <= E <= 1149) to 24 bits. Returns the float's bits without the sign and, in
// *r, the signed remainder x - h in units of 2^(E - 1075) (|r| <= 2^28).
GW_HD uint32_t round_hi(uint32_t hx, uint32_t lx, uint32_t E, int32_t* r) {
  const uint32_t rem = lx & 0x1FFFFFFFu;  // the 29 significand bits a float drops
  uint32_t f = ((E - 896u) << 23) | ((hx & 0xFFFFFu) << 3) | (lx >> 29);
  const uint32_t up = (rem > 0x10000000u) || (rem == 0x10000000u && (f & 1u));
  f += up;  // a carry out of the significand steps the exponent, as rounding does
  *r = (int32_t)rem - (int32_t)(up << 29);
  return f;
}

GW_HD float d2f(double x) {
  const uint64_t u = dbits(x);
  const uint32_t hx = (uint32_t)(u >> 32), lx = (uint32_t)u;
  const uint32_t E = (hx >> 20) & 0x7FFu;
  if (E < 897u || E > 1149u) return d2f_hw(x);
  int32_t r;
  return fbits(round_hi(hx, lx, E, &r) | (hx & 0x80000000u));
}

GW_HD void d2ff(double x, float& h, float& l) {
  const uint64_t u = dbits(x);
  const uint32_t hx = (uint32_t)(u >> 32), lx = (uint32_t)u;
  const uint32_t E = (hx >> 20) & 0x7FFu;
  if (E < 949u || E > 1149u) {
    h = d2f_hw(x);
    l = d2f_hw(x - (double)h);
    return;
  }
  int32_t r;
  h = fbits(round_hi(hx, lx, E, &r) | (hx & 0x80000000u));
  if (hx >> 31) r = -r;
  // x - h = r 2^(E - 1075): RN of the integer, then an exact scaling by a power of two
  // (the product is a normal float since |r| >= 1 and E >= 949)
  l = i2f_rn(r) * fbits((E - 948u) << 23);
}

// float -> double, exact: the exponent re-biased (127 -> 1023) and the significand widened, for
// every normal float; zeros, subnormals, infinities and nan take the conversion instruction.
GW_HD double f2d(float x) {
  const uint32_t u = ubits(x);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return f2d_hw(x);
  return dfrom(((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29));
}

}  // namespace cvt
}  // namespace gwi
