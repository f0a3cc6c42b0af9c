// FP64 -> FP32 conversion by integer arithmetic on the IEEE 754 bit
// patterns. On this GPU the FP64 unit retires about 1/64 of the FP32 and
// integer rate, and a hardware conversion from double runs on it; the
// residual gather converts every local row, so that conversion is done on
// the integer units instead. It restates IEEE 754 binary64 -> binary32
// rounding to nearest, ties to even, for results that are normal floats and
// for zeros; the rare rest (results below the smallest normal float,
// overflow, infinities, NaN) goes to the compiler's conversion. Host and
// device share the code, so a host test checks it bit for bit against the C
// cast.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define RAS_CVT_HD __host__ __device__ __forceinline__
#else
#define RAS_CVT_HD inline
#endif

namespace ras {

RAS_CVT_HD uint64_t cvt_bits_f64(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t u;
  memcpy(&u, &v, 8);
  return u;
#endif
}
RAS_CVT_HD float cvt_f32_bits(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float v;
  memcpy(&v, &u, 4);
  return v;
#endif
}

// double -> float, round to nearest, ties to even.
RAS_CVT_HD float f64_to_f32_rn(double v) {
  const uint64_t u = cvt_bits_f64(v);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);  // biased binary64 exponent
  if (e == 0) return cvt_f32_bits(sign);     // zero or a binary64 subnormal: rounds to +-0
  // binary32 normal range: binary64 exponents 1023 - 126 .. 1023 + 127
  if (e < 897 || e > 1150) return (float)v;
  // sign | rebiased exponent | the top 23 of the 52 fraction bits ...
  uint32_t f = sign | ((uint32_t)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  // ... rounded on the 29 dropped bits; a carry out of the fraction steps the
  // exponent (up to infinity from the largest binade, as IEEE rounding does)
  const uint32_t rest = lo & 0x1fffffffu, half = 0x10000000u;
  f += (rest > half || (rest == half && (f & 1u))) ? 1u : 0u;
  return cvt_f32_bits(f);
}

}  // namespace ras
