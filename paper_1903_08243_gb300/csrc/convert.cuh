// double <-> float conversions on the integer pipe.
//
// On GB300 the F2F conversion instructions issue on the FP64 pipe (2 lanes
// per clock per SM), so converting one input and one output value per dof
// would cost the FP32 kernels more than their arithmetic.  These versions
// work on the IEEE-754 bit fields with integer instructions.
//
// d2f: round to nearest, ties to even, for |x| in the normal float range;
// magnitudes below the smallest normal float (1.2e-38) become signed zero,
// magnitudes above the largest float become infinity, NaN stays NaN.
// f2d: exact for normal floats and zero; float subnormals become zero.
#pragma once

#include <cuda_runtime.h>

namespace mfa {

__device__ __forceinline__ float d2f_bits(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u));
  const int fe = e - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 of the 52 fraction bits
  const unsigned rest = lo & 0x1fffffffu;                   // the 29 dropped bits
  unsigned f = sign | ((unsigned)fe << 23) | m;
  if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) f += 1u;  // a carry may bump the exponent: correct
  return __uint_as_float(f);
}

__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0) return __longlong_as_double((long long)((unsigned long long)sign << 32));
  unsigned hi;
  if (e == 0xff) hi = sign | 0x7ff00000u | ((u & 0x7fffffu) >> 3) | ((u & 0x7fffffu) ? 0x80000u : 0u);
  else hi = sign | ((e - 127u + 1023u) << 20) | ((u & 0x7fffffu) >> 3);
  const unsigned lo = (u & 0x7u) << 29;
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

}  // namespace mfa
