// FP32 functions defined as fixed sequences of correctly rounded operations.
//
// Results that two implementations must reproduce bit for bit (the CDF
// tables every encoder and decoder build, and the integer lifting of
// lossless streams, whose predict / update outputs are rounded to integers
// (Fig. 2 caption)) may not depend on a math library's exp or tanh, nor on
// the compiler contracting a multiply and an add. Every operation here is
// an explicitly rounded intrinsic (__fmul_rn, __fadd_rn, __fsub_rn,
// __fdiv_rn: IEEE round to nearest even, never fused), so the same sequence
// evaluated by any IEEE FP32 arithmetic gives the same bits.
#pragma once

#include <cuda_runtime.h>

namespace pw {

// exp(z) for z <= 0: z < -80 gives 0; otherwise k = rint(z / ln 2) (as
// z * log2(e)), r = (z - k ln2_hi) - k ln2_lo (Cody-Waite reduction with a
// 16-bit ln2_hi so that k ln2_hi is exact), p = the degree-6 Taylor
// polynomial of e^r (coefficients 1/n!) in Horner order, result p * 2^k with
// 2^k built from its bit pattern (exact).
__device__ __forceinline__ float exp32_spec(float z) {
  if (z < -80.f) return 0.f;
  const float kLog2e = 0x1.715476p+0f;     // float nearest 1/ln 2
  const float kLn2Hi = 0x1.62e4p-1f;       // 0.693145751953125
  const float kLn2Lo = 0x1.7f7d1cp-20f;    // float nearest ln 2 - kLn2Hi
  const float c6 = 0x1.6c16c2p-10f, c5 = 0x1.111112p-7f, c4 = 0x1.555556p-5f,
              c3 = 0x1.555556p-3f, c2 = 0.5f, c1 = 1.f, c0 = 1.f;
  float k = rintf(__fmul_rn(z, kLog2e));
  float r = __fsub_rn(z, __fmul_rn(k, kLn2Hi));
  r = __fsub_rn(r, __fmul_rn(k, kLn2Lo));
  float p = c6;
  p = __fadd_rn(__fmul_rn(p, r), c5);
  p = __fadd_rn(__fmul_rn(p, r), c4);
  p = __fadd_rn(__fmul_rn(p, r), c3);
  p = __fadd_rn(__fmul_rn(p, r), c2);
  p = __fadd_rn(__fmul_rn(p, r), c1);
  p = __fadd_rn(__fmul_rn(p, r), c0);
  float scale = __int_as_float(((int)k + 127) << 23);
  return __fmul_rn(p, scale);
}

// tanh(x), written through the identity tanh(a) = -m / (2 + m) with
// m = e^(-2a) - 1 and a = |x|, then given the sign of x. m comes from its
// Taylor series m = z + z^2/2! + ... + z^11/11! (z = -2a, Horner order
// z * (1 + z * (1/2! + z * (... + z / 11!)))) when z >= -1, where e^z - 1
// would cancel, and from exp32_spec(z) - 1 below that (e^z <= 1/e there).
// The truncated series is accurate to 4e-9 relative on its range; the whole
// function stays within a few FP32 ulps of tanh (checked against FP64 tanh).
__device__ __forceinline__ float tanh32_spec(float x) {
  const float a = fabsf(x);
  const float z = __fmul_rn(-2.f, a);
  float m;
  if (z >= -1.f) {
    const float c11 = 0x1.ae6456p-26f, c10 = 0x1.27e4fcp-22f, c9 = 0x1.71de3ap-19f,
                c8 = 0x1.a01a02p-16f, c7 = 0x1.a01a02p-13f, c6 = 0x1.6c16c2p-10f,
                c5 = 0x1.111112p-7f, c4 = 0x1.555556p-5f, c3 = 0x1.555556p-3f;
    float p = c11;
    p = __fadd_rn(__fmul_rn(p, z), c10);
    p = __fadd_rn(__fmul_rn(p, z), c9);
    p = __fadd_rn(__fmul_rn(p, z), c8);
    p = __fadd_rn(__fmul_rn(p, z), c7);
    p = __fadd_rn(__fmul_rn(p, z), c6);
    p = __fadd_rn(__fmul_rn(p, z), c5);
    p = __fadd_rn(__fmul_rn(p, z), c4);
    p = __fadd_rn(__fmul_rn(p, z), c3);
    p = __fadd_rn(__fmul_rn(p, z), 0.5f);
    p = __fadd_rn(__fmul_rn(p, z), 1.f);
    m = __fmul_rn(p, z);
  } else {
    m = __fsub_rn(exp32_spec(z), 1.f);
  }
  const float t = __fdiv_rn(-m, __fadd_rn(2.f, m));
  return copysignf(t, x);
}

}  // namespace pw
