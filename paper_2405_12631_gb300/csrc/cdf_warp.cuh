// Integer CDF table of one distribution from its FP32 edge values, built by
// one warp. Shared by the Laplace table bank and the logistic-mixture
// tables, whose definitions differ only in F.
#pragma once

#include "pw_internal.cuh"

namespace pw {

// Lane l owns symbols 4l .. 4l+3 (kNSym = 127 symbols) and CDF entries
// 4l .. 4l+3 (128 entries: cdf[0] = 0 .. cdf[127] = M). F[i] is the
// distribution function at edge 4l + i (edge e separates symbols e and
// e + 1; edges 126 and 127 do not exist and their F is ignored).
// p_s = F(s) - F(s - 1) with F(-1) = 0 and F(126) = 1, f_s = 1 +
// floor(max(p_s, 0) (M - 127)), the signed remainder M - sum f added to the
// first largest f. Returns the lane's f in f[] and cdf[4l] (the sum of f
// over the symbols before 4l); entry 4l + i is that plus f[0 .. i-1].
__device__ __forceinline__ int warp_cdf(const float F[4], int lane, int f[4]) {
  float prevF = __shfl_up_sync(0xffffffffu, F[3], 1);
  if (lane == 0) prevF = 0.f;
  int sum = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int s = 4 * lane + i;
    const float lo = (i == 0) ? prevF : F[i - 1];
    const float hi = (s == kNSym - 1) ? 1.f : F[i];
    float p = (s == 0) ? F[0] : __fsub_rn(hi, lo);
    p = fmaxf(p, 0.f);
    const int q = (int)floorf(__fmul_rn(p, (float)(kM - kNSym)));
    f[i] = (s < kNSym) ? 1 + q : 0;
    sum += f[i];
  }
  // warp sum and first argmax
  int best = -1, bidx = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (f[i] > best) { best = f[i]; bidx = 4 * lane + i; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const int ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
  }
  const int rem = (int)kM - sum;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (4 * lane + i == bidx) f[i] += rem;
  // exclusive scan of the lanes' block sums
  const int local = f[0] + f[1] + f[2] + f[3];
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  return incl - local;
}

}  // namespace pw
