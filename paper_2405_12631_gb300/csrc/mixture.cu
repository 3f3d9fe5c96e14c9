// Logistic-mixture (K = 3) probability model: the alternative to the
// Laplace model of Section 3.1 that the paper's experiments compare
// (Section 4). Each symbol gets its own integer CDF table, so instead of an
// index into a fixed bank the context model's head produces a key that
// every encoder and decoder turns into the same table:
//
//   parameters (per position): weight logits w_k, means mu_k and scales
//   sigma_k = softplus(rho_k) from the head's 9 outputs (w, mu, rho);
//   decision (FP32): a = the first k of largest w_k, ctr = rint(mu_a)
//   (|ctr| <= 2^23), q_k = clamp(rint(8 (mu_k - ctr)), -255, 255),
//   g_k = clamp(rint(4 (w_k - w_a)), -31, 0), j_k = the scale bin of sigma_k
//   (8 bins per octave above 0.125, as for the Laplace tables);
//   table of r = y - ctr: edges u_e = e - 62.5 (e = 0..125), m_k = q_k / 8,
//   inv_k = 1 / b_{j_k} (b_j the middle of bin j), om_k = exp(g_k / 4),
//   W = (om_0 + om_1) + om_2, z = (u_e - m_k) inv_k,
//   S(z) = 1 / (1 + exp(-z)) (z >= 0) or e / (1 + e), e = exp(z) (z < 0),
//   F(u_e) = ((om_0 S_0 + om_1 S_1) + om_2 S_2) / W; then frequencies, the
//   remainder and the escapes exactly as for the Laplace tables.
// Every operation is one explicitly rounded FP32 operation and exp is the
// library's own exp32_spec, so the tables do not depend on the GPU, the
// compiler or the batch.
//
// Decoding: the last convolution of each coding step stores z' (the head's
// input); k_mix_head then takes one warp per symbol of the step: the 9 head
// outputs (lanes split the channels, butterfly sums, which leave the same
// value in every lane), the decision, the 127-symbol table (4 per lane) and
// its 16 coarse entries, written as one 288-byte row that the rANS decoder
// reads in place of a bank table. Encoding runs the same kernel with the
// symbol values known and keeps only each symbol's (cdf, frequency) pair.
#include <cstdint>

#include "cdf_warp.cuh"
#include "ctx_kernels.cuh"
#include "pw_internal.cuh"
#include "spec_math.cuh"

namespace pw {

__device__ __forceinline__ float sigmoid32_spec(float z) {
  if (z >= 0.f) return __fdiv_rn(1.f, __fadd_rn(1.f, exp32_spec(-z)));
  const float e = exp32_spec(z);
  return __fdiv_rn(e, __fadd_rn(1.f, e));
}

// Decision of one position from its parameters (identical in every lane).
// Key: q_k + 255 (9 bits each) at bits 0, 9, 18; j_k (7 bits) at 27, 34,
// 41; -g_k (5 bits) at 48, 53, 58.
__device__ __forceinline__ void mix_decide(const float w[3], const float mu[3],
                                           const float sg[3], int &ctr, uint64_t &key) {
  // the first component of largest weight logit: its w and mu
  float wa = w[0], mua = mu[0];
  if (w[1] > wa) { wa = w[1]; mua = mu[1]; }
  if (w[2] > wa) { wa = w[2]; mua = mu[2]; }
  float t = rintf(mua);
  t = fminf(fmaxf(t, -8388608.f), 8388608.f);
  ctr = (int)t;
  key = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int q = (int)rintf(__fmul_rn(__fsub_rn(mu[k], (float)ctr), 8.f));
    q = min(max(q, -255), 255);
    int g = (int)rintf(__fmul_rn(__fsub_rn(w[k], wa), 4.f));
    g = min(max(g, -31), 0);
    int j = (__float_as_int(sg[k]) - 0x3E000000) >> 20;
    j = min(max(j, 0), kNJ - 1);
    key |= (uint64_t)(q + 255) << (9 * k);
    key |= (uint64_t)j << (27 + 7 * k);
    key |= (uint64_t)(-g) << (48 + 5 * k);
  }
}

// F at the lane's four edges for key (q, j, g).
__device__ __forceinline__ void mix_edges(const int q[3], const int j[3], const int g[3],
                                          int lane, float F[4]) {
  float m[3], inv[3], om[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    m[k] = __fdiv_rn((float)q[k], 8.f);
    inv[k] = __fdiv_rn(1.f, __int_as_float(0x3E000000 + (j[k] << 20) + (1 << 19)));
    om[k] = exp32_spec(__fmul_rn((float)g[k], 0.25f));
  }
  const float W = __fadd_rn(__fadd_rn(om[0], om[1]), om[2]);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = 4 * lane + i;
    const float u = __fsub_rn((float)e, 62.5f);
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float z = __fmul_rn(__fsub_rn(u, m[k]), inv[k]);
      const float t = __fmul_rn(om[k], sigmoid32_spec(z));
      acc = k == 0 ? t : __fadd_rn(acc, t);
    }
    F[i] = (e < kNSym - 1) ? __fdiv_rn(acc, W) : 1.f;
  }
}

__device__ __forceinline__ void unpack_key(uint64_t key, int q[3], int j[3], int g[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    q[k] = (int)((key >> (9 * k)) & 511u) - 255;
    j[k] = (int)((key >> (27 + 7 * k)) & 127u);
    g[k] = -(int)((key >> (48 + 5 * k)) & 31u);
  }
}

// One table row: cdf[0..127] then the coarse entries cdf[0], cdf[8], ...,
// cdf[120] (kMixRow u16, 16-byte aligned rows).
__device__ __forceinline__ void write_row(uint16_t *row, const int f[4], int run, int lane) {
  if ((lane & 1) == 0) row[kNSym + 1 + (lane >> 1)] = (uint16_t)run;
  uint32_t v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int s = 4 * lane + i;
    v[i] = s == kNSym ? kM : (uint32_t)run;
    run += f[i];
  }
  reinterpret_cast<uint2 *>(row)[lane] = make_uint2(v[0] | (v[1] << 16), v[2] | (v[3] << 16));
}

// Stage kernel: tables of n keys given as (q, j, g) triples.
__global__ void k_mix_tables(const int32_t *__restrict__ key9, int64_t n,
                             uint16_t *__restrict__ rows) {
  const int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wi >= n) return;
  const int32_t *k9 = key9 + wi * 9;
  int q[3], j[3], g[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    q[k] = min(max(k9[k], -255), 255);
    j[k] = min(max(k9[3 + k], 0), kNJ - 1);
    g[k] = min(max(k9[6 + k], -31), 0);
  }
  float F[4];
  mix_edges(q, j, g, lane, F);
  int f[4];
  const int run = warp_cdf(F, lane, f);
  write_row(rows + wi * kMixRow, f, run, lane);
}

// Head, decision and table of every symbol of one coding step.
template <int NCH>
__global__ void __launch_bounds__(256) k_mix_head(MixHeadParams a) {
  const int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wi >= (int64_t)a.P * a.nk) return;
  const int p = (int)(wi / a.nk);
  const int qi = (int)(wi - (int64_t)p * a.nk);
  // step-order index -> position
  const int ae = step_phase(a.step, 0), ao = step_phase(a.step, 1);
  const int ne = row_count(a.W, ae), pair = ne + row_count(a.W, ao);
  const int y2 = qi / pair, rr = qi - y2 * pair;
  const int y = rr < ne ? 2 * y2 : 2 * y2 + 1;
  const int x = rr < ne ? ae + 4 * rr : ao + 4 * (rr - ne);
  const int64_t pix = ((int64_t)p * a.H + y) * a.W + x;
  const float *zr = a.z + pix * (NCH * 32);
  float zc[NCH];
#pragma unroll
  for (int t = 0; t < NCH; ++t) zc[t] = zr[lane + 32 * t];
  float h[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float v = 0.f;
#pragma unroll
    for (int t = 0; t < NCH; ++t) v = fmaf(__ldg(a.wh + k * NCH * 32 + lane + 32 * t), zc[t], v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    h[k] = __fadd_rn(v, __ldg(a.bh + k));
  }
  float sg[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float rho = h[6 + k];
    sg[k] = rho > 20.f ? rho : log1pf(expf(rho));
  }
  int ctr;
  uint64_t key;
  mix_decide(h, h + 3, sg, ctr, key);
  if (a.par && lane < 9) {
    float v = h[0];
#pragma unroll
    for (int k = 1; k < 9; ++k)
      if (lane == k) v = k >= 6 ? sg[k - 6] : h[k];
    a.par[pix * 9 + lane] = v;
  }
  if (lane == 0) a.ctr[wi] = ctr;
  int q[3], j[3], g[3];
  unpack_key(key, q, j, g);
  float F[4];
  mix_edges(q, j, g, lane, F);
  int f[4];
  const int run = warp_cdf(F, lane, f);
  if (a.rows) write_row(a.rows + wi * kMixRow, f, run, lane);
  if (a.cf) {
    // the symbol this position codes: r = y - ctr, escapes at both ends
    const int r = a.q[pix] - ctr;
    const int s = r < -kT ? 0 : (r > kT ? kNSym - 1 : r + kT + 1);
    if ((s >> 2) == lane) {
      int c = run;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i < (s & 3)) c += f[i];
      int fs = f[0];
#pragma unroll
      for (int i = 1; i < 4; ++i)
        if (i == (s & 3)) fs = f[i];
      a.cf[wi] = (uint32_t)c | ((uint32_t)fs << 16);
    }
  }
}

void launch_mix_tables(const int32_t *key9, int64_t n, uint16_t *rows, cudaStream_t st) {
  if (n <= 0) return;
  k_mix_tables<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(key9, n, rows);
}

void launch_mix_head(const MixHeadParams &a, cudaStream_t st) {
  const int64_t n = (int64_t)a.P * a.nk;
  if (n <= 0) return;
  const unsigned grid = (unsigned)((n + 7) / 8);
  switch (a.C) {
    case 32: k_mix_head<1><<<grid, 256, 0, st>>>(a); return;
    case 64: k_mix_head<2><<<grid, 256, 0, st>>>(a); return;
    case 128: k_mix_head<4><<<grid, 256, 0, st>>>(a); return;
    default:
      set_last_error("mixture head: unsupported channel count");
      launch_failed() = true;
  }
}

}  // namespace pw
