// Autoregressive context model of the LL subband (pWave++'s default, Section
// 3.2 and Table 1: the first subband is coded position by position with
// spatial context from LL itself only).
//
// Model (a reading of the text; the architecture is in a missing figure):
// a 5x5 mask-A convolution (taps strictly before the centre in raster order:
// 12 taps) 1 -> C, LeakyReLU, 1x1 C -> C, LeakyReLU, 1x1 C -> 2 giving the
// Laplace mean and softplus^-1 scale (in the integer-network class: the
// same layers in integer arithmetic, the head giving 16 mu and the scale
// bin directly). The decoder runs one warp per plane
// over the LL positions in raster order: the warp evaluates the model at the
// next position from symbols already decoded, lane 0 decodes that symbol
// from the plane's single-state rANS chunk and the warp moves on. The
// encoder evaluates the same device function at every position in parallel
// (all symbols known), so both sides derive bit-identical table indices.
#include <algorithm>

#include "codec.h"
#include "ll_ar.h"
#include "pw_internal.cuh"

namespace pw {

constexpr int kArTaps = 12;   // 5x5 mask A: rows 0-1 (10 taps) + row 2, cols 0-1

struct ArSmem {
  // weights (FP32): w5t[tap][C], b5[C], w1t[in][out], b1[C], wh[2][C], bh[2]
  float *w5t, *b5, *w1t, *b1, *wh, *bh, *f;
};

__device__ __forceinline__ int ar_tap_dy(int t) { return t < 10 ? t / 5 : 2; }
__device__ __forceinline__ int ar_tap_dx(int t) { return t < 10 ? t % 5 : t - 10; }

// Integer-network class helpers: the sums below are exact integers in FP32
// (|sum| < 2^24); requantisation by n bits rounds half up, LeakyReLU has
// slope 1/128 (floor division), activations are clamped to +-127.
__device__ __forceinline__ long long ar_rq(long long x, int n) {
  return n > 0 ? ((x + (1LL << (n - 1))) >> n) : (x << (-n));
}
__device__ __forceinline__ float ar_act_i(float v, int n) {
  long long x = (long long)v;
  x = x >= 0 ? x : (x >> 7);
  x = ar_rq(x, n);
  return (float)(x > 127 ? 127 : (x < -127 ? -127 : x));
}

// Parameters at (y, x) of one plane from its symbols s (int32 plane of
// h x w, read through `get`): the packed table index, and mu and sigma for
// the optional parameter outputs. Executed by a full warp; returns the same
// values in every lane. C in {32, 64, 128}: lane owns channels lane + 32 i.
template <int C, class Get>
__device__ __forceinline__ void ar_params(const ArSmem &S, const ArWeightsDev &wd, int h, int w,
                                          int y, int x, Get get, uint32_t &pk, float &mu,
                                          float &sg) {
  const int lane = threadIdx.x & 31;
  constexpr int NPL = C / 32;
  float nb[kArTaps];
#pragma unroll
  for (int t = 0; t < kArTaps; ++t) {
    const int yy = y + ar_tap_dy(t) - 2, xx = x + ar_tap_dx(t) - 2;
    int32_t v = (yy >= 0 && yy < h && xx >= 0 && xx < w) ? get(yy * w + xx) : 0;
    if (wd.iq) v = min(max(v, -127), 127);   // integer class input
    nb[t] = (float)v;
  }
  float f[NPL];
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int c = lane + 32 * i;
    float v = S.b5[c];
#pragma unroll
    for (int t = 0; t < kArTaps; ++t) v = fmaf(S.w5t[t * C + c], nb[t], v);
    v = wd.iq ? ar_act_i(v, wd.n5) : (v >= 0.f ? v : 0.01f * v);
    f[i] = v;
    S.f[(threadIdx.x >> 5) * C + c] = v;
  }
  __syncwarp();
  const float *fs = S.f + (threadIdx.x >> 5) * C;
  float hsum[NPL];
#pragma unroll
  for (int i = 0; i < NPL; ++i) hsum[i] = S.b1[lane + 32 * i];
  for (int j = 0; j < C; ++j) {
    const float fj = fs[j];
#pragma unroll
    for (int i = 0; i < NPL; ++i) hsum[i] = fmaf(S.w1t[j * C + lane + 32 * i], fj, hsum[i]);
  }
  float pm = 0.f, pr = 0.f;
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int c = lane + 32 * i;
    const float hv = wd.iq ? ar_act_i(hsum[i], wd.n1) : (hsum[i] >= 0.f ? hsum[i] : 0.01f * hsum[i]);
    pm = fmaf(S.wh[c], hv, pm);
    pr = fmaf(S.wh[C + c], hv, pr);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pm += __shfl_xor_sync(0xffffffffu, pm, o);
    pr += __shfl_xor_sync(0xffffffffu, pr, o);
  }
  __syncwarp();  // f is rewritten at the next position
  const float m = pm + S.bh[0], rho = pr + S.bh[1];
  if (wd.iq) {
    // integer head: t = 16 mu and the scale bin j directly
    long long t = ar_rq((long long)m, wd.n_mu);
    t = t > (1LL << 23) ? (1LL << 23) : (t < -(1LL << 23) ? -(1LL << 23) : t);
    long long j = ar_rq((long long)rho, wd.n_rho) + 24;
    j = j < 0 ? 0 : (j > kNJ - 1 ? kNJ - 1 : j);
    pk = ((uint32_t)(t + (1 << 23)) << 7) | (uint32_t)j;
    mu = (float)t * 0.0625f;
    sg = __int_as_float(0x3E000000 + ((int)j << 20) + (1 << 19));
  } else {
    pk = pack_index(m, rho);
    mu = m;
    sg = rho > 20.f ? rho : log1pf(expf(rho));
  }
  (void)f;
}

template <int C>
__device__ void ar_load_weights(const ArWeightsDev &wd, float *base, int nwarps, ArSmem &S) {
  S.w5t = base;
  S.b5 = S.w5t + kArTaps * C;
  S.w1t = S.b5 + C;
  S.b1 = S.w1t + C * C;
  S.wh = S.b1 + C;
  S.bh = S.wh + 2 * C;
  S.f = S.bh + 2;
  for (int e = threadIdx.x; e < kArTaps * C; e += blockDim.x) {
    const int t = e / C, c = e % C;
    S.w5t[e] = wd.w5[c * 25 + ar_tap_dy(t) * 5 + ar_tap_dx(t)];
  }
  for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
    const int j = e / C, c = e % C;  // w1 is [out][in]
    S.w1t[e] = wd.w1[c * C + j];
  }
  for (int e = threadIdx.x; e < C; e += blockDim.x) { S.b5[e] = wd.b5[e]; S.b1[e] = wd.b1[e]; }
  for (int e = threadIdx.x; e < 2 * C; e += blockDim.x) S.wh[e] = wd.wh[e];
  if (threadIdx.x < 2) S.bh[threadIdx.x] = wd.bh[threadIdx.x];
  (void)nwarps;
  __syncthreads();
}

size_t ar_smem_weights(int C, int nwarps) {
  return sizeof(float) * ((size_t)kArTaps * C + C + (size_t)C * C + C + 2 * C + 2 + (size_t)nwarps * C);
}

// Encoder side: one warp per position, all planes.
template <int C>
__global__ void k_ll_ar_params(const int32_t *__restrict__ Q, int P, int h, int w,
                               ArWeightsDev wd, uint32_t *__restrict__ idx, float *mu_out,
                               float *sg_out) {
  extern __shared__ float smem[];
  ArSmem S;
  ar_load_weights<C>(wd, smem, blockDim.x / 32, S);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int n = h * w;
  for (int e = warp; e < P * n; e += nw) {
    const int p = e / n, pos = e % n;
    const int32_t *sp = Q + (int64_t)p * n;
    uint32_t pk;
    float mu, sg;
    ar_params<C>(S, wd, h, w, pos / w, pos % w, [&](int i) { return sp[i]; }, pk, mu, sg);
    if ((threadIdx.x & 31) == 0) {
      idx[(int64_t)p * n + pos] = pk;
      if (mu_out) {
        mu_out[(int64_t)p * n + pos] = mu;
        sg_out[(int64_t)p * n + pos] = sg;
      }
    }
  }
}

__device__ __forceinline__ int find_sym(const uint16_t *__restrict__ t, uint32_t slot) {
  int lo = 0, hi = kNSym;
#pragma unroll
  for (int it = 0; it < 7; ++it) {
    const int mid = (lo + hi) >> 1;
    if (mid > lo) {
      if ((uint32_t)__ldg(t + mid) <= slot) lo = mid; else hi = mid;
    }
  }
  return lo;
}

// Decoder: one warp per plane (one warp per CTA); the plane's symbols live
// in shared memory while it is decoded. Ragged batches (ext): plane p's LL
// is (ext[p].x >> esh) x (ext[p].y >> esh), written into the canvas's
// h x w plane.
template <int C>
__global__ void k_ll_ar_decode(const DecChunk *__restrict__ chunks, int P, int h, int w,
                               ArWeightsDev wd, const uint16_t *__restrict__ bank,
                               int32_t *__restrict__ Q, uint32_t *status,
                               const int2 *__restrict__ ext, int esh) {
  extern __shared__ float smem[];
  ArSmem S;
  ar_load_weights<C>(wd, smem, 1, S);
  int32_t *s_sym = reinterpret_cast<int32_t *>(S.f + C);
  const int p = blockIdx.x;
  if (p >= P) return;
  const int lane = threadIdx.x & 31;
  const DecChunk ch = chunks[p];
  const int hv = ext ? min(ext[p].x >> esh, h) : h, wv = ext ? min(ext[p].y >> esh, w) : w;
  const int n = hv * wv;
  bool bad = ch.lanes != 1 || ch.count != (uint32_t)n || ch.nbytes < 4 || ((ch.nbytes - 4) & 1);
  uint32_t x = kRansL, ptr = 0, nwords = 0;
  const uint8_t *wp = ch.data + 4;
  if (!bad) {
    nwords = (ch.nbytes - 4) >> 1;
    x = (uint32_t)ch.data[0] | ((uint32_t)ch.data[1] << 8) | ((uint32_t)ch.data[2] << 16) |
        ((uint32_t)ch.data[3] << 24);
  }
  auto word = [&](uint32_t &st) {
    if (ptr < nwords) {
      st = (st << 16) | (uint32_t)wp[2 * ptr] | ((uint32_t)wp[2 * ptr + 1] << 8);
      ++ptr;
    } else {
      bad = true;
    }
  };
  for (int pos = 0; pos < n; ++pos) {
    if (__shfl_sync(0xffffffffu, bad ? 1 : 0, 0)) break;
    uint32_t pk;
    float mu, sg;
    ar_params<C>(S, wd, hv, wv, pos / wv, pos % wv, [&](int i) { return s_sym[i]; }, pk, mu,
                 sg);
    if (lane == 0) {
      int ctr, tid;
      unpack_index(pk, ctr, tid);
      const uint16_t *t = bank + (size_t)tid * (kNSym + 1);
      uint32_t slot = x & (kM - 1);
      const int s = find_sym(t, slot);
      const uint32_t c0 = __ldg(t + s), c1 = __ldg(t + s + 1);
      x = (c1 - c0) * (x >> kLogM) + slot - c0;
      if (x < kRansL) word(x);
      int r = s - kT - 1;
      if (s == 0 || s == kNSym - 1) {
        // Exp-Golomb-0 excess in bypass bits: k ones, a zero, k bits
        int k = 0;
        uint32_t v = 1;
        bool phase1 = false;
        for (int guard = 0; guard < 2 * kMaxEscBits + 2 && !bad; ++guard) {
          slot = x & (kM - 1);
          const uint32_t bit = slot >> (kLogM - 1);
          x = (kM >> 1) * (x >> kLogM) + (slot & ((kM >> 1) - 1));
          if (x < kRansL) word(x);
          if (!phase1) {
            if (bit) { if (++k > kMaxEscBits) bad = true; }
            else { phase1 = true; if (k == 0) break; }
          } else {
            v = (v << 1) | bit;
            if (--k == 0) break;
          }
        }
        const int e = (int)(v - 1);
        r = (s == 0) ? -(e + kT + 1) : e + kT + 1;
      }
      s_sym[pos] = ctr + r;
    }
    __syncwarp();
  }
  if (lane == 0 && (x != kRansL || ptr != nwords)) bad = true;
  for (int i = lane; i < n; i += 32) Q[(int64_t)p * h * w + (int64_t)(i / wv) * w + i % wv] = s_sym[i];
  if (lane == 0 && bad) atomicOr(status, kStCorrupt);
}

int launch_ll_ar_params(const int32_t *Q, int P, int h, int w, int C, const ArWeightsDev &wd,
                        uint32_t *idx, float *mu, float *sg, cudaStream_t st) {
  const int warps = 8;
  const size_t sm = ar_smem_weights(C, warps);
  const int64_t need = (int64_t)P * h * w;
  int blocks = (int)std::min<int64_t>((need + warps - 1) / warps, 152 * 8);
#define PW_AR(C_)                                                                           \
  if (C == C_) {                                                                            \
    cudaFuncSetAttribute(k_ll_ar_params<C_>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                         (int)sm);                                                          \
    k_ll_ar_params<C_><<<blocks, 32 * warps, sm, st>>>(Q, P, h, w, wd, idx, mu, sg);        \
    return PW_OK;                                                                           \
  }
  PW_AR(32) PW_AR(64) PW_AR(128)
#undef PW_AR
  return PW_EUNSUPPORTED;
}

int launch_ll_ar_decode(const DecChunk *chunks, int P, int h, int w, int C, const ArWeightsDev &wd,
                        const uint16_t *bank, int32_t *Q, uint32_t *status, cudaStream_t st,
                        const int2 *ext, int esh) {
  const size_t sm = ar_smem_weights(C, 1) + (size_t)h * w * sizeof(int32_t);
  if (sm > 227 * 1024) {
    set_last_error("autoregressive LL subband too large for one CTA");
    return PW_EUNSUPPORTED;
  }
#define PW_AR(C_)                                                                           \
  if (C == C_) {                                                                            \
    cudaFuncSetAttribute(k_ll_ar_decode<C_>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                         (int)sm);                                                          \
    k_ll_ar_decode<C_><<<P, 32, sm, st>>>(chunks, P, h, w, wd, bank, Q, status, ext, esh);  \
    return PW_OK;                                                                           \
  }
  PW_AR(32) PW_AR(64) PW_AR(128)
#undef PW_AR
  return PW_EUNSUPPORTED;
}

}  // namespace pw
