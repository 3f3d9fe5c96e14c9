// Context model of pWave++ (Section 3.2, Figs. 3-5) on FP32 SIMT cores: the
// plain FP32 path. Activations are NHWC float tensors [P, H, W, C] (P =
// planes: images x colour components). Every kernel here computes each
// output from a fixed sequence of FP32 operations, so results do not depend
// on batch composition or launch order (encoder and decoder agree bit for bit).
//
// Layers (a reading of the text; the paper's figures are not available):
//  ConvLSTM: e = conv3x3(1->C)(up(s_prev)), [i f o g] = conv3x3(2C->4C)([e, up(h)]),
//            c = sig(f) up(c) + sig(i) tanh(g), h = sig(o) tanh(c), l = h.
//  step 1:   z = 1x1(l); z += 1x1(dw3x3(lrelu(1x1 z))); z += 1x1(lrelu(1x1(2C) z));
//            (mu, rho) = 1x1(C->2) z.
//  steps 2-4: a = conv3x3(1->C)(m_<k s); z = 1x1(2C->C)[a, l];
//            z += conv3x3(lrelu(conv3x3 z)); (mu, rho) = 1x1(C->2) z.
// The integer-network class runs the same kernels on integers held exactly
// in floats, with integer epilogues (requantisation, clamps, LeakyReLU
// slope 1/128, hard sigmoid / tanh cell, log-scale head): see rq_ll below.
#include "pw_internal.cuh"
#include "ctx_kernels.cuh"
#include "f32x2.cuh"

namespace pw {

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }
__device__ __forceinline__ float lrelu(float x) { return x >= 0.f ? x : 0.01f * x; }

// Integer-network class. Every sum is of integers below 2^24 in magnitude
// (at most 2304 products of weights |w| <= 56 and activations |a| <= 127,
// plus a bias |b| <= 2^18), so FP32 FMAs compute it exactly in any order;
// these helpers then work on the exact integer: requantisation by n bits
// (round half up: floor((x + 2^(n-1)) / 2^n); n <= 0 shifts left),
// clamping, LeakyReLU with slope 1/128 (floor division), hard sigmoid
// clamp(2x + 64, 0, 128) and hard tanh clamp(8x, -128, 128) (7 fractional
// bits).
__device__ __forceinline__ long long rq_ll(long long x, int n) {
  return n > 0 ? ((x + (1LL << (n - 1))) >> n) : (x << (-n));
}
__device__ __forceinline__ long long clamp_ll(long long x, long long lim) {
  return x > lim ? lim : (x < -lim ? -lim : x);
}
__device__ __forceinline__ float rq_f(float v, int n, long long lim) {
  return (float)clamp_ll(rq_ll((long long)v, n), lim);
}
__device__ __forceinline__ float lrelu_i(float v) {
  const long long x = (long long)v;
  return (float)(x >= 0 ? x : (x >> 7));
}
__device__ __forceinline__ long long hsig_i(long long x) {
  return x * 2 + 64 < 0 ? 0 : (x * 2 + 64 > 128 ? 128 : x * 2 + 64);
}
__device__ __forceinline__ long long htanh_i(long long x) { return clamp_ll(8 * x, 128); }

// Generic NHWC convolution, KS x KS (KS = 1 or 3, zero padding), output
// channels [blockIdx.y * CO_T, +CO_T). Tile: 8 rows x 16 columns of one
// plane (blockIdx.z); 256 threads, each 4 consecutive pixels x CO_T/8
// channels. Weights are [KS*KS][cin][cout_total].
template <int KS, int CO_T, int EPI>
__global__ void __launch_bounds__(256) k_conv_simt(ConvParams a) {
  constexpr int TH = 8, TW = 16, CI = (CO_T >= 128 ? 4 : 8), R = KS / 2;
  constexpr int HH = TH + KS - 1, HW = TW + KS - 1;
  constexpr int NC = CO_T / 8;
  // input tile, one plane per channel; the plane stride avoids shared-memory
  // bank conflicts of the channel-fastest fill below
  constexpr int PS = HH * HW + ((HH * HW) % 32 == 0 ? 4 : 0);
  __shared__ float s_in[CI * PS];
  __shared__ __align__(16) float s_w[KS * KS][CI][CO_T];
  __shared__ float s_head[EPI == EPI_HEAD ? 8 : 1][TH * TW][2];

  const int t = threadIdx.x;
  const int pg = t & 31, cg = t >> 5;
  const int prow = pg >> 2, pcol = (pg & 3) * 4;
  const int p = blockIdx.z;
  const int tiles_x = (a.W + TW - 1) / TW;
  const int y0 = (blockIdx.x / tiles_x) * TH, x0 = (blockIdx.x % tiles_x) * TW;
  const int co0 = blockIdx.y * CO_T;
  const float *inp = a.in + (int64_t)p * a.H * a.W * a.in_cs + a.in_co;

  // accumulators of output channels (2k, 2k + 1) of pixel i in one packed
  // FP32 pair: each element takes the same fused multiply-adds in the same
  // order as a scalar accumulator (bit-identical results, half the
  // instructions)
  uint64_t accp[4][NC / 2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < NC / 2; ++k) accp[i][k] = 0ull;

  for (int c0 = 0; c0 < a.cin; c0 += CI) {
    __syncthreads();
    // channel fastest: consecutive threads read a pixel's consecutive
    // channels (one 32-byte sector per pixel for CI = 8)
    for (int e = t; e < CI * HH * HW; e += 256) {
      const int c = e % CI, r = e / CI;
      const int yy = y0 + r / HW - R, xx = x0 + r % HW - R;
      float v = 0.f;
      if (c0 + c < a.cin && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
        v = inp[((int64_t)yy * a.W + xx) * a.in_cs + c0 + c];
      s_in[c * PS + r] = v;
    }
    for (int e = t; e < KS * KS * CI * CO_T; e += 256) {
      int tap = e / (CI * CO_T), r = e % (CI * CO_T);
      int c = r / CO_T, o = r % CO_T;
      float v = 0.f;
      if (c0 + c < a.cin && co0 + o < a.cout_total)
        v = a.w[((int64_t)tap * a.cin + c0 + c) * a.cout_total + co0 + o];
      s_w[tap][c][o] = v;
    }
    __syncthreads();
#pragma unroll
    for (int tap = 0; tap < KS * KS; ++tap) {
      const int dy = tap / KS, dx = tap % KS;
#pragma unroll
      for (int c = 0; c < CI; ++c) {
        float xv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xv[i] = s_in[c * PS + (prow + dy) * HW + pcol + i + dx];
        const uint64_t *wrow = reinterpret_cast<const uint64_t *>(&s_w[tap][c][cg * NC]);
        uint64_t wp[NC / 2];
#pragma unroll
        for (int k = 0; k < NC / 2; ++k) wp[k] = wrow[k];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint64_t xx = f2pack(xv[i], xv[i]);
#pragma unroll
          for (int k = 0; k < NC / 2; ++k) accp[i][k] = fma2(wp[k], xx, accp[i][k]);
        }
      }
    }
  }
  float acc[4][NC];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < NC / 2; ++k) f2unpack(accp[i][k], acc[i][2 * k], acc[i][2 * k + 1]);

  const int y = y0 + prow;
  if (EPI == EPI_STORE) {
    // four channels per 16-byte access (channel counts are multiples of
    // 32, channel offsets and row strides multiples of 4 floats)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int x = x0 + pcol + i;
      if (y >= a.H || x >= a.W) continue;
      const int64_t pix = ((int64_t)p * a.H + y) * a.W + x;
#pragma unroll
      for (int j = 0; j < NC; j += 4) {
        const int co = co0 + cg * NC + j;
        if (co >= a.cout_total) continue;
        const float4 bb = *reinterpret_cast<const float4 *>(a.b + co);
        float v[4] = {acc[i][j] + bb.x, acc[i][j + 1] + bb.y, acc[i][j + 2] + bb.z,
                      acc[i][j + 3] + bb.w};
        float r[4] = {0.f, 0.f, 0.f, 0.f};
        if (a.res) {
          const float4 rr = *reinterpret_cast<const float4 *>(a.res + pix * a.res_cs + a.res_co + co);
          r[0] = rr.x; r[1] = rr.y; r[2] = rr.z; r[3] = rr.w;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (a.iq) {
            // integer class: act on the accumulator, requantise, then the
            // residual (an activation at the same binary point)
            if (a.act) v[k] = lrelu_i(v[k]);
            v[k] = rq_f(v[k], a.rq, 127);
            if (a.res) v[k] = (float)clamp_ll((long long)v[k] + (long long)r[k], 127);
          } else {
            if (a.res) v[k] += r[k];
            if (a.act) v[k] = lrelu(v[k]);
          }
        }
        *reinterpret_cast<float4 *>(a.out + pix * a.out_cs + a.out_co + co) =
            make_float4(v[0], v[1], v[2], v[3]);
      }
    }
  } else if (EPI == EPI_LSTM) {
    // output channel o = 4 * ch + gate (gate order i, f, o, g)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int x = x0 + pcol + i;
      if (y >= a.H || x >= a.W) continue;
      const int64_t pix = ((int64_t)p * a.H + y) * a.W + x;
      const int Hp = a.H >> a.up, Wp = a.W >> a.up;
      const int64_t ppix = ((int64_t)p * Hp + (y >> a.up)) * Wp + (x >> a.up);
#pragma unroll
      for (int j = 0; j < NC; j += 4) {
        const int o = co0 + cg * NC + j;
        const int ch = o >> 2;
        float gi = acc[i][j] + a.b[o], gf = acc[i][j + 1] + a.b[o + 1];
        float go = acc[i][j + 2] + a.b[o + 2], gg = acc[i][j + 3] + a.b[o + 3];
        float cp = a.first ? 0.f : a.c_prev[ppix * a.C + ch];
        if (a.iq) {
          // integer cell: gates requantised to 4 fractional bits, hard
          // sigmoid / tanh, c and h with 7
          const long long si = hsig_i((long long)rq_f(gi, a.rq, 127));
          const long long sf = hsig_i((long long)rq_f(gf, a.rq, 127));
          const long long so = hsig_i((long long)rq_f(go, a.rq, 127));
          const long long tg = htanh_i((long long)rq_f(gg, a.rq, 127));
          const long long c = clamp_ll(rq_ll(sf * (long long)cp + si * tg, 7), 32767);
          const long long hq = clamp_ll(rq_ll(so * clamp_ll(c, 128), 7), 127);
          a.c_new[pix * a.C + ch] = (float)c;
          a.out[pix * a.out_cs + a.out_co + ch] = (float)hq;
          continue;
        }
        float cn = sigm(gf) * cp + sigm(gi) * tanhf(gg);
        float hn = sigm(go) * tanhf(cn);
        a.c_new[pix * a.C + ch] = cn;
        a.out[pix * a.out_cs + a.out_co + ch] = hn;
      }
    }
  } else {  // EPI_HEAD: z' = res + acc + b over all C channels, then 1x1(C->2)
    float pm[4], pr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { pm[i] = 0.f; pr[i] = 0.f; }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int x = x0 + pcol + i;
      const bool in = y < a.H && x < a.W;
      const int64_t pix = ((int64_t)p * a.H + min(y, a.H - 1)) * a.W + min(x, a.W - 1);
      float rv[NC];
#pragma unroll
      for (int j = 0; j < NC; j += 4) {  // the residual, 16 bytes at a time
        float4 r4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (in) r4 = *reinterpret_cast<const float4 *>(a.res + pix * a.res_cs + a.res_co + cg * NC + j);
        rv[j] = r4.x; rv[j + 1] = r4.y; rv[j + 2] = r4.z; rv[j + 3] = r4.w;
      }
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int co = cg * NC + j;
        float v = acc[i][j] + a.b[co];
        if (a.iq) {
          v = rq_f(v, a.rq, 127);
          if (in) v = (float)clamp_ll((long long)v + (long long)rv[j], 127);
        } else if (in) {
          v += rv[j];
        }
        pm[i] = fmaf(a.wh[co], v, pm[i]);
        pr[i] = fmaf(a.wh[a.cout_total + co], v, pr[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      s_head[cg][prow * TW + pcol + i][0] = pm[i];
      s_head[cg][prow * TW + pcol + i][1] = pr[i];
    }
    __syncthreads();
    if (t < TH * TW) {
      const int yy = y0 + t / TW, xx = x0 + t % TW;
      if (yy < a.H && xx < a.W && step_of(yy, xx) == a.step) {
        float mu = a.bh[0], rho = a.bh[1];
#pragma unroll
        for (int g = 0; g < 8; ++g) { mu += s_head[g][t][0]; rho += s_head[g][t][1]; }
        const int q = step_index(a.W, a.step, yy, xx);
        if (a.iq) {
          // integer head: t = 16 mu and the scale bin j directly
          const long long ti = clamp_ll(rq_ll((long long)mu, a.rq_mu), 1LL << 23);
          long long j = rq_ll((long long)rho, a.rq_rho) + 24;
          j = j < 0 ? 0 : (j > kNJ - 1 ? kNJ - 1 : j);
          a.idx[(int64_t)p * a.idx_stride + q] =
              ((uint32_t)(ti + (1 << 23)) << 7) | (uint32_t)j;
          if (a.mu_out) {
            const int64_t o = (int64_t)p * a.H * a.W + (int64_t)yy * a.W + xx;
            a.mu_out[o] = (float)ti * 0.0625f;
            a.sg_out[o] = __int_as_float(0x3E000000 + ((int)j << 20) + (1 << 19));
          }
        } else {
          a.idx[(int64_t)p * a.idx_stride + q] = pack_index(mu, rho);
          if (a.mu_out) {
            const int64_t o = (int64_t)p * a.H * a.W + (int64_t)yy * a.W + xx;
            a.mu_out[o] = mu;
            a.sg_out[o] = rho > 20.f ? rho : log1pf(expf(rho));
          }
        }
      }
    }
  }
}

// ConvLSTM input: X[..., 0:C] = conv3x3(1->C)(up(s_prev)) + be,
// X[..., C:2C] = up(h_prev) (zero for the first LSTM step).
__global__ void k_lstm_in(const int32_t *__restrict__ s_prev, const float *__restrict__ h_prev,
                          int h_cs, int h_co, const float *__restrict__ we,
                          const float *__restrict__ be, float *__restrict__ X, int P, int H,
                          int W, int C, int up, int first, int rqn) {
  const int64_t n = (int64_t)P * H * W * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int64_t pix = e / C;
    const int x = (int)(pix % W);
    const int y = (int)((pix / W) % H);
    const int p = (int)(pix / ((int64_t)W * H));
    const int Hp = H >> up, Wp = W >> up;
    const int32_t *sp = s_prev + (int64_t)p * Hp * Wp;
    float v = be[c];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
      int32_t sv = sp[(int64_t)(yy >> up) * Wp + (xx >> up)];
      if (rqn != kRqFloat) sv = min(max(sv, -127), 127);   // integer class input
      v = fmaf(we[c * 9 + tap], (float)sv, v);
    }
    X[pix * 2 * C + c] = rqn != kRqFloat ? rq_f(v, rqn, 127) : v;
    float hv = 0.f;
    if (!first) {
      const int64_t pp = ((int64_t)p * Hp + (y >> up)) * Wp + (x >> up);
      hv = h_prev[pp * h_cs + h_co + c];
    }
    X[pix * 2 * C + C + c] = hv;
  }
}

// Masked spatial input of steps 2-4: out[..., 0:C] = conv3x3(1->C)(m_<k s) + b.
__global__ void k_masked_in(const int32_t *__restrict__ s, const float *__restrict__ wa,
                            const float *__restrict__ ba, float *__restrict__ out, int out_cs,
                            int P, int H, int W, int C, int step, int rqn) {
  const int64_t n = (int64_t)P * H * W * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int64_t pix = e / C;
    const int x = (int)(pix % W);
    const int y = (int)((pix / W) % H);
    const int p = (int)(pix / ((int64_t)W * H));
    const int32_t *sp = s + (int64_t)p * H * W;
    float v = ba[c];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
      if (step_of(yy, xx) >= step) continue;
      int32_t sv = sp[(int64_t)yy * W + xx];
      if (rqn != kRqFloat) sv = min(max(sv, -127), 127);   // integer class input
      v = fmaf(wa[c * 9 + tap], (float)sv, v);
    }
    out[pix * out_cs + c] = rqn != kRqFloat ? rq_f(v, rqn, 127) : v;
  }
}

// Depthwise 3x3 (zero padding): out = dw(in) + b, NHWC with C channels.
__global__ void k_dw3x3(const float *__restrict__ in, const float *__restrict__ w,
                        const float *__restrict__ b, float *__restrict__ out, int P, int H,
                        int W, int C, int rqn) {
  const int64_t n = (int64_t)P * H * W * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int64_t pix = e / C;
    const int x = (int)(pix % W);
    const int y = (int)((pix / W) % H);
    const int64_t pbase = pix - ((int64_t)y * W + x);
    float v = b[c];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
      v = fmaf(w[c * 9 + tap], in[(pbase + (int64_t)yy * W + xx) * C + c], v);
    }
    out[pix * C + c] = rqn != kRqFloat ? rq_f(v, rqn, 127) : v;
  }
}

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 152 * 64 ? 152 * 64 : (g < 1 ? 1 : g));
}

bool &launch_failed() {
  static thread_local bool f = false;
  return f;
}

void launch_conv_simt(int ks, const ConvParams &a, int epi, cudaStream_t st) {
  const int tiles = ((a.H + 7) / 8) * ((a.W + 15) / 16);
  int co_t = a.cout_total >= 64 ? 64 : 32;
  if (epi == EPI_HEAD) co_t = a.cout_total;
  dim3 grid(tiles, (a.cout_total + co_t - 1) / co_t, a.P);
#define PW_CONV_CASE(KS_, CO_, EPI_)                                         \
  if (ks == KS_ && co_t == CO_ && epi == EPI_) {                             \
    k_conv_simt<KS_, CO_, EPI_><<<grid, 256, 0, st>>>(a);                    \
    return;                                                                  \
  }
  PW_CONV_CASE(1, 32, EPI_STORE) PW_CONV_CASE(1, 64, EPI_STORE)
  PW_CONV_CASE(3, 32, EPI_STORE) PW_CONV_CASE(3, 64, EPI_STORE)
  PW_CONV_CASE(3, 32, EPI_LSTM) PW_CONV_CASE(3, 64, EPI_LSTM)
  PW_CONV_CASE(1, 32, EPI_HEAD) PW_CONV_CASE(1, 64, EPI_HEAD) PW_CONV_CASE(1, 128, EPI_HEAD)
  PW_CONV_CASE(3, 32, EPI_HEAD) PW_CONV_CASE(3, 64, EPI_HEAD) PW_CONV_CASE(3, 128, EPI_HEAD)
#undef PW_CONV_CASE
  set_last_error("no convolution kernel for this shape");
  launch_failed() = true;
}

void launch_lstm_in(const int32_t *s_prev, const float *h_prev, int h_cs, int h_co,
                    const float *we, const float *be, float *X, int P, int H, int W, int C,
                    int up, int first, cudaStream_t st, int rqn) {
  int64_t n = (int64_t)P * H * W * C;
  k_lstm_in<<<grid_for(n), 256, 0, st>>>(s_prev, h_prev, h_cs, h_co, we, be, X, P, H, W, C,
                                          up, first, rqn);
}
void launch_masked_in(const int32_t *s, const float *wa, const float *ba, float *out,
                      int out_cs, int P, int H, int W, int C, int step, cudaStream_t st,
                      int rqn) {
  int64_t n = (int64_t)P * H * W * C;
  k_masked_in<<<grid_for(n), 256, 0, st>>>(s, wa, ba, out, out_cs, P, H, W, C, step, rqn);
}
void launch_dw3x3(const float *in, const float *w, const float *b, float *out, int P, int H,
                  int W, int C, cudaStream_t st, int rqn) {
  int64_t n = (int64_t)P * H * W * C;
  k_dw3x3<<<grid_for(n), 256, 0, st>>>(in, w, b, out, P, H, W, C, rqn);
}

}  // namespace pw
