// Context model of pWave++ (Section 3.2) on the 5th-generation tensor cores:
// BF16 implicit-GEMM convolutions with tcgen05.mma, FP32 accumulators in
// tensor memory, operand tiles brought in by TMA, fused epilogues.
//
// Activations are BF16 in a channel-group-blocked layout [P][G][H][W][8]
// (G = channels / 8), so that a TMA box ((tile width + halo) x 8 channels,
// tile height + halo, groups) lands in shared memory as one slab of 16-byte
// pixel rows per channel group: exactly the no-swizzle K-major core-matrix
// layout of the MMA A operand. A 3x3 tap is then just a shifted start address into
// the halo tile, so every input pixel is loaded once per K-block.
//
// GEMM view: M = 128 output pixels (16 rows x 8 columns of one plane),
// N = output channels of the CTA (32, 64 or 128), K = taps x input channels,
// processed in K-blocks of 64 (32) channels. Weights of the CTA's N block
// stay resident in shared memory for the whole persistent kernel.
// Warp roles: warp 0 = TMA producer, warp 1 = MMA issuer (and TMEM owner),
// warps 2-5 = epilogue (one TMEM lane quadrant each). Accumulators are
// double-buffered in TMEM so the epilogue of one tile overlaps the MMAs of
// the next. Every wait is bounded: on expiry the kernel sets an error flag,
// lets in-flight copies land, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <cmath>
#include <cstring>
#include <mutex>

#include "ctx_tc.h"
#include "prof.h"
#include "tc_ptx.cuh"
#include "f32x2.cuh"

namespace pw {

struct TcWeights {
  // per conv: packed BF16 weights [nb][kblock][tap][kb/8][ncta][8] + FP32 bias
  struct Conv {
    __nv_bfloat16 *w = nullptr;   // BF16 weights, or (f8) E4M3 bytes in the same order
    float *b = nullptr;
    float *sw = nullptr;          // f8: per-output-column scale of the accumulator
    // ConvLSTM gates: BF16 weights of the v block (K-block 0, see
    // TcConvArgs::wtv); w then holds the h block only (cin = C)
    __nv_bfloat16 *wv = nullptr;
    int cin = 0, cout = 0, ks = 1, kb = 64, ncta = 64, nb = 1;
    bool f8 = false;
  };
  Conv gates;
  Conv s0_in, s0_w1, s0_w2, s0_w3, s0_w4;        // sb set, step 0
  // step 1: in_ = 1x1 z = Win l + bin (run on the step-1 positions only),
  // w1 = the composite 1x1 W1 Win, W1 bin + b1 (u = lrelu(w1 l), there is no
  // nonlinearity between the two 1x1 layers)
  Conv sk_c1[3], sk_c2[3];                      // sb set, steps 1..3
  Conv l0_in, l0_w1, l0_w2, l0_w3, l0_w4;       // ll set
  Conv lk_c1[3], lk_c2[3];
  // steps 2-4 with the masked input conv folded into the 1x1: zt = 1x1 over
  // [T (v block: the 9 masked neighbour values as BF16, zero padding),
  // l (C channels)]; the bias includes the folded bias
  Conv sk_zt[3], lk_zt[3];
  // FP8 precision: E4M3 copies of the 3x3 convolutions (gates, steps 2-4
  // residual blocks) with the input channels' static scales folded in, and
  // the scales (value * scale = stored E4M3 value) of the FP8 activations:
  // z (residual-block input, per step), u (hidden layer, per step) and h
  // (l_i, fixed 256 since |h| < 1); the gates' v block stays BF16
  bool has_f8 = false;
  Conv gates8, sk_c1_8[3], sk_c2_8[3], lk_c1_8[3], lk_c2_8[3];
  float *h_scale = nullptr;
  float *sk_z_scale[3] = {}, *sk_u_scale[3] = {}, *lk_z_scale[3] = {}, *lk_u_scale[3] = {};
  std::vector<void *> allocs;
};

struct TcAct {  // BF16 activations in [P][G][H][W][8]
  // X: (2C; channels C..2C-1 hold up(h) when h_{i-1} is at another
  // resolution); L[2]: long-term context l_i of the
  // current and previous subband (C each, ping-pong so the gates conv can
  // read h_{i-1} while its epilogue writes h_i); Z, V, Z2 (C); U (2C).
  __nv_bfloat16 *X = nullptr, *L[2] = {nullptr, nullptr}, *Z = nullptr, *U = nullptr,
                *V = nullptr, *Z2 = nullptr;
  // Step-1 tail on the step-1 positions only, in the compact layout
  // [P][G][ceil(h/2)][n_even + n_odd][8] (row pair, index within the pair):
  // Vc = dw3x3 output, Zc = block input (residual), Z2c = block output (C
  // each), U2c = feed-forward hidden layer (2C).
  __nv_bfloat16 *Vc = nullptr, *Zc = nullptr, *Z2c = nullptr, *U2c = nullptr;
  // V16: the ConvLSTM gates' v block [P][2][H][W][8] (9 neighbour values of
  // the upsampled previous subband, an inside indicator, zeros)
  __nv_bfloat16 *V16 = nullptr;
  // T: masked neighbour values of steps 2-4 (16 channels, see TcWeights)
  __nv_bfloat16 *T = nullptr;
  // FP8 precision: E4M3 activations [P][G16][H][W][16]: X8 (2C; channels
  // C..2C-1 hold up(h) when h_{i-1} is at another resolution), L8[2] = l_i
  // (C, ping-pong like L), Z8 / U8 = residual-block input and hidden layer (C)
  uint8_t *X8 = nullptr, *L8[2] = {nullptr, nullptr}, *Z8 = nullptr, *U8 = nullptr;
  int *err = nullptr;
  void *base = nullptr;
};

__device__ __forceinline__ float sigm_f(float x) { return 1.f / (1.f + __expf(-x)); }
__device__ __forceinline__ float sigm_fast(float x) { return fmaf(0.5f, tanh_fast(0.5f * x), 0.5f); }
__device__ __forceinline__ float lrelu_f(float x) { return x >= 0.f ? x : 0.01f * x; }

// ---------------------------------------------------------------------------
// TE_HEADC: the residual + head 3x3 conv of steps 2-4 evaluated at the
// step's own positions only (see the compact head below). TE_STOREV: a plain
// store whose K-block 0 is a BF16 v block (the steps 2-4 z conv); TE_LSTM
// always has one too. Convs without a v block compile without its code.
enum { TE_STORE = 0, TE_LSTM = 1, TE_HEAD = 2, TE_HEADC = 3, TE_STOREV = 4 };

struct TcConvArgs {
  int P, H, W;
  int ks, cin, kb, nkb, in_goff;
  int ncta, nb;
  int tiles_x, tiles_y, tiles;  // tiles per N block
  int step_dx, step_dy, step_dp;  // the CTA stride in (tiles_x, tiles_y) digits
  int pairs;                      // MMA issue of two tiles per round (see the issuer)
  int stages, halo_x, halo_y;
  uint32_t stage_bytes, w_bytes;
  const __nv_bfloat16 *wt;      // [nb][kblock][tap][kb/8][ncta][8]
  // K-block 0 may be a 16-channel BF16 "v" block with its own weights wtv
  // [nb][tap][2][ncta][8] (wv_bytes per N block), read through the first
  // tensor map (vstage_bytes), either into the first K-block's stage after
  // its hstage_bytes of the other input (one barrier and one commit for
  // both) or, when hstage_bytes is 0, as K-block 0 in a stage of its own:
  // for the ConvLSTM gates the 9
  // neighbour values of the upsampled previous subband and an inside
  // indicator (in place of e), for the steps 2-4 z conv the 9 masked
  // neighbour values; wt then holds the remaining K-blocks
  const __nv_bfloat16 *wtv;
  uint32_t wv_bytes, vstage_bytes, hstage_bytes;
  const float *bias;            // [nb * ncta]
  int epi, act;
  __nv_bfloat16 *out;
  int out_G, out_goff;
  const __nv_bfloat16 *res;
  int res_G, res_goff;
  // ConvLSTM cell state, BF16 [P][H][W][C] (previous subband's resolution
  // for c_prev)
  const __nv_bfloat16 *c_prev;
  __nv_bfloat16 *c_new;
  int up, first, C;
  const float *wh, *bh;
  int step;
  uint32_t *idx;
  int64_t idx_stride;
  float *mu_out, *sg_out;
  int nkb0;                     // K-blocks read through the first tensor map
  int in1_goff;                 // group offset of the second tensor map
  // TE_HEAD on a compact step layout (H x W = row pairs x positions per
  // pair): compact_n = number of step positions (0: full-plane layout),
  // full_W = width of the subband (for the mu / sigma planes)
  int compact_n, full_W, full_H;
  // step-compact BF16 copy of a plain store's output: the positions of step
  // `step` only, [P][G][n][8] in step order (outc_n = n positions per plane);
  // a head reads its residual from such a copy when res_compact_n > 0
  __nv_bfloat16 *outc;
  int outc_n, res_compact_n;
  // FP8 (E4M3) operands: per-output-column scale applied to the accumulator
  // (acc * w_scale[n] + bias[n]); optional second output in FP8, blocked
  // [P][G16][H][W][16], value = output * out8_scale[channel]
  const float *w_scale;
  uint8_t *out8;
  int out8_G16;
  const float *out8_scale;
  // out / out8 in the compact head's input layout when set: pixel-major and
  // split by column phase, [P][H][4][W4 / 4][channels] (x = 4 j + phase,
  // W4 = W rounded up to a multiple of 4; columns W .. W4 - 1 are written
  // with zeros)
  int out_ps;
  // TE_HEADC: tile = cR rows of one parity x cJ step positions per row
  // (cR * cJ = 128, cJ = 1 << cJlog); tps = taps per pipeline stage (1, 3
  // or 9)
  int cR, cJ, cJlog, tps;
  int *err;
};

constexpr int kTileH = 16, kTileW = 8;

// Tile coordinates of a persistent CTA's tiles t = t0, t0 + step, ...:
// (tx, ty, p) advanced like an odometer by the step's digits (dx, dy, dp)
// in the (tiles_x, tiles_y) radix, which the host precomputes, so the loop
// needs no division and holds three registers.
struct TileIter {
  int tx, ty, p;
  __device__ __forceinline__ TileIter(int t0, int tiles_x, int tiles_y) {
    tx = t0 % tiles_x; ty = (t0 / tiles_x) % tiles_y; p = t0 / (tiles_x * tiles_y);
  }
  __device__ __forceinline__ void next(int dx, int dy, int dp, int nx, int ny) {
    tx += dx;
    int cy = 0;
    if (tx >= nx) { tx -= nx; cy = 1; }
    ty += dy + cy;
    int cp = 0;
    if (ty >= ny) { ty -= ny; cp = 1; }
    p += dp + cp;
  }
};

__device__ __forceinline__ void store_bf16x8(__nv_bfloat16 *p, const float *v) {
  uint4 u;
  __nv_bfloat162 t0 = __floats2bfloat162_rn(v[0], v[1]), t1 = __floats2bfloat162_rn(v[2], v[3]),
                 t2 = __floats2bfloat162_rn(v[4], v[5]), t3 = __floats2bfloat162_rn(v[6], v[7]);
  u.x = *reinterpret_cast<uint32_t *>(&t0);
  u.y = *reinterpret_cast<uint32_t *>(&t1);
  u.z = *reinterpret_cast<uint32_t *>(&t2);
  u.w = *reinterpret_cast<uint32_t *>(&t3);
  *reinterpret_cast<uint4 *>(p) = u;
}
__device__ __forceinline__ void load_bf16x8(const __nv_bfloat16 *p, float *v) {
  uint4 u = *reinterpret_cast<const uint4 *>(p);
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 f = __bfloat1622float2(h[i]);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

// 16 floats -> 16 E4M3 bytes (round to nearest, saturating), one 16-byte store
__device__ __forceinline__ void store_fp8x16(uint8_t *p, const float *v) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i], v[4 * i + 1]),
                                                 __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i + 2], v[4 * i + 3]),
                                                 __NV_SATFINITE, __NV_E4M3);
    w[i] = lo | (hi << 16);
  }
  *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void mma_fp8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// pipeline stages at most (the barrier arrays below hold this many)
constexpr int kMaxStages = 24;

// shared memory: barriers [0, 1024), epilogue constants [1024, 4096)
// (5 x NCTA floats), head partial sums [4096, 8192), then the resident
// weights and the stages
constexpr int kConvHeader = 8192;

// Epilogue warps: 16 (four per TMEM lane quadrant, 16 columns each) for the
// 1x1 plain stores of 64 columns, whose short epilogue is latency-bound
// (measured: 1x1 class 9.04 -> 8.53 ms per batch of 24; the 3x3 stores lost
// as much, their MMA and load warps need the issue slots), else 8 (two per
// quadrant, NCTA / 2 columns each).
__host__ __device__ constexpr int conv_epi_warps(int ks, int epi, int ncta) {
  return (ks == 1 && (epi == TE_STORE || epi == TE_STOREV) && ncta == 64) ? 16 : 8;
}
__host__ __device__ constexpr int conv_threads(int ks, int epi, int ncta) {
  return 64 + 32 * conv_epi_warps(ks, epi, ncta);
}
constexpr int kAcc = 4;                         // TMEM accumulator buffers

// KB: input channels per K-block; F8: E4M3 operands (kind::f8f6f4, 16
// channels per 16-byte core-matrix row) instead of BF16 (8 per row).
template <int KS, int KB, int NCTA, int EPI, bool F8>
__global__ void __launch_bounds__(conv_threads(KS, EPI, NCTA), 1) k_conv_tc(const __grid_constant__ CUtensorMap tmap,
                                                    const __grid_constant__ CUtensorMap tmap1,
                                                    const TcConvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // [0, 384): stage barriers; [384, 456): accumulator and weight barriers;
  // 456: abort flag; 464: TMEM base; [512, 640): head barriers
  uint64_t *full = reinterpret_cast<uint64_t *>(smem);       // [kMaxStages]
  uint64_t *empty = full + kMaxStages;                       // [kMaxStages]
  uint64_t *accf = empty + kMaxStages;                       // [kAcc]
  uint64_t *acce = accf + kAcc;                              // [kAcc]
  uint64_t *wbar = acce + kAcc;                              // [1]
  volatile int *s_abort = reinterpret_cast<volatile int *>(wbar + 1);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + 464);
  static_assert(2 * kMaxStages * 8 + (2 * kAcc + 1) * 8 + 4 <= 464, "barrier area");
  // TE_HEAD: the column halves of a lane quadrant exchange partial (mu, rho)
  // sums through s_part[acc][quadrant][lane], signalled by hbar[acc][quadrant]
  uint64_t *hbar = reinterpret_cast<uint64_t *>(smem + 512);        // [kAcc * 4]
  float2 *s_part = reinterpret_cast<float2 *>(smem + 4096);          // [kAcc][4][32]
  // per-column epilogue constants of this CTA's N block (loaded once):
  // bias, accumulator scale (F8), FP8 output scale, head weights [2][NCTA]
  float *s_bias = reinterpret_cast<float *>(smem + 1024);
  float *s_wsc = s_bias + NCTA;
  float *s_osc = s_wsc + NCTA;
  float *s_wh = s_osc + NCTA;
  uint8_t *wsm = smem + kConvHeader;
  uint8_t *stg = wsm + ((a.wv_bytes + a.w_bytes + 1023) / 1024) * 1024;

  // the head epilogue (residual + 1x1 C->2) on full tiles or compact ones
  constexpr bool HEADK = EPI == TE_HEAD || EPI == TE_HEADC;
  // plain stores; convs with a v block; the gates' v block shares the h
  // block's stage (one wait and one commit per tile), the z conv's has a
  // stage of its own (both measured the faster choice)
  constexpr bool STORE = EPI == TE_STORE || EPI == TE_STOREV;
  constexpr bool HV = EPI == TE_LSTM || EPI == TE_STOREV;
  constexpr bool VMERGE = EPI == TE_LSTM;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = blockIdx.x % a.nb;
  const int cta = blockIdx.x / a.nb;
  const int nctas = gridDim.x / a.nb;
  constexpr uint32_t kCols = NCTA * kAcc <= 32 ? 32 : NCTA * kAcc;  // power of two

  // a plain store whose only output is FP8: the output scale is folded into
  // the accumulator scale and bias (lrelu commutes with a positive scale)
  const bool fold8 = STORE && a.out8 && !a.out && !a.res && !a.outc;
  {
    const int nb0 = (blockIdx.x % a.nb) * NCTA;
    // FP8 output scale per output channel: the LSTM's outputs are channels
    // (4 gate columns each), the other epilogues' outputs are columns
    const int nosc = (EPI == TE_LSTM) ? NCTA / 4 : NCTA;
    const int osc0 = (EPI == TE_LSTM) ? nb0 / 4 : nb0;
    for (int j = threadIdx.x; j < NCTA; j += blockDim.x) {
      const float os = (a.out8_scale && j < nosc) ? a.out8_scale[osc0 + j] : 0.f;
      const float k = fold8 ? os : 1.f;
      s_bias[j] = a.bias[nb0 + j] * k;
      s_wsc[j] = (F8 ? a.w_scale[nb0 + j] : 1.f) * k;
      s_osc[j] = os;
      // head weights interleaved: (w_mu[j], w_rho[j]) as one FP32 pair
      if (HEADK) { s_wh[2 * j] = a.wh[j]; s_wh[2 * j + 1] = a.wh[NCTA + j]; }
    }
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.stages; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
    for (int i = 0; i < kAcc; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], conv_epi_warps(KS, EPI, NCTA));
    }
    if (HEADK)
      for (int i = 0; i < kAcc * 4; ++i) mbar_init(&hbar[i], 1);
    mbar_init(wbar, 1);
    // the compact head's swizzled stages must start on 1024-byte boundaries
    // (the swizzle pattern's period), else the kernel reports an error
    *s_abort = (EPI == TE_HEADC && (smem_u32(stg) & 1023u)) ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(s_tmem)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  // The set-up above reads constants only (model weights and scales, which
  // host copies write once at model load, never a kernel), so under a
  // programmatic dependent launch it overlaps the previous kernel's tail;
  // activations are read and written only after griddep_wait. The producer
  // starts its (constant) weight loads first, and lets the next kernel be
  // scheduled once it has issued its last load (measured faster than at
  // the start, when the next kernel's blocks would wait beside this one).
  if (threadIdx.x != 0) griddep_wait();
  const uint32_t tbase = *s_tmem;
  constexpr int taps = KS * KS;
  constexpr int R = KS / 2;
  constexpr int HX = kTileW + 2 * R, HY = kTileH + 2 * R;   // halo tile
  constexpr int EPG = F8 ? 16 : 8;          // channels per 16-byte group
  constexpr int GPK = KB / EPG;             // groups per K-block
  constexpr int KSTEPS = GPK / 2;           // MMAs per tap (32 bytes of K each)

  if (warp == 0 && lane == 0) {
    // ---- producer: weights once, then halo K-blocks ----------------------
    const uint8_t *wsrc = reinterpret_cast<const uint8_t *>(a.wt) + (size_t)nb * a.w_bytes;
    mbar_expect_tx(wbar, a.wv_bytes + a.w_bytes);
    if (a.wv_bytes) {   // v block first, then the rest
      const uint8_t *vsrc = reinterpret_cast<const uint8_t *>(a.wtv) + (size_t)nb * a.wv_bytes;
      for (uint32_t off = 0; off < a.wv_bytes; off += 32768u)
        bulk_load(wsm + off, vsrc + off, min(32768u, a.wv_bytes - off), wbar);
    }
    for (uint32_t off = 0; off < a.w_bytes; off += 32768u) {
      const uint32_t n = min(32768u, a.w_bytes - off);
      bulk_load(wsm + a.wv_bytes + off, wsrc + off, n, wbar);
    }
    griddep_wait();
    int stage = 0;
    uint32_t phase = 0;
    int issued = 0;
    // Tiles come in rounds of one, or two (paired issue: the MMA warp
    // interleaves two tiles into two accumulators) whose stages alternate:
    // K-step k of the first tile, K-step k of the second, k + 1, ...
    const bool pairs = a.pairs && a.stages >= 2;
    TileIter ti(cta, a.tiles_x, a.tiles_y);
    for (int t = cta; t < a.tiles && !*s_abort;) {
      const bool two = pairs && t + nctas < a.tiles;
      TileIter t1 = ti;
      t1.next(a.step_dx, a.step_dy, a.step_dp, a.tiles_x, a.tiles_y);   // tile t + nctas
      bool stop = false;
      for (int kbi = 0; kbi < a.nkb && !stop; ++kbi) {
        for (int u = 0; u < (two ? 2 : 1); ++u) {
          const TileIter &tt = u ? t1 : ti;
          const int tx = tt.tx, ty = tt.ty, p = tt.p;
          if (!mbar_wait(&empty[stage], phase ^ 1, s_abort, 500)) { stop = true; break; }
          const bool vk = HV && kbi == 0;    // the stage holds the v block
          const bool vsep = vk && !VMERGE;   // ... and nothing else
          const uint32_t hb = VMERGE ? a.hstage_bytes : a.stage_bytes;
          mbar_expect_tx(&full[stage], vsep ? a.vstage_bytes : vk ? hb + a.vstage_bytes : hb);
          if constexpr (EPI == TE_HEADC) {
            // compact head: K-step kbi = a.tps taps (9 / a.tps steps per
            // tile), one box per tap of cR rows x cJ positions x all
            // channels (one 128-row swizzled K-major slab). Output (row, j)
            // of the tile is at y = 2 (i0 + row) + par, x = aph + 4 (j0 + j);
            // tap (dy, dx) reads row 2 (i0 + row) + v, v = par + dy, through
            // the map of rows of parity v & 1 (index i0 + row + (v >> 1)),
            // and column 4 (j0 + j) + w, w = aph + dx, as phase w & 3 of
            // position j0 + j + (w >> 2). Out-of-range boxes read zeros (the
            // padding).
            const int par = ty & 1, i0 = (ty >> 1) * a.cR, j0 = tx * a.cJ;
            const int aph = step_phase(a.step, par);
            const uint32_t box = a.stage_bytes / a.tps;
            for (int k = 0; k < a.tps; ++k) {
              const int tap = kbi * a.tps + k;
              const int v = par + tap / 3 - 1, w = aph + tap % 3 - 1;
              const CUtensorMap *mp = (v & 1) ? &tmap1 : &tmap;
              tma_load_5d(stg + (size_t)stage * a.stage_bytes + k * box, mp, &full[stage], 0,
                          j0 + (w >> 2), w & 3, i0 + (v >> 1), p);
            }
          } else {
            // K-blocks [0, nkb0) come through tmap (group offset in_goff),
            // the rest through tmap1 (groups counted from 0); innermost
            // coordinate = pixel x * 8 channels (a multiple of 8 elements =
            // 16 bytes, also when negative at the left border)
            if (vk)
              tma_load_4d(stg + (size_t)stage * a.stage_bytes + a.hstage_bytes, &tmap,
                          &full[stage], (tx * kTileW - R) * 8, ty * kTileH - R, 0, p);
            if (vsep) {
            } else if (kbi < a.nkb0)
              tma_load_4d(stg + (size_t)stage * a.stage_bytes, &tmap, &full[stage],
                          (tx * kTileW - R) * EPG, ty * kTileH - R, a.in_goff + kbi * GPK, p);
            else
              tma_load_4d(stg + (size_t)stage * a.stage_bytes, &tmap1, &full[stage],
                          (tx * kTileW - R) * EPG, ty * kTileH - R,
                          a.in1_goff + (kbi - a.nkb0) * GPK, p);
          }
          ++issued;
          if (++stage == a.stages) { stage = 0; phase ^= 1; }
        }
      }
      if (stop) break;
      t += (two ? 2 : 1) * nctas;
      if (two) {
        ti = t1;
        ti.next(a.step_dx, a.step_dy, a.step_dp, a.tiles_x, a.tiles_y);
      } else {
        ti = t1;
      }
    }
    griddep_launch();
    // let every copy this thread issued land before the CTA can exit
    {
      int s = stage;
      uint32_t ph = phase;
      for (int i = 0; i < min(issued, a.stages); ++i) {
        if (--s < 0) { s = a.stages - 1; ph ^= 1; }
        mbar_wait_drain(&full[s], ph);
      }
      mbar_wait_drain(wbar, 0);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ---------------------------------------------------------
    // All descriptor offsets are compile-time constants: one K-block is
    // taps x KB/16 MMAs whose descriptors differ from the block's base
    // descriptors by fixed amounts (addresses enter descriptors >> 4).
    // instruction descriptor: FP32 accumulate; A/B format BF16 (1) for
    // kind::f16, E4M3 (0) for kind::f8f6f4; K-major; N, M = 128
    constexpr uint32_t fmt = F8 ? 0u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NCTA >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    constexpr uint32_t slab = (uint32_t)HX * HY * 16u;
    constexpr uint32_t wblock = (uint32_t)taps * GPK * NCTA * 16u;  // bytes per K-block
    bool ok = mbar_wait(wbar, 0, s_abort);
    int stage = 0, acc = 0;
    uint32_t phase = 0, aphase = 0;
    // a.pairs: two tiles per round (the producer alternates their K-blocks,
    // so two stages suffice), their MMAs interleaved into two accumulators so that
    // consecutive MMAs never depend on each other's accumulator (the
    // autotuner decides per shape class: faster for the FP8 3x3 convs,
    // slower for the HBM-bound 1x1 convs)
    const bool pairs = a.pairs && a.stages >= 2;
    for (int t = cta; ok && t < a.tiles; t += (pairs ? 2 : 1) * nctas) {
      const bool two = pairs && t + nctas < a.tiles;
      const int acc1 = acc + 1 == kAcc ? 0 : acc + 1;
      const uint32_t aphase1 = acc + 1 == kAcc ? aphase ^ 1 : aphase;
      if (!mbar_wait(&acce[acc], aphase ^ 1, s_abort, 200)) break;
      if (two && !mbar_wait(&acce[acc1], aphase1 ^ 1, s_abort, 200)) break;
      fence_after();
      const uint32_t d0 = tbase + (uint32_t)(acc * NCTA), d1 = tbase + (uint32_t)(acc1 * NCTA);
      uint32_t accum = 0;
      if constexpr (EPI == TE_HEADC) {
        // a.nkb = 9 / a.tps stages per tile, a.tps taps per stage: A =
        // 128 positions x KB channels per tap, rows of KB * element bytes
        // (32, 64 or 128) swizzled like the TMA wrote them; each MMA takes
        // the next 32 bytes of K within the rows
        constexpr uint32_t rowb = KB * (F8 ? 1 : 2);
        constexpr uint32_t swz = rowb == 128 ? 2u : rowb == 64 ? 4u : 6u;
        const uint64_t b0 = sdesc(smem_u32(wsm), NCTA * 16u, 128u);
        const uint32_t boxd = (128u * rowb) >> 4;   // descriptor step per tap
        for (int kbi = 0; kbi < a.nkb; ++kbi) {
          // stages of K-step kbi: the first tile's, then (paired) the second's
          int s0 = stage + (two ? 2 * kbi : kbi);
          uint32_t p0 = phase;
          while (s0 >= a.stages) { s0 -= a.stages; p0 ^= 1; }
          int s1 = s0 + 1;
          uint32_t p1 = p0;
          if (s1 >= a.stages) { s1 -= a.stages; p1 ^= 1; }
          if (!mbar_wait(&full[s0], p0, s_abort)) { ok = false; break; }
          if (two && !mbar_wait(&full[s1], p1, s_abort)) { ok = false; break; }
          fence_after();
          const uint64_t a0 = sdesc_sw(smem_u32(stg + (size_t)s0 * a.stage_bytes), 8u * rowb, swz);
          const uint64_t a1 = sdesc_sw(smem_u32(stg + (size_t)s1 * a.stage_bytes), 8u * rowb, swz);
          for (int tt = 0; tt < a.tps; ++tt) {
            const int tap = kbi * a.tps + tt;
#pragma unroll
            for (int s = 0; s < KSTEPS; ++s) {
              const uint32_t aoff = tt * boxd + ((32u * s) >> 4);
              const uint32_t boff = ((uint32_t)(tap * GPK + 2 * s) * (NCTA * 16u)) >> 4;
              if (F8) mma_fp8(d0, a0 + aoff, b0 + boff, idesc, accum);
              else mma_bf16(d0, a0 + aoff, b0 + boff, idesc, accum);
              if (two) {
                if (F8) mma_fp8(d1, a1 + aoff, b0 + boff, idesc, accum);
                else mma_bf16(d1, a1 + aoff, b0 + boff, idesc, accum);
              }
              accum = 1;
            }
          }
          mma_commit(&empty[s0]);
          if (two) mma_commit(&empty[s1]);
        }
      } else
      for (int kbi = 0; kbi < a.nkb; ++kbi) {
        // stages of this K-block: the first tile's, then (paired) the second's
        int s0 = stage + (two ? 2 * kbi : kbi);
        uint32_t p0 = phase;
        while (s0 >= a.stages) { s0 -= a.stages; p0 ^= 1; }
        int s1 = s0 + 1;
        uint32_t p1 = p0;
        if (s1 >= a.stages) { s1 -= a.stages; p1 ^= 1; }
        if (!mbar_wait(&full[s0], p0, s_abort)) { ok = false; break; }
        if (two && !mbar_wait(&full[s1], p1, s_abort)) { ok = false; break; }
        fence_after();
        const uint64_t a0 = sdesc(smem_u32(stg + (size_t)s0 * a.stage_bytes), slab, HX * 16u);
        const uint64_t a1 = sdesc(smem_u32(stg + (size_t)s1 * a.stage_bytes), slab, HX * 16u);
        if (HV && kbi == 0) {
          // v block (after the first K-block in the same stage, or alone
          // in its stage): one BF16 MMA (K = 16, the block's two 16-byte
          // groups) per tap, accumulating with the K-blocks' MMAs
          const uint32_t idv = (1u << 4) | (1u << 7) | (1u << 10) |
                               ((uint32_t)(NCTA >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
          const uint64_t bv = sdesc(smem_u32(wsm), NCTA * 16u, 128u);
          const uint32_t vo = VMERGE ? a.hstage_bytes >> 4 : 0u;
#pragma unroll
          for (int tap = 0; tap < taps; ++tap) {
            const uint32_t aoff = vo + (((uint32_t)((tap / KS) * HX + tap % KS) * 16u) >> 4);
            const uint32_t boff = ((uint32_t)(tap * 2) * (NCTA * 16u)) >> 4;
            mma_bf16(d0, a0 + aoff, bv + boff, idv, accum);
            if (two) mma_bf16(d1, a1 + aoff, bv + boff, idv, accum);
            accum = 1;
          }
          if (!VMERGE) {
            mma_commit(&empty[s0]);
            if (two) mma_commit(&empty[s1]);
            continue;
          }
        }
        const int kh = kbi - (HV && !VMERGE ? 1 : 0);   // index in wt
        const uint64_t b0 = sdesc(smem_u32(wsm) + a.wv_bytes + (uint32_t)kh * wblock, NCTA * 16u, 128u);
#pragma unroll
        for (int tap = 0; tap < taps; ++tap) {
#pragma unroll
          for (int s = 0; s < KSTEPS; ++s) {
            const uint32_t aoff = ((uint32_t)(2 * s) * slab + (uint32_t)((tap / KS) * HX + tap % KS) * 16u) >> 4;
            const uint32_t boff = ((uint32_t)(tap * GPK + 2 * s) * (NCTA * 16u)) >> 4;
            if (F8) mma_fp8(d0, a0 + aoff, b0 + boff, idesc, accum);
            else mma_bf16(d0, a0 + aoff, b0 + boff, idesc, accum);
            if (two) {
              if (F8) mma_fp8(d1, a1 + aoff, b0 + boff, idesc, accum);
              else mma_bf16(d1, a1 + aoff, b0 + boff, idesc, accum);
            }
            accum = 1;
          }
        }
        mma_commit(&empty[s0]);
        if (two) mma_commit(&empty[s1]);
      }
      if (!ok) break;
      mma_commit(&accf[acc]);
      if (two) mma_commit(&accf[acc1]);
      // advance past the consumed stages and accumulators
      const int used = (two ? 2 : 1) * a.nkb;
      stage += used;
      while (stage >= a.stages) { stage -= a.stages; phase ^= 1; }
      acc += two ? 2 : 1;
      if (acc >= kAcc) { acc -= kAcc; aphase ^= 1; }
    }
  } else if (warp >= 2) {
    // ---- epilogue: warps 2 .. 2 + EW - 1; warp w reads TMEM lanes
    // 32 (w % 4) .. +31 (output pixels), part (w - 2) / 4 of the columns
    // (two halves, or four quarters for the 16-warp plain stores; the head
    // epilogue needs all columns of a pixel and runs on half 0 only) -----
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    constexpr int NH = NCTA / (conv_epi_warps(KS, EPI, NCTA) / 4);
    const bool work = true;
    const int col0 = half * NH;
    const int m = 32 * q + lane;
    const int r = m / kTileW, c = m % kTileW;
    int acc = 0;
    uint32_t aphase = 0;
    const int G = a.out_G;
    const int n0 = nb * NCTA + col0;   // first output column handled here
    const int64_t hw = (int64_t)a.H * a.W;
    // output position of this thread in tile tt
    auto tile_pos = [&](const TileIter &tt, int &y, int &x) {
      if constexpr (EPI == TE_HEADC) {
        const int par = tt.ty & 1;
        y = 2 * ((tt.ty >> 1) * a.cR + (m >> a.cJlog)) + par;
        x = step_phase(a.step, par) + 4 * (tt.tx * a.cJ + (m & (a.cJ - 1)));
      } else {
        y = tt.ty * kTileH + r;
        x = tt.tx * kTileW + c;
      }
    };
    // Global operands of the epilogue (cell state, residual) do not depend
    // on the accumulator: they are loaded one tile ahead, so that their
    // latency overlaps the processing of the tile before (the epilogue, not
    // the MMAs, is the slower side of these kernels).
    constexpr int NPF = (EPI == TE_LSTM) ? NH / 4 : 8;
    static_assert(NPF % 8 == 0, "cell state in 8-channel groups");
    constexpr int NRES = (HEADK || STORE) ? NH / 8 : 1;
    // (the cell state stays packed BF16 until it is used: registers are
    // scarce in the ConvLSTM epilogue)
    constexpr int NCP = NPF / 8;
    auto load_ops = [&](const TileIter &tt, uint4 *cpo, uint4 *preso) {
      int y, x;
      tile_pos(tt, y, x);
      if (!(work && y < a.H && x < a.W)) return;
      const int p = tt.p;
      const int64_t pix = (int64_t)y * a.W + x;
      if (EPI == TE_LSTM) {
        const int Hp = a.H >> a.up, Wp = a.W >> a.up;
        const int64_t ppix = ((int64_t)p * Hp + (y >> a.up)) * Wp + (x >> a.up);
#pragma unroll
        for (int k = 0; k < NCP; ++k)
          cpo[k] = a.first ? make_uint4(0u, 0u, 0u, 0u)
                           : __ldg(reinterpret_cast<const uint4 *>(a.c_prev + ppix * a.C + n0 / 4 + 8 * k));
      } else if (HEADK || (STORE && a.res)) {
        const bool need = STORE ||
                          (a.compact_n ? pix < a.compact_n : step_of(y, x) == a.step);
        if (need) {
          if (HEADK && a.res_compact_n) {
            const int64_t qn = step_index(a.W, a.step, y, x);
#pragma unroll
            for (int g = 0; g < NRES; ++g)
              preso[g] = __ldg(reinterpret_cast<const uint4 *>(
                  a.res + (((int64_t)p * a.res_G + (n0 >> 3) + g) * a.res_compact_n + qn) * 8));
          } else {
#pragma unroll
            for (int g = 0; g < NRES; ++g)
              preso[g] = __ldg(reinterpret_cast<const uint4 *>(
                  a.res + (((int64_t)p * a.res_G + a.res_goff + (n0 >> 3) + g) * hw + pix) * 8));
          }
        }
      }
    };
    TileIter ti(cta, a.tiles_x, a.tiles_y);
    uint4 cpq[NCP];      // operands of the next tile to process
    uint4 presq[NRES];
    // only the epilogues that read such operands pay for the lookahead (the
    // z conv never has a residual, conv 1 and most plain stores neither)
    constexpr bool PREF = EPI == TE_LSTM || HEADK || EPI == TE_STORE;
    const bool has_ops = PREF && (EPI != TE_STORE || a.res != nullptr);
    if (has_ops && cta < a.tiles) load_ops(ti, cpq, presq);
    for (int t = cta; t < a.tiles;
         t += nctas, ti.next(a.step_dx, a.step_dy, a.step_dp, a.tiles_x, a.tiles_y)) {
      const int p = ti.p;
      int y, x;
      tile_pos(ti, y, x);
      const bool valid = y < a.H && x < a.W;
      const int64_t pix = (int64_t)y * a.W + x;
      uint4 cpk[NCP];
      uint4 pres[NRES];
#pragma unroll
      for (int k = 0; k < NCP; ++k) cpk[k] = cpq[k];
#pragma unroll
      for (int g = 0; g < NRES; ++g) pres[g] = presq[g];
      if (has_ops && t + nctas < a.tiles) {
        TileIter tn = ti;
        tn.next(a.step_dx, a.step_dy, a.step_dp, a.tiles_x, a.tiles_y);
        load_ops(tn, cpq, presq);
      }
      // warp-uniform wait: lane 0 decides, the others then observe the
      // completed phase themselves (their try_wait succeeds at once)
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&accf[acc], aphase, s_abort, 200) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      if (lane != 0) mbar_wait(&accf[acc], aphase, s_abort);
      __syncwarp();
      fence_after();
      float v[NH];
      const uint32_t taddr = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * NCTA + col0);
      if (work) tmem_ld<NH>(taddr, v);
      fence_before();
      __syncwarp();
      // the head's half 0 releases the accumulator only after it has read its
      // partner's partial sums for this tile (which then cannot be overwritten)
      const int cur_acc = acc;
      const uint32_t cur_phase = aphase;
      if (lane == 0 && !(HEADK && half == 0)) mbar_arrive(&acce[acc]);
      if (++acc == kAcc) { acc = 0; aphase ^= 1; }
      if (!work) continue;

      if constexpr (STORE) {
        // column pairs in packed FP32 (per element the same fmaf / add)
        const uint64_t *wsc2 = reinterpret_cast<const uint64_t *>(s_wsc + col0);
        const uint64_t *bia2 = reinterpret_cast<const uint64_t *>(s_bias + col0);
        if (F8 || fold8) {
#pragma unroll
          for (int j = 0; j < NH / 2; ++j)
            f2unpack(fma2(f2pack(v[2 * j], v[2 * j + 1]), wsc2[j], bia2[j]), v[2 * j],
                     v[2 * j + 1]);
        } else {
#pragma unroll
          for (int j = 0; j < NH / 2; ++j)
            f2unpack(add2(f2pack(v[2 * j], v[2 * j + 1]), bia2[j]), v[2 * j], v[2 * j + 1]);
        }
      } else if (F8) {
#pragma unroll
        for (int j = 0; j < NH; ++j) v[j] = fmaf(v[j], s_wsc[col0 + j], s_bias[col0 + j]);
      } else {
#pragma unroll
        for (int j = 0; j < NH; ++j) v[j] += s_bias[col0 + j];
      }
      // (the head's halves must both reach the partial-sum handoff, so
      // invalid positions only skip the work inside it)
      // element offsets of this thread's 16-byte chunk g in out (BF16) and
      // out8 (bytes): blocked planes, or the phase-split pixel-major layout
      const int64_t psix = (((int64_t)p * a.H + y) * 4 + (x & 3)) * (((a.W + 3) & ~3) >> 2) + (x >> 2);
      auto off_out = [&](int g) -> int64_t {
        return a.out_ps ? psix * (int64_t)(G * 8) + n0 + 8 * g
                        : (((int64_t)p * G + a.out_goff + (n0 >> 3) + g) * hw + pix) * 8;
      };
      auto off_out8 = [&](int g) -> int64_t {
        return a.out_ps ? psix * (int64_t)(a.out8_G16 * 16) + n0 + 16 * g
                        : (((int64_t)p * a.out8_G16 + (n0 >> 4) + g) * hw + pix) * 16;
      };
      if (STORE && !valid) {
        // pad columns of the phase-split layout: zeros
        if (a.out_ps && y < a.H && x < ((a.W + 3) & ~3)) {
          if (a.out) {
#pragma unroll
            for (int g = 0; g < NH / 8; ++g)
              *reinterpret_cast<uint4 *>(a.out + off_out(g)) = make_uint4(0u, 0u, 0u, 0u);
          }
          if (NH % 16 == 0 && a.out8) {
#pragma unroll
            for (int g = 0; g < NH / 16; ++g)
              *reinterpret_cast<uint4 *>(a.out8 + off_out8(g)) = make_uint4(0u, 0u, 0u, 0u);
          }
        }
        continue;
      }
      if (!valid && !HEADK) continue;
      if (STORE) {
#pragma unroll
        for (int g = 0; g < NH / 8; ++g) {
          if (a.res) {
            float rv[8];
            load_bf16x8(reinterpret_cast<const __nv_bfloat16 *>(&pres[g]), rv);
#pragma unroll
            for (int e = 0; e < 8; ++e) v[8 * g + e] += rv[e];
          }
          if (a.act) {
            // lrelu(x) = max(x, 0.01 x), the products in packed FP32
            const uint64_t k01 = f2pack(0.01f, 0.01f);
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              float lo, hi;
              f2unpack(mul2(f2pack(v[8 * g + e], v[8 * g + e + 1]), k01), lo, hi);
              v[8 * g + e] = fmaxf(v[8 * g + e], lo);
              v[8 * g + e + 1] = fmaxf(v[8 * g + e + 1], hi);
            }
          }
          if (a.out) store_bf16x8(a.out + off_out(g), v + 8 * g);
        }
        if (a.outc && step_of(y, x) == a.step) {
          const int64_t qn = step_index(a.W, a.step, y, x);
#pragma unroll
          for (int g = 0; g < NH / 8; ++g)
            store_bf16x8(a.outc + (((int64_t)p * G + (n0 >> 3) + g) * a.outc_n + qn) * 8, v + 8 * g);
        }
        if (NH % 16 == 0 && a.out8) {
#pragma unroll
          for (int g = 0; g < NH / 16; ++g) {
            float f[16];
            if (fold8) {
#pragma unroll
              for (int e = 0; e < 16; ++e) f[e] = v[16 * g + e];
            } else {
              // the output scale in packed FP32 pairs (per element one fmul)
              const uint64_t *osc2 = reinterpret_cast<const uint64_t *>(s_osc + col0 + 16 * g);
#pragma unroll
              for (int e = 0; e < 16; e += 2)
                f2unpack(mul2(f2pack(v[16 * g + e], v[16 * g + e + 1]), osc2[e / 2]), f[e],
                         f[e + 1]);
            }
            store_fp8x16(a.out8 + off_out8(g), f);
          }
        }
      } else if (EPI == TE_LSTM) {
        // column 4 * ch + gate (i, f, o, g) within the CTA's N block
        const int ch0 = n0 / 4;
        float cp[NPF];
#pragma unroll
        for (int k = 0; k < NCP; ++k)
          load_bf16x8(reinterpret_cast<const __nv_bfloat16 *>(&cpk[k]), cp + 8 * k);
        float hv[NH / 4], cn[NH / 4];
#pragma unroll
        for (int k = 0; k < NH / 4; ++k) {
          cn[k] = sigm_fast(v[4 * k + 1]) * cp[k] + sigm_fast(v[4 * k]) * tanh_fast(v[4 * k + 3]);
          hv[k] = sigm_fast(v[4 * k + 2]) * tanh_fast(cn[k]);
        }
#pragma unroll
        for (int k = 0; k < NH / 4; k += 8)
          store_bf16x8(a.c_new + ((int64_t)p * hw + pix) * a.C + ch0 + k, cn + k);
#pragma unroll
        for (int g = 0; g < NH / 32; ++g)
          store_bf16x8(a.out + (((int64_t)p * G + a.out_goff + (ch0 >> 3) + g) * hw + pix) * 8,
                       hv + 8 * g);
        if (NH % 64 == 0 && a.out8) {
#pragma unroll
          for (int g = 0; g < NH / 64; ++g) {
            float f[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) f[e] = hv[16 * g + e] * s_osc[col0 / 4 + 16 * g + e];
            store_fp8x16(a.out8 + (((int64_t)p * a.out8_G16 + (ch0 >> 4) + g) * hw + pix) * 16, f);
          }
        }
      } else {  // TE_HEAD: z' = res + acc + b over all C columns, then 1x1(C->2)
        const bool mine =
            valid && (a.compact_n ? pix < a.compact_n : step_of(y, x) == a.step);
        // partial sums of this half's columns (half 0 adds the head bias)
        float mu = half == 0 ? a.bh[0] : 0.f, rho = half == 0 ? a.bh[1] : 0.f;
        if (mine) {
          // (mu, rho) as one packed FP32 pair: per element the same fmaf
          // chain over the columns in order
          const uint64_t *wh2 = reinterpret_cast<const uint64_t *>(s_wh) + col0;
          uint64_t mr = f2pack(mu, rho);
#pragma unroll
          for (int g = 0; g < NH / 8; ++g) {
            float rv[8];
            load_bf16x8(reinterpret_cast<const __nv_bfloat16 *>(&pres[g]), rv);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float z = v[8 * g + e] + rv[e];
              mr = fma2(wh2[8 * g + e], f2pack(z, z), mr);
            }
          }
          f2unpack(mr, mu, rho);
        }
        float2 *slot = s_part + (cur_acc * 4 + q) * 32 + lane;
        if (half == 1) {
          *slot = make_float2(mu, rho);
          __syncwarp();
          if (lane == 0) mbar_arrive(&hbar[cur_acc * 4 + q]);
          continue;
        }
        int hok = 1;
        if (lane == 0) hok = mbar_wait(&hbar[cur_acc * 4 + q], cur_phase, s_abort, 100) ? 1 : 0;
        hok = __shfl_sync(0xffffffffu, hok, 0);
        if (!hok) break;
        if (lane != 0) mbar_wait(&hbar[cur_acc * 4 + q], cur_phase, s_abort);
        const float2 other = *slot;
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[cur_acc]);
        mu += other.x;
        rho += other.y;
        if (mine) {
          int qi;
          int64_t fpix, fhw;
          if (a.compact_n) {
            qi = (int)pix;
            int fy, fx;
            step_pos(a.full_W, a.step, qi, fy, fx);
            fpix = (int64_t)fy * a.full_W + fx;
            fhw = (int64_t)a.full_H * a.full_W;
          } else {
            qi = step_index(a.W, a.step, y, x);
            fpix = pix;
            fhw = hw;
          }
          a.idx[(int64_t)p * a.idx_stride + qi] = pack_index(mu, rho);
          if (a.mu_out) {
            a.mu_out[(int64_t)p * fhw + fpix] = mu;
            a.sg_out[(int64_t)p * fhw + fpix] = rho > 20.f ? rho : log1pf(expf(rho));
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols));
  }
  if (threadIdx.x == 0 && *s_abort) atomicExch(a.err, 1);
}

// ---------------------------------------------------------------------------
// SIMT helper kernels on the blocked BF16 layout.

// ConvLSTM gates input v (see pack_gates_v), one block per row (plane p,
// row y): V16[p][g][y][x][8] = 16 BF16 channels: the previous subband s
// (nearest-upsampled by `up` levels) at the 9 neighbours (0 outside the
// plane), 1 (inside indicator), zeros.
__global__ void __launch_bounds__(256) k_lstm_v(const int32_t *__restrict__ s_prev,
                                                __nv_bfloat16 *__restrict__ V16, int P, int H,
                                                int W, int up) {
  const int y = blockIdx.x % H;
  const int64_t p = blockIdx.x / H;
  const int Hp = H >> up, Wp = W >> up;
  const int64_t hw = (int64_t)H * W;
  const int32_t *sp = s_prev + p * Hp * Wp;
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    float v[16];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      v[tap] = (yy >= 0 && yy < H && xx >= 0 && xx < W)
                   ? (float)__ldg(sp + (int64_t)(yy >> up) * Wp + (xx >> up))
                   : 0.f;
    }
    v[9] = 1.f;
#pragma unroll
    for (int k = 10; k < 16; ++k) v[k] = 0.f;
    const int64_t pix = (int64_t)y * W + x;
    store_bf16x8(V16 + ((p * 2 + 0) * hw + pix) * 8, v);
    store_bf16x8(V16 + ((p * 2 + 1) * hw + pix) * 8, v + 8);
  }
}

// 16-byte channel groups of a blocked plane set, nearest-upsampled by `up`
// levels (zeros when zero is set): dst[p][dst_goff + g][y][x] =
// src[p][g][y >> up][x >> up] for g < ng, one block per row (plane, row).
__global__ void __launch_bounds__(256) k_copy_up16(const uint4 *__restrict__ src, int src_G,
                                                   uint4 *__restrict__ dst, int dst_G,
                                                   int dst_goff, int ng, int P, int H, int W,
                                                   int up, int zero) {
  const int y = blockIdx.x % H;
  const int64_t p = blockIdx.x / H;
  const int Hp = H >> up, Wp = W >> up;
  for (int it = threadIdx.x; it < ng * W; it += blockDim.x) {
    const int g = it / W, x = it - g * W;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (!zero) v = src[((p * src_G + g) * Hp + (y >> up)) * (int64_t)Wp + (x >> up)];
    dst[((p * dst_G + dst_goff + g) * H + y) * (int64_t)W + x] = v;
  }
}

// Compact step tail input: for the q-th position (y, x) of step `step`,
// Vc[q] = dw3x3(U)(y, x) + b and Zc[q] = Z(y, x) (C channels each, blocked
// layout; q indexes the compact plane of hc x wc positions).
__global__ void __launch_bounds__(256) k_dw3x3_compact(
    const __nv_bfloat16 *__restrict__ U, const __nv_bfloat16 *__restrict__ Z,
    const float *__restrict__ w, const float *__restrict__ b, __nv_bfloat16 *__restrict__ Vc,
    __nv_bfloat16 *__restrict__ Zc, int P, int H, int W, int C, int step, int n, int64_t chw) {
  // one block per compact row (plane p, row pair yc); item = group-major
  // (g, xc); xc < n_even lies on row 2 yc, the rest on row 2 yc + 1
  __shared__ float sw[9 * 128], sb[128];
  for (int i = threadIdx.x; i < 9 * C; i += blockDim.x) sw[i] = w[i];
  for (int i = threadIdx.x; i < C; i += blockDim.x) sb[i] = b[i];
  __syncthreads();
  const int G = C / 8;
  const int hc = (H + 1) >> 1;
  const int yc = blockIdx.x % hc;
  const int64_t p = blockIdx.x / hc;
  const int ae = step_phase(step, 0), ao = step_phase(step, 1);
  const int ne = row_count(W, ae), wc = ne + row_count(W, ao);
  const int64_t hw = (int64_t)H * W;
  for (int it = threadIdx.x; it < G * wc; it += blockDim.x) {
    const int g = it / wc, xc = it - g * wc;
    const int y = xc < ne ? 2 * yc : 2 * yc + 1;
    const int x = xc < ne ? ae + 4 * xc : ao + 4 * (xc - ne);
    if (y >= H) continue;  // odd height: the last pair has no odd row
    const int64_t pg = p * G + g;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = sb[8 * g + k];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
      float u[8];
      load_bf16x8(U + (pg * hw + (int64_t)yy * W + xx) * 8, u);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = fmaf(sw[(8 * g + k) * 9 + tap], u[k], v[k]);
    }
    const int64_t q = (int64_t)yc * wc + xc;
    store_bf16x8(Vc + (pg * chw + q) * 8, v);
    *reinterpret_cast<uint4 *>(Zc + (pg * chw + q) * 8) =
        *reinterpret_cast<const uint4 *>(Z + (pg * hw + (int64_t)y * W + x) * 8);
  }
}

// T = the 9 masked neighbour values of every position for step `step`
// (neighbours coded in an earlier step, else 0) as BF16 channels 0..8,
// channels 9..15 = 0 (the z conv's v block). One thread per position;
// blocked layout [P][2][H][W][8].
// One block per row (plane p, row y), threads along x: no integer division
// per element. Which of the 9 taps come from an earlier step depends only
// on (y mod 2, x mod 4): a 9-bit mask per class, built once per block.
__global__ void __launch_bounds__(128) k_masked_taps(const int32_t *__restrict__ s,
                                                     __nv_bfloat16 *__restrict__ T, int P, int H,
                                                     int W, int step) {
  __shared__ uint32_t smask[8];
  const int y = blockIdx.x % H;
  const int64_t p = blockIdx.x / H;
  if (threadIdx.x < 8) {
    const int ry = threadIdx.x >> 2, rx = threadIdx.x & 3;
    uint32_t m = 0;
    for (int tap = 0; tap < 9; ++tap)
      if (step_of(ry + 2 + tap / 3 - 1, rx + 4 + tap % 3 - 1) < step) m |= 1u << tap;
    smask[threadIdx.x] = m;
  }
  __syncthreads();
  const int64_t hw = (int64_t)H * W;
  const int32_t *sp = s + p * hw;
  const bool yin = y > 0 && y + 1 < H;
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    const uint32_t mask = smask[((y & 1) << 2) | (x & 3)];
    const bool interior = yin && x > 0 && x + 1 < W;
    float v[16];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      const bool use = ((mask >> tap) & 1u) &&
                       (interior || (yy >= 0 && yy < H && xx >= 0 && xx < W));
      v[tap] = use ? (float)__ldg(sp + (int64_t)yy * W + xx) : 0.f;
    }
#pragma unroll
    for (int c = 9; c < 16; ++c) v[c] = 0.f;
    const int64_t pix = (int64_t)y * W + x;
    store_bf16x8(T + ((p * 2 + 0) * hw + pix) * 8, v);
    store_bf16x8(T + ((p * 2 + 1) * hw + pix) * 8, v + 8);
  }
}

// ---------------------------------------------------------------------------
// Host side.
static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_encode{nullptr};

static int get_encoder() {
  if (g_encode.load()) return PW_OK;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    set_last_error("cuTensorMapEncodeTiled not available");
    return PW_ECUDA;
  }
  g_encode.store(reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn));
  return PW_OK;
}

// Tensor map over a blocked BF16 tensor [P][G][H][W][8], viewed as 4-D
// (W * 8 elements, H, G, P) so that each box row is one contiguous run of
// box_x * 16 bytes; box = one K-block halo tile.
// With f8 the tensor holds E4M3 bytes [P][G][H][W][16] (G = channels / 16)
// and the map's elements are bytes; the byte geometry is the same.
static int make_map(CUtensorMap *map, const void *base, int P, int G, int H, int W,
                    int box_x, int box_y, int box_g, bool f8 = false) {
  int s = get_encoder();
  if (s) return s;
  const cuuint64_t epg = f8 ? 16 : 8;
  cuuint64_t dims[4] = {(cuuint64_t)W * epg, (cuuint64_t)H, (cuuint64_t)G, (cuuint64_t)P};
  cuuint64_t strides[3] = {(cuuint64_t)W * 16, (cuuint64_t)H * W * 16,
                           (cuuint64_t)G * H * W * 16};
  cuuint32_t box[4] = {(cuuint32_t)(box_x * epg), (cuuint32_t)box_y, (cuuint32_t)box_g, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = g_encode.load()(map, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                        4, (void *)base, dims, strides, box,
                        es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return PW_ECUDA;
  }
  return PW_OK;
}

// Compact-head view of a phase-split pixel-major activation
// [P][H][4][W4 / 4][C] (x = 4 j + phase): the rows of parity `par` as a 5-D
// tensor (channels, j, phase, row / 2, plane); a box is R rows x J positions
// of one phase with all C channels, landing as 128 rows of C elements in
// the swizzled K-major layout of the row size (32, 64 or 128 bytes).
static int make_map_hc(CUtensorMap *map, const void *base, int P, int C, int H, int W4, int par,
                       int R, int J, bool f8) {
  int s = get_encoder();
  if (s) return s;
  const cuuint64_t rowb = (cuuint64_t)C * (f8 ? 1 : 2);
  cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)W4 / 4, 4, (cuuint64_t)(H + 1 - par) / 2,
                        (cuuint64_t)P};
  cuuint64_t strides[4] = {rowb, rowb * (W4 / 4), rowb * W4 * 2, rowb * W4 * H};
  cuuint32_t box[5] = {(cuuint32_t)C, (cuuint32_t)J, 1, (cuuint32_t)R, 1};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUtensorMapSwizzle sw = rowb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : rowb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                             : CU_TENSOR_MAP_SWIZZLE_32B;
  void *b = (void *)(static_cast<const uint8_t *>(base) + (size_t)par * W4 * rowb);
  CUresult r = g_encode.load()(map, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                               5, b, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return PW_ECUDA;
  }
  return PW_OK;
}

// The compact head applies to subbands of at least 4 rows and 8 columns.
static bool headc_ok(int h, int w) { return h >= 4 && w >= 8; }


// ---- autotuner -------------------------------------------------------------
// Per (kernel variant, size class = log2 of the tile count) the MMA issue
// schedule: one or two tiles per round. The candidates are sampled in place,
// round robin, on the real launches of the decode / encode pipeline (each
// launch bracketed by events that are read back later without a
// synchronisation), so that the choice reflects the caches and concurrency
// the kernel really sees; after kSamples samples of every candidate the
// fastest median wins (the median ignores a one-off outlier such as the
// first launch of a kernel, which loads its module). Results do not depend
// on the schedule.
// Candidates: bit 0 = paired MMA issue, bit 1 = the alternative pipeline
// shape (a shallower pipeline for the plain convolutions, the second-best
// tile shape for the compact head).
constexpr int kTuneCand = 4, kSamples = 3;
struct TuneChoice {
  int pairs = 0;
  int shape = 0;
  int cand() const { return pairs | (shape << 1); }
};
struct TuneEntry {
  bool tuned = false;
  TuneChoice choice;
  int next = 0;                        // candidate of the next sample
  int issued[kTuneCand] = {};          // samples launched
  int n[kTuneCand] = {};               // samples read back
  float us[kTuneCand][kSamples] = {};  // their times
  double median(int c) const {
    if (n[c] == 0) return -1.0;
    float v[kSamples];
    for (int i = 0; i < n[c]; ++i) v[i] = us[c][i];
    std::sort(v, v + n[c]);
    return v[n[c] / 2];
  }
};
struct TunePending {
  uint64_t key;
  int cand;
  cudaEvent_t e0, e1;
};
static std::mutex g_tune_mu;
static std::map<uint64_t, TuneEntry> g_tune;
static std::vector<TunePending> g_tune_pending;
static std::atomic<int> g_tune_on{1};
// launches of a class still being tuned (sampled or waiting for read-back)
static std::atomic<uint64_t> g_untuned_uses{0};

static uint64_t tune_key(const TcWeights::Conv &cv, int epi, int tiles) {
  int cls = 0;
  while ((1 << (cls + 1)) <= tiles && cls < 30) ++cls;
  int dev = 0;
  cudaGetDevice(&dev);
  return ((uint64_t)dev << 40) | ((uint64_t)cv.ks << 32) | ((uint64_t)cv.kb << 24) |
         ((uint64_t)cv.ncta << 14) | ((uint64_t)epi << 10) | ((uint64_t)cv.f8 << 9) |
         (uint64_t)cls;
}

// Read back finished samples (lock held).
static void tune_poll_locked() {
  size_t w = 0;
  for (size_t i = 0; i < g_tune_pending.size(); ++i) {
    TunePending &q = g_tune_pending[i];
    const cudaError_t e = cudaEventQuery(q.e1);
    if (e == cudaErrorNotReady) { g_tune_pending[w++] = q; continue; }
    float ms = 0.f;
    if (e == cudaSuccess && cudaEventElapsedTime(&ms, q.e0, q.e1) == cudaSuccess) {
      TuneEntry &t = g_tune[q.key];
      if (t.n[q.cand] < kSamples) t.us[q.cand][t.n[q.cand]++] = 1e3f * ms;
      bool done = !t.tuned;
      for (int c = 0; c < kTuneCand; ++c) done = done && (t.issued[c] == 0 || t.n[c] >= kSamples);
      if (done) {
        double best = 1e30;
        for (int c = 0; c < kTuneCand; ++c)
          if (t.n[c] && t.median(c) < best) {
            best = t.median(c);
            t.choice.pairs = c & 1;
            t.choice.shape = c >> 1;
          }
        t.tuned = true;
      }
    } else {
      cudaGetLastError();
    }
    cudaEventDestroy(q.e0);
    cudaEventDestroy(q.e1);
  }
  g_tune_pending.resize(w);
}

// The schedule of the next launch of a class. While the class is being tuned
// (sample = true) the launch is a sample of candidate `cand`.
static TuneChoice tune_next(uint64_t key, bool can_pair, bool has_alt, cudaStream_t st,
                            bool &sample, int &cand) {
  TuneChoice c;
  c.pairs = ((key >> 32) & 0xFF) == 3 && ((key >> 9) & 1) && can_pair;  // default
  sample = false;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_poll_locked();
  TuneEntry &t = g_tune[key];
  if (t.tuned) {
    c.pairs = t.choice.pairs && can_pair;
    c.shape = t.choice.shape && has_alt;
    return c;
  }
  if (!g_tune_on.load()) return c;
  g_untuned_uses.fetch_add(1);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return c;
  }
  auto valid = [&](int k) { return (!(k & 1) || can_pair) && (!(k & 2) || has_alt); };
  int nvalid = 0;
  for (int k = 0; k < kTuneCand; ++k) nvalid += valid(k) ? 1 : 0;
  if (nvalid == 1) {  // nothing to choose
    t.tuned = true;
    t.choice = TuneChoice{};
    return c;
  }
  while (!valid(t.next)) t.next = (t.next + 1) % kTuneCand;
  cand = t.next;
  if (t.issued[cand] >= kSamples) return c;  // enough in flight; wait for read-back
  do { t.next = (t.next + 1) % kTuneCand; } while (!valid(t.next));
  t.issued[cand] += 1;
  c.pairs = cand & 1;
  c.shape = cand >> 1;
  sample = true;
  return c;
}

static void tune_record(uint64_t key, int cand, cudaEvent_t e0, cudaEvent_t e1) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_pending.push_back(TunePending{key, cand, e0, e1});
}

uint64_t tune_untuned_uses() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_poll_locked();
  return g_untuned_uses.load();
}

int tune_set_enabled(int on) {
  const int old = g_tune_on.load();
  g_tune_on.store(on ? 1 : 0);
  return old;
}
// One line per tuned class: "ks kb ncta epi f8 log2tiles choice t0 t1 t2 t3"
// (choice = the kept candidate, bit 0 paired issue, bit 1 alternative
// pipeline shape; t = median sampled time of each candidate in microseconds,
// -1 = not sampled).
std::string tune_report() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_poll_locked();
  std::string out;
  char line[256];
  for (const auto &kv : g_tune) {
    if (!kv.second.tuned) continue;
    const uint64_t k = kv.first;
    const TuneEntry &t = kv.second;
    snprintf(line, sizeof(line), "%d %d %d %d %d %d %d %.1f %.1f %.1f %.1f\n",
             (int)((k >> 32) & 0xFF), (int)((k >> 24) & 0xFF), (int)((k >> 14) & 0x3FF),
             (int)((k >> 10) & 0xF), (int)((k >> 9) & 1), (int)(k & 0x1FF), t.choice.cand(),
             t.median(0), t.median(1), t.median(2), t.median(3));
    out += line;
  }
  return out;
}

// Launch a tensor-core convolution with a programmatic dependency on the
// previous kernel of the stream (its set-up overlaps that kernel's tail; it
// touches activations only after griddep_wait).
template <typename K>
static int launch_pdl(pw_ctx *ctx, K kern, int threads, int grid, size_t smem, cudaStream_t st,
                      const CUtensorMap &map, const CUtensorMap &map1, const TcConvArgs &la) {
  const cudaError_t e = launch_dep(kern, dim3((unsigned)grid), dim3((unsigned)threads), smem, st,
                                   map, map1, la);
  if (e != cudaSuccess) {
    set_last_error(std::string("tensor-core conv launch: ") + cudaGetErrorString(e));
    return PW_ECUDA;
  }
  ctx->launches += 1;
  return PW_OK;
}

// Launch one tensor-core convolution.
// in / in_G / in_goff: the input tensor of the first nkb0 K-blocks (all of
// them when in1 is null); in1 / in1_G: the input of the remaining K-blocks.
// With a v block (cv.wv) `in` holds its two BF16 groups, the K-blocks come
// through in1 and the nkb0 argument is not used.
// in_G / in1_G / goffs count 16-byte channel groups (8 BF16 or 16 E4M3
// channels; cv.f8 selects the operand type).
static int conv_tc(pw_ctx *ctx, const TcWeights::Conv &cv, const void *in, int in_G,
                   int in_goff, int P, int H, int W, TcConvArgs a, int *err,
                   const void *in1 = nullptr, int in1_G = 0, int in1_goff = 0,
                   int nkb0 = -1) {
  const int R = cv.ks / 2;
  a.P = P; a.H = H; a.W = W; a.ks = cv.ks; a.cin = cv.cin; a.kb = cv.kb; a.nkb = cv.cin / cv.kb;
  a.in_goff = in_goff; a.ncta = cv.ncta; a.nb = cv.nb;
  a.halo_x = kTileW + 2 * R; a.halo_y = kTileH + 2 * R;
  a.tiles_x = (W + kTileW - 1) / kTileW; a.tiles_y = (H + kTileH - 1) / kTileH;
  a.tiles = P * a.tiles_x * a.tiles_y;
  const int esz = cv.f8 ? 1 : 2, epg = cv.f8 ? 16 : 8;
  a.stage_bytes = (uint32_t)a.halo_x * a.halo_y * cv.kb * esz;
  a.w_bytes = (uint32_t)(cv.ks * cv.ks) * cv.cin * cv.ncta * esz;
  a.wt = cv.w; a.bias = cv.b; a.w_scale = cv.sw; a.err = err;
  if (cv.wv) {
    // ConvLSTM gates: K-block 0 = the BF16 v block through `in` (2 groups),
    // the h block (cin channels) through in1
    a.wtv = cv.wv;
    a.wv_bytes = (uint32_t)(cv.ks * cv.ks) * 2u * cv.ncta * 16u;
    a.vstage_bytes = (uint32_t)a.halo_x * a.halo_y * 32u;
    if (a.epi == TE_LSTM) {
      // the gates: the v block follows the h block in its stage
      a.hstage_bytes = a.stage_bytes;
      a.stage_bytes += a.vstage_bytes;
    } else {
      // the z conv: the v block is K-block 0 in a stage of its own
      if (a.epi == TE_STORE) a.epi = TE_STOREV;
      a.hstage_bytes = 0;
      a.nkb += 1;
    }
  }
  if ((a.epi == TE_LSTM || a.epi == TE_STOREV) != (cv.wv != nullptr)) {
    set_last_error("tensor-core conv: v block and epilogue do not match");
    return PW_EUNSUPPORTED;
  }
  const bool hc = a.epi == TE_HEADC;
  // compact head: tiles of R rows of one parity x J step positions. The
  // shapes with the fewest and the second-fewest tiles (ties: the wider one)
  // are the tuner's two shape candidates.
  int lj_best = -1, lj_alt = -1;
  int npos = 0, nrows = 0;
  if (hc) {
    npos = std::max(row_count(W, step_phase(a.step, 0)), row_count(W, step_phase(a.step, 1)));
    nrows = (H + 1) / 2;
    int best = -1, second = -1;
    for (int lj = 3; lj <= 7; ++lj) {
      const int J = 1 << lj, Rr = 128 / J;
      const int n = ((npos + J - 1) / J) * ((nrows + Rr - 1) / Rr);
      if (best < 0 || n <= best) {
        second = best; lj_alt = lj_best;
        best = n; lj_best = lj;
      } else if (second < 0 || n <= second) {
        second = n; lj_alt = lj;
      }
    }
  }
  auto set_hc_shape = [&](int lj) {
    a.cJlog = lj;
    a.cJ = 1 << a.cJlog; a.cR = 128 / a.cJ;
    a.tiles_x = (npos + a.cJ - 1) / a.cJ;
    a.tiles_y = 2 * ((nrows + a.cR - 1) / a.cR);
    a.tiles = P * a.tiles_x * a.tiles_y;
    // taps per stage: 3 (three commits per tile), or 1 where three 3-tap
    // stages do not fit next to the weights
    const uint32_t tapb = 128u * (uint32_t)cv.cin * esz;   // one tap: 128 rows x C
    const size_t room = 227 * 1024 - kConvHeader - (a.w_bytes + 1023) / 1024 * 1024;
    a.tps = room >= 3 * 3 * (size_t)tapb ? 3 : 1;
    a.nkb = 9 / a.tps;                           // stages per tile
    a.stage_bytes = (uint32_t)a.tps * tapb;
  };
  if (hc) set_hc_shape(lj_best);
  const size_t fixed = kConvHeader + (a.wv_bytes + a.w_bytes + 1023) / 1024 * 1024;
  const size_t maxsm = 227 * 1024;
  auto depth = [&](int cap) {
    const int n = (int)((maxsm - fixed) / a.stage_bytes);
    return n > cap ? cap : n;
  };
  // deep pipelines keep enough bytes in flight for the HBM-bound 1x1 convs;
  // the alternative shape of the plain convs is a shallower pipeline
  const int st_def = depth(hc ? std::min(kMaxStages, 2 * a.nkb + 2) : (cv.ks == 1 ? 16 : 6));
  if (st_def < 2) { set_last_error("tensor-core conv does not fit in shared memory"); return PW_EUNSUPPORTED; }
  int st_alt = -1;
  if (!hc) {
    const int v = depth(cv.ks == 1 ? 8 : 4);
    if (v >= 2 && v != st_def) st_alt = v;
  }
  const bool has_alt = hc ? lj_alt >= 0 : st_alt >= 0;
  // tuning class: the variant (epilogue 4 = a plain store with a v block,
  // the steps 2-4 z conv) and the size (tiles of the default shape)
  const uint64_t key = tune_key(cv, a.epi, a.tiles);
  bool sample = false;
  int cand = 0;
  const TuneChoice ch = tune_next(key, true, has_alt, ctx->stream, sample, cand);
  a.pairs = ch.pairs;
  if (ch.shape && hc) set_hc_shape(lj_alt);
  a.stages = (ch.shape && !hc) ? st_alt : st_def;
  const size_t smem = fixed + (size_t)a.stages * a.stage_bytes;
  CUtensorMap map, map1;
  int s;
  if (hc) {
    const int W4 = (W + 3) & ~3;
    if ((s = make_map_hc(&map, in, P, cv.cin, H, W4, 0, a.cR, a.cJ, cv.f8))) return s;
    if ((s = make_map_hc(&map1, in, P, cv.cin, H, W4, 1, a.cR, a.cJ, cv.f8))) return s;
  } else if (cv.wv) {
    if (!in1) { set_last_error("gates conv needs the h input"); return PW_EINVAL; }
    if ((s = make_map(&map, in, P, 2, H, W, a.halo_x, a.halo_y, 2, false))) return s;
  } else if ((s = make_map(&map, in, P, in_G, H, W, a.halo_x, a.halo_y, cv.kb / epg, cv.f8))) {
    return s;
  }
  a.nkb0 = a.nkb;
  a.in1_goff = in1_goff;
  if (in1 && !hc) {
    a.nkb0 = cv.wv ? (a.epi == TE_LSTM ? 0 : 1) : nkb0;
    if ((s = make_map(&map1, in1, P, in1_G, H, W, a.halo_x, a.halo_y, cv.kb / epg, cv.f8)))
      return s;
  } else if (!hc) {
    map1 = map;
  }
  cudaStream_t st = ctx->stream;
  // one launch with a persistent grid of SMs / frac CTAs per N block
  auto launch = [&](TcConvArgs &la, int frac) -> int {
    int per_nb = sm_count() / cv.nb / frac;
    if (per_nb < 1) per_nb = 1;
    if (per_nb > la.tiles) per_nb = la.tiles;
    const int grid = per_nb * cv.nb;
    la.step_dx = per_nb % la.tiles_x;
    la.step_dy = (per_nb / la.tiles_x) % la.tiles_y;
    la.step_dp = per_nb / (la.tiles_x * la.tiles_y);
#define PW_TC_CASE(KS_, KB_, N_, E_, F8_)                                                   \
    if (cv.ks == KS_ && cv.kb == KB_ && cv.ncta == N_ && la.epi == E_ && cv.f8 == F8_) {    \
      static std::atomic<uint64_t> attr{0};                                                 \
      once_per_device(attr, [&] {                                                           \
        cudaFuncSetAttribute(k_conv_tc<KS_, KB_, N_, E_, F8_>,                              \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxsm);      \
      });                                                                                   \
      return launch_pdl(ctx, k_conv_tc<KS_, KB_, N_, E_, F8_>, conv_threads(KS_, E_, N_), grid, smem, \
                        st, map, map1, la);                                                  \
    }
    // BF16 plain stores (all shapes the stage entry accepts)
    PW_TC_CASE(1, 32, 32, TE_STORE, false) PW_TC_CASE(1, 32, 64, TE_STORE, false)
    PW_TC_CASE(1, 32, 128, TE_STORE, false) PW_TC_CASE(1, 64, 32, TE_STORE, false)
    PW_TC_CASE(1, 64, 64, TE_STORE, false) PW_TC_CASE(1, 64, 128, TE_STORE, false)
    PW_TC_CASE(3, 32, 32, TE_STORE, false) PW_TC_CASE(3, 32, 64, TE_STORE, false)
    PW_TC_CASE(3, 32, 128, TE_STORE, false) PW_TC_CASE(3, 64, 32, TE_STORE, false)
    PW_TC_CASE(3, 64, 64, TE_STORE, false) PW_TC_CASE(3, 64, 128, TE_STORE, false)
    // z conv of steps 2-4 (v block + l)
    PW_TC_CASE(1, 32, 32, TE_STOREV, false) PW_TC_CASE(1, 64, 64, TE_STOREV, false)
    // ConvLSTM gates (K-block = C channels)
    PW_TC_CASE(3, 32, 64, TE_LSTM, false) PW_TC_CASE(3, 64, 64, TE_LSTM, false)
    // residual + head: 3x3 C->C of steps 2-4, 1x1 2C->C of step 1
    PW_TC_CASE(3, 32, 32, TE_HEAD, false) PW_TC_CASE(3, 64, 64, TE_HEAD, false)
    PW_TC_CASE(1, 64, 32, TE_HEAD, false) PW_TC_CASE(1, 64, 64, TE_HEAD, false)
    // FP8: gates (N = 128 per CTA), residual-block convs of steps 2-4
    PW_TC_CASE(3, 32, 128, TE_LSTM, true) PW_TC_CASE(3, 64, 128, TE_LSTM, true)
    PW_TC_CASE(3, 32, 32, TE_STORE, true) PW_TC_CASE(3, 64, 64, TE_STORE, true)
    PW_TC_CASE(3, 32, 32, TE_HEAD, true) PW_TC_CASE(3, 64, 64, TE_HEAD, true)
    // compact heads of steps 2-4
    PW_TC_CASE(3, 32, 32, TE_HEADC, false) PW_TC_CASE(3, 64, 64, TE_HEADC, false)
    PW_TC_CASE(3, 32, 32, TE_HEADC, true) PW_TC_CASE(3, 64, 64, TE_HEADC, true)
#undef PW_TC_CASE
    set_last_error("no tensor-core conv for this shape");
    return PW_EUNSUPPORTED;
  };
  if (!sample) return launch(a, 1);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  s = launch(a, 1);
  cudaEventRecord(e1, st);
  tune_record(key, cand, e0, e1);
  return s;
}

// ---- weights -------------------------------------------------------------
// kb: channels per K-block (0 = min(cin, 64)); the ConvLSTM gates use kb = C
// so that every K-block is either all e channels or all h channels.
static int pack_conv(TcWeights &tw, TcWeights::Conv &cv, const std::vector<float> &w,
                     const std::vector<float> &b, int cout, int cin, int ks, int ncta,
                     int kb = 0) {
  // w: [cout][cin][ks*ks] (output order as the kernel's columns)
  cv.cin = cin; cv.cout = cout; cv.ks = ks; cv.kb = kb ? kb : (cin >= 64 ? 64 : cin);
  cv.ncta = ncta;
  cv.nb = cout / ncta;
  const int taps = ks * ks, nkb = cin / cv.kb, gpb = cv.kb / 8;
  std::vector<__nv_bfloat16> h((size_t)cout * cin * taps);
  size_t o = 0;
  for (int nb = 0; nb < cv.nb; ++nb)
    for (int kbi = 0; kbi < nkb; ++kbi)
      for (int t = 0; t < taps; ++t)
        for (int g = 0; g < gpb; ++g)
          for (int n = 0; n < ncta; ++n)
            for (int e = 0; e < 8; ++e) {
              const int co = nb * ncta + n, ci = kbi * cv.kb + g * 8 + e;
              h[o++] = __float2bfloat16(w[((size_t)co * cin + ci) * taps + t]);
            }
  if (cudaMalloc(&cv.w, h.size() * 2) != cudaSuccess || cudaMalloc(&cv.b, cout * 4) != cudaSuccess) {
    set_last_error("weight allocation failed");
    return PW_ENOMEM;
  }
  tw.allocs.push_back(cv.w);
  tw.allocs.push_back(cv.b);
  cudaMemcpy(cv.w, h.data(), h.size() * 2, cudaMemcpyHostToDevice);
  cudaMemcpy(cv.b, b.data(), cout * 4, cudaMemcpyHostToDevice);
  return PW_OK;
}

// ConvLSTM gates without the e channels (Section 3.2): e = we * u + be (a
// 3x3 conv of the upsampled previous subband u) has no nonlinearity before
// the gates conv, so We * e = sum over taps of (We[tap] [we | be]) v, with
// v = the 9 neighbour values of u and an inside indicator (zero outside the
// plane, like e under the gates conv's zero padding): 10 input channels
// instead of C. Returns the h-only weights [4C][C][9] of wg ([4C][2C][9],
// inputs e then h) in wh and packs the v block as BF16 [nb][tap][2][ncta][8]
// (channels 10..15 zero), each output column divided by colscale[n] (the
// FP8 accumulator scale; null = 1).
static int pack_gates_v(TcWeights &tw, TcWeights::Conv &cv, const std::vector<float> &wg,
                        const std::vector<float> &we, const std::vector<float> &be, int C,
                        int ncta, const std::vector<float> *colscale, std::vector<float> &wh) {
  const int cout = 4 * C, nb = cout / ncta;
  wh.assign((size_t)cout * C * 9, 0.f);
  for (int n = 0; n < cout; ++n)
    for (int c = 0; c < C; ++c)
      for (int t = 0; t < 9; ++t)
        wh[((size_t)n * C + c) * 9 + t] = wg[((size_t)n * 2 * C + C + c) * 9 + t];
  std::vector<__nv_bfloat16> h((size_t)nb * 9 * 2 * ncta * 8, __float2bfloat16(0.f));
  for (int n = 0; n < cout; ++n) {
    const int b = n / ncta, nn = n % ncta;
    const double cs = colscale ? (double)(*colscale)[n] : 1.0;
    for (int t = 0; t < 9; ++t)
      for (int j = 0; j < 10; ++j) {
        double acc = 0.0;
        for (int c = 0; c < C; ++c)
          acc += (double)wg[((size_t)n * 2 * C + c) * 9 + t] * (j < 9 ? we[c * 9 + j] : be[c]);
        const int g = j / 8, e = j % 8;
        h[((((size_t)b * 9 + t) * 2 + g) * ncta + nn) * 8 + e] = __float2bfloat16((float)(acc / cs));
      }
  }
  if (cudaMalloc(&cv.wv, h.size() * 2) != cudaSuccess) {
    set_last_error("weight allocation failed");
    return PW_ENOMEM;
  }
  tw.allocs.push_back(cv.wv);
  cudaMemcpy(cv.wv, h.data(), h.size() * 2, cudaMemcpyHostToDevice);
  return PW_OK;
}

int Model::ensure_tc() {
  if (tc) return PW_OK;
  if (C != 32 && C != 64) {
    set_last_error("the tensor-core path supports C = 32 or 64");
    return PW_EUNSUPPORTED;
  }
  std::unique_ptr<TcWeights> t(new TcWeights());
  int s;
  auto H = [&](const std::string &n) -> const std::vector<float> & { return host.at(n); };
  {
    std::vector<float> wh;
    if ((s = pack_gates_v(*t, t->gates, H("lstm.wg.perm"), H("lstm.we"), H("lstm.be"), C, 64,
                          nullptr, wh)))
      return s;
    if ((s = pack_conv(*t, t->gates, wh, H("lstm.bg.perm"), 4 * C, C, 3, 64, C))) return s;
  }
  auto set = [&](const std::string &ns, TcWeights::Conv &in_, TcWeights::Conv &w1,
                 TcWeights::Conv &w2, TcWeights::Conv &w3, TcWeights::Conv &w4,
                 TcWeights::Conv *k1, TcWeights::Conv *k2) -> int {
    int r;
    const std::string p = ns + ".s0.";
    const std::vector<float> &win = H(p + "win"), &bin = H(p + "bin"), &wa = H(p + "w1"),
                             &ba = H(p + "b1");
    if ((r = pack_conv(*t, in_, win, bin, C, C, 1, C))) return r;
    {
      std::vector<float> wc((size_t)C * C), bc(C);
      for (int c = 0; c < C; ++c) {
        double bacc = ba[c];
        for (int k = 0; k < C; ++k) bacc += (double)wa[(size_t)c * C + k] * bin[k];
        bc[c] = (float)bacc;
        for (int j = 0; j < C; ++j) {
          double acc = 0.0;
          for (int k = 0; k < C; ++k) acc += (double)wa[(size_t)c * C + k] * win[(size_t)k * C + j];
          wc[(size_t)c * C + j] = (float)acc;
        }
      }
      if ((r = pack_conv(*t, w1, wc, bc, C, C, 1, C))) return r;
    }
    if ((r = pack_conv(*t, w2, H(p + "w2"), H(p + "b2"), C, C, 1, C))) return r;
    if ((r = pack_conv(*t, w3, H(p + "w3"), H(p + "b3"), 2 * C, C, 1, 2 * C))) return r;
    if ((r = pack_conv(*t, w4, H(p + "w4"), H(p + "b4"), C, 2 * C, 1, C))) return r;
    for (int k = 1; k < 4; ++k) {
      const std::string q = ns + ".s" + std::to_string(k) + ".";
      if ((r = pack_conv(*t, k1[k - 1], H(q + "w1"), H(q + "b1"), C, C, 3, C))) return r;
      if ((r = pack_conv(*t, k2[k - 1], H(q + "w2"), H(q + "b2"), C, C, 3, C))) return r;
    }
    return PW_OK;
  };
  if ((s = set("sb", t->s0_in, t->s0_w1, t->s0_w2, t->s0_w3, t->s0_w4, t->sk_c1, t->sk_c2)))
    return s;
  // Steps 2-4: z = Wz [a; l] + bz with a = Wa * (m s) + ba is linear in a,
  // so z = Wz_l l + sum_tap (Wz_a Wa[:, tap]) (m s)(tap) + (Wz_a ba + bz):
  // one 1x1 over l and a v block of the 9 masked neighbour values (BF16).
  auto fold = [&](const std::string &ns, TcWeights::Conv *zt) -> int {
    for (int k = 1; k < 4; ++k) {
      const std::string q = ns + ".s" + std::to_string(k) + ".";
      const std::vector<float> &wz = H(q + "wz"), &bz = H(q + "bz"), &wa = H(q + "wa"),
                               &ba = H(q + "ba");
      std::vector<float> wk((size_t)C * C, 0.f), bf(C);
      std::vector<__nv_bfloat16> wv((size_t)2 * C * 8, __float2bfloat16(0.f));  // [2][C][8]
      for (int c = 0; c < C; ++c) {
        double bacc = bz[c];
        for (int j = 0; j < C; ++j) {
          wk[(size_t)c * C + j] = wz[(size_t)c * 2 * C + C + j];
          bacc += (double)wz[(size_t)c * 2 * C + j] * ba[j];
        }
        bf[c] = (float)bacc;
        for (int tap = 0; tap < 9; ++tap) {
          double acc = 0.0;
          for (int j = 0; j < C; ++j) acc += (double)wz[(size_t)c * 2 * C + j] * wa[j * 9 + tap];
          wv[((size_t)(tap / 8) * C + c) * 8 + tap % 8] = __float2bfloat16((float)acc);
        }
      }
      int r;
      if ((r = pack_conv(*t, zt[k - 1], wk, bf, C, C, 1, C))) return r;
      if (cudaMalloc(&zt[k - 1].wv, wv.size() * 2) != cudaSuccess) {
        set_last_error("weight allocation failed");
        return PW_ENOMEM;
      }
      t->allocs.push_back(zt[k - 1].wv);
      cudaMemcpy(zt[k - 1].wv, wv.data(), wv.size() * 2, cudaMemcpyHostToDevice);
    }
    return PW_OK;
  };
  if ((s = fold("sb", t->sk_zt))) return s;
  if (ll_mode == 0 && (s = fold("ll", t->lk_zt))) return s;
  if (ll_mode == 0 &&
      (s = set("ll", t->l0_in, t->l0_w1, t->l0_w2, t->l0_w3, t->l0_w4, t->lk_c1, t->lk_c2)))
    return s;
  tc = t.release();
  return PW_OK;
}

// E4M3 copy of a convolution whose input channel k is stored as value *
// in_scale[k]: W'[n][k] = W[n][k] / in_scale[k], per output column
// sw[n] = max |W'[n][.]| / 448, stored E4M3(W' / sw) in the BF16 packing
// order with 16 channels per 16-byte group. The epilogue computes
// acc * sw[n] + b[n].
static int pack_conv_f8(TcWeights &tw, TcWeights::Conv &cv, const std::vector<float> &w,
                        const std::vector<float> &b, const std::vector<float> &in_scale,
                        int cout, int cin, int ks, int ncta, int kb,
                        std::vector<float> *sw_out = nullptr) {
  cv.cin = cin; cv.cout = cout; cv.ks = ks; cv.kb = kb; cv.ncta = ncta; cv.nb = cout / ncta;
  cv.f8 = true;
  const int taps = ks * ks, nkb = cin / kb, gpb = kb / 16;
  std::vector<float> sw(cout, 1.f);
  for (int n = 0; n < cout; ++n) {
    double mx = 0.0;
    for (int k = 0; k < cin; ++k)
      for (int t = 0; t < taps; ++t)
        mx = std::max(mx, std::fabs((double)w[((size_t)n * cin + k) * taps + t] / in_scale[k]));
    if (mx > 0.0) sw[n] = (float)(mx / 448.0);
  }
  std::vector<uint8_t> h((size_t)cout * cin * taps);
  size_t o = 0;
  for (int nb = 0; nb < cv.nb; ++nb)
    for (int kbi = 0; kbi < nkb; ++kbi)
      for (int t = 0; t < taps; ++t)
        for (int g = 0; g < gpb; ++g)
          for (int n = 0; n < ncta; ++n)
            for (int e = 0; e < 16; ++e) {
              const int co = nb * ncta + n, ci = kbi * kb + g * 16 + e;
              const float v = (float)((double)w[((size_t)co * cin + ci) * taps + t] /
                                      in_scale[ci] / sw[co]);
              h[o++] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
            }
  if (cudaMalloc(&cv.w, h.size()) != cudaSuccess || cudaMalloc(&cv.b, cout * 4) != cudaSuccess ||
      cudaMalloc(&cv.sw, cout * 4) != cudaSuccess) {
    set_last_error("weight allocation failed");
    return PW_ENOMEM;
  }
  tw.allocs.push_back(cv.w);
  tw.allocs.push_back(cv.b);
  tw.allocs.push_back(cv.sw);
  cudaMemcpy(cv.w, h.data(), h.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(cv.b, b.data(), cout * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(cv.sw, sw.data(), cout * 4, cudaMemcpyHostToDevice);
  if (sw_out) *sw_out = sw;
  return PW_OK;
}

// FP8 activation scales (stored E4M3 value = activation * scale), fixed per
// model from the weights alone: a root-mean-square estimate of every
// channel, propagated through the layers from assumed input magnitudes
// (quantised symbols RMS 8, l_i RMS 0.5), is mapped to 16. E4M3 then holds
// 28x that RMS before saturating and keeps full precision down to 1/1000 of
// it. l_i = h is bounded by 1 and is stored * 256.
int Model::ensure_fp8() {
  int s = ensure_tc();
  if (s) return s;
  if (tc->has_f8) return PW_OK;
  TcWeights &t = *tc;
  auto H = [&](const std::string &n) -> const std::vector<float> & { return host.at(n); };
  constexpr double kSigS = 8.0, kSigL = 0.5, kTarget = 16.0;
  auto dev = [&](const std::vector<float> &v, float **out) -> int {
    if (cudaMalloc(out, v.size() * 4) != cudaSuccess) return PW_ENOMEM;
    t.allocs.push_back(*out);
    cudaMemcpy(*out, v.data(), v.size() * 4, cudaMemcpyHostToDevice);
    return PW_OK;
  };
  std::vector<float> hs(C, 256.f);
  if ((s = dev(hs, &t.h_scale))) return s;
  {
    // gates: E4M3 h block (input scale hs), BF16 v block divided by the
    // h block's accumulator scale so that both accumulate on one scale
    std::vector<float> wh, sw;
    {
      std::vector<float> tmp;
      const std::vector<float> &wg = H("lstm.wg.perm");
      wh.assign((size_t)4 * C * C * 9, 0.f);
      for (int n = 0; n < 4 * C; ++n)
        for (int c = 0; c < C; ++c)
          for (int tp = 0; tp < 9; ++tp)
            wh[((size_t)n * C + c) * 9 + tp] = wg[((size_t)n * 2 * C + C + c) * 9 + tp];
    }
    if ((s = pack_conv_f8(t, t.gates8, wh, H("lstm.bg.perm"), hs, 4 * C, C, 3, 128, C, &sw)))
      return s;
    std::vector<float> unused;
    if ((s = pack_gates_v(t, t.gates8, H("lstm.wg.perm"), H("lstm.we"), H("lstm.be"), C, 128,
                          &sw, unused)))
      return s;
  }
  // steps 2-4: z = Wz [a; l] + bz (a = Wa (m s) + ba), u = lrelu(conv3x3 z)
  auto steps = [&](const std::string &ns, TcWeights::Conv *c1, TcWeights::Conv *c2,
                   float **zsc, float **usc) -> int {
    for (int k = 1; k < 4; ++k) {
      const std::string q = ns + ".s" + std::to_string(k) + ".";
      const std::vector<float> &wz = H(q + "wz"), &bz = H(q + "bz"), &wa = H(q + "wa"),
                               &ba = H(q + "ba"), &w1 = H(q + "w1"), &b1 = H(q + "b1");
      std::vector<double> sa(C), sz(C);
      for (int j = 0; j < C; ++j) {
        double v = (double)ba[j] * ba[j];
        for (int tap = 0; tap < 9; ++tap) v += (double)wa[j * 9 + tap] * wa[j * 9 + tap] * kSigS * kSigS;
        sa[j] = v;
      }
      std::vector<float> zs(C), us(C);
      for (int c = 0; c < C; ++c) {
        double v = (double)bz[c] * bz[c];
        for (int j = 0; j < C; ++j) {
          const double wa_ = wz[(size_t)c * 2 * C + j], wl = wz[(size_t)c * 2 * C + C + j];
          v += wa_ * wa_ * sa[j] + wl * wl * kSigL * kSigL;
        }
        sz[c] = v;
        zs[c] = (float)(kTarget / std::sqrt(std::max(v, 1e-12)));
      }
      for (int c = 0; c < C; ++c) {
        double v = (double)b1[c] * b1[c];
        for (int j = 0; j < C; ++j)
          for (int tap = 0; tap < 9; ++tap) {
            const double ww = w1[((size_t)c * C + j) * 9 + tap];
            v += ww * ww * sz[j];
          }
        us[c] = (float)(kTarget / std::sqrt(std::max(v, 1e-12)));
      }
      int r;
      if ((r = dev(zs, &zsc[k - 1])) || (r = dev(us, &usc[k - 1]))) return r;
      if ((r = pack_conv_f8(t, c1[k - 1], w1, b1, zs, C, C, 3, C, C))) return r;
      if ((r = pack_conv_f8(t, c2[k - 1], H(q + "w2"), H(q + "b2"), us, C, C, 3, C, C))) return r;
    }
    return PW_OK;
  };
  if ((s = steps("sb", t.sk_c1_8, t.sk_c2_8, t.sk_z_scale, t.sk_u_scale))) return s;
  if (ll_mode == 0 && (s = steps("ll", t.lk_c1_8, t.lk_c2_8, t.lk_z_scale, t.lk_u_scale)))
    return s;
  t.has_f8 = true;
  return PW_OK;
}

int Model::prepare(int precision) {
  if (mix && precision != PW_PREC_FP32) {
    set_last_error("logistic-mixture models run in the FP32 precision class only");
    return PW_EUNSUPPORTED;
  }
  if (precision == PW_PREC_INT8) {
    if (!intn) {
      set_last_error("the integer-network class needs a Laplace model loaded in an INT8 "
                     "context");
      return PW_EUNSUPPORTED;
    }
    return PW_OK;
  }
  if (precision == PW_PREC_FP32) return PW_OK;
  std::lock_guard<std::mutex> lk(mu);
  return precision == PW_PREC_FP8 ? ensure_fp8() : ensure_tc();
}

void Model::free_tc() {
  if (!tc) return;
  for (void *p : tc->allocs) cudaFree(p);
  delete tc;
  tc = nullptr;
}

// ---- workspace -----------------------------------------------------------
// Positions of the compact step-1 plane of an h x w subband (row pairs x
// step-1 positions per pair).
static int64_t compact_elems(int h, int w) {
  return (int64_t)((h + 1) >> 1) * (row_count(w, step_phase(0, 0)) + row_count(w, step_phase(0, 1)));
}

// Largest subband with its width rounded up to a multiple of 4 (the pitched
// u of the compact head), at least the largest plain subband.
static int64_t pitched_elems(const Geometry &g) {
  int64_t m = 0;
  for (int sb = 0; sb < g.nsb; ++sb)
    m = std::max(m, (int64_t)g.sh[sb] * std::max((g.sw[sb] + 3) & ~3, g.sw[sb]));
  return m;
}

int64_t tc_workspace_bytes(const Geometry &g, int P, int C, bool f8) {
  const int64_t big = (int64_t)P * g.sh.back() * g.sw.back();
  const int64_t big4 = (int64_t)P * pitched_elems(g);
  int64_t cmax = 0;
  for (int sb = 0; sb < g.nsb; ++sb) cmax = std::max(cmax, compact_elems(g.sh[sb], g.sw[sb]));
  cmax *= P;
  auto al = [](int64_t b) { return (b + 1023) / 1024 * 1024; };
  int64_t tot = 1024 + al(big * 2 * C * 2) + 4 * al(big * C * 2) +
                al(std::max(big * 2, big4) * C * 2) + al(big * C * 2) +
                3 * al(cmax * C * 2) + al(cmax * 2 * C * 2) + al(big * 32) + al(big * 32);
  if (f8) tot += al(big * 2 * C) + 3 * al(big * C) + al(big4 * C);
  return tot;
}

int tc_workspace_alloc(Workspace *ws, const Geometry &g, int C, bool f8) {
  const int64_t big = (int64_t)ws->P * g.sh.back() * g.sw.back();
  const int64_t big4 = (int64_t)ws->P * pitched_elems(g);
  int64_t cmax = 0;
  for (int sb = 0; sb < g.nsb; ++sb) cmax = std::max(cmax, compact_elems(g.sh[sb], g.sw[sb]));
  cmax *= ws->P;
  auto al = [](int64_t b) { return (b + 1023) / 1024 * 1024; };
  // X (2C), L0 (C), L1 (C), Z (C), U (2C), V (C), Z2 (C); compact Vc, Zc,
  // Z2c (C), U2c (2C); T (32); bf16. FP8: X8 (2C), L8 x 2, Z8, U8 (C) bytes.
  // U and U8 also hold the pitched input of the compact head (big4)
  constexpr int kN = 13, kN8 = 5;
  const int64_t sizes[kN] = {big * 2 * C * 2, big * C * 2,  big * C * 2,      big * C * 2,
                             std::max(big * 2, big4) * C * 2, big * C * 2,  big * C * 2,
                             cmax * C * 2,    cmax * C * 2, cmax * C * 2, cmax * 2 * C * 2,
                             big * 32,        big * 32};
  const int64_t sizes8[kN8] = {big * 2 * C, big * C, big * C, big * C, big4 * C};
  int64_t tot = 1024;
  for (int64_t v : sizes) tot += al(v);
  if (f8)
    for (int64_t v : sizes8) tot += al(v);
  TcAct *t = new TcAct();
  if (pool_alloc(&t->base, (size_t)tot, ws->stream) != PW_OK) {
    delete t;
    set_last_error("tensor-core workspace allocation failed");
    return PW_ENOMEM;
  }
  uint8_t *b = static_cast<uint8_t *>(t->base);
  t->err = reinterpret_cast<int *>(b);
  cudaMemsetAsync(t->err, 0, 1024, ws->stream);
  int64_t o = 1024;
  __nv_bfloat16 **dst[kN] = {&t->X,  &t->L[0], &t->L[1], &t->Z,   &t->U,  &t->V,
                             &t->Z2, &t->Vc,   &t->Zc,   &t->Z2c, &t->U2c, &t->T, &t->V16};
  for (int i = 0; i < kN; ++i) { *dst[i] = reinterpret_cast<__nv_bfloat16 *>(b + o); o += al(sizes[i]); }
  if (f8) {
    uint8_t **dst8[kN8] = {&t->X8, &t->L8[0], &t->L8[1], &t->Z8, &t->U8};
    for (int i = 0; i < kN8; ++i) { *dst8[i] = b + o; o += al(sizes8[i]); }
  }
  ws->tc = t;
  return PW_OK;
}

void tc_workspace_free(Workspace *ws) {
  TcAct *t = static_cast<TcAct *>(ws->tc);
  if (!t) return;
  pool_free(t->base, ws->stream);
  delete t;
  ws->tc = nullptr;
}

int tc_run_lstm(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws, int sb,
                const int32_t *sprev, int up, int first, int cur) {
  TcAct &t = *static_cast<TcAct *>(ws.tc);
  const bool f8 = ctx->precision == PW_PREC_FP8;
  const int h = g.sh[sb], w = g.sw[sb], C = m.C, P = ws.P, G = C / 8, G16 = C / 16;
  const double pix = (double)P * h * w;
  __nv_bfloat16 *lprev = t.L[(sb - 1) & 1], *lout = t.L[sb & 1];
  const TcWeights::Conv &gates = f8 ? m.tc->gates8 : m.tc->gates;
  // h_{i-1} is copied (upsampled, or zeros for the first subband) into the
  // second half of X / X8 when it is not at this resolution; otherwise the
  // gates conv reads it from the previous l buffer directly
  const int copy_h = (up || first) ? 1 : 0;
  {
    ProfScope ps(ctx, KC_SMALL_CTX, 0.0, pix * (4.0 + 32.0 + (copy_h ? (f8 ? 2.0 : 4.0) * C : 0)));
    k_lstm_v<<<P * h, 256, 0, ctx->stream>>>(sprev, t.V16, P, h, w, up);
    ctx->launches += 1;
    if (ws.ext) {  // ragged batch: the gates conv reads v over 3 x 3 neighbourhoods
      launch_zero_outside(t.V16, ZL_GROUP, P, h, w, 2, ws.ext, sb_level(g, sb), ctx->stream);
      ctx->launches += 1;
    }
    if (copy_h) {
      if (f8)
        k_copy_up16<<<P * h, 256, 0, ctx->stream>>>(
            reinterpret_cast<const uint4 *>(t.L8[(sb - 1) & 1]), G16,
            reinterpret_cast<uint4 *>(t.X8), 2 * G16, G16, G16, P, h, w, up, first);
      else
        k_copy_up16<<<P * h, 256, 0, ctx->stream>>>(
            reinterpret_cast<const uint4 *>(lprev), G, reinterpret_cast<uint4 *>(t.X), 2 * G, G,
            G, P, h, w, up, first);
      ctx->launches += 1;
    }
  }
  TcConvArgs a{};
  a.epi = TE_LSTM;
  a.out = lout; a.out_G = G; a.out_goff = 0;
  // the cell state is BF16 on the tensor-core path (half the bytes of the
  // FP32 buffers it lives in)
  a.c_prev = reinterpret_cast<const __nv_bfloat16 *>(ws.Cst[cur]);
  a.c_new = reinterpret_cast<__nv_bfloat16 *>(ws.Cst[cur ^ 1]);
  a.up = up; a.first = first; a.C = C;
  if (f8) { a.out8 = t.L8[sb & 1]; a.out8_G16 = G16; a.out8_scale = m.tc->h_scale; }
  // MMA work: the 16-channel v block and the C h channels, 9 taps, 4C outputs
  ProfScope ps(ctx, KC_LSTM_GATES, 2.0 * pix * 9 * (16 + C) * 4 * C,
               pix * (32.0 + (f8 ? 1.0 : 2.0) * C + 2.0 * C + 4.0 * C + (f8 ? C : 0)));
  int s;
  if (f8) {
    if (copy_h) s = conv_tc(ctx, gates, t.V16, 2, 0, P, h, w, a, t.err, t.X8, 2 * G16, G16, 0);
    else s = conv_tc(ctx, gates, t.V16, 2, 0, P, h, w, a, t.err, t.L8[(sb - 1) & 1], G16, 0, 0);
  } else {
    if (copy_h) s = conv_tc(ctx, gates, t.V16, 2, 0, P, h, w, a, t.err, t.X, 2 * G, G, 0);
    else s = conv_tc(ctx, gates, t.V16, 2, 0, P, h, w, a, t.err, lprev, G, 0, 0);
  }
  if (s == PW_OK && ws.ext) {
    // ragged batch: h feeds the next gates conv over 3 x 3 neighbourhoods
    launch_zero_outside(lout, ZL_GROUP, P, h, w, G, ws.ext, sb_level(g, sb), ctx->stream);
    if (f8) launch_zero_outside(t.L8[sb & 1], ZL_GROUP, P, h, w, G16, ws.ext, sb_level(g, sb),
                                ctx->stream);
    ctx->launches += f8 ? 2 : 1;
  }
  return s;
}

int tc_run_step(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws, int sb, int step,
                StepNetDev &n, const int32_t *Qi, uint32_t *idx, int64_t nk, float *mu,
                float *sgp) {
  TcAct &t = *static_cast<TcAct *>(ws.tc);
  TcWeights &W = *m.tc;
  const bool ll = sb == 0;
  const int h = g.sh[sb], w = g.sw[sb], C = m.C, P = ws.P, G = C / 8;
  cudaStream_t st = ctx->stream;
  const double pix = (double)P * h * w;
  __nv_bfloat16 *l = t.L[sb & 1];
  auto conv = [&](const TcWeights::Conv &cv, const __nv_bfloat16 *in, int in_G, int in_goff,
                  TcConvArgs a, double extra_flops) {
    ProfScope ps(ctx, cv.ks == 3 ? KC_CONV3 : KC_CONV1,
                 2.0 * pix * cv.ks * cv.ks * cv.cin * cv.cout + extra_flops,
                 pix * 2.0 * (cv.cin + cv.cout + (a.res ? cv.cout : 0)));
    return conv_tc(ctx, cv, in, in_G, in_goff, P, h, w, a, t.err);
  };
  int s;
  // ragged batch: zero a buffer outside the planes' extents before a
  // spatial convolution reads it (NG 16-byte units per position)
  auto mask = [&](void *buf, int layout, int NG) {
    if (!ws.ext) return;
    launch_zero_outside(buf, layout, P, h, w, NG, ws.ext, sb_level(g, sb), st);
    ctx->launches += 1;
  };
  if (ll && step == 0) {  // l = 0 for LL
    cudaMemsetAsync(l, 0, (size_t)P * h * w * C * 2, st);
    if (ctx->precision == PW_PREC_FP8) cudaMemsetAsync(t.L8[sb & 1], 0, (size_t)P * h * w * C, st);
  }
  if (step == 0) {
    const TcWeights::Conv &cin_ = ll ? W.l0_in : W.s0_in, &c1 = ll ? W.l0_w1 : W.s0_w1,
                          &c2 = ll ? W.l0_w2 : W.s0_w2, &c3 = ll ? W.l0_w3 : W.s0_w3,
                          &c4 = ll ? W.l0_w4 : W.s0_w4;
    TcConvArgs a{};
    a.epi = TE_STORE; a.act = 1; a.out = t.U; a.out_G = G;
    if ((s = conv(c1, l, G, 0, a, 0))) return s;                   // u = lrelu(W1 Win l + .)
    mask(t.U, ZL_GROUP, G);
    // Everything after the depthwise conv is per position and only the
    // step-1 positions' parameters are used: run it on those alone, in the
    // compact layout (hc row pairs x wc positions per pair).
    const int hc = (h + 1) >> 1;
    const int wc = row_count(w, step_phase(0, 0)) + row_count(w, step_phase(0, 1));
    const int n0 = step_count(h, w, 0);
    const int64_t chw = (int64_t)hc * wc;
    const double cpix = (double)P * n0;
    auto cconv = [&](const TcWeights::Conv &cv, const __nv_bfloat16 *in, int in_G,
                     TcConvArgs a2) {
      ProfScope ps(ctx, KC_CONV1, 2.0 * cpix * cv.cin * cv.cout,
                   cpix * 2.0 * (cv.cin + cv.cout + (a2.res ? cv.cout : 0)));
      return conv_tc(ctx, cv, in, in_G, 0, P, hc, wc, a2, t.err);
    };
    {
      ProfScope ps(ctx, KC_SMALL_CTX, 2.0 * cpix * 9 * C, cpix * 2.0 * C * 4);
      k_dw3x3_compact<<<P * hc, 256, 0, st>>>(
          t.U, l, n.wdw, n.bdw, t.Vc, t.Zc, P, h, w, C, 0, n0, chw);  // Zc <- l gathered
      ctx->launches += 1;
    }
    // the block input z = Win l + bin on the step-1 positions (compact, in Z)
    a = TcConvArgs{}; a.epi = TE_STORE; a.out = t.Z; a.out_G = G;
    if ((s = cconv(cin_, t.Zc, G, a))) return s;
    a = TcConvArgs{}; a.epi = TE_STORE; a.out = t.Z2c; a.out_G = G; a.res = t.Z; a.res_G = G;
    if ((s = cconv(c2, t.Vc, G, a))) return s;                     // z2 = z + 1x1(v)
    a = TcConvArgs{}; a.epi = TE_STORE; a.act = 1; a.out = t.U2c; a.out_G = 2 * G;
    if ((s = cconv(c3, t.Z2c, G, a))) return s;                    // u2 = lrelu(1x1 z2)
    a = TcConvArgs{}; a.epi = TE_HEAD; a.res = t.Z2c; a.res_G = G;
    a.wh = n.wh; a.bh = n.bh; a.step = 0; a.idx = idx; a.idx_stride = nk;
    a.mu_out = mu; a.sg_out = sgp;
    a.compact_n = n0; a.full_W = w; a.full_H = h;
    return cconv(c4, t.U2c, 2 * G, a);                             // head
  }
  const TcWeights::Conv &zt = ll ? W.lk_zt[step - 1] : W.sk_zt[step - 1];
  const bool f8 = ctx->precision == PW_PREC_FP8;
  const TcWeights::Conv &c1 = f8 ? (ll ? W.lk_c1_8[step - 1] : W.sk_c1_8[step - 1])
                                 : (ll ? W.lk_c1[step - 1] : W.sk_c1[step - 1]);
  const TcWeights::Conv &c2 = f8 ? (ll ? W.lk_c2_8[step - 1] : W.sk_c2_8[step - 1])
                                 : (ll ? W.lk_c2[step - 1] : W.sk_c2[step - 1]);
  const float *zsc = ll ? W.lk_z_scale[step - 1] : W.sk_z_scale[step - 1];
  const float *usc = ll ? W.lk_u_scale[step - 1] : W.sk_u_scale[step - 1];
  const int G16 = C / 16;
  {
    ProfScope ps(ctx, KC_SMALL_CTX, 0.0, pix * (4.0 + 32.0));
    k_masked_taps<<<P * h, 128, 0, st>>>(Qi, t.T, P, h, w, step);   // T: 16 channels
    ctx->launches += 1;
  }
  TcConvArgs a{};
  a.epi = TE_STORE; a.out = t.Z; a.out_G = G;
  // FP8: the residual-block input feeds conv 1 as E4M3 and the head's
  // residual as a dense BF16 copy of this step's positions (in Zc)
  if (f8) {
    a.out = nullptr; a.out8 = t.Z8; a.out8_G16 = G16; a.out8_scale = zsc;
    a.outc = t.Zc; a.outc_n = (int)nk; a.step = step;
  }
  {
    // z = 1x1 over [T (v block, 16 BF16 channels), l (C channels)]
    ProfScope ps(ctx, KC_CONV1, 2.0 * pix * (16 + zt.cin) * zt.cout,
                 pix * (32.0 + 2.0 * zt.cin + (f8 ? C + C / 2 : 2.0 * zt.cout)));
    if ((s = conv_tc(ctx, zt, t.T, 2, 0, P, h, w, a, t.err, l, G, 0, 0))) return s;
  }
  if (f8) mask(t.Z8, ZL_GROUP, G16);
  else mask(t.Z, ZL_GROUP, G);
  // The head conv's outputs are used at this step's positions only (a
  // quarter of the plane): where the subband is large enough it runs on
  // those alone (TE_HEADC), reading u in the phase-split layout.
  const bool hcm = headc_ok(h, w);
  const int ups = hcm ? 1 : 0;
  const double kpix = hcm ? (double)P * nk : pix;   // positions the head computes
  if (f8) {
    a = TcConvArgs{}; a.epi = TE_STORE; a.act = 1; a.out = nullptr; a.out_G = G;
    a.out8 = t.U8; a.out8_G16 = G16; a.out8_scale = usc; a.out_ps = ups;
    {
      ProfScope ps(ctx, KC_CONV3, 2.0 * pix * 9 * C * C, pix * 2.0 * C);
      if ((s = conv_tc(ctx, c1, t.Z8, G16, 0, P, h, w, a, t.err))) return s;  // u = lrelu(3x3 z)
    }
    mask(t.U8, ups ? ZL_PHASE : ZL_GROUP, G16);
    a = TcConvArgs{}; a.epi = hcm ? TE_HEADC : TE_HEAD; a.res = t.Zc; a.res_G = G;
    a.res_compact_n = (int)nk;
    a.wh = n.wh; a.bh = n.bh; a.step = step; a.idx = idx; a.idx_stride = nk;
    a.mu_out = mu; a.sg_out = sgp;
    ProfScope ps(ctx, KC_HEAD3, 2.0 * kpix * 9 * C * C, pix * C + kpix * 2.0 * C);
    return conv_tc(ctx, c2, t.U8, G16, 0, P, h, w, a, t.err);               // head
  }
  a = TcConvArgs{}; a.epi = TE_STORE; a.act = 1; a.out = t.U; a.out_G = G; a.out_ps = ups;
  if ((s = conv(c1, t.Z, G, 0, a, 0))) return s;                  // u = lrelu(conv3x3 z)
  mask(t.U, ups ? ZL_PHASE : ZL_GROUP, G);
  a = TcConvArgs{}; a.epi = hcm ? TE_HEADC : TE_HEAD; a.res = t.Z; a.res_G = G;
  a.wh = n.wh; a.bh = n.bh; a.step = step; a.idx = idx; a.idx_stride = nk;
  a.mu_out = mu; a.sg_out = sgp;
  ProfScope ps(ctx, KC_HEAD3, 2.0 * kpix * 9 * C * C, pix * 2.0 * C + kpix * 4.0 * C);
  return conv_tc(ctx, c2, t.U, G, 0, P, h, w, a, t.err);          // head
}

// Stage entry: one tensor-core convolution on host data (testing).
int tc_conv_host(pw_ctx *ctx, int P, int H, int W, int cin, int cout, int ks, int act,
                 const float *x, const float *w, const float *b, float *y) {
  if (!(ks == 1 || ks == 3) || cin % 32 || (cin > 64 && cin % 64) ||
      (cout != 32 && cout != 64 && cout != 128 && cout != 192 && cout != 256) ||
      P < 1 || H < 1 || W < 1) {
    set_last_error("unsupported convolution shape");
    return PW_EUNSUPPORTED;
  }
  TcWeights tw;
  TcWeights::Conv cv;
  const int ncta = cout <= 128 ? cout : 64;
  std::vector<float> wv(w, w + (size_t)cout * cin * ks * ks), bv(b, b + cout);
  int s = pack_conv(tw, cv, wv, bv, cout, cin, ks, ncta);
  if (s) { for (void *q : tw.allocs) cudaFree(q); return s; }
  const int Gi = cin / 8, Go = cout / 8;
  const int64_t hw = (int64_t)H * W;
  std::vector<__nv_bfloat16> xb((size_t)P * cin * hw);
  for (int p = 0; p < P; ++p)
    for (int64_t i = 0; i < hw; ++i)
      for (int c = 0; c < cin; ++c)
        xb[(((size_t)p * Gi + c / 8) * hw + i) * 8 + c % 8] =
            __float2bfloat16(x[((size_t)p * hw + i) * cin + c]);
  void *dx = nullptr, *dy = nullptr, *derr = nullptr;
  const size_t ybytes = (size_t)P * cout * hw * 2;
  if (cudaMalloc(&dx, xb.size() * 2) != cudaSuccess || cudaMalloc(&dy, ybytes) != cudaSuccess ||
      cudaMalloc(&derr, 16) != cudaSuccess) {
    cudaFree(dx); cudaFree(dy); cudaFree(derr);
    for (void *q : tw.allocs) cudaFree(q);
    set_last_error("allocation failed");
    return PW_ENOMEM;
  }
  cudaMemcpy(dx, xb.data(), xb.size() * 2, cudaMemcpyHostToDevice);
  cudaMemset(dy, 0, ybytes);
  cudaMemset(derr, 0, 16);
  TcConvArgs a{};
  a.epi = TE_STORE; a.act = act; a.out = (__nv_bfloat16 *)dy; a.out_G = Go;
  s = conv_tc(ctx, cv, (const __nv_bfloat16 *)dx, Gi, 0, P, H, W, a, (int *)derr);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  int err = 0;
  if (e == cudaSuccess) cudaMemcpy(&err, derr, 4, cudaMemcpyDeviceToHost);
  if (s == PW_OK && e == cudaSuccess && !err) {
    std::vector<__nv_bfloat16> yb((size_t)P * cout * hw);
    cudaMemcpy(yb.data(), dy, ybytes, cudaMemcpyDeviceToHost);
    for (int p = 0; p < P; ++p)
      for (int64_t i = 0; i < hw; ++i)
        for (int c = 0; c < cout; ++c)
          y[((size_t)p * hw + i) * cout + c] =
              __bfloat162float(yb[(((size_t)p * Go + c / 8) * hw + i) * 8 + c % 8]);
  }
  cudaFree(dx); cudaFree(dy); cudaFree(derr);
  for (void *q : tw.allocs) cudaFree(q);
  if (s) return s;
  if (e != cudaSuccess) { set_last_error(std::string("CUDA: ") + cudaGetErrorString(e)); return PW_ECUDA; }
  if (err) { set_last_error("tensor-core convolution timed out (bounded wait expired)"); return PW_ETIMEOUT; }
  return PW_OK;
}

void tc_error_reset(Workspace &ws, cudaStream_t st) {
  TcAct *t = static_cast<TcAct *>(ws.tc);
  if (t) cudaMemsetAsync(t->err, 0, 4, st);
}

int tc_error(Workspace &ws) {
  TcAct *t = static_cast<TcAct *>(ws.tc);
  if (!t) return 0;
  int e = 0;
  cudaMemcpy(&e, t->err, 4, cudaMemcpyDeviceToHost);
  return e;
}

}  // namespace pw
