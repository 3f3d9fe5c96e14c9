// CNN lifting wavelet transform (Section 3.1, Fig. 2), temporal lifting
// (Section 3.3), colour conversion and the scalar quantiser.
//
// One lifting half-step computes v = lin(src) + CNN(src) along a direction
// and writes out = other + sign * v; the inverse transform runs the steps
// of the forward transform backwards, so it reconstructs perfectly for any
// network weights. The CNN residual is conv3x3(1->16), tanh,
// conv3x3(16->16), tanh, conv3x3(16->1) with zero padding, fused in one
// kernel per 16x16 output tile (halo of 3, all activations in shared
// memory). Linear parts: LeGall 5/3 (P = (s[n] + s[n+1]) / 2,
// U = (s[n-1] + s[n]) / 4, edges clamped = whole-sample symmetric) for the
// spatial transform; Haar (P = s, U = s / 2) for the temporal one. Integer
// mode (lossless) rounds P with floor(v) and U with floor(v + 1/2), which
// makes the transform the JPEG 2000 reversible 5/3 when the CNN is zero.
//
// An integer lifting step reconstructs exactly only if encoder and decoder
// round the same P and U values, so in integer mode the CNN is evaluated as
// a fixed sequence of FP32 operations that any IEEE implementation
// reproduces bit for bit: every layer starts from its bias and adds, tap by
// tap in raster order (dy, dx) and within a tap input channel by input
// channel in ascending order, the product w * x (product and sum each
// rounded to nearest even, never fused), the activation is tanh32_spec, and
// v = lin + CNN is one rounded addition before the floor. The lossy steps
// keep fused multiply-adds and the CUDA tanh.
#include <cuda_bf16.h>

#include <mutex>

#include "pw_internal.cuh"
#include "lift_kernels.cuh"
#include "spec_math.cuh"
#include "f32x2.cuh"
#include "tc_ptx.cuh"

namespace pw {

constexpr int LT = 16;            // output tile
constexpr int LF = 16;            // CNN channels
constexpr int L1 = LT + 4;        // layer-1 region (20)
constexpr int L2 = LT + 2;        // layer-2 region (18)
constexpr int LI = LT + 6;        // input region (22)

// Shared memory of one tile. Weights are stored tap-major with the output
// (or input) channel innermost so that 16 of them come in four broadcast
// 128-bit loads: w1t[tap][c], w2t[tap][ci][c], w3t[tap][ci].
struct LiftSmem {
  alignas(16) float in[LI * LI];
  alignas(16) float a1[L1 * L1 * LF];
  alignas(16) float a2[L2 * L2 * LF];
  alignas(16) float w1t[9 * LF];
  alignas(16) float w2t[9 * LF * LF];
  alignas(16) float w3t[9 * LF];
  alignas(16) float b1[LF];
  alignas(16) float b2[LF];
  alignas(16) float b3[4];
};

__device__ __forceinline__ void ld16(const float *p, float *v) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 f = q[i];
    v[4 * i] = f.x; v[4 * i + 1] = f.y; v[4 * i + 2] = f.z; v[4 * i + 3] = f.w;
  }
}

// acc + w * x: one fused multiply-add, or (kExact) a rounded product and a
// rounded sum; the activation: CUDA's tanhf, or (kExact) tanh32_spec.
template <bool kExact>
__device__ __forceinline__ float mac(float acc, float w, float x) {
  return kExact ? __fadd_rn(acc, __fmul_rn(w, x)) : fmaf(w, x, acc);
}
template <bool kExact>
__device__ __forceinline__ float act(float v) {
  return kExact ? tanh32_spec(v) : tanhf(v);
}

// Two accumulators of mac<kExact> at once (per element the same operations:
// a fused multiply-add, or (kExact) a rounded product and a rounded sum).
template <bool kExact>
__device__ __forceinline__ uint64_t mac2(uint64_t acc, uint64_t w, uint64_t x) {
  return kExact ? add2(acc, mul2(w, x)) : fma2(w, x, acc);
}

__device__ __forceinline__ float acc_get(const PlaneAcc &a, int p, int y, int x) {
  return a.p[(int64_t)p * a.ps + (int64_t)y * a.rs + (int64_t)x * a.cs];
}
__device__ __forceinline__ void acc_set(const PlaneAcc &a, int p, int y, int x, float v) {
  a.p[(int64_t)p * a.ps + (int64_t)y * a.rs + (int64_t)x * a.cs] = v;
}

// Layer 3 of the CNN (conv3x3 16 -> 1 over the 18 x 18 layer-2 region a2,
// null when the step has no CNN), the linear part and the output of one
// 16 x 16 tile; thread t handles output (t / 16, t % 16). in: the 22 x 22
// input region (origin y0 - 3, x0 - 3).
// rout (optional): the CNN residual of the tile's outputs, already computed.
template <bool kExact>
__device__ __forceinline__ void lift_finish(const LiftStepParams &a, int p, int H, int W, int y0,
                                            int x0, const float *in, const float *a2,
                                            const float *w3t, const float *b3,
                                            const float *rout = nullptr) {
  const int t = threadIdx.x;
  const int ly = t / LT, lx = t % LT;
  float r_out = 0.f;
  if (rout) {
    r_out = rout[t];
  } else if (a2) {
    float v = b3[0];
    for (int tap = 0; tap < 9; ++tap) {
      float xv[LF], w[LF];
      ld16(a2 + ((ly + tap / 3) * L2 + lx + tap % 3) * LF, xv);
      ld16(w3t + tap * LF, w);
#pragma unroll
      for (int ci = 0; ci < LF; ++ci) v = mac<kExact>(v, w[ci], xv[ci]);
    }
    r_out = v;
  }
  const int y = y0 + ly, x = x0 + lx;
  if (y >= H || x >= W) return;
  const float s0 = in[(ly + 3) * LI + lx + 3];
  float lin;
  if (a.lin == LIN_P53) {
    const float s1 = a.dir == 0 ? (x + 1 < W ? in[(ly + 3) * LI + lx + 4] : s0)
                                : (y + 1 < H ? in[(ly + 4) * LI + lx + 3] : s0);
    lin = 0.5f * (s0 + s1);
  } else if (a.lin == LIN_U53) {
    const float sm = a.dir == 0 ? (x > 0 ? in[(ly + 3) * LI + lx + 2] : s0)
                                : (y > 0 ? in[(ly + 2) * LI + lx + 3] : s0);
    lin = 0.25f * (sm + s0);
  } else if (a.lin == LIN_ID) {
    lin = s0;
  } else if (a.lin == LIN_HALF) {
    lin = 0.5f * s0;
  } else {  // LIN_ZERO: the CNN alone (post-processing)
    lin = 0.f;
  }
  float v = kExact ? __fadd_rn(lin, r_out) : lin + r_out;
  if (a.round == 1) v = floorf(v);
  else if (a.round == 2) v = floorf(v + 0.5f);
  const float o = acc_get(a.other, p, y, x);
  acc_set(a.out, p, y, x, a.sign > 0 ? o + v : o - v);
  if (a.copy.p) acc_set(a.copy, p, y, x, s0);
}

template <bool kExact>
__global__ void __launch_bounds__(256) k_lift_step(LiftStepParams a) {
  extern __shared__ float smem_raw[];
  LiftSmem &S = *reinterpret_cast<LiftSmem *>(smem_raw);
  const int t = threadIdx.x;
  const int p = blockIdx.z;
  const int tiles_x = (a.W + LT - 1) / LT;
  const int y0 = (blockIdx.x / tiles_x) * LT, x0 = (blockIdx.x % tiles_x) * LT;
  const bool cnn = a.net.w1 != nullptr;
  int H, W;
  lift_extent(a, p, H, W);
  if (y0 >= H || x0 >= W) return;  // a tile beyond this plane of a ragged batch

  for (int e = t; e < LI * LI; e += 256) {
    int yy = y0 + e / LI - 3, xx = x0 + e % LI - 3;
    S.in[e] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? acc_get(a.src, p, yy, xx) : 0.f;
  }
  if (cnn) {
    for (int e = t; e < LF * 9; e += 256) {
      const int c = e / 9, tap = e % 9;  // source [c][tap]
      S.w1t[tap * LF + c] = a.net.w1[e];
      S.w3t[tap * LF + c] = a.net.w3[e];
    }
    for (int e = t; e < LF * LF * 9; e += 256) {
      const int c = e / (LF * 9), ci = (e / 9) % LF, tap = e % 9;  // source [c][ci][tap]
      S.w2t[(tap * LF + ci) * LF + c] = a.net.w2[e];
    }
    if (t < LF) { S.b1[t] = a.net.b1[t]; S.b2[t] = a.net.b2[t]; }
    if (t == 0) S.b3[0] = a.net.b3[0];
  }
  __syncthreads();
  if (cnn) {
    // layer 1 on the 20 x 20 region (origin y0 - 2, x0 - 2)
    for (int e = t; e < L1 * L1; e += 256) {
      const int ly = e / L1, lx = e % L1;
      const int yy = y0 + ly - 2, xx = x0 + lx - 2;
      const bool inside = yy >= 0 && yy < H && xx >= 0 && xx < W;
      // output channels in pairs (packed FP32): each accumulator sees the
      // same sequence of operations as one mac<kExact> chain
      uint64_t accp[LF / 2];
#pragma unroll
      for (int c = 0; c < LF / 2; ++c) accp[c] = f2pack(S.b1[2 * c], S.b1[2 * c + 1]);
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const float iv = S.in[(ly + tap / 3) * LI + lx + tap % 3];
        const uint64_t xv = f2pack(iv, iv);
        const uint64_t *wp = reinterpret_cast<const uint64_t *>(S.w1t + tap * LF);
#pragma unroll
        for (int c = 0; c < LF / 2; ++c) accp[c] = mac2<kExact>(accp[c], wp[c], xv);
      }
      float acc[LF];
#pragma unroll
      for (int c = 0; c < LF / 2; ++c) f2unpack(accp[c], acc[2 * c], acc[2 * c + 1]);
      float4 *dst = reinterpret_cast<float4 *>(S.a1 + e * LF);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        dst[i] = inside ? make_float4(act<kExact>(acc[4 * i]), act<kExact>(acc[4 * i + 1]),
                                      act<kExact>(acc[4 * i + 2]), act<kExact>(acc[4 * i + 3]))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    // layer 2 on the 18 x 18 region (origin y0 - 1, x0 - 1): 324 positions,
    // two per thread (threads 0..161) so that every weight load feeds 32 FMAs
    constexpr int kHalf = L2 * L2 / 2;
    if (t < kHalf) {
      const int e0 = t, e1 = t + kHalf;
      const int ly0 = e0 / L2, lx0 = e0 % L2, ly1 = e1 / L2, lx1 = e1 % L2;
      // output channels in pairs (packed FP32), as in layer 1
      uint64_t p0[LF / 2], p1[LF / 2];
#pragma unroll
      for (int c = 0; c < LF / 2; ++c) p0[c] = p1[c] = f2pack(S.b2[2 * c], S.b2[2 * c + 1]);
      for (int tap = 0; tap < 9; ++tap) {
        float in0v[LF], in1v[LF];
        ld16(S.a1 + ((ly0 + tap / 3) * L1 + lx0 + tap % 3) * LF, in0v);
        ld16(S.a1 + ((ly1 + tap / 3) * L1 + lx1 + tap % 3) * LF, in1v);
#pragma unroll
        for (int ci = 0; ci < LF; ++ci) {
          const uint64_t *wp = reinterpret_cast<const uint64_t *>(S.w2t + (tap * LF + ci) * LF);
          const uint64_t x0 = f2pack(in0v[ci], in0v[ci]), x1 = f2pack(in1v[ci], in1v[ci]);
#pragma unroll
          for (int c = 0; c < LF / 2; ++c) {
            const uint64_t w = wp[c];
            p0[c] = mac2<kExact>(p0[c], w, x0);
            p1[c] = mac2<kExact>(p1[c], w, x1);
          }
        }
      }
      float acc0[LF], acc1[LF];
#pragma unroll
      for (int c = 0; c < LF / 2; ++c) {
        f2unpack(p0[c], acc0[2 * c], acc0[2 * c + 1]);
        f2unpack(p1[c], acc1[2 * c], acc1[2 * c + 1]);
      }
      const int yy0 = y0 + ly0 - 1, xx0 = x0 + lx0 - 1, yy1 = y0 + ly1 - 1, xx1 = x0 + lx1 - 1;
      const bool in0 = yy0 >= 0 && yy0 < H && xx0 >= 0 && xx0 < W;
      const bool in1 = yy1 >= 0 && yy1 < H && xx1 >= 0 && xx1 < W;
      float4 *d0 = reinterpret_cast<float4 *>(S.a2 + e0 * LF);
      float4 *d1 = reinterpret_cast<float4 *>(S.a2 + e1 * LF);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        d0[i] = in0 ? make_float4(act<kExact>(acc0[4 * i]), act<kExact>(acc0[4 * i + 1]),
                                  act<kExact>(acc0[4 * i + 2]), act<kExact>(acc0[4 * i + 3]))
                    : make_float4(0.f, 0.f, 0.f, 0.f);
        d1[i] = in1 ? make_float4(act<kExact>(acc1[4 * i]), act<kExact>(acc1[4 * i + 1]),
                                  act<kExact>(acc1[4 * i + 2]), act<kExact>(acc1[4 * i + 3]))
                    : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
  }
  lift_finish<kExact>(a, p, H, W, y0, x0, S.in, cnn ? S.a2 : nullptr, S.w3t, S.b3);
}

// ---------------------------------------------------------------------------
// Lifting step with the CNN's second and third layers (conv3x3 16 -> 16 and
// 16 -> 1, 95 % of its FLOPs) on the tensor cores: BF16 operands, FP32
// accumulation in tensor memory. Layer 1, the linear part and the output
// stay FP32.
//
// Rows of every GEMM are positions of a region laid out with a row stride of
// RS = 24 positions: row m = r * RS + c. Layer 1 (20 x 20 region) and layer 2
// (18 x 18) are stored as BF16 slabs with that stride, so tap (dy, dx) of row
// m reads position m + dy * RS + dx of the layer below: each tap is one MMA
// per 128-row block whose A operand is the slab shifted by a constant
// (columns c >= 18, resp. 16, are padding whose results are never used).
// Slabs: [2 channel groups][positions][8] BF16 (K-major core matrices, no
// swizzle); B: [tap][2][16 outputs][8] (layer 3: output 0 only, rest zero).
constexpr int kRS = 24;                   // row stride of the regions
constexpr int kMT = 4;                    // layer-2 blocks (18 * 24 = 432 rows)
constexpr int kMT3 = 3;                   // layer-3 blocks (16 * 24 = 384 rows)
constexpr int kA = 576;                   // layer-1 positions kept (> 511 + 2 * 24 + 2)
constexpr int kA2 = 448;                  // layer-2 positions kept (> 383 + 2 * 24 + 2)

struct LiftTcSmem {
  // layer-1 slab; once the layer-2 MMAs have completed, the layer-2 slab
  // (2 * kA2 * 8 elements) is written over it
  alignas(128) __nv_bfloat16 a1[2 * kA * 8];
  alignas(128) __nv_bfloat16 w2[9 * 2 * LF * 8];
  alignas(128) __nv_bfloat16 w3[9 * 2 * LF * 8];
  alignas(16) float in[LI * LI];
  alignas(16) float rout[LT * LT];
  alignas(16) float w1t[9 * LF];
  alignas(16) float b1[LF];
  alignas(16) float b2[LF];
  alignas(8) uint64_t bar;
  uint32_t tmem;
  float b3;
};

// Bounded wait of every thread for completion phase `parity` of the MMA
// barrier (lane 0 polls, the rest follow); false on expiry.
__device__ __forceinline__ bool lift_mma_wait(uint64_t *bar, uint32_t parity) {
  const int lane = threadIdx.x & 31;
  int ok = 1;
  if (lane == 0) {
    // suspended try_wait: the waiting warps leave the issue slots to the
    // other CTAs' warps on the SM instead of spinning
    const long long t0 = clock64();
    while (!mbar_try_sleep(bar, parity, 2000u))
      if (clock64() - t0 > kWaitCycles) { ok = 0; break; }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && lane != 0) while (!mbar_try(bar, parity)) {}
  __syncwarp();
  fence_after();
  return ok != 0;
}

// (six resident CTAs per SM: 40 registers instead of 48, which allowed five;
// lifting class 4.50 -> 4.45 ms per batch of 24)
__global__ void __launch_bounds__(256, 6) k_lift_tc(LiftStepParams a) {
  extern __shared__ __align__(1024) uint8_t lsm_raw[];
  LiftTcSmem &S = *reinterpret_cast<LiftTcSmem *>(lsm_raw);
  __nv_bfloat16 *const a2 = S.a1;   // layer-2 slab over the consumed layer-1 slab
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int p = blockIdx.z;
  const int tiles_x = (a.W + LT - 1) / LT;
  const int y0 = (blockIdx.x / tiles_x) * LT, x0 = (blockIdx.x % tiles_x) * LT;
  int H, W;
  lift_extent(a, p, H, W);
  if (y0 >= H || x0 >= W) return;  // a tile beyond this plane of a ragged batch (uniform)
  // TMEM columns: layer 2 in [0, 64) (4 blocks x 16), then layer 3 in
  // [0, 48) once the layer-2 epilogue has read them
  constexpr uint32_t kCols = 64;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 32) {
    mbar_init(&S.bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = t; e < LI * LI; e += 256) {
    const int yy = y0 + e / LI - 3, xx = x0 + e % LI - 3;
    S.in[e] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? acc_get(a.src, p, yy, xx) : 0.f;
  }
  for (int e = t; e < LF * 9; e += 256) {
    const int c = e / 9, tap = e % 9;  // source [c][tap]
    S.w1t[tap * LF + c] = a.net.w1[e];
  }
  {
    // the packed B operands of layers 2 and 3 (9 x 2 x 16 x 8 BF16 each)
    constexpr int kB16 = 9 * 2 * LF * 8 * 2 / 16;
    const uint4 *src2 = reinterpret_cast<const uint4 *>(a.net.w2b);
    const uint4 *src3 = reinterpret_cast<const uint4 *>(a.net.w3b);
    for (int i = t; i < kB16; i += 256) {
      reinterpret_cast<uint4 *>(S.w2)[i] = __ldg(src2 + i);
      reinterpret_cast<uint4 *>(S.w3)[i] = __ldg(src3 + i);
    }
  }
  if (t < LF) { S.b1[t] = a.net.b1[t]; S.b2[t] = a.net.b2[t]; }
  if (t == 0) S.b3 = a.net.b3[0];
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = S.tmem;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(LF >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);

  // layer 1 on the 20 x 24 region (origin y0 - 2, x0 - 2), one position and
  // one group of 8 channels per item; padding positions are written as 0
  for (int it = t; it < 2 * kA; it += 256) {
    const int pos = it >> 1, g = it & 1;
    const int r = pos / kRS, c = pos % kRS;
    const int yy = y0 - 2 + r, xx = x0 - 2 + c;
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r < L1 && c < L1 && yy >= 0 && yy < H && xx >= 0 && xx < W) {
      // channel pairs in packed FP32 FMAs (the same rounding as fmaf)
      uint64_t acc[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] = f2pack(S.b1[8 * g + 2 * k], S.b1[8 * g + 2 * k + 1]);
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const float iv = S.in[(r + tap / 3) * LI + c + tap % 3];
        const uint64_t iv2 = f2pack(iv, iv);
        const float4 wa = *reinterpret_cast<const float4 *>(S.w1t + tap * LF + 8 * g);
        const float4 wb = *reinterpret_cast<const float4 *>(S.w1t + tap * LF + 8 * g + 4);
        acc[0] = fma2(f2pack(wa.x, wa.y), iv2, acc[0]);
        acc[1] = fma2(f2pack(wa.z, wa.w), iv2, acc[1]);
        acc[2] = fma2(f2pack(wb.x, wb.y), iv2, acc[2]);
        acc[3] = fma2(f2pack(wb.z, wb.w), iv2, acc[3]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) f2unpack(acc[k], v[2 * k], v[2 * k + 1]);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = tanh_fast(v[k]);
    }
    __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) hb[k] = __float2bfloat16_rn(v[k]);
    *reinterpret_cast<uint4 *>(S.a1 + ((size_t)g * kA + pos) * 8) =
        *reinterpret_cast<const uint4 *>(hb);
  }
  fence_proxy_async();
  __syncthreads();

  // layer 2: 4 blocks x 9 taps MMAs (M = 128, N = 16, K = 16), one thread
  if (t == 0) {
    fence_after();
    const uint32_t abase = smem_u32(S.a1), bbase = smem_u32(S.w2);
#pragma unroll
    for (int i = 0; i < kMT; ++i) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const uint32_t arow = (uint32_t)(i * 128 + (tap / 3) * kRS + tap % 3);
        const uint64_t ad = sdesc(abase + arow * 16u, kA * 16u, 128u);
        const uint64_t bd = sdesc(bbase + (uint32_t)tap * (2 * LF * 16), LF * 16u, 128u);
        mma_bf16(tbase + (uint32_t)(i * LF), ad, bd, idesc, tap > 0 ? 1u : 0u);
      }
    }
    mma_commit(&S.bar);
  }
  bool ok = lift_mma_wait(&S.bar, 0);
  // layer-2 epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of blocks
  // w / 4 and w / 4 + 2 -> tanh(acc + b2) (0 outside the image and in the
  // padding rows / columns) into the layer-2 slab
  if (ok) {
    const int q = warp & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = (warp >> 2) + 2 * h;
      float v[LF];
      tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(i * LF), v);
      const int m = i * 128 + 32 * q + lane;
      if (m < kA2) {
        const int r2 = m / kRS, c2 = m % kRS;
        const int yy = y0 - 1 + r2, xx = x0 - 1 + c2;
        const bool live = r2 < L2 && c2 < L2 && yy >= 0 && yy < H && xx >= 0 && xx < W;
        __align__(16) __nv_bfloat16 hb[LF];
#pragma unroll
        for (int k = 0; k < LF; ++k)
          hb[k] = __float2bfloat16_rn(live ? tanh_fast(v[k] + S.b2[k]) : 0.f);
        *reinterpret_cast<uint4 *>(a2 + (size_t)m * 8) = *reinterpret_cast<const uint4 *>(hb);
        *reinterpret_cast<uint4 *>(a2 + ((size_t)kA2 + m) * 8) =
            *reinterpret_cast<const uint4 *>(hb + 8);
      }
    }
  }
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();

  // layer 3: 3 blocks x 9 taps MMAs into TMEM columns 64 + 16 i
  if (t == 0 && ok) {
    const uint32_t abase = smem_u32(a2), bbase = smem_u32(S.w3);
#pragma unroll
    for (int i = 0; i < kMT3; ++i) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const uint32_t arow = (uint32_t)(i * 128 + (tap / 3) * kRS + tap % 3);
        const uint64_t ad = sdesc(abase + arow * 16u, kA2 * 16u, 128u);
        const uint64_t bd = sdesc(bbase + (uint32_t)tap * (2 * LF * 16), LF * 16u, 128u);
        mma_bf16(tbase + (uint32_t)(i * LF), ad, bd, idesc, tap > 0 ? 1u : 0u);
      }
    }
    mma_commit(&S.bar);
  }
  if (ok) ok = lift_mma_wait(&S.bar, 1);
  if (!ok && lane == 0) atomicOr(a.status, kStTimeout);
  // layer-3 epilogue: column 0 of each block -> residual of output (r, c)
  if (ok) {
    const int q = warp & 3;
    for (int i = warp >> 2; i < kMT3; i += 2) {
      float v[LF];
      tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(i * LF), v);
      const int m = i * 128 + 32 * q + lane;
      const int r = m / kRS, c = m % kRS;
      if (r < LT && c < LT) S.rout[r * LT + c] = v[0] + S.b3;
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols));
  }
  if (ok) lift_finish<false>(a, p, H, W, y0, x0, S.in, nullptr, nullptr, nullptr, S.rout);
}

// Component planes [B][nc][Hp][Wp] -> interleaved samples (crop, inverse
// colour transform, floor(v + 1/2), clip).
__global__ void k_colour_out(const float *__restrict__ planes, int B, int nc, int Hp, int Wp,
                             int H, int W, int colour, int bitdepth, void *out,
                             int64_t img_stride, int64_t row_stride, int out16) {
  const int64_t n = (int64_t)B * H * W;
  const float off = (float)(1 << (bitdepth - 1));
  const float maxv = (float)((1 << bitdepth) - 1);
  const float kr = 0.299f, kb = 0.114f, kg = 1.f - 0.299f - 0.114f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % W);
    const int y = (int)((e / W) % H);
    const int b = (int)(e / ((int64_t)W * H));
    const float *pl = planes + (int64_t)b * nc * Hp * Wp + (int64_t)y * Wp + x;
    float v[3];
    if (nc == 1) {
      v[0] = pl[0] + off;
    } else {
      const float Y = pl[0] + off, Cb = pl[(int64_t)Hp * Wp], Cr = pl[2 * (int64_t)Hp * Wp];
      if (colour == 2) {
        const float G = Y - floorf((Cb + Cr) * 0.25f);
        v[0] = Cr + G; v[1] = G; v[2] = Cb + G;
      } else {
        const float R = Y + 2.f * (1.f - kr) * Cr;
        const float Bv = Y + 2.f * (1.f - kb) * Cb;
        v[0] = R; v[2] = Bv; v[1] = (Y - kr * R - kb * Bv) / kg;
      }
    }
    for (int c = 0; c < nc; ++c) {
      float s = fminf(fmaxf(floorf(v[c] + 0.5f), 0.f), maxv);
      const int64_t o = (int64_t)b * img_stride + (int64_t)y * row_stride;
      if (out16) reinterpret_cast<uint16_t *>((uint8_t *)out + o)[(int64_t)x * nc + c] = (uint16_t)s;
      else ((uint8_t *)out + o)[(int64_t)x * nc + c] = (uint8_t)s;
    }
  }
}

// Interleaved samples -> component planes [B][nc][Hp][Wp] (colour
// transform, level shift, whole-sample mirror padding).
__global__ void k_colour_in(const void *in, int64_t img_stride, int64_t row_stride, int in16,
                            int B, int nc, int H, int W, int Hp, int Wp, int lossless,
                            int bitdepth, float *__restrict__ planes) {
  const int64_t n = (int64_t)B * Hp * Wp;
  const float off = (float)(1 << (bitdepth - 1));
  const float kr = 0.299f, kb = 0.114f, kg = 1.f - 0.299f - 0.114f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % Wp);
    const int y = (int)((e / Wp) % Hp);
    const int b = (int)(e / ((int64_t)Wp * Hp));
    int sy = y < H ? y : 2 * (H - 1) - y;
    int sx = x < W ? x : 2 * (W - 1) - x;
    sy = min(max(sy, 0), H - 1);
    sx = min(max(sx, 0), W - 1);
    const int64_t o = (int64_t)b * img_stride + (int64_t)sy * row_stride;
    float s[3];
    for (int c = 0; c < nc; ++c)
      s[c] = in16 ? (float)reinterpret_cast<const uint16_t *>((const uint8_t *)in + o)[(int64_t)sx * nc + c]
                  : (float)((const uint8_t *)in + o)[(int64_t)sx * nc + c];
    float *pl = planes + (int64_t)b * nc * Hp * Wp + (int64_t)y * Wp + x;
    const int64_t ps = (int64_t)Hp * Wp;
    if (nc == 1) {
      pl[0] = s[0] - off;
    } else if (lossless) {
      pl[0] = floorf((s[0] + 2.f * s[1] + s[2]) * 0.25f) - off;
      pl[ps] = s[2] - s[1];
      pl[2 * ps] = s[0] - s[1];
    } else {
      const float Y = kr * s[0] + kg * s[1] + kb * s[2];
      pl[0] = Y - off;
      pl[ps] = (s[2] - Y) / (2.f * (1.f - kb));
      pl[2 * ps] = (s[0] - Y) / (2.f * (1.f - kr));
    }
  }
}

__global__ void k_quantise(const float *__restrict__ y, int64_t n, float delta,
                           int32_t *__restrict__ q) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    q[e] = (int32_t)rintf(__fmul_rn(y[e], delta));
}

__global__ void k_dequantise(const int32_t *__restrict__ q, int64_t n, float delta,
                             float *__restrict__ y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = __fdiv_rn((float)q[e], delta);
}

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 152 * 32 ? 152 * 32 : (g < 1 ? 1 : g));
}

void launch_lift_step(const LiftStepParams &a, cudaStream_t st) {
  if (a.tc && a.net.w1 && a.round == 0) {
    static std::atomic<uint64_t> attr_tc{0};
    once_per_device(attr_tc, [] {
      cudaFuncSetAttribute(k_lift_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(LiftTcSmem) + 1024);
    });
    const int tiles = ((a.H + LT - 1) / LT) * ((a.W + LT - 1) / LT);
    dim3 grid(tiles, 1, a.P);
    k_lift_tc<<<grid, 256, sizeof(LiftTcSmem) + 1024, st>>>(a);
    return;
  }
  static std::atomic<uint64_t> attr{0};
  once_per_device(attr, [] {
    cudaFuncSetAttribute(k_lift_step<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(LiftSmem));
    cudaFuncSetAttribute(k_lift_step<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(LiftSmem));
  });
  const int tiles = ((a.H + LT - 1) / LT) * ((a.W + LT - 1) / LT);
  dim3 grid(tiles, 1, a.P);
  // integer (lossless) steps take the exact operation sequence
  if (a.round != 0) k_lift_step<true><<<grid, 256, sizeof(LiftSmem), st>>>(a);
  else k_lift_step<false><<<grid, 256, sizeof(LiftSmem), st>>>(a);
}
void launch_colour_out(const float *planes, int B, int nc, int Hp, int Wp, int H, int W,
                       int colour, int bitdepth, void *out, int64_t img_stride,
                       int64_t row_stride, cudaStream_t st) {
  int64_t n = (int64_t)B * H * W;
  k_colour_out<<<grid_for(n), 256, 0, st>>>(planes, B, nc, Hp, Wp, H, W, colour, bitdepth,
                                             out, img_stride, row_stride, bitdepth > 8);
}
void launch_colour_in(const void *in, int64_t img_stride, int64_t row_stride, int B, int nc,
                      int H, int W, int Hp, int Wp, int lossless, int bitdepth, float *planes,
                      cudaStream_t st) {
  int64_t n = (int64_t)B * Hp * Wp;
  k_colour_in<<<grid_for(n), 256, 0, st>>>(in, img_stride, row_stride, bitdepth > 8, B, nc,
                                            H, W, Hp, Wp, lossless, bitdepth, planes);
}
void launch_quantise(const float *y, int64_t n, float delta, int32_t *q, cudaStream_t st) {
  k_quantise<<<grid_for(n), 256, 0, st>>>(y, n, delta, q);
}
void launch_dequantise(const int32_t *q, int64_t n, float delta, float *y, cudaStream_t st) {
  k_dequantise<<<grid_for(n), 256, 0, st>>>(q, n, delta, y);
}

}  // namespace pw
