// Motion-compensated temporal lifting (Section 3.3): the predict step of
// the temporal wavelet warps the even frame towards the odd one with block
// motion vectors, and the update step re-uses the same vectors to map the
// highpass band back onto the even frame's grid (inverse motion
// compensation).
//
// Motion model (the paper defers it to its reference): integer-pel vectors
// (dy, dx), |dy|, |dx| <= kMcRange, one per kMcBlock x kMcBlock block of the
// odd frame on the padded frame grid;
//   MC(f)[y, x]  = f[clamp(y + dy), clamp(x + dx)],
//   IMC(h)[y, x] = h[clamp(y - dy), clamp(x - dx)],
// with (dy, dx) the vector of the block containing (y, x). Vectors of
// temporal level l, pair m come from a full search of original frame
// 2^l m + 2^(l-1) against original frame 2^l m on an integer luma (the gray
// sample or floor((R + 2G + B) / 4) of the 8-bit samples, mirror-padded like
// the colour planes): minimum sum of absolute differences, ties to the
// smaller |dy| + |dx|, then the smaller dy, then the smaller dx. Integer
// arithmetic throughout, so every implementation finds the same vectors.
#include <cstdint>

#include "codec.h"
#include "lift_kernels.cuh"
#include "pw_internal.cuh"

namespace pw {

// Interleaved 8-bit frames [nf][H][W][nc] -> integer luma [nf][Hp][Wp]
// (whole-sample mirror padding, as the colour planes).
__global__ void k_gop_luma(const uint8_t *__restrict__ img, int64_t img_stride, int64_t row_stride,
                           int nf, int nc, int H, int W, int Hp, int Wp, int32_t *__restrict__ luma) {
  const int64_t n = (int64_t)nf * Hp * Wp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % Wp);
    const int y = (int)((e / Wp) % Hp);
    const int f = (int)(e / ((int64_t)Wp * Hp));
    int sy = y < H ? y : 2 * (H - 1) - y;
    int sx = x < W ? x : 2 * (W - 1) - x;
    sy = min(max(sy, 0), H - 1);
    sx = min(max(sx, 0), W - 1);
    const uint8_t *p = img + (int64_t)f * img_stride + (int64_t)sy * row_stride + (int64_t)sx * nc;
    luma[e] = nc == 1 ? (int32_t)p[0] : ((int32_t)p[0] + 2 * (int32_t)p[1] + (int32_t)p[2]) >> 2;
  }
}

// One CTA per (block, field): the reference window of the block
// ((B + 2R)^2 samples, coordinates clamped to the frame) and the block in
// shared memory, one candidate per thread at a time, then the minimum of the
// packed key (SAD << 24 | (|dy| + |dx|) << 16 | (dy + R) << 8 | (dx + R))
// over the CTA, which orders candidates exactly as the definition does.
constexpr int kWin = kMcBlock + 2 * kMcRange;

__global__ void __launch_bounds__(256) k_motion_search(const int32_t *__restrict__ luma, int nf,
                                                       int Hp, int Wp, int8_t *__restrict__ mv) {
  __shared__ int32_t win[kWin * kWin];
  __shared__ int32_t blk[kMcBlock * kMcBlock];
  __shared__ unsigned long long red[8];
  const int bx = blockIdx.x, by = blockIdx.y, field = blockIdx.z;
  const int nbx = gridDim.x, nby = gridDim.y;
  // field -> (level, pair): fields of level 1 first, nf / 2 of them, ...
  int lv = 1, m = field, cnt = nf >> 1;
  while (m >= cnt && cnt > 0) { m -= cnt; ++lv; cnt >>= 1; }
  const int ref_f = (1 << lv) * m, cur_f = ref_f + (1 << (lv - 1));
  const int32_t *ref = luma + (int64_t)ref_f * Hp * Wp;
  const int32_t *cur = luma + (int64_t)cur_f * Hp * Wp;
  const int y0 = by * kMcBlock, x0 = bx * kMcBlock;
  for (int e = threadIdx.x; e < kWin * kWin; e += blockDim.x) {
    const int yy = min(max(y0 - kMcRange + e / kWin, 0), Hp - 1);
    const int xx = min(max(x0 - kMcRange + e % kWin, 0), Wp - 1);
    win[e] = ref[(int64_t)yy * Wp + xx];
  }
  for (int e = threadIdx.x; e < kMcBlock * kMcBlock; e += blockDim.x) {
    const int yy = y0 + e / kMcBlock, xx = x0 + e % kMcBlock;
    blk[e] = (yy < Hp && xx < Wp) ? cur[(int64_t)yy * Wp + xx] : 0;
  }
  __syncthreads();
  const int bh = min(kMcBlock, Hp - y0), bw = min(kMcBlock, Wp - x0);
  constexpr int side = 2 * kMcRange + 1;
  unsigned long long best = ~0ull;
  for (int c = threadIdx.x; c < side * side; c += blockDim.x) {
    const int dy = c / side - kMcRange, dx = c % side - kMcRange;
    uint32_t sad = 0;
    for (int i = 0; i < bh; ++i) {
      // window row of block row i displaced by dy; the window's clamping
      // equals clamping the frame coordinates
      const int32_t *wr = win + (i + dy + kMcRange) * kWin + kMcRange + dx;
      const int32_t *br = blk + i * kMcBlock;
      for (int j = 0; j < bw; ++j) sad += (uint32_t)abs(br[j] - wr[j]);
    }
    const unsigned long long key = ((unsigned long long)sad << 24) |
                                   ((unsigned long long)(abs(dy) + abs(dx)) << 16) |
                                   ((unsigned long long)(dy + kMcRange) << 8) |
                                   (unsigned long long)(dx + kMcRange);
    best = key < best ? key : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
    best = v < best ? v : best;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = red[w] < best ? red[w] : best;
    int8_t *o = mv + (((int64_t)field * nby + by) * nbx + bx) * 2;
    o[0] = (int8_t)((int)((best >> 8) & 0xFF) - kMcRange);
    o[1] = (int8_t)((int)(best & 0xFF) - kMcRange);
  }
}

// out[p][y][x] = in[p][clamp(y + sign dy)][clamp(x + sign dx)], (dy, dx) the
// vector of field field0 + p at block (y / B, x / B).
__global__ void k_mc_warp(PlaneAcc src, PlaneAcc dst, int P, int H, int W,
                          const int8_t *__restrict__ mv, int field0, int nby, int nbx, int sign) {
  const int64_t n = (int64_t)P * H * W;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % W);
    const int y = (int)((e / W) % H);
    const int p = (int)(e / ((int64_t)W * H));
    const int8_t *v = mv + (((int64_t)(field0 + p) * nby + y / kMcBlock) * nbx + x / kMcBlock) * 2;
    const int sy = min(max(y + sign * (int)v[0], 0), H - 1);
    const int sx = min(max(x + sign * (int)v[1], 0), W - 1);
    dst.p[(int64_t)p * dst.ps + (int64_t)y * dst.rs + x] =
        src.p[(int64_t)p * src.ps + (int64_t)sy * src.rs + sx];
  }
}

static int grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 152 * 32 ? 152 * 32 : (g < 1 ? 1 : g));
}

void launch_gop_luma(const uint8_t *img, int64_t img_stride, int64_t row_stride, int nf, int nc,
                     int H, int W, int Hp, int Wp, int32_t *luma, cudaStream_t st) {
  k_gop_luma<<<grid_of((int64_t)nf * Hp * Wp), 256, 0, st>>>(img, img_stride, row_stride, nf, nc,
                                                             H, W, Hp, Wp, luma);
}

void launch_motion_search(const int32_t *luma, int nf, int Hp, int Wp, int8_t *mv,
                          cudaStream_t st) {
  const int nby = (Hp + kMcBlock - 1) / kMcBlock, nbx = (Wp + kMcBlock - 1) / kMcBlock;
  dim3 grid(nbx, nby, nf - 1);   // 2^T - 1 fields over all levels
  k_motion_search<<<grid, 256, 0, st>>>(luma, nf, Hp, Wp, mv);
}

void launch_mc_warp(const PlaneAcc &src, const PlaneAcc &dst, int P, int H, int W,
                    const int8_t *mv, int field0, int sign, cudaStream_t st) {
  const int nby = (H + kMcBlock - 1) / kMcBlock, nbx = (W + kMcBlock - 1) / kMcBlock;
  k_mc_warp<<<grid_of((int64_t)P * H * W), 256, 0, st>>>(src, dst, P, H, W, mv, field0, nby, nbx,
                                                         sign);
}

}  // namespace pw
