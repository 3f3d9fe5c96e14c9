// Declarations of the lifting / colour / quantiser kernels' launchers.
#pragma once
#include "pw_internal.cuh"

namespace pw {

// Strided view of a stack of planes: element (p, y, x) at
// p[p * ps + y * rs + x * cs].
struct PlaneAcc {
  float *p;
  int64_t ps;
  int64_t rs;
  int64_t cs;
};

struct LiftNetDev {
  const float *w1, *b1, *w2, *b2, *w3, *b3;  // [16][9], [16], [16][16][9], [16], [16][9], [1]
  // BF16 MMA B operands of layers 2 and 3 for the tensor-core step, packed
  // [tap][2 channel groups][16 outputs][8] (layer 3: output 0, rest zero)
  const void *w2b, *w3b;
};

enum { LIN_P53 = 0, LIN_U53 = 1, LIN_ID = 2, LIN_HALF = 3, LIN_ZERO = 4 };

struct LiftStepParams {
  PlaneAcc src, other, out, copy;  // copy.p may be null
  int P, H, W;                     // plane count and src/out plane size
  LiftNetDev net;                  // net.w1 == null: linear part only
  int lin, dir;                    // dir 0: along x (rows), 1: along y (columns)
  int sign;                        // out = other + sign * v
  int round;                       // 0 none, 1 floor(v), 2 floor(v + 1/2)
  int tc;                          // 1: middle CNN layer on the tensor cores
                                   // (BF16 operands; round must be 0)
  uint32_t *status;                // kStTimeout is set here (tc only)
  // ragged batches (planes of different sizes on one canvas of P x H x W):
  // plane p's own extent is ((ext[p].x >> esh) * ehmul) x (ext[p].y >> esh)
  // (ext = the planes' padded full-resolution sizes); tiles beyond it do no
  // work and its borders take the place of the canvas's. Null: every plane
  // is H x W.
  const int2 *ext;
  int esh, ehmul;
};
// Extent of plane p of a lifting step (see LiftStepParams::ext).
__host__ __device__ __forceinline__ void lift_extent(const LiftStepParams &a, int p, int &H,
                                                     int &W) {
  if (a.ext) {
    H = (a.ext[p].x >> a.esh) * a.ehmul;
    W = a.ext[p].y >> a.esh;
  } else {
    H = a.H;
    W = a.W;
  }
}

void launch_lift_step(const LiftStepParams &a, cudaStream_t st);
void launch_colour_out(const float *planes, int B, int nc, int Hp, int Wp, int H, int W,
                       int colour, int bitdepth, void *out, int64_t img_stride,
                       int64_t row_stride, cudaStream_t st);
void launch_colour_in(const void *in, int64_t img_stride, int64_t row_stride, int B, int nc,
                      int H, int W, int Hp, int Wp, int lossless, int bitdepth, float *planes,
                      cudaStream_t st);
void launch_quantise(const float *y, int64_t n, float delta, int32_t *q, cudaStream_t st);
void launch_dequantise(const int32_t *q, int64_t n, float delta, float *y, cudaStream_t st);

}  // namespace pw
