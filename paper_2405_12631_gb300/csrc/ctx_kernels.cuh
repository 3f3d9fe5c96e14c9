// Declarations of the context-model, lifting and entropy kernels' launchers.
#pragma once
#include "pw_internal.cuh"

namespace pw {

enum { EPI_STORE = 0, EPI_LSTM = 1, EPI_HEAD = 2 };

// Parameters of the generic NHWC convolution (FP32 SIMT path).
struct ConvParams {
  const float *in;      // [P, H, W, in_cs], channels [in_co, in_co + cin)
  int in_cs, in_co, cin;
  const float *w;       // [KS*KS][cin][cout_total]
  const float *b;       // [cout_total]
  int cout_total;
  int P, H, W;
  // EPI_STORE: out = act(acc + b + res)
  float *out;
  int out_cs, out_co;
  int act;
  const float *res;
  int res_cs, res_co;
  // EPI_LSTM: gates -> c_new, h (h written to out at out_cs/out_co)
  const float *c_prev;  // [P, H >> up, W >> up, C]
  float *c_new;         // [P, H, W, C]
  int up, first, C;
  // EPI_HEAD: z' = res + acc + b; (mu, rho) = wh z' + bh at step positions
  const float *wh;      // [2][cout_total]
  const float *bh;      // [2]
  int step;
  uint32_t *idx;        // packed indices, [P][idx_stride] in step order
  int64_t idx_stride;
  float *mu_out, *sg_out;  // optional [P, H, W]
  // integer-network class: inputs, weights and biases are integers held
  // exactly in floats; the output is requantised by rq bits (round half
  // up) and clamped (EPI_STORE: residual added after; EPI_LSTM: the gates;
  // EPI_HEAD: z'), the head by rq_mu / rq_rho bits (see the launchers)
  int iq, rq, rq_mu, rq_rho;
};
// Integer class of the SIMT producers below: rqn = kRqFloat selects the
// float definition, otherwise their outputs are requantised by rqn bits.
constexpr int kRqFloat = -1000;

void launch_conv_simt(int ks, const ConvParams &a, int epi, cudaStream_t st);

// Logistic-mixture head of one coding step (mixture.cu): one warp per
// symbol of the step ([P][nk] in step order).
struct MixHeadParams {
  const float *z;       // z' [P, H, W, C]
  const float *wh;      // [9][C]
  const float *bh;      // [9]
  int C, P, H, W, step;
  int64_t nk;           // symbols of the step per plane
  int32_t *ctr;         // [P][nk] centres (written)
  uint16_t *rows;       // decoding: [P * nk][kMixRow] table rows, or null
  const int32_t *q;     // encoding: quantised subband [P, H, W] ...
  uint32_t *cf;         // ... and [P][nk] (cdf | frequency << 16) of each symbol, or null
  float *par;           // optional [P, H, W, 9] (w, mu, sigma) at the step's positions
};
void launch_mix_head(const MixHeadParams &a, cudaStream_t st);
// Stage entry: rows of n keys given as int32 (q0 q1 q2 j0 j1 j2 g0 g1 g2).
void launch_mix_tables(const int32_t *key9, int64_t n, uint16_t *rows, cudaStream_t st);
// Ragged batches (planes of different sizes decoded on one canvas of
// P x H x W): zero every 16-byte unit of an activation buffer that lies
// outside its plane's own extent (ext[p] >> esh, the padded full-resolution
// sizes shifted to the subband level), so that a convolution over the
// canvas sees the same zero padding as one over the plane alone. Layouts
// of the NG units per position: group-major [P][NG][H][W], pixel-major
// [P][H][W][NG], or phase-split pixel-major [P][H][4][W4 / 4][NG]
// (x = 4 j + phase, W4 = W rounded up to a multiple of 4).
enum { ZL_GROUP = 0, ZL_PIXEL = 1, ZL_PHASE = 2 };
void launch_zero_outside(void *buf, int layout, int P, int H, int W, int NG, const int2 *ext,
                         int esh, cudaStream_t st);
// Set when a launcher found no kernel for its arguments (checked and cleared
// by the host drivers).
bool &launch_failed();
void launch_lstm_in(const int32_t *s_prev, const float *h_prev, int h_cs, int h_co,
                    const float *we, const float *be, float *X, int P, int H, int W, int C,
                    int up, int first, cudaStream_t st, int rqn = kRqFloat);
void launch_masked_in(const int32_t *s, const float *wa, const float *ba, float *out,
                      int out_cs, int P, int H, int W, int C, int step, cudaStream_t st,
                      int rqn = kRqFloat);
void launch_dw3x3(const float *in, const float *w, const float *b, float *out, int P, int H,
                  int W, int C, cudaStream_t st, int rqn = kRqFloat);

// entropy.cu
struct DecChunk {
  const uint8_t *data;
  uint32_t nbytes;
  uint32_t count;
  uint32_t first;
  uint16_t lanes;
  uint16_t plane;
};
struct EncChunk {
  uint64_t sym_base;     // element offset of the chunk's first symbol (idx / vals)
  uint64_t scratch_end;  // word index one past the chunk's scratch region
  uint32_t count, lanes;
};
// bank: 2048 x 128 CDF tables; coarse (may be null): every 8th entry, 2048 x 16
void launch_cdf_bank(uint16_t *bank, uint16_t *coarse, cudaStream_t st);
// mix: per-symbol tables (logistic mixture) - bank is then the step's
// [P * idx_stride][kMixRow] rows (row of symbol plane * idx_stride + first
// + i), coarse is unused and idx holds the symbols' centres (int32).
void launch_rans_decode(const DecChunk *chunks, int nchunks, const uint16_t *bank,
                        const uint16_t *coarse, const uint32_t *idx, int64_t idx_stride,
                        int32_t *out, int64_t out_stride, int h, int w, int step,
                        uint32_t *status, cudaStream_t st, bool mix = false,
                        const int2 *ext = nullptr, int esh = 0);
// cf (logistic mixture, else null): per symbol (cdf | frequency << 16) of its
// coded symbol; idx then holds the centres (int32) and bank is unused.
void launch_rans_count_ops(const EncChunk *chunks, int nchunks, const uint32_t *idx,
                           const int32_t *vals, uint32_t *ops, cudaStream_t st,
                           bool mix = false);
void launch_rans_encode(const EncChunk *chunks, int nchunks, const uint16_t *bank,
                        const uint32_t *idx, const int32_t *vals, uint16_t *scratch,
                        uint32_t *states, uint32_t *nwords, uint32_t *status,
                        cudaStream_t st, const uint32_t *cf = nullptr);
void launch_rans_pack(const EncChunk *chunks, int nchunks, const uint16_t *scratch,
                      const uint32_t *states, const uint32_t *nwords,
                      const uint64_t *out_off, uint8_t *payload, cudaStream_t st);
void launch_pack_index(const float *mu, const float *s, int64_t n, int is_sigma,
                       uint32_t *idx, cudaStream_t st);

}  // namespace pw
