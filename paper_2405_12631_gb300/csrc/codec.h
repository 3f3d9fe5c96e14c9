// Host-side objects of libpwave: context, model, stream header, plans.
#pragma once

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "ctx_kernels.cuh"
#include "lift_kernels.cuh"
#include "pw_internal.cuh"

struct pw_ctx;

namespace pw {

// Precision classes whose context convolutions run on the tensor cores.
inline bool tc_precision(int p) { return p == PW_PREC_BF16 || p == PW_PREC_FP8; }

struct StepNetDev {
  // step 1 (DepthConvBlock net)
  float *win = nullptr, *bin = nullptr, *w1 = nullptr, *b1 = nullptr, *wdw = nullptr,
        *bdw = nullptr, *w2 = nullptr, *b2 = nullptr, *w3 = nullptr, *b3 = nullptr,
        *w4 = nullptr, *b4 = nullptr;
  // steps 2-4 (residual-block nets)
  float *wa = nullptr, *ba = nullptr, *wz = nullptr, *bz = nullptr, *c1w = nullptr,
        *c1b = nullptr, *c2w = nullptr, *c2b = nullptr;
  // head
  float *wh = nullptr, *bh = nullptr;
};

// Integer-network class (PW_PREC_INT8): the context model's weights and
// biases quantised to integers (held exactly as floats, in the FP32 path's
// layouts) and the requantisation shift of every layer's output.
struct IntStepNet {
  StepNetDev d;
  int n_win = 0, n_w1 = 0, n_dw = 0, n_w2 = 0, n_w3 = 0, n_w4 = 0;  // step 1
  int n_wa = 0, n_wz = 0, n_c1 = 0, n_c2 = 0;                       // steps 2-4
  int n_mu = 0, n_rho = 0;                                          // head
};
struct IntNets {
  float *we = nullptr, *be = nullptr, *wg = nullptr, *bg = nullptr;  // ConvLSTM
  int n_e = 0, n_g = 0;
  IntStepNet sb[4], ll[4];
  // autoregressive LL model (ll_mode 1): masked 5x5 conv, 1x1, head
  float *ar_w5 = nullptr, *ar_b5 = nullptr, *ar_w1 = nullptr, *ar_b1 = nullptr,
        *ar_wh = nullptr, *ar_bh = nullptr;
  int ar_n5 = 0, ar_n1 = 0, ar_nmu = 0, ar_nrho = 0;
};

// Tensor-core (BF16) copies of the context-model weights, see ctx_tc.cu.
struct TcWeights;

struct Model {
  pw_ctx *ctx = nullptr;
  int levels = 4, C = 32, F = 16, ll_mode = 0;
  // probability model: Laplace (heads of 2 outputs) or the logistic mixture
  // of 3 (9 outputs; FP32 precision class and four-step LL only)
  int nh = 2;
  bool mix = false;
  IntNets *intn = nullptr;   // built when loaded in an INT8 context (Laplace models)
  uint64_t hash = 0;
  uint64_t uid = 0;          // unique per loaded model (keys cached workspaces)
  std::vector<float *> allocs;
  std::map<std::string, std::vector<float>> host;
  LiftNetDev lift[2][2];   // [row, col][P, U]
  LiftNetDev tlift[2];     // [P, U]
  // post-processing CNN after the inverse transform (present when the blob
  // carries "post.*" tensors; lossy images only)
  LiftNetDev post{};
  bool has_post = false;
  float *lstm_we = nullptr, *lstm_be = nullptr, *lstm_wg = nullptr, *lstm_bg = nullptr;
  StepNetDev sb[4], ll[4];
  float *ar_w5 = nullptr, *ar_b5 = nullptr, *ar_w1 = nullptr, *ar_b1 = nullptr,
        *ar_wh = nullptr, *ar_bh = nullptr;
  TcWeights *tc = nullptr;
  std::mutex mu;     // guards the lazy tensor-core weight builds
  int load(pw_ctx *c, const void *blob, size_t n);
  int ensure_tc();   // builds tc on first use (BF16 contexts)
  int ensure_fp8();  // adds the E4M3 convolutions to tc (FP8 contexts)
  // weights a context of this precision needs (thread-safe)
  int prepare(int precision);
  void free_tc();
  ~Model();
};

#pragma pack(push, 1)
struct StreamHeader {
  char magic[4];
  uint16_t version, flags;
  uint32_t width, height;
  uint8_t ncomp, levels, bitdepth, colour;
  float delta_l, delta_h;
  uint16_t T;
  uint8_t log2m, lanes;
  uint32_t chunk_symbols, n_chunks;
  uint64_t model_hash;
  uint32_t payload_bytes;
  uint8_t lane_shift;          // 0: the default 2^7 symbols per state
  uint8_t reserved[11];
};
#pragma pack(pop)
static_assert(sizeof(StreamHeader) == 64, "stream header is 64 bytes");

enum : uint16_t {
  FLAG_LOSSLESS = 1, FLAG_LL_AR = 2, FLAG_PREC_SHIFT = 2, FLAG_BALANCED = 16,
  FLAG_MIX = 32   // logistic-mixture probability model
};

// One chunk of the per-component layout (same for every image of a class).
struct ChunkTpl {
  int sb, step;            // step -1: single-state autoregressive LL chunk
  uint32_t first, count;
  uint16_t lanes;
};

// Geometry shared by all images of a plan.
struct Geometry {
  int H = 0, W = 0, Hp = 0, Wp = 0, nc = 1, levels = 4, colour = 0, bitdepth = 8;
  int lossless = 0, ll_ar = 0, chunk = 16384;
  // chunk layout of a step's symbols: 0 = chunks of `chunk` symbols and a
  // shorter last one; 1 (balanced, header flag FLAG_BALANCED) = the fewest
  // chunks of at most `chunk` symbols, of equal length to within one
  int balanced = 1;
  // symbols per interleaved rANS state: 2^lane_shift (5..7; header byte 52,
  // where 0 stands for the default 7)
  int lane_shift = kLaneShift;
  int nsb = 13;
  std::vector<int> sh, sw;          // subband sizes in coding order
  std::vector<int64_t> soff;        // per-plane element offset of subband i
  int64_t plane_elems = 0;          // Hp * Wp
  std::vector<int64_t> ioff;        // [sb * 4 + step] per-plane offset in idx arena
  std::vector<ChunkTpl> chunks;     // per-component chunk list (stream order)
  std::vector<int> group_first;     // [sb * 4 + step] first chunk index, or -1
  std::vector<int> group_count;     // [sb * 4 + step]
  void build(int H, int W, int nc, int levels, int colour, int bitdepth, int lossless,
             int ll_ar, int chunk, int balanced = 1, int lane_shift = kLaneShift);
};

// Device buffers for a batch of planes of one geometry.
// Stream-ordered device allocations from a per-device memory pool that keeps
// freed memory for reuse: freeing never synchronises the device, so plans
// of one context can come and go while other streams keep decoding.
int pool_alloc(void **p, size_t n, cudaStream_t st);
void pool_free(void *p, cudaStream_t st);

struct Workspace {
  int P = 0;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;   // the stream alloc() ran on (frees go there)
  uint8_t *base = nullptr;
  int32_t *Q = nullptr;        // quantised latent, [sb][P][h][w]
  float *Yf = nullptr;         // float latent (dequantised / forward output)
  uint32_t *idx = nullptr;     // packed table indices, [sb*4+step][P][n]
  float *X = nullptr, *X2 = nullptr, *Z = nullptr, *U = nullptr, *V = nullptr, *Z2 = nullptr;
  float *Cst[2] = {nullptr, nullptr};
  float *T0 = nullptr, *T1 = nullptr, *T2 = nullptr;  // lifting temporaries
  float *planes = nullptr;     // component planes [P][Hp][Wp]
  float *mu = nullptr, *sg = nullptr;  // optional parameter outputs [P][Hp*Wp]
  // logistic-mixture models: table rows of the current step ([P * largest
  // step][kMixRow], decoding), (cdf | frequency << 16) of every symbol in the
  // idx layout (encoding), optional parameters [P][Hp*Wp][9]
  uint16_t *mrows = nullptr;
  uint32_t *mcf = nullptr;
  float *mpar = nullptr;
  void *tc = nullptr;          // BF16 / FP8 activations (tensor-core path)
  int lstm_cur = 0;            // which Cst holds the current cell state
  // ragged batches: the planes' own padded sizes (Hp, Wp) on the device, one
  // per plane, when they differ from the workspace's geometry (the canvas);
  // the passes then zero activations outside every plane's extent before a
  // spatial convolution reads them. Not owned; null for plain batches.
  const int2 *ext = nullptr;
  // prec: the context's pw_precision (tensor-core buffers unless FP32)
  // mix: buffers of the logistic-mixture model
  int alloc(const Geometry &g, int P, int C, bool params, int prec, cudaStream_t st,
            bool mix = false);
  // upper bound of the device bytes alloc() takes for these arguments
  static int64_t estimate(const Geometry &g, int P, int C, bool params, int prec,
                          bool mix = false);
  void release();
  ~Workspace() { release(); }
};

// Decomposition level of subband sb (coding order: LL_L, then HL/LH/HH of
// levels L .. 1).
inline int sb_level(const Geometry &g, int sb) {
  return sb == 0 ? g.levels : g.levels - (sb - 1) / 3;
}

// Host entry points implemented in codec.cu (all on ctx's stream).
int run_context_pass(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws, int sb,
                     int step, bool decoding);
int run_lstm(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws, int sb);
int lift_inverse_planes(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws,
                        float *dst_planes);
int lift_forward_planes(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws,
                        const float *src_planes);
// Post-processing of the reconstructed component planes ([P][Hp][Wp]):
// dst = src + CNN_post(src) (dst != src).
// ext: ragged batches' per-plane padded sizes (see Workspace::ext) or null.
int post_process_planes(pw_ctx *ctx, Model &m, const Geometry &g, int P, const float *src,
                        float *dst, const int2 *ext = nullptr);
// Temporal lifting of a GOP (Section 3.3). mv: device block motion vectors
// of every level and pair (the order of the motion search: level 1 pairs
// first), or null for zero motion; twarp: (nf / 2) frames of scratch for the
// motion-compensated operands (unused without vectors).
int temporal_planes(pw_ctx *ctx, Model &m, int nf, int nc, int Hp, int Wp, const float *in,
                    float *out, float *tmp0, float *tmp1, bool forward,
                    const int8_t *mv = nullptr, float *twarp = nullptr);

// Motion model of the temporal lifting (motion.cu): integer-pel vectors of
// kMcBlock x kMcBlock blocks, |dy|, |dx| <= kMcRange.
constexpr int kMcBlock = 16, kMcRange = 16;
void launch_gop_luma(const uint8_t *img, int64_t img_stride, int64_t row_stride, int nf, int nc,
                     int H, int W, int Hp, int Wp, int32_t *luma, cudaStream_t st);
void launch_motion_search(const int32_t *luma, int nf, int Hp, int Wp, int8_t *mv,
                          cudaStream_t st);
void launch_mc_warp(const PlaneAcc &src, const PlaneAcc &dst, int P, int H, int W,
                    const int8_t *mv, int field0, int sign, cudaStream_t st);
// Batch decode of B streams of one geometry (api.cu) and release of a
// context's cached workspaces; used by the decode server.
int decode_batch(pw_ctx *ctx, Model &m, int B, const uint8_t *const *bs, const size_t *n,
                 int on_dev, pw_image *out);
void drop_plans(pw_ctx *ctx);
// Validate a host stream's header against the model and the context's
// precision and derive its geometry (api.cu).
int stream_geometry(pw_ctx *ctx, const Model &m, const uint8_t *bs, size_t n, Geometry &g);

}  // namespace pw

struct pw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = PW_PREC_FP32;
  uint16_t *bank = nullptr;        // CDF table bank (built by k_cdf_bank)
  uint16_t *coarse = nullptr;      // its coarse level (same allocation, after the bank)
  uint32_t *status = nullptr;      // device status word
  uint64_t launches = 0;
  void *plan_cache = nullptr;      // cached workspaces per geometry (api.cu)
  void *prof = nullptr;            // per-kernel-class event timing (prof.cpp)
  int lane_shift = 7;              // encoders: 2^lane_shift symbols per rANS state
  // image decodes replay a CUDA graph of their plan's pass chain once a
  // direct run of the plan used only tuned schedules (pw_ctx_set_graphs)
  int graphs = 1;
  cudaStream_t cap_stream = nullptr;   // private stream the chains are captured on
  uint64_t graph_replays = 0;
  // GOP decodes: a second context on its own non-blocking stream decodes the
  // lowpass band while this one decodes the highpass bands (created on first
  // use, destroyed with this context)
  pw_ctx *aux = nullptr;
  cudaStream_t aux_stream = nullptr;
};

struct pw_model {
  pw::Model m;
};
