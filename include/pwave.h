/*
 * pwave.h - C ABI of the GB300 pWave++ codec library (libpwave.so).
 *
 * The library implements the decode path of the learned wavelet coder of
 * "Efficient Learned Wavelet Image and Video Coding" (pWave++ / pMCTF):
 * the four-step parallel context model (Section 3.2), entropy parameters ->
 * integer CDF tables -> rANS decoding (standing in for the paper's
 * arithmetic coder, Section 3.1), and the CNN lifting inverse wavelet
 * transform (Section 3.1, Fig. 2), plus the matching encoder and the
 * temporal lifting stage for groups of pictures (Section 3.3).
 *
 * Conventions for every call:
 *  - the return value is a pw_status (PW_OK = 0); no call aborts the process;
 *  - all GPU work is enqueued on the context's CUDA stream; calls that return
 *    host results synchronise that stream before returning;
 *  - the library never frees memory it did not allocate; buffers it returns
 *    (bitstreams) are released with pw_free;
 *  - "device" pointers are CUDA device pointers of the context's device;
 *    "host" pointers are ordinary (pageable or pinned) host memory;
 *  - a pw_ctx is not thread-safe: use one context per host thread.
 */
#ifndef PWAVE_H
#define PWAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PW_OK = 0,
  PW_EINVAL = 1,        /* bad argument, or stream made by another model  */
  PW_ENOMEM = 2,        /* device or host allocation failed               */
  PW_ECORRUPT = 3,      /* malformed or truncated bitstream               */
  PW_EUNSUPPORTED = 4,  /* valid but unsupported configuration            */
  PW_ETIMEOUT = 5,      /* a bounded wait expired                         */
  PW_EAGAIN = 6,        /* resource temporarily exhausted (server budget) */
  PW_ECUDA = 7          /* a CUDA runtime/driver call failed              */
} pw_status;

/* Arithmetic of the context-model and lifting convolutions. FP32 is the
 * plain SIMT path; INT8 is the integer-network context model (int8 weights
 * with one power-of-two scale per tensor, int8 activations at fixed binary
 * points, round-half-up requantisation, hard sigmoid / tanh ConvLSTM, a head
 * whose outputs are the table indices: every operation exact integer
 * arithmetic, so any two implementations derive identical tables; four-step
 * LL Laplace models, loaded in an INT8 context; lifting as FP32);
 * BF16 runs the convolutions on tcgen05 tensor cores with
 * FP32 accumulation (and, for lossy streams, layers 2 and 3 of the inverse
 * lifting CNN); FP8 is BF16 with the three 3x3 context convolutions (ConvLSTM
 * gates, residual blocks of steps 2-4) in E4M3 with per-channel scales and
 * FP32 accumulation. The entropy-parameter -> table decision and the CDF
 * tables are FP32/integer in every mode. A stream decodes only with the
 * precision class that encoded it (recorded in the stream header). */
typedef enum {
  PW_PREC_FP32 = 0, PW_PREC_BF16 = 1, PW_PREC_FP8 = 2, PW_PREC_INT8 = 3
} pw_precision;

typedef struct pw_ctx pw_ctx;
typedef struct pw_model pw_model;

/* An interleaved (HWC) image. bitdepth 8 means uint8 samples, 9..16 means
 * uint16 samples. stride_bytes = 0 means tightly packed rows. */
typedef struct {
  int32_t width, height, channels; /* channels: 1 (gray) or 3 (RGB)      */
  int32_t bitdepth;
  int32_t is_device;               /* data is a device pointer             */
  int32_t reserved;
  void *data;
  int64_t stride_bytes;
} pw_image;

typedef struct {
  float q;                /* quantiser step: Delta_L = Delta_H = 1/q (Section 3.1) */
  int32_t lossless;       /* integer lifting + RCT, no quantiser (Fig. 2 caption) */
  int32_t chunk_symbols;  /* max symbols per rANS chunk (0 = 16384)              */
} pw_codec_opts;

/* ---- context and model ------------------------------------------------- */

/* Create a context on CUDA device `device` that enqueues its work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * Errors: PW_EINVAL (bad device/precision), PW_ECUDA. */
int pw_ctx_create(int device, void *cuda_stream, int precision, pw_ctx **out);
void pw_ctx_destroy(pw_ctx *ctx);
/* Precision the context was created with. */
int pw_ctx_precision(const pw_ctx *ctx);
/* Stream-format option of the streams this context encodes (the coder
 * stands in for the paper's arithmetic coder, Section 3.1; the paper has no
 * such parameter): a chunk of n symbols is coded with min(32, max(1,
 * n >> s)) interleaved rANS states, s = log2_symbols_per_state in 5..7
 * (default 7). Every state costs a 4-byte flush in the stream, and a chunk
 * decodes in ceil(n / states) serial rounds, so a smaller s trades rate for
 * decode latency on small subbands. The stream header records s (byte 52);
 * decoders read any of them. Errors: PW_EINVAL (s outside 5..7). */
int pw_ctx_set_lane_rule(pw_ctx *ctx, int log2_symbols_per_state);

/* Load a weight blob ("PWMB" format: lifting nets, ConvLSTM, four-step
 * context nets; one blob per lambda model, Section 4.1). The blob is a host
 * buffer of n bytes; the library copies what it needs to the device.
 * Errors: PW_EINVAL (bad magic, missing tensor, shape mismatch). */
int pw_model_load(pw_ctx *ctx, const void *blob, size_t n, pw_model **out);
void pw_model_free(pw_model *m);
/* 64-bit hash of the blob; every stream records the hash of its model. */
uint64_t pw_model_hash(const pw_model *m);
/* 1 when the model's probability model is the logistic mixture of three
 * components (heads of 9 outputs in the blob: weight logits, means, scale
 * pre-activations), 0 for the Laplace model (heads of 2). The paper's
 * experiments compare both (Section 4). Mixture models are four-step LL
 * models and run in the FP32 precision class only (pw_model_load returns
 * PW_EUNSUPPORTED in a BF16 or FP8 context); their streams record the model
 * in header flag 32, and each symbol is coded with its own CDF table built
 * from its key (see pw_mix_tables). */
int pw_model_mixture(const pw_model *m);

/* Architecture of a random-init model: wavelet levels (1..6), context
 * channels C (32, 64 or 128), lifting CNN channels F (16), LL mode (0: the
 * four-step nets also for LL4, 1: the autoregressive LL model, Section 3.2). */
typedef struct {
  int32_t levels, C, F, ll_mode;
} pw_model_cfg;

/* Seeded random-init weights of that architecture as a weight blob: the
 * stand-in for a trained lambda model (Section 4.1). Every tensor of the
 * format, uniform in +-b with a Kaiming-style bound per tensor role (0.05
 * for biases; head biases fixed at (0, softplus^-1(1.5))), drawn by
 * SplitMix64 keyed by (seed, tensor index, element index); the same seed
 * gives the same bytes on every host. Host-only: needs no device.
 * buf == NULL: size query (*n = bytes). Otherwise writes *n bytes to the
 * caller's buffer of cap bytes. Errors: PW_EINVAL (cfg NULL, cap too small),
 * PW_EUNSUPPORTED (configuration the library does not load). */
int pw_model_random_blob(const pw_model_cfg *cfg, uint64_t seed, void *buf, size_t cap,
                         size_t *n);
/* pw_model_random_blob followed by pw_model_load on ctx. Errors: those of
 * both. */
int pw_model_init_random(pw_ctx *ctx, const pw_model_cfg *cfg, uint64_t seed,
                         pw_model **out);

/* Graph replay of image decodes (on by default). The device work of a
 * batch image decode - stream parsing, every context-model pass, the rANS
 * passes, dequantisation, inverse lifting and post-processing - depends only
 * on the cached plan (image size, channels, batch, model, chunk layout), so
 * after a direct run of a plan in which every convolution used its final
 * (tuned) schedule, the context captures that chain into a CUDA graph (on a private
 * stream, so any user stream works, including the legacy default stream)
 * and replays it for later decodes of the plan: one launch instead of
 * hundreds. While per-kernel profiling is on, decodes run directly.
 * Results are identical either way. pw_ctx_set_graphs returns the previous
 * setting (or a negative pw_status); pw_ctx_graph_replays counts the
 * decodes served by a replayed graph. */
int pw_ctx_set_graphs(pw_ctx *ctx, int enable);
uint64_t pw_ctx_graph_replays(const pw_ctx *ctx);

/* ---- images (Sections 3.1, 3.2) ----------------------------------------- */

/* Encode one image (host or device samples) into a newly allocated host
 * bitstream *bs of *n bytes (free with pw_free). */
int pw_encode_image(pw_ctx *ctx, const pw_model *m, const pw_image *in,
                    const pw_codec_opts *opts, uint8_t **bs, size_t *n);

/* Decode one host bitstream into `out`. out->data must hold
 * height * width * channels samples of the stream's bit depth (checked
 * against out->width/height/channels, which must match the stream). With
 * out->data == NULL the library allocates a packed host image of the
 * stream's size and fills all of *out (release out->data with pw_free).
 * Errors: PW_EINVAL (model hash or size mismatch), PW_ECORRUPT, PW_ENOMEM. */
int pw_decode_image(pw_ctx *ctx, const pw_model *m, const uint8_t *bs, size_t n,
                    pw_image *out);

/* Batched encode: count images of identical size and channel count (at most
 * 65535 planes, count x channels, per call: PW_EUNSUPPORTED beyond);
 * bs[i], n[i] receive the streams (free each with pw_free). */
int pw_encode_batch(pw_ctx *ctx, const pw_model *m, int count, const pw_image *in,
                    const pw_codec_opts *opts, uint8_t **bs, size_t *n);

/* Batched decode of count streams of one model into out[0..count-1]
 * (out[i] sized like stream i). bs[i] are host pointers unless bs_on_device
 * is set, in which case they are device pointers (the streams never visit
 * the host: one kernel gathers their 64-byte headers, which the host reads
 * to form the batch, and the parse kernel validates them again). The
 * streams may differ in image size (not in channels, levels, bit depth,
 * colour mode, lossless / LL-model flags, precision class or coder layout:
 * PW_EINVAL): such a ragged batch is
 * decoded on a canvas of the largest padded size, every convolution, coder
 * pass and lifting step covering all streams in one launch, and each image
 * is bit-identical to its single decode (logistic-mixture models decode it
 * as one batch per size). Page-locked host streams and host images (pinned
 * or registered memory) are copied to and from the device directly;
 * pageable ones go through the library's pinned staging. At most 65535
 * planes (count x channels) per call: PW_EUNSUPPORTED beyond. */
int pw_decode_batch(pw_ctx *ctx, const pw_model *m, int count,
                    const uint8_t *const *bs, const size_t *n, int bs_on_device,
                    pw_image *out);

/* ---- video GOPs (Section 3.3) -------------------------------------------- */

/* Encode a group of nframes = 2^k frames: motion-compensated temporal
 * lifting (Section 3.3: the predict step warps the even frame with block
 * motion vectors, the update step maps the highpass band back with the same
 * vectors; the blob's temporal CNNs), then the lowpass band coded as an
 * image with m_low and the nframes - 1 highpass bands (batched) with m_high.
 * The vectors (16 x 16 blocks of the frames padded to 2^levels, |dy|, |dx|
 * <= 16) come from pw_motion_search's full search on the frames' integer
 * luma. frames are 8-bit gray or RGB images of one size (host or device).
 * *bs (host, free with pw_free) is a "PWGP" version-2 container: 36-byte
 * header (magic, version, nframes, width, height, temporal levels,
 * components, the two model hashes), the vectors (nframes - 1 fields of
 * ceil(Hp/16) x ceil(Wp/16) int8 (dy, dx) pairs, temporal level 1 first),
 * then, per band, a u32 length and a "PWBS" stream. */
int pw_encode_gop(pw_ctx *ctx, const pw_model *m_low, const pw_model *m_high, int nframes,
                  const pw_image *frames, const pw_codec_opts *opts, uint8_t **bs, size_t *n);
/* Inverse of pw_encode_gop into frames[0..nframes-1]; also decodes version-1
 * containers (no vectors: zero motion). The lowpass band is decoded by an
 * auxiliary context of ctx (same device and class, its own non-blocking
 * stream, created on first use and destroyed with ctx) from a second host
 * thread while ctx decodes the highpass bands; the call returns after both.
 * Errors: PW_EINVAL (models / sizes do not match the stream), PW_ECORRUPT. */
int pw_decode_gop(pw_ctx *ctx, const pw_model *m_low, const pw_model *m_high, const uint8_t *bs,
                  size_t n, int nframes, pw_image *frames);
/* Temporal lifting alone on nframes host planes of H x W floats ([frame]
 * [H][W]) with zero motion: forward writes the bands [L_T, H_T, H_{T-1}...,
 * H_1] (the highs of a level in frame order), inverse reads them back
 * (Section 3.3). */
int pw_temporal_lift(pw_ctx *ctx, const pw_model *m, int nframes, int H, int W, int forward,
                     const float *in, float *out);
/* pw_temporal_lift with motion compensation (Section 3.3): mv (host) holds
 * nframes - 1 fields of ceil(H/16) x ceil(W/16) (dy, dx) int8 pairs, level 1
 * pairs first (the layout pw_motion_search writes). Level l, pair m warps
 * frame 2m of that level by MC(f)[y, x] = f[y + dy, x + dx] for the predict
 * step and the highpass band by f[y - dy, x - dx] for the update step,
 * coordinates clamped. Errors: PW_EINVAL. */
int pw_temporal_lift_mc(pw_ctx *ctx, const pw_model *m, int nframes, int H, int W, int forward,
                        const int8_t *mv, const float *in, float *out);
/* Block motion search of a GOP (the encoder's side of Section 3.3's
 * motion-compensated prediction): luma (host, nframes x H x W int32,
 * integer samples) -> mv (host, the layout of pw_temporal_lift_mc). Field
 * (l, m) searches frame 2^l m + 2^(l-1) against frame 2^l m: per 16 x 16
 * block the (dy, dx) in [-16, 16]^2 with the least sum of absolute
 * differences (reference coordinates clamped), ties to the smaller
 * |dy| + |dx|, then dy, then dx. Exact integer arithmetic. */
int pw_motion_search(pw_ctx *ctx, int nframes, int H, int W, const int32_t *luma, int8_t *mv);

/* ---- stages of the decode path (for testing and composition) ----------- */

/* Build the 2048 x 128 uint16 CDF table bank (table id (phi + 8) * 128 + j)
 * into device buffer dev_bank (2048 * 128 * 2 bytes). Deterministic FP32
 * definition; identical on every GPU and to the reference definition. */
int pw_cdf_bank(pw_ctx *ctx, uint16_t *dev_bank);

/* Entropy-parameter index decision for n (mu, sigma) pairs (host arrays):
 * writes packed indices ((rint(16 mu) + 2^23) << 7) | j to host idx. */
int pw_entropy_index(pw_ctx *ctx, const float *mu, const float *sigma, int64_t n,
                     uint32_t *idx);

/* rANS-decode `nchunks` chunks (host arrays): chunk c holds count[c]
 * symbols coded with lanes[c] interleaved states, its bytes at
 * payload + offset[c] (nbytes[c] long). idx gives the packed table index of
 * every symbol (chunks concatenated, host); out receives the decoded
 * values ctr + r (host int32, same order). Errors: PW_ECORRUPT. */
int pw_rans_decode(pw_ctx *ctx, const uint8_t *payload, size_t payload_bytes,
                   int nchunks, const uint32_t *offset, const uint32_t *nbytes,
                   const uint32_t *count, const uint32_t *lanes,
                   const uint32_t *idx, int32_t *out);

/* Inverse of pw_rans_decode: encodes values with the given indices into a
 * new host payload (*payload, *payload_bytes; free with pw_free) and fills
 * offset[c] and nbytes[c]. */
int pw_rans_encode(pw_ctx *ctx, int nchunks, const uint32_t *count,
                   const uint32_t *lanes, const uint32_t *idx, const int32_t *values,
                   uint8_t **payload, size_t *payload_bytes, uint32_t *offset,
                   uint32_t *nbytes);

/* Allocation-free variant of pw_rans_decode, for callers that must not
 * allocate device memory while decoding (a plug-in living inside a host
 * application's fixed device-memory budget, or a real-time pipeline that
 * cannot afford cudaMalloc / cudaFree, which synchronise the device). The
 * paper has no counterpart to this call; it is a deployment convenience.
 * All arrays are DEVICE pointers: payload (payload_bytes long), the
 * per-chunk offset / nbytes / count / lanes arrays (nchunks each), idx (one
 * packed table index per symbol, chunks concatenated) and out (one int32 per
 * symbol). No context is needed: work is enqueued on cuda_stream (NULL =
 * legacy default stream) and the call returns after synchronising it.
 * The table bank, chunk descriptors and a status word live in one fixed
 * device array of about 1 MiB that every GPU loading the library holds until
 * the process exits; at most 16384 chunks per call (PW_EINVAL beyond).
 * The first call on a device looks the array's address up (make it before
 * any stream capture) and keeps it for the life of the process, so a
 * cudaDeviceReset while the library is loaded is not supported. Every call
 * reuses the array, so calls that overlap on the GPU race: serialise them.
 * Errors: PW_EINVAL (chunk limit, null pointer, value out of range),
 * PW_ECORRUPT (a corrupt or truncated chunk, and also a chunk whose offset +
 * nbytes exceeds payload_bytes or whose lane count is not 1..32: the checks
 * run on the device, where pw_rans_decode reports those two as PW_EINVAL),
 * PW_ETIMEOUT (the decoder's bounded wait for its table copy expired),
 * PW_EUNSUPPORTED, PW_ECUDA. */
int pw_rans_decode_noalloc(void *cuda_stream, const uint8_t *payload, size_t payload_bytes,
                           int nchunks, const uint32_t *offset, const uint32_t *nbytes,
                           const uint32_t *count, const uint32_t *lanes, const uint32_t *idx,
                           int32_t *out);

/* Context model on fully known quantised subbands of one component
 * (Section 3.2): q holds the 3*levels+1 subbands in coding order, each
 * (H >> lv) x (W >> lv) int32, concatenated (host). Writes mu and sigma
 * (host float, same layout) of every position as the decoder computes them
 * step by step. H and W must be multiples of 2^levels. In the INT8 class
 * mu = t / 16 and sigma = the middle of scale bin j, (t, j) the integer
 * head's outputs (exact). */
int pw_context_params(pw_ctx *ctx, const pw_model *m, int H, int W,
                      const int32_t *q, float *mu, float *sigma);

/* Logistic-mixture counterpart of pw_context_params: par (host float,
 * 9 per position, positions in the layout of pw_context_params) receives
 * (w_0, w_1, w_2, mu_0, mu_1, mu_2, sigma_0, sigma_1, sigma_2) of every
 * position as the decoder computes them, sigma_k = softplus of the head's
 * scale outputs. Errors: PW_EUNSUPPORTED for a Laplace model (and
 * pw_context_params returns PW_EUNSUPPORTED for a mixture model). */
int pw_context_mixture(pw_ctx *ctx, const pw_model *m, int H, int W,
                       const int32_t *q, float *par);

/* CDF tables of n logistic-mixture keys. key9 (host int32, 9 per key):
 * q_0 q_1 q_2 (mean offsets from the centre in 1/8 steps, -255..255),
 * j_0 j_1 j_2 (scale bins 0..127, the Laplace tables' bins), g_0 g_1 g_2
 * (log-weights in 1/4 steps, -31..0), each clamped to its range. cdf (host
 * uint16, 128 per key) receives cdf[0] = 0 .. cdf[127] = 2^15 of the 127
 * symbols (escape, residuals -62..62 around the centre, escape): the
 * mixture sum_k exp(g_k / 4) S((u - q_k / 8) / b_{j_k}) / sum_k exp(g_k / 4),
 * S the logistic function, at the 126 symbol edges u, quantised like the
 * Laplace tables, every step one correctly rounded FP32 operation (the
 * exponential the library's own), so encoders and decoders on any GPU build
 * identical tables. The decision of a key from the mixture parameters
 * (w, mu, sigma): a = the first component of largest w, centre
 * rint(mu_a), q_k = rint(8 (mu_k - centre)), g_k = rint(4 (w_k - w_a)),
 * j_k = the bin of sigma_k, all in FP32. */
int pw_mix_tables(pw_ctx *ctx, int64_t n, const int32_t *key9, uint16_t *cdf);

/* Forward / inverse learned lifting DWT of one plane (Section 3.1, Fig. 2)
 * on host float arrays: x is H x W; sb holds the subbands in coding order
 * (same layout as pw_context_params). lossless selects integer lifting. */
int pw_lift_forward(pw_ctx *ctx, const pw_model *m, int H, int W, int lossless,
                    const float *x, float *sb);
int pw_lift_inverse(pw_ctx *ctx, const pw_model *m, int H, int W, int lossless,
                    const float *sb, float *x);

/* Decode only the quantised coefficients of a host stream (context model +
 * rANS, no inverse transform). q (host int32) receives ncomp * Hp * Wp
 * values, Hp / Wp the sizes padded to multiples of 2^levels, laid out
 * subband-major: subband i (coding order) of component c at
 * q[ncomp * off_i + c * h_i * w_i + y * w_i + x], off_i = sum of h_j * w_j
 * over j < i. */
int pw_decode_symbols(pw_ctx *ctx, const pw_model *m, const uint8_t *bs, size_t n,
                      int32_t *q);

/* Encoder analysis only: colour transform, forward lifting DWT and
 * quantiser of one image; q as in pw_decode_symbols. */
int pw_analyse(pw_ctx *ctx, const pw_model *m, const pw_image *in,
               const pw_codec_opts *opts, int32_t *q);

/* Entropy-code a given quantised latent (host q, layout as in
 * pw_decode_symbols) into a stream for an image of the given size, channel
 * count, bit depth and colour code (0 gray, 1 YCbCr, 2 RCT, 3 raw planes). */
int pw_encode_latent(pw_ctx *ctx, const pw_model *m, const int32_t *q, int width,
                     int height, int channels, int bitdepth, int colour,
                     const pw_codec_opts *opts, uint8_t **bs, size_t *n);

/* One context-model convolution on the tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation), for testing the building block of Section 3.2's nets:
 * y = act(conv_ks(x) + b) with zero padding, act = LeakyReLU(0.01) if act.
 * x: host [P][H][W][cin] float (rounded to BF16), w: host [cout][cin][ks][ks],
 * b: host [cout], y: host [P][H][W][cout] (BF16-rounded results as float).
 * ks in {1, 3}; cin a multiple of 32 (of 64 above 64); cout in {32, 64, 128,
 * 192, 256}. Errors: PW_EUNSUPPORTED (shape), PW_ETIMEOUT (a bounded
 * wait expired). */
int pw_conv_bf16(pw_ctx *ctx, int P, int H, int W, int cin, int cout, int ks, int act,
                 const float *x, const float *w, const float *b, float *y);

/* ---- decode server ------------------------------------------------------- */
/* A decode server for a stream of requests of mixed sizes (the serving
 * workload: images that arrive one at a time at random instants). The paper
 * decodes one image per call; the server adds continuous batching around
 * that same decode path and changes no result.
 *
 * pw_server_create starts `lanes` worker threads (1..16). Each lane owns a
 * CUDA stream and a context of ctx's device and precision; all lanes share
 * the model m (read only; m and ctx must outlive the server, and ctx itself
 * is not used by the lanes). A lane repeatedly takes the oldest queued
 * request together with queued requests of the same format (channels, bit
 * depth, levels, coder layout; at most max_batch) whose sizes are close:
 * a request joins while the batch's canvas (its largest padded size) times
 * its image count stays within 1.5 times the images' own padded area. The
 * batch is decoded in one call (a ragged batch when the sizes differ, see
 * pw_decode_batch; logistic-mixture models batch equal sizes only). A
 * batch starts only when its device workspace fits in hbm_budget
 * bytes next to the workspaces the other lanes hold; an idle lane frees its
 * workspace. Lanes run concurrently, so different sizes overlap on the GPU.
 * Each result is bit-identical to pw_decode_image of the same stream on a
 * context of the same precision.
 *
 * pw_server_submit copies the host stream bs[0..n) and returns at once with
 * a ticket. Errors: those of the header checks of pw_decode_image (PW_ECORRUPT
 * not a stream, PW_EINVAL another model or precision class),
 * PW_EAGAIN (one request alone exceeds hbm_budget, or 4096 requests are
 * queued). pw_server_poll waits up to timeout_ms for a ticket (0: do not
 * wait) and copies the decoded image into out (host or device, packed or
 * strided, as pw_decode_image); the ticket is then released. It returns the
 * decode's status (a failed batch is re-decoded one request at a time, so a
 * corrupt stream fails only its own ticket), PW_EAGAIN (timeout_ms = 0, not
 * done), PW_ETIMEOUT, or PW_EINVAL (unknown ticket, or out does not match
 * the image; the ticket then stays valid).
 * The submit / poll / stats calls are thread-safe. pw_server_destroy
 * finishes the batches in flight, drops queued requests and frees all. */
typedef struct pw_server pw_server;
typedef struct {
  uint64_t submitted, completed, failed, rejected, queued, batches;
  uint64_t held_bytes;       /* workspace bytes the lanes hold now          */
  double p50_ms, p99_ms;     /* submit -> result ready, completed requests  */
  double mpix_per_s;         /* decoded pixels / (last result - first submit) */
} pw_stats;
/* Estimated device workspace bytes for decoding `count` streams of the
 * geometry of host stream bs[0..n) in one batch on ctx (the figure the
 * server's admission uses). Errors as pw_decode_image's header checks. */
int pw_decode_footprint(pw_ctx *ctx, const pw_model *m, const uint8_t *bs, size_t n, int count,
                        uint64_t *bytes);
int pw_server_create(pw_ctx *ctx, const pw_model *m, size_t hbm_budget, int lanes,
                     int max_batch, pw_server **out);
int pw_server_submit(pw_server *s, const uint8_t *bs, size_t n, uint64_t *ticket);
int pw_server_poll(pw_server *s, uint64_t ticket, pw_image *out, int timeout_ms);
int pw_server_stats(pw_server *s, pw_stats *out);
void pw_server_destroy(pw_server *s);

/* ---- misc ---------------------------------------------------------------- */
void pw_free(void *p);
const char *pw_strerror(int status);
/* Message of the last failure on the calling thread. */
const char *pw_last_error(void);
/* Number of kernels this library launched on the context so far. */
uint64_t pw_ctx_launch_count(const pw_ctx *ctx);

/* Autotuner of the tensor-core convolutions. For every convolution variant
 * and size class (log2 of its tile count) it picks, among up to four
 * candidates, the MMA issue schedule (one tile or two interleaved tiles per
 * round) crossed with the pipeline shape (the default or a shallower
 * pipeline for the plain convolutions; for the compact head, the tile shape
 * with the fewest or the second-fewest tiles), by sampling the candidates
 * round robin on the first real launches of the class in the process (CUDA
 * events read back without synchronising, 3 samples each) and keeping the
 * fastest median; results never depend on the choice.
 * pw_autotune(0 / 1) disables / enables sampling of classes not tuned yet
 * (default on; disabled classes use the default schedule) and returns the
 * previous setting. pw_autotune_report writes one line per tuned class
 * ("ks kb ncta epilogue fp8 log2tiles choice t0 t1 t2 t3": choice bit 0 =
 * paired issue, bit 1 = alternative shape; t = median sample time of each
 * candidate in microseconds, -1 = not sampled; epilogue 0 store, 1 ConvLSTM
 * gates, 2 head, 3 compact head, 4 store with a 16-channel BF16 input block)
 * into buf (NUL-terminated, truncated to n) and returns the full length. */
int pw_autotune(int enable);
int pw_autotune_report(char *buf, size_t n);
/* 1 when no convolution launch since the previous call (the first call:
 * since the library loaded) was of a class still being tuned, else 0. A
 * service can repeat its warm-up decodes until a decode is followed by 1,
 * so that no later launch of those shapes is a tuning sample. */
int pw_autotune_settled(void);

/* Per-kernel-class timing. pw_ctx_profile(ctx, 1) resets the counters and
 * records a CUDA event pair on the context's stream around every launch that
 * follows (adds a few microseconds per launch); 0 stops recording.
 * pw_ctx_kernel_stats fills up to max entries and returns the number of
 * classes seen (negative pw_status on error). flops / bytes are the
 * algorithmic work of the recorded launches (not hardware counters). */
typedef struct {
  char name[40];
  uint64_t launches;
  double ms, flops, bytes;
} pw_kernel_stat;
int pw_ctx_profile(pw_ctx *ctx, int enable);
int pw_ctx_kernel_stats(pw_ctx *ctx, pw_kernel_stat *out, int max);
/* Like pw_ctx_profile, but records only the kernel classes whose bit is set
 * in class_mask (bit k = class index k, see pw_kernel_class; 0 stops), so
 * that one class can be timed with little perturbation of the others. */
int pw_ctx_profile_classes(pw_ctx *ctx, uint32_t class_mask);
/* Class index of a name that pw_ctx_kernel_stats reports, or -1. */
int pw_kernel_class(const char *name);

#ifdef __cplusplus
}
#endif
#endif /* PWAVE_H */
