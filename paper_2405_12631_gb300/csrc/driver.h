// Device-side stream parsing, (de)quantisation and gathers: declarations.
#pragma once
#include "codec.h"

namespace pw {

struct ParseExpect {
  uint32_t width, height;
  uint32_t ncomp, levels, bitdepth, colour;
  uint32_t flags, chunk;
  uint64_t hash;
  uint32_t lane_byte;   // header byte 52 (lane rule) of the batch's streams
};

// Per-component chunk template on the device: where the chunk's decode
// descriptor goes (group block base, chunks per plane in the group, index
// within the group) and its symbol range.
struct TplDev {
  int64_t gbase;
  int32_t gcount, j;
  uint32_t first, count, lanes;
};

// Ragged batches: one entry per (stream, component, chunk); streams of one
// class (format, model) but their own sizes, so every entry says where its
// descriptor goes and which chunk of which stream it is.
struct RagTpl {
  int64_t out;            // index of the decode descriptor
  uint32_t first, count;
  uint16_t lanes, comp;
  uint32_t b;             // stream
  uint32_t gc, nch;       // chunk index within the stream, chunks in the stream
};

struct SbTable {
  int nsb;
  int64_t base[20];  // element offset of subband i over all planes (+ end)
  int64_t hw[20];
};

SbTable make_sbtable(const Geometry &g, int P);
void launch_gather_step(const int32_t *Qi, int P, int h, int w, int step, int32_t *vals,
                        int64_t nk, cudaStream_t st);
void launch_dequant_all(const int32_t *Q, float *Yf, int64_t n, const SbTable &tb, int nc,
                        const float *deltas, cudaStream_t st);
void launch_quant_all(const float *Yf, int32_t *Q, int64_t n, const SbTable &tb, float dl,
                      float dh, cudaStream_t st);
void launch_parse_streams(const uint8_t *const *streams, const uint64_t *lens, int B,
                          const ParseExpect &ex, const TplDev *tpl, int nck, DecChunk *out,
                          float *deltas, uint32_t *status, cudaStream_t st);
// out[b * 64 ..]: the first 64 bytes of device stream b (zeros past its end)
void launch_gather_headers(const uint8_t *const *ptrs, const uint64_t *lens, int B, uint8_t *out,
                           cudaStream_t st);
// wh: the streams' expected (width, height), 2 per stream
void launch_parse_ragged(const uint8_t *const *streams, const uint64_t *lens,
                         const uint32_t *wh, const ParseExpect &ex, const RagTpl *tpl,
                         int64_t ntpl, DecChunk *out, float *deltas, uint32_t *status,
                         cudaStream_t st);

}  // namespace pw
