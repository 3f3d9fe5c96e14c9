// Batch encode / decode drivers and their small device kernels (stream
// parsing, dequantisation, step gathers).
#include <algorithm>
#include <cstring>

#include "codec.h"
#include "driver.h"

namespace pw {

// ---------------------------------------------------------------------------
// Device kernels

__device__ __forceinline__ uint32_t rd32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
__device__ __forceinline__ uint16_t rd16(const uint8_t *p) {
  return (uint16_t)((uint32_t)p[0] | ((uint32_t)p[1] << 8));
}

// Header check of one stream (a mismatch with the plan: kStHeader) and
// the byte range of its chunk gc (out of range or out of order:
// kStCorrupt). Returns the chunk's descriptor fields.
__device__ __forceinline__ void parse_chunk(const uint8_t *s, uint64_t len,
                                            const ParseExpect &ex, uint32_t width,
                                            uint32_t height, uint32_t nch, uint32_t gc,
                                            bool &hdr, bool &ok, const uint8_t *&data,
                                            uint32_t &nbytes) {
  const uint64_t base = 64ull + 4ull * (nch + 1);
  hdr = s != nullptr && len >= base;
  if (hdr) {
    hdr = s[0] == 'P' && s[1] == 'W' && s[2] == 'B' && s[3] == 'S' && rd16(s + 4) == 1 &&
         rd16(s + 6) == ex.flags && rd32(s + 8) == width && rd32(s + 12) == height &&
         s[16] == ex.ncomp && s[17] == ex.levels && s[18] == ex.bitdepth &&
         s[19] == ex.colour && rd16(s + 28) == kT && s[30] == kLogM && s[31] == kMaxLanes &&
         rd32(s + 32) == ex.chunk && rd32(s + 36) == nch &&
         rd32(s + 40) == (uint32_t)ex.hash && rd32(s + 44) == (uint32_t)(ex.hash >> 32) &&
         s[52] == ex.lane_byte;
  }
  const uint32_t pb = hdr ? rd32(s + 48) : 0;
  ok = hdr && base + pb <= len;
  uint32_t o0 = 0, o1 = 0;
  if (ok) {
    o0 = rd32(s + 64 + 4 * gc);
    o1 = rd32(s + 64 + 4 * (gc + 1));
    ok = o0 <= o1 && o1 <= pb;
  }
  data = ok ? s + base + o0 : nullptr;
  nbytes = ok ? o1 - o0 : 0;
}

// The stream's quantiser steps (delta_L, delta_H) into deltas[2 b ..].
__device__ __forceinline__ void parse_deltas(const uint8_t *s, bool ok, int b, float *deltas,
                                             uint32_t *status) {
  float dl = 1.f, dh = 1.f;
  if (ok) {
    dl = __uint_as_float(rd32(s + 20));
    dh = __uint_as_float(rd32(s + 24));
  }
  if (!(dl > 0.f) || !(dh > 0.f)) { dl = dh = 1.f; atomicOr(status, kStHeader); }
  deltas[2 * b] = dl;
  deltas[2 * b + 1] = dh;
}

// Validate every stream's header against the plan and fill the decode
// chunk descriptors (bitstream parse, done on the device). One thread per
// (image, component, chunk of the component).
__global__ void k_parse_streams(const uint8_t *const *streams, const uint64_t *lens, int B,
                                ParseExpect ex, const TplDev *tpl, int nck,
                                DecChunk *out, float *deltas, uint32_t *status) {
  const int64_t n = (int64_t)B * ex.ncomp * nck;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % nck);
    const int comp = (int)((e / nck) % ex.ncomp);
    const int b = (int)(e / ((int64_t)nck * ex.ncomp));
    const uint8_t *s = streams[b];
    bool hdr, ok;
    DecChunk d;
    parse_chunk(s, lens[b], ex, ex.width, ex.height, (uint32_t)nck * ex.ncomp,
                (uint32_t)(comp * nck + c), hdr, ok, d.data, d.nbytes);
    const TplDev t = tpl[c];
    d.count = t.count;
    d.first = t.first;
    d.lanes = (uint16_t)t.lanes;
    const int p = b * ex.ncomp + comp;
    d.plane = (uint16_t)p;
    out[t.gbase + (int64_t)p * t.gcount + t.j] = d;
    if (!hdr) atomicOr(status, kStHeader);
    else if (!ok) atomicOr(status, kStCorrupt);
    if (comp == 0 && c == 0) parse_deltas(s, ok, b, deltas, status);
  }
}

// The same for a ragged batch: one thread per entry of the host-built
// table (every stream checked against its own width and height).
__global__ void k_parse_ragged(const uint8_t *const *streams, const uint64_t *lens,
                               const uint32_t *wh, ParseExpect ex, const RagTpl *tpl,
                               int64_t ntpl, DecChunk *out, float *deltas, uint32_t *status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ntpl;
       e += (int64_t)gridDim.x * blockDim.x) {
    const RagTpl t = tpl[e];
    const uint8_t *s = streams[t.b];
    bool hdr, ok;
    DecChunk d;
    parse_chunk(s, lens[t.b], ex, wh[2 * t.b], wh[2 * t.b + 1], t.nch, t.gc, hdr, ok, d.data,
                d.nbytes);
    d.count = t.count;
    d.first = t.first;
    d.lanes = t.lanes;
    d.plane = (uint16_t)(t.b * ex.ncomp + t.comp);
    out[t.out] = d;
    if (!hdr) atomicOr(status, kStHeader);
    else if (!ok) atomicOr(status, kStCorrupt);
    if (t.gc == 0) parse_deltas(s, ok, (int)t.b, deltas, status);
  }
}

// The 64-byte headers of device-resident streams (zeros past a stream's
// end), one block per stream: read on the host to form a batch.
__global__ void k_gather_headers(const uint8_t *const *ptrs, const uint64_t *lens, int B,
                                 uint8_t *out) {
  const int b = blockIdx.x, i = threadIdx.x;
  if (b >= B || i >= 64) return;
  const uint8_t *s = ptrs[b];
  out[(int64_t)b * 64 + i] = (s && (uint64_t)i < lens[b]) ? s[i] : 0;
}

// Ragged batches: zero the 16-byte units of an activation buffer outside
// each plane's extent. One block per canvas row (plane p, row y).
__global__ void __launch_bounds__(128) k_zero_outside(uint4 *__restrict__ buf, int layout,
                                                      int P, int H, int W, int NG,
                                                      const int2 *__restrict__ ext, int esh) {
  const int row = blockIdx.x;
  const int p = row / H, y = row - p * H;
  if (p >= P) return;
  const int hv = ext[p].x >> esh, wv = ext[p].y >> esh;
  const int x0 = y >= hv ? 0 : wv;
  if (x0 >= W) return;
  const int nx = W - x0;
  const int64_t n = (int64_t)nx * NG;
  const int64_t w4q = ((W + 3) & ~3) >> 2;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    int64_t o;
    if (layout == ZL_GROUP) {
      const int g = (int)(e / nx), x = x0 + (int)(e % nx);
      o = (((int64_t)p * NG + g) * H + y) * W + x;
    } else {
      const int x = x0 + (int)(e / NG), g = (int)(e % NG);
      o = layout == ZL_PIXEL ? (((int64_t)p * H + y) * W + x) * NG + g
                             : ((((int64_t)p * H + y) * 4 + (x & 3)) * w4q + (x >> 2)) * NG + g;
    }
    buf[o] = make_uint4(0u, 0u, 0u, 0u);
  }
}

__global__ void k_dequant_all(const int32_t *__restrict__ Q, float *__restrict__ Yf,
                              int64_t n, SbTable tb, int nc, const float *__restrict__ deltas) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = 0;
    while (i + 1 < tb.nsb && tb.base[i + 1] <= e) ++i;
    const int p = (int)((e - tb.base[i]) / tb.hw[i]);
    const int b = p / nc;
    const float d = deltas[2 * b + (i > 0 ? 1 : 0)];
    Yf[e] = __fdiv_rn((float)Q[e], d);
  }
}

__global__ void k_quant_all(const float *__restrict__ Yf, int32_t *__restrict__ Q, int64_t n,
                            SbTable tb, float dl, float dh) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float d = e < tb.base[1] ? dl : dh;
    Q[e] = (int32_t)rintf(__fmul_rn(Yf[e], d));
  }
}

__global__ void k_gather_step(const int32_t *__restrict__ Qi, int P, int h, int w, int step,
                              int32_t *__restrict__ vals, int64_t nk) {
  const int64_t n = (int64_t)P * nk;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / nk);
    const int q = (int)(e % nk);
    int y, x;
    if (step >= 0) step_pos(w, step, q, y, x);
    else { y = q / w; x = q % w; }
    vals[e] = Qi[(int64_t)p * h * w + (int64_t)y * w + x];
  }
}

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 152 * 32 ? 152 * 32 : (g < 1 ? 1 : g));
}

// ---------------------------------------------------------------------------
SbTable make_sbtable(const Geometry &g, int P) {
  SbTable t{};
  t.nsb = g.nsb;
  for (int i = 0; i < g.nsb; ++i) {
    t.base[i] = (int64_t)P * g.soff[i];
    t.hw[i] = (int64_t)g.sh[i] * g.sw[i];
  }
  t.base[g.nsb] = (int64_t)P * g.plane_elems;
  return t;
}

void launch_gather_step(const int32_t *Qi, int P, int h, int w, int step, int32_t *vals,
                        int64_t nk, cudaStream_t st) {
  k_gather_step<<<grid_for((int64_t)P * nk), 256, 0, st>>>(Qi, P, h, w, step, vals, nk);
}
void launch_dequant_all(const int32_t *Q, float *Yf, int64_t n, const SbTable &tb, int nc,
                        const float *deltas, cudaStream_t st) {
  k_dequant_all<<<grid_for(n), 256, 0, st>>>(Q, Yf, n, tb, nc, deltas);
}
void launch_quant_all(const float *Yf, int32_t *Q, int64_t n, const SbTable &tb, float dl,
                      float dh, cudaStream_t st) {
  k_quant_all<<<grid_for(n), 256, 0, st>>>(Yf, Q, n, tb, dl, dh);
}
void launch_parse_streams(const uint8_t *const *streams, const uint64_t *lens, int B,
                          const ParseExpect &ex, const TplDev *tpl, int nck, DecChunk *out,
                          float *deltas, uint32_t *status, cudaStream_t st) {
  int64_t n = (int64_t)B * ex.ncomp * nck;
  k_parse_streams<<<grid_for(n), 256, 0, st>>>(streams, lens, B, ex, tpl, nck, out, deltas,
                                                status);
}

void launch_parse_ragged(const uint8_t *const *streams, const uint64_t *lens,
                         const uint32_t *wh, const ParseExpect &ex, const RagTpl *tpl,
                         int64_t ntpl, DecChunk *out, float *deltas, uint32_t *status,
                         cudaStream_t st) {
  k_parse_ragged<<<grid_for(ntpl), 256, 0, st>>>(streams, lens, wh, ex, tpl, ntpl, out, deltas,
                                                 status);
}
void launch_gather_headers(const uint8_t *const *ptrs, const uint64_t *lens, int B, uint8_t *out,
                           cudaStream_t st) {
  if (B > 0) k_gather_headers<<<B, 64, 0, st>>>(ptrs, lens, B, out);
}
void launch_zero_outside(void *buf, int layout, int P, int H, int W, int NG, const int2 *ext,
                         int esh, cudaStream_t st) {
  if (P < 1 || H < 1 || W < 1 || NG < 1 || !ext) return;
  k_zero_outside<<<P * H, 128, 0, st>>>(static_cast<uint4 *>(buf), layout, P, H, W, NG, ext,
                                        esh);
}

}  // namespace pw
