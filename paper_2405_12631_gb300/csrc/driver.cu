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
    const uint64_t len = lens[b];
    const uint32_t nch = (uint32_t)nck * ex.ncomp;
    const uint64_t base = 64ull + 4ull * (nch + 1);
    // header fields that must match the plan (a mismatch: kStHeader), then
    // the payload and offset table (out of range or out of order: kStCorrupt)
    bool hdr = s != nullptr && len >= base;
    if (hdr) {
      hdr = s[0] == 'P' && s[1] == 'W' && s[2] == 'B' && s[3] == 'S' && rd16(s + 4) == 1 &&
           rd16(s + 6) == ex.flags && rd32(s + 8) == ex.width && rd32(s + 12) == ex.height &&
           s[16] == ex.ncomp && s[17] == ex.levels && s[18] == ex.bitdepth &&
           s[19] == ex.colour && rd16(s + 28) == kT && s[30] == kLogM && s[31] == kMaxLanes &&
           rd32(s + 32) == ex.chunk && rd32(s + 36) == nch &&
           rd32(s + 40) == (uint32_t)ex.hash && rd32(s + 44) == (uint32_t)(ex.hash >> 32) &&
           s[52] == ex.lane_byte;
    }
    uint32_t pb = hdr ? rd32(s + 48) : 0;
    bool ok = hdr && base + pb <= len;
    const int gc = comp * nck + c;
    uint32_t o0 = 0, o1 = 0;
    if (ok) {
      o0 = rd32(s + 64 + 4 * gc);
      o1 = rd32(s + 64 + 4 * (gc + 1));
      ok = o0 <= o1 && o1 <= pb;
    }
    const TplDev t = tpl[c];
    DecChunk d;
    d.data = ok ? s + base + o0 : nullptr;
    d.nbytes = ok ? o1 - o0 : 0;
    d.count = t.count;
    d.first = t.first;
    d.lanes = (uint16_t)t.lanes;
    const int p = b * ex.ncomp + comp;
    d.plane = (uint16_t)p;
    out[t.gbase + (int64_t)p * t.gcount + t.j] = d;
    if (!hdr) atomicOr(status, kStHeader);
    else if (!ok) atomicOr(status, kStCorrupt);
    if (comp == 0 && c == 0) {
      float dl = 1.f, dh = 1.f;
      if (ok) {
        uint32_t a = rd32(s + 20), bb = rd32(s + 24);
        dl = __uint_as_float(a);
        dh = __uint_as_float(bb);
      }
      if (!(dl > 0.f) || !(dh > 0.f)) { dl = dh = 1.f; atomicOr(status, kStHeader); }
      deltas[2 * b] = dl;
      deltas[2 * b + 1] = dh;
    }
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

}  // namespace pw
