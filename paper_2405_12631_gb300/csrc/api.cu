// C ABI of libpwave (include/pwave.h) and the host-side batch drivers.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <thread>

#include "codec.h"
#include "ctx_tc.h"
#include "driver.h"
#include "ll_ar.h"
#include "prof.h"

namespace pw {

// Planes (images x components) of one batch: every launch indexes them with
// a 16-bit descriptor field or as the grid's z dimension.
constexpr int64_t kMaxPlanes = 65535;

static thread_local std::string g_last_error;
void set_last_error(const std::string &s) { g_last_error = s; }

static inline void bump(pw_ctx *ctx, int n = 1) { ctx->launches += (uint64_t)n; }

// Device buffer of a plan that grows on demand, from the context's
// stream-ordered pool.
struct PoolBuf {
  void *p = nullptr;
  size_t cap = 0;
  cudaStream_t st = nullptr;
  int ensure(size_t n) {
    if (n <= cap) return PW_OK;
    pool_free(p, st);
    p = nullptr;
    cap = 0;
    if (pool_alloc(&p, n ? n : 1, st) != PW_OK) return PW_ENOMEM;
    cap = n;
    return PW_OK;
  }
  ~PoolBuf() { pool_free(p, st); }
};

// Device buffer that grows on demand.
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  int ensure(size_t n) {
    if (n <= cap) return PW_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc(&p, n ? n : 1) != cudaSuccess) { set_last_error("device allocation failed"); return PW_ENOMEM; }
    cap = n;
    return PW_OK;
  }
  ~DevBuf() { if (p) cudaFree(p); }
};
struct HostBuf {  // pinned
  void *p = nullptr;
  size_t cap = 0;
  int ensure(size_t n) {
    if (n <= cap) return PW_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    if (cudaMallocHost(&p, n ? n : 1) != cudaSuccess) { set_last_error("pinned allocation failed"); return PW_ENOMEM; }
    cap = n;
    return PW_OK;
  }
  ~HostBuf() { if (p) cudaFreeHost(p); }
};

struct Plan {
  std::string key;
  Geometry g;
  int B = 0;
  Workspace ws;
  // decode
  PoolBuf d_chunks, d_tpl, d_deltas, d_ptrs, d_lens, d_stage, d_out;
  HostBuf h_stage, h_small, h_out;
  // ragged batches: the streams' sizes, the planes' extents and the parse
  // table (one pinned host image, one device copy)
  PoolBuf d_rag;
  HostBuf h_rag;
  std::vector<int64_t> gbase;   // decode descriptor block of each group
  // encode
  PoolBuf d_enc, d_ops, d_scratch, d_states, d_nwords, d_outoff, d_payload, d_img;
  // the decode chain as a CUDA graph (captured after one direct run)
  cudaStream_t stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const float *graph_recon = nullptr;   // its reconstructed planes
  uint64_t graph_launches = 0;          // kernel launches it holds
  bool tuned_run = false;               // the last direct run used final schedules only
  bool graph_bad = false;               // capture failed: stay direct
  ~Plan() {
    if (gexec) {
      cudaStreamSynchronize(stream);
      cudaGraphExecDestroy(gexec);
    }
  }
  void set_stream(cudaStream_t s) {
    stream = s;
    for (PoolBuf *b : {&d_chunks, &d_tpl, &d_deltas, &d_ptrs, &d_lens, &d_stage, &d_out, &d_rag, &d_enc,
                       &d_ops, &d_scratch, &d_states, &d_nwords, &d_outoff, &d_payload, &d_img})
      b->st = s;
  }
};

// Scratch of the GOP calls, kept per context and grown on demand: hundreds
// of MB per 1080p GOP, which allocating and freeing on every call would
// cost (each cudaFree synchronises the device), and pinned staging for
// host frames.
struct GopBufs {
  DevBuf bands, frames, t0, t1, img, mv, warp, luma;
  HostBuf h_img;
};

struct PlanCache {
  std::vector<std::unique_ptr<Plan>> plans;
  GopBufs gop;
  // headers of device-resident stream batches (pointer table and headers)
  DevBuf d_hdr;
  HostBuf h_hdr;
};

Prof &prof_of(pw_ctx *ctx) { return *reinterpret_cast<Prof *>(ctx->prof); }

static PlanCache &cache_of(pw_ctx *ctx) {
  return *reinterpret_cast<PlanCache *>(ctx->plan_cache);
}

static std::string geo_key(const char *kind, const Geometry &g, int B, const Model &m, int params) {
  char buf[256];
  // the model's unique id and channel count: a workspace is sized by both;
  // the chunk layout (balanced flag, lane rule) shapes the plan's chunk tables
  snprintf(buf, sizeof(buf), "%s:%d:%d:%d:%d:%d:%d:%d:%d:%d:%d:%d:%d:%llu:%d:%d", kind, g.H, g.W,
           g.nc, g.levels, g.colour, g.bitdepth, g.lossless, g.ll_ar, g.chunk, g.balanced,
           g.lane_shift, B, (unsigned long long)m.uid, m.C, params);
  return buf;
}

static int get_plan(pw_ctx *ctx, Model &m, const Geometry &g, int B, const char *kind,
                    bool params, Plan **out) {
  const std::string key = geo_key(kind, g, B, m, params ? 1 : 0);
  auto &pc = cache_of(ctx);
  for (auto &p : pc.plans)
    if (p->key == key) { *out = p.get(); return PW_OK; }
  // keep the cache small: drop the oldest plans beyond 6
  while (pc.plans.size() >= 6) pc.plans.erase(pc.plans.begin());
  std::unique_ptr<Plan> p(new Plan());
  p->key = key;
  p->g = g;
  p->B = B;
  p->set_stream(ctx->stream);
  int s = m.prepare(ctx->precision);
  if (s != PW_OK) return s;
  s = p->ws.alloc(g, B * g.nc, m.C, params, ctx->precision, ctx->stream, m.mix);
  if (s != PW_OK) return s;
  if (!strcmp(kind, "dec") || !strcmp(kind, "sym")) {
    // decode descriptor layout: group blocks of P x count
    const int P = B * g.nc;
    p->gbase.assign(g.nsb * 4, 0);
    int64_t acc = 0;
    for (int gi = 0; gi < g.nsb * 4; ++gi) {
      p->gbase[gi] = acc;
      acc += (int64_t)P * g.group_count[gi];
    }
    s = p->d_chunks.ensure(std::max<int64_t>(acc, 1) * sizeof(DecChunk));
    if (s) return s;
    const int nck = (int)g.chunks.size();
    std::vector<TplDev> tpl(nck);
    for (int c = 0; c < nck; ++c) {
      const ChunkTpl &t = g.chunks[c];
      const int gi = t.sb * 4 + (t.step < 0 ? 0 : t.step);
      tpl[c].gbase = p->gbase[gi];
      tpl[c].gcount = g.group_count[gi];
      tpl[c].j = c - g.group_first[gi];
      tpl[c].first = t.first;
      tpl[c].count = t.count;
      tpl[c].lanes = t.lanes;
    }
    if ((s = p->d_tpl.ensure(std::max(nck, 1) * sizeof(TplDev)))) return s;
    if (nck)
      cudaMemcpyAsync(p->d_tpl.p, tpl.data(), nck * sizeof(TplDev), cudaMemcpyHostToDevice,
                      ctx->stream);
    if ((s = p->d_deltas.ensure(2 * B * sizeof(float)))) return s;
    if ((s = p->d_ptrs.ensure(B * sizeof(void *)))) return s;
    if ((s = p->d_lens.ensure(B * sizeof(uint64_t)))) return s;
    if ((s = p->h_small.ensure(B * 16 + 64))) return s;
  } else if (!strcmp(kind, "rag")) {
    // ragged batches build their descriptor tables per call
    if ((s = p->d_deltas.ensure(2 * B * sizeof(float)))) return s;
    if ((s = p->d_ptrs.ensure(B * sizeof(void *)))) return s;
    if ((s = p->d_lens.ensure(B * sizeof(uint64_t)))) return s;
    if ((s = p->h_small.ensure(B * 16 + 64))) return s;
  }
  pc.plans.push_back(std::move(p));
  *out = pc.plans.back().get();
  return PW_OK;
}

// Release every cached workspace of the context (after its work finished).
void drop_plans(pw_ctx *ctx) {
  cudaStreamSynchronize(ctx->stream);
  cache_of(ctx).plans.clear();
}

static int check_status(pw_ctx *ctx, Workspace *ws = nullptr) {
  if (launch_failed()) { launch_failed() = false; return PW_EUNSUPPORTED; }
  if (ws && tc_precision(ctx->precision)) {
    cudaStreamSynchronize(ctx->stream);
    if (tc_error(*ws)) { set_last_error("a tensor-core kernel's bounded wait expired"); return PW_ETIMEOUT; }
  }
  uint32_t st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, ctx->status, 4, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) { set_last_error(std::string("CUDA: ") + cudaGetErrorString(e)); return PW_ECUDA; }
  e = cudaGetLastError();
  if (e != cudaSuccess) { set_last_error(std::string("CUDA launch: ") + cudaGetErrorString(e)); return PW_ECUDA; }
  if (st & kStHeader) { set_last_error("stream header does not match (model, size or format)"); return PW_EINVAL; }
  if (st & kStCorrupt) { set_last_error("corrupt or truncated bitstream"); return PW_ECORRUPT; }
  if (st & kStRange) { set_last_error("value outside the coder's range"); return PW_EINVAL; }
  if (st & kStTimeout) { set_last_error("a kernel's bounded wait expired"); return PW_ETIMEOUT; }
  return PW_OK;
}

// Synchronise and report launch / kernel errors (no status word).
static int finish(pw_ctx *ctx) {
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) { set_last_error(std::string("CUDA: ") + cudaGetErrorString(e)); return PW_ECUDA; }
  if (launch_failed()) { launch_failed() = false; return PW_EUNSUPPORTED; }
  return PW_OK;
}

// The autoregressive LL model's weights for this context's class (the
// integer-network class uses the quantised copy).
static ArWeightsDev ar_weights(const pw_ctx *ctx, const Model &m) {
  if (ctx->precision == PW_PREC_INT8 && m.intn) {
    const IntNets &n = *m.intn;
    ArWeightsDev w{n.ar_w5, n.ar_b5, n.ar_w1, n.ar_b1, n.ar_wh, n.ar_bh};
    w.iq = 1; w.n5 = n.ar_n5; w.n1 = n.ar_n1; w.n_mu = n.ar_nmu; w.n_rho = n.ar_nrho;
    return w;
  }
  return ArWeightsDev{m.ar_w5, m.ar_b5, m.ar_w1, m.ar_b1, m.ar_wh, m.ar_bh};
}

static uint16_t prec_flags(pw_ctx *ctx) {
  return (uint16_t)(ctx->precision << FLAG_PREC_SHIFT);
}

// --------------------------------------------------------------------------
// Symbol decoding of a batch (context model + rANS), shared by decode and
// pw_decode_symbols. Streams are device pointers in ptrs (host array).
// Host half of a batch decode's stream table: the streams' device pointers
// and lengths into the plan's pinned staging, which the device work below
// copies to the device (so that a captured chain reads the current table).
static void fill_stream_table(Plan &pl, const uint8_t *const *ptrs, const size_t *lens) {
  uint64_t *hs = reinterpret_cast<uint64_t *>(pl.h_small.p);
  for (int b = 0; b < pl.B; ++b) { hs[b] = (uint64_t)(uintptr_t)ptrs[b]; hs[pl.B + b] = lens[b]; }
}

// Device work of a batch decode up to the quantised latent (stream table
// filled by fill_stream_table). Every size and flag it uses is fixed by the
// plan (geometry, batch, model, chunk layout), so it can be captured once
// and replayed for other streams of the plan.
static int decode_symbols_dev(pw_ctx *ctx, Model &m, Plan &pl, const StreamHeader &h0) {
  const Geometry &g = pl.g;
  const int B = pl.B, P = B * g.nc;
  cudaStream_t st = ctx->stream;
  // pointer / length tables -> device
  const uint64_t *hs = reinterpret_cast<const uint64_t *>(pl.h_small.p);
  PW_CUDA_TRY(cudaMemcpyAsync(pl.d_ptrs.p, hs, B * 8, cudaMemcpyHostToDevice, st));
  PW_CUDA_TRY(cudaMemcpyAsync(pl.d_lens.p, hs + B, B * 8, cudaMemcpyHostToDevice, st));
  PW_CUDA_TRY(cudaMemsetAsync(ctx->status, 0, 4, st));
  if (tc_precision(ctx->precision)) tc_error_reset(pl.ws, st);
  ParseExpect ex{};
  ex.width = h0.width; ex.height = h0.height; ex.ncomp = g.nc; ex.levels = g.levels;
  ex.bitdepth = g.bitdepth; ex.colour = g.colour; ex.flags = h0.flags; ex.chunk = g.chunk;
  ex.lane_byte = h0.lane_shift;
  ex.hash = m.hash;
  DecChunk *dch = reinterpret_cast<DecChunk *>(pl.d_chunks.p);
  double stream_bytes = 0;
  for (int b = 0; b < B; ++b) stream_bytes += (double)hs[B + b];
  const double total_syms = (double)P * g.plane_elems;
  {
  ProfScope ps(ctx, KC_PARSE, 0.0, (double)B * g.nc * g.chunks.size() * (8 + sizeof(DecChunk)));
  launch_parse_streams(reinterpret_cast<const uint8_t *const *>(pl.d_ptrs.p),
                       reinterpret_cast<const uint64_t *>(pl.d_lens.p), B, ex,
                       reinterpret_cast<const TplDev *>(pl.d_tpl.p), (int)g.chunks.size(), dch,
                       reinterpret_cast<float *>(pl.d_deltas.p), ctx->status, st);
  }
  {
    ProfScope ps(ctx, KC_CDF, 0.0, (double)kNTables * (kNSym + 1) * 2);
    launch_cdf_bank(ctx->bank, ctx->coarse, st);
  }
  bump(ctx, 2);
  for (int sb = 0; sb < g.nsb; ++sb) {
    if (sb == 0 && g.ll_ar) {
      // autoregressive LL: one warp per plane walks the positions in raster
      // order, decoding each symbol from the plane's single-state chunk
      if (g.group_count[0] != 1) { set_last_error("bad LL chunk layout"); return PW_ECORRUPT; }
      ProfScope ps(ctx, KC_RANS_DEC, 0.0, (double)P * g.sh[0] * g.sw[0] * 8.0);
      int s = launch_ll_ar_decode(dch + pl.gbase[0], P, g.sh[0], g.sw[0], m.C, ar_weights(ctx, m),
                                  ctx->bank, pl.ws.Q, ctx->status, st);
      bump(ctx);
      if (s) return s;
      continue;
    }
    if (sb >= 1) {
      int s = run_lstm(ctx, m, g, pl.ws, sb);
      if (s) return s;
    }
    for (int k = 0; k < 4; ++k) {
      int s = run_context_pass(ctx, m, g, pl.ws, sb, k, true);
      if (s) return s;
      const int gi = sb * 4 + k;
      const int cnt = g.group_count[gi];
      if (!cnt) continue;
      const int h = g.sh[sb], w = g.sw[sb];
      const double nsym = (double)P * step_count(h, w, k);
      ProfScope ps(ctx, KC_RANS_DEC, 0.0, nsym * 8.0 + stream_bytes * nsym / total_syms);
      // logistic mixture: the step's own table rows instead of the bank
      launch_rans_decode(dch + pl.gbase[gi], P * cnt, m.mix ? pl.ws.mrows : ctx->bank,
                         ctx->coarse, pl.ws.idx + (int64_t)P * g.ioff[gi], step_count(h, w, k),
                         pl.ws.Q + (int64_t)P * g.soff[sb], (int64_t)h * w, h, w, k,
                         ctx->status, st, m.mix);
      bump(ctx);
    }
  }
  return PW_OK;
}

static int read_header(const uint8_t *bs, size_t n, int on_dev, StreamHeader &h) {
  if (!bs || n < sizeof(StreamHeader)) { set_last_error("stream too short"); return PW_ECORRUPT; }
  if (on_dev) {
    PW_CUDA_TRY(cudaMemcpy(&h, bs, sizeof(h), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(&h, bs, sizeof(h));
  }
  if (std::memcmp(h.magic, "PWBS", 4) != 0 || h.version != 1) { set_last_error("not a PWBS stream"); return PW_ECORRUPT; }
  return PW_OK;
}

// Headers of B device-resident streams: one gather kernel and one copy.
static int read_headers_dev(pw_ctx *ctx, int B, const uint8_t *const *bs, const size_t *n,
                            std::vector<StreamHeader> &hd) {
  PlanCache &pc = *reinterpret_cast<PlanCache *>(ctx->plan_cache);
  const size_t tab = (size_t)B * 16, bytes = tab + (size_t)B * 64;
  int s;
  if ((s = pc.d_hdr.ensure(bytes)) || (s = pc.h_hdr.ensure(bytes))) return s;
  uint64_t *ht = static_cast<uint64_t *>(pc.h_hdr.p);
  for (int b = 0; b < B; ++b) { ht[b] = (uint64_t)(uintptr_t)bs[b]; ht[B + b] = n[b]; }
  uint8_t *dt = static_cast<uint8_t *>(pc.d_hdr.p);
  PW_CUDA_TRY(cudaMemcpyAsync(dt, ht, tab, cudaMemcpyHostToDevice, ctx->stream));
  launch_gather_headers(reinterpret_cast<const uint8_t *const *>(dt),
                        reinterpret_cast<const uint64_t *>(dt + (size_t)B * 8), B, dt + tab,
                        ctx->stream);
  bump(ctx);
  uint8_t *hh = static_cast<uint8_t *>(pc.h_hdr.p) + tab;
  PW_CUDA_TRY(cudaMemcpyAsync(hh, dt + tab, (size_t)B * 64, cudaMemcpyDeviceToHost, ctx->stream));
  PW_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  hd.resize(B);
  for (int b = 0; b < B; ++b) {
    if (!bs[b] || n[b] < sizeof(StreamHeader)) { set_last_error("stream too short"); return PW_ECORRUPT; }
    std::memcpy(&hd[b], hh + (size_t)b * 64, sizeof(StreamHeader));
    if (std::memcmp(hd[b].magic, "PWBS", 4) != 0 || hd[b].version != 1) {
      set_last_error("not a PWBS stream");
      return PW_ECORRUPT;
    }
  }
  return PW_OK;
}

static int check_header_model(pw_ctx *ctx, const Model &m, const StreamHeader &h) {
  if (h.model_hash != m.hash) { set_last_error("stream was made with another model"); return PW_EINVAL; }
  if (h.levels != m.levels || ((h.flags & FLAG_LL_AR) ? 1 : 0) != m.ll_mode) {
    set_last_error("stream levels / LL mode do not match the model"); return PW_EINVAL;
  }
  if (((h.flags & FLAG_MIX) ? true : false) != m.mix) {
    set_last_error("stream and model use different probability models"); return PW_EINVAL;
  }
  if (((h.flags >> FLAG_PREC_SHIFT) & 3) != ctx->precision) {
    set_last_error("stream was encoded with another precision class"); return PW_EINVAL;
  }
  if (h.T != kT || h.log2m != kLogM || h.lanes != kMaxLanes || h.chunk_symbols == 0 ||
      (h.lane_shift != 0 && (h.lane_shift < 5 || h.lane_shift > 7)) ||
      (h.ncomp != 1 && h.ncomp != 3) || h.width == 0 || h.height == 0 || h.bitdepth < 1 ||
      h.bitdepth > 16 || h.colour > 3) {
    set_last_error("unsupported stream parameters"); return PW_EUNSUPPORTED;
  }
  return PW_OK;
}

static int build_geo(const StreamHeader &h, Geometry &g) {
  g.build((int)h.height, (int)h.width, h.ncomp, h.levels, h.colour, h.bitdepth,
          (h.flags & FLAG_LOSSLESS) ? 1 : 0, (h.flags & FLAG_LL_AR) ? 1 : 0,
          (int)h.chunk_symbols, (h.flags & FLAG_BALANCED) ? 1 : 0,
          h.lane_shift ? h.lane_shift : kLaneShift);
  if ((uint64_t)g.chunks.size() * g.nc != h.n_chunks) { set_last_error("chunk count mismatch"); return PW_ECORRUPT; }
  return PW_OK;
}

int stream_geometry(pw_ctx *ctx, const Model &m, const uint8_t *bs, size_t n, Geometry &g) {
  StreamHeader h;
  int s = read_header(bs, n, 0, h);
  if (s || (s = check_header_model(ctx, m, h))) return s;
  return build_geo(h, g);
}

// Stage host streams in device memory; fills ptrs.
// True when host memory at p is page-locked (registered or allocated
// pinned): copies from or to it run asynchronously without staging.
static bool pinned_host(const void *p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

static int stage_streams(pw_ctx *ctx, Plan &pl, int B, const uint8_t *const *bs, const size_t *n,
                         int on_dev, std::vector<const uint8_t *> &ptrs) {
  ptrs.resize(B);
  if (on_dev) {
    for (int b = 0; b < B; ++b) ptrs[b] = bs[b];
    return PW_OK;
  }
  size_t tot = 0;
  std::vector<size_t> off(B);
  for (int b = 0; b < B; ++b) { off[b] = tot; tot += (n[b] + 255) / 256 * 256; }
  int s;
  if ((s = pl.d_stage.ensure(tot))) return s;
  bool pinned = true;
  for (int b = 0; b < B && pinned; ++b) pinned = pinned_host(bs[b]);
  if (pinned) {
    // page-locked streams: copied to the device directly
    for (int b = 0; b < B; ++b)
      PW_CUDA_TRY(cudaMemcpyAsync(static_cast<uint8_t *>(pl.d_stage.p) + off[b], bs[b], n[b],
                                  cudaMemcpyHostToDevice, ctx->stream));
  } else {
    if ((s = pl.h_stage.ensure(tot))) return s;
    uint8_t *hp = static_cast<uint8_t *>(pl.h_stage.p);
    for (int b = 0; b < B; ++b) std::memcpy(hp + off[b], bs[b], n[b]);
    PW_CUDA_TRY(cudaMemcpyAsync(pl.d_stage.p, hp, tot, cudaMemcpyHostToDevice, ctx->stream));
  }
  for (int b = 0; b < B; ++b) ptrs[b] = static_cast<uint8_t *>(pl.d_stage.p) + off[b];
  return PW_OK;
}

// Decode B host streams (same geometry) to component planes; on success
// *planes points into the plan's workspace ([B][nc][Hp][Wp] floats) and *geo
// describes them. The planes stay valid until the next call on this plan.
static int decode_to_planes(pw_ctx *ctx, Model &m, int B, const uint8_t *const *bs,
                            const size_t *n, float **planes, Geometry *geo) {
  StreamHeader h0;
  int s = read_header(bs[0], n[0], 0, h0);
  if (s || (s = check_header_model(ctx, m, h0))) return s;
  Geometry g;
  if ((s = build_geo(h0, g))) return s;
  Plan *pl;
  if ((s = get_plan(ctx, m, g, B, "dec", false, &pl))) return s;
  std::vector<const uint8_t *> ptrs;
  if ((s = stage_streams(ctx, *pl, B, bs, n, 0, ptrs))) return s;
  fill_stream_table(*pl, ptrs.data(), n);
  if ((s = decode_symbols_dev(ctx, m, *pl, h0))) return s;
  const int P = B * g.nc;
  SbTable tb = make_sbtable(g, P);
  launch_dequant_all(pl->ws.Q, pl->ws.Yf, (int64_t)P * g.plane_elems, tb, g.nc,
                     reinterpret_cast<float *>(pl->d_deltas.p), ctx->stream);
  bump(ctx);
  if ((s = lift_inverse_planes(ctx, m, g, pl->ws, pl->ws.planes))) return s;
  if ((s = check_status(ctx, &pl->ws))) return s;
  *planes = pl->ws.planes;
  *geo = g;
  return PW_OK;
}

// Device work of an image decode after the stream table: symbols,
// dequantisation, inverse transform and post-processing (Section 3.1, of
// lossy images, into the dequantised subbands' buffer, which the inverse
// transform has consumed). *recon: the reconstructed planes (plan-owned).
static int decode_chain(pw_ctx *ctx, Model &m, Plan &pl, const StreamHeader &h0,
                        const float **recon) {
  const Geometry &g = pl.g;
  const int P = pl.B * g.nc;
  int s;
  if ((s = decode_symbols_dev(ctx, m, pl, h0))) return s;
  SbTable tb = make_sbtable(g, P);
  {
    ProfScope ps(ctx, KC_QUANT, 0.0, (double)P * g.plane_elems * 8.0);
    launch_dequant_all(pl.ws.Q, pl.ws.Yf, (int64_t)P * g.plane_elems, tb, g.nc,
                       reinterpret_cast<float *>(pl.d_deltas.p), ctx->stream);
  }
  bump(ctx);
  if ((s = lift_inverse_planes(ctx, m, g, pl.ws, pl.ws.planes))) return s;
  *recon = pl.ws.planes;
  if (m.has_post && !g.lossless) {
    if ((s = post_process_planes(ctx, m, g, P, pl.ws.planes, pl.ws.Yf))) return s;
    *recon = pl.ws.Yf;
  }
  return PW_OK;
}

// Capture the plan's decode chain on the context's private stream into a
// CUDA graph. On any failure the plan stays on direct launches.
static void capture_chain(pw_ctx *ctx, Model &m, Plan &pl, const StreamHeader &h0) {
  if (!ctx->cap_stream &&
      cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    pl.graph_bad = true;
    return;
  }
  cudaStream_t user = ctx->stream;
  ctx->stream = ctx->cap_stream;
  const uint64_t l0 = ctx->launches;
  cudaGraph_t graph = nullptr;
  const float *recon = nullptr;
  int s = PW_ECUDA;
  if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
    s = decode_chain(ctx, m, pl, h0, &recon);
    if (cudaStreamEndCapture(ctx->cap_stream, &graph) != cudaSuccess) s = PW_ECUDA;
  }
  ctx->stream = user;
  const uint64_t nl = ctx->launches - l0;
  ctx->launches = l0;
  if (launch_failed()) { launch_failed() = false; s = PW_EUNSUPPORTED; }
  if (s == PW_OK && graph && cudaGraphInstantiate(&pl.gexec, graph, 0) == cudaSuccess) {
    pl.graph_launches = nl;
    pl.graph_recon = recon;
  } else {
    pl.gexec = nullptr;
    pl.graph_bad = true;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
}

// decode_chain, replayed from the plan's graph once a direct run of the plan
// (kernel attributes set, buffers in place) launched no convolution of a
// class still being tuned; direct while the context profiles kernels.
static int run_decode_chain(pw_ctx *ctx, Model &m, Plan &pl, const StreamHeader &h0,
                            const float **recon) {
  const bool eligible = ctx->graphs && !prof_of(ctx).on && !pl.graph_bad && pl.tuned_run;
  if (eligible && !pl.gexec) capture_chain(ctx, m, pl, h0);
  if (eligible && pl.gexec) {
    PW_CUDA_TRY(cudaGraphLaunch(pl.gexec, ctx->stream));
    ctx->launches += pl.graph_launches;
    ctx->graph_replays += 1;
    *recon = pl.graph_recon;
    return PW_OK;
  }
  const uint64_t u0 = tune_untuned_uses();
  const int s = decode_chain(ctx, m, pl, h0, recon);
  pl.tuned_run = s == PW_OK && tune_untuned_uses() == u0;
  return s;
}

// --------------------------------------------------------------------------
// Ragged batches: streams of one class (format, model, precision class)
// whose image sizes differ, decoded together on a canvas of the largest
// padded size. Every convolution, coder pass and lifting step of the chain
// covers all streams in one launch; each plane keeps its own extent
// (Workspace::ext): activations are zeroed outside it before a spatial
// convolution reads them, the coder maps each chunk's symbols to its own
// plane's step positions and the lifting steps take each plane's borders,
// so every image decodes exactly as it does alone.
struct RagTables {
  std::vector<int64_t> gbase, gtot;   // descriptor block and chunk count of each group
};

static int decode_ragged_dev(pw_ctx *ctx, Model &m, Plan &pl, const StreamHeader &h0,
                             const RagTables &rt, const uint32_t *d_wh, const RagTpl *d_tpl,
                             int64_t ntpl, double stream_bytes) {
  const Geometry &g = pl.g;
  const int B = pl.B, P = B * g.nc;
  cudaStream_t st = ctx->stream;
  const uint64_t *hs = reinterpret_cast<const uint64_t *>(pl.h_small.p);
  PW_CUDA_TRY(cudaMemcpyAsync(pl.d_ptrs.p, hs, B * 8, cudaMemcpyHostToDevice, st));
  PW_CUDA_TRY(cudaMemcpyAsync(pl.d_lens.p, hs + B, B * 8, cudaMemcpyHostToDevice, st));
  PW_CUDA_TRY(cudaMemsetAsync(ctx->status, 0, 4, st));
  if (tc_precision(ctx->precision)) tc_error_reset(pl.ws, st);
  // symbols outside every plane's extent stay 0 (the context convolutions'
  // zero padding)
  PW_CUDA_TRY(cudaMemsetAsync(pl.ws.Q, 0, (size_t)P * g.plane_elems * 4, st));
  ParseExpect ex{};
  ex.ncomp = g.nc; ex.levels = g.levels; ex.bitdepth = g.bitdepth; ex.colour = g.colour;
  ex.flags = h0.flags; ex.chunk = g.chunk; ex.lane_byte = h0.lane_shift; ex.hash = m.hash;
  DecChunk *dch = reinterpret_cast<DecChunk *>(pl.d_chunks.p);
  const double total_syms = (double)P * g.plane_elems;
  {
    ProfScope ps(ctx, KC_PARSE, 0.0, (double)ntpl * (8 + sizeof(DecChunk) + sizeof(RagTpl)));
    launch_parse_ragged(reinterpret_cast<const uint8_t *const *>(pl.d_ptrs.p),
                        reinterpret_cast<const uint64_t *>(pl.d_lens.p), d_wh, ex, d_tpl, ntpl,
                        dch, reinterpret_cast<float *>(pl.d_deltas.p), ctx->status, st);
  }
  {
    ProfScope ps(ctx, KC_CDF, 0.0, (double)kNTables * (kNSym + 1) * 2);
    launch_cdf_bank(ctx->bank, ctx->coarse, st);
  }
  bump(ctx, 2);
  for (int sb = 0; sb < g.nsb; ++sb) {
    const int lv = sb_level(g, sb);
    if (sb == 0 && g.ll_ar) {
      if (rt.gtot[0] != P) { set_last_error("bad LL chunk layout"); return PW_ECORRUPT; }
      ProfScope ps(ctx, KC_RANS_DEC, 0.0, (double)P * g.sh[0] * g.sw[0] * 8.0);
      int s = launch_ll_ar_decode(dch + rt.gbase[0], P, g.sh[0], g.sw[0], m.C, ar_weights(ctx, m),
                                  ctx->bank, pl.ws.Q, ctx->status, st, pl.ws.ext, lv);
      bump(ctx);
      if (s) return s;
      continue;
    }
    if (sb >= 1) {
      int s = run_lstm(ctx, m, g, pl.ws, sb);
      if (s) return s;
    }
    for (int k = 0; k < 4; ++k) {
      int s = run_context_pass(ctx, m, g, pl.ws, sb, k, true);
      if (s) return s;
      const int gi = sb * 4 + k;
      if (!rt.gtot[gi]) continue;
      const int h = g.sh[sb], w = g.sw[sb];
      const double nsym = (double)P * step_count(h, w, k);
      ProfScope ps(ctx, KC_RANS_DEC, 0.0, nsym * 8.0 + stream_bytes * nsym / total_syms);
      launch_rans_decode(dch + rt.gbase[gi], (int)rt.gtot[gi], ctx->bank, ctx->coarse,
                         pl.ws.idx + (int64_t)P * g.ioff[gi], step_count(h, w, k),
                         pl.ws.Q + (int64_t)P * g.soff[sb], (int64_t)h * w, h, w, k,
                         ctx->status, st, false, pl.ws.ext, lv);
      bump(ctx);
    }
  }
  return PW_OK;
}

static int decode_ragged(pw_ctx *ctx, Model &m, int B, const uint8_t *const *bs, const size_t *n,
                         const std::vector<StreamHeader> &hd, pw_image *out, int on_dev) {
  const StreamHeader &h0 = hd[0];
  std::vector<Geometry> gs(B);
  int Hc = 0, Wc = 0, s;
  for (int b = 0; b < B; ++b) {
    const StreamHeader &h = hd[b];
    if (h.flags != h0.flags || h.ncomp != h0.ncomp || h.levels != h0.levels ||
        h.bitdepth != h0.bitdepth || h.colour != h0.colour ||
        h.chunk_symbols != h0.chunk_symbols || h.lane_shift != h0.lane_shift) {
      set_last_error("streams of a batch differ in format (only their sizes may differ)");
      return PW_EINVAL;
    }
    if ((s = check_header_model(ctx, m, h)) || (s = build_geo(h, gs[b]))) return s;
    Hc = std::max(Hc, gs[b].Hp);
    Wc = std::max(Wc, gs[b].Wp);
  }
  const Geometry &g0 = gs[0];
  Geometry gc;
  gc.build(Hc, Wc, g0.nc, g0.levels, g0.colour, g0.bitdepth, g0.lossless, g0.ll_ar, g0.chunk,
           g0.balanced, g0.lane_shift);
  const int bps = gc.bitdepth > 8 ? 2 : 1, nc = gc.nc, P = B * nc, NG = gc.nsb * 4;
  for (int b = 0; b < B; ++b)
    if (out[b].width != gs[b].W || out[b].height != gs[b].H || out[b].channels != nc ||
        !out[b].data || (out[b].bitdepth > 8 ? 2 : 1) != bps) {
      set_last_error("output image does not match the stream (size, channels, bit depth)");
      return PW_EINVAL;
    }
  Plan *pl;
  if ((s = get_plan(ctx, m, gc, B, "rag", false, &pl))) return s;
  // descriptor blocks: group gi holds, stream by stream and component by
  // component, every chunk of that group
  RagTables rt;
  rt.gtot.assign(NG, 0);
  rt.gbase.assign(NG, 0);
  for (int b = 0; b < B; ++b)
    for (int gi = 0; gi < NG; ++gi) rt.gtot[gi] += (int64_t)nc * gs[b].group_count[gi];
  int64_t total = 0;
  for (int gi = 0; gi < NG; ++gi) { rt.gbase[gi] = total; total += rt.gtot[gi]; }
  int64_t ntpl = 0;
  for (int b = 0; b < B; ++b) ntpl += (int64_t)nc * gs[b].chunks.size();
  // pinned image of the tables: [wh: 2B u32][ext: P int2][tpl]
  const size_t o_ext = ((size_t)B * 8 + 15) / 16 * 16;
  const size_t o_tpl = (o_ext + (size_t)P * sizeof(int2) + 15) / 16 * 16;
  const size_t nbytes = o_tpl + (size_t)std::max<int64_t>(ntpl, 1) * sizeof(RagTpl);
  if ((s = pl->h_rag.ensure(nbytes)) || (s = pl->d_rag.ensure(nbytes)) ||
      (s = pl->d_chunks.ensure(std::max<int64_t>(total, 1) * sizeof(DecChunk))))
    return s;
  uint8_t *hb = static_cast<uint8_t *>(pl->h_rag.p);
  uint32_t *wh = reinterpret_cast<uint32_t *>(hb);
  int2 *ext = reinterpret_cast<int2 *>(hb + o_ext);
  RagTpl *tpl = reinterpret_cast<RagTpl *>(hb + o_tpl);
  std::vector<int64_t> run(rt.gbase);   // next free descriptor of each group
  int64_t e = 0;
  for (int b = 0; b < B; ++b) {
    const Geometry &g = gs[b];
    wh[2 * b] = (uint32_t)g.W;
    wh[2 * b + 1] = (uint32_t)g.H;
    const int nck = (int)g.chunks.size();
    for (int c = 0; c < nc; ++c) ext[b * nc + c] = make_int2(g.Hp, g.Wp);
    for (int comp = 0; comp < nc; ++comp)
      for (int c = 0; c < nck; ++c) {
        const ChunkTpl &t = g.chunks[c];
        const int gi = t.sb * 4 + (t.step < 0 ? 0 : t.step);
        RagTpl &r = tpl[e++];
        r.out = run[gi] + (int64_t)comp * g.group_count[gi] + (c - g.group_first[gi]);
        r.first = t.first;
        r.count = t.count;
        r.lanes = t.lanes;
        r.comp = (uint16_t)comp;
        r.b = (uint32_t)b;
        r.gc = (uint32_t)(comp * nck + c);
        r.nch = (uint32_t)(nck * nc);
      }
    for (int gi = 0; gi < NG; ++gi) run[gi] += (int64_t)nc * g.group_count[gi];
  }
  cudaStream_t st = ctx->stream;
  PW_CUDA_TRY(cudaMemcpyAsync(pl->d_rag.p, hb, nbytes, cudaMemcpyHostToDevice, st));
  uint8_t *db = static_cast<uint8_t *>(pl->d_rag.p);
  pl->ws.ext = reinterpret_cast<const int2 *>(db + o_ext);
  std::vector<const uint8_t *> ptrs;
  if ((s = stage_streams(ctx, *pl, B, bs, n, on_dev, ptrs))) return s;
  fill_stream_table(*pl, ptrs.data(), n);
  double stream_bytes = 0;
  for (int b = 0; b < B; ++b) stream_bytes += (double)n[b];
  if ((s = decode_ragged_dev(ctx, m, *pl, h0, rt, reinterpret_cast<const uint32_t *>(db),
                             reinterpret_cast<const RagTpl *>(db + o_tpl), ntpl, stream_bytes)))
    return s;
  {
    ProfScope ps(ctx, KC_QUANT, 0.0, (double)P * gc.plane_elems * 8.0);
    launch_dequant_all(pl->ws.Q, pl->ws.Yf, (int64_t)P * gc.plane_elems, make_sbtable(gc, P), nc,
                       reinterpret_cast<float *>(pl->d_deltas.p), st);
  }
  bump(ctx);
  if ((s = lift_inverse_planes(ctx, m, gc, pl->ws, pl->ws.planes))) return s;
  const float *recon = pl->ws.planes;
  if (m.has_post && !gc.lossless) {
    if ((s = post_process_planes(ctx, m, gc, P, pl->ws.planes, pl->ws.Yf, pl->ws.ext))) return s;
    recon = pl->ws.Yf;
  }
  // colour conversion per stream: device outputs directly, host outputs
  // through a packed device image
  std::vector<int64_t> off(B + 1, 0);
  for (int b = 0; b < B; ++b) off[b + 1] = off[b] + (int64_t)gs[b].W * nc * bps * gs[b].H;
  bool any_host = false;
  for (int b = 0; b < B; ++b) any_host = any_host || !out[b].is_device;
  if (any_host && (s = pl->d_out.ensure((size_t)off[B]))) return s;
  const int64_t cplane = (int64_t)gc.Hp * gc.Wp;
  for (int b = 0; b < B; ++b) {
    const Geometry &g = gs[b];
    const int64_t row = (int64_t)g.W * nc * bps;
    const int64_t rs = out[b].is_device ? (out[b].stride_bytes ? out[b].stride_bytes : row) : row;
    void *dst = out[b].is_device ? out[b].data : static_cast<uint8_t *>(pl->d_out.p) + off[b];
    ProfScope ps(ctx, KC_COLOUR, 0.0, (double)nc * g.H * g.W * 4.0 + (double)row * g.H);
    launch_colour_out(recon + (int64_t)b * nc * cplane, 1, nc, gc.Hp, gc.Wp, g.H, g.W, gc.colour,
                      gc.bitdepth, dst, row * g.H, rs, st);
    bump(ctx);
  }
  bool any_staged = false;
  for (int b = 0; b < B; ++b) {
    if (out[b].is_device) continue;
    const int64_t row = (int64_t)gs[b].W * nc * bps;
    const int64_t rs = out[b].stride_bytes ? out[b].stride_bytes : row;
    if (pinned_host(out[b].data)) {
      PW_CUDA_TRY(cudaMemcpy2DAsync(out[b].data, rs, static_cast<uint8_t *>(pl->d_out.p) + off[b],
                                    row, row, gs[b].H, cudaMemcpyDeviceToHost, st));
    } else {
      any_staged = true;
    }
  }
  if (any_staged) {
    if ((s = pl->h_out.ensure((size_t)off[B]))) return s;
    PW_CUDA_TRY(cudaMemcpyAsync(pl->h_out.p, pl->d_out.p, (size_t)off[B], cudaMemcpyDeviceToHost,
                                st));
  }
  if ((s = check_status(ctx, &pl->ws))) return s;
  if (any_staged) {
    const uint8_t *hp = static_cast<const uint8_t *>(pl->h_out.p);
    for (int b = 0; b < B; ++b) {
      if (out[b].is_device || pinned_host(out[b].data)) continue;
      const int64_t row = (int64_t)gs[b].W * nc * bps;
      const int64_t rs = out[b].stride_bytes ? out[b].stride_bytes : row;
      for (int y = 0; y < gs[b].H; ++y)
        std::memcpy((uint8_t *)out[b].data + y * rs, hp + off[b] + y * row, (size_t)row);
    }
  }
  return PW_OK;
}

int decode_batch(pw_ctx *ctx, Model &m, int B, const uint8_t *const *bs, const size_t *n,
                 int on_dev, pw_image *out) {
  if (B < 1 || !bs || !n || !out) { set_last_error("bad arguments"); return PW_EINVAL; }
  StreamHeader h0;
  std::vector<StreamHeader> hd;
  int s;
  if (on_dev && B > 1) {
    // every header of a device batch (one gather and one copy)
    if ((s = read_headers_dev(ctx, B, bs, n, hd))) return s;
    h0 = hd[0];
  } else if ((s = read_header(bs[0], n[0], on_dev, h0))) {
    return s;
  }
  if ((s = check_header_model(ctx, m, h0))) return s;
  if ((int64_t)B * h0.ncomp > kMaxPlanes) {
    set_last_error("too many planes in one batch");
    return PW_EUNSUPPORTED;
  }
  if (B > 1) {
    // streams of different sizes: one ragged batch (the mixture model: one
    // batch per size)
    if (!on_dev) {
      hd.resize(B);
      hd[0] = h0;
      for (int b = 1; b < B; ++b)
        if ((s = read_header(bs[b], n[b], 0, hd[b]))) return s;
    }
    bool ragged = false;
    for (int b = 1; b < B; ++b)
      ragged = ragged || hd[b].width != h0.width || hd[b].height != h0.height;
    if (ragged && !m.mix) return decode_ragged(ctx, m, B, bs, n, hd, out, on_dev);
    if (ragged) {
      std::vector<char> done(B, 0);
      for (int b = 0; b < B; ++b) {
        if (done[b]) continue;
        std::vector<const uint8_t *> sp;
        std::vector<size_t> sn;
        std::vector<pw_image> so;
        for (int c = b; c < B; ++c)
          if (!done[c] && hd[c].width == hd[b].width && hd[c].height == hd[b].height) {
            sp.push_back(bs[c]); sn.push_back(n[c]); so.push_back(out[c]);
            done[c] = 1;
          }
        if ((s = decode_batch(ctx, m, (int)sp.size(), sp.data(), sn.data(), on_dev, so.data())))
          return s;
      }
      return PW_OK;
    }
  }
  Geometry g;
  if ((s = build_geo(h0, g))) return s;
  const int bps = g.bitdepth > 8 ? 2 : 1;
  for (int b = 0; b < B; ++b) {
    if (out[b].width != (int)h0.width || out[b].height != (int)h0.height ||
        out[b].channels != g.nc || !out[b].data || (out[b].bitdepth > 8 ? 2 : 1) != bps) {
      set_last_error("output image does not match the stream (size, channels, bit depth)");
      return PW_EINVAL;
    }
  }
  Plan *pl;
  if ((s = get_plan(ctx, m, g, B, "dec", false, &pl))) return s;
  std::vector<const uint8_t *> ptrs;
  if ((s = stage_streams(ctx, *pl, B, bs, n, on_dev, ptrs))) return s;
  fill_stream_table(*pl, ptrs.data(), n);
  const float *recon = nullptr;
  if ((s = run_decode_chain(ctx, m, *pl, h0, &recon))) return s;
  cudaStream_t st = ctx->stream;
  const int P = B * g.nc;
  // output: direct when the batch is one contiguous packed device buffer
  const int64_t row = (int64_t)g.W * g.nc * bps, img = row * g.H;
  bool direct = true;
  for (int b = 0; b < B; ++b) {
    const int64_t rs = out[b].stride_bytes ? out[b].stride_bytes : row;
    if (!out[b].is_device || rs != row ||
        (uint8_t *)out[b].data != (uint8_t *)out[0].data + b * img)
      direct = false;
  }
  void *dst = out[0].data;
  if (!direct) {
    if ((s = pl->d_out.ensure((size_t)img * B))) return s;
    dst = pl->d_out.p;
  }
  {
    ProfScope ps(ctx, KC_COLOUR, 0.0, (double)P * g.H * g.W * 4.0 + (double)img * B);
    launch_colour_out(recon, B, g.nc, g.Hp, g.Wp, g.H, g.W, g.colour, g.bitdepth, dst,
                      img, row, st);
  }
  bump(ctx);
  // host outputs: page-locked ones are written by the copy engine directly;
  // pageable ones get one copy into pinned staging, then a host memcpy
  // (a DMA to pageable memory would go through the driver's bounce buffer)
  bool any_staged = false;
  if (!direct) {
    for (int b = 0; b < B; ++b) {
      const int64_t rs = out[b].stride_bytes ? out[b].stride_bytes : row;
      if (out[b].is_device) {
        PW_CUDA_TRY(cudaMemcpy2DAsync(out[b].data, rs, (uint8_t *)dst + b * img, row, row, g.H,
                                      cudaMemcpyDeviceToDevice, st));
      } else if (pinned_host(out[b].data)) {
        PW_CUDA_TRY(cudaMemcpy2DAsync(out[b].data, rs, (uint8_t *)dst + b * img, row, row, g.H,
                                      cudaMemcpyDeviceToHost, st));
      } else {
        any_staged = true;
      }
    }
    if (any_staged) {
      if ((s = pl->h_out.ensure((size_t)img * B))) return s;
      PW_CUDA_TRY(cudaMemcpyAsync(pl->h_out.p, dst, (size_t)img * B, cudaMemcpyDeviceToHost, st));
    }
  }
  if ((s = check_status(ctx, &pl->ws))) return s;
  if (!direct && any_staged) {
    const uint8_t *hp = static_cast<const uint8_t *>(pl->h_out.p);
    for (int b = 0; b < B; ++b) {
      if (out[b].is_device || pinned_host(out[b].data)) continue;
      const int64_t rs = out[b].stride_bytes ? out[b].stride_bytes : row;
      if (rs == row) {
        std::memcpy(out[b].data, hp + b * img, (size_t)img);
      } else {
        for (int y = 0; y < g.H; ++y)
          std::memcpy((uint8_t *)out[b].data + y * rs, hp + b * img + y * row, (size_t)row);
      }
    }
  }
  return PW_OK;
}

// --------------------------------------------------------------------------
// Encoding.
static int encode_from_latent(pw_ctx *ctx, Model &m, Plan &pl, int B, float dl, float dh,
                              uint8_t **bs, size_t *n) {
  const Geometry &g = pl.g;
  const int P = B * g.nc;
  cudaStream_t st = ctx->stream;
  Workspace &ws = pl.ws;
  if (tc_precision(ctx->precision)) tc_error_reset(ws, st);
  launch_cdf_bank(ctx->bank, ctx->coarse, st);
  bump(ctx);
  for (int sb = 0; sb < g.nsb; ++sb) {
    int s;
    if (sb == 0 && g.ll_ar) {
      // all LL symbols are known: the AR model runs at every position at once
      if ((s = launch_ll_ar_params(ws.Q, P, g.sh[0], g.sw[0], m.C, ar_weights(ctx, m), ws.idx, nullptr,
                                   nullptr, st)))
        return s;
      bump(ctx);
      continue;
    }
    if (sb >= 1 && (s = run_lstm(ctx, m, g, ws, sb))) return s;
    for (int k = 0; k < 4; ++k)
      if ((s = run_context_pass(ctx, m, g, ws, sb, k, false))) return s;
  }
  // gather values in coding order (same layout as idx): step order, or
  // raster order for the autoregressive LL chunk
  int32_t *vals = reinterpret_cast<int32_t *>(ws.T0);
  for (int sb = 0; sb < g.nsb; ++sb)
    for (int k = 0; k < 4; ++k) {
      const bool ar = sb == 0 && g.ll_ar;
      if (ar && k > 0) continue;
      const int64_t nk = ar ? (int64_t)g.sh[0] * g.sw[0] : step_count(g.sh[sb], g.sw[sb], k);
      if (!nk) continue;
      launch_gather_step(ws.Q + (int64_t)P * g.soff[sb], P, g.sh[sb], g.sw[sb], ar ? -1 : k,
                         vals + (int64_t)P * g.ioff[sb * 4 + k], nk, st);
      bump(ctx);
    }
  // chunk list in stream order per image
  const int nck = (int)g.chunks.size();
  const int nall = B * g.nc * nck;
  std::vector<EncChunk> ec(nall);
  for (int b = 0; b < B; ++b)
    for (int c = 0; c < g.nc; ++c)
      for (int j = 0; j < nck; ++j) {
        const ChunkTpl &t = g.chunks[j];
        const int p = b * g.nc + c;
        const int gi = t.sb * 4 + (t.step < 0 ? 0 : t.step);
        const int64_t nk = t.step < 0 ? (int64_t)g.sh[t.sb] * g.sw[t.sb]
                                      : step_count(g.sh[t.sb], g.sw[t.sb], t.step);
        EncChunk &e = ec[(b * g.nc + c) * nck + j];
        e.sym_base = (uint64_t)((int64_t)P * g.ioff[gi] + (int64_t)p * nk + t.first);
        e.count = t.count;
        e.lanes = t.lanes;
        e.scratch_end = 0;
      }
  int s;
  if ((s = pl.d_enc.ensure(std::max(nall, 1) * sizeof(EncChunk))) ||
      (s = pl.d_ops.ensure(std::max(nall, 1) * 4)) ||
      (s = pl.d_nwords.ensure(std::max(nall, 1) * 4)) ||
      (s = pl.d_states.ensure(std::max(nall, 1) * 32 * 4)) ||
      (s = pl.d_outoff.ensure(std::max(nall, 1) * 8)))
    return s;
  EncChunk *d_ec = reinterpret_cast<EncChunk *>(pl.d_enc.p);
  PW_CUDA_TRY(cudaMemcpyAsync(d_ec, ec.data(), nall * sizeof(EncChunk), cudaMemcpyHostToDevice, st));
  PW_CUDA_TRY(cudaMemsetAsync(ctx->status, 0, 4, st));
  launch_rans_count_ops(d_ec, nall, ws.idx, vals, reinterpret_cast<uint32_t *>(pl.d_ops.p), st,
                        m.mix);
  bump(ctx);
  std::vector<uint32_t> ops(nall);
  PW_CUDA_TRY(cudaMemcpyAsync(ops.data(), pl.d_ops.p, nall * 4, cudaMemcpyDeviceToHost, st));
  PW_CUDA_TRY(cudaStreamSynchronize(st));
  uint64_t tot = 0;
  for (int i = 0; i < nall; ++i) { tot += ops[i]; ec[i].scratch_end = tot; }
  if ((s = pl.d_scratch.ensure(std::max<uint64_t>(tot, 1) * 2))) return s;
  PW_CUDA_TRY(cudaMemcpyAsync(d_ec, ec.data(), nall * sizeof(EncChunk), cudaMemcpyHostToDevice, st));
  launch_rans_encode(d_ec, nall, ctx->bank, ws.idx, vals,
                     reinterpret_cast<uint16_t *>(pl.d_scratch.p),
                     reinterpret_cast<uint32_t *>(pl.d_states.p),
                     reinterpret_cast<uint32_t *>(pl.d_nwords.p), ctx->status, st,
                     m.mix ? ws.mcf : nullptr);
  bump(ctx);
  std::vector<uint32_t> nw(nall);
  PW_CUDA_TRY(cudaMemcpyAsync(nw.data(), pl.d_nwords.p, nall * 4, cudaMemcpyDeviceToHost, st));
  if ((s = check_status(ctx, &ws))) return s;
  // payload layout: per image, chunks in stream order
  std::vector<uint64_t> outoff(nall);
  std::vector<uint64_t> img_start(B + 1);
  uint64_t pos = 0;
  for (int b = 0; b < B; ++b) {
    img_start[b] = pos;
    for (int i = 0; i < g.nc * nck; ++i) {
      const int ci = b * g.nc * nck + i;
      outoff[ci] = pos;
      pos += 4ull * ec[ci].lanes + 2ull * nw[ci];
    }
  }
  img_start[B] = pos;
  if ((s = pl.d_payload.ensure(std::max<uint64_t>(pos, 1)))) return s;
  PW_CUDA_TRY(cudaMemcpyAsync(pl.d_outoff.p, outoff.data(), nall * 8, cudaMemcpyHostToDevice, st));
  launch_rans_pack(d_ec, nall, reinterpret_cast<uint16_t *>(pl.d_scratch.p),
                   reinterpret_cast<uint32_t *>(pl.d_states.p),
                   reinterpret_cast<uint32_t *>(pl.d_nwords.p),
                   reinterpret_cast<uint64_t *>(pl.d_outoff.p),
                   reinterpret_cast<uint8_t *>(pl.d_payload.p), st);
  bump(ctx);
  std::vector<uint8_t> payload(pos);
  PW_CUDA_TRY(cudaMemcpyAsync(payload.data(), pl.d_payload.p, pos, cudaMemcpyDeviceToHost, st));
  if ((s = check_status(ctx))) return s;
  const int nch = g.nc * nck;
  for (int b = 0; b < B; ++b) {
    StreamHeader h{};
    std::memcpy(h.magic, "PWBS", 4);
    h.version = 1;
    h.flags = (uint16_t)((g.lossless ? FLAG_LOSSLESS : 0) | (g.ll_ar ? FLAG_LL_AR : 0) |
                         (g.balanced ? FLAG_BALANCED : 0) | (m.mix ? FLAG_MIX : 0) |
                         prec_flags(ctx));
    h.width = g.W; h.height = g.H; h.ncomp = (uint8_t)g.nc; h.levels = (uint8_t)g.levels;
    h.bitdepth = (uint8_t)g.bitdepth; h.colour = (uint8_t)g.colour;
    h.delta_l = dl; h.delta_h = dh; h.T = kT; h.log2m = kLogM; h.lanes = kMaxLanes;
    h.chunk_symbols = g.chunk; h.n_chunks = nch; h.model_hash = m.hash;
    h.lane_shift = (uint8_t)(g.lane_shift == kLaneShift ? 0 : g.lane_shift);
    const uint64_t pb = img_start[b + 1] - img_start[b];
    h.payload_bytes = (uint32_t)pb;
    const size_t total = 64 + 4 * (size_t)(nch + 1) + pb;
    uint8_t *o = static_cast<uint8_t *>(std::malloc(total));
    if (!o) { set_last_error("host allocation failed"); return PW_ENOMEM; }
    std::memcpy(o, &h, 64);
    uint32_t *offs = reinterpret_cast<uint32_t *>(o + 64);
    for (int i = 0; i < nch; ++i)
      offs[i] = (uint32_t)(outoff[b * nch + i] - img_start[b]);
    offs[nch] = (uint32_t)pb;
    std::memcpy(o + 64 + 4 * (nch + 1), payload.data() + img_start[b], pb);
    bs[b] = o;
    n[b] = total;
  }
  return PW_OK;
}

// Encode B x nc device planes ([B][nc][Hp][Wp], colour code 3 = raw
// planes) with model m.
static int encode_planes_dev(pw_ctx *ctx, Model &m, int B, int nc, int H, int W,
                             const float *planes, const pw_codec_opts *o, uint8_t **bs,
                             size_t *n) {
  const int lossless = o && o->lossless ? 1 : 0;
  if (!lossless && !(o && o->q > 0.f)) { set_last_error("quantiser step must be > 0"); return PW_EINVAL; }
  const int chunk = (o && o->chunk_symbols > 0) ? o->chunk_symbols : 16384;
  Geometry g;
  g.build(H, W, nc, m.levels, 3, 8, lossless, m.ll_mode, chunk, 1, ctx->lane_shift);
  Plan *pl;
  int s;
  if ((s = get_plan(ctx, m, g, B, "enc", false, &pl))) return s;
  const int P = B * nc;
  PW_CUDA_TRY(cudaMemcpyAsync(pl->ws.planes, planes, (size_t)P * g.Hp * g.Wp * 4,
                              cudaMemcpyDeviceToDevice, ctx->stream));
  if ((s = lift_forward_planes(ctx, m, g, pl->ws, pl->ws.planes))) return s;
  const float d = lossless ? 1.f : 1.f / o->q;
  SbTable tb = make_sbtable(g, P);
  launch_quant_all(pl->ws.Yf, pl->ws.Q, (int64_t)P * g.plane_elems, tb, d, d, ctx->stream);
  bump(ctx);
  return encode_from_latent(ctx, m, *pl, B, d, d, bs, n);
}

static int image_geo(pw_ctx *ctx, const Model &m, const pw_image &im, const pw_codec_opts *o,
                     Geometry &g) {
  if (im.width < 1 || im.height < 1 || (im.channels != 1 && im.channels != 3) || !im.data ||
      im.bitdepth < 1 || im.bitdepth > 16) {
    set_last_error("bad input image"); return PW_EINVAL;
  }
  const int lossless = o && o->lossless ? 1 : 0;
  const int colour = im.channels == 1 ? 0 : (lossless ? 2 : 1);
  const int chunk = (o && o->chunk_symbols > 0) ? o->chunk_symbols : 16384;
  g.build(im.height, im.width, im.channels, m.levels, colour, im.bitdepth, lossless, m.ll_mode,
          chunk, 1, ctx->lane_shift);
  return PW_OK;
}

static int encode_batch(pw_ctx *ctx, Model &m, int B, const pw_image *in,
                        const pw_codec_opts *o, uint8_t **bs, size_t *n) {
  if (B < 1 || !in || !bs || !n) { set_last_error("bad arguments"); return PW_EINVAL; }
  Geometry g;
  int s = image_geo(ctx, m, in[0], o, g);
  if (s) return s;
  for (int b = 1; b < B; ++b)
    if (in[b].width != in[0].width || in[b].height != in[0].height ||
        in[b].channels != in[0].channels || in[b].bitdepth != in[0].bitdepth) {
      set_last_error("batch images differ in size or format"); return PW_EINVAL;
    }
  if (!g.lossless && !(o && o->q > 0.f)) { set_last_error("quantiser step must be > 0"); return PW_EINVAL; }
  if ((int64_t)B * g.nc > kMaxPlanes) { set_last_error("too many planes in one batch"); return PW_EUNSUPPORTED; }
  Plan *pl;
  if ((s = get_plan(ctx, m, g, B, "enc", false, &pl))) return s;
  const int bps = g.bitdepth > 8 ? 2 : 1;
  const int64_t row = (int64_t)g.W * g.nc * bps, img = row * g.H;
  if ((s = pl->d_img.ensure((size_t)img * B))) return s;
  cudaStream_t st = ctx->stream;
  for (int b = 0; b < B; ++b) {
    const int64_t rs = in[b].stride_bytes ? in[b].stride_bytes : row;
    PW_CUDA_TRY(cudaMemcpy2DAsync((uint8_t *)pl->d_img.p + b * img, row, in[b].data, rs, row,
                                  g.H, in[b].is_device ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice,
                                  st));
  }
  const int P = B * g.nc;
  launch_colour_in(pl->d_img.p, img, row, B, g.nc, g.H, g.W, g.Hp, g.Wp, g.lossless,
                   g.bitdepth, pl->ws.planes, st);
  bump(ctx);
  if ((s = lift_forward_planes(ctx, m, g, pl->ws, pl->ws.planes))) return s;
  const float d = g.lossless ? 1.f : 1.f / o->q;
  SbTable tb = make_sbtable(g, P);
  launch_quant_all(pl->ws.Yf, pl->ws.Q, (int64_t)P * g.plane_elems, tb, d, d, st);
  bump(ctx);
  return encode_from_latent(ctx, m, *pl, B, d, d, bs, n);
}

}  // namespace pw

using namespace pw;

// ===========================================================================
// C ABI
extern "C" {

const char *pw_strerror(int status) {
  switch (status) {
    case PW_OK: return "ok";
    case PW_EINVAL: return g_last_error.empty() ? "invalid argument" : g_last_error.c_str();
    case PW_ENOMEM: return "out of memory";
    case PW_ECORRUPT: return "corrupt bitstream";
    case PW_EUNSUPPORTED: return g_last_error.empty() ? "unsupported" : g_last_error.c_str();
    case PW_ETIMEOUT: return "timeout";
    case PW_EAGAIN: return "try again";
    case PW_ECUDA: return g_last_error.empty() ? "CUDA error" : g_last_error.c_str();
    default: return "unknown error";
  }
}

const char *pw_last_error(void) { return g_last_error.c_str(); }

void pw_free(void *p) { std::free(p); }

int pw_ctx_create(int device, void *stream, int precision, pw_ctx **out) {
  if (!out || (precision != PW_PREC_FP32 && precision != PW_PREC_BF16 &&
               precision != PW_PREC_FP8 && precision != PW_PREC_INT8)) {
    set_last_error("bad precision"); return PW_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    set_last_error("no such CUDA device"); return PW_EINVAL;
  }
  PW_CUDA_TRY(cudaSetDevice(device));
  pw_ctx *c = new pw_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  c->precision = precision;
  c->plan_cache = new PlanCache();
  c->prof = new Prof();
  if (cudaMalloc(&c->bank, kNTables * (kNSym + 1 + kCoarse) * 2) != cudaSuccess ||
      cudaMalloc(&c->status, 256) != cudaSuccess) {
    delete reinterpret_cast<PlanCache *>(c->plan_cache);
    delete reinterpret_cast<Prof *>(c->prof);
    delete c;
    set_last_error("device allocation failed");
    return PW_ENOMEM;
  }
  c->coarse = c->bank + (size_t)kNTables * (kNSym + 1);
  *out = c;
  return PW_OK;
}

void pw_ctx_destroy(pw_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->aux) {
    pw_ctx_destroy(c->aux);
    cudaStreamDestroy(c->aux_stream);
  }
  delete reinterpret_cast<PlanCache *>(c->plan_cache);
  delete reinterpret_cast<Prof *>(c->prof);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  cudaFree(c->bank);
  cudaFree(c->status);
  delete c;
}

int pw_ctx_precision(const pw_ctx *c) { return c ? c->precision : -1; }

int pw_ctx_set_lane_rule(pw_ctx *c, int log2_symbols_per_state) {
  if (!c || log2_symbols_per_state < 5 || log2_symbols_per_state > 7) {
    set_last_error("lane rule: 2^5 .. 2^7 symbols per state");
    return PW_EINVAL;
  }
  c->lane_shift = log2_symbols_per_state;
  return PW_OK;
}

int pw_ctx_profile(pw_ctx *c, int enable) {
  if (!c) return PW_EINVAL;
  Prof &p = prof_of(c);
  cudaStreamSynchronize(c->stream);
  p.reset();
  p.on = enable != 0;
  p.mask = ~0u;
  return PW_OK;
}

int pw_ctx_profile_classes(pw_ctx *c, uint32_t class_mask) {
  if (!c) return PW_EINVAL;
  Prof &p = prof_of(c);
  cudaStreamSynchronize(c->stream);
  p.reset();
  p.on = class_mask != 0;
  p.mask = class_mask;
  return PW_OK;
}

int pw_kernel_class(const char *name) {
  if (!name) return -1;
  for (int k = 0; k < KC_COUNT; ++k)
    if (std::strcmp(name, kclass_name(k)) == 0) return k;
  return -1;
}

int pw_ctx_kernel_stats(pw_ctx *c, pw_kernel_stat *out, int max) {
  if (!c || (max > 0 && !out)) return -PW_EINVAL;
  Prof &p = prof_of(c);
  p.resolve();
  int n = 0;
  for (int k = 0; k < KC_COUNT; ++k) {
    if (!p.launches[k]) continue;
    if (n < max) {
      std::memset(out[n].name, 0, sizeof(out[n].name));
      std::strncpy(out[n].name, kclass_name(k), sizeof(out[n].name) - 1);
      out[n].launches = p.launches[k];
      out[n].ms = p.ms[k];
      out[n].flops = p.flops[k];
      out[n].bytes = p.bytes[k];
    }
    ++n;
  }
  return n;
}
uint64_t pw_ctx_launch_count(const pw_ctx *c) { return c ? c->launches : 0; }

int pw_autotune(int enable) { return tune_set_enabled(enable); }

int pw_autotune_settled(void) {
  static std::atomic<uint64_t> last{~0ull};
  const uint64_t now = tune_untuned_uses();
  return last.exchange(now) == now ? 1 : 0;
}

int pw_autotune_report(char *buf, size_t n) {
  const std::string r = tune_report();
  if (buf && n) {
    const size_t k = r.size() < n - 1 ? r.size() : n - 1;
    std::memcpy(buf, r.data(), k);
    buf[k] = 0;
  }
  return (int)r.size();
}

int pw_model_load(pw_ctx *c, const void *blob, size_t n, pw_model **out) {
  if (!c || !blob || !out) { set_last_error("bad arguments"); return PW_EINVAL; }
  pw_model *m = new pw_model();
  int s = m->m.load(c, blob, n);
  if (s == PW_OK) s = m->m.prepare(c->precision);
  if (s != PW_OK) { delete m; return s; }
  *out = m;
  return PW_OK;
}

void pw_model_free(pw_model *m) { delete m; }
uint64_t pw_model_hash(const pw_model *m) { return m ? m->m.hash : 0; }

int pw_encode_batch(pw_ctx *c, const pw_model *m, int count, const pw_image *in,
                    const pw_codec_opts *o, uint8_t **bs, size_t *n) {
  if (!c || !m) return PW_EINVAL;
  return encode_batch(c, const_cast<pw_model *>(m)->m, count, in, o, bs, n);
}

int pw_encode_image(pw_ctx *c, const pw_model *m, const pw_image *in, const pw_codec_opts *o,
                    uint8_t **bs, size_t *n) {
  return pw_encode_batch(c, m, 1, in, o, bs, n);
}

int pw_decode_batch(pw_ctx *c, const pw_model *m, int count, const uint8_t *const *bs,
                    const size_t *n, int on_dev, pw_image *out) {
  if (!c || !m) return PW_EINVAL;
  return decode_batch(c, const_cast<pw_model *>(m)->m, count, bs, n, on_dev, out);
}

int pw_decode_image(pw_ctx *c, const pw_model *m, const uint8_t *bs, size_t n, pw_image *out) {
  if (!c || !m || !out) return PW_EINVAL;
  if (out->data) return pw_decode_batch(c, m, 1, &bs, &n, 0, out);
  // no buffer given: a host image of the stream's size, owned by the caller
  StreamHeader h;
  int s = read_header(bs, n, 0, h);
  if (s) return s;
  const int bps = h.bitdepth > 8 ? 2 : 1;
  const size_t bytes = (size_t)h.width * h.height * h.ncomp * bps;
  void *buf = std::malloc(bytes ? bytes : 1);
  if (!buf) { set_last_error("host allocation failed"); return PW_ENOMEM; }
  pw_image im{(int)h.width, (int)h.height, (int)h.ncomp, (int)h.bitdepth, 0, 0, buf, 0};
  s = pw_decode_batch(c, m, 1, &bs, &n, 0, &im);
  if (s != PW_OK) { std::free(buf); return s; }
  *out = im;
  return PW_OK;
}

// ---- video GOPs (Section 3.3) ----------------------------------------------
#pragma pack(push, 1)
struct GopHeader {
  char magic[4];
  uint16_t version, nframes;
  uint32_t width, height;
  uint8_t tlevels, ncomp;
  uint16_t zero;
  uint64_t hash_low, hash_high;
};
#pragma pack(pop)
static_assert(sizeof(GopHeader) == 36, "GOP header is 36 bytes");

// Bytes of the block motion vectors of a GOP (version 2): nframes - 1
// fields of ceil(Hp / 16) x ceil(Wp / 16) (dy, dx) int8 pairs.
static size_t gop_mv_bytes(int nframes, int Hp, int Wp) {
  const size_t nby = (Hp + kMcBlock - 1) / kMcBlock, nbx = (Wp + kMcBlock - 1) / kMcBlock;
  return (size_t)(nframes - 1) * nby * nbx * 2;
}

int pw_encode_gop(pw_ctx *c, const pw_model *ml, const pw_model *mh, int nframes,
                  const pw_image *frames, const pw_codec_opts *o, uint8_t **bs, size_t *n) {
  if (!c || !ml || !mh || !frames || !bs || !n || nframes < 2 || (nframes & (nframes - 1))) {
    set_last_error("GOP: need 2^k frames, models and outputs"); return PW_EINVAL;
  }
  Model &L = const_cast<pw_model *>(ml)->m, &Hm = const_cast<pw_model *>(mh)->m;
  if (L.levels != Hm.levels) { set_last_error("GOP models differ in levels"); return PW_EINVAL; }
  if (o && o->lossless) { set_last_error("lossless GOPs are not supported"); return PW_EUNSUPPORTED; }
  const pw_image &f0 = frames[0];
  for (int f = 0; f < nframes; ++f)
    if (frames[f].width != f0.width || frames[f].height != f0.height ||
        frames[f].channels != f0.channels || frames[f].bitdepth != 8 || !frames[f].data) {
      set_last_error("GOP frames must be 8-bit images of one size"); return PW_EINVAL;
    }
  const int nc = f0.channels, H = f0.height, W = f0.width;
  const int mult = 1 << L.levels;
  const int Hp = (H + mult - 1) / mult * mult, Wp = (W + mult - 1) / mult * mult;
  const int64_t F = (int64_t)nc * Hp * Wp;
  const int64_t row = (int64_t)W * nc, img = row * H;
  const size_t mv_bytes = gop_mv_bytes(nframes, Hp, Wp);
  GopBufs &gb = cache_of(c).gop;
  DevBuf &dimg = gb.img, &dframes = gb.frames, &dbands = gb.bands, &dt0 = gb.t0, &dt1 = gb.t1,
         &dluma = gb.luma, &dmv = gb.mv, &dwarp = gb.warp;
  int s;
  if ((s = dimg.ensure((size_t)img * nframes)) || (s = dframes.ensure((size_t)F * nframes * 4)) ||
      (s = dbands.ensure((size_t)F * nframes * 4)) || (s = dt0.ensure((size_t)F * nframes * 2)) ||
      (s = dt1.ensure((size_t)F * nframes * 2)) ||
      (s = dluma.ensure((size_t)nframes * Hp * Wp * 4)) || (s = dmv.ensure(mv_bytes)) ||
      (s = dwarp.ensure((size_t)F * (nframes / 2) * 4)))
    return s;
  cudaStream_t st = c->stream;
  // host frames go through pinned staging (one copy to the device)
  bool any_host = false;
  for (int f = 0; f < nframes; ++f) any_host = any_host || !frames[f].is_device;
  if (any_host && (s = gb.h_img.ensure((size_t)img * nframes))) return s;
  for (int f = 0; f < nframes; ++f) {
    const int64_t rs = frames[f].stride_bytes ? frames[f].stride_bytes : row;
    if (frames[f].is_device) {
      PW_CUDA_TRY(cudaMemcpy2DAsync((uint8_t *)dimg.p + f * img, row, frames[f].data, rs, row, H,
                                    cudaMemcpyDeviceToDevice, st));
    } else {
      uint8_t *hp = static_cast<uint8_t *>(gb.h_img.p) + f * img;
      for (int y = 0; y < H; ++y)
        std::memcpy(hp + y * row, static_cast<const uint8_t *>(frames[f].data) + y * rs,
                    (size_t)row);
    }
  }
  if (any_host) {
    for (int f = 0; f < nframes; ++f)
      if (!frames[f].is_device)
        PW_CUDA_TRY(cudaMemcpyAsync((uint8_t *)dimg.p + f * img,
                                    static_cast<uint8_t *>(gb.h_img.p) + f * img, (size_t)img,
                                    cudaMemcpyHostToDevice, st));
  }
  launch_colour_in(dimg.p, img, row, nframes, nc, H, W, Hp, Wp, 0, 8, (float *)dframes.p, st);
  // motion of every temporal level and pair on the frames' integer luma
  launch_gop_luma((const uint8_t *)dimg.p, img, row, nframes, nc, H, W, Hp, Wp,
                  (int32_t *)dluma.p, st);
  launch_motion_search((const int32_t *)dluma.p, nframes, Hp, Wp, (int8_t *)dmv.p, st);
  bump(c, 3);
  std::vector<int8_t> hmv(mv_bytes);
  PW_CUDA_TRY(cudaMemcpyAsync(hmv.data(), dmv.p, mv_bytes, cudaMemcpyDeviceToHost, st));
  if ((s = temporal_planes(c, L, nframes, nc, Hp, Wp, (float *)dframes.p, (float *)dbands.p,
                           (float *)dt0.p, (float *)dt1.p, true, (const int8_t *)dmv.p,
                           (float *)dwarp.p)))
    return s;
  std::vector<uint8_t *> sb(nframes, nullptr);
  std::vector<size_t> sn(nframes, 0);
  if ((s = encode_planes_dev(c, L, 1, nc, H, W, (float *)dbands.p, o, sb.data(), sn.data())))
    return s;
  if ((s = encode_planes_dev(c, Hm, nframes - 1, nc, H, W, (float *)dbands.p + F, o, sb.data() + 1,
                             sn.data() + 1))) {
    std::free(sb[0]);
    return s;
  }
  GopHeader gh{};
  std::memcpy(gh.magic, "PWGP", 4);
  gh.version = 2; gh.nframes = (uint16_t)nframes; gh.width = W; gh.height = H;
  int T = 0;
  while ((1 << T) < nframes) ++T;
  gh.tlevels = (uint8_t)T; gh.ncomp = (uint8_t)nc; gh.hash_low = L.hash; gh.hash_high = Hm.hash;
  size_t total = sizeof(gh) + mv_bytes;
  for (int f = 0; f < nframes; ++f) total += 4 + sn[f];
  uint8_t *out = static_cast<uint8_t *>(std::malloc(total));
  if (!out) { for (auto q : sb) std::free(q); return PW_ENOMEM; }
  size_t pos = 0;
  std::memcpy(out, &gh, sizeof(gh));
  pos += sizeof(gh);
  std::memcpy(out + pos, hmv.data(), mv_bytes);   // synchronised by the encodes above
  pos += mv_bytes;
  for (int f = 0; f < nframes; ++f) {
    const uint32_t len = (uint32_t)sn[f];
    std::memcpy(out + pos, &len, 4);
    std::memcpy(out + pos + 4, sb[f], sn[f]);
    pos += 4 + sn[f];
    std::free(sb[f]);
  }
  *bs = out;
  *n = total;
  return PW_OK;
}

// The auxiliary context of GOP decodes (same device and precision class,
// own non-blocking stream), or null when it cannot be made (the decode then
// runs both band sets on the caller's context, one after the other).
static pw_ctx *gop_aux(pw_ctx *c) {
  if (c->aux) return c->aux;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  pw_ctx *a = nullptr;
  if (pw_ctx_create(c->device, s, c->precision, &a) != PW_OK) {
    cudaStreamDestroy(s);
    return nullptr;
  }
  a->lane_shift = c->lane_shift;
  a->graphs = c->graphs;
  c->aux = a;
  c->aux_stream = s;
  return a;
}

int pw_decode_gop(pw_ctx *c, const pw_model *ml, const pw_model *mh, const uint8_t *bs, size_t n,
                  int nframes, pw_image *frames) {
  if (!c || !ml || !mh || !bs || !frames || n < sizeof(GopHeader)) return PW_EINVAL;
  Model &L = const_cast<pw_model *>(ml)->m, &Hm = const_cast<pw_model *>(mh)->m;
  GopHeader gh;
  std::memcpy(&gh, bs, sizeof(gh));
  if (std::memcmp(gh.magic, "PWGP", 4) || (gh.version != 1 && gh.version != 2)) {
    set_last_error("not a PWGP stream"); return PW_ECORRUPT;
  }
  if (gh.hash_low != L.hash || gh.hash_high != Hm.hash) { set_last_error("GOP made with other models"); return PW_EINVAL; }
  if ((int)gh.nframes != nframes || nframes < 2 || (1 << gh.tlevels) != nframes ||
      (gh.ncomp != 1 && gh.ncomp != 3)) {
    set_last_error("GOP frame count mismatch"); return PW_EINVAL;
  }
  const int nc = gh.ncomp, H = gh.height, W = gh.width;
  for (int f = 0; f < nframes; ++f)
    if (frames[f].width != W || frames[f].height != H || frames[f].channels != nc ||
        frames[f].bitdepth != 8 || !frames[f].data) {
      set_last_error("GOP output frames do not match the stream"); return PW_EINVAL;
    }
  std::vector<const uint8_t *> bp(nframes);
  std::vector<size_t> bn(nframes);
  size_t pos = sizeof(gh);
  const int mult0 = 1 << L.levels;
  const size_t mv_bytes = gh.version == 2 ? gop_mv_bytes(nframes, (H + mult0 - 1) / mult0 * mult0,
                                                         (W + mult0 - 1) / mult0 * mult0) : 0;
  const uint8_t *mv_src = bs + pos;
  if (pos + mv_bytes > n) { set_last_error("truncated GOP"); return PW_ECORRUPT; }
  pos += mv_bytes;
  for (int f = 0; f < nframes; ++f) {
    uint32_t len;
    if (pos + 4 > n) { set_last_error("truncated GOP"); return PW_ECORRUPT; }
    std::memcpy(&len, bs + pos, 4);
    pos += 4;
    if (pos + len > n) { set_last_error("truncated GOP"); return PW_ECORRUPT; }
    bp[f] = bs + pos;
    bn[f] = len;
    pos += len;
  }
  const int mult = 1 << L.levels;
  const int Hp = (H + mult - 1) / mult * mult, Wp = (W + mult - 1) / mult * mult;
  const int64_t F = (int64_t)nc * Hp * Wp;
  GopBufs &gb = cache_of(c).gop;
  DevBuf &dbands = gb.bands, &dframes = gb.frames, &dt0 = gb.t0, &dt1 = gb.t1, &dimg = gb.img,
         &dmv = gb.mv, &dwarp = gb.warp;
  const int64_t row = (int64_t)W * nc, img = row * H;
  int s;
  if ((s = dbands.ensure((size_t)F * nframes * 4)) || (s = dframes.ensure((size_t)F * nframes * 4)) ||
      (s = dt0.ensure((size_t)F * nframes * 2)) || (s = dt1.ensure((size_t)F * nframes * 2)) ||
      (s = dimg.ensure((size_t)img * nframes)) ||
      (mv_bytes && ((s = dmv.ensure(mv_bytes)) ||
                    (s = dwarp.ensure((size_t)F * (nframes / 2) * 4)))))
    return s;
  cudaStream_t st = c->stream;
  if (mv_bytes) {
    PW_CUDA_TRY(cudaMemcpyAsync(dmv.p, mv_src, mv_bytes, cudaMemcpyHostToDevice, st));
  }
  // the lowpass band (one image, model L) and the highpass bands (a batch,
  // model H) are independent: the auxiliary context decodes the former on
  // its own stream from a second host thread while this one decodes the
  // latter, so that the single-image decode's latency-bound passes overlap
  // the batch
  pw_ctx *ax = gop_aux(c);
  float *lplanes = nullptr, *planes = nullptr;
  Geometry lg, g;
  int ls = PW_OK;
  std::string lerr;
  if (ax) {
    const uint64_t l0 = ax->launches;
    std::thread th([&] {
      cudaSetDevice(c->device);
      ls = decode_to_planes(ax, L, 1, bp.data(), bn.data(), &lplanes, &lg);
      if (ls) lerr = pw_last_error();
    });
    s = decode_to_planes(c, Hm, nframes - 1, bp.data() + 1, bn.data() + 1, &planes, &g);
    th.join();
    c->launches += ax->launches - l0;
    if (ls) { set_last_error(lerr); return ls; }
  } else {
    if ((s = decode_to_planes(c, L, 1, bp.data(), bn.data(), &lplanes, &lg))) return s;
    PW_CUDA_TRY(cudaMemcpyAsync(dbands.p, lplanes, (size_t)F * 4, cudaMemcpyDeviceToDevice, st));
    lplanes = nullptr;
    s = decode_to_planes(c, Hm, nframes - 1, bp.data() + 1, bn.data() + 1, &planes, &g);
  }
  if (s) return s;
  if (g.H != H || g.W != W || g.nc != nc || g.colour != 3 ||
      (lplanes && (lg.H != H || lg.W != W || lg.nc != nc || lg.colour != 3))) {
    set_last_error("GOP band geometry"); return PW_ECORRUPT;
  }
  if (lplanes)  // the auxiliary decode has completed (it synchronised its stream)
    PW_CUDA_TRY(cudaMemcpyAsync(dbands.p, lplanes, (size_t)F * 4, cudaMemcpyDeviceToDevice, st));
  PW_CUDA_TRY(cudaMemcpyAsync((float *)dbands.p + F, planes, (size_t)F * (nframes - 1) * 4,
                              cudaMemcpyDeviceToDevice, st));
  if ((s = temporal_planes(c, L, nframes, nc, Hp, Wp, (float *)dbands.p, (float *)dframes.p,
                           (float *)dt0.p, (float *)dt1.p, false,
                           mv_bytes ? (const int8_t *)dmv.p : nullptr, (float *)dwarp.p)))
    return s;
  launch_colour_out((float *)dframes.p, nframes, nc, Hp, Wp, H, W, nc == 3 ? 1 : 0, 8, dimg.p, img,
                    row, st);
  bump(c);
  // device and page-locked host frames directly; pageable host frames
  // through one copy into pinned staging
  bool any_host = false;
  std::vector<char> staged(nframes, 0);
  for (int f = 0; f < nframes; ++f) {
    const int64_t rs = frames[f].stride_bytes ? frames[f].stride_bytes : row;
    if (frames[f].is_device || pinned_host(frames[f].data)) {
      PW_CUDA_TRY(cudaMemcpy2DAsync(frames[f].data, rs, (uint8_t *)dimg.p + f * img, row, row, H,
                                    frames[f].is_device ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyDeviceToHost, st));
    } else {
      any_host = true;
      staged[f] = 1;
    }
  }
  if (any_host) {
    if ((s = gb.h_img.ensure((size_t)img * nframes))) return s;
    PW_CUDA_TRY(cudaMemcpyAsync(gb.h_img.p, dimg.p, (size_t)img * nframes, cudaMemcpyDeviceToHost,
                                st));
  }
  if ((s = finish(c))) return s;
  for (int f = 0; f < nframes; ++f) {
    if (!staged[f]) continue;
    const int64_t rs = frames[f].stride_bytes ? frames[f].stride_bytes : row;
    const uint8_t *hp = static_cast<const uint8_t *>(gb.h_img.p) + f * img;
    for (int y = 0; y < H; ++y)
      std::memcpy(static_cast<uint8_t *>(frames[f].data) + y * rs, hp + y * row, (size_t)row);
  }
  return PW_OK;
}

int pw_temporal_lift(pw_ctx *c, const pw_model *mm, int nframes, int H, int W, int forward,
                     const float *in, float *out) {
  if (!c || !mm || !in || !out || H < 1 || W < 1) return PW_EINVAL;
  Model &m = const_cast<pw_model *>(mm)->m;
  const int64_t F = (int64_t)H * W;
  DevBuf din, dout, dt0, dt1;
  int s;
  if ((s = din.ensure((size_t)F * nframes * 4)) || (s = dout.ensure((size_t)F * nframes * 4)) ||
      (s = dt0.ensure((size_t)F * nframes * 2)) || (s = dt1.ensure((size_t)F * nframes * 2)))
    return s;
  PW_CUDA_TRY(cudaMemcpyAsync(din.p, in, (size_t)F * nframes * 4, cudaMemcpyHostToDevice, c->stream));
  if ((s = temporal_planes(c, m, nframes, 1, H, W, (float *)din.p, (float *)dout.p, (float *)dt0.p,
                           (float *)dt1.p, forward != 0)))
    return s;
  PW_CUDA_TRY(cudaMemcpyAsync(out, dout.p, (size_t)F * nframes * 4, cudaMemcpyDeviceToHost, c->stream));
  return finish(c);
}

int pw_temporal_lift_mc(pw_ctx *c, const pw_model *mm, int nframes, int H, int W, int forward,
                        const int8_t *mv, const float *in, float *out) {
  if (!c || !mm || !in || !out || !mv || H < 1 || W < 1 || nframes < 2 ||
      (nframes & (nframes - 1)))
    return PW_EINVAL;
  Model &m = const_cast<pw_model *>(mm)->m;
  const int64_t F = (int64_t)H * W;
  const size_t mv_bytes = gop_mv_bytes(nframes, H, W);
  DevBuf din, dout, dt0, dt1, dmv, dwarp;
  int s;
  if ((s = din.ensure((size_t)F * nframes * 4)) || (s = dout.ensure((size_t)F * nframes * 4)) ||
      (s = dt0.ensure((size_t)F * nframes * 2)) || (s = dt1.ensure((size_t)F * nframes * 2)) ||
      (s = dmv.ensure(mv_bytes)) || (s = dwarp.ensure((size_t)F * (nframes / 2) * 4)))
    return s;
  PW_CUDA_TRY(cudaMemcpyAsync(din.p, in, (size_t)F * nframes * 4, cudaMemcpyHostToDevice, c->stream));
  PW_CUDA_TRY(cudaMemcpyAsync(dmv.p, mv, mv_bytes, cudaMemcpyHostToDevice, c->stream));
  if ((s = temporal_planes(c, m, nframes, 1, H, W, (float *)din.p, (float *)dout.p, (float *)dt0.p,
                           (float *)dt1.p, forward != 0, (const int8_t *)dmv.p, (float *)dwarp.p)))
    return s;
  PW_CUDA_TRY(cudaMemcpyAsync(out, dout.p, (size_t)F * nframes * 4, cudaMemcpyDeviceToHost, c->stream));
  return finish(c);
}

int pw_motion_search(pw_ctx *c, int nframes, int H, int W, const int32_t *luma, int8_t *mv) {
  if (!c || !luma || !mv || H < 1 || W < 1 || nframes < 2 || (nframes & (nframes - 1)))
    return PW_EINVAL;
  const size_t mv_bytes = gop_mv_bytes(nframes, H, W);
  DevBuf dl, dmv;
  int s;
  if ((s = dl.ensure((size_t)nframes * H * W * 4)) || (s = dmv.ensure(mv_bytes))) return s;
  PW_CUDA_TRY(cudaMemcpyAsync(dl.p, luma, (size_t)nframes * H * W * 4, cudaMemcpyHostToDevice,
                              c->stream));
  launch_motion_search((const int32_t *)dl.p, nframes, H, W, (int8_t *)dmv.p, c->stream);
  bump(c);
  PW_CUDA_TRY(cudaMemcpyAsync(mv, dmv.p, mv_bytes, cudaMemcpyDeviceToHost, c->stream));
  return finish(c);
}

// ---- stages ---------------------------------------------------------------
int pw_cdf_bank(pw_ctx *c, uint16_t *dev_bank) {
  if (!c || !dev_bank) return PW_EINVAL;
  launch_cdf_bank(dev_bank, nullptr, c->stream);
  bump(c);
  return finish(c);
}

int pw_entropy_index(pw_ctx *c, const float *mu, const float *sigma, int64_t n, uint32_t *idx) {
  if (!c || n < 0 || (n && (!mu || !sigma || !idx))) return PW_EINVAL;
  if (!n) return PW_OK;
  DevBuf d;
  int s;
  if ((s = d.ensure((size_t)n * 12))) return s;
  float *dm = (float *)d.p, *ds = dm + n;
  uint32_t *di = (uint32_t *)(ds + n);
  PW_CUDA_TRY(cudaMemcpyAsync(dm, mu, n * 4, cudaMemcpyHostToDevice, c->stream));
  PW_CUDA_TRY(cudaMemcpyAsync(ds, sigma, n * 4, cudaMemcpyHostToDevice, c->stream));
  launch_pack_index(dm, ds, n, 1, di, c->stream);
  bump(c);
  PW_CUDA_TRY(cudaMemcpyAsync(idx, di, n * 4, cudaMemcpyDeviceToHost, c->stream));
  PW_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PW_OK;
}

int pw_rans_decode(pw_ctx *c, const uint8_t *payload, size_t payload_bytes, int nchunks,
                   const uint32_t *offset, const uint32_t *nbytes, const uint32_t *count,
                   const uint32_t *lanes, const uint32_t *idx, int32_t *out) {
  if (!c || nchunks < 0) return PW_EINVAL;
  uint64_t nsym = 0;
  for (int i = 0; i < nchunks; ++i) {
    if ((uint64_t)offset[i] + nbytes[i] > payload_bytes || lanes[i] < 1 || lanes[i] > 32) {
      set_last_error("chunk outside payload or bad lane count"); return PW_EINVAL;
    }
    nsym += count[i];
  }
  DevBuf dp, di, dout, dch;
  int s;
  if ((s = dp.ensure(payload_bytes + 16)) || (s = di.ensure(nsym * 4 + 4)) ||
      (s = dout.ensure(nsym * 4 + 4)) || (s = dch.ensure((nchunks + 1) * sizeof(DecChunk))))
    return s;
  std::vector<DecChunk> ch(nchunks);
  uint64_t first = 0;
  for (int i = 0; i < nchunks; ++i) {
    ch[i].data = (const uint8_t *)dp.p + offset[i];
    ch[i].nbytes = nbytes[i];
    ch[i].count = count[i];
    ch[i].first = (uint32_t)first;
    ch[i].lanes = (uint16_t)lanes[i];
    ch[i].plane = 0;
    first += count[i];
  }
  cudaStream_t st = c->stream;
  if (payload_bytes)
    PW_CUDA_TRY(cudaMemcpyAsync(dp.p, payload, payload_bytes, cudaMemcpyHostToDevice, st));
  if (nsym) PW_CUDA_TRY(cudaMemcpyAsync(di.p, idx, nsym * 4, cudaMemcpyHostToDevice, st));
  if (nchunks)
    PW_CUDA_TRY(cudaMemcpyAsync(dch.p, ch.data(), nchunks * sizeof(DecChunk), cudaMemcpyHostToDevice, st));
  PW_CUDA_TRY(cudaMemsetAsync(c->status, 0, 4, st));
  launch_cdf_bank(c->bank, c->coarse, st);
  launch_rans_decode((DecChunk *)dch.p, nchunks, c->bank, c->coarse, (uint32_t *)di.p, 0,
                     (int32_t *)dout.p, 0, 0, 0, -1, c->status, st);
  bump(c, 2);
  if (nsym) PW_CUDA_TRY(cudaMemcpyAsync(out, dout.p, nsym * 4, cudaMemcpyDeviceToHost, st));
  return check_status(c);
}

int pw_rans_encode(pw_ctx *c, int nchunks, const uint32_t *count, const uint32_t *lanes,
                   const uint32_t *idx, const int32_t *values, uint8_t **payload,
                   size_t *payload_bytes, uint32_t *offset, uint32_t *nbytes) {
  if (!c || nchunks < 0 || !payload || !payload_bytes) return PW_EINVAL;
  uint64_t nsym = 0;
  for (int i = 0; i < nchunks; ++i) {
    if (lanes[i] < 1 || lanes[i] > 32) { set_last_error("bad lane count"); return PW_EINVAL; }
    nsym += count[i];
  }
  cudaStream_t st = c->stream;
  DevBuf di, dv, dec, dops, dsc, dstates, dnw, doff, dpay;
  int s;
  if ((s = di.ensure(nsym * 4 + 4)) || (s = dv.ensure(nsym * 4 + 4)) ||
      (s = dec.ensure((nchunks + 1) * sizeof(EncChunk))) || (s = dops.ensure(nchunks * 4 + 4)) ||
      (s = dstates.ensure(nchunks * 128 + 4)) || (s = dnw.ensure(nchunks * 4 + 4)) ||
      (s = doff.ensure(nchunks * 8 + 8)))
    return s;
  std::vector<EncChunk> ec(nchunks);
  uint64_t first = 0;
  for (int i = 0; i < nchunks; ++i) {
    ec[i].sym_base = first; ec[i].count = count[i]; ec[i].lanes = lanes[i]; ec[i].scratch_end = 0;
    first += count[i];
  }
  if (nsym) {
    PW_CUDA_TRY(cudaMemcpyAsync(di.p, idx, nsym * 4, cudaMemcpyHostToDevice, st));
    PW_CUDA_TRY(cudaMemcpyAsync(dv.p, values, nsym * 4, cudaMemcpyHostToDevice, st));
  }
  if (nchunks)
    PW_CUDA_TRY(cudaMemcpyAsync(dec.p, ec.data(), nchunks * sizeof(EncChunk), cudaMemcpyHostToDevice, st));
  launch_cdf_bank(c->bank, c->coarse, st);
  launch_rans_count_ops((EncChunk *)dec.p, nchunks, (uint32_t *)di.p, (int32_t *)dv.p,
                        (uint32_t *)dops.p, st);
  bump(c, 2);
  std::vector<uint32_t> ops(nchunks);
  if (nchunks) PW_CUDA_TRY(cudaMemcpyAsync(ops.data(), dops.p, nchunks * 4, cudaMemcpyDeviceToHost, st));
  PW_CUDA_TRY(cudaStreamSynchronize(st));
  uint64_t tot = 0;
  for (int i = 0; i < nchunks; ++i) { tot += ops[i]; ec[i].scratch_end = tot; }
  if ((s = dsc.ensure(tot * 2 + 2))) return s;
  if (nchunks)
    PW_CUDA_TRY(cudaMemcpyAsync(dec.p, ec.data(), nchunks * sizeof(EncChunk), cudaMemcpyHostToDevice, st));
  PW_CUDA_TRY(cudaMemsetAsync(c->status, 0, 4, st));
  launch_rans_encode((EncChunk *)dec.p, nchunks, c->bank, (uint32_t *)di.p, (int32_t *)dv.p,
                     (uint16_t *)dsc.p, (uint32_t *)dstates.p, (uint32_t *)dnw.p, c->status, st);
  bump(c);
  std::vector<uint32_t> nw(nchunks);
  if (nchunks) PW_CUDA_TRY(cudaMemcpyAsync(nw.data(), dnw.p, nchunks * 4, cudaMemcpyDeviceToHost, st));
  if ((s = check_status(c))) return s;
  std::vector<uint64_t> off(nchunks);
  uint64_t pos = 0;
  for (int i = 0; i < nchunks; ++i) {
    off[i] = pos;
    offset[i] = (uint32_t)pos;
    nbytes[i] = 4 * lanes[i] + 2 * nw[i];
    pos += nbytes[i];
  }
  if ((s = dpay.ensure(pos + 4))) return s;
  if (nchunks) {
    PW_CUDA_TRY(cudaMemcpyAsync(doff.p, off.data(), nchunks * 8, cudaMemcpyHostToDevice, st));
    launch_rans_pack((EncChunk *)dec.p, nchunks, (uint16_t *)dsc.p, (uint32_t *)dstates.p,
                     (uint32_t *)dnw.p, (uint64_t *)doff.p, (uint8_t *)dpay.p, st);
    bump(c);
  }
  uint8_t *o = static_cast<uint8_t *>(std::malloc(pos ? pos : 1));
  if (!o) return PW_ENOMEM;
  if (pos) PW_CUDA_TRY(cudaMemcpyAsync(o, dpay.p, pos, cudaMemcpyDeviceToHost, st));
  PW_CUDA_TRY(cudaStreamSynchronize(st));
  *payload = o;
  *payload_bytes = pos;
  return PW_OK;
}

// The context model over a fully known latent (every step at once); the
// plan's workspace then holds the entropy parameters.
static int context_all(pw_ctx *c, Model &m, int H, int W, const int32_t *q, Plan **plo,
                       Geometry &g) {
  const int mult = 1 << m.levels;
  if (H < mult || W < mult || H % mult || W % mult) {
    set_last_error("H and W must be positive multiples of 2^levels"); return PW_EINVAL;
  }
  g.build(H, W, 1, m.levels, 0, 8, 0, m.ll_mode, 16384);
  Plan *pl;
  int s;
  if ((s = get_plan(c, m, g, 1, "par", true, &pl))) return s;
  *plo = pl;
  cudaStream_t st = c->stream;
  PW_CUDA_TRY(cudaMemcpyAsync(pl->ws.Q, q, g.plane_elems * 4, cudaMemcpyHostToDevice, st));
  if (tc_precision(c->precision)) tc_error_reset(pl->ws, st);
  for (int sb = 0; sb < g.nsb; ++sb) {
    if (sb == 0 && m.ll_mode == 1) {
      if ((s = launch_ll_ar_params(pl->ws.Q, 1, g.sh[0], g.sw[0], m.C, ar_weights(c, m), pl->ws.idx,
                                   pl->ws.mu, pl->ws.sg, st)))
        return s;
      bump(c);
      continue;
    }
    if (sb >= 1 && (s = run_lstm(c, m, g, pl->ws, sb))) return s;
    for (int k = 0; k < 4; ++k)
      if ((s = run_context_pass(c, m, g, pl->ws, sb, k, false))) return s;
  }
  return PW_OK;
}

int pw_context_params(pw_ctx *c, const pw_model *mm, int H, int W, const int32_t *q, float *mu,
                      float *sigma) {
  if (!c || !mm || !q || !mu || !sigma) return PW_EINVAL;
  Model &m = const_cast<pw_model *>(mm)->m;
  if (m.mix) {
    set_last_error("a mixture model's parameters come from pw_context_mixture");
    return PW_EUNSUPPORTED;
  }
  Plan *pl;
  Geometry g;
  int s = context_all(c, m, H, W, q, &pl, g);
  if (s) return s;
  cudaStream_t st = c->stream;
  PW_CUDA_TRY(cudaMemcpyAsync(mu, pl->ws.mu, g.plane_elems * 4, cudaMemcpyDeviceToHost, st));
  PW_CUDA_TRY(cudaMemcpyAsync(sigma, pl->ws.sg, g.plane_elems * 4, cudaMemcpyDeviceToHost, st));
  if ((s = finish(c))) return s;
  if (tc_precision(c->precision) && tc_error(pl->ws)) {
    set_last_error("a tensor-core kernel's bounded wait expired");
    return PW_ETIMEOUT;
  }
  return PW_OK;
}

int pw_context_mixture(pw_ctx *c, const pw_model *mm, int H, int W, const int32_t *q,
                       float *par) {
  if (!c || !mm || !q || !par) return PW_EINVAL;
  Model &m = const_cast<pw_model *>(mm)->m;
  if (!m.mix) {
    set_last_error("not a mixture model (pw_context_params gives its parameters)");
    return PW_EUNSUPPORTED;
  }
  Plan *pl;
  Geometry g;
  int s = context_all(c, m, H, W, q, &pl, g);
  if (s) return s;
  PW_CUDA_TRY(cudaMemcpyAsync(par, pl->ws.mpar, g.plane_elems * 9 * 4, cudaMemcpyDeviceToHost,
                              c->stream));
  return finish(c);
}

int pw_mix_tables(pw_ctx *c, int64_t n, const int32_t *key9, uint16_t *cdf) {
  if (!c || n < 0 || (n && (!key9 || !cdf))) return PW_EINVAL;
  if (!n) return PW_OK;
  DevBuf dk, dr;
  int s;
  if ((s = dk.ensure((size_t)n * 9 * 4)) || (s = dr.ensure((size_t)n * kMixRow * 2))) return s;
  cudaStream_t st = c->stream;
  PW_CUDA_TRY(cudaMemcpyAsync(dk.p, key9, (size_t)n * 9 * 4, cudaMemcpyHostToDevice, st));
  launch_mix_tables((const int32_t *)dk.p, n, (uint16_t *)dr.p, st);
  bump(c);
  PW_CUDA_TRY(cudaMemcpy2DAsync(cdf, (kNSym + 1) * 2, dr.p, kMixRow * 2, (kNSym + 1) * 2,
                                (size_t)n, cudaMemcpyDeviceToHost, st));
  return finish(c);
}

int pw_model_mixture(const pw_model *m) { return m && m->m.mix ? 1 : 0; }

int pw_ctx_set_graphs(pw_ctx *c, int enable) {
  if (!c) return -PW_EINVAL;
  const int old = c->graphs;
  c->graphs = enable ? 1 : 0;
  if (c->aux) c->aux->graphs = c->graphs;
  return old;
}

uint64_t pw_ctx_graph_replays(const pw_ctx *c) { return c ? c->graph_replays : 0; }

static int lift_stage(pw_ctx *c, const pw_model *mm, int H, int W, int lossless, const float *in,
                      float *out, bool fwd) {
  if (!c || !mm || !in || !out) return PW_EINVAL;
  Model &m = const_cast<pw_model *>(mm)->m;
  const int mult = 1 << m.levels;
  if (H < mult || W < mult || H % mult || W % mult) {
    set_last_error("H and W must be positive multiples of 2^levels"); return PW_EINVAL;
  }
  Geometry g;
  g.build(H, W, 1, m.levels, 0, 8, lossless ? 1 : 0, 0, 16384);
  Plan *pl;
  int s;
  if ((s = get_plan(c, m, g, 1, "lift", false, &pl))) return s;
  cudaStream_t st = c->stream;
  const size_t bytes = (size_t)g.plane_elems * 4;
  PW_CUDA_TRY(cudaMemsetAsync(c->status, 0, 4, st));
  if (fwd) {
    PW_CUDA_TRY(cudaMemcpyAsync(pl->ws.planes, in, bytes, cudaMemcpyHostToDevice, st));
    if ((s = lift_forward_planes(c, m, g, pl->ws, pl->ws.planes))) return s;
    PW_CUDA_TRY(cudaMemcpyAsync(out, pl->ws.Yf, bytes, cudaMemcpyDeviceToHost, st));
  } else {
    PW_CUDA_TRY(cudaMemcpyAsync(pl->ws.Yf, in, bytes, cudaMemcpyHostToDevice, st));
    if ((s = lift_inverse_planes(c, m, g, pl->ws, pl->ws.planes))) return s;
    PW_CUDA_TRY(cudaMemcpyAsync(out, pl->ws.planes, bytes, cudaMemcpyDeviceToHost, st));
  }
  return check_status(c);
}

int pw_lift_forward(pw_ctx *c, const pw_model *m, int H, int W, int lossless, const float *x,
                    float *sb) {
  return lift_stage(c, m, H, W, lossless, x, sb, true);
}
int pw_lift_inverse(pw_ctx *c, const pw_model *m, int H, int W, int lossless, const float *sb,
                    float *x) {
  return lift_stage(c, m, H, W, lossless, sb, x, false);
}

int pw_conv_bf16(pw_ctx *c, int P, int H, int W, int cin, int cout, int ks, int act,
                 const float *x, const float *w, const float *b, float *y) {
  if (!c || !x || !w || !b || !y) return PW_EINVAL;
  return tc_conv_host(c, P, H, W, cin, cout, ks, act, x, w, b, y);
}

int pw_decode_symbols(pw_ctx *c, const pw_model *mm, const uint8_t *bs, size_t n, int32_t *q) {
  if (!c || !mm || !bs || !q) return PW_EINVAL;
  Model &m = const_cast<pw_model *>(mm)->m;
  StreamHeader h0;
  int s = read_header(bs, n, 0, h0);
  if (s || (s = check_header_model(c, m, h0))) return s;
  Geometry g;
  if ((s = build_geo(h0, g))) return s;
  Plan *pl;
  if ((s = get_plan(c, m, g, 1, "sym", false, &pl))) return s;
  std::vector<const uint8_t *> ptrs;
  const uint8_t *const bsp[1] = {bs};
  if ((s = stage_streams(c, *pl, 1, bsp, &n, 0, ptrs))) return s;
  fill_stream_table(*pl, ptrs.data(), &n);
  if ((s = decode_symbols_dev(c, m, *pl, h0))) return s;
  PW_CUDA_TRY(cudaMemcpyAsync(q, pl->ws.Q, (size_t)g.nc * g.plane_elems * 4,
                              cudaMemcpyDeviceToHost, c->stream));
  return check_status(c, &pl->ws);
}

int pw_analyse(pw_ctx *c, const pw_model *mm, const pw_image *in, const pw_codec_opts *o,
               int32_t *q) {
  if (!c || !mm || !in || !q) return PW_EINVAL;
  Model &m = const_cast<pw_model *>(mm)->m;
  Geometry g;
  int s = image_geo(c, m, *in, o, g);
  if (s) return s;
  if (!g.lossless && !(o && o->q > 0.f)) { set_last_error("quantiser step must be > 0"); return PW_EINVAL; }
  Plan *pl;
  if ((s = get_plan(c, m, g, 1, "ana", false, &pl))) return s;
  const int bps = g.bitdepth > 8 ? 2 : 1;
  const int64_t row = (int64_t)g.W * g.nc * bps, img = row * g.H;
  if ((s = pl->d_img.ensure((size_t)img))) return s;
  cudaStream_t st = c->stream;
  const int64_t rs = in->stride_bytes ? in->stride_bytes : row;
  PW_CUDA_TRY(cudaMemcpy2DAsync(pl->d_img.p, row, in->data, rs, row, g.H,
                                in->is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  launch_colour_in(pl->d_img.p, img, row, 1, g.nc, g.H, g.W, g.Hp, g.Wp, g.lossless, g.bitdepth,
                   pl->ws.planes, st);
  bump(c);
  if ((s = lift_forward_planes(c, m, g, pl->ws, pl->ws.planes))) return s;
  const float d = g.lossless ? 1.f : 1.f / o->q;
  SbTable tb = make_sbtable(g, g.nc);
  launch_quant_all(pl->ws.Yf, pl->ws.Q, (int64_t)g.nc * g.plane_elems, tb, d, d, st);
  bump(c);
  PW_CUDA_TRY(cudaMemcpyAsync(q, pl->ws.Q, (size_t)g.nc * g.plane_elems * 4,
                              cudaMemcpyDeviceToHost, st));
  return finish(c);
}

int pw_encode_latent(pw_ctx *c, const pw_model *mm, const int32_t *q, int width, int height,
                     int channels, int bitdepth, int colour, const pw_codec_opts *o,
                     uint8_t **bs, size_t *n) {
  if (!c || !mm || !q || !bs || !n || (channels != 1 && channels != 3) || width < 1 ||
      height < 1 || colour < 0 || colour > 3)
    return PW_EINVAL;
  Model &m = const_cast<pw_model *>(mm)->m;
  const int lossless = o && o->lossless ? 1 : 0;
  if (!lossless && !(o && o->q > 0.f)) { set_last_error("quantiser step must be > 0"); return PW_EINVAL; }
  const int chunk = (o && o->chunk_symbols > 0) ? o->chunk_symbols : 16384;
  Geometry g;
  g.build(height, width, channels, m.levels, colour, bitdepth, lossless, m.ll_mode, chunk, 1,
          c->lane_shift);
  Plan *pl;
  int s;
  if ((s = get_plan(c, m, g, 1, "lat", false, &pl))) return s;
  PW_CUDA_TRY(cudaMemcpyAsync(pl->ws.Q, q, (size_t)channels * g.plane_elems * 4,
                              cudaMemcpyHostToDevice, c->stream));
  const float d = lossless ? 1.f : 1.f / o->q;
  return encode_from_latent(c, m, *pl, 1, d, d, bs, n);
}

}  // extern "C"
