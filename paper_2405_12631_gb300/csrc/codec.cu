// Decode / encode drivers of the pWave++ path.
//
// Decode (Sections 3.1, 3.2): parse the streams on the device, build the CDF
// table bank, then for every subband in coding order run the ConvLSTM
// context prediction (subbands 2..13) and the four coding steps (context
// fusion net -> entropy parameters -> table indices -> rANS decoding of the
// step's positions), then dequantise, run the inverse lifting transform
// level by level and convert colour. Encoding runs the same context kernels
// on the fully known latent (each step's net masks the positions of later
// steps, so it sees exactly what the decoder sees) and rANS-encodes.
#include <algorithm>
#include <mutex>
#include <cstring>

#include "codec.h"
#include "ctx_tc.h"
#include "prof.h"

namespace pw {

static inline void bump(pw_ctx *ctx, int n = 1) { ctx->launches += (uint64_t)n; }

// ---------------------------------------------------------------------------
void Geometry::build(int H_, int W_, int nc_, int levels_, int colour_, int bitdepth_,
                     int lossless_, int ll_ar_, int chunk_, int balanced_,
                     int lane_shift_) {
  H = H_; W = W_; nc = nc_; levels = levels_; colour = colour_; bitdepth = bitdepth_;
  lossless = lossless_; ll_ar = ll_ar_; chunk = chunk_; balanced = balanced_;
  lane_shift = lane_shift_;
  const int mult = 1 << levels;
  Hp = (H + mult - 1) / mult * mult;
  Wp = (W + mult - 1) / mult * mult;
  nsb = 3 * levels + 1;
  sh.clear(); sw.clear(); soff.clear();
  sh.push_back(Hp >> levels); sw.push_back(Wp >> levels);
  for (int lv = levels; lv >= 1; --lv)
    for (int o = 0; o < 3; ++o) { sh.push_back(Hp >> lv); sw.push_back(Wp >> lv); }
  int64_t acc = 0;
  for (int i = 0; i < nsb; ++i) { soff.push_back(acc); acc += (int64_t)sh[i] * sw[i]; }
  plane_elems = acc;
  ioff.assign(nsb * 4, 0);
  acc = 0;
  for (int i = 0; i < nsb; ++i)
    for (int k = 0; k < 4; ++k) {
      ioff[i * 4 + k] = acc;
      acc += (i == 0 && ll_ar) ? (k == 0 ? (int64_t)sh[0] * sw[0] : 0)
                               : step_count(sh[i], sw[i], k);
    }
  chunks.clear();
  group_first.assign(nsb * 4, -1);
  group_count.assign(nsb * 4, 0);
  for (int i = 0; i < nsb; ++i) {
    if (i == 0 && ll_ar) {
      const int n = sh[0] * sw[0];
      if (n) {
        group_first[0] = (int)chunks.size();
        group_count[0] = 1;
        chunks.push_back({0, -1, 0u, (uint32_t)n, 1});
      }
      continue;
    }
    for (int k = 0; k < 4; ++k) {
      const int n = step_count(sh[i], sw[i], k);
      group_first[i * 4 + k] = (int)chunks.size();
      if (balanced) {
        // ceil(n / chunk) chunks; the first n % nch get one symbol more
        const int nch = (n + chunk - 1) / chunk;
        for (int j = 0, f = 0; j < nch; ++j) {
          const int cnt = n / nch + (j < n % nch ? 1 : 0);
          chunks.push_back({i, k, (uint32_t)f, (uint32_t)cnt,
                            (uint16_t)chunk_lanes(cnt, lane_shift)});
          f += cnt;
        }
      } else {
        for (int f = 0; f < n; f += chunk) {
          const int cnt = std::min(chunk, n - f);
          chunks.push_back({i, k, (uint32_t)f, (uint32_t)cnt,
                            (uint16_t)chunk_lanes(cnt, lane_shift)});
        }
      }
      group_count[i * 4 + k] = (int)chunks.size() - group_first[i * 4 + k];
    }
  }
}

// ---------------------------------------------------------------------------
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

static cudaMemPool_t device_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;  // keep freed memory in the pool
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

int pool_alloc(void **p, size_t n, cudaStream_t st) {
  *p = nullptr;
  cudaMemPool_t pool = device_pool();
  if (!pool || cudaMallocFromPoolAsync(p, n ? n : 1, pool, st) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_last_error("device allocation failed");
    return PW_ENOMEM;
  }
  return PW_OK;
}

void pool_free(void *p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// Symbols of the largest coding step of one plane.
static int64_t max_step_symbols(const Geometry &g) {
  int64_t m = 0;
  for (int sb = 0; sb < g.nsb; ++sb)
    for (int k = 0; k < 4; ++k) m = std::max(m, (int64_t)step_count(g.sh[sb], g.sw[sb], k));
  return m;
}

int Workspace::alloc(const Geometry &g, int P_, int C, bool params, int prec, cudaStream_t st,
                     bool mix) {
  const bool bf16 = tc_precision(prec);
  release();
  stream = st;
  P = P_;
  const int64_t pe = (int64_t)P * g.Hp * g.Wp;
  const int64_t big = (int64_t)P * g.sh.back() * g.sw.back();  // largest subband
  auto al = [](int64_t b) { return (b + 255) / 256 * 256; };
  std::vector<std::pair<void **, int64_t>> parts = {
      {(void **)&Q, al(pe * 4)},        {(void **)&Yf, al(pe * 4)},
      {(void **)&idx, al(pe * 4)},      {(void **)&T0, al(pe * 4)},
      {(void **)&T1, al(pe * 4)},       {(void **)&T2, al(pe * 4)},
      {(void **)&planes, al(pe * 4)}};
  if (!bf16) {
    parts.push_back({(void **)&X, al(big * 2 * C * 4)});
    parts.push_back({(void **)&X2, al(big * 2 * C * 4)});
    parts.push_back({(void **)&Z, al(big * C * 4)});
    parts.push_back({(void **)&U, al(big * 2 * C * 4)});
    parts.push_back({(void **)&V, al(big * C * 4)});
    parts.push_back({(void **)&Z2, al(big * C * 4)});
  }
  parts.push_back({(void **)&Cst[0], al(big * C * 4)});
  parts.push_back({(void **)&Cst[1], al(big * C * 4)});
  if (params) {
    parts.push_back({(void **)&mu, al(pe * 4)});
    parts.push_back({(void **)&sg, al(pe * 4)});
  }
  if (mix) {
    parts.push_back({(void **)&mrows, al((int64_t)P * max_step_symbols(g) * kMixRow * 2)});
    parts.push_back({(void **)&mcf, al(pe * 4)});
    if (params) parts.push_back({(void **)&mpar, al(pe * 9 * 4)});
  }
  int64_t tot = 0;
  for (auto &p : parts) tot += p.second;
  void *b = nullptr;
  if (pool_alloc(&b, (size_t)tot, stream) != PW_OK) {
    base = nullptr;
    set_last_error("workspace allocation failed");
    return PW_ENOMEM;
  }
  base = static_cast<uint8_t *>(b);
  bytes = (size_t)tot;
  int64_t o = 0;
  for (auto &p : parts) { *p.first = base + o; o += p.second; }
  if (bf16) {
    int s = tc_workspace_alloc(this, g, C, prec == PW_PREC_FP8);
    if (s != PW_OK) return s;
  }
  return PW_OK;
}

int64_t Workspace::estimate(const Geometry &g, int P, int C, bool params, int prec, bool mix) {
  const bool bf16 = tc_precision(prec);
  const int64_t pe = (int64_t)P * g.Hp * g.Wp;
  const int64_t big = (int64_t)P * g.sh.back() * g.sw.back();
  auto al = [](int64_t b) { return (b + 1023) / 1024 * 1024; };
  int64_t tot = 7 * al(pe * 4) + 2 * al(big * C * 4);
  if (!bf16) tot += 3 * al(big * 2 * C * 4) + 3 * al(big * C * 4);
  else tot += tc_workspace_bytes(g, P, C, prec == PW_PREC_FP8);
  if (params) tot += 2 * al(pe * 4);
  if (mix)
    tot += al((int64_t)P * max_step_symbols(g) * kMixRow * 2) + al(pe * 4) +
           (params ? al(pe * 9 * 4) : 0);
  return tot;
}

void Workspace::release() {
  if (tc) tc_workspace_free(this);
  pool_free(base, stream);
  base = nullptr;
  bytes = 0;
}

// ---------------------------------------------------------------------------
// ConvLSTM context prediction for subband sb >= 1 (Section 3.2). The cell
// state ping-pongs between ws.Cst[0] and ws.Cst[1] (the previous state is
// read at half resolution when the level changes).
int run_lstm(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws, int sb) {
  const int h = g.sh[sb], w = g.sw[sb], C = m.C, P = ws.P;
  const int up = g.sh[sb - 1] < h ? 1 : 0;
  const int first = sb == 1 ? 1 : 0;
  if (first) ws.lstm_cur = 0;
  const int cur = ws.lstm_cur;
  const int32_t *sprev = ws.Q + (int64_t)P * g.soff[sb - 1];
  if (tc_precision(ctx->precision)) {
    int s = tc_run_lstm(ctx, m, g, ws, sb, sprev, up, first, cur);
    ws.lstm_cur = cur ^ 1;
    return s;
  }
  const double pix = (double)P * h * w;
  // integer-network class: the quantised weights and requantisation shifts
  const IntNets *in = ctx->precision == PW_PREC_INT8 ? m.intn : nullptr;
  {
    ProfScope ps(ctx, KC_SMALL_CTX, 2.0 * pix * 9 * C, pix * (4.0 + 3.0 * C * 4));
    launch_lstm_in(sprev, ws.X2, 2 * C, C, in ? in->we : m.lstm_we, in ? in->be : m.lstm_be,
                   ws.X, P, h, w, C, up, first, ctx->stream, in ? in->n_e : kRqFloat);
  }
  if (ws.ext) {  // the gates conv reads X over 3 x 3 neighbourhoods
    launch_zero_outside(ws.X, ZL_PIXEL, P, h, w, 2 * C / 4, ws.ext, sb_level(g, sb), ctx->stream);
    bump(ctx);
  }
  ConvParams a{};
  a.in = ws.X; a.in_cs = 2 * C; a.in_co = 0; a.cin = 2 * C;
  a.w = in ? in->wg : m.lstm_wg; a.b = in ? in->bg : m.lstm_bg; a.cout_total = 4 * C;
  a.iq = in ? 1 : 0; a.rq = in ? in->n_g : 0;
  a.P = P; a.H = h; a.W = w;
  a.out = ws.X2; a.out_cs = 2 * C; a.out_co = C;
  a.c_prev = ws.Cst[cur]; a.c_new = ws.Cst[cur ^ 1]; a.up = up; a.first = first; a.C = C;
  {
    ProfScope ps(ctx, KC_LSTM_GATES, 2.0 * pix * 9 * 2 * C * 4 * C, pix * 4.0 * (2 * C + 3 * C));
    launch_conv_simt(3, a, EPI_LSTM, ctx->stream);
  }
  ws.lstm_cur = cur ^ 1;
  bump(ctx, 2);
  return PW_OK;
}

// One coding step's context fusion net -> packed table indices (Laplace),
// or centres plus table rows (decoding) / per-symbol (cdf, frequency)
// pairs (encoding) of the logistic mixture.
int run_context_pass(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws, int sb,
                     int step, bool decoding) {
  const int h = g.sh[sb], w = g.sw[sb], C = m.C, P = ws.P;
  // integer-network class: the quantised nets and their requantisation
  // shifts (iq marks every convolution of the pass)
  IntStepNet *in = nullptr;
  if (ctx->precision == PW_PREC_INT8) in = sb == 0 ? &m.intn->ll[step] : &m.intn->sb[step];
  const int iq = in ? 1 : 0;
  StepNetDev &n = in ? in->d : ((sb == 0) ? m.ll[step] : m.sb[step]);
  const int32_t *Qi = ws.Q + (int64_t)P * g.soff[sb];
  uint32_t *idx = ws.idx + (int64_t)P * g.ioff[sb * 4 + step];
  const int64_t nk = step_count(h, w, step);
  float *mu = ws.mu ? ws.mu + (int64_t)P * g.soff[sb] : nullptr;
  float *sgp = ws.sg ? ws.sg + (int64_t)P * g.soff[sb] : nullptr;
  if (tc_precision(ctx->precision))
    return tc_run_step(ctx, m, g, ws, sb, step, n, Qi, idx, nk, mu, sgp);
  cudaStream_t st = ctx->stream;
  if (sb == 0 && step == 0) {
    cudaMemsetAsync(ws.X2, 0, (size_t)P * h * w * 2 * C * 4, st);  // l = 0 for LL
  }
  // logistic mixture: the last convolution stores z' (in place over its
  // residual input), then the mixture head runs on the step's symbols
  auto mix_head = [&](const float *zp) {
    MixHeadParams mp{};
    mp.z = zp; mp.wh = n.wh; mp.bh = n.bh; mp.C = C; mp.P = P; mp.H = h; mp.W = w;
    mp.step = step; mp.nk = nk;
    mp.ctr = reinterpret_cast<int32_t *>(idx);
    if (decoding) {
      mp.rows = ws.mrows;
    } else {
      mp.q = Qi;
      mp.cf = ws.mcf + (int64_t)P * g.ioff[sb * 4 + step];
      mp.par = ws.mpar ? ws.mpar + (int64_t)P * g.soff[sb] * 9 : nullptr;
    }
    const double ns = (double)P * nk;
    ProfScope ps(ctx, KC_MIX, ns * (2.0 * 9 * C + 3.0 * 126 * 8),
                 ns * (4.0 * C + 4.0 + (decoding ? 2.0 * kMixRow : 8.0)));
    launch_mix_head(mp, st);
  };
  const double pix = (double)P * h * w;
  auto conv = [&](int ks, const ConvParams &cp, int epi) {
    const double fl = 2.0 * pix * ks * ks * cp.cin * cp.cout_total;
    const double by = pix * 4.0 * (cp.cin + cp.cout_total + (cp.res ? cp.cout_total : 0));
    ProfScope ps(ctx, ks == 3 ? (epi == EPI_HEAD ? KC_HEAD3 : KC_CONV3) : KC_CONV1, fl, by);
    launch_conv_simt(ks, cp, epi, st);
  };
  // ragged batches: zero a C-channel buffer outside the planes' extents
  // before a spatial convolution reads it
  auto mask = [&](float *buf) {
    if (!ws.ext) return;
    launch_zero_outside(buf, ZL_PIXEL, P, h, w, C / 4, ws.ext, sb_level(g, sb), st);
    bump(ctx);
  };
  ConvParams a{};
  a.P = P; a.H = h; a.W = w;
  auto base = [&]() {
    ConvParams b{};
    b.P = P; b.H = h; b.W = w;
    return b;
  };
  if (step == 0) {
    a = base();  // z = 1x1(l)
    a.in = ws.X2; a.in_cs = 2 * C; a.in_co = C; a.cin = C;
    a.w = n.win; a.b = n.bin; a.cout_total = C;
    a.out = ws.Z; a.out_cs = C;
    a.iq = iq; a.rq = iq ? in->n_win : 0;
    conv(1, a, EPI_STORE);
    a = base();  // u = lrelu(1x1 z)
    a.in = ws.Z; a.in_cs = C; a.cin = C; a.w = n.w1; a.b = n.b1; a.cout_total = C;
    a.out = ws.U; a.out_cs = C; a.act = 1;
    a.iq = iq; a.rq = iq ? in->n_w1 : 0;
    conv(1, a, EPI_STORE);
    mask(ws.U);
    {
      ProfScope ps(ctx, KC_SMALL_CTX, 2.0 * pix * 9 * C, pix * 8.0 * C);
      launch_dw3x3(ws.U, n.wdw, n.bdw, ws.V, P, h, w, C, st, iq ? in->n_dw : kRqFloat);
    }
    a = base();  // z2 = z + 1x1(v)
    a.in = ws.V; a.in_cs = C; a.cin = C; a.w = n.w2; a.b = n.b2; a.cout_total = C;
    a.out = ws.Z2; a.out_cs = C; a.res = ws.Z; a.res_cs = C;
    a.iq = iq; a.rq = iq ? in->n_w2 : 0;
    conv(1, a, EPI_STORE);
    a = base();  // u2 = lrelu(1x1(C->2C) z2)
    a.in = ws.Z2; a.in_cs = C; a.cin = C; a.w = n.w3; a.b = n.b3; a.cout_total = 2 * C;
    a.out = ws.U; a.out_cs = 2 * C; a.act = 1;
    a.iq = iq; a.rq = iq ? in->n_w3 : 0;
    conv(1, a, EPI_STORE);
    a = base();  // z3 = z2 + 1x1(2C->C) u2; head
    a.in = ws.U; a.in_cs = 2 * C; a.cin = 2 * C; a.w = n.w4; a.b = n.b4; a.cout_total = C;
    a.res = ws.Z2; a.res_cs = C;
    a.iq = iq; a.rq = iq ? in->n_w4 : 0;
    a.rq_mu = iq ? in->n_mu : 0; a.rq_rho = iq ? in->n_rho : 0;
    if (m.mix) {
      a.out = ws.Z2; a.out_cs = C;
      conv(1, a, EPI_STORE);
      mix_head(ws.Z2);
      bump(ctx, 7);
      return PW_OK;
    }
    a.wh = n.wh; a.bh = n.bh; a.step = 0; a.idx = idx; a.idx_stride = nk;
    a.mu_out = mu; a.sg_out = sgp;
    conv(1, a, EPI_HEAD);
    bump(ctx, 6);
  } else {
    {
      ProfScope ps(ctx, KC_SMALL_CTX, 2.0 * pix * 9 * C, pix * (4.0 + 4.0 * C));
      launch_masked_in(Qi, n.wa, n.ba, ws.X2, 2 * C, P, h, w, C, step, st,
                       iq ? in->n_wa : kRqFloat);
    }
    a = base();  // z = 1x1(2C->C)[a, l]
    a.in = ws.X2; a.in_cs = 2 * C; a.cin = 2 * C; a.w = n.wz; a.b = n.bz; a.cout_total = C;
    a.out = ws.Z; a.out_cs = C;
    a.iq = iq; a.rq = iq ? in->n_wz : 0;
    conv(1, a, EPI_STORE);
    mask(ws.Z);
    a = base();  // u = lrelu(conv3x3 z)
    a.in = ws.Z; a.in_cs = C; a.cin = C; a.w = n.c1w; a.b = n.c1b; a.cout_total = C;
    a.out = ws.U; a.out_cs = C; a.act = 1;
    a.iq = iq; a.rq = iq ? in->n_c1 : 0;
    conv(3, a, EPI_STORE);
    mask(ws.U);
    a = base();  // z' = z + conv3x3 u; head
    a.in = ws.U; a.in_cs = C; a.cin = C; a.w = n.c2w; a.b = n.c2b; a.cout_total = C;
    a.res = ws.Z; a.res_cs = C;
    a.iq = iq; a.rq = iq ? in->n_c2 : 0;
    a.rq_mu = iq ? in->n_mu : 0; a.rq_rho = iq ? in->n_rho : 0;
    if (m.mix) {
      a.out = ws.Z; a.out_cs = C;
      conv(3, a, EPI_STORE);
      mix_head(ws.Z);
      bump(ctx, 5);
      return PW_OK;
    }
    a.wh = n.wh; a.bh = n.bh; a.step = step; a.idx = idx; a.idx_stride = nk;
    a.mu_out = mu; a.sg_out = sgp;
    conv(3, a, EPI_HEAD);
    bump(ctx, 4);
  }
  return PW_OK;
}

// ---------------------------------------------------------------------------
// Lifting drivers (Section 3.1, Fig. 2). Subbands in ws.Yf ([sb][P][h][w]).
static PlaneAcc acc(float *p, int64_t ps, int64_t rs, int64_t cs = 1) { return {p, ps, rs, cs}; }

// One lifting half-step: CNN (9*16 + 9*16*16 + 9*16 MACs per sample) plus
// the linear part; algorithmic bytes: read src and other, write out (+copy).
static void lift_step(pw_ctx *ctx, const LiftStepParams &a) {
  const double n = (double)a.P * a.H * a.W;
  ProfScope ps(ctx, KC_LIFT, 2.0 * n * (9 * 16 + 9 * 16 * 16 + 9 * 16),
               n * 4.0 * (a.copy.p ? 4 : 3));
  launch_lift_step(a, ctx->stream);
}

int post_process_planes(pw_ctx *ctx, Model &m, const Geometry &g, int P, const float *src,
                        float *dst, const int2 *ext) {
  LiftStepParams a{};
  a.P = P; a.H = g.Hp; a.W = g.Wp; a.dir = 0; a.lin = LIN_ZERO; a.sign = +1; a.round = 0;
  a.ext = ext; a.esh = 0; a.ehmul = 1;
  a.net = m.post; a.status = ctx->status;
  a.tc = tc_precision(ctx->precision) ? 1 : 0;
  const int64_t hw = (int64_t)g.Hp * g.Wp;
  a.src = acc(const_cast<float *>(src), hw, g.Wp);
  a.other = acc(const_cast<float *>(src), hw, g.Wp);
  a.out = acc(dst, hw, g.Wp);
  a.copy = acc(nullptr, 0, 0);
  lift_step(ctx, a);
  bump(ctx);
  return PW_OK;
}

int lift_inverse_planes(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws,
                        float *dst) {
  const int P = ws.P, L = g.levels;
  const int rP = g.lossless ? 1 : 0, rU = g.lossless ? 2 : 0;
  // BF16 / FP8 precision class, lossy: the CNNs' middle layer on the tensor cores
  const int tc = (tc_precision(ctx->precision) && !g.lossless) ? 1 : 0;
  float *cur = ws.Yf;  // LL_L, plane stride h*w
  for (int lv = L; lv >= 1; --lv) {
    const int h = g.Hp >> lv, w = g.Wp >> lv;
    const int64_t hw = (int64_t)h * w;
    const int iHL = 1 + 3 * (L - lv);
    float *HL = ws.Yf + (int64_t)P * g.soff[iHL];
    float *LH = ws.Yf + (int64_t)P * g.soff[iHL + 1];
    float *HH = ws.Yf + (int64_t)P * g.soff[iHL + 2];
    float *Lo = ws.T0, *Hi = ws.T0 + (int64_t)P * 2 * hw, *E = ws.T1;
    float *X = (lv == 1) ? dst : ws.T2;
    auto colinv = [&](float *Lb, float *Hb, float *out) {
      LiftStepParams a{};
      a.P = P; a.H = h; a.W = w; a.dir = 1; a.tc = tc; a.status = ctx->status;
      a.ext = ws.ext; a.esh = lv; a.ehmul = 1;
      a.src = acc(Hb, hw, w); a.other = acc(Lb, hw, w); a.out = acc(E, hw, w);
      a.copy = acc(nullptr, 0, 0); a.net = m.lift[1][1]; a.lin = LIN_U53; a.sign = -1;
      a.round = rU;
      lift_step(ctx, a);
      a.src = acc(E, hw, w); a.other = acc(Hb, hw, w);
      a.out = acc(out + w, 2 * hw, 2 * w); a.copy = acc(out, 2 * hw, 2 * w);
      a.net = m.lift[1][0]; a.lin = LIN_P53; a.sign = 1; a.round = rP;
      lift_step(ctx, a);
    };
    colinv(cur, LH, Lo);
    colinv(HL, HH, Hi);
    LiftStepParams a{};
    a.P = P; a.H = 2 * h; a.W = w; a.dir = 0; a.tc = tc; a.status = ctx->status;
    a.ext = ws.ext; a.esh = lv; a.ehmul = 2;
    a.src = acc(Hi, 2 * hw, w); a.other = acc(Lo, 2 * hw, w); a.out = acc(E, 2 * hw, w);
    a.copy = acc(nullptr, 0, 0); a.net = m.lift[0][1]; a.lin = LIN_U53; a.sign = -1;
    a.round = rU;
    lift_step(ctx, a);
    a.src = acc(E, 2 * hw, w); a.other = acc(Hi, 2 * hw, w);
    a.out = acc(X + 1, 4 * hw, 2 * w, 2); a.copy = acc(X, 4 * hw, 2 * w, 2);
    a.net = m.lift[0][0]; a.lin = LIN_P53; a.sign = 1; a.round = rP;
    lift_step(ctx, a);
    bump(ctx, 6);
    cur = X;
  }
  return PW_OK;
}

int lift_forward_planes(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws,
                        const float *src) {
  const int P = ws.P, L = g.levels;
  const int rP = g.lossless ? 1 : 0, rU = g.lossless ? 2 : 0;
  float *cur = const_cast<float *>(src);
  for (int lv = 1; lv <= L; ++lv) {
    const int h = g.Hp >> lv, w = g.Wp >> lv;
    const int64_t hw = (int64_t)h * w;
    const int iHL = 1 + 3 * (L - lv);
    float *HL = ws.Yf + (int64_t)P * g.soff[iHL];
    float *LH = ws.Yf + (int64_t)P * g.soff[iHL + 1];
    float *HH = ws.Yf + (int64_t)P * g.soff[iHL + 2];
    float *Lo = ws.T0, *Hi = ws.T0 + (int64_t)P * 2 * hw;
    float *nxt = (lv == L) ? ws.Yf : ((lv & 1) ? ws.T1 : ws.T2);
    LiftStepParams a{};
    a.P = P; a.H = 2 * h; a.W = w; a.dir = 0; a.copy = acc(nullptr, 0, 0);
    // rows: Hi = odd - P(even); Lo = even + U(Hi)
    a.src = acc(cur, 4 * hw, 2 * w, 2); a.other = acc(cur + 1, 4 * hw, 2 * w, 2);
    a.out = acc(Hi, 2 * hw, w); a.net = m.lift[0][0]; a.lin = LIN_P53; a.sign = -1;
    a.round = rP;
    lift_step(ctx, a);
    a.src = acc(Hi, 2 * hw, w); a.other = acc(cur, 4 * hw, 2 * w, 2);
    a.out = acc(Lo, 2 * hw, w); a.net = m.lift[0][1]; a.lin = LIN_U53; a.sign = 1;
    a.round = rU;
    lift_step(ctx, a);
    // columns on Lo -> (LL, LH), on Hi -> (HL, HH)
    auto colfwd = [&](float *Sb, float *lowout, float *highout) {
      LiftStepParams b{};
      b.P = P; b.H = h; b.W = w; b.dir = 1; b.copy = acc(nullptr, 0, 0);
      b.src = acc(Sb, 2 * hw, 2 * w); b.other = acc(Sb + w, 2 * hw, 2 * w);
      b.out = acc(highout, hw, w); b.net = m.lift[1][0]; b.lin = LIN_P53; b.sign = -1;
      b.round = rP;
      lift_step(ctx, b);
      b.src = acc(highout, hw, w); b.other = acc(Sb, 2 * hw, 2 * w);
      b.out = acc(lowout, hw, w); b.net = m.lift[1][1]; b.lin = LIN_U53; b.sign = 1;
      b.round = rU;
      lift_step(ctx, b);
    };
    colfwd(Lo, nxt, LH);
    colfwd(Hi, HL, HH);
    bump(ctx, 6);
    cur = nxt;
  }
  return PW_OK;
}

// ---------------------------------------------------------------------------
// Temporal lifting of a GOP (Section 3.3, identity motion): frames are
// nf x nc planes [frame][comp][Hp][Wp]. Forward: per level, pairs (f_e, f_o)
// -> H = f_o - (f_e + CNN_P(f_e)), L = f_e + (H / 2 + CNN_U(H)); bands are
// written as [L_T, H_T, H_{T-1} ..., H_1] (highs of a level in frame order).
// Inverse runs the same steps backwards. tmp holds nf / 2 frames.
int temporal_planes(pw_ctx *ctx, Model &m, int nf, int nc, int Hp, int Wp, const float *in,
                    float *out, float *tmp0, float *tmp1, bool forward, const int8_t *mv,
                    float *twarp) {
  const int64_t HW = (int64_t)Hp * Wp;
  const int64_t F = (int64_t)nc * HW;  // one frame
  int T = 0;
  while ((1 << T) < nf) ++T;
  if ((1 << T) != nf || nf < 2) { set_last_error("GOP size must be a power of two >= 2"); return PW_EINVAL; }
  if (mv && !twarp) { set_last_error("motion-compensated lifting needs scratch"); return PW_EINVAL; }
  // the inverse (decoder) runs the CNNs' middle layers on the tensor cores in
  // the BF16 / FP8 classes, as the spatial inverse lifting does; the
  // encoder's forward transform stays FP32
  const int tc = (!forward && tc_precision(ctx->precision)) ? 1 : 0;
  auto step = [&](const float *src, int64_t ssrc, const float *oth, int64_t soth, float *dst,
                  int64_t sdst, int P, int lin, int sign, const LiftNetDev &net) {
    LiftStepParams a{};
    a.P = P; a.H = Hp; a.W = Wp; a.dir = 0; a.lin = lin; a.sign = sign; a.round = 0; a.net = net;
    a.tc = tc; a.status = ctx->status;
    a.src = acc(const_cast<float *>(src), ssrc, Wp);
    a.other = acc(const_cast<float *>(oth), soth, Wp);
    a.out = acc(dst, sdst, Wp);
    a.copy = acc(nullptr, 0, 0);
    lift_step(ctx, a);
  };
  // MC (sign +1) or inverse MC (-1) of P planes with the vectors of fields
  // field0 .. field0 + P - 1 into the scratch planes (stride F)
  auto warp = [&](const float *src, int64_t ssrc, int P, int field0, int sign) {
    launch_mc_warp(acc(const_cast<float *>(src), ssrc, Wp), acc(twarp, F, Wp), P, Hp, Wp, mv,
                   field0, sign, ctx->stream);
    bump(ctx);
    return twarp;
  };
  // first field of level lv (fields of level 1 first, nf / 2 of them)
  auto field0_of = [&](int lv) {
    int f = 0;
    for (int l = 1; l < lv; ++l) f += nf >> l;
    return f;
  };
  if (forward) {
    const float *cur = in;
    float *bufs[2] = {tmp0, tmp1};
    for (int lv = 1; lv <= T; ++lv) {
      const int n = nf >> (lv - 1), h = n / 2;
      const int f0 = field0_of(lv);
      float *L = (lv == T) ? out : bufs[lv & 1];
      for (int c = 0; c < nc; ++c) {
        const float *fe = cur + c * HW, *fo = cur + F + c * HW;
        float *Hb = out + (int64_t)h * F + c * HW;
        if (mv) {
          // H = fo - P(MC(fe)); L = fe + U(IMC(H))
          step(warp(fe, 2 * F, h, f0, +1), F, fo, 2 * F, Hb, F, h, LIN_ID, -1,
               m.tlift[0]);
          step(warp(Hb, F, h, f0, -1), F, fe, 2 * F, L + c * HW, F, h, LIN_HALF, +1, m.tlift[1]);
        } else {
          step(fe, 2 * F, fo, 2 * F, Hb, F, h, LIN_ID, -1, m.tlift[0]);
          step(Hb, F, fe, 2 * F, L + c * HW, F, h, LIN_HALF, +1, m.tlift[1]);
        }
      }
      ctx->launches += 2 * nc;
      cur = L;
    }
  } else {
    // bands in `in`; start from L_T, rebuild level by level
    const float *cur = in;  // L of the current level: frame 0 of the bands
    float *bufs[2] = {tmp0, tmp1};
    for (int lv = T; lv >= 1; --lv) {
      const int n = nf >> (lv - 1), h = n / 2;
      const int f0 = field0_of(lv);
      float *dst = (lv == 1) ? out : bufs[lv & 1];
      for (int c = 0; c < nc; ++c) {
        const float *Hb = in + (int64_t)h * F + c * HW, *L = cur + c * HW;
        float *fe = dst + c * HW, *fo = dst + F + c * HW;
        if (mv) {
          // fe = L - U(IMC(H)); fo = H + P(MC(fe))
          step(warp(Hb, F, h, f0, -1), F, L, F, fe, 2 * F, h, LIN_HALF, -1, m.tlift[1]);
          step(warp(fe, 2 * F, h, f0, +1), F, Hb, F, fo, 2 * F, h, LIN_ID, +1, m.tlift[0]);
        } else {
          step(Hb, F, L, F, fe, 2 * F, h, LIN_HALF, -1, m.tlift[1]);
          step(fe, 2 * F, Hb, F, fo, 2 * F, h, LIN_ID, +1, m.tlift[0]);
        }
      }
      ctx->launches += 2 * nc;
      cur = dst;
    }
  }
  return PW_OK;
}

}  // namespace pw
