// Weight-blob parsing and device weight layouts.
//
// A blob ("PWMB") holds one lambda model (Section 4.1): the lifting
// predict/update CNNs (Section 3.1), the temporal lifting nets (Section
// 3.3), the ConvLSTM context prediction module and the four-step context
// fusion nets (Section 3.2). Tensors are found by name; their shapes are
// checked against the configuration in the blob header.
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <map>

#include <cuda_bf16.h>

#include "codec.h"

namespace pw {

namespace {

struct BlobTensor {
  std::vector<int> shape;
  const float *data;
};

uint64_t poly_hash(const uint8_t *p, size_t n) {
  // h = sum_i (w_i + 1) * P^(i+1) mod 2^64 over little-endian u32 words
  const uint64_t P = 0x100000001B3ull;
  uint64_t h = 0, pw = 1;
  for (size_t i = 0; i + 4 <= n; i += 4) {
    uint32_t w;
    std::memcpy(&w, p + i, 4);
    pw *= P;
    h += ((uint64_t)w + 1ull) * pw;
  }
  return h;
}

// ---- integer-network weights ----------------------------------------------
// Largest integer k with m 2^k <= lim (m > 0), found exactly.
int max_shift(double m, double lim) {
  int k = (int)std::floor(std::log2(lim / m));
  while (std::ldexp(m, k + 1) <= lim) ++k;
  while (std::ldexp(m, k) > lim) --k;
  return k;
}

struct QGroup {
  int c0, n, fa;  // input channels [c0, c0 + n) carrying fa fractional bits
};
constexpr double kWMax = 56.0, kBMax = 262144.0;  // |w_q| <= 56, |b_q| <= 2^18

// Quantise a convolution's weights w ([cout][cin][kk], the blob's layout)
// and bias b: k_g = the largest k with max|w_g| 2^k <= 56 per input group,
// S = min_g (k_g + fa_g), lowered so that max|b| 2^S <= 2^18; w_q =
// rint(w 2^(S - fa_g)), b_q = rint(b 2^S) (round half to even), kept as
// exact float integers in the same layout. Returns S.
int quantise(const std::vector<float> &w, const std::vector<float> &b, int cout, int cin, int kk,
             std::initializer_list<QGroup> groups, std::vector<float> &wq,
             std::vector<float> &bq) {
  int S = 0;
  bool any = false;
  for (const QGroup &g : groups) {
    double m = 0.0;
    for (int o = 0; o < cout; ++o)
      for (int ci = g.c0; ci < g.c0 + g.n; ++ci)
        for (int t = 0; t < kk; ++t)
          m = std::max(m, std::fabs((double)w[((size_t)o * cin + ci) * kk + t]));
    if (m > 0.0) {
      const int k = max_shift(m, kWMax) + g.fa;
      S = any ? std::min(S, k) : k;
      any = true;
    }
  }
  if (!any) S = 30;
  double mb = 0.0;
  for (float v : b) mb = std::max(mb, std::fabs((double)v));
  if (mb > 0.0) S = std::min(S, max_shift(mb, kBMax));
  wq.assign(w.size(), 0.f);
  for (const QGroup &g : groups)
    for (int o = 0; o < cout; ++o)
      for (int ci = g.c0; ci < g.c0 + g.n; ++ci)
        for (int t = 0; t < kk; ++t) {
          const size_t i = ((size_t)o * cin + ci) * kk + t;
          wq[i] = (float)std::nearbyint(std::ldexp((double)w[i], S - g.fa));
        }
  bq.resize(b.size());
  for (size_t i = 0; i < b.size(); ++i) bq[i] = (float)std::nearbyint(std::ldexp((double)b[i], S));
  return S;
}

}  // namespace

int Model::load(pw_ctx *c, const void *blob, size_t n) {
  static uint64_t next_uid = 1;
  ctx = c;
  uid = __atomic_fetch_add(&next_uid, 1, __ATOMIC_RELAXED);
  const uint8_t *b = static_cast<const uint8_t *>(blob);
  if (n < 32 || std::memcmp(b, "PWMB", 4) != 0) {
    set_last_error("weight blob: bad magic");
    return PW_EINVAL;
  }
  uint32_t hdr[7];
  std::memcpy(hdr, b + 4, sizeof(hdr));
  if (hdr[0] != 1) { set_last_error("weight blob: unsupported version"); return PW_EINVAL; }
  levels = (int)hdr[1]; C = (int)hdr[2]; F = (int)hdr[3]; ll_mode = (int)hdr[4];
  const uint32_t nt = hdr[5];
  if (levels < 1 || levels > 6 || F != 16 || (C != 32 && C != 64 && C != 128) || ll_mode > 1 ||
      32ull + 64ull * nt > n || (n & 3)) {
    set_last_error("weight blob: unsupported configuration (levels 1..6, F = 16, C in {32, 64, 128})");
    return PW_EUNSUPPORTED;
  }
  std::map<std::string, BlobTensor> ts;
  for (uint32_t i = 0; i < nt; ++i) {
    const uint8_t *r = b + 32 + 64 * i;
    char name[41];
    std::memcpy(name, r, 40);
    name[40] = 0;
    uint32_t f[6];
    std::memcpy(f, r + 40, sizeof(f));
    if (f[0] < 1 || f[0] > 4) { set_last_error("weight blob: bad rank"); return PW_EINVAL; }
    BlobTensor t;
    size_t cnt = 1;
    for (uint32_t d = 0; d < f[0]; ++d) { t.shape.push_back((int)f[1 + d]); cnt *= f[1 + d]; }
    if ((size_t)f[5] + 4 * cnt > n || (f[5] & 3)) {
      set_last_error(std::string("weight blob: tensor out of range: ") + name);
      return PW_EINVAL;
    }
    t.data = reinterpret_cast<const float *>(b + f[5]);
    ts[name] = t;
  }
  hash = poly_hash(b, n);

  auto get = [&](const std::string &name, std::vector<int> shape,
                 std::vector<float> &out) -> bool {
    auto it = ts.find(name);
    if (it == ts.end() || it->second.shape != shape) {
      set_last_error("weight blob: missing or mis-shaped tensor " + name);
      return false;
    }
    size_t cnt = 1;
    for (int s : shape) cnt *= (size_t)s;
    out.resize(cnt);
    std::memcpy(out.data(), it->second.data, cnt * 4);
    return true;
  };
  std::vector<float> t0, t1;
  // layout converters
  auto conv_tap_major = [](const std::vector<float> &w, int co, int ci, int k) {
    // [co][ci][k][k] -> [tap][ci][co]
    std::vector<float> o((size_t)co * ci * k * k);
    for (int a = 0; a < co; ++a)
      for (int c = 0; c < ci; ++c)
        for (int t = 0; t < k * k; ++t)
          o[((size_t)t * ci + c) * co + a] = w[((size_t)a * ci + c) * k * k + t];
    return o;
  };
  auto transpose = [](const std::vector<float> &w, int co, int ci) {
    std::vector<float> o((size_t)co * ci);
    for (int a = 0; a < co; ++a)
      for (int c = 0; c < ci; ++c) o[(size_t)c * co + a] = w[(size_t)a * ci + c];
    return o;
  };

  int st = PW_OK;
  auto up = [&](const std::vector<float> &h) -> float * {
    float *d = nullptr;
    if (cudaMalloc(&d, h.size() * 4) != cudaSuccess) { st = PW_ENOMEM; return nullptr; }
    cudaMemcpy(d, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
    allocs.push_back(d);
    return d;
  };
  host.clear();
  auto keep = [&](const std::string &name, const std::vector<float> &v) { host[name] = v; };

  // lifting nets: w1 [16,1,3,3], w2 [16,16,3,3], w3 [1,16,3,3] (already [co][ci][9])
  auto load_lift = [&](const std::string &p, LiftNetDev &n) -> bool {
    std::vector<float> w1, b1, w2, b2, w3, b3;
    if (!get(p + "w1", {16, 1, 3, 3}, w1) || !get(p + "b1", {16}, b1) ||
        !get(p + "w2", {16, 16, 3, 3}, w2) || !get(p + "b2", {16}, b2) ||
        !get(p + "w3", {1, 16, 3, 3}, w3) || !get(p + "b3", {1}, b3))
      return false;
    n.w1 = up(w1); n.b1 = up(b1); n.w2 = up(w2); n.b2 = up(b2); n.w3 = up(w3); n.b3 = up(b3);
    {
      // packed BF16 B operands: [tap][ci / 8][c][ci % 8]
      std::vector<__nv_bfloat16> b2p(9 * 2 * 16 * 8), b3p(9 * 2 * 16 * 8, __float2bfloat16(0.f));
      for (int c = 0; c < 16; ++c)
        for (int ci = 0; ci < 16; ++ci)
          for (int tap = 0; tap < 9; ++tap) {
            const size_t o = ((size_t)(tap * 2 + ci / 8) * 16 + c) * 8 + ci % 8;
            b2p[o] = __float2bfloat16(w2[((size_t)c * 16 + ci) * 9 + tap]);
            if (c == 0) b3p[o] = __float2bfloat16(w3[(size_t)ci * 9 + tap]);
          }
      void *d2 = nullptr, *d3 = nullptr;
      if (cudaMalloc(&d2, b2p.size() * 2) != cudaSuccess ||
          cudaMalloc(&d3, b3p.size() * 2) != cudaSuccess) {
        cudaFree(d2);
        st = PW_ENOMEM;
        return false;
      }
      allocs.push_back(static_cast<float *>(d2));
      allocs.push_back(static_cast<float *>(d3));
      cudaMemcpy(d2, b2p.data(), b2p.size() * 2, cudaMemcpyHostToDevice);
      cudaMemcpy(d3, b3p.data(), b3p.size() * 2, cudaMemcpyHostToDevice);
      n.w2b = d2;
      n.w3b = d3;
    }
    keep(p + "w2", w2); keep(p + "w1", w1); keep(p + "w3", w3);
    keep(p + "b1", b1); keep(p + "b2", b2); keep(p + "b3", b3);
    return true;
  };
  const char *dirs[2] = {"row", "col"};
  const char *ops[2] = {"P", "U"};
  for (int d = 0; d < 2; ++d)
    for (int o = 0; o < 2; ++o)
      if (!load_lift(std::string("lift.") + dirs[d] + "." + ops[o] + ".", lift[d][o]))
        return PW_EINVAL;
  for (int o = 0; o < 2; ++o)
    if (!load_lift(std::string("tlift.") + ops[o] + ".", tlift[o])) return PW_EINVAL;
  // optional post-processing net (same structure as the lifting nets)
  has_post = false;
  if (ts.count("post.w1")) {
    if (!load_lift("post.", post)) return PW_EINVAL;
    has_post = true;
  }

  // ConvLSTM
  {
    std::vector<float> we, be, wg, bg;
    if (!get("lstm.we", {C, 1, 3, 3}, we) || !get("lstm.be", {C}, be) ||
        !get("lstm.wg", {4 * C, 2 * C, 3, 3}, wg) || !get("lstm.bg", {4 * C}, bg))
      return PW_EINVAL;
    lstm_we = up(we);
    lstm_be = up(be);
    // permute output channels: gate * C + ch -> 4 * ch + gate
    std::vector<float> wgp(wg.size()), bgp(bg.size());
    for (int g = 0; g < 4; ++g)
      for (int ch = 0; ch < C; ++ch) {
        const int o = g * C + ch, o2 = 4 * ch + g;
        bgp[o2] = bg[o];
        std::memcpy(&wgp[(size_t)o2 * 2 * C * 9], &wg[(size_t)o * 2 * C * 9], 2 * C * 9 * 4);
      }
    lstm_wg = up(conv_tap_major(wgp, 4 * C, 2 * C, 3));
    lstm_bg = up(bgp);
    keep("lstm.wg.perm", wgp);
    keep("lstm.bg.perm", bgp);
    keep("lstm.we", we);
    keep("lstm.be", be);
  }
  // heads: 2 outputs (Laplace mean and scale) or, four-step LL models only,
  // 9 (logistic mixture of 3: weight logits, means, scale pre-activations)
  {
    auto it = ts.find("sb.s0.wh");
    nh = (ll_mode == 0 && it != ts.end() && !it->second.shape.empty() &&
          it->second.shape[0] == 9) ? 9 : 2;
    mix = nh == 9;
  }
  // four-step nets
  auto load_set = [&](const std::string &ns, StepNetDev *nets) -> bool {
    {
      StepNetDev &s = nets[0];
      const std::string p = ns + ".s0.";
      std::vector<float> w, bb;
      if (!get(p + "win", {C, C}, w) || !get(p + "bin", {C}, bb)) return false;
      s.win = up(transpose(w, C, C)); s.bin = up(bb); keep(p + "win", w); keep(p + "bin", bb);
      if (!get(p + "w1", {C, C}, w) || !get(p + "b1", {C}, bb)) return false;
      s.w1 = up(transpose(w, C, C)); s.b1 = up(bb); keep(p + "w1", w); keep(p + "b1", bb);
      if (!get(p + "wdw", {C, 3, 3}, w) || !get(p + "bdw", {C}, bb)) return false;
      s.wdw = up(w); s.bdw = up(bb);
      if (!get(p + "w2", {C, C}, w) || !get(p + "b2", {C}, bb)) return false;
      s.w2 = up(transpose(w, C, C)); s.b2 = up(bb); keep(p + "w2", w); keep(p + "b2", bb);
      if (!get(p + "w3", {2 * C, C}, w) || !get(p + "b3", {2 * C}, bb)) return false;
      s.w3 = up(transpose(w, 2 * C, C)); s.b3 = up(bb); keep(p + "w3", w); keep(p + "b3", bb);
      if (!get(p + "w4", {C, 2 * C}, w) || !get(p + "b4", {C}, bb)) return false;
      s.w4 = up(transpose(w, C, 2 * C)); s.b4 = up(bb); keep(p + "w4", w); keep(p + "b4", bb);
      if (!get(p + "wh", {nh, C}, w) || !get(p + "bh", {nh}, bb)) return false;
      s.wh = up(w); s.bh = up(bb); keep(p + "wh", w); keep(p + "bh", bb);
    }
    for (int k = 1; k < 4; ++k) {
      StepNetDev &s = nets[k];
      const std::string p = ns + ".s" + std::to_string(k) + ".";
      std::vector<float> w, bb;
      if (!get(p + "wa", {C, 1, 3, 3}, w) || !get(p + "ba", {C}, bb)) return false;
      s.wa = up(w); s.ba = up(bb); keep(p + "wa", w); keep(p + "ba", bb);
      if (!get(p + "wz", {C, 2 * C}, w) || !get(p + "bz", {C}, bb)) return false;
      s.wz = up(transpose(w, C, 2 * C)); s.bz = up(bb); keep(p + "wz", w); keep(p + "bz", bb);
      if (!get(p + "w1", {C, C, 3, 3}, w) || !get(p + "b1", {C}, bb)) return false;
      s.c1w = up(conv_tap_major(w, C, C, 3)); s.c1b = up(bb); keep(p + "w1", w); keep(p + "b1", bb);
      if (!get(p + "w2", {C, C, 3, 3}, w) || !get(p + "b2", {C}, bb)) return false;
      s.c2w = up(conv_tap_major(w, C, C, 3)); s.c2b = up(bb); keep(p + "w2", w); keep(p + "b2", bb);
      if (!get(p + "wh", {nh, C}, w) || !get(p + "bh", {nh}, bb)) return false;
      s.wh = up(w); s.bh = up(bb); keep(p + "wh", w); keep(p + "bh", bb);
    }
    return true;
  };
  if (!load_set("sb", sb)) return PW_EINVAL;
  if (ll_mode == 0) {
    if (!load_set("ll", ll)) return PW_EINVAL;
  } else {
    std::vector<float> w, bb;
    if (!get("ar.w5", {C, 1, 5, 5}, w) || !get("ar.b5", {C}, bb)) return PW_EINVAL;
    ar_w5 = up(w); ar_b5 = up(bb);
    if (!get("ar.w1", {C, C}, w) || !get("ar.b1", {C}, bb)) return PW_EINVAL;
    ar_w1 = up(w); ar_b1 = up(bb);
    if (!get("ar.wh", {2, C}, w) || !get("ar.bh", {2}, bb)) return PW_EINVAL;
    ar_wh = up(w); ar_bh = up(bb);
  }
  // integer-network class: quantised copies of the context model
  delete intn;
  intn = nullptr;
  if (c->precision == PW_PREC_INT8 && !mix && st == PW_OK) {
    const int FA = 4, FH = 7;
    IntNets *in = new IntNets();
    std::vector<float> w, bb, wq, bq;
    bool ok = true;
    // shifts of layer outputs with 4 fractional bits (head: 4 for 16 mu, 3
    // for the 8-per-octave scale bins)
    auto shift_ok = [&](int n) { ok = ok && n >= -30 && n <= 62; return n; };
    if (!get("lstm.we", {C, 1, 3, 3}, w) || !get("lstm.be", {C}, bb)) ok = false;
    if (ok) {
      in->n_e = shift_ok(quantise(w, bb, C, 1, 9, {{0, 1, 0}}, wq, bq) - FA);
      in->we = up(wq); in->be = up(bq);
    }
    if (ok && get("lstm.wg", {4 * C, 2 * C, 3, 3}, w) && get("lstm.bg", {4 * C}, bb)) {
      in->n_g = shift_ok(quantise(w, bb, 4 * C, 2 * C, 9, {{0, C, FA}, {C, C, FH}}, wq, bq) - FA);
      std::vector<float> wp(wq.size()), bp(bq.size());
      for (int g = 0; g < 4; ++g)
        for (int ch = 0; ch < C; ++ch) {
          const int o = g * C + ch, o2 = 4 * ch + g;  // gate-interleaved outputs
          bp[o2] = bq[o];
          std::memcpy(&wp[(size_t)o2 * 2 * C * 9], &wq[(size_t)o * 2 * C * 9], 2 * C * 9 * 4);
        }
      in->wg = up(conv_tap_major(wp, 4 * C, 2 * C, 3));
      in->bg = up(bp);
    } else {
      ok = false;
    }
    if (ok && ll_mode == 1) {
      // autoregressive LL: the 5x5 weights masked to the 12 causal taps
      // before quantisation (the mask decides the scale)
      if (get("ar.w5", {C, 1, 5, 5}, w) && get("ar.b5", {C}, bb)) {
        for (int co = 0; co < C; ++co)
          for (int t = 0; t < 25; ++t)
            if (!(t < 10 || t == 10 || t == 11)) w[(size_t)co * 25 + t] = 0.f;
        in->ar_n5 = shift_ok(quantise(w, bb, C, 1, 25, {{0, 1, 0}}, wq, bq) - FA);
        in->ar_w5 = up(wq); in->ar_b5 = up(bq);
      } else {
        ok = false;
      }
      if (ok && get("ar.w1", {C, C}, w) && get("ar.b1", {C}, bb)) {
        in->ar_n1 = shift_ok(quantise(w, bb, C, C, 1, {{0, C, FA}}, wq, bq) - FA);
        in->ar_w1 = up(wq); in->ar_b1 = up(bq);
      } else {
        ok = false;
      }
      if (ok && get("ar.wh", {2, C}, w) && get("ar.bh", {2}, bb)) {
        const int Sh = quantise(w, bb, 2, C, 1, {{0, C, FA}}, wq, bq);
        in->ar_nmu = shift_ok(Sh - 4);
        in->ar_nrho = shift_ok(Sh - 3);
        in->ar_wh = up(wq); in->ar_bh = up(bq);
      } else {
        ok = false;
      }
    }
    for (int set = 0; set < (ll_mode == 0 ? 2 : 1) && ok; ++set) {
      const std::string ns = set ? "ll" : "sb";
      IntStepNet *nets = set ? in->ll : in->sb;
      auto q1 = [&](const std::string &name, int co, int ci, int kk,
                    std::initializer_list<QGroup> g, float *&dw, float *&db, bool tap_major,
                    bool transp) -> int {
        std::vector<int> shp = kk == 9 ? std::vector<int>{co, ci, 3, 3} : std::vector<int>{co, ci};
        if (name.find("wdw") != std::string::npos) shp = {co, 3, 3};
        if (!get(name, shp, w)) { ok = false; return 0; }
        // its bias: "w..." -> "b..." in the last name component
        const std::string bn = name.substr(0, name.rfind('.') + 1) + "b" +
                               name.substr(name.rfind('.') + 2);
        if (!get(bn, {co}, bb)) { ok = false; return 0; }
        const int S = quantise(w, bb, co, ci, kk, g, wq, bq);
        dw = up(tap_major ? conv_tap_major(wq, co, ci, 3) : transp ? transpose(wq, co, ci) : wq);
        db = up(bq);
        return S;
      };
      {
        IntStepNet &s0 = nets[0];
        const std::string p = ns + ".s0.";
        s0.n_win = shift_ok(q1(p + "win", C, C, 1, {{0, C, FH}}, s0.d.win, s0.d.bin, false, true) - FA);
        s0.n_w1 = shift_ok(q1(p + "w1", C, C, 1, {{0, C, FA}}, s0.d.w1, s0.d.b1, false, true) - FA);
        s0.n_dw = shift_ok(q1(p + "wdw", C, 1, 9, {{0, 1, FA}}, s0.d.wdw, s0.d.bdw, false, false) - FA);
        s0.n_w2 = shift_ok(q1(p + "w2", C, C, 1, {{0, C, FA}}, s0.d.w2, s0.d.b2, false, true) - FA);
        s0.n_w3 = shift_ok(q1(p + "w3", 2 * C, C, 1, {{0, C, FA}}, s0.d.w3, s0.d.b3, false, true) - FA);
        s0.n_w4 = shift_ok(q1(p + "w4", C, 2 * C, 1, {{0, 2 * C, FA}}, s0.d.w4, s0.d.b4, false, true) - FA);
        const int Sh = q1(p + "wh", 2, C, 1, {{0, C, FA}}, s0.d.wh, s0.d.bh, false, false);
        s0.n_mu = shift_ok(Sh - 4);
        s0.n_rho = shift_ok(Sh - 3);
      }
      for (int k = 1; k < 4 && ok; ++k) {
        IntStepNet &sk = nets[k];
        const std::string p = ns + ".s" + std::to_string(k) + ".";
        sk.n_wa = shift_ok(q1(p + "wa", C, 1, 9, {{0, 1, 0}}, sk.d.wa, sk.d.ba, false, false) - FA);
        sk.n_wz = shift_ok(q1(p + "wz", C, 2 * C, 1, {{0, C, FA}, {C, C, FH}}, sk.d.wz, sk.d.bz, false, true) - FA);
        sk.n_c1 = shift_ok(q1(p + "w1", C, C, 9, {{0, C, FA}}, sk.d.c1w, sk.d.c1b, true, false) - FA);
        sk.n_c2 = shift_ok(q1(p + "w2", C, C, 9, {{0, C, FA}}, sk.d.c2w, sk.d.c2b, true, false) - FA);
        const int Sh = q1(p + "wh", 2, C, 1, {{0, C, FA}}, sk.d.wh, sk.d.bh, false, false);
        sk.n_mu = shift_ok(Sh - 4);
        sk.n_rho = shift_ok(Sh - 3);
      }
    }
    if (ok && st == PW_OK) {
      intn = in;
    } else {
      delete in;
      if (!ok) set_last_error("integer-network weights: a tensor is missing or out of range");
    }
  }
  cudaDeviceSynchronize();
  return st;
}

Model::~Model() {
  for (float *p : allocs) cudaFree(p);
  free_tc();
  delete intn;
}

}  // namespace pw
