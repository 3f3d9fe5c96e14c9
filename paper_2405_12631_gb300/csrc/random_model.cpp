// Seeded random-init weights of the model architecture, serialised as a
// weight blob ("PWMB"). The paper trains one model per rate-distortion
// trade-off (Section 4.1); without trained weights, a random-init model of
// the same architecture (lifting predict/update CNNs of Section 3.1, the
// temporal lifting nets of Section 3.3, the ConvLSTM and the four-step
// context fusion nets of Section 3.2) stands in, and C callers can create
// one here without any other tool.
//
// Tensors, shapes, order and per-tensor uniform bounds are those of every
// random-init blob of this format; the numbers come from SplitMix64 (Steele,
// Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
// 2014) keyed by (seed, tensor index, element index), so any element can be
// drawn independently of the others. Host code only.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "codec.h"

namespace pw {
namespace {

struct Spec {
  std::string name;
  std::vector<uint32_t> shape;
};

// (name, shape) of every parameter tensor in blob order; 1x1 weights are
// [Cout, Cin], 3x3 weights [Cout, Cin, 3, 3], depthwise [C, 3, 3].
std::vector<Spec> tensor_specs(uint32_t C, uint32_t F, int ll_mode) {
  std::vector<Spec> s;
  auto cnn = [&](const std::string &p) {
    s.push_back({p + "w1", {F, 1, 3, 3}});
    s.push_back({p + "b1", {F}});
    s.push_back({p + "w2", {F, F, 3, 3}});
    s.push_back({p + "b2", {F}});
    s.push_back({p + "w3", {1, F, 3, 3}});
    s.push_back({p + "b3", {1}});
  };
  for (const char *d : {"row", "col"})
    for (const char *op : {"P", "U"}) cnn(std::string("lift.") + d + "." + op + ".");
  for (const char *op : {"P", "U"}) cnn(std::string("tlift.") + op + ".");
  s.push_back({"lstm.we", {C, 1, 3, 3}});
  s.push_back({"lstm.be", {C}});
  s.push_back({"lstm.wg", {4 * C, 2 * C, 3, 3}});
  s.push_back({"lstm.bg", {4 * C}});
  std::vector<std::string> sets = {"sb"};
  if (ll_mode == 0) sets.push_back("ll");
  for (const std::string &ns : sets) {
    const std::string p = ns + ".s0.";
    s.push_back({p + "win", {C, C}});
    s.push_back({p + "bin", {C}});
    s.push_back({p + "w1", {C, C}});
    s.push_back({p + "b1", {C}});
    s.push_back({p + "wdw", {C, 3, 3}});
    s.push_back({p + "bdw", {C}});
    s.push_back({p + "w2", {C, C}});
    s.push_back({p + "b2", {C}});
    s.push_back({p + "w3", {2 * C, C}});
    s.push_back({p + "b3", {2 * C}});
    s.push_back({p + "w4", {C, 2 * C}});
    s.push_back({p + "b4", {C}});
    s.push_back({p + "wh", {2, C}});
    s.push_back({p + "bh", {2}});
    for (int k = 1; k <= 3; ++k) {
      const std::string q = ns + ".s" + std::to_string(k) + ".";
      s.push_back({q + "wa", {C, 1, 3, 3}});
      s.push_back({q + "ba", {C}});
      s.push_back({q + "wz", {C, 2 * C}});
      s.push_back({q + "bz", {C}});
      s.push_back({q + "w1", {C, C, 3, 3}});
      s.push_back({q + "b1", {C}});
      s.push_back({q + "w2", {C, C, 3, 3}});
      s.push_back({q + "b2", {C}});
      s.push_back({q + "wh", {2, C}});
      s.push_back({q + "bh", {2}});
    }
  }
  if (ll_mode == 1) {
    s.push_back({"ar.w5", {C, 1, 5, 5}});
    s.push_back({"ar.b5", {C}});
    s.push_back({"ar.w1", {C, C}});
    s.push_back({"ar.b1", {C}});
    s.push_back({"ar.wh", {2, C}});
    s.push_back({"ar.bh", {2}});
  }
  return s;
}

// Bound b of the uniform draw in [-b, b): Kaiming-uniform style for weights
// (sqrt(3 / fan_in) with a per-role gain), 0.05 for biases.
double init_bound(const Spec &t) {
  const std::string leaf = t.name.substr(t.name.rfind('.') + 1);
  if (leaf[0] == 'b') return 0.05;
  double fan_in = 1.0;
  for (size_t i = 1; i < t.shape.size(); ++i) fan_in *= t.shape[i];
  const double base = std::sqrt(3.0 / (fan_in > 1.0 ? fan_in : 1.0));
  const bool lift = t.name.rfind("lift.", 0) == 0 || t.name.rfind("tlift.", 0) == 0;
  if (lift) {
    if (leaf == "w1") return base * (5.0 / 3.0) / 64.0;   // inputs of order +-128
    if (leaf == "w2") return base * (5.0 / 3.0);
    return base * 0.5;                                     // residual output of order 1
  }
  if (t.name == "lstm.we" || t.name == "ar.w5" || leaf == "wa") return base * 0.25;
  if (leaf == "wh") return base * 0.1;                     // initial means near zero
  if (t.name == "lstm.wg") return base;
  return base * std::sqrt(2.0);                            // leaky-ReLU gain
}

uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Uniform in [-1, 1) from the top 53 bits of one SplitMix64 output.
double draw(uint64_t seed, uint64_t tensor, uint64_t elem) {
  const uint64_t key = splitmix64(seed ^ splitmix64(tensor + 1));
  const uint64_t r = splitmix64(key + elem);
  return (double)(r >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// Serialise a random-init model; returns PW_OK or PW_EUNSUPPORTED for a
// configuration the library does not load.
int random_blob(const pw_model_cfg &cfg, uint64_t seed, std::vector<uint8_t> &out) {
  if (cfg.levels < 1 || cfg.levels > 6 || cfg.F != 16 ||
      (cfg.C != 32 && cfg.C != 64 && cfg.C != 128) || cfg.ll_mode < 0 || cfg.ll_mode > 1) {
    set_last_error("random model: unsupported configuration (levels 1..6, F = 16, "
                   "C in {32, 64, 128}, ll_mode 0 or 1)");
    return PW_EUNSUPPORTED;
  }
  const std::vector<Spec> specs = tensor_specs((uint32_t)cfg.C, (uint32_t)cfg.F, cfg.ll_mode);
  const size_t rec_end = 32 + 64 * specs.size();
  std::vector<size_t> offs(specs.size());
  size_t off = round256(rec_end);
  for (size_t i = 0; i < specs.size(); ++i) {
    size_t cnt = 1;
    for (uint32_t d : specs[i].shape) cnt *= d;
    offs[i] = off;
    off = round256(off + 4 * cnt);
  }
  out.assign(off, 0);
  uint8_t *b = out.data();
  auto put32 = [](uint8_t *p, uint32_t v) {
    for (int k = 0; k < 4; ++k) p[k] = (uint8_t)(v >> (8 * k));   // little endian
  };
  std::memcpy(b, "PWMB", 4);
  const uint32_t head[7] = {1u, (uint32_t)cfg.levels, (uint32_t)cfg.C, (uint32_t)cfg.F,
                            (uint32_t)cfg.ll_mode, (uint32_t)specs.size(), 0u};
  for (int k = 0; k < 7; ++k) put32(b + 4 + 4 * k, head[k]);
  for (size_t i = 0; i < specs.size(); ++i) {
    const Spec &t = specs[i];
    uint8_t *r = b + 32 + 64 * i;
    std::memcpy(r, t.name.data(), t.name.size());            // NUL padded to 40
    put32(r + 40, (uint32_t)t.shape.size());
    for (int d = 0; d < 4; ++d)
      put32(r + 44 + 4 * d, d < (int)t.shape.size() ? t.shape[d] : 1u);
    put32(r + 60, (uint32_t)offs[i]);
    size_t cnt = 1;
    for (uint32_t d : t.shape) cnt *= d;
    const bool head_bias = t.name.size() > 3 && t.name.compare(t.name.size() - 3, 3, ".bh") == 0;
    const double bound = init_bound(t);
    for (size_t e = 0; e < cnt; ++e) {
      // head biases: mean 0, scale softplus^-1(1.5) (about 1.5 quantiser steps)
      const float v = head_bias ? (e == 0 ? 0.f : (float)std::log(std::expm1(1.5)))
                                : (float)(bound * draw(seed, i, e));
      uint32_t u;
      std::memcpy(&u, &v, 4);
      put32(b + offs[i] + 4 * e, u);
    }
  }
  return PW_OK;
}

}  // namespace pw

int pw_model_random_blob(const pw_model_cfg *cfg, uint64_t seed, void *buf, size_t cap,
                         size_t *n) {
  if (!cfg) { pw::set_last_error("bad arguments"); return PW_EINVAL; }
  std::vector<uint8_t> blob;
  const int s = pw::random_blob(*cfg, seed, blob);
  if (s != PW_OK) return s;
  if (n) *n = blob.size();
  if (!buf) return PW_OK;   // size query
  if (cap < blob.size()) { pw::set_last_error("random model: buffer too small"); return PW_EINVAL; }
  std::memcpy(buf, blob.data(), blob.size());
  return PW_OK;
}

int pw_model_init_random(pw_ctx *ctx, const pw_model_cfg *cfg, uint64_t seed, pw_model **out) {
  if (!ctx || !cfg || !out) { pw::set_last_error("bad arguments"); return PW_EINVAL; }
  std::vector<uint8_t> blob;
  const int s = pw::random_blob(*cfg, seed, blob);
  if (s != PW_OK) return s;
  return pw_model_load(ctx, blob.data(), blob.size(), out);
}
