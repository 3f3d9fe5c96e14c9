// Per-kernel-class timing (see prof.h).
#include "prof.h"

namespace pw {

const char *kclass_name(int c) {
  static const char *n[KC_COUNT] = {"ctx_lstm_gates_conv3x3", "ctx_conv3x3", "ctx_conv1x1",
                                    "ctx_small", "rans_decode", "rans_encode", "cdf_bank",
                                    "lift_step", "colour", "parse", "quant",
                                    "ctx_head_conv3x3", "mix_head"};
  return (c >= 0 && c < KC_COUNT) ? n[c] : "?";
}

cudaEvent_t Prof::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Prof::resolve() {
  for (auto &p : pending) {
    float t = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      launches[p.cls] += 1;
      ms[p.cls] += t;
      flops[p.cls] += p.flops;
      bytes[p.cls] += p.bytes;
    }
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
}

void Prof::reset() {
  resolve();
  for (int i = 0; i < KC_COUNT; ++i) { launches[i] = 0; ms[i] = flops[i] = bytes[i] = 0.0; }
}

Prof::~Prof() {
  for (auto &p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : pool) cudaEventDestroy(e);
}

ProfScope::ProfScope(pw_ctx *c, int k, double f, double b) : ctx(c), cls(k), flops(f), bytes(b) {
  Prof &p = prof_of(ctx);
  if (p.on && ((p.mask >> k) & 1u)) {
    a = p.get();
    cudaEventRecord(a, ctx->stream);
  }
}

ProfScope::~ProfScope() {
  if (!a) return;
  Prof &p = prof_of(ctx);
  cudaEvent_t b = p.get();
  cudaEventRecord(b, ctx->stream);
  p.pending.push_back({cls, a, b, flops, bytes});
  if (p.pending.size() > 4096) p.resolve();
}

}  // namespace pw
