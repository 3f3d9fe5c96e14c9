// Optional per-kernel-class timing with CUDA events on the context's stream.
#pragma once
#include <string>
#include <vector>

#include "codec.h"

namespace pw {

enum KClass {
  KC_LSTM_GATES = 0, KC_CONV3, KC_CONV1, KC_SMALL_CTX, KC_RANS_DEC, KC_RANS_ENC, KC_CDF,
  KC_LIFT, KC_COLOUR, KC_PARSE, KC_QUANT,
  KC_HEAD3,  // steps 2-4 second residual conv fused with the head (3x3)
  KC_MIX,    // logistic-mixture head, decision and per-symbol tables
  KC_COUNT
};
const char *kclass_name(int c);

struct Prof {
  bool on = false;
  uint32_t mask = ~0u;   // classes recorded while on (bit = KClass)
  struct Pending {
    int cls;
    cudaEvent_t a, b;
    double flops, bytes;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  uint64_t launches[KC_COUNT] = {};
  double ms[KC_COUNT] = {}, flops[KC_COUNT] = {}, bytes[KC_COUNT] = {};
  cudaEvent_t get();
  void resolve();
  void reset();
  ~Prof();
};

// Records events around the launches issued during its lifetime when the
// context's profiling is on.
struct ProfScope {
  pw_ctx *ctx;
  int cls;
  double flops, bytes;
  cudaEvent_t a = nullptr;
  ProfScope(pw_ctx *c, int k, double f, double b);
  ~ProfScope();
};

Prof &prof_of(pw_ctx *ctx);

}  // namespace pw
