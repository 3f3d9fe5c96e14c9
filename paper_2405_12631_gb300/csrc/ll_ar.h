// Autoregressive LL model (ll_ar.cu): declarations.
#pragma once
#include "ctx_kernels.cuh"

namespace pw {

struct ArWeightsDev {
  const float *w5;  // [C][25] (5x5, only the 12 causal taps are used)
  const float *b5;  // [C]
  const float *w1;  // [C][C] (out, in)
  const float *b1;  // [C]
  const float *wh;  // [2][C]
  const float *bh;  // [2]
};

int launch_ll_ar_params(const int32_t *Q, int P, int h, int w, int C, const ArWeightsDev &wd,
                        uint32_t *idx, float *mu, float *sg, cudaStream_t st);
int launch_ll_ar_decode(const DecChunk *chunks, int P, int h, int w, int C, const ArWeightsDev &wd,
                        const uint16_t *bank, int32_t *Q, uint32_t *status, cudaStream_t st);

}  // namespace pw
