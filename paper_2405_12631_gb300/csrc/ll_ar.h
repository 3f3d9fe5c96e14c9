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
  // integer-network class: the arrays hold quantised integers, iq = 1, and
  // the layers' outputs are requantised by n5 / n1 bits (head: n_mu, n_rho)
  int iq = 0, n5 = 0, n1 = 0, n_mu = 0, n_rho = 0;
};

int launch_ll_ar_params(const int32_t *Q, int P, int h, int w, int C, const ArWeightsDev &wd,
                        uint32_t *idx, float *mu, float *sg, cudaStream_t st);
// ext / esh: ragged batches (every plane's own LL extent, see the kernel)
int launch_ll_ar_decode(const DecChunk *chunks, int P, int h, int w, int C, const ArWeightsDev &wd,
                        const uint16_t *bank, int32_t *Q, uint32_t *status, cudaStream_t st,
                        const int2 *ext = nullptr, int esh = 0);

}  // namespace pw
