// Tensor-core (tcgen05, BF16 / FP8) context-model path: declarations.
#pragma once
#include "codec.h"

namespace pw {
// f8: also the E4M3 activation buffers of the FP8 precision
int tc_workspace_alloc(Workspace *ws, const Geometry &g, int C, bool f8);
// Device bytes tc_workspace_alloc takes for P planes of geometry g.
int64_t tc_workspace_bytes(const Geometry &g, int P, int C, bool f8);
void tc_workspace_free(Workspace *ws);
int tc_run_lstm(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws, int sb,
                const int32_t *sprev, int up, int first, int cur);
int tc_run_step(pw_ctx *ctx, Model &m, const Geometry &g, Workspace &ws, int sb, int step,
                StepNetDev &n, const int32_t *Qi, uint32_t *idx, int64_t nk, float *mu,
                float *sg);
// Non-zero when a tensor-core kernel hit a bounded-wait expiry since the last
// reset (reads the workspace's device error word; synchronous).
int tc_error(Workspace &ws);
void tc_error_reset(Workspace &ws, cudaStream_t st);
int tc_conv_host(pw_ctx *ctx, int P, int H, int W, int cin, int cout, int ks, int act,
                 const float *x, const float *w, const float *b, float *y);
// Autotuner of the tensor-core convolutions (ctx_tc.cu): enable / disable
// (returns the previous setting) and a text report of the tuned classes.
int tune_set_enabled(int on);
// Count of convolution launches so far whose class was still being tuned
// (sampled, or waiting for its samples to be read back; read-backs are
// polled first). A pass chain during which it did not change used final
// schedules only, so it can be captured into a CUDA graph.
uint64_t tune_untuned_uses();
std::string tune_report();
}  // namespace pw
