// Tensor-core (tcgen05, BF16) context-model path.
#include "ctx_tc.h"

namespace pw {
int tc_workspace_alloc(Workspace *, const Geometry &, int) {
  set_last_error("BF16 path not built");
  return PW_EUNSUPPORTED;
}
void tc_workspace_free(Workspace *) {}
int tc_run_lstm(pw_ctx *, Model &, const Geometry &, Workspace &, int, const int32_t *, int,
                int, int) {
  return PW_EUNSUPPORTED;
}
int tc_run_step(pw_ctx *, Model &, const Geometry &, Workspace &, int, int, StepNetDev &,
                const int32_t *, uint32_t *, int64_t, float *, float *) {
  return PW_EUNSUPPORTED;
}
int Model::ensure_tc() { return PW_EUNSUPPORTED; }
void Model::free_tc() {}
}  // namespace pw
