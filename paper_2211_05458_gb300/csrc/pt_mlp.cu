// pt_mlp.cu -- learned Newton start: training pairs, FP32 training kernels,
// BF16 export (no counterpart in the paper).
#include <cuda_runtime.h>

#include <cstring>

#include "pt_ctx.h"
#include "pt_internal.h"

struct pt_mlp_state {
  int dummy;
};

DevMLP pt_dev_mlp(const pt_ctx* c) {
  DevMLP m;
  std::memset(&m, 0, sizeof m);
  (void)c;
  return m;
}

void pt_mlp_release(pt_ctx* c) {
  delete c->mlp;
  c->mlp = nullptr;
}

static pt_status notyet(pt_ctx* c) {
  if (c) c->err = "learned guess: not available in this build";
  return PT_ERR_STATE;
}

extern "C" {
int32_t pt_mlp_nparams(void) { return PT_MLP_NP; }
pt_status pt_mlp_make_pairs(pt_ctx* c, int64_t, uint64_t, float*, float*) { return notyet(c); }
pt_status pt_mlp_train(pt_ctx* c, int64_t, const float*, const float*, int32_t, int32_t, float,
                       uint64_t, float*) {
  return notyet(c);
}
pt_status pt_mlp_features(pt_ctx* c, int64_t, const double*, const int32_t*, float*) {
  return notyet(c);
}
pt_status pt_mlp_set(pt_ctx* c, const float*, const float*) { return notyet(c); }
pt_status pt_mlp_get(pt_ctx* c, float*, float*) { return notyet(c); }
pt_status pt_mlp_forward(pt_ctx* c, int32_t, const float*, float*) { return notyet(c); }
pt_status pt_mlp_grad(pt_ctx* c, int32_t, const float*, const float*, float*, float*) {
  return notyet(c);
}
pt_status pt_push_batch(pt_ctx* const* ctxs, const pt_particles*, int32_t, int32_t, double,
                        pt_stats*) {
  return notyet(ctxs ? ctxs[0] : nullptr);
}
}
