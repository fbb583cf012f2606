// Square-free part in Z[x] (placeholder until the multi-modular version lands).
#include "ctx.cuh"

extern "C" int bs_squarefree_part(bs_ctx* ctx, const bs_upoly* r, bs_upoly* out) {
  if (!ctx || !r || !out) return BS_ERR_ARG;
  return ctx_fail(ctx, BS_ERR_RANGE, "square-free part: not built yet");
}
