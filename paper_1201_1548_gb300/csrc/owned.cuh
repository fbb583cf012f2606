// Host-side helpers for pipelines composed of the library's own entry points: an integer
// polynomial held in a host buffer, and the two-call pattern (size query, then the
// computation) of the entry points that write a caller-owned bs_upoly.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "ctx.cuh"

namespace bs {

struct HostPoly {
  std::vector<uint32_t> c;
  bs_upoly u{-1, 1, nullptr};
};

// call a bs_upoly-producing entry point twice: size query, then the computation
template <class F>
static int fetch(HostPoly* h, F&& call) {
  h->u = bs_upoly{0, 0, nullptr};
  int rc = call(&h->u);
  if (rc) return rc;
  h->c.assign((size_t)(std::max(h->u.deg, 0) + 1) * std::max(h->u.limbs, 1), 0u);
  h->u.limbs = std::max(h->u.limbs, 1);
  h->u.deg = std::max(h->u.deg, 0);
  h->u.c = h->c.data();
  return call(&h->u);
}

// bs_modgcd_batch with owned outputs: a size query, then the computation
static inline int modgcd_owned(bs_ctx* ctx, const std::vector<int>& kind, const std::vector<bs_upoly>& a,
                               const std::vector<bs_upoly>& b, std::vector<HostPoly>* out) {
  const int n = (int)kind.size();
  out->assign(n, HostPoly{});
  std::vector<bs_upoly> o(n, bs_upoly{0, 0, nullptr});
  int rc = bs_modgcd_batch(ctx, n, kind.data(), a.data(), b.empty() ? nullptr : b.data(), o.data());
  if (rc) return rc;
  for (int j = 0; j < n; ++j) {
    HostPoly& p = (*out)[j];
    p.c.assign((size_t)(std::max(o[j].deg, 0) + 1) * std::max(o[j].limbs, 1), 0u);
    o[j].deg = std::max(o[j].deg, 0);
    o[j].limbs = std::max(o[j].limbs, 1);
    o[j].c = p.c.data();
  }
  rc = bs_modgcd_batch(ctx, n, kind.data(), a.data(), b.empty() ? nullptr : b.data(), o.data());
  if (rc) return rc;
  for (int j = 0; j < n; ++j) (*out)[j].u = o[j];
  return BS_OK;
}

}  // namespace bs
