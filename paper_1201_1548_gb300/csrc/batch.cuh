// Host-planned batches of resultants and of modular gcds, split into planning (no device
// work), launching (staging, upload, stages and download enqueued on the context's
// stream, inside a device region the caller provides) and finishing (after the stream
// has been synchronised).  The blocking entry points and the serving loop share them.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "ctx.cuh"

namespace bs {

struct HostBatch {
  int n = 0, var = 1;
  std::vector<Plan> plans;
  std::vector<int64_t> in_f, in_g;  // input limb words per job
  int needT = 1, needLog = 0, kmax = 1, lmax = 1, maxN = 1;
  int cls_count[kNumUniClasses] = {0, 0, 0, 0, 0, 0};
  int ecls_count[kNumEvalClasses] = {0, 0, 0, 0, 0, 0};
  // layout: [upload | compute | download], offsets from the region's base
  size_t o_jobs = 0, o_eoff = 0, o_ioff = 0, o_iwoff = 0, o_coff = 0;
  size_t o_cids[kNumUniClasses] = {}, o_coffs[kNumUniClasses] = {};
  size_t o_eids[kNumEvalClasses] = {}, o_eoffs[kNumEvalClasses] = {};
  size_t o_status = 0, o_pstat = 0, o_in = 0, up_bytes = 0;
  std::vector<size_t> o_ev, o_vals, o_rmod, o_sel, o_out;
  // reconstruction of many primes (k_need > kCrtWarpMaxK): weighted-sum workspace and lists
  std::vector<char> big;
  std::vector<size_t> o_wsM, o_wsY, o_wsS;
  size_t o_cbt = 0, o_cbg = 0, o_cbc = 0, o_cbf = 0;
  int kmax_big = 1, lmax_big = 1;
  size_t dn_start = 0, o_status_dn = 0, dn_bytes = 0, total = 0;
  // statistics
  int64_t instances = 0, mulmods = 0, k_need_sum = 0, k_total_sum = 0;
  int maxpts = 0, maxprimes = 0;
};

// validate and plan; computes the layout (total device bytes, upload and download bytes)
int batch_plan(bs_ctx* ctx, int n, const bs_bipoly* f, const bs_bipoly* g, int var, HostBatch* hb);
// stage the inputs in h_up (>= up_bytes), upload into dev (>= total bytes), enqueue the
// stages and the download into h_down (>= dn_bytes); the tables must already cover the
// batch (needT, needLog)
int batch_launch(bs_ctx* ctx, HostBatch& hb, const bs_bipoly* f, const bs_bipoly* g, char* dev,
                 char* h_up, char* h_down, bool use_graph);
// read the status and format the results from h_down into caller buffers
int batch_finish(bs_ctx* ctx, const HostBatch& hb, const char* h_down, bs_upoly* out);

// modular gcd batches (gcd in Z[x] and square-free parts); kind 0 gcd(a, b), kind 1
// square-free part of a (b unused).  Jobs whose result needs no device work (a zero
// input, a constant) are answered on the host ("special").
struct MgBatch {
  int n = 0;
  std::vector<int> kind, k_need, k_total, cap, out_limbs, da, db, swap;
  std::vector<int> special, special_deg, special_limbs;
  std::vector<std::vector<uint32_t>> special_out;
  std::vector<int> gen;  // indices of the jobs that run on the device
  int kmax = 1, lmax = 1, needT = 1;
  int in_limbs = 1;  // widest input coefficient
  int64_t items = 0;
  size_t smem = 0;
  int threads = 32;
  size_t o_jobs = 0, o_items = 0, o_crt = 0, o_toff = 0, o_ids1 = 0, o_ids2 = 0, o_in = 0;
  size_t up_bytes = 0;
  std::vector<size_t> o_qp, o_dg, o_sel, o_rmod, o_cont, o_cmul, o_cinv, o_h, o_info, o_out;
  size_t dn_start = 0, dn_bytes = 0, total = 0;
};

int mg_plan(bs_ctx* ctx, int n, const int* kind, const bs_upoly* a, const bs_upoly* b, MgBatch* mb);
int mg_launch(bs_ctx* ctx, MgBatch& mb, const bs_upoly* a, const bs_upoly* b, char* dev,
              char* h_up, char* h_down);
// job_status (may be null) receives each job's status; returns the first failure
int mg_finish(bs_ctx* ctx, const MgBatch& mb, const char* h_down, bs_upoly* out, int* job_status);
// upper bounds of job j's result shape
void mg_result_shape(const MgBatch& mb, int j, int* deg, int* limbs);

}  // namespace bs

int ensure_pinned(bs_ctx* ctx, size_t up, size_t down);
