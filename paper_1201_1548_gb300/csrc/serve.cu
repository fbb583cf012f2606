// Serving loop: continuous batching of resultant and gcd jobs on one GPU.
//
// Jobs are submitted from any host thread and queued with copies of their inputs.  A
// fixed number of slot threads, each with its own CUDA stream and executable graph,
// take work from the queue: a slot forms a batch from the queued jobs of one type and
// one work class (first come first served, up to a job limit), reserves device memory
// for it in the server's arena (admission: the batch waits while the arena cannot hold
// it), launches it, waits for its stream, posts the results and frees the memory.  Slots
// run concurrently, so a batch admitted while others are on the GPU overlaps with them.
// All slots share the context's prime tables; a slot that needs larger tables waits
// until no batch is in flight before growing them.
//
// Work classes keep small jobs from waiting behind large ones: a resultant is large when
// its plan counts more than kLargeWork multiply-reduce operations (the univariate
// eliminations of all its (prime, point) images), tiny when it counts at most kTinyWork,
// small otherwise, and a batch never mixes classes, since every job of a batch finishes
// when the batch does.  With two or more slots the last half of them (at least one) take
// tiny and small jobs only, so those find a slot even while the others run large
// batches.  Every slot launches small batches on a stream of the highest
// priority and large batches on one of the lowest, and a large batch's grids are sized by
// its work (short blocks) instead of persistent blocks on every SM: the block scheduler
// then starts the blocks of a small batch as soon as blocks of the large kernel end, and
// a large batch alone still has the whole GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <shared_mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "ctx.cuh"

namespace bs {

// first-fit allocator over [0, size) with coalescing free blocks (256-byte granules)
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    size_ = size & ~(size_t)255;
    if (size_) free_[0] = size_;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t start = it->first + bytes;
      free_.erase(it);
      if (rest) free_[start] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t largest_free() const {
    size_t m = 0;
    for (const auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0, peak_ = 0;
};

using Clock = std::chrono::steady_clock;

struct Ticket {
  int kind = 0;  // BS_JOB_*
  int var = 1;
  // resultant inputs
  bs_bipoly f{}, g{};
  std::vector<uint32_t> fc, gc;
  // gcd / square-free inputs
  bs_upoly a{}, b{};
  std::vector<uint32_t> ac, bc;
  size_t bytes = 0;  // device bytes of the job as a batch of one (admission estimate)
  int large = 0;     // 1: more than kLargeWork operations
  int work = 0;      // work class: 0 up to kTinyWork operations, 1 up to kLargeWork, 2 above
  int state = 0;     // 0 queued, 1 running, 2 done
  int status = 0;
  int deg = -1, limbs = 1;
  std::vector<uint32_t> out;
  Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace bs

struct bs_server {
  bs_ctx* parent = nullptr;
  int max_batch = 64;
  char* arena_base = nullptr;
  bs::Arena arena;
  std::vector<bs_ctx*> slots;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, bs::Ticket> tickets;
  std::shared_mutex tables_mu;
  bool stop = false;
  uint64_t next_ticket = 1;
  // statistics
  int64_t submitted = 0, completed = 0, batches = 0, jobs_in_batches = 0;
  int inflight = 0, max_inflight = 0;
  double phase_ms[3] = {0, 0, 0};  // host planning, device (launch to stream idle), formatting
};

namespace bs {

static int job_type(const Ticket& t) { return t.kind == BS_JOB_RESULTANT ? (t.var ? 1 : 0) : 2; }

// jobs of one batch: the same type and the same work class
static int batch_class(const Ticket& t) { return job_type(t) * 3 + t.work; }

// work of a large job: about a millisecond of the GPU's multiply pipe
constexpr double kLargeWork = 2e9;
// work of a tiny job (a tenth of that): tiny jobs are not batched with larger small ones,
// whose batch would hold them back
constexpr double kTinyWork = 2e8;
// pinned staging of a slot allocated at start (each way)
constexpr size_t kSlotPinnedBytes = size_t(64) << 20;

// device bytes reserved for a batch: the jobs' bytes as batches of one bound the batch's
// layout (a batch shares its headers); the slack covers alignment
constexpr size_t kBatchSlack = 64 * 1024;

static size_t jobs_bytes(const std::vector<Ticket*>& jobs) {
  size_t s = kBatchSlack;
  for (const Ticket* t : jobs) s += t->bytes;
  return s;
}

// the slot context: two streams (small batches at the highest priority, large ones at
// the lowest), status word and graph; the parent's tables
static int make_slot(bs_ctx* parent, bs_ctx** out) {
  bs_ctx* c = new bs_ctx();
  c->device = parent->device;
  c->sms = parent->sms;
  c->smem_optin = parent->smem_optin;
  c->budget = parent->budget;
  c->tabs = parent->tabs;
  c->parent = parent;
  for (int i = 0; i < kNumUniClasses; ++i)
    for (int t = 0; t < 3; ++t) c->occ[i][t] = parent->occ[i][t];
  c->tune = parent->tune;
  int lo = 0, hi = 0;  // numerically lower is higher priority
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (cudaStreamCreateWithPriority(&c->own_stream, cudaStreamNonBlocking, hi) != cudaSuccess) {
    delete c;
    return BS_ERR_CUDA;
  }
  if (cudaStreamCreateWithPriority(&c->aux_stream, cudaStreamNonBlocking, lo) != cudaSuccess) {
    cudaStreamDestroy(c->own_stream);
    delete c;
    return BS_ERR_CUDA;
  }
  c->stream = c->own_stream;
  // pinned staging sized up front: a later growth waits for the whole device (cudaFreeHost,
  // cudaMallocHost), i.e. for the longest batch in flight on the other slots
  if (ensure_pinned(c, kSlotPinnedBytes, kSlotPinnedBytes) != 0) {
    if (c->h_up) cudaFreeHost(c->h_up);
    if (c->h_down) cudaFreeHost(c->h_down);
    cudaStreamDestroy(c->own_stream);
    cudaStreamDestroy(c->aux_stream);
    delete c;
    return BS_ERR_NOMEM;
  }
  if (cudaMalloc(&c->d_status, sizeof(int32_t) * 4) != cudaSuccess) {
    cudaStreamDestroy(c->own_stream);
    cudaStreamDestroy(c->aux_stream);
    delete c;
    return BS_ERR_CUDA;
  }
  cudaMemset(c->d_status, 0, sizeof(int32_t) * 4);
  *out = c;
  return 0;
}

static double ms_since(Clock::time_point& t0) {
  const auto t1 = Clock::now();
  const double ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  t0 = t1;
  return ms;
}

// run one batch of tickets (all of one type) on slot context c, inside dev; fills the
// tickets' results (called without the server lock) and adds the wall time of its host
// planning, device work and result formatting to ph[0..2]
static void run_batch(bs_server* S, bs_ctx* c, std::vector<Ticket*>& jobs, char* dev, double* ph) {
  NvtxScope nv(jobs[0]->large ? "bs.serve.large_batch" : "bs.serve.batch");
  auto t0 = Clock::now();
  const int n = (int)jobs.size();
  const int type = job_type(*jobs[0]);
  // a large batch: low priority, short blocks (small batches' blocks start between them)
  c->stream = jobs[0]->large ? c->aux_stream : c->own_stream;
  c->fine_grids = jobs[0]->large != 0;
  int rc = 0;
  std::vector<bs_upoly> outs(n);
  auto fail_all = [&](int code) {
    for (Ticket* t : jobs) {
      t->status = code;
      t->deg = -1;
      t->out.clear();
    }
  };
  if (type <= 1) {
    std::vector<bs_bipoly> f(n), g(n);
    for (int i = 0; i < n; ++i) {
      f[i] = jobs[i]->f;
      g[i] = jobs[i]->g;
    }
    HostBatch B;
    rc = batch_plan(c, n, f.data(), g.data(), type, &B);
    if (!rc && B.total > jobs_bytes(jobs)) rc = BS_ERR_INTERNAL;
    if (rc) return fail_all(rc);
    ph[0] += ms_since(t0);
    {
      std::shared_lock<std::shared_mutex> lk(S->tables_mu, std::defer_lock);
      for (;;) {
        lk.lock();
        if (c->tabs->Tt >= B.needT && c->tabs->Tg >= B.needT && c->tabs->logNT >= B.needLog) break;
        lk.unlock();
        std::unique_lock<std::shared_mutex> ulk(S->tables_mu);
        rc = c->tabs->ensure(B.needT, B.needLog, S->parent->stream);
        if (rc) return fail_all(rc);
      }
      rc = ensure_pinned(c, B.up_bytes, B.dn_bytes);
      if (!rc) rc = batch_launch(c, B, f.data(), g.data(), dev, (char*)c->h_up, (char*)c->h_down, true);
      if (!rc) rc = ctx_cuda(c, cudaStreamSynchronize(c->stream), "stream");
    }
    ph[1] += ms_since(t0);
    if (rc) return fail_all(rc);
    for (int i = 0; i < n; ++i) {
      const Plan& P = B.plans[i];
      jobs[i]->limbs = P.out_limbs;
      jobs[i]->out.assign((size_t)(std::max(P.D, 0) + 1) * P.out_limbs, 0u);
      outs[i] = bs_upoly{std::max(P.D, 0), P.out_limbs, jobs[i]->out.data()};
    }
    rc = batch_finish(c, B, (const char*)c->h_down, outs.data());
    ph[2] += ms_since(t0);
    if (rc) return fail_all(rc);
    for (int i = 0; i < n; ++i) {
      jobs[i]->status = 0;
      jobs[i]->deg = outs[i].deg;
    }
    return;
  }
  std::vector<int> kind(n);
  std::vector<bs_upoly> a(n), b(n);
  for (int i = 0; i < n; ++i) {
    kind[i] = jobs[i]->kind == BS_JOB_GCD ? 0 : 1;
    a[i] = jobs[i]->a;
    b[i] = jobs[i]->b;
  }
  MgBatch B;
  rc = mg_plan(c, n, kind.data(), a.data(), b.data(), &B);
  if (!rc && B.total > jobs_bytes(jobs)) rc = BS_ERR_INTERNAL;
  if (rc) return fail_all(rc);
  ph[0] += ms_since(t0);
  {
    std::shared_lock<std::shared_mutex> lk(S->tables_mu, std::defer_lock);
    for (;;) {
      lk.lock();
      if (c->tabs->Tt >= B.needT && c->tabs->Tg >= B.needT) break;
      lk.unlock();
      std::unique_lock<std::shared_mutex> ulk(S->tables_mu);
      rc = c->tabs->ensure(B.needT, 0, S->parent->stream);
      if (rc) return fail_all(rc);
    }
    rc = ensure_pinned(c, B.up_bytes, B.dn_bytes);
    if (!rc) rc = mg_launch(c, B, a.data(), b.data(), dev, (char*)c->h_up, (char*)c->h_down);
    if (!rc) rc = ctx_cuda(c, cudaStreamSynchronize(c->stream), "stream");
  }
  ph[1] += ms_since(t0);
  if (rc) return fail_all(rc);
  for (int i = 0; i < n; ++i) {
    int d, l;
    mg_result_shape(B, i, &d, &l);
    jobs[i]->limbs = l;
    jobs[i]->out.assign((size_t)(std::max(d, 0) + 1) * l, 0u);
    outs[i] = bs_upoly{std::max(d, 0), l, jobs[i]->out.data()};
  }
  std::vector<int> st(n, 0);
  mg_finish(c, B, (const char*)c->h_down, outs.data(), st.data());
  ph[2] += ms_since(t0);
  for (int i = 0; i < n; ++i) {
    jobs[i]->status = st[i];
    jobs[i]->deg = st[i] ? -1 : outs[i].deg;
  }
}

static void slot_main(bs_server* S, int slot) {
  bs_ctx* c = S->slots[slot];
  cudaSetDevice(c->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    // form a batch: the head job's type, then later jobs of the same type, while the
    // arena can hold them
    std::vector<uint64_t> ids;
    std::vector<Ticket*> jobs;
    size_t off = 0, bytes = 0;
    // the last half of the slots (at least one of two or more) take no large jobs
    const int ns = (int)S->slots.size();
    const bool small_only = ns >= 2 && slot >= ns - std::max(1, ns / 2);
    for (;;) {
      if (S->stop && S->queue.empty()) return;
      // the head: the oldest queued job (the oldest small one for the small-job slot)
      size_t h = 0;
      if (small_only)
        while (h < S->queue.size() && S->tickets[S->queue[h]].large) ++h;
      if (h < S->queue.size()) {
        Ticket& head = S->tickets[S->queue[h]];
        const int type = batch_class(head);
        size_t sum = kBatchSlack;
        std::vector<size_t> pos;
        for (size_t q = h; q < S->queue.size() && (int)pos.size() < S->max_batch; ++q) {
          Ticket& t = S->tickets[S->queue[q]];
          if (batch_class(t) != type) continue;
          if (!pos.empty() && sum + t.bytes > S->arena.largest_free()) break;
          sum += t.bytes;
          pos.push_back(q);
        }
        if (S->arena.alloc(sum, &off)) {
          bytes = sum;
          for (size_t k = pos.size(); k-- > 0;) {
            const uint64_t id = S->queue[pos[k]];
            S->queue.erase(S->queue.begin() + (std::ptrdiff_t)pos[k]);
            ids.insert(ids.begin(), id);
          }
          break;
        }
      }
      S->cv_work.wait(lk);  // new work or freed memory
    }
    const auto now = Clock::now();
    for (uint64_t id : ids) {
      Ticket& t = S->tickets[id];
      t.state = 1;
      t.t_admit = now;
      jobs.push_back(&t);
    }
    ++S->batches;
    S->jobs_in_batches += (int64_t)jobs.size();
    ++S->inflight;
    S->max_inflight = std::max(S->max_inflight, S->inflight);
    lk.unlock();
    double ph[3] = {0, 0, 0};
    run_batch(S, c, jobs, S->arena_base + off, ph);
    lk.lock();
    for (int i = 0; i < 3; ++i) S->phase_ms[i] += ph[i];
    --S->inflight;
    S->arena.release(off, bytes);
    const auto done = Clock::now();
    for (Ticket* t : jobs) {
      t->state = 2;
      t->t_done = done;
      ++S->completed;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace bs

using namespace bs;

extern "C" int bs_serve_start(bs_ctx* ctx, int slots, int max_batch, size_t arena_bytes) {
  if (!ctx || ctx->parent) return BS_ERR_ARG;
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "serving loop already running");
  if (slots < 1 || slots > 16 || max_batch < 1) return ctx_fail(ctx, BS_ERR_ARG, "bad slot or batch count");
  cudaSetDevice(ctx->device);
  if (arena_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    arena_bytes = std::min(ctx->budget, fr / 2);
  }
  if (arena_bytes > ctx->budget) return ctx_fail(ctx, BS_ERR_NOMEM, "arena above the memory budget");
  bs_server* S = new bs_server();
  S->parent = ctx;
  S->max_batch = max_batch;
  if (cudaMalloc(&S->arena_base, arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return ctx_fail(ctx, BS_ERR_NOMEM, "cudaMalloc of the serving arena failed");
  }
  S->arena.reset(arena_bytes);
  for (int i = 0; i < slots; ++i) {
    bs_ctx* c = nullptr;
    if (make_slot(ctx, &c) != 0) {
      for (bs_ctx* d : S->slots) bs_free(d);
      cudaFree(S->arena_base);
      delete S;
      return ctx_fail(ctx, BS_ERR_CUDA, "slot stream creation failed");
    }
    S->slots.push_back(c);
  }
  ctx->server = S;
  for (int i = 0; i < slots; ++i) S->threads.emplace_back(slot_main, S, i);
  return BS_OK;
}

extern "C" int bs_serve_stop(bs_ctx* ctx) {
  if (!ctx) return BS_ERR_ARG;
  bs_server* S = ctx->server;
  if (!S) return BS_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->threads) t.join();
  for (bs_ctx* c : S->slots) bs_free(c);
  cudaFree(S->arena_base);
  ctx->server = nullptr;
  delete S;
  return BS_OK;
}

static int copy_upoly(const bs_upoly* u, bs_upoly* dst, std::vector<uint32_t>* store) {
  if (!u || u->deg < -1 || u->limbs < 1 || u->limbs > kMaxUniLimbs || (u->deg >= 0 && !u->c)) return 1;
  store->assign(u->c, u->c + (size_t)(u->deg + 1) * u->limbs);
  *dst = bs_upoly{u->deg, u->limbs, store->data()};
  return 0;
}

extern "C" int bs_submit(bs_ctx* ctx, const bs_job* job, uint64_t* ticket) {
  if (!ctx || !job || !ticket) return BS_ERR_ARG;
  bs_server* S = ctx->server;
  if (!S) return ctx_fail(ctx, BS_ERR_ARG, "no serving loop (bs_serve_start)");
  Ticket t;
  t.kind = job->kind;
  t.var = job->var;
  if (job->kind == BS_JOB_RESULTANT) {
    if (job->var != 0 && job->var != 1) return ctx_fail(ctx, BS_ERR_ARG, "bad var");
    for (int w = 0; w < 2; ++w) {
      const bs_bipoly& p = w ? job->g : job->f;
      if (p.deg_x < 0 || p.deg_y < 0 || p.limbs < 1 || p.limbs > kMaxLimbs || !p.c)
        return ctx_fail(ctx, BS_ERR_ARG, "bad bivariate operand");
      std::vector<uint32_t>& st = w ? t.gc : t.fc;
      st.assign(p.c, p.c + (size_t)(p.deg_x + 1) * (p.deg_y + 1) * p.limbs);
      (w ? t.g : t.f) = bs_bipoly{p.deg_x, p.deg_y, p.limbs, st.data()};
    }
    HostBatch B;  // plan as a batch of one: validation, admission estimate, work class
    const int rc = batch_plan(ctx, 1, &t.f, &t.g, t.var, &B);
    if (rc) return rc;
    t.bytes = B.total;
    t.large = (double)B.mulmods > kLargeWork;
    t.work = t.large ? 2 : (double)B.mulmods > kTinyWork ? 1 : 0;
  } else if (job->kind == BS_JOB_GCD || job->kind == BS_JOB_SQFREE) {
    if (copy_upoly(&job->a, &t.a, &t.ac)) return ctx_fail(ctx, BS_ERR_ARG, "bad operand a");
    if (job->kind == BS_JOB_GCD) {
      if (copy_upoly(&job->b, &t.b, &t.bc)) return ctx_fail(ctx, BS_ERR_ARG, "bad operand b");
    } else {
      t.b = bs_upoly{-1, 1, nullptr};
    }
    MgBatch B;
    const int kd = job->kind == BS_JOB_GCD ? 0 : 1;
    const int rc = mg_plan(ctx, 1, &kd, &t.a, &t.b, &B);
    if (rc) return rc;
    t.bytes = B.total;
  } else {
    return ctx_fail(ctx, BS_ERR_ARG, "unknown job kind");
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (t.bytes + kBatchSlack > S->arena.size())
    return ctx_fail(ctx, BS_ERR_NOMEM, "job needs more device memory than the serving arena holds");
  if (S->stop) return ctx_fail(ctx, BS_ERR_ARG, "serving loop is stopping");
  const uint64_t id = S->next_ticket++;
  t.t_submit = Clock::now();
  // vectors keep their heap buffers when moved, so the operand pointers stay valid
  S->tickets.emplace(id, std::move(t));
  S->queue.push_back(id);
  ++S->submitted;
  *ticket = id;
  S->cv_work.notify_all();  // the small-job slot must not absorb the wake-up of a large job
  return BS_OK;
}

static void fill_result(const Ticket& t, bs_result* r) {
  r->status = t.status;
  r->deg = t.deg;
  r->limbs = t.limbs;
  auto ms = [](Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
  };
  r->queue_ms = ms(t.t_submit, t.t_admit);
  r->latency_ms = ms(t.t_submit, t.t_done);
}

extern "C" int bs_poll(bs_ctx* ctx, uint64_t ticket, bs_result* r) {
  if (!ctx || !r) return BS_ERR_ARG;
  bs_server* S = ctx->server;
  if (!S) return ctx_fail(ctx, BS_ERR_ARG, "no serving loop (bs_serve_start)");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return ctx_fail(ctx, BS_ERR_ARG, "unknown ticket");
  const Ticket& t = it->second;
  if (t.state != 2) return BS_PENDING;
  fill_result(t, r);
  if (!r->c) return BS_OK;
  const size_t words = (size_t)(t.deg + 1) * t.limbs;
  if (r->cap_words < (int64_t)words) return ctx_fail(ctx, BS_ERR_CAPACITY, "result buffer too small");
  if (words) std::memcpy(r->c, t.out.data(), words * sizeof(uint32_t));
  S->tickets.erase(it);
  return BS_OK;
}

extern "C" int bs_wait(bs_ctx* ctx, uint64_t ticket, int timeout_ms) {
  if (!ctx) return BS_ERR_ARG;
  bs_server* S = ctx->server;
  if (!S) return ctx_fail(ctx, BS_ERR_ARG, "no serving loop (bs_serve_start)");
  std::unique_lock<std::mutex> lk(S->mu);
  auto ready = [&] {
    auto it = S->tickets.find(ticket);
    return it == S->tickets.end() || it->second.state == 2;
  };
  if (timeout_ms < 0) {
    S->cv_done.wait(lk, ready);
    return BS_OK;
  }
  return S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready) ? BS_OK : BS_ERR_TIMEOUT;
}

extern "C" int bs_serve_stats(bs_ctx* ctx, bs_serve_info* out) {
  if (!ctx || !out) return BS_ERR_ARG;
  bs_server* S = ctx->server;
  if (!S) return ctx_fail(ctx, BS_ERR_ARG, "no serving loop (bs_serve_start)");
  std::lock_guard<std::mutex> lk(S->mu);
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->batches = S->batches;
  out->jobs_in_batches = S->jobs_in_batches;
  out->queued = (int64_t)S->queue.size();
  out->inflight = S->inflight;
  out->max_inflight = S->max_inflight;
  out->arena_bytes = (int64_t)S->arena.size();
  out->arena_used = (int64_t)S->arena.used();
  out->arena_peak = (int64_t)S->arena.peak();
  out->host_plan_ms = S->phase_ms[0];
  out->device_ms = S->phase_ms[1];
  out->host_finish_ms = S->phase_ms[2];
  return BS_OK;
}
