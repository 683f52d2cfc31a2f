// Serving: a persistent request loop around pc_extract.
//
// Requests (network + box) arrive at any time through pc_server_submit.  A
// request whose estimated device memory exceeds the per-request limit is
// rejected at once (PC_ERR_TOO_LARGE); the others wait in a FIFO queue.  Each
// of max_slots worker threads owns one extraction context and one CUDA
// stream; a free worker admits the request at the head of the queue as soon
// as the sum of the running requests' estimates plus its own fits the memory
// budget, runs the extraction on its stream (the context keeps the growing
// vertex, edge and sign-vector arrays on the device and grows them on
// overflow), and records the result.  Requests that arrive while others run
// are admitted as slots and memory free up, and their kernels overlap on the
// device.  With max_slots = 1 the same code is the plain per-request path
// (FIFO, one request at a time, the same kernels).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pc.h"

// Frees a context's extraction buffers (pc_core.cu); the next extraction
// allocates them again.
void pc_release_buffers(pc_ctx* c);

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  int L = 0;
  std::vector<int32_t> widths;
  std::vector<double> params, lo, hi;
  pc_result res{};
  bool done = false;
  std::vector<double> X;
  std::vector<int32_t> E;
  std::vector<uint64_t> SIG;
  int S = 0;
  std::string err;
};

}  // namespace

// Device bytes a slot's context may keep between requests.
constexpr int64_t kTrimBytes = int64_t(8) << 30;

struct pc_server {
  int device = 0;
  pc_server_options opt{};
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, std::unique_ptr<Request>> all;
  uint64_t next_id = 1;
  int64_t in_use = 0, peak_in_use = 0;
  int running = 0, pending = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<pc_ctx*> ctxs;              // one extraction context per slot
  std::vector<cudaStream_t> streams;      // one stream per slot

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void worker(int slot);
};

void pc_server::worker(int slot) {
  cudaSetDevice(device);
  cudaStream_t stream = streams[slot];
  pc_ctx* ctx = ctxs[slot];
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] {
        if (stop) return true;
        if (queue.empty()) return false;
        const int64_t est = queue.front()->res.est_bytes;
        return running == 0 || in_use + est <= opt.mem_budget_bytes;
      });
      if (stop && queue.empty()) break;
      if (stop) break;
      r = queue.front();
      queue.pop_front();
      in_use += r->res.est_bytes;
      peak_in_use = std::max(peak_in_use, in_use);
      ++running;
      r->res.start_s = now();
      r->res.slot = slot;
    }
    pc_status st = ctx ? pc_extract(ctx, r->L, r->widths.data(), r->params.data(), r->lo.data(), r->hi.data(),
                                     stream)
                       : PC_ERR_CUDA;
    if (st == PC_OK) {
      int64_t nv = 0, ne = 0;
      int32_t sw = 0, dim = 0, nent = 0;
      pc_counts(ctx, &nv, &ne, &sw, &dim, &nent);
      r->res.n_vertices = nv;
      r->res.n_edges = ne;
      int64_t d[10] = {0};
      pc_diagnostics(ctx, d, 10);
      r->res.held_bytes = d[8];
      if (opt.keep_outputs) {
        r->X.resize(size_t(dim) * nv);
        r->E.resize(size_t(2) * ne);
        r->SIG.resize(size_t(sw) * nv);
        r->S = sw;
        pc_vertices(ctx, nullptr, nullptr, r->X.data());
        pc_edges(ctx, nullptr, nullptr, r->E.data());
        pc_signvectors(ctx, nullptr, nullptr, r->SIG.data());
      }
    }
    if (st != PC_OK) r->err = ctx ? pc_last_error(ctx) : "context creation failed";
    // a slot that grew large for this request gives its buffers back, so
    // that idle slots do not hold memory the admission budget does not see
    if (ctx) {
      int64_t d[10] = {0};
      pc_diagnostics(ctx, d, 10);
      if (d[8] > kTrimBytes) pc_release_buffers(ctx);
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      r->res.status = st;
      r->res.finish_s = now();
      r->done = true;
      in_use -= r->res.est_bytes;
      --running;
      --pending;
    }
    cv_work.notify_all();
    cv_done.notify_all();
  }
}

extern "C" {

int64_t pc_estimate_bytes(int L, const int32_t* widths) {
  if (L < 1 || !widths) return -1;
  const int D = widths[0];
  double N = 0.0;
  int hmax = 0;
  for (int l = 1; l <= L; ++l) {
    N += widths[l];
    hmax = std::max(hmax, int(widths[l]));
  }
  // vertices ~ 1.2 N^D / D! for generic random ReLU nets (1.2 covers the
  // measured 0.4 - 1.2); edges ~ D V; sign words S = (2D + N + 31) / 32
  double fact = 1.0;
  for (int k = 2; k <= D; ++k) fact *= k;
  const double V = 1.2 * std::pow(N, D) / fact + double(1 << D);
  const double E = D * V + double(D << (D - 1));
  const double S = std::ceil((2.0 * D + N) / 32.0);
  // per vertex: coordinates, two value buffers (float), error estimates, signs;
  // per edge: endpoints, two 16-byte splitting-edge lists, the pairing record
  // and two flag bits; two hash tables of about E / 2 16-byte slots each
  const double bytes = V * (8.0 * D + 2 * 4.0 * hmax + 8 + 8.0 * S) + E * (8 + 32 + 16 + 0.25) + 16.0 * E;
  // capacity growth doubles buffers: budget for the worst case of 2x
  const double total = 2.0 * bytes + 64.0 * 1024 * 1024;
  return total > 9.0e18 ? INT64_MAX : int64_t(total);
}

void pc_server_default_options(pc_server_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_slots = 8;
  o->precision = PC_PREC_MIXED;
  o->exec = PC_EXEC_STEPWISE;
  o->polish = 0;
  o->mem_budget_bytes = int64_t(160) << 30;
  o->request_max_bytes = int64_t(64) << 30;
}

pc_status pc_server_create(pc_server** out, int device, const pc_server_options* opt) {
  if (!out) return PC_ERR_INVALID;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return PC_ERR_CUDA;
  }
  pc_server* s = new pc_server();
  s->device = device;
  pc_server_default_options(&s->opt);
  if (opt) s->opt = *opt;
  if (s->opt.max_slots < 1 || s->opt.max_slots > 64) {
    delete s;
    return PC_ERR_INVALID;
  }
  // contexts and streams are created here, before any worker runs
  cudaSetDevice(device);
  pc_options o;
  pc_default_options(&o);
  o.precision = s->opt.precision;
  o.exec = s->opt.exec;
  o.polish = s->opt.polish;
  for (int k = 0; k < s->opt.max_slots; ++k) {
    pc_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    const pc_status cs = pc_create(&ctx, device, &o);
    if (cs != PC_OK || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      if (ctx) pc_destroy(ctx);
      for (auto* c : s->ctxs) pc_destroy(c);
      for (auto q : s->streams) cudaStreamDestroy(q);
      delete s;
      return PC_ERR_CUDA;
    }
    s->ctxs.push_back(ctx);
    s->streams.push_back(st);
  }
  s->t0 = Clock::now();
  for (int k = 0; k < s->opt.max_slots; ++k) s->workers.emplace_back([s, k] { s->worker(k); });
  *out = s;
  return PC_OK;
}

pc_status pc_server_submit(pc_server* s, int L, const int32_t* widths, const double* params, const double* lo,
                           const double* hi, uint64_t* id) {
  if (!s || !widths || !params || !lo || !hi || !id || L < 1) return PC_ERR_INVALID;
  auto r = std::make_unique<Request>();
  r->L = L;
  r->widths.assign(widths, widths + L + 1);
  size_t np = 0;
  for (int l = 0; l < L; ++l) np += size_t(widths[l + 1]) * (widths[l] + 1);
  r->params.assign(params, params + np);
  r->lo.assign(lo, lo + widths[0]);
  r->hi.assign(hi, hi + widths[0]);
  r->res.est_bytes = pc_estimate_bytes(L, widths);
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  r->res.arrival_s = s->now();
  *id = r->id;
  Request* raw = r.get();
  s->all[r->id] = std::move(r);
  if (raw->res.est_bytes < 0 || raw->res.est_bytes > s->opt.request_max_bytes) {
    raw->res.status = PC_ERR_TOO_LARGE;
    raw->res.start_s = raw->res.finish_s = raw->res.arrival_s;
    raw->res.slot = -1;
    raw->done = true;
    return PC_OK;
  }
  raw->res.status = PC_PENDING;
  ++s->pending;
  s->queue.push_back(raw);
  s->cv_work.notify_all();
  return PC_OK;
}

pc_status pc_server_poll(pc_server* s, uint64_t id, pc_result* out) {
  if (!s || !out) return PC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return PC_ERR_INVALID;
  *out = it->second->res;
  return it->second->done ? PC_OK : PC_PENDING;
}

pc_status pc_server_wait_all(pc_server* s, double timeout_s) {
  if (!s) return PC_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return s->pending == 0; });
  return ok ? PC_OK : PC_ERR_TIMEOUT;
}

pc_status pc_server_outputs(pc_server* s, uint64_t id, double* X, int32_t* E, uint64_t* SIG) {
  if (!s) return PC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end() || !it->second->done) return PC_ERR_INVALID;
  Request* r = it->second.get();
  if (r->res.status != PC_OK || !s->opt.keep_outputs) return PC_ERR_INVALID;
  if (X) std::memcpy(X, r->X.data(), r->X.size() * sizeof(double));
  if (E) std::memcpy(E, r->E.data(), r->E.size() * sizeof(int32_t));
  if (SIG) std::memcpy(SIG, r->SIG.data(), r->SIG.size() * sizeof(uint64_t));
  return PC_OK;
}

const char* pc_server_error(pc_server* s, uint64_t id) {
  if (!s) return "null server";
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return "unknown request";
  return it->second->err.c_str();
}

pc_status pc_server_release(pc_server* s, uint64_t id) {
  if (!s) return PC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end() || !it->second->done) return PC_ERR_INVALID;
  s->all.erase(it);
  return PC_OK;
}

pc_status pc_server_stats(pc_server* s, int64_t* peak_bytes, int64_t* in_use_bytes) {
  if (!s) return PC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (peak_bytes) *peak_bytes = s->peak_in_use;
  if (in_use_bytes) *in_use_bytes = s->in_use;
  return PC_OK;
}

pc_status pc_server_destroy(pc_server* s) {
  if (!s) return PC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto* c : s->ctxs) pc_destroy(c);
  for (auto q : s->streams) cudaStreamDestroy(q);
  delete s;
  return PC_OK;
}

}  // extern "C"
