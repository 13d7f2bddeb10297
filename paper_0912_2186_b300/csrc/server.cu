// Continuous-batching solve server.  Gauge fields and their multigrid hierarchies stay
// resident in HBM (one context per field); each field has a worker thread and its own CUDA
// stream, so the work of different fields overlaps on the device.  Requests (a mass and 1..n
// right-hand sides) queue per field; the worker's outer-solver slot engine admits their
// right-hand sides into free slots at every restart boundary, so requests that arrive while
// a batch is running join it as slots free up, and every slot of a launch shares the field's
// hierarchy (different masses differ only by a diagonal shift).  Fields are admitted by
// their HBM footprint against the server's budget.  Each request records its latency from
// submission to completion.
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "ctx.h"
#include "solver.h"

using namespace wmg;

namespace {

using clk = std::chrono::steady_clock;

struct Request {
  long long id = 0;
  int field = 0;
  double mass = 0.0;
  const double* b = nullptr;  // host, canonical, nrhs spinors
  double* x = nullptr;        // host, canonical
  int nrhs = 0;
  int admitted = 0, finished = 0;
  std::vector<wmg_info> info;
  clk::time_point t_submit, t_done;
  bool done = false;
  wmg_status status = WMG_OK;
};

struct Field;

}  // namespace

struct wmg_server {
  size_t budget = 0, used = 0;
  std::vector<Field*> fields;
  std::mutex mu;  // guards requests, queues and completion state
  std::condition_variable cv_done;
  std::map<long long, Request*> reqs;
  long long next_id = 1;
};

namespace {

struct Field {
  wmg_server* srv = nullptr;
  wmg_ctx* ctx = nullptr;
  int nslots = 0;
  size_t footprint = 0;
  std::thread th;
  std::deque<Request*> queue;
  std::condition_variable cv;
  bool stop = false;
  std::vector<std::pair<Request*, int>> owner;  // slot -> (request, rhs index)
  void* bstage = nullptr;                       // device canonical staging, one spinor per slot
  void* xstage = nullptr;
  double* hstage = nullptr;                     // pinned host staging, one spinor
  wmg_status err = WMG_OK;
};

struct ServerSource : SlotSource {
  Field* f;
  explicit ServerSource(Field* f_) : f(f_) {}
  size_t spinor_bytes() const { return (size_t)f->ctx->fine.V * 12 * sizeof(cd); }

  void admit(wmg_ctx* c, const std::vector<int>& free_slots, std::vector<Admission>& out) override {
    std::vector<std::pair<Request*, int>> take;
    {
      std::lock_guard<std::mutex> lock(f->srv->mu);
      for (int slot : free_slots) {
        if (f->queue.empty()) break;
        Request* q = f->queue.front();
        take.push_back({q, q->admitted});
        f->owner[slot] = {q, q->admitted};
        out.push_back({slot, (const double*)((char*)f->bstage + spinor_bytes() * slot), q->mass});
        if (++q->admitted == q->nrhs) f->queue.pop_front();
      }
    }
    // copy the admitted right-hand sides to the device (host buffers belong to the caller)
    for (size_t i = 0; i < take.size(); ++i) {
      const Request* q = take[i].first;
      const int r = take[i].second;
      std::memcpy(f->hstage, q->b + (size_t)c->fine.V * 24 * r, spinor_bytes());
      cudaMemcpyAsync((char*)f->bstage + spinor_bytes() * out[out.size() - take.size() + i].slot, f->hstage,
                      spinor_bytes(), cudaMemcpyHostToDevice, c->stream);
      cudaStreamSynchronize(c->stream);
    }
  }

  wmg_status finish(wmg_ctx* c, int slot, const void* x64, const wmg_info& info) override {
    Request* q = f->owner[slot].first;
    const int r = f->owner[slot].second;
    f->owner[slot] = {nullptr, 0};
    void* xs = (char*)f->xstage + spinor_bytes() * slot;
    unpack_spinor(WMG_PREC_DOUBLE, x64, (double*)xs, c->fine.V, 1, c->stream);
    cudaError_t e = cudaMemcpyAsync(f->hstage, xs, spinor_bytes(), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, e, "server: copy x");
    std::memcpy(q->x + (size_t)c->fine.V * 24 * r, f->hstage, spinor_bytes());
    std::lock_guard<std::mutex> lock(f->srv->mu);
    q->info[r] = info;
    if (!info.converged) q->status = WMG_ENOCONV;
    if (++q->finished == q->nrhs) {
      q->t_done = clk::now();
      q->done = true;
      f->srv->cv_done.notify_all();
    }
    return WMG_OK;
  }
};

void worker(Field* f) {
  cudaSetDevice(f->ctx->device);
  while (true) {
    {
      std::unique_lock<std::mutex> lock(f->srv->mu);
      f->cv.wait(lock, [&] { return f->stop || !f->queue.empty(); });
      if (f->stop && f->queue.empty()) return;
    }
    ServerSource src(f);
    wmg_status st = fgcr_engine(f->ctx, f->nslots, src, true);
    if (st != WMG_OK) {
      // fail every request that is queued or in a slot, keep serving
      std::lock_guard<std::mutex> lock(f->srv->mu);
      f->err = st;
      auto fail_req = [&](Request* q) {
        if (!q || q->done) return;
        q->status = st;
        q->done = true;
        q->t_done = clk::now();
      };
      for (auto& o : f->owner) fail_req(o.first), o = {nullptr, 0};
      for (Request* q : f->queue) fail_req(q);
      f->queue.clear();
      f->srv->cv_done.notify_all();
    }
  }
}

// device bytes held by a context for its field and hierarchy plus the slot workspaces
size_t field_footprint(const wmg_ctx* c, int nslots) {
  const double V = c->fine.V;
  // links and every operator copy as allocated, plus the slot workspaces of nslots
  double b = 0.0;
  {
    size_t ops = context_device_bytes(c);
    for (const auto& kv : c->ws) ops -= kv.second.second;
    b = (double)ops;
  }
  const int m = c->prm.gcr_restart;
  const double lo = c->prm.prec_sloppy == WMG_PREC_DOUBLE ? 16 : 8;
  b += nslots * V * 12 * (4 * 16 + (1 + 2 * m + 3) * lo + 2 * 16);  // engine, smoother and staging vectors
  return (size_t)b;
}

}  // namespace

extern "C" {

wmg_status wmg_server_create(wmg_server** out, size_t hbm_budget_bytes) {
  if (!out) return WMG_EINVAL;
  wmg_server* s = new wmg_server();
  s->budget = hbm_budget_bytes;
  *out = s;
  return WMG_OK;
}

wmg_status wmg_server_add_field(wmg_server* s, wmg_ctx* ctx, int nslots, int* field_id) {
  if (!s || !ctx || !field_id || nslots < 1 || nslots > kMaxRhs) return WMG_EINVAL;
  if (!ctx->have_hier) return WMG_ESTATE;
  const size_t fp = field_footprint(ctx, nslots);
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->used + fp > s->budget) {
    ctx->err = "server: field footprint exceeds the HBM budget";
    return WMG_ENOMEM;
  }
  Field* f = new Field();
  f->srv = s;
  f->ctx = ctx;
  f->nslots = nslots;
  f->footprint = fp;
  f->owner.assign(nslots, {nullptr, 0});
  const size_t sb = (size_t)ctx->fine.V * 12 * sizeof(cd);
  if (cudaMalloc(&f->bstage, sb * nslots) != cudaSuccess || cudaMalloc(&f->xstage, sb * nslots) != cudaSuccess ||
      cudaMallocHost((void**)&f->hstage, sb) != cudaSuccess) {
    if (f->bstage) cudaFree(f->bstage);
    if (f->xstage) cudaFree(f->xstage);
    delete f;
    return WMG_ENOMEM;
  }
  s->used += fp;
  *field_id = (int)s->fields.size();
  s->fields.push_back(f);
  f->th = std::thread(worker, f);
  return WMG_OK;
}

wmg_status wmg_server_submit(wmg_server* s, int field_id, double mass, const double* b_host, double* x_host,
                             int nrhs, long long* ticket) {
  if (!s || !b_host || !x_host || nrhs < 1 || !ticket) return WMG_EINVAL;
  if (field_id < 0 || field_id >= (int)s->fields.size() || !(mass == mass)) return WMG_EINVAL;
  Request* q = new Request();
  q->field = field_id;
  q->mass = mass;
  q->b = b_host;
  q->x = x_host;
  q->nrhs = nrhs;
  q->info.assign(nrhs, wmg_info{});
  q->t_submit = clk::now();
  Field* f = s->fields[field_id];
  {
    std::lock_guard<std::mutex> lock(s->mu);
    q->id = s->next_id++;
    s->reqs[q->id] = q;
    f->queue.push_back(q);
  }
  f->cv.notify_one();
  *ticket = q->id;
  return WMG_OK;
}

wmg_status wmg_server_poll(wmg_server* s, long long ticket, int* done) {
  if (!s || !done) return WMG_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return WMG_EINVAL;
  *done = it->second->done;
  return WMG_OK;
}

wmg_status wmg_server_wait(wmg_server* s, long long ticket, wmg_info* info, double* latency_s) {
  if (!s) return WMG_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return WMG_EINVAL;
  Request* q = it->second;
  s->cv_done.wait(lock, [&] { return q->done; });
  if (info)
    for (int r = 0; r < q->nrhs; ++r) info[r] = q->info[r];
  if (latency_s) *latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
  const wmg_status st = q->status;
  s->reqs.erase(it);
  delete q;
  return st;
}

wmg_status wmg_server_destroy(wmg_server* s) {
  if (!s) return WMG_EINVAL;
  for (Field* f : s->fields) {
    {
      std::lock_guard<std::mutex> lock(s->mu);
      f->stop = true;
    }
    f->cv.notify_all();
  }
  for (Field* f : s->fields) {
    if (f->th.joinable()) f->th.join();
    cudaFree(f->bstage);
    cudaFree(f->xstage);
    cudaFreeHost(f->hstage);
    delete f;
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return WMG_OK;
}

}  // extern "C"
