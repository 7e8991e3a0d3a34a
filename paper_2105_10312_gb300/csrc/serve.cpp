// serve.cpp — the serving loop (gpa_serve_*): a host queue of admission
// queries, a batcher thread that packs them into micro-batches and runs
// them on several streams while earlier batches are still on the GPU
// (continuous batching), and tenant state resident in device memory.
//
// Ordering: a micro-batch holds at most one request per tenant, and a
// tenant with a request in flight takes no new one until it completes, so
// each tenant sees its requests in submission order and every result
// depends only on that tenant's history.  Admission by memory: a new tenant
// needs a device slot; when none is free the pool grows by one allocation
// if the device keeps `reserve_bytes` free afterwards, otherwise the ADMIT
// waits in the queue (it is never failed for lack of memory).
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "gpa.h"
#include "gpa_ctx.h"
#include "serve_types.h"

using namespace gpa;
using Clock = std::chrono::steady_clock;

namespace {

struct Pending {
  uint64_t id;
  int op;
  int64_t tenant;
  int index;
  int n;
  std::vector<int64_t> T, D, A, B, u;
  std::vector<uint8_t> type;
  Clock::time_point t0;
};

struct TenantInfo {
  int slot;
  int n;
  bool busy;
};

struct StreamCtx {
  cudaStream_t stream = nullptr;
  ServeReq* h_req = nullptr;  // pinned
  ServeResp* h_resp = nullptr;
  long long* h_pay = nullptr;  // 5 x cap int64
  unsigned char* h_type = nullptr;
  ServeReq* d_req = nullptr;
  ServeResp* d_resp = nullptr;
  long long* d_pay = nullptr;
  unsigned char* d_type = nullptr;
  std::vector<Pending> batch;
  std::vector<int> slot_of;  // slot per batch entry
  int64_t pay_used = 0;
  bool busy = false;
  bool done = false;  // set by the completion callback
};

}  // namespace

struct ServeState {
  gpa_ctx* ctx = nullptr;
  gpa_serve_cfg cfg{};
  DevModel md{};
  gpa_params prm{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // batcher wakes up
  std::condition_variable cv_done;  // pollers wake up
  std::deque<Pending> queue;
  std::unordered_map<uint64_t, gpa_response> completed;
  std::unordered_set<uint64_t> outstanding;
  std::unordered_map<int64_t, TenantInfo> tenants;
  std::vector<int> free_slots;
  std::vector<TenantSlot*> chunks;
  TenantSlot** d_chunks = nullptr;
  cudaStream_t setup_stream = nullptr;
  std::vector<StreamCtx> streams;
  uint64_t next_id = 0;
  bool stop = false;
  std::thread worker;
  int64_t n_completed = 0, n_batches = 0, max_batch_seen = 0, n_overlapped = 0;
  int64_t pay_cap = 0;
  unsigned int* d_err = nullptr;
  unsigned short* d_sizes = nullptr;  // admissible sizes and rank table, or none
};

namespace {

void CUDART_CB on_batch_done(void* arg) {
  auto* pr = static_cast<std::pair<ServeState*, StreamCtx*>*>(arg);
  {
    std::lock_guard<std::mutex> lk(pr->first->mu);
    pr->second->done = true;
  }
  pr->first->cv_work.notify_one();
  delete pr;
}

// Add one chunk of tenant slots if the device keeps reserve_bytes free.
// Called by the batcher thread with the lock RELEASED (cudaMalloc may
// synchronise with work whose completion callbacks need the lock); only
// that thread changes the chunk list.
bool grow_slots(ServeState* S, std::unique_lock<std::mutex>* lk) {
  const int per = kSlotsPerChunkMax;
  const int idx = (int)S->chunks.size();
  if (idx >= kMaxChunks) return false;
  if ((int64_t)(idx + 1) * per > S->cfg.max_tenants + per) return false;
  if (lk) lk->unlock();
  bool ok = false;
  TenantSlot* c = nullptr;
  size_t free_b = 0, total_b = 0;
  const size_t bytes = sizeof(TenantSlot) * (size_t)per;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && free_b >= bytes + (size_t)S->cfg.reserve_bytes &&
      cudaMalloc(&c, bytes) == cudaSuccess) {
    ok = cudaMemcpyAsync(S->d_chunks + idx, &c, sizeof(TenantSlot*), cudaMemcpyHostToDevice, S->setup_stream) ==
             cudaSuccess &&
         cudaStreamSynchronize(S->setup_stream) == cudaSuccess;
    if (!ok) cudaFree(c);
  }
  if (lk) lk->lock();
  if (!ok) return false;
  S->chunks.push_back(c);
  for (int k = per - 1; k >= 0; k--) S->free_slots.push_back(idx * per + k);
  return true;
}

gpa_response error_response(const Pending& p, int32_t status) {
  gpa_response r;
  std::memset(&r, 0, sizeof r);
  r.req_id = p.id;
  r.status = status;
  r.latency_us = std::chrono::duration<double, std::micro>(Clock::now() - p.t0).count();
  return r;
}

// Complete a finished micro-batch (lock held).
void harvest(ServeState* S, StreamCtx& sc) {
  const auto now = Clock::now();
  for (size_t k = 0; k < sc.batch.size(); k++) {
    const Pending& p = sc.batch[k];
    const ServeResp& d = sc.h_resp[k];
    gpa_response r;
    std::memset(&r, 0, sizeof r);
    r.req_id = p.id;
    r.status = d.status == 1 ? GPA_ERR_RANGE : d.status == 2 ? GPA_ERR_TIMEOUT : GPA_OK;
    r.verdict = d.verdict;
    r.reason = d.reason;
    r.path = d.path;
    r.n_tasks = d.n_tasks;
    r.n_parts = d.n_parts;
    r.Pi = d.Pi;
    r.W = d.W;
    std::memcpy(r.part_of_task, d.part, sizeof r.part_of_task);
    std::memcpy(r.size_of_part, d.size, sizeof r.size_of_part);
    r.latency_us = std::chrono::duration<double, std::micro>(now - p.t0).count();
    auto it = S->tenants.find(p.tenant);
    if (it != S->tenants.end()) {
      TenantInfo& ti = it->second;
      ti.busy = false;
      const bool drop = (p.op == GPA_SERVE_EVICT) || (p.op == GPA_SERVE_ADMIT && !d.verdict) ||
                        (p.op == GPA_SERVE_ADMIT && d.status == 1);
      if (drop) {
        S->free_slots.push_back(ti.slot);
        S->tenants.erase(it);
      } else {
        ti.n = d.n_tasks;
      }
    }
    S->completed[p.id] = r;
    S->n_completed++;
  }
  sc.batch.clear();
  sc.slot_of.clear();
  sc.busy = false;
  sc.done = false;
}

// Pack one micro-batch for sc into its pinned staging buffers (lock held;
// no CUDA call).  Returns false if the queue had nothing launchable;
// *need_slots is set when an ADMIT waits for a free tenant slot.
bool form_batch(ServeState* S, StreamCtx& sc, bool* need_slots) {
  std::unordered_set<int64_t> blocked;
  int64_t pay_used = 0;
  const int cap = S->cfg.max_batch;
  for (auto it = S->queue.begin(); it != S->queue.end() && (int)sc.batch.size() < cap;) {
    Pending& p = *it;
    if (blocked.count(p.tenant)) {
      ++it;
      continue;
    }
    auto ti = S->tenants.find(p.tenant);
    int32_t err = GPA_OK;
    if (p.op == GPA_SERVE_ADMIT) {
      if (ti != S->tenants.end()) {
        if (ti->second.busy) {  // an EVICT of this tenant is still in flight: keep the order
          blocked.insert(p.tenant);
          ++it;
          continue;
        }
        err = GPA_ERR_ARG;  // tenant already exists
      }
    } else if (ti == S->tenants.end()) {
      err = GPA_ERR_NOTFOUND;
    } else if (ti->second.busy) {
      blocked.insert(p.tenant);
      ++it;
      continue;
    } else if (p.op == GPA_SERVE_ADD && ti->second.n >= GPA_SERVE_NMAX) {
      err = GPA_ERR_RANGE;
    } else if (p.op == GPA_SERVE_REMOVE && (p.index < 0 || p.index >= ti->second.n)) {
      err = GPA_ERR_RANGE;
    }
    if (err != GPA_OK) {
      S->completed[p.id] = error_response(p, err);
      S->n_completed++;
      it = S->queue.erase(it);
      continue;
    }
    if (pay_used + p.n > S->pay_cap) break;
    int slot = -1;
    if (p.op == GPA_SERVE_ADMIT) {
      if (S->free_slots.empty()) {
        *need_slots = true;
        blocked.insert(p.tenant);  // waits for a slot (or for memory to add one)
        ++it;
        continue;
      }
      slot = S->free_slots.back();
      S->free_slots.pop_back();
      S->tenants[p.tenant] = TenantInfo{slot, 0, true};
    } else {
      slot = ti->second.slot;
      ti->second.busy = true;
    }
    const int k = (int)sc.batch.size();
    ServeReq& rq = sc.h_req[k];
    rq.op = p.op;
    rq.slot = slot;
    rq.index = p.index;
    rq.n = p.n;
    rq.payload = pay_used;
    for (int i = 0; i < p.n; i++) {
      sc.h_pay[0 * S->pay_cap + pay_used + i] = p.T[(size_t)i];
      sc.h_pay[1 * S->pay_cap + pay_used + i] = p.D[(size_t)i];
      sc.h_pay[2 * S->pay_cap + pay_used + i] = p.A[(size_t)i];
      sc.h_pay[3 * S->pay_cap + pay_used + i] = p.B[(size_t)i];
      sc.h_pay[4 * S->pay_cap + pay_used + i] = p.u[(size_t)i];
      sc.h_type[pay_used + i] = p.type[(size_t)i];
    }
    pay_used += p.n;
    blocked.insert(p.tenant);
    sc.batch.push_back(std::move(p));
    sc.slot_of.push_back(slot);
    it = S->queue.erase(it);
  }
  if (sc.batch.empty()) return false;
  sc.pay_used = pay_used;
  sc.busy = true;
  sc.done = false;
  S->n_batches++;
  if ((int64_t)sc.batch.size() > S->max_batch_seen) S->max_batch_seen = (int64_t)sc.batch.size();
  for (auto& o : S->streams)
    if (&o != &sc && o.busy && !o.done) {
      S->n_overlapped++;
      break;
    }
  return true;
}

// Enqueue a formed batch (lock RELEASED: a launch may block until earlier
// work, whose completion callback takes the lock, has drained).
void issue_batch(ServeState* S, StreamCtx& sc) {
  const int nreq = (int)sc.batch.size();
  const int64_t pay_used = sc.pay_used;
  cudaStream_t st = sc.stream;
  cudaMemcpyAsync(sc.d_req, sc.h_req, sizeof(ServeReq) * (size_t)nreq, cudaMemcpyHostToDevice, st);
  if (pay_used > 0) {
    for (int c = 0; c < 5; c++)
      cudaMemcpyAsync(sc.d_pay + c * S->pay_cap, sc.h_pay + c * S->pay_cap, sizeof(long long) * (size_t)pay_used,
                      cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(sc.d_type, sc.h_type, (size_t)pay_used, cudaMemcpyHostToDevice, st);
  }
  ServePayload pay{sc.d_pay, sc.d_pay + S->pay_cap, sc.d_pay + 2 * S->pay_cap, sc.d_pay + 3 * S->pay_cap,
                   sc.d_pay + 4 * S->pay_cap, sc.d_type};
  launch_serve_batch(sc.d_req, nreq, S->d_chunks, pay, sc.d_resp, S->md, S->prm, S->ctx->d_mdiv, S->d_err, st);
  cudaMemcpyAsync(sc.h_resp, sc.d_resp, sizeof(ServeResp) * (size_t)nreq, cudaMemcpyDeviceToHost, st);
  cudaLaunchHostFunc(st, on_batch_done, new std::pair<ServeState*, StreamCtx*>(S, &sc));
}

void worker_main(ServeState* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool any_busy = false;
    for (auto& sc : S->streams) {
      if (sc.busy && sc.done) harvest(S, sc);
      any_busy = any_busy || sc.busy;
    }
    S->cv_done.notify_all();
    bool launched = false, need_slots = false;
    if (!S->queue.empty())
      for (auto& sc : S->streams)
        if (!sc.busy && form_batch(S, sc, &need_slots)) {
          lk.unlock();
          issue_batch(S, sc);
          lk.lock();
          S->ctx->launches += 1;
          launched = true;
          any_busy = true;
        }
    if (need_slots && grow_slots(S, &lk)) launched = true;  // retry the waiting ADMITs at once
    if (S->stop && S->queue.empty() && !any_busy) break;
    if (launched) continue;
    // sleep until a submission or a completion (bounded, so a queue blocked
    // on memory is retried)
    S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
  }
}

void free_state(ServeState* S) {
  for (auto& sc : S->streams) {
    if (sc.stream) cudaStreamSynchronize(sc.stream);
    cudaFreeHost(sc.h_req);
    cudaFreeHost(sc.h_resp);
    cudaFreeHost(sc.h_pay);
    cudaFreeHost(sc.h_type);
    cudaFree(sc.d_req);
    cudaFree(sc.d_resp);
    cudaFree(sc.d_pay);
    cudaFree(sc.d_type);
    if (sc.stream) cudaStreamDestroy(sc.stream);
  }
  for (auto* c : S->chunks) cudaFree(c);
  cudaFree(S->d_chunks);
  cudaFree(S->d_err);
  cudaFree(S->d_sizes);
  if (S->setup_stream) cudaStreamDestroy(S->setup_stream);
}

}  // namespace

void gpa_serve_teardown(gpa_ctx* c) {
  if (c && c->serve) gpa_serve_stop(c);
}

extern "C" int32_t gpa_serve_start(gpa_ctx* c, const gpa_serve_cfg* cfg) {
  if (!c || !cfg) return gpa_fail(GPA_ERR_ARG, "gpa_serve_start: NULL argument");
  if (c->serve) return gpa_fail(GPA_ERR_BUSY, "gpa_serve_start: a server is already running on this context");
  if (cfg->g < 1 || cfg->M < 1 || cfg->M > GPA_MMAX || cfg->M % cfg->g || cfg->k_c_pm < 1000 ||
      cfg->k_c_pm > 16000 || cfg->k_m_pm < 1000 || cfg->k_m_pm > 16000)
    return gpa_fail(GPA_ERR_RANGE, "gpa_serve_start: model out of range");
  if (cfg->policy != GPA_POLICY_SMS && cfg->policy != GPA_POLICY_BF)
    return gpa_fail(GPA_ERR_ARG, "gpa_serve_start: policy must be SMS or BF");
  if (cfg->sched != GPA_SCHED_DM && cfg->sched != GPA_SCHED_EDF)
    return gpa_fail(GPA_ERR_ARG, "gpa_serve_start: unknown scheduling policy");
  if (cfg->nsizes < 0 || cfg->nsizes > GPA_MMAX || (cfg->nsizes > 0 && !cfg->sizes))
    return gpa_fail(GPA_ERR_RANGE, "gpa_serve_start: size list out of range");
  for (int k = 0; k < cfg->nsizes; k++) {
    const int z = cfg->sizes[k];
    if (z < cfg->g || z > cfg->M || z % cfg->g != 0 || (k > 0 && z <= cfg->sizes[k - 1]))
      return gpa_fail(GPA_ERR_RANGE, "gpa_serve_start: size list must increase over multiples of g in [g, M]");
  }
  if (cfg->max_batch < 1 || cfg->max_batch > 4096 || cfg->nstreams < 1 || cfg->nstreams > 8 || cfg->queue_cap < 1 ||
      cfg->max_tenants < 1 || cfg->max_tenants > (int64_t)kSlotsPerChunkMax * kMaxChunks || cfg->reserve_bytes < 0)
    return gpa_fail(GPA_ERR_RANGE, "gpa_serve_start: configuration out of range");
  cudaSetDevice(c->device);
  cudaError_t e = serve_kernels_init();
  if (e != cudaSuccess) return gpa_cuda_fail(e, "serve kernel attributes");
  auto* S = new ServeState();
  S->ctx = c;
  S->cfg = *cfg;
  S->device = c->device;
  S->md = DevModel{cfg->M, cfg->g, cfg->k_c_pm, cfg->k_m_pm, cfg->sched, 0, nullptr, nullptr};
  S->cfg.sizes = nullptr;  // the list is copied to the device below, not kept by pointer
  S->prm = gpa_params{cfg->policy, cfg->act, 1, 0};
  S->pay_cap = (int64_t)cfg->max_batch * GPA_SERVE_NMAX;
  bool ok = cudaStreamCreateWithFlags(&S->setup_stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&S->d_chunks, sizeof(TenantSlot*) * kMaxChunks) == cudaSuccess &&
            cudaMemset(S->d_chunks, 0, sizeof(TenantSlot*) * kMaxChunks) == cudaSuccess &&
            cudaMalloc(&S->d_err, sizeof(unsigned int)) == cudaSuccess &&
            cudaMemset(S->d_err, 0, sizeof(unsigned int)) == cudaSuccess;
  S->streams.resize((size_t)cfg->nstreams);
  for (auto& sc : S->streams) {
    if (!ok) break;
    const size_t nb = (size_t)cfg->max_batch, pb = (size_t)S->pay_cap;
    ok = cudaStreamCreateWithFlags(&sc.stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaMallocHost(&sc.h_req, sizeof(ServeReq) * nb) == cudaSuccess &&
         cudaMallocHost(&sc.h_resp, sizeof(ServeResp) * nb) == cudaSuccess &&
         cudaMallocHost(&sc.h_pay, sizeof(long long) * 5 * pb) == cudaSuccess &&
         cudaMallocHost(&sc.h_type, pb) == cudaSuccess &&
         cudaMalloc(&sc.d_req, sizeof(ServeReq) * nb) == cudaSuccess &&
         cudaMalloc(&sc.d_resp, sizeof(ServeResp) * nb) == cudaSuccess &&
         cudaMalloc(&sc.d_pay, sizeof(long long) * 5 * pb) == cudaSuccess &&
         cudaMalloc(&sc.d_type, pb) == cudaSuccess;
  }
  if (ok && cfg->nsizes > 0) {
    // the admissible sizes and their rank table over [0, M + 1] (see gpa_model)
    std::vector<unsigned short> host((size_t)cfg->nsizes + (size_t)cfg->M + 2);
    for (int k = 0; k < cfg->nsizes; k++) host[(size_t)k] = (unsigned short)cfg->sizes[k];
    int below = 0;
    for (int m = 0; m <= cfg->M + 1; m++) {
      host[(size_t)cfg->nsizes + (size_t)m] = (unsigned short)below;
      if (below < cfg->nsizes && cfg->sizes[below] == m) below++;
    }
    ok = cudaMalloc(&S->d_sizes, sizeof(unsigned short) * host.size()) == cudaSuccess &&
         cudaMemcpy(S->d_sizes, host.data(), sizeof(unsigned short) * host.size(), cudaMemcpyHostToDevice) ==
             cudaSuccess;
    if (ok) {
      S->md.nz = cfg->nsizes;
      S->md.zlist = S->d_sizes;
      S->md.zrank = S->d_sizes + cfg->nsizes;
    }
  }
  if (ok) {
    const int want = cfg->slots_per_chunk > 0 ? cfg->slots_per_chunk : kSlotsPerChunkMax;
    for (int got = 0; got < want && ok; got += kSlotsPerChunkMax) ok = grow_slots(S, nullptr);
  }
  if (!ok) {
    free_state(S);
    delete S;
    return gpa_fail(GPA_ERR_NOMEM, "gpa_serve_start: device or pinned allocation failed");
  }
  c->serve = S;
  S->worker = std::thread(worker_main, S);
  return GPA_OK;
}

extern "C" int32_t gpa_serve_submit(gpa_ctx* c, const gpa_request* r, uint64_t* req_id) {
  if (!c || !c->serve || !r || !req_id) return gpa_fail(GPA_ERR_ARG, "gpa_serve_submit: no server or NULL argument");
  ServeState* S = c->serve;
  if (r->op < GPA_SERVE_ADMIT || r->op > GPA_SERVE_EVICT || r->tenant < 0)
    return gpa_fail(GPA_ERR_ARG, "gpa_serve_submit: bad op or tenant");
  Pending p;
  p.op = r->op;
  p.tenant = r->tenant;
  p.index = r->index;
  p.n = 0;
  if (r->op == GPA_SERVE_ADMIT || r->op == GPA_SERVE_ADD) {
    const int n = r->op == GPA_SERVE_ADD ? 1 : r->n;
    if (n < 0 || n > GPA_SERVE_NMAX) return gpa_fail(GPA_ERR_RANGE, "gpa_serve_submit: %d tasks", n);
    if (n > 0 && (!r->T || !r->D || !r->A || !r->B || !r->u_ppm || !r->type))
      return gpa_fail(GPA_ERR_ARG, "gpa_serve_submit: NULL task column");
    for (int i = 0; i < n; i++) {
      const int64_t T = r->T[i], D = r->D[i], A = r->A[i], B = r->B[i], u = r->u_ppm[i];
      const bool ok = D >= 1 && D <= T && T <= 2147483647LL && A >= 0 && B >= 0 && A + B >= 1 &&
                      A + B <= (1LL << 36) && u >= 0 && u <= 4294967295LL && r->type[i] <= 1;
      if (!ok) return gpa_fail(GPA_ERR_RANGE, "gpa_serve_submit: task %d violates the bounds", i);
    }
    p.n = n;
    p.T.assign(r->T, r->T + n);
    p.D.assign(r->D, r->D + n);
    p.A.assign(r->A, r->A + n);
    p.B.assign(r->B, r->B + n);
    p.u.assign(r->u_ppm, r->u_ppm + n);
    p.type.assign(r->type, r->type + n);
  }
  p.t0 = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return gpa_fail(GPA_ERR_ARG, "gpa_serve_submit: the server is stopping");
    if ((int)S->queue.size() >= S->cfg.queue_cap) return gpa_fail(GPA_ERR_BUSY, "gpa_serve_submit: queue full");
    p.id = ++S->next_id;
    *req_id = p.id;
    S->outstanding.insert(p.id);
    S->queue.push_back(std::move(p));
  }
  S->cv_work.notify_one();
  return GPA_OK;
}

extern "C" int32_t gpa_serve_poll(gpa_ctx* c, uint64_t req_id, gpa_response* out, int64_t timeout_us) {
  if (!c || !c->serve || !out) return gpa_fail(GPA_ERR_ARG, "gpa_serve_poll: no server or NULL argument");
  ServeState* S = c->serve;
  std::unique_lock<std::mutex> lk(S->mu);
  if (!S->outstanding.count(req_id)) return gpa_fail(GPA_ERR_NOTFOUND, "gpa_serve_poll: unknown request %llu",
                                                     (unsigned long long)req_id);
  const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  for (;;) {
    auto it = S->completed.find(req_id);
    if (it != S->completed.end()) {
      *out = it->second;
      S->completed.erase(it);
      S->outstanding.erase(req_id);
      return GPA_OK;
    }
    if (timeout_us <= 0 || Clock::now() >= deadline) return gpa_fail(GPA_ERR_TIMEOUT, "gpa_serve_poll: not done");
    S->cv_done.wait_until(lk, deadline);
  }
}

extern "C" int32_t gpa_serve_stop(gpa_ctx* c) {
  if (!c || !c->serve) return gpa_fail(GPA_ERR_ARG, "gpa_serve_stop: no server");
  ServeState* S = c->serve;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_one();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  free_state(S);
  delete S;
  c->serve = nullptr;
  return GPA_OK;
}

extern "C" int32_t gpa_serve_stats(gpa_ctx* c, int64_t* completed, int64_t* batches, int64_t* max_batch,
                                   int64_t* overlapped, int64_t* slots) {
  if (!c || !c->serve) return gpa_fail(GPA_ERR_ARG, "gpa_serve_stats: no server");
  ServeState* S = c->serve;
  std::lock_guard<std::mutex> lk(S->mu);
  if (completed) *completed = S->n_completed;
  if (batches) *batches = S->n_batches;
  if (max_batch) *max_batch = S->max_batch_seen;
  if (overlapped) *overlapped = S->n_overlapped;
  if (slots) *slots = (int64_t)S->chunks.size() * kSlotsPerChunkMax;
  return GPA_OK;
}
