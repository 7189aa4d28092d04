// sg_server.cu -- serving runtime over the C ABI: admission of requests
// against a device byte budget and a pool of slots (one handle, one CUDA
// stream and one host worker thread each), continuous batching of small
// requests into sgagg_aggregate_batched calls, per-request timestamps.
//
// Host code only.  The admission and batching decisions live in Scheduler,
// which the server and the virtual-time simulator (sgagg_server_simulate)
// share, so that the decisions are testable without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <queue>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/sgagg.h"

namespace {

int64_t clock_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Pending {
  int64_t ticket;
  int64_t rows;
  int64_t footprint;
  bool batchable;  // can share a batched call
};

// Requests a batched call runs in one pass: at most one chunk (any key
// width, a CTA each), or keys of at most 32 bits (composite key).
constexpr int64_t kDirectRows = 8192;
bool batchable(const sgagg_server_config& c, int64_t rows, int key_bytes) {
  return c.small_rows > 0 && rows <= c.small_rows && (rows <= kDirectRows || key_bytes <= 4);
}

// FIFO admission: the oldest waiting request starts when a slot is free and
// its footprint fits the budget left; small requests behind it join its call.
class Scheduler {
 public:
  explicit Scheduler(const sgagg_server_config& c) : cfg_(c), busy_((size_t)c.slots, false) {}

  void push(const Pending& p) { q_.push_back(p); }
  bool empty() const { return q_.empty(); }

  // Start the next call if one can start now, on `want` (>= 0: that slot,
  // which must be free) or on the lowest free slot.  Fills the tickets it
  // covers (in arrival order), their total rows and footprint, and the slot.
  bool next(int want, std::vector<int64_t>* ids, int64_t* rows, int64_t* fp, int* slot) {
    if (q_.empty()) return false;
    int sl = want;
    if (sl < 0) {
      for (int i = 0; i < cfg_.slots; ++i)
        if (!busy_[(size_t)i]) {
          sl = i;
          break;
        }
      if (sl < 0) return false;
    } else if (busy_[(size_t)sl]) {
      return false;
    }
    const Pending& h = q_.front();
    if (in_use_ + h.footprint > cfg_.device_budget_bytes) return false;
    ids->clear();
    int64_t f = 0, r = 0;
    if (h.batchable) {
      const int cap = std::max(1, cfg_.max_batch);
      while (!q_.empty()) {
        const Pending& p = q_.front();
        if (!p.batchable || (int)ids->size() >= cap) break;
        if (!ids->empty() && r + p.rows > cfg_.max_batch_rows) break;
        if (in_use_ + f + p.footprint > cfg_.device_budget_bytes) break;
        ids->push_back(p.ticket);
        f += p.footprint;
        r += p.rows;
        q_.pop_front();
      }
    } else {
      ids->push_back(h.ticket);
      f = h.footprint;
      r = h.rows;
      q_.pop_front();
    }
    in_use_ += f;
    busy_[(size_t)sl] = true;
    *rows = r;
    *fp = f;
    *slot = sl;
    return true;
  }

  void done(int slot, int64_t fp) {
    in_use_ -= fp;
    busy_[(size_t)slot] = false;
  }

 private:
  sgagg_server_config cfg_;
  std::deque<Pending> q_;
  std::vector<bool> busy_;
  int64_t in_use_ = 0;
};

bool config_ok(const sgagg_server_config* c) {
  return c && c->slots >= 1 && c->slots <= 256 && c->device_budget_bytes > 0 && c->memory_budget_rows >= 1 &&
         c->small_rows >= 0 && c->max_batch >= 1 && c->max_batch_rows >= 1;
}

struct Req {
  sgagg_request r;
  std::vector<const int64_t*> pay;
  std::vector<int64_t*> oa;
  sgagg_request_result res;
  bool done = false;
};

struct Slot {
  sgagg_t h = nullptr;
  cudaStream_t st = nullptr;
  std::thread th;
  void* dptr = nullptr;   // batched call: device pointer arrays and row counts
  void* hptr = nullptr;   // pinned host copy of the same
  size_t cap = 0;
};

}  // namespace

struct sgagg_server {
  sgagg_server_config cfg;
  std::vector<sgagg_agg> aggs;
  sgagg_spec spec;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  Scheduler sched;
  std::unordered_map<int64_t, Req*> reqs;
  int64_t next_ticket = 1;
  std::vector<Slot> slots;

  explicit sgagg_server(const sgagg_server_config& c) : cfg(c), spec{0, nullptr}, sched(c) {}
};

namespace {

sgagg_status grow_staging(Slot& sl, size_t bytes) {
  if (bytes <= sl.cap) return SGAGG_OK;
  size_t nb = std::max(bytes, sl.cap * 2);
  void* d = nullptr;
  void* hp = nullptr;
  if (cudaMalloc(&d, nb) != cudaSuccess) return SGAGG_ENOMEM;
  if (cudaMallocHost(&hp, nb) != cudaSuccess) {
    cudaFree(d);
    return SGAGG_ENOMEM;
  }
  if (sl.dptr) cudaFree(sl.dptr);
  if (sl.hptr) cudaFreeHost(sl.hptr);
  sl.dptr = d;
  sl.hptr = hp;
  sl.cap = nb;
  return SGAGG_OK;
}

// One request alone: the plain path on the slot's handle and stream.
void run_one(sgagg_server* s, Slot& sl, Req* q) {
  if (q->r.ready) cudaStreamWaitEvent(sl.st, (cudaEvent_t)q->r.ready, 0);
  int32_t kb = q->r.key_bytes;
  const void* kc = q->r.keys;
  sgagg_keys k{1, &kb, &kc};
  void* ok = q->r.out_keys;
  int64_t rows = -1;
  sgagg_status st = sgagg_aggregate(sl.h, &k, q->pay.data(), q->r.n_payload, q->r.n, &s->spec, &ok, q->oa.data(),
                                    q->r.out_capacity, sl.st);
  if (st == SGAGG_OK) st = sgagg_result_rows(sl.h, &rows);
  q->res.status = st;
  q->res.rows = st == SGAGG_OK ? rows : -1;
}

// Several small requests: one batched call.
void run_batch(sgagg_server* s, Slot& sl, const std::vector<Req*>& qs) {
  const int k = (int)qs.size();
  const int S = s->spec.n_aggs;
  size_t words = (size_t)k;  // out_rows
  for (Req* q : qs) words += (size_t)q->r.n_payload + (size_t)S;
  sgagg_status st = grow_staging(sl, words * 8);
  if (st == SGAGG_OK) {
    int64_t* hw = static_cast<int64_t*>(sl.hptr);
    int64_t* dw = static_cast<int64_t*>(sl.dptr);
    std::vector<sgagg_instance> inst((size_t)k);
    size_t at = (size_t)k;
    for (int i = 0; i < k; ++i) {
      Req* q = qs[(size_t)i];
      if (q->r.ready) cudaStreamWaitEvent(sl.st, (cudaEvent_t)q->r.ready, 0);
      sgagg_instance& d = inst[(size_t)i];
      d.keys = q->r.keys;
      d.key_bytes = q->r.key_bytes;
      d.n_payload = q->r.n_payload;
      d.payload = reinterpret_cast<const int64_t* const*>(dw + at);
      for (int c = 0; c < q->r.n_payload; ++c) hw[at++] = (int64_t)(intptr_t)q->pay[(size_t)c];
      d.n = q->r.n;
      d.out_keys = q->r.out_keys;
      d.out_aggs = reinterpret_cast<int64_t* const*>(dw + at);
      for (int a = 0; a < S; ++a) hw[at++] = (int64_t)(intptr_t)q->oa[(size_t)a];
      d.out_capacity = q->r.out_capacity;
      d.out_rows = dw + i;
      hw[i] = -1;
    }
    if (cudaMemcpyAsync(dw, hw, words * 8, cudaMemcpyHostToDevice, sl.st) != cudaSuccess) st = SGAGG_ECUDA;
    if (st == SGAGG_OK) st = sgagg_aggregate_batched(sl.h, inst.data(), k, &s->spec, sl.st);
    int64_t total = 0;
    if (st == SGAGG_OK) st = sgagg_result_rows(sl.h, &total);
    if (st == SGAGG_OK) {
      if (cudaMemcpyAsync(hw, dw, (size_t)k * 8, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess ||
          cudaStreamSynchronize(sl.st) != cudaSuccess)
        st = SGAGG_ECUDA;
    }
    if (st == SGAGG_OK) {
      for (int i = 0; i < k; ++i) {
        Req* q = qs[(size_t)i];
        q->res.rows = hw[i];
        q->res.status = hw[i] < 0 ? SGAGG_ECAPACITY : SGAGG_OK;
      }
      return;
    }
  }
  for (Req* q : qs) {
    q->res.status = st;
    q->res.rows = -1;
  }
}

void worker(sgagg_server* s, int i) {
  cudaSetDevice(s->device);
  Slot& sl = s->slots[(size_t)i];
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    std::vector<int64_t> ids;
    int64_t rows = 0, fp = 0;
    int slot = -1;
    while (!s->sched.next(i, &ids, &rows, &fp, &slot)) {
      if (s->stop && s->sched.empty()) return;
      s->cv.wait(lk);
    }
    std::vector<Req*> qs;
    const int64_t t0 = clock_ns();
    for (int64_t t : ids) {
      Req* q = s->reqs[t];
      q->res.start_ns = t0;
      q->res.slot = i;
      q->res.batch_size = (int32_t)ids.size();
      qs.push_back(q);
    }
    lk.unlock();
    if (qs.size() == 1) run_one(s, sl, qs[0]);
    else run_batch(s, sl, qs);
    const int64_t t1 = clock_ns();
    lk.lock();
    s->sched.done(i, fp);
    for (Req* q : qs) {
      q->res.done_ns = t1;
      q->done = true;
    }
    s->cv.notify_all();
  }
}

}  // namespace

extern "C" {

int64_t sgagg_request_footprint(int64_t n, int32_t key_bytes, int32_t n_payload, int32_t n_aggs,
                                int64_t out_capacity, int64_t memory_budget_rows) {
  if (n < 0 || out_capacity < 0 || n_payload < 0 || n_aggs < 0) return -1;
  const int64_t in = n * (key_bytes + 8ll * n_payload);
  const int64_t out = out_capacity * (key_bytes + 8ll * n_aggs);
  const int64_t m = memory_budget_rows > 0 ? std::min(n, memory_budget_rows) : n;
  const int64_t ws = 8 * m * (3 + 3ll * n_payload + 3ll * (1 + n_aggs));
  const int64_t runs = (memory_budget_rows > 0 && n > memory_budget_rows) ? 8 * n * (1ll + n_aggs) : 0;
  return in + out + ws + runs + (64ll << 20);
}

int64_t sgagg_server_now_ns(void) { return clock_ns(); }

sgagg_status sgagg_server_create(const sgagg_server_config* cfg, const sgagg_spec* spec, sgagg_server_t* out) {
  if (!out) return SGAGG_EINVAL;
  *out = nullptr;
  if (!config_ok(cfg) || !spec || spec->n_aggs < 0 || (spec->n_aggs > 0 && !spec->aggs)) return SGAGG_EINVAL;
  sgagg_server* s = new sgagg_server(*cfg);
  s->aggs.assign(spec->aggs, spec->aggs + spec->n_aggs);
  s->spec.n_aggs = spec->n_aggs;
  s->spec.aggs = s->aggs.data();
  cudaGetDevice(&s->device);
  s->slots.resize((size_t)cfg->slots);
  sgagg_status st = SGAGG_OK;
  for (auto& sl : s->slots) {
    if ((st = sgagg_create(cfg->memory_budget_rows, &sl.h)) != SGAGG_OK) break;
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess) {
      st = SGAGG_ECUDA;
      break;
    }
  }
  if (st != SGAGG_OK) {
    for (auto& sl : s->slots) {
      if (sl.h) sgagg_destroy(sl.h);
      if (sl.st) cudaStreamDestroy(sl.st);
    }
    delete s;
    return st;
  }
  for (int i = 0; i < cfg->slots; ++i) s->slots[(size_t)i].th = std::thread(worker, s, i);
  *out = s;
  return SGAGG_OK;
}

sgagg_status sgagg_server_submit(sgagg_server_t s, const sgagg_request* req, int64_t* ticket) {
  if (!s || !req || !ticket) return SGAGG_EINVAL;
  const sgagg_request& r = *req;
  const int kb = r.key_bytes;
  if (kb != 1 && kb != 2 && kb != 4 && kb != 8) return SGAGG_EINVAL;
  if (r.n < 0 || r.out_capacity < 0 || r.n_payload < 0 || r.n_payload > 1024) return SGAGG_EINVAL;
  if (r.n > 0 && (!r.keys || (r.n_payload > 0 && !r.payload))) return SGAGG_EINVAL;
  if (s->spec.n_aggs > 0 && !r.out_aggs) return SGAGG_EINVAL;
  for (int a = 0; a < s->spec.n_aggs; ++a)
    if (s->spec.aggs[a].op != SGAGG_COUNT && s->spec.aggs[a].col >= r.n_payload) return SGAGG_EINVAL;
  const int64_t fp = sgagg_request_footprint(r.n, kb, r.n_payload, s->spec.n_aggs, r.out_capacity,
                                             s->cfg.memory_budget_rows);
  if (fp > s->cfg.device_budget_bytes) return SGAGG_ECAPACITY;
  Req* q = new Req();
  q->r = r;
  if (r.n_payload > 0 && r.payload) q->pay.assign(r.payload, r.payload + r.n_payload);
  q->pay.resize((size_t)std::max(1, r.n_payload), nullptr);
  if (s->spec.n_aggs > 0) q->oa.assign(r.out_aggs, r.out_aggs + s->spec.n_aggs);
  q->oa.resize((size_t)std::max(1, s->spec.n_aggs), nullptr);
  q->r.payload = nullptr;
  q->r.out_aggs = nullptr;
  q->res = sgagg_request_result{};
  q->res.status = SGAGG_OK;
  q->res.slot = -1;
  q->res.rows = -1;
  q->res.submit_ns = clock_ns();
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t t = s->next_ticket++;
  s->reqs[t] = q;
  s->sched.push(Pending{t, r.n, fp, batchable(s->cfg, r.n, kb)});
  *ticket = t;
  s->cv.notify_all();
  return SGAGG_OK;
}

sgagg_status sgagg_server_poll(sgagg_server_t s, int64_t ticket, int32_t* done, sgagg_request_result* out) {
  if (!s || !done || !out) return SGAGG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SGAGG_EINVAL;
  *done = it->second->done ? 1 : 0;
  if (*done) {
    *out = it->second->res;
    delete it->second;
    s->reqs.erase(it);
  }
  return SGAGG_OK;
}

sgagg_status sgagg_server_wait(sgagg_server_t s, int64_t ticket, sgagg_request_result* out) {
  if (!s || !out) return SGAGG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SGAGG_EINVAL;
  Req* q = it->second;
  s->cv.wait(lk, [q] { return q->done; });
  *out = q->res;
  delete q;
  s->reqs.erase(ticket);
  return SGAGG_OK;
}

void sgagg_server_destroy(sgagg_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  for (auto& sl : s->slots)
    if (sl.th.joinable()) sl.th.join();
  for (auto& sl : s->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.h) sgagg_destroy(sl.h);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.dptr) cudaFree(sl.dptr);
    if (sl.hptr) cudaFreeHost(sl.hptr);
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
}

sgagg_status sgagg_server_simulate(const sgagg_server_config* cfg, int32_t n_payload, int32_t n_aggs, int32_t count,
                                   const int64_t* rows, const double* arrive_us, const double* cost_us,
                                   double* start_us, double* finish_us, int32_t* slot, int32_t* batch) {
  if (!config_ok(cfg) || count < 0 || n_payload < 0 || n_aggs < 0) return SGAGG_EINVAL;
  if (count > 0 && (!rows || !arrive_us || !cost_us || !start_us || !finish_us || !slot || !batch))
    return SGAGG_EINVAL;
  std::vector<int> order((size_t)count);
  for (int i = 0; i < count; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return arrive_us[a] < arrive_us[b]; });
  Scheduler sched(*cfg);
  struct Run {
    double finish;
    int slot;
    int64_t fp;
    bool operator>(const Run& o) const { return finish > o.finish; }
  };
  std::priority_queue<Run, std::vector<Run>, std::greater<Run>> running;
  size_t next = 0;
  int nbatch = 0;
  double t = 0.0;
  for (;;) {
    const bool have_a = next < order.size();
    const bool have_f = !running.empty();
    if (!have_a && !have_f) break;
    if (have_a && (!have_f || arrive_us[order[next]] <= running.top().finish)) {
      const int i = order[next++];
      t = std::max(t, arrive_us[i]);
      if (rows[i] < 0) return SGAGG_EINVAL;
      const int64_t fp = sgagg_request_footprint(rows[i], 8, n_payload, n_aggs, rows[i], cfg->memory_budget_rows);
      if (fp > cfg->device_budget_bytes) {
        start_us[i] = finish_us[i] = t;
        slot[i] = -1;
        batch[i] = -1;
      } else {
        sched.push(Pending{i, rows[i], fp, batchable(*cfg, rows[i], 8)});
      }
    } else {
      const Run r = running.top();
      running.pop();
      t = r.finish;
      sched.done(r.slot, r.fp);
    }
    std::vector<int64_t> ids;
    int64_t r = 0, fp = 0;
    int sl = -1;
    while (sched.next(-1, &ids, &r, &fp, &sl)) {
      const double dur = cost_us[0] + cost_us[1] * (double)r + cost_us[2] * (double)ids.size();
      for (int64_t id : ids) {
        start_us[id] = t;
        finish_us[id] = t + dur;
        slot[id] = sl;
        batch[id] = nbatch;
      }
      ++nbatch;
      running.push(Run{t + dur, sl, fp});
    }
  }
  return SGAGG_OK;
}

}  // extern "C"
