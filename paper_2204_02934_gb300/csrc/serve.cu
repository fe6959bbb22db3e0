// serve.cu -- a request loop for coarsening requests (one level: MIS-2,
// aggregation, coarse graph per request) with continuous batching: requests
// are admitted as device memory and execution slots free up, each slot owns
// a resident context (status arrays, worklists, staging buffers) and its own
// stream, so requests admitted while others run overlap on the GPU.
//
// A request's result does not depend on what else runs: every slot computes
// with its own scratch, and the computation itself is deterministic.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

uint64_t fnv1a(uint64_t h, const void* p, size_t bytes) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < bytes; i++) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct Request {
  int64_t ticket = 0;
  mis2_csr g{};
  uint64_t seed = 0;
  int64_t need = 0;  // bytes charged against the memory budget
  Clock::time_point t_arrive;
};

struct Slot {
  mis2_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  uint8_t* in_set = nullptr;  // pinned host outputs
  int32_t *roots = nullptr, *labels = nullptr, *c_rowptr = nullptr, *c_colind = nullptr;
  int64_t cap_cci = 0;
};

}  // namespace

struct mis2_server {
  mis2_server_config cfg{};
  std::vector<Slot> slots;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::vector<mis2_result> done;  // indexed by ticket
  std::vector<char> finished;
  int64_t next_ticket = 0;
  int64_t mem_in_use = 0;
  int64_t max_in_flight = 0, in_flight = 0;
  bool stop = false;
  int device = 0;
  Clock::time_point t0;
};

namespace {

// Bytes a request holds on the device while it runs: its CSR and outputs
// (the slot's scratch is resident and charged once at creation).
int64_t request_bytes(const mis2_csr& g) {
  const int64_t rp = (g.n + 1) * (g.rowptr_is_64 ? 8 : 4);
  return rp + 4 * g.nnz + g.n * (1 + 4 + 4) + 4 * (g.n + 1) + 4 * g.nnz;
}

double secs(const mis2_server* s, Clock::time_point t) {
  return std::chrono::duration<double>(t - s->t0).count();
}

void worker_main(mis2_server* s, int slot_id) {
  cudaSetDevice(s->device);
  Slot& sl = s->slots[slot_id];
  for (;;) {
    Request rq;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // admission: FIFO head, a free slot (this thread) and room in the budget
      s->cv_work.wait(lk, [&] {
        return s->stop || (!s->queue.empty() && s->mem_in_use + s->queue.front().need <= s->cfg.mem_budget);
      });
      if (s->stop && s->queue.empty()) return;
      rq = s->queue.front();
      s->queue.pop_front();
      s->mem_in_use += rq.need;
      s->in_flight++;
      s->max_in_flight = std::max(s->max_in_flight, s->in_flight);
    }
    mis2_result res{};
    res.ticket = rq.ticket;
    res.slot = slot_id;
    res.n = rq.g.n;
    res.nnz = rq.g.nnz;
    res.t_arrive = secs(s, rq.t_arrive);
    res.t_start = secs(s, Clock::now());
    int64_t nr = 0, na = 0, cn = 0;
    int rc = mis2_coarsen_level_host(sl.ctx, &rq.g, rq.seed, sl.in_set, sl.roots, sl.labels, sl.c_rowptr,
                                     sl.c_colind, sl.cap_cci, &nr, &na, &cn, sl.stream);
    res.t_done = secs(s, Clock::now());
    res.status = rc;
    if (rc == MIS2_OK) {
      res.n_roots = nr;
      res.n_aggs = na;
      res.c_nnz = cn;
      uint64_t h = 1469598103934665603ull;
      h = fnv1a(h, sl.roots, (size_t)nr * 4);
      h = fnv1a(h, sl.labels, (size_t)rq.g.n * 4);
      h = fnv1a(h, sl.c_rowptr, (size_t)(na + 1) * 4);
      h = fnv1a(h, sl.c_colind, (size_t)cn * 4);
      res.checksum = h;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->mem_in_use -= rq.need;
      s->in_flight--;
      s->done[rq.ticket] = res;
      s->finished[rq.ticket] = 1;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
}

}  // namespace

using namespace mis2;

extern "C" {

void mis2_server_config_default(mis2_server_config* c) {
  if (c == nullptr) return;
  memset(c, 0, sizeof(*c));
  c->slots = 4;
  c->mem_budget = (int64_t)8 << 30;
  c->slot_max_n = (int64_t)1 << 22;
  c->slot_max_nnz = (int64_t)1 << 25;
  mis2_config_default(&c->cfg);
  c->cfg.loop = MIS2_LOOP_HOST;
}

int mis2_server_create(mis2_server** out, const mis2_server_config* cfg) {
  if (out == nullptr || cfg == nullptr) return MIS2_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->slots < 1 || cfg->slots > 64 || cfg->slot_max_n < 1 || cfg->slot_max_nnz < 1 || cfg->mem_budget < 1)
    return MIS2_ERR_INVALID_ARG;
  mis2_server* s = new mis2_server();
  s->cfg = *cfg;
  s->t0 = Clock::now();
  cudaGetDevice(&s->device);
  s->slots.resize(cfg->slots);
  for (int i = 0; i < cfg->slots; i++) {
    Slot& sl = s->slots[i];
    int rc = mis2_ctx_create(&sl.ctx, cfg->slot_max_n, cfg->slot_max_nnz, &cfg->cfg);
    if (rc == MIS2_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
      rc = MIS2_ERR_CUDA;
    if (rc != MIS2_OK) {
      mis2_server_destroy(s);
      return rc;
    }
    const int64_t n = cfg->slot_max_n, nnz = cfg->slot_max_nnz;
    sl.cap_cci = nnz;
    if (cudaMallocHost(&sl.in_set, n) != cudaSuccess || cudaMallocHost(&sl.roots, 4 * n) != cudaSuccess ||
        cudaMallocHost(&sl.labels, 4 * n) != cudaSuccess || cudaMallocHost(&sl.c_rowptr, 4 * (n + 1)) != cudaSuccess ||
        cudaMallocHost(&sl.c_colind, 4 * nnz) != cudaSuccess) {
      mis2_server_destroy(s);
      return MIS2_ERR_OUT_OF_MEMORY;
    }
    // one tiny request sets up the slot's staging buffers before serving
    int64_t rp[2] = {0, 0};
    mis2_csr tiny{1, 0, 1, 0, rp, nullptr};
    int64_t a, b2, c2;
    rc = mis2_coarsen_level_host(sl.ctx, &tiny, 0, sl.in_set, sl.roots, sl.labels, sl.c_rowptr, sl.c_colind,
                                 sl.cap_cci, &a, &b2, &c2, sl.stream);
    if (rc != MIS2_OK) {
      mis2_server_destroy(s);
      return rc;
    }
  }
  for (int i = 0; i < cfg->slots; i++) s->workers.emplace_back(worker_main, s, i);
  *out = s;
  return MIS2_OK;
}

int mis2_server_destroy(mis2_server* s) {
  if (s == nullptr) return MIS2_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& sl : s->slots) {
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ctx) mis2_ctx_destroy(sl.ctx);
    for (void* p : {(void*)sl.in_set, (void*)sl.roots, (void*)sl.labels, (void*)sl.c_rowptr, (void*)sl.c_colind})
      if (p) cudaFreeHost(p);
  }
  delete s;
  return MIS2_OK;
}

int mis2_server_submit(mis2_server* s, const mis2_csr* g_host, uint64_t seed, int64_t* ticket) {
  if (s == nullptr || g_host == nullptr || ticket == nullptr) return MIS2_ERR_INVALID_ARG;
  if (g_host->n < 0 || g_host->nnz < 0 || g_host->rowptr == nullptr) return MIS2_ERR_INVALID_ARG;
  if (g_host->n > s->cfg.slot_max_n || g_host->nnz > s->cfg.slot_max_nnz) return MIS2_ERR_OUT_OF_MEMORY;
  Request rq;
  rq.g = *g_host;
  rq.seed = seed;
  rq.need = request_bytes(*g_host);
  if (rq.need > s->cfg.mem_budget) return MIS2_ERR_OUT_OF_MEMORY;
  rq.t_arrive = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    rq.ticket = s->next_ticket++;
    s->done.emplace_back();
    s->finished.push_back(0);
    s->queue.push_back(rq);
  }
  s->cv_work.notify_all();
  *ticket = rq.ticket;
  return MIS2_OK;
}

int mis2_server_wait(mis2_server* s, int64_t ticket, mis2_result* out) {
  if (s == nullptr || out == nullptr) return MIS2_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket < 0 || ticket >= s->next_ticket) return MIS2_ERR_INVALID_ARG;
  s->cv_done.wait(lk, [&] { return s->finished[ticket] != 0; });
  *out = s->done[ticket];
  return MIS2_OK;
}

int mis2_server_replay(mis2_server* s, int32_t n_pool, const mis2_csr* pool_host, int64_t n_req,
                       const double* arrival_s, const int32_t* pool_index, uint64_t seed, mis2_result* results,
                       int64_t* max_in_flight) {
  if (s == nullptr || pool_host == nullptr || arrival_s == nullptr || pool_index == nullptr || results == nullptr ||
      n_pool < 1 || n_req < 0)
    return MIS2_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->max_in_flight = 0;
  }
  std::vector<int64_t> tickets(n_req);
  const Clock::time_point start = Clock::now();
  for (int64_t i = 0; i < n_req; i++) {
    if (pool_index[i] < 0 || pool_index[i] >= n_pool) return MIS2_ERR_INVALID_ARG;
    const Clock::time_point due =
        start + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
    std::this_thread::sleep_until(due);
    MIS2_TRY(mis2_server_submit(s, &pool_host[pool_index[i]], seed, &tickets[i]));
  }
  for (int64_t i = 0; i < n_req; i++) MIS2_TRY(mis2_server_wait(s, tickets[i], &results[i]));
  if (max_in_flight) {
    std::lock_guard<std::mutex> lk(s->mu);
    *max_in_flight = s->max_in_flight;
  }
  return MIS2_OK;
}

}  // extern "C"
