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

// SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Adds sum_i mix(mix((k << 40) + i) ^ (uint32)a[i]) to *out (mod 2^64): a
// position-dependent fingerprint whose value does not depend on the order in
// which the terms are added.
__global__ void k_fingerprint(const int32_t* a, int64_t n, uint64_t k, unsigned long long* out) {
  uint64_t acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += mix64(mix64((k << 40) + (uint64_t)i) ^ (uint64_t)(uint32_t)a[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0) atomicAdd(out, (unsigned long long)acc);
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
  unsigned long long* d_sum = nullptr;  // device fingerprint accumulator
  unsigned long long* h_sum = nullptr;  // pinned landing
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
  std::mutex coop_mu;  // one device-loop kernel of the slots at a time
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

// Fingerprint of the slot's last results (the device copies the host-buffer
// entry point left in the context's stage).
int fingerprint(mis2_ctx* c, Slot& sl, int64_t n, int64_t nr, int64_t na, int64_t cn, uint64_t* out) {
  const mis2::HostStage& h = c->stage;
  MIS2_CUDA(cudaMemsetAsync(sl.d_sum, 0, sizeof(unsigned long long), sl.stream));
  const int32_t* arr[4] = {h.roots, h.labels, h.c_rowptr, h.c_colind};
  const int64_t len[4] = {nr, n, na + 1, cn};
  for (int k = 0; k < 4; k++) {
    if (len[k] <= 0) continue;
    const int blocks = (int)std::min<int64_t>((len[k] + 255) / 256, (int64_t)c->sm_count * 4);
    k_fingerprint<<<blocks, 256, 0, sl.stream>>>(arr[k], len[k], (uint64_t)k, sl.d_sum);
  }
  MIS2_CUDA(cudaGetLastError());
  MIS2_CUDA(cudaMemcpyAsync(sl.h_sum, sl.d_sum, sizeof(unsigned long long), cudaMemcpyDeviceToHost, sl.stream));
  MIS2_CUDA(cudaStreamSynchronize(sl.stream));
  uint64_t f = *sl.h_sum;
  const int64_t cnt[3] = {nr, na, cn};
  for (int j = 0; j < 3; j++) f += mix64(((uint64_t)(5 + j) << 40) ^ (uint64_t)cnt[j]);
  *out = f;
  return MIS2_OK;
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
      res.status = fingerprint(sl.ctx, sl, rq.g.n, nr, na, cn, &res.checksum);
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
  c->cfg.loop = MIS2_LOOP_DEVICE;
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
    if (rc == MIS2_OK && cudaEventCreateWithFlags(&sl.ctx->coop_done, cudaEventDisableTiming) != cudaSuccess)
      rc = MIS2_ERR_CUDA;
    if (rc == MIS2_OK) sl.ctx->coop_lock = &s->coop_mu;
    if (rc != MIS2_OK) {
      mis2_server_destroy(s);
      return rc;
    }
    const int64_t n = cfg->slot_max_n, nnz = cfg->slot_max_nnz;
    sl.cap_cci = nnz;
    if (cudaMallocHost(&sl.in_set, n) != cudaSuccess || cudaMallocHost(&sl.roots, 4 * n) != cudaSuccess ||
        cudaMallocHost(&sl.labels, 4 * n) != cudaSuccess || cudaMallocHost(&sl.c_rowptr, 4 * (n + 1)) != cudaSuccess ||
        cudaMallocHost(&sl.c_colind, 4 * nnz) != cudaSuccess || cudaMalloc(&sl.d_sum, 8) != cudaSuccess ||
        cudaMallocHost(&sl.h_sum, 8) != cudaSuccess) {
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
    if (sl.ctx && sl.ctx->coop_done) cudaEventDestroy(sl.ctx->coop_done);
    if (sl.ctx) mis2_ctx_destroy(sl.ctx);
    for (void* p : {(void*)sl.in_set, (void*)sl.roots, (void*)sl.labels, (void*)sl.c_rowptr, (void*)sl.c_colind,
                    (void*)sl.h_sum})
      if (p) cudaFreeHost(p);
    if (sl.d_sum) cudaFree(sl.d_sum);
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

int mis2_server_cancel(mis2_server* s, int64_t ticket, int32_t* cancelled) {
  if (s == nullptr || cancelled == nullptr) return MIS2_ERR_INVALID_ARG;
  *cancelled = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket < 0 || ticket >= s->next_ticket) return MIS2_ERR_INVALID_ARG;
    auto it = std::find_if(s->queue.begin(), s->queue.end(), [&](const Request& r) { return r.ticket == ticket; });
    if (it == s->queue.end()) return MIS2_OK;  // running or finished: its result stands
    mis2_result res{};
    res.ticket = ticket;
    res.n = it->g.n;
    res.nnz = it->g.nnz;
    res.t_arrive = secs(s, it->t_arrive);
    res.t_start = res.t_done = secs(s, Clock::now());
    res.status = MIS2_ERR_CANCELLED;
    res.slot = -1;
    s->queue.erase(it);
    s->done[ticket] = res;
    s->finished[ticket] = 1;
    *cancelled = 1;
  }
  s->cv_work.notify_all();  // the new queue head may fit the budget
  s->cv_done.notify_all();
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
