// serve.cu -- a request loop for coarsening requests (one level: MIS-2,
// aggregation, coarse graph per request) with continuous batching: requests
// are admitted as device memory and execution slots free up, each slot owns
// a resident context (status arrays, worklists, staging buffers) and its own
// stream, so requests admitted while others run overlap on the GPU.
//
// With batch_max >= 2 a slot instead takes every queued request that fits
// (same seed, at most batch_max, its union capacity in total) and runs them
// as one block-diagonal union through the batched engine: one persistent
// MIS-2 launch, one aggregation and one coarse-graph pass for all of them,
// each graph keeping the tuples, ids and tie-breaks it would have alone.
//
// A request's result does not depend on what else runs: every slot computes
// with its own scratch, the union preserves each graph's computation, and
// the computation itself is deterministic.
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
  mis2_request_out out{};  // caller's result buffers (null pointers: not returned)
};

struct Slot {
  mis2_ctx* ctx = nullptr;      // one request at a time (batch_max <= 1)
  mis2_batch* batch = nullptr;  // merged requests (batch_max >= 2)
  cudaStream_t stream = nullptr;
  uint8_t* in_set = nullptr;  // pinned host outputs
  int32_t *roots = nullptr, *labels = nullptr, *c_rowptr = nullptr, *c_colind = nullptr;
  int64_t cap_cci = 0;
  unsigned long long* d_sum = nullptr;  // device fingerprint accumulator
  unsigned long long* h_sum = nullptr;  // pinned landing
  // batch_max >= 2: device staging of the merged requests' CSRs and of one
  // request's results
  unsigned char* d_rp = nullptr;
  int32_t* d_ci = nullptr;
  int32_t *d_roots = nullptr, *d_labels = nullptr, *d_crp = nullptr, *d_cci = nullptr;
  int64_t cap_rp_bytes = 0, cap_ci = 0;
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

// The array terms of one request's fingerprint, summed into *acc on the
// stream (no synchronisation): roots[nr], labels[n], c_rowptr[na + 1],
// c_colind[cn] in device memory.
int fingerprint_enqueue(cudaStream_t st, int sm_count, const int32_t* roots, const int32_t* labels,
                        const int32_t* c_rowptr, const int32_t* c_colind, int64_t n, int64_t nr, int64_t na,
                        int64_t cn, unsigned long long* acc) {
  MIS2_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), st));
  const int32_t* arr[4] = {roots, labels, c_rowptr, c_colind};
  const int64_t len[4] = {nr, n, na + 1, cn};
  for (int k = 0; k < 4; k++) {
    if (len[k] <= 0) continue;
    const int blocks = (int)std::min<int64_t>((len[k] + 255) / 256, (int64_t)sm_count * 4);
    k_fingerprint<<<blocks, 256, 0, st>>>(arr[k], len[k], (uint64_t)k, acc);
  }
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

// The fingerprint from the summed array terms and the three counts.
uint64_t fingerprint_counts(uint64_t f, int64_t nr, int64_t na, int64_t cn) {
  const int64_t cnt[3] = {nr, na, cn};
  for (int j = 0; j < 3; j++) f += mix64(((uint64_t)(5 + j) << 40) ^ (uint64_t)cnt[j]);
  return f;
}

// Fingerprint of one request's results in device memory (synchronises).
int fingerprint_of(Slot& sl, int sm_count, const int32_t* roots, const int32_t* labels, const int32_t* c_rowptr,
                   const int32_t* c_colind, int64_t n, int64_t nr, int64_t na, int64_t cn, uint64_t* out) {
  MIS2_TRY(fingerprint_enqueue(sl.stream, sm_count, roots, labels, c_rowptr, c_colind, n, nr, na, cn, sl.d_sum));
  MIS2_CUDA(cudaMemcpyAsync(sl.h_sum, sl.d_sum, sizeof(unsigned long long), cudaMemcpyDeviceToHost, sl.stream));
  MIS2_CUDA(cudaStreamSynchronize(sl.stream));
  *out = fingerprint_counts(*sl.h_sum, nr, na, cn);
  return MIS2_OK;
}

// Fingerprint of the slot's last results (the device copies the host-buffer
// entry point left in the context's stage).
int fingerprint(mis2_ctx* c, Slot& sl, int64_t n, int64_t nr, int64_t na, int64_t cn, uint64_t* out) {
  const mis2::HostStage& h = c->stage;
  return fingerprint_of(sl, c->sm_count, h.roots, h.labels, h.c_rowptr, h.c_colind, n, nr, na, cn, out);
}

// The request's results, from host copies (the slot's pinned buffers at the
// request's offsets), into the caller's buffers.
int deliver(const Request& rq, const uint8_t* in_set, const int32_t* roots, const int32_t* labels,
            const int32_t* c_rowptr, const int32_t* c_colind, int64_t nr, int64_t na, int64_t cn) {
  const mis2_request_out& o = rq.out;
  const int64_t n = rq.g.n;
  if (o.c_colind != nullptr && cn > o.c_colind_cap) return MIS2_ERR_INVALID_ARG;
  if (o.in_set && n > 0) memcpy(o.in_set, in_set, (size_t)n);
  if (o.roots && nr > 0) memcpy(o.roots, roots, (size_t)nr * 4);
  if (o.labels && n > 0) memcpy(o.labels, labels, (size_t)n * 4);
  if (o.c_rowptr) memcpy(o.c_rowptr, c_rowptr, (size_t)(na + 1) * 4);
  if (o.c_colind && cn > 0) memcpy(o.c_colind, c_colind, (size_t)cn * 4);
  return MIS2_OK;
}

void finish(mis2_server* s, const std::vector<Request>& rqs, std::vector<mis2_result>& res) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < rqs.size(); i++) {
      s->mem_in_use -= rqs[i].need;
      s->in_flight--;
      s->done[rqs[i].ticket] = res[i];
      s->finished[rqs[i].ticket] = 1;
    }
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
}

// Merged launches (batch_max >= 2): the queued requests that fit run as one
// union; each then gets its results renumbered, fingerprinted, copied to the
// host and delivered in turn.
void worker_batch_main(mis2_server* s, int slot_id) {
  cudaSetDevice(s->device);
  Slot& sl = s->slots[slot_id];
  mis2_ctx* bc = mis2::batch_context(sl.batch);
  std::vector<Request> rqs;
  std::vector<mis2_result> res;
  std::vector<mis2_csr> dg;
  for (;;) {
    rqs.clear();
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        return s->stop || (!s->queue.empty() && s->mem_in_use + s->queue.front().need <= s->cfg.mem_budget);
      });
      if (s->stop && s->queue.empty()) return;
      int64_t sn = 0, snnz = 0, need = 0;
      while (!s->queue.empty() && (int)rqs.size() < s->cfg.batch_max) {
        const Request& h = s->queue.front();
        if (!rqs.empty() && (h.seed != rqs[0].seed || sn + h.g.n > s->cfg.slot_max_n ||
                             snnz + h.g.nnz > s->cfg.slot_max_nnz ||
                             s->mem_in_use + need + h.need > s->cfg.mem_budget))
          break;
        sn += h.g.n;
        snnz += h.g.nnz;
        need += h.need;
        rqs.push_back(h);
        s->queue.pop_front();
      }
      s->mem_in_use += need;
      s->in_flight += (int64_t)rqs.size();
      s->max_in_flight = std::max(s->max_in_flight, s->in_flight);
    }
    const double t_start = secs(s, Clock::now());
    res.assign(rqs.size(), mis2_result{});
    for (size_t i = 0; i < rqs.size(); i++) {
      res[i].ticket = rqs[i].ticket;
      res[i].slot = slot_id;
      res[i].n = rqs[i].g.n;
      res[i].nnz = rqs[i].g.nnz;
      res[i].t_arrive = secs(s, rqs[i].t_arrive);
      res[i].t_start = t_start;
    }
    // inputs to the device: rowptr regions 16-byte aligned, colind regions
    // padded to 4 entries (keeps 16-byte loads aligned)
    int rc = MIS2_OK;
    dg.assign(rqs.size(), mis2_csr{});
    int64_t rp_off = 0, ci_off = 0;
    for (size_t i = 0; i < rqs.size() && rc == MIS2_OK; i++) {
      const mis2_csr& g = rqs[i].g;
      const int64_t rp_bytes = (g.n + 1) * (g.rowptr_is_64 ? 8 : 4);
      dg[i] = g;
      dg[i].rowptr = sl.d_rp + rp_off;
      dg[i].colind = sl.d_ci + ci_off;
      if (cudaMemcpyAsync(sl.d_rp + rp_off, g.rowptr, (size_t)rp_bytes, cudaMemcpyHostToDevice, sl.stream) !=
              cudaSuccess ||
          (g.nnz > 0 && cudaMemcpyAsync(sl.d_ci + ci_off, g.colind, (size_t)g.nnz * 4, cudaMemcpyHostToDevice,
                                        sl.stream) != cudaSuccess))
        rc = mis2::set_cuda_error(cudaGetLastError());
      rp_off += (rp_bytes + 15) / 16 * 16;
      ci_off += (g.nnz + 3) / 4 * 4;
    }
    int32_t levels = 0;
    if (rc == MIS2_OK)
      rc = mis2_batch_coarsen(sl.batch, (int32_t)rqs.size(), dg.data(), rqs[0].seed, 1, 1, &levels, sl.stream);
    // every request's results: renumbered into its own region of the
    // slot's device buffers, fingerprinted and copied to the host, all
    // queued before one synchronisation
    std::vector<int64_t> nr(rqs.size(), 0), na(rqs.size(), 0), cn(rqs.size(), 0);
    std::vector<int64_t> vo(rqs.size() + 1, 0), eo(rqs.size() + 1, 0);
    std::vector<int> st_i(rqs.size(), rc);
    for (size_t i = 0; i < rqs.size(); i++) {
      vo[i + 1] = vo[i] + rqs[i].g.n + 1;  // + 1: room for c_rowptr's last entry
      eo[i + 1] = eo[i] + rqs[i].g.nnz;
    }
    for (size_t i = 0; i < rqs.size(); i++) {
      int& r = st_i[i];
      const int64_t n = rqs[i].g.n;
      int32_t *roots = sl.d_roots + vo[i], *labels = sl.d_labels + vo[i], *crp = sl.d_crp + vo[i],
              *cci = sl.d_cci + eo[i];
      if (r == MIS2_OK && n > 0)
        r = mis2::batch_level0_result(sl.batch, (int32_t)i, roots, labels, crp, cci, &nr[i], &na[i], &cn[i],
                                      sl.stream);
      if (r == MIS2_OK && n == 0 && cudaMemsetAsync(crp, 0, sizeof(int32_t), sl.stream) != cudaSuccess)
        r = MIS2_ERR_CUDA;
      if (r == MIS2_OK)
        r = fingerprint_enqueue(sl.stream, bc->sm_count, roots, labels, crp, cci, n, nr[i], na[i], cn[i],
                                sl.d_sum + i);
      if (r == MIS2_OK &&
          ((nr[i] > 0 && cudaMemcpyAsync(sl.roots + vo[i], roots, (size_t)nr[i] * 4, cudaMemcpyDeviceToHost,
                                         sl.stream) != cudaSuccess) ||
           (n > 0 && cudaMemcpyAsync(sl.labels + vo[i], labels, (size_t)n * 4, cudaMemcpyDeviceToHost, sl.stream) !=
                         cudaSuccess) ||
           cudaMemcpyAsync(sl.c_rowptr + vo[i], crp, (size_t)(na[i] + 1) * 4, cudaMemcpyDeviceToHost, sl.stream) !=
               cudaSuccess ||
           (cn[i] > 0 && cudaMemcpyAsync(sl.c_colind + eo[i], cci, (size_t)cn[i] * 4, cudaMemcpyDeviceToHost,
                                         sl.stream) != cudaSuccess)))
        r = mis2::set_cuda_error(cudaGetLastError());
    }
    if (cudaMemcpyAsync(sl.h_sum, sl.d_sum, rqs.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        sl.stream) != cudaSuccess ||
        cudaStreamSynchronize(sl.stream) != cudaSuccess) {
      const int e = mis2::set_cuda_error(cudaGetLastError());
      for (int& r : st_i)
        if (r == MIS2_OK) r = e;
    }
    const double t_done = secs(s, Clock::now());
    for (size_t i = 0; i < rqs.size(); i++) {
      int r = st_i[i];
      const int64_t n = rqs[i].g.n;
      if (r == MIS2_OK && n > 0) {
        uint8_t* fl = sl.in_set + vo[i];
        memset(fl, 0, (size_t)n);
        for (int64_t k = 0; k < nr[i]; k++) fl[sl.roots[vo[i] + k]] = 1;
      }
      if (r == MIS2_OK) {
        res[i].checksum = fingerprint_counts(sl.h_sum[i], nr[i], na[i], cn[i]);
        r = deliver(rqs[i], sl.in_set + vo[i], sl.roots + vo[i], sl.labels + vo[i], sl.c_rowptr + vo[i],
                    sl.c_colind + eo[i], nr[i], na[i], cn[i]);
      }
      res[i].status = r;
      res[i].n_roots = nr[i];
      res[i].n_aggs = na[i];
      res[i].c_nnz = cn[i];
      res[i].t_done = t_done;
    }
    finish(s, rqs, res);
  }
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
      if (res.status == MIS2_OK)
        res.status = deliver(rq, sl.in_set, sl.roots, sl.labels, sl.c_rowptr, sl.c_colind, nr, na, cn);
    }
    std::vector<Request> one{rq};
    std::vector<mis2_result> r1{res};
    finish(s, one, r1);
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
  // several slots: the host-driven rounds of different requests interleave
  // on the GPU, where device-loop kernels would run one at a time
  c->cfg.loop = MIS2_LOOP_HOST;
}

int mis2_server_create(mis2_server** out, const mis2_server_config* cfg) {
  if (out == nullptr || cfg == nullptr) return MIS2_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->slots < 1 || cfg->slots > 64 || cfg->slot_max_n < 1 || cfg->slot_max_nnz < 1 || cfg->mem_budget < 1 ||
      cfg->batch_max < 0 || cfg->batch_max > 4096)
    return MIS2_ERR_INVALID_ARG;
  mis2_server* s = new mis2_server();
  s->cfg = *cfg;
  s->t0 = Clock::now();
  cudaGetDevice(&s->device);
  s->slots.resize(cfg->slots);
  for (int i = 0; i < cfg->slots; i++) {
    Slot& sl = s->slots[i];
    const bool merged = cfg->batch_max >= 2;
    int rc = merged ? mis2_batch_create(&sl.batch, cfg->batch_max, cfg->slot_max_n, cfg->slot_max_nnz, &cfg->cfg)
                    : mis2_ctx_create(&sl.ctx, cfg->slot_max_n, cfg->slot_max_nnz, &cfg->cfg);
    mis2_ctx* lc = merged ? (sl.batch ? mis2::batch_context(sl.batch) : nullptr) : sl.ctx;
    if (rc == MIS2_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
      rc = MIS2_ERR_CUDA;
    if (rc == MIS2_OK && cudaEventCreateWithFlags(&lc->coop_done, cudaEventDisableTiming) != cudaSuccess)
      rc = MIS2_ERR_CUDA;
    if (rc == MIS2_OK) lc->coop_lock = &s->coop_mu;
    if (rc != MIS2_OK) {
      mis2_server_destroy(s);
      return rc;
    }
    const int64_t n = cfg->slot_max_n, nnz = cfg->slot_max_nnz;
    if (merged) {
      sl.cap_rp_bytes = 8 * (n + cfg->batch_max) + 16 * (int64_t)cfg->batch_max;
      sl.cap_ci = nnz + 4 * (int64_t)cfg->batch_max;
      const int64_t nb = n + cfg->batch_max;  // every request's region has one extra entry
      if (cudaMalloc(&sl.d_rp, (size_t)sl.cap_rp_bytes) != cudaSuccess ||
          cudaMalloc(&sl.d_ci, (size_t)sl.cap_ci * 4) != cudaSuccess ||
          cudaMalloc(&sl.d_roots, (size_t)nb * 4) != cudaSuccess || cudaMalloc(&sl.d_labels, (size_t)nb * 4) != cudaSuccess ||
          cudaMalloc(&sl.d_crp, (size_t)nb * 4) != cudaSuccess ||
          cudaMalloc(&sl.d_cci, (size_t)std::max<int64_t>(nnz, 1) * 4) != cudaSuccess) {
        cudaGetLastError();
        mis2_server_destroy(s);
        return MIS2_ERR_OUT_OF_MEMORY;
      }
    }
    sl.cap_cci = nnz;
    const int64_t nh = n + std::max(cfg->batch_max, 1);  // merged: one extra entry per request region
    const size_t sums = 8 * (size_t)std::max(cfg->batch_max, 1);
    if (cudaMallocHost(&sl.in_set, nh) != cudaSuccess || cudaMallocHost(&sl.roots, 4 * nh) != cudaSuccess ||
        cudaMallocHost(&sl.labels, 4 * nh) != cudaSuccess || cudaMallocHost(&sl.c_rowptr, 4 * nh) != cudaSuccess ||
        cudaMallocHost(&sl.c_colind, 4 * nnz) != cudaSuccess || cudaMalloc(&sl.d_sum, sums) != cudaSuccess ||
        cudaMallocHost(&sl.h_sum, sums) != cudaSuccess) {
      mis2_server_destroy(s);
      return MIS2_ERR_OUT_OF_MEMORY;
    }
    // one tiny request sets up the slot's staging buffers before serving
    if (!merged) {
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
  }
  for (int i = 0; i < cfg->slots; i++)
    s->workers.emplace_back(cfg->batch_max >= 2 ? worker_batch_main : worker_main, s, i);
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
    mis2_ctx* lc = sl.batch ? mis2::batch_context(sl.batch) : sl.ctx;
    if (lc && lc->coop_done) cudaEventDestroy(lc->coop_done);
    if (sl.ctx) mis2_ctx_destroy(sl.ctx);
    if (sl.batch) mis2_batch_destroy(sl.batch);
    for (void* p : {(void*)sl.d_rp, (void*)sl.d_ci, (void*)sl.d_roots, (void*)sl.d_labels, (void*)sl.d_crp,
                    (void*)sl.d_cci})
      if (p) cudaFree(p);
    for (void* p : {(void*)sl.in_set, (void*)sl.roots, (void*)sl.labels, (void*)sl.c_rowptr, (void*)sl.c_colind,
                    (void*)sl.h_sum})
      if (p) cudaFreeHost(p);
    if (sl.d_sum) cudaFree(sl.d_sum);
  }
  delete s;
  return MIS2_OK;
}

int mis2_server_submit(mis2_server* s, const mis2_csr* g_host, uint64_t seed, int64_t* ticket) {
  return mis2_server_submit_out(s, g_host, seed, nullptr, ticket);
}

int mis2_server_submit_out(mis2_server* s, const mis2_csr* g_host, uint64_t seed, const mis2_request_out* out,
                           int64_t* ticket) {
  if (s == nullptr || g_host == nullptr || ticket == nullptr) return MIS2_ERR_INVALID_ARG;
  if (out != nullptr && out->c_colind_cap < 0) return MIS2_ERR_INVALID_ARG;
  if (g_host->n < 0 || g_host->nnz < 0 || g_host->rowptr == nullptr) return MIS2_ERR_INVALID_ARG;
  if (g_host->n > s->cfg.slot_max_n || g_host->nnz > s->cfg.slot_max_nnz) return MIS2_ERR_OUT_OF_MEMORY;
  Request rq;
  rq.g = *g_host;
  rq.seed = seed;
  if (out != nullptr) rq.out = *out;
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
