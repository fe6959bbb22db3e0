// cupti_trace.cpp -- GPU activity trace of a stretch of host code: every
// kernel, memset and memcpy the process runs on the device between
// mis2_trace_start and mis2_trace_stop, with its device start and end time,
// written one record per line to a text file.  Built apart from the library
// (it links CUPTI) and used only by measurement code; the library's compute
// path never calls it.
//
// Record lines: "<K|S|C> <start ns> <end ns> <stream id> <name>", K a kernel
// (its mangled name), S a memset ("memset_<bytes>"), C a memcpy
// ("memcpy_<kind>_<bytes>").
#include <cupti.h>

#include <cstdio>
#include <cstdlib>
#include <mutex>

namespace {

FILE* g_out = nullptr;
std::mutex g_mu;

void CUPTIAPI buffer_requested(uint8_t** buf, size_t* size, size_t* max_records) {
  *size = 8u << 20;
  *buf = static_cast<uint8_t*>(aligned_alloc(8, *size));
  *max_records = 0;
}

void CUPTIAPI buffer_completed(CUcontext, uint32_t, uint8_t* buf, size_t, size_t valid) {
  std::lock_guard<std::mutex> lk(g_mu);
  CUpti_Activity* rec = nullptr;
  while (cuptiActivityGetNextRecord(buf, valid, &rec) == CUPTI_SUCCESS) {
    if (g_out == nullptr) continue;
    switch (rec->kind) {
      case CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL:
      case CUPTI_ACTIVITY_KIND_KERNEL: {
        const auto* k = reinterpret_cast<const CUpti_ActivityKernel10*>(rec);
        fprintf(g_out, "K %llu %llu %u %s\n", (unsigned long long)k->start, (unsigned long long)k->end, k->streamId,
                k->name);
        break;
      }
      case CUPTI_ACTIVITY_KIND_MEMSET: {
        const auto* m = reinterpret_cast<const CUpti_ActivityMemset4*>(rec);
        fprintf(g_out, "S %llu %llu %u memset_%llu\n", (unsigned long long)m->start, (unsigned long long)m->end,
                m->streamId, (unsigned long long)m->bytes);
        break;
      }
      case CUPTI_ACTIVITY_KIND_MEMCPY: {
        const auto* m = reinterpret_cast<const CUpti_ActivityMemcpy6*>(rec);
        fprintf(g_out, "C %llu %llu %u memcpy_%d_%llu\n", (unsigned long long)m->start, (unsigned long long)m->end,
                m->streamId, (int)m->copyKind, (unsigned long long)m->bytes);
        break;
      }
      default:
        break;
    }
  }
  free(buf);
}

const CUpti_ActivityKind kKinds[] = {CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL, CUPTI_ACTIVITY_KIND_MEMSET,
                                     CUPTI_ACTIVITY_KIND_MEMCPY};

}  // namespace

extern "C" {

// Starts recording into the file at `path` (overwritten).  Returns 0, or a
// nonzero code when the file cannot be opened (-1) or CUPTI refuses
// (its CUptiResult).
int mis2_trace_start(const char* path) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_out = fopen(path, "w");
    if (g_out == nullptr) return -1;
  }
  CUptiResult r = cuptiActivityRegisterCallbacks(buffer_requested, buffer_completed);
  if (r != CUPTI_SUCCESS) return (int)r;
  for (CUpti_ActivityKind k : kKinds) {
    r = cuptiActivityEnable(k);
    if (r != CUPTI_SUCCESS) return (int)r;
  }
  return 0;
}

// Flushes every pending record and closes the file.  The caller
// synchronises the device first, so that the traced work has finished.
int mis2_trace_stop() {
  cuptiActivityFlushAll(1);
  for (CUpti_ActivityKind k : kKinds) cuptiActivityDisable(k);
  cuptiActivityFlushAll(1);
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_out != nullptr) fclose(g_out);
  g_out = nullptr;
  return 0;
}

}  // extern "C"
