// rowclass.cu -- rows split by length for the host-driven round kernels of
// distance-k MIS and of the colouring: short rows stay with the kernels that
// give each row G lanes, medium rows get a warp each and long rows a block
// each, from two ascending lists built once per call.
#include "internal.h"

namespace mis2 {

namespace {

template <typename I>
__global__ void __launch_bounds__(kBlock) k_class_flags(const I* rowptr, int64_t n, int64_t light_max,
                                                        int64_t heavy_min, uint8_t* medium, uint8_t* heavy) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const int64_t d = (int64_t)rowptr[v + 1] - (int64_t)rowptr[v];
    medium[v] = d > light_max && d <= heavy_min;
    heavy[v] = d > heavy_min;
  }
}

}  // namespace

int classify_rows(mis2_ctx* c, const GraphArgs& g, int64_t light_max, int64_t heavy_min, LenLists* rl,
                  cudaStream_t st) {
  Scratch& s = c->s;
  uint8_t* fm = s.qflag;
  uint8_t* fh = reinterpret_cast<uint8_t*>(s.aggsize);
  rl->medium = s.left_mid;
  rl->heavy = s.large;
  rl->n_medium_dev = s.ctr + kCtrLeftMid;
  rl->n_heavy_dev = s.ctr + kCtrHeavy;
  if (g.n > 0) {
    const int blocks = grid_for(c, g.n, kBlock);
    if (g.rp64)
      k_class_flags<int64_t><<<blocks, kBlock, 0, st>>>(static_cast<const int64_t*>(g.rowptr), g.n, light_max,
                                                        heavy_min, fm, fh);
    else
      k_class_flags<int32_t><<<blocks, kBlock, 0, st>>>(static_cast<const int32_t*>(g.rowptr), g.n, light_max,
                                                        heavy_min, fm, fh);
    c->launches++;
    MIS2_CUDA(cudaGetLastError());
  }
  MIS2_TRY(compact_flags(c, fm, nullptr, g.n, s.left_mid, s.ctr + kCtrLeftMid, st));
  MIS2_TRY(compact_flags(c, fh, nullptr, g.n, s.large, s.ctr + kCtrHeavy, st));
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  rl->n_medium = c->h_ctr[kCtrLeftMid];
  rl->n_heavy = c->h_ctr[kCtrHeavy];
  return MIS2_OK;
}

}  // namespace mis2
