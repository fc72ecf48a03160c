// Dispatch of the batched step kernels (instances in lb_batch_f32.cu,
// lb_batch_f64.cu, lb_batch_f16s.cu) and the step counter.
#include "lb_batch.cuh"
#include "lb_batch_dispatch.h"

namespace lbp {

void batch_kernels_f32(BatchKernelSet* ks);
void batch_kernels_f64(BatchKernelSet* ks);
void batch_kernels_f16s(BatchKernelSet* ks);

bool batch_kernels(int precision, BatchKernelSet* ks) {
  if (precision == PR_F32) { batch_kernels_f32(ks); return true; }
  if (precision == PR_F64) { batch_kernels_f64(ks); return true; }
  if (precision == PR_F16S) { batch_kernels_f16s(ks); return true; }
  return false;
}

void batch_advance(long long* step, cudaStream_t s) { batch_advance_kernel<<<1, 32, 0, s>>>(step); }

}  // namespace lbp
