// Batched step kernel instances for population storage F32.
#include "lb_batch_inst.cuh"

namespace lbp {
void batch_kernels_f32(BatchKernelSet* ks) { batch_fill<PR_F32>(ks); }
}  // namespace lbp
