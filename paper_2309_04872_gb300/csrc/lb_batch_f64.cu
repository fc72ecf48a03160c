// Batched step kernel instances for population storage F64.
#include "lb_batch_inst.cuh"

namespace lbp {
void batch_kernels_f64(BatchKernelSet* ks) { batch_fill<PR_F64>(ks); }
}  // namespace lbp
