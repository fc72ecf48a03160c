// Batched step kernel instances for population storage F16S.
#include "lb_batch_inst.cuh"

namespace lbp {
void batch_kernels_f16s(BatchKernelSet* ks) { batch_fill<PR_F16S>(ks); }
}  // namespace lbp
