// Kernel instances for population storage F32 with exact set sums.
#include "lb_inst.cuh"

namespace lbp {
bool kernels_f32c(int dim, int closure, KernelSet* ks) { return kernels_for<PR_F32C>(dim, closure, ks); }
}  // namespace lbp
