// Kernel instances for population storage F32.
#include "lb_inst.cuh"

namespace lbp {
bool kernels_f32(int dim, int closure, KernelSet* ks) { return kernels_for<PR_F32>(dim, closure, ks); }
}  // namespace lbp
