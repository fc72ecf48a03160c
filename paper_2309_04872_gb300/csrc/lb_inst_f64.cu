// Kernel instances for population storage F64.
#include "lb_inst.cuh"

namespace lbp {
bool kernels_f64(int dim, int closure, KernelSet* ks) { return kernels_for<PR_F64>(dim, closure, ks); }
}  // namespace lbp
