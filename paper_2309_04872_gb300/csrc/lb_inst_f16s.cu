// Kernel instances for population storage F16S.
#include "lb_inst.cuh"

namespace lbp {
bool kernels_f16s(int dim, int closure, KernelSet* ks) { return kernels_for<PR_F16S>(dim, closure, ks); }
}  // namespace lbp
