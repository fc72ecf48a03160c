// Kernel table of the discrete adjoint for one (dimension, closure,
// precision); the runtime picks one when a run starts recording.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace lbp {

struct AdjParams;
struct GradParams;
struct StepParams;

struct AdjKernelSet {
  int K, NG, NPREV, NTAPE;
  int tz, tx;  // tile of the per-node kernels
  int spt;     // sets per thread of the per-(node, set) kernels: grid.z = ceil(K / spt)
  // per (node, set), grid.z = K: the gather of the next state's population
  // adjoints, before adj_local
  void (*coll)(const AdjParams&, dim3 grid, cudaStream_t);
  void (*local)(const AdjParams&, dim3 grid, cudaStream_t);
  void (*field)(const AdjParams&, dim3 grid, cudaStream_t);
  void (*init_rows)(const StepParams&, const void* lE, const void* lB, const double* Kx, double* rows, dim3 grid,
                    cudaStream_t);
  void (*seed)(void* lE, long long idx, double v, cudaStream_t);
  void (*read_slot)(const void* E, const void* Elo, long long idx, double* out, cudaStream_t);
};

// 1D/2D, LEC/WARMC, FP64/FP32 storage; false otherwise.
bool adjoint_kernels(int dim, int closure, int precision, AdjKernelSet* ks);
// Row sets -> per-set partial gradients -> running sums (fixed order).
void launch_grad(const GradParams& G, cudaStream_t s);

}  // namespace lbp
