// Kernel table of the batched step: per closure (index CL_LEC, CL_WARMC),
// one entry per candidate tile.
#pragma once

#include <cuda_runtime.h>

namespace lbp {

struct BatchArgs;

struct BatchKernelSet {
  int ncand;
  int tz[4], tx[4];
  cudaError_t (*prepare[2][4])();
  void (*launch[2][4])(const BatchArgs&, int grid, cudaStream_t);
  int (*occupancy[2][4])();
};

bool batch_kernels(int precision, BatchKernelSet* ks);
void batch_advance(long long* step, cudaStream_t s);

}  // namespace lbp
