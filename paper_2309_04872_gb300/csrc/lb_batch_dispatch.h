// Kernel table of the batched step (one entry per candidate tile).
#pragma once

#include <cuda_runtime.h>

namespace lbp {

struct BatchArgs;

struct BatchKernelSet {
  int ncand;
  int tz[4], tx[4];
  cudaError_t (*prepare[4])();
  void (*launch[4])(const BatchArgs&, int grid, cudaStream_t);
  int (*occupancy[4])();
};

bool batch_kernels(int precision, BatchKernelSet* ks);
void batch_advance(long long* step, cudaStream_t s);

}  // namespace lbp
