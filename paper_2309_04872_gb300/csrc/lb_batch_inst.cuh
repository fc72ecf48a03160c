// Instances of the batched step kernel for one storage precision: each
// closure, three candidate tiles for the autotuner (one translation unit per
// precision, so the units compile in parallel).
#pragma once

#include "lb_batch.cuh"
#include "lb_batch_dispatch.h"

namespace lbp {
template <int PR, int TZ, int TX, int CL>
struct BatchImpl {
  using Cfg = BatchCfg<PR, TZ, TX, CL>;
  static cudaError_t prepare() {
    return cudaFuncSetAttribute(lb_step_batch_kernel<PR, TZ, TX, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg::smem_bytes);
  }
  static void launch(const BatchArgs& A, int grid, cudaStream_t s) {
    lb_step_batch_kernel<PR, TZ, TX, CL><<<grid, TZ * TX, Cfg::smem_bytes, s>>>(A);
  }
  static int occupancy() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lb_step_batch_kernel<PR, TZ, TX, CL>, TZ * TX, Cfg::smem_bytes);
    return n;
  }
};

template <int PR, int CL>
void fill_closure(BatchKernelSet* ks, int c) {
  ks->prepare[c][0] = &BatchImpl<PR, 32, 8, CL>::prepare;
  ks->prepare[c][1] = &BatchImpl<PR, 64, 4, CL>::prepare;
  ks->prepare[c][2] = &BatchImpl<PR, 16, 16, CL>::prepare;
  ks->launch[c][0] = &BatchImpl<PR, 32, 8, CL>::launch;
  ks->launch[c][1] = &BatchImpl<PR, 64, 4, CL>::launch;
  ks->launch[c][2] = &BatchImpl<PR, 16, 16, CL>::launch;
  ks->occupancy[c][0] = &BatchImpl<PR, 32, 8, CL>::occupancy;
  ks->occupancy[c][1] = &BatchImpl<PR, 64, 4, CL>::occupancy;
  ks->occupancy[c][2] = &BatchImpl<PR, 16, 16, CL>::occupancy;
}

template <int PR>
void batch_fill(BatchKernelSet* ks) {
  ks->ncand = 3;
  ks->tz[0] = 32; ks->tx[0] = 8;
  ks->tz[1] = 64; ks->tx[1] = 4;
  ks->tz[2] = 16; ks->tx[2] = 16;
  fill_closure<PR, CL_LEC>(ks, CL_LEC);
  fill_closure<PR, CL_WARMC>(ks, CL_WARMC);
}
}  // namespace lbp
