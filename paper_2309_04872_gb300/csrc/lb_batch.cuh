// Batched 2D step: one persistent launch advances many runs (uneven grids,
// both closures) by one time step.  The work list holds (run, tile) items;
// CTA b takes items b, b + gridDim.x, ...  Each item copies its run's launch
// parameters into shared memory, sets the step's time and buffer parity from
// a device-side step counter (so a captured CUDA graph can be replayed from
// any step) and runs the same three-phase step as a single run, with the
// LEC or WARMC body chosen per item (block-uniform branch).
#pragma once

#include "lb_batch_types.cuh"
#include "lb_step.cuh"

namespace lbp {

// Time of step s written without contraction, as the host computes it for
// single runs (z0 + s dt in round-to-nearest, no fused multiply-add).
__device__ __forceinline__ double batch_zeta0(double z0, long long s, double dt) {
  return __dadd_rn(z0, __dmul_rn((double)s, dt));
}

template <int CL, int PR, int TZ, int TX>
__device__ __forceinline__ void batch_item(const StepParams& P, unsigned char* smem, int tz, int tx) {
  using real = typename Prec<PR>::real;
  GlobalPull<2, CL, PR> pull{P};
  FieldPF<real> F;
  if (tile_is_bulk<2, TZ, TX, 1>(P, tz, tx, 0)) {
    prefetch_own<2, real, false, TZ, TX, 1>(P, F, tz, tx, 0);
    step_body<2, CL, PR, TZ, TX, 1, false>(P, smem, pull, F, tz, tx, 0);
  } else {
    prefetch_own<2, real, true, TZ, TX, 1>(P, F, tz, tx, 0);
    step_body<2, CL, PR, TZ, TX, 1, true>(P, smem, pull, F, tz, tx, 0);
  }
}

template <int PR, int TZ, int TX>
struct BatchCfg {
  static constexpr size_t smem_lec = StepCfg<2, CL_LEC, PR, TZ, TX, 1>::smem_bytes;
  static constexpr size_t smem_warmc = StepCfg<2, CL_WARMC, PR, TZ, TX, 1>::smem_bytes;
  static constexpr size_t smem_bytes = smem_lec > smem_warmc ? smem_lec : smem_warmc;
};

template <int PR, int TZ, int TX>
__global__ void __launch_bounds__(TZ* TX) lb_step_batch_kernel(const BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) StepParams Ps;
  const long long step = *A.step;
  const int parity = (int)(step & 1);
  for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
    const int2 w = A.items[it];
    const BatchRun* R = A.runs + w.x;
    {
      const int* src = reinterpret_cast<const int*>(&R->P[parity]);
      int* dst = reinterpret_cast<int*>(&Ps);
      for (int q = threadIdx.x; q < (int)(sizeof(StepParams) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double z = batch_zeta0(R->z0, step, R->dt);
      Ps.cd.zeta0 = z;
      Ps.cf.zeta0 = (float)z;
      Ps.have_prev = step > R->prev_from ? 1 : 0;
    }
    __syncthreads();
    const int tz = w.y % R->ntz, tx = w.y / R->ntz;
    if (R->closure == CL_LEC) batch_item<CL_LEC, PR, TZ, TX>(Ps, smem_raw, tz, tx);
    else batch_item<CL_WARMC, PR, TZ, TX>(Ps, smem_raw, tz, tx);
    __syncthreads();  // Ps and the records are reused by the next item
  }
}

static __global__ void batch_advance_kernel(long long* step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

}  // namespace lbp
