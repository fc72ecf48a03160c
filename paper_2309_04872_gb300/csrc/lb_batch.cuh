// Batched 2D step: one persistent launch per closure advances many runs
// (uneven grids) by one time step.  The closure's work list holds (run, tile)
// items; CTA b takes items b, b + gridDim.x, ...  Each item copies its run's
// launch parameters into shared memory, sets the step's time and buffer
// parity from a device-side step counter (so a captured CUDA graph can be
// replayed from any step) and runs the same three-phase step as a single
// run.  One kernel per closure keeps each at its own register budget and
// occupancy (LEC needs far fewer registers than WARMC).
#pragma once

#include "lb_batch_types.cuh"
#include "lb_step.cuh"

namespace lbp {

// Time of step s written without contraction, as the host computes it for
// single runs (z0 + s dt in round-to-nearest, no fused multiply-add).
__device__ __forceinline__ double batch_zeta0(double z0, long long s, double dt) {
  return __dadd_rn(z0, __dmul_rn((double)s, dt));
}

// AXI: an axisymmetric (z, r) run (the axis rules and 1/r sources of
// step_body's AXI mode).
template <int CL, int PR, int TZ, int TX, bool AXI>
__device__ __forceinline__ void batch_item(const StepParams& P, unsigned char* smem, int tz, int tx) {
  using real = typename Prec<PR>::real;
  using Pull = GlobalPull<2, CL, PR, false, AXI>;
  Pull pull{P};
  FieldPF<real> F;
  if (tile_is_bulk<2, TZ, TX, 1>(P, tz, tx, 0)) {
    prefetch_own<2, real, false, TZ, TX, 1>(P, F, tz, tx, 0);
    step_body<2, CL, PR, TZ, TX, 1, false, Pull, NoHook, false, AXI>(P, smem, pull, F, tz, tx, 0);
  } else {
    prefetch_own<2, real, true, TZ, TX, 1>(P, F, tz, tx, 0);
    step_body<2, CL, PR, TZ, TX, 1, true, Pull, NoHook, false, AXI>(P, smem, pull, F, tz, tx, 0);
  }
}

template <int PR, int TZ, int TX, int CL>
struct BatchCfg {
  static constexpr size_t smem_bytes = StepCfg<2, CL, PR, TZ, TX, 1>::smem_bytes;
  // resident CTAs the register budget is held to in FP32 and FP16S: three
  // for LEC (as the single-run LEC kernel runs), two for WARMC
  static constexpr int MINB = (PR == PR_F32 || PR == PR_F16S) ? (CL == CL_LEC ? 3 : 2) : 1;
};

template <int PR, int TZ, int TX, int CL>
__global__ void __launch_bounds__(TZ* TX, (BatchCfg<PR, TZ, TX, CL>::MINB)) lb_step_batch_kernel(const BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) StepParams Ps;
  __shared__ int s_ntz, s_axi;
  const long long step = *A.step;
  const int parity = (int)(step & 1);
  // the CTA's items are mostly consecutive tiles of one run: the run's launch
  // parameters are copied only when the run changes, and the next item's
  // index is loaded one item ahead
  int run = -1;
  int it = blockIdx.x;
  int2 w = it < A.nitems ? A.items[it] : make_int2(0, 0);
  for (; it < A.nitems; it += gridDim.x) {
    const int itn = it + gridDim.x;
    const int2 wn = itn < A.nitems ? A.items[itn] : w;
    if (w.x != run) {
      const BatchRun* R = A.runs + w.x;
      const int* src = reinterpret_cast<const int*>(&R->P[parity]);
      int* dst = reinterpret_cast<int*>(&Ps);
      for (int q = threadIdx.x; q < (int)(sizeof(StepParams) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
      __syncthreads();
      if (threadIdx.x == 0) {
        const double z = batch_zeta0(R->z0, step, R->dt);
        Ps.cd.zeta0 = z;
        Ps.cf.zeta0 = (float)z;
        Ps.have_prev = step > R->prev_from ? 1 : 0;
        s_ntz = R->ntz;
        s_axi = R->axi;
      }
      __syncthreads();
      run = w.x;
    }
    const int tz = w.y % s_ntz, tx = w.y / s_ntz;
    // the run's geometry is uniform over the CTA
    if (s_axi) batch_item<CL, PR, TZ, TX, true>(Ps, smem_raw, tz, tx);
    else batch_item<CL, PR, TZ, TX, false>(Ps, smem_raw, tz, tx);
    __syncthreads();  // Ps and the records are reused by the next item
    w = wn;
  }
}

static __global__ void batch_advance_kernel(long long* step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

}  // namespace lbp
