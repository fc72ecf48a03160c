// Instantiation of the adjoint kernels (lb_adjoint.cuh).
#include "lb_adjoint.cuh"
#include "lb_adjoint_dispatch.h"

namespace lbp {

namespace {

template <int DIM> struct AdjTile;
template <> struct AdjTile<1> { static constexpr int TZ = 128, TX = 1; };
// 2D: 32 x 4 tiles, so the 512 x 256 grid's 1024 CTAs spread evenly over the
// SMs (32 x 8: 3.085-3.094 cost ratio of the sweep, 32 x 4: 3.052-3.06)
template <> struct AdjTile<2> { static constexpr int TZ = 32, TX = 4; };

// Resident CTAs per SM the per-node kernels' register budget is held to
// (latency-bound chains want warps; the counts below are for 256-thread
// CTAs, the 128-thread CTAs of the 32 x 4 tile run twice as many).  FP32 WARMC 2D, 1000-step reverse sweep
// with the population gathers inside them: 1/1 CTAs 117 ms, 2/2 103, 3/3
// 107, 3/4 101; with the gathers in the per-set kernels: 3/4 74 ms, 4/4 70,
// 4/5 76 (adj_local at 5 spills).  FP64 unconstrained.
template <typename real> struct AdjMinBlocks { static constexpr int LOCAL = 1, FIELD = 1; };
template <> struct AdjMinBlocks<float> { static constexpr int LOCAL = 8, FIELD = 8; };

// Launch with programmatic stream serialization (the kernels wait for
// their predecessor themselves, pdl_enter).
template <typename... Args>
void launch_pdl(void (*kernel)(Args...), dim3 g, unsigned threads, cudaStream_t s, const AdjParams& A) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = g;
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, A);
}

template <int DIM, int CL, int PR>
struct AdjImpl {
  using real = typename Prec<PR>::real;
  using T = AdjTile<DIM>;
  static void coll(const AdjParams& A, dim3 g, cudaStream_t s) {
    launch_pdl(adj_coll_kernel<DIM, CL, real, T::TZ, T::TX>, g, T::TZ * T::TX, s, A);
  }
  static void local(const AdjParams& A, dim3 g, cudaStream_t s) {
    launch_pdl(adj_local_kernel<DIM, CL, real, T::TZ, T::TX, AdjMinBlocks<real>::LOCAL>, g, T::TZ * T::TX, s, A);
  }
  static void field(const AdjParams& A, dim3 g, cudaStream_t s) {
    launch_pdl(adj_field_kernel<DIM, CL, real, T::TZ, T::TX, AdjMinBlocks<real>::FIELD>, g, T::TZ * T::TX, s, A);
  }
  static void init_rows(const StepParams& P, const void* lE, const void* lB, const double* Kx, double* rows,
                        dim3 g, cudaStream_t s) {
    if constexpr (DIM == 2)
      adj_init_rows_kernel<real, T::TZ, T::TX><<<g, T::TZ * T::TX, 0, s>>>(P, (const real*)lE, (const real*)lB, Kx,
                                                                            rows);
  }
  static void seed(void* lE, long long idx, double v, cudaStream_t s) {
    adj_seed_kernel<real><<<1, 32, 0, s>>>((real*)lE, idx, v);
  }
  static void read_slot(const void* E, const void* Elo, long long idx, double* out, cudaStream_t s) {
    read_slot_kernel<real><<<1, 32, 0, s>>>((const real*)E, (const real*)Elo, idx, out);
  }
  static void fill(AdjKernelSet* k) {
    using AM = AdjModel<DIM, CL>;
    k->K = AM::K;
    k->NG = AM::NG;
    k->NPREV = AM::NPREV;
    k->NTAPE = AM::NTAPE;
    k->tz = T::TZ;
    k->tx = T::TX;
    k->spt = kAdjSetsPerThread;
    k->coll = &coll;
    k->local = &local;
    k->field = &field;
    k->init_rows = &init_rows;
    k->seed = &seed;
    k->read_slot = &read_slot;
  }
};

template <int PR>
bool pick(int dim, int closure, AdjKernelSet* k) {
  if (dim == 1 && closure == CL_LEC) { AdjImpl<1, CL_LEC, PR>::fill(k); return true; }
  if (dim == 1 && closure == CL_WARMC) { AdjImpl<1, CL_WARMC, PR>::fill(k); return true; }
  if (dim == 2 && closure == CL_LEC) { AdjImpl<2, CL_LEC, PR>::fill(k); return true; }
  if (dim == 2 && closure == CL_WARMC) { AdjImpl<2, CL_WARMC, PR>::fill(k); return true; }
  return false;
}

}  // namespace

bool adjoint_kernels(int dim, int closure, int precision, AdjKernelSet* k) {
  if (precision == PR_F64) return pick<PR_F64>(dim, closure, k);
  if (precision == PR_F32) return pick<PR_F32>(dim, closure, k);
  return false;
}

void launch_grad(const GradParams& G, cudaStream_t s) {
  if (G.nsets <= 0) return;
  grad_sets_kernel<<<G.nsets, 256, 0, s>>>(G);
  const int nout = G.plen > 3 ? G.plen : 3;
  grad_accum_kernel<<<(nout + 127) / 128, 128, 0, s>>>(G);
}

}  // namespace lbp
