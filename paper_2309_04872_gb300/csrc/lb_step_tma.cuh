// 2D fused step with the tile's population neighbourhood staged in shared
// memory by one TMA bulk-tensor load (cp.async.bulk.tensor, mbarrier
// completion).  The box covers z in [z0 - h, z0 + TZ + h) (h = 16 bytes of
// elements, so the start stays 16-byte aligned), x in [x0 - 2, x0 + TX + 2)
// and all K*Q population planes: every pull of the tile and of its one-node
// decode halo reads from it.  Open boundaries only (the clamped pull sources
// stay inside the box; periodic wrap would leave it).
#pragma once

#include <cuda.h>

#include "lb_step.cuh"

namespace lbp {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

template <int CL, int PR> struct TmaTile2D;
// Tile and resident CTAs per SM (the shared-memory box sets the occupancy;
// the register budget is held to match it).
template <> struct TmaTile2D<CL_LEC, PR_F32> { static constexpr int TZ = 64, TX = 8, MINB = 2; };
template <> struct TmaTile2D<CL_LEC, PR_F16S> { static constexpr int TZ = 64, TX = 8, MINB = 2; };
template <> struct TmaTile2D<CL_LEC, PR_F64> { static constexpr int TZ = 32, TX = 8, MINB = 2; };
template <> struct TmaTile2D<CL_WARMC, PR_F32> { static constexpr int TZ = 32, TX = 4, MINB = 2; };
template <> struct TmaTile2D<CL_WARMC, PR_F16S> { static constexpr int TZ = 32, TX = 8, MINB = 2; };
template <> struct TmaTile2D<CL_WARMC, PR_F64> { static constexpr int TZ = 0, TX = 0, MINB = 1; };  // not staged

template <int CL, int PR>
struct TmaCfg2D {
  using M = Model<2, CL>;
  using store = typename Prec<PR>::store;
  static constexpr int TZ = TmaTile2D<CL, PR>::TZ, TX = TmaTile2D<CL, PR>::TX, MINB = TmaTile2D<CL, PR>::MINB;
  static constexpr bool enabled = TZ > 0;
  static constexpr int HZ = 16 / (int)sizeof(store);
  static constexpr int BZ = TZ + 2 * HZ, BX = TX + 4, BK = M::K * M::Q;
  static constexpr size_t box_bytes = (size_t)BZ * BX * BK * sizeof(store);
  static constexpr size_t box_pad = (box_bytes + 127) / 128 * 128;
  using Body = StepCfg<2, CL, PR, (TZ > 0 ? TZ : 1), (TX > 0 ? TX : 1), 1>;
  static constexpr size_t smem_bytes = 128 + box_pad + 16 + Body::smem_bytes;
};

// Pull from the staged box (open boundaries: a boundary node reads as its
// nearest bulk node, Eq. open-bc).
template <int CL, int PR>
struct SmemPull2D {
  using T = TmaCfg2D<CL, PR>;
  using real = typename Prec<PR>::real;
  using store = typename Prec<PR>::store;
  const StepParams& P;
  const store* box;
  int oz, ox;
  __device__ __forceinline__ void operator()(int z, int x, int, int k, real* df) const {
    using L = Lattice<2>;
    const int bz = min(max(z, 1), P.n[0] - 2) - oz;
    const int bx = min(max(x, 1), P.n[1] - 2) - ox;
    const float is = P.inv_scale[k];
    const store* bk = box + (size_t)k * L::Q * T::BX * T::BZ;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const store v = bk[(i * T::BX + (bx - L::c(i, 1))) * T::BZ + (bz - L::c(i, 0))];
      if constexpr (PR == PR_F16S) df[i] = __half2float(v) * is;
      else df[i] = v;
    }
  }
};

template <int CL, int PR>
__global__ void __launch_bounds__(TmaCfg2D<CL, PR>::TZ* TmaCfg2D<CL, PR>::TX, TmaCfg2D<CL, PR>::MINB)
lb_step_tma2d_kernel(const StepParams P, const __grid_constant__ CUtensorMap tmap) {
  using T = TmaCfg2D<CL, PR>;
  using store = typename Prec<PR>::store;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  store* box = reinterpret_cast<store*>(base);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + T::box_pad);
  unsigned char* body = base + T::box_pad + 16;
  const int oz = blockIdx.x * T::TZ - T::HZ;
  const int ox = blockIdx.y * T::TX - 2;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
    mbar_arrive_expect_tx(bar, (uint32_t)T::box_bytes);
    tma_load_3d(box, &tmap, bar, oz, ox, 0);
  }
  __syncthreads();
  // bounded wait for the box; on timeout flag the error and leave
  bool done = false;
  for (uint32_t spin = 0; spin < (1u << 24) && !(done = mbar_try_wait(bar, 0)); ++spin) {
  }
  if (!__syncthreads_and(done)) {
    if (threadIdx.x == 0 && P.err) atomicOr(P.err, 1);
    return;
  }
  SmemPull2D<CL, PR> pull{P, box, oz, ox};
  step_body<2, CL, PR, T::TZ, T::TX, 1>(P, body, pull);
}

}  // namespace lbp
