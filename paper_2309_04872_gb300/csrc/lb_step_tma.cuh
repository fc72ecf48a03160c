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

// Bounded wait on one phase of an mbarrier: at most `polls` polls, false when
// they ran out.  A tile's first wait polls P.wait_limit times (2^24 unless the
// host lowered it to exercise the timeout path); the drain after a timeout,
// which lets the copy in flight land before the CTA leaves, keeps the long
// limit kDrainPolls.
constexpr uint32_t kDrainPolls = 1u << 24;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t polls) {
  for (uint32_t spin = 0; spin < polls; ++spin)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <int CL, int PR> struct TmaTile2D;
// Tile and resident CTAs per SM (the shared-memory box sets the occupancy;
// the register budget is held to match it).
template <> struct TmaTile2D<CL_LEC, PR_F32> { static constexpr int TZ = 32, TX = 8, MINB = 3; };
template <> struct TmaTile2D<CL_LEC, PR_F16S> { static constexpr int TZ = 64, TX = 8, MINB = 2; };
template <> struct TmaTile2D<CL_LEC, PR_F64> { static constexpr int TZ = 32, TX = 8, MINB = 2; };
template <> struct TmaTile2D<CL_WARMC, PR_F32> { static constexpr int TZ = 32, TX = 4, MINB = 2; };
template <> struct TmaTile2D<CL_WARMC, PR_F16S> { static constexpr int TZ = 32, TX = 8, MINB = 2; };
template <> struct TmaTile2D<CL_WARMC, PR_F64> { static constexpr int TZ = 0, TX = 0, MINB = 1; };  // not staged
template <int CL> struct TmaTile2D<CL, PR_F32C> : TmaTile2D<CL, PR_F32> {};

template <int CL, int PR>
struct TmaCfg2D {
  using M = Model<2, CL>;
  using store = typename Prec<PR>::store;
  static constexpr int TZ = TmaTile2D<CL, PR>::TZ, TX = TmaTile2D<CL, PR>::TX, MINB = TmaTile2D<CL, PR>::MINB;
  static constexpr bool enabled = TZ > 0;
  static constexpr int HZ = 16 / (int)sizeof(store);
  // K*Q population planes, then the rest populations' low parts (FP16S)
  static constexpr int KQ = M::K * M::Q, BZ = TZ + 2 * HZ, BX = TX + 4, BK = KQ + M::K * Codec<PR>::kLoPlanes;
  static constexpr size_t box_bytes = (size_t)BZ * BX * BK * sizeof(store);
  static constexpr size_t box_pad = (box_bytes + 127) / 128 * 128;
  using Body = StepCfg<2, CL, PR, (TZ > 0 ? TZ : 1), (TX > 0 ? TX : 1), 1>;
  static constexpr size_t smem_bytes = 128 + box_pad + 16 + Body::smem_bytes;
};

// Pull from the staged box (open boundaries: a boundary node reads as its
// nearest bulk node, Eq. open-bc), in storage units as pulled_dev.
template <int CL, int PR>
struct SmemPull2D {
  using T = TmaCfg2D<CL, PR>;
  using real = typename Prec<PR>::real;
  using store = typename Prec<PR>::store;
  const StepParams& P;
  const store* box;
  int oz, ox;
  template <bool EDGE>
  __device__ __forceinline__ void get(int z, int x, int, int k, real* df) const {
    using L = Lattice<2>;
    const int bz = (EDGE ? min(max(z, 1), P.n[0] - 2) : z) - oz;
    const int bx = (EDGE ? min(max(x, 1), P.n[1] - 2) : x) - ox;
    const store* bk = box + (size_t)k * L::Q * T::BX * T::BZ;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const store v = bk[(i * T::BX + (bx - L::c(i, 1))) * T::BZ + (bz - L::c(i, 0))];
      if constexpr (PR == PR_F16S) df[i] = __half2float(v);  // storage units
      else df[i] = v;
    }
    if constexpr (Codec<PR>::kLoPlanes > 0) {
      // the rest population with its low part (staged after the K*Q planes)
      const store* lo = box + ((size_t)T::KQ + k) * T::BX * T::BZ;
      df[0] = Codec<PR>::join_u(bk[bx * T::BZ + bz], lo[bx * T::BZ + bz]);
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
  using real = typename Prec<PR>::real;
  const int oz = blockIdx.x * T::TZ - T::HZ;
  const int ox = blockIdx.y * T::TX - 2;
  const bool bulk = tile_is_bulk<2, T::TZ, T::TX, 1>(P, blockIdx.x, blockIdx.y, 0);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
    mbar_arrive_expect_tx(bar, (uint32_t)T::box_bytes);
    tma_load_3d(box, &tmap, bar, oz, ox, 0);
  }
  __syncthreads();
  // the own node's fields load while the box is in flight
  FieldPF<real> F;
  if (bulk) prefetch_own<2, real, false, T::TZ, T::TX, 1>(P, F, blockIdx.x, blockIdx.y, 0);
  else prefetch_own<2, real, true, T::TZ, T::TX, 1>(P, F, blockIdx.x, blockIdx.y, 0);
  // bounded wait for the box; on timeout flag the error, let the copy in
  // flight land in shared memory, and leave
  const bool done = mbar_wait_bounded(bar, 0, P.wait_limit);
  if (!__syncthreads_and(done)) {
    if (threadIdx.x == 0) {
      if (P.err) atomicOr(P.err, 1);
      mbar_wait_bounded(bar, 0, kDrainPolls);
    }
    return;
  }
  SmemPull2D<CL, PR> pull{P, box, oz, ox};
  if (bulk) step_body<2, CL, PR, T::TZ, T::TX, 1, false>(P, body, pull, F, blockIdx.x, blockIdx.y, 0);
  else step_body<2, CL, PR, T::TZ, T::TX, 1, true>(P, body, pull, F, blockIdx.x, blockIdx.y, 0);
}

// Persistent form for the LEC closure: MINB CTAs per SM walk the tiles
// (t = blockIdx.x, + gridDim.x, ...) with one box each.  LEC keeps the own
// node's populations in registers (K*Q = 27 <= 32), so the box is free once
// the decode phase has passed its barrier: the TMA load of the CTA's next
// tile is issued there and streams in while the E/B update and the collide
// of the current tile run.  The CTAs of an SM thus overlap loads and compute
// without the lockstep waves of one launch-per-tile grid.
// Tile, CTAs per SM, and whether the automatic kernel choice takes this form
// (measured on the 1024 x 512 LEC workload: FP32 32 x 8 with three CTAs per
// SM runs 17.0 GLUPS against 14.9 for one box per launched CTA, FP16S 16.4
// against 16.0; FP64 is faster with one box per CTA).
template <int CL, int PR> struct PersistTile2D;
template <> struct PersistTile2D<CL_LEC, PR_F32> { static constexpr int TZ = 32, TX = 8, MINB = 3, AUTO = 1; };
template <> struct PersistTile2D<CL_LEC, PR_F16S> { static constexpr int TZ = 32, TX = 8, MINB = 3, AUTO = 1; };
template <> struct PersistTile2D<CL_LEC, PR_F64> { static constexpr int TZ = 32, TX = 8, MINB = 2, AUTO = 0; };
template <> struct PersistTile2D<CL_WARMC, PR_F32> { static constexpr int TZ = 0, TX = 0, MINB = 1, AUTO = 0; };
template <> struct PersistTile2D<CL_WARMC, PR_F16S> { static constexpr int TZ = 0, TX = 0, MINB = 1, AUTO = 0; };
template <> struct PersistTile2D<CL_WARMC, PR_F64> { static constexpr int TZ = 0, TX = 0, MINB = 1, AUTO = 0; };
template <int CL> struct PersistTile2D<CL, PR_F32C> : PersistTile2D<CL, PR_F32> {};

template <int CL, int PR>
struct PersistCfg2D {
  using M = Model<2, CL>;
  using store = typename Prec<PR>::store;
  static constexpr int TZ = PersistTile2D<CL, PR>::TZ, TX = PersistTile2D<CL, PR>::TX;
  static constexpr int MINB = PersistTile2D<CL, PR>::MINB;
  static constexpr bool enabled = TZ > 0;
  static constexpr bool automatic = enabled && PersistTile2D<CL, PR>::AUTO != 0;
  static_assert(!enabled || M::K * Lattice<2>::Q <= 32, "the box is refilled after the decode phase");
  static constexpr int HZ = 16 / (int)sizeof(store);
  // K*Q population planes, then the rest populations' low parts (FP16S)
  static constexpr int KQ = M::K * M::Q, BZ = TZ + 2 * HZ, BX = TX + 4, BK = KQ + M::K * Codec<PR>::kLoPlanes;
  static constexpr size_t box_bytes = (size_t)BZ * BX * BK * sizeof(store);
  static constexpr size_t box_pad = (box_bytes + 127) / 128 * 128;
  using Body = StepCfg<2, CL, PR, (TZ > 0 ? TZ : 1), (TX > 0 ? TX : 1), 1>;
  static constexpr size_t smem_bytes = 128 + box_pad + 16 + Body::smem_bytes;
};

// AXI: the x = 0 row is the r = 0 boundary node of an axisymmetric grid; its
// odd sets take the mirrored velocity (as pulled_dev).
template <int CL, int PR, bool AXI = false>
struct SmemPullBox2D {
  using T = PersistCfg2D<CL, PR>;
  using real = typename Prec<PR>::real;
  using store = typename Prec<PR>::store;
  const StepParams& P;
  const store* box;
  int oz, ox;
  template <bool EDGE>
  __device__ __forceinline__ void get(int z, int x, int, int k, real* df) const {
    using L = Lattice<2>;
    const bool mirror = AXI && EDGE && x == 0 && odd_in_r<CL>(k);
    const int bz = (EDGE ? min(max(z, 1), P.n[0] - 2) : z) - oz;
    const int bx = (EDGE ? min(max(x, 1), P.n[1] - 2) : x) - ox;
    const store* bk = box + (size_t)k * L::Q * T::BX * T::BZ;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const store v = bk[(i * T::BX + (bx - L::c(i, 1))) * T::BZ + (bz - L::c(i, 0))];
      if constexpr (PR == PR_F16S) df[i] = __half2float(v);  // storage units
      else df[i] = v;
    }
    if constexpr (Codec<PR>::kLoPlanes > 0) {
      // the rest population with its low part (staged after the K*Q planes)
      const store* lo = box + ((size_t)T::KQ + k) * T::BX * T::BZ;
      df[0] = Codec<PR>::join_u(bk[bx * T::BZ + bz], lo[bx * T::BZ + bz]);
    }
    if constexpr (AXI) {
      if (mirror) {
        // D2Q9 with x reversed: 3 <-> 4, 5 <-> 7, 6 <-> 8
        real t;
        t = df[3]; df[3] = df[4]; df[4] = t;
        t = df[5]; df[5] = df[7]; df[7] = t;
        t = df[6]; df[6] = df[8]; df[8] = t;
      }
    }
  }
};

// AXI: the axisymmetric (z, r) step (the axis rules and 1/r sources of
// step_body's AXI mode).
template <int CL, int PR, bool AXI = false>
__global__ void __launch_bounds__(PersistCfg2D<CL, PR>::TZ* PersistCfg2D<CL, PR>::TX, PersistCfg2D<CL, PR>::MINB)
lb_step_persist2d_kernel(const StepParams P, const __grid_constant__ CUtensorMap tmap, int ntz, int ntiles) {
  using T = PersistCfg2D<CL, PR>;
  using store = typename Prec<PR>::store;
  using real = typename Prec<PR>::real;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  store* box = reinterpret_cast<store*>(base);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + T::box_pad);
  unsigned char* body = base + T::box_pad + 16;
  const int G = gridDim.x;
  int t = blockIdx.x;
  if (t >= ntiles) return;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
    mbar_arrive_expect_tx(bar, (uint32_t)T::box_bytes);
    tma_load_3d(box, &tmap, bar, (t % ntz) * T::TZ - T::HZ, (t / ntz) * T::TX - 2, 0);
  }
  __syncthreads();
  for (uint32_t j = 0; t < ntiles; ++j, t += G) {
    const int tz = t % ntz, tx = t / ntz;
    const int tn = t + G;
    const bool bulk = tile_is_bulk<2, T::TZ, T::TX, 1>(P, tz, tx, 0);
    FieldPF<real> F;
    if (bulk) prefetch_own<2, real, false, T::TZ, T::TX, 1>(P, F, tz, tx, 0);
    else prefetch_own<2, real, true, T::TZ, T::TX, 1>(P, F, tz, tx, 0);
    // bounded wait for this tile's box (the barrier's phase j); on timeout
    // flag the error, let the copy in flight land, and leave
    const bool done = mbar_wait_bounded(bar, j & 1u, P.wait_limit);
    if (!__syncthreads_and(done)) {
      if (threadIdx.x == 0) {
        if (P.err) atomicOr(P.err, 1);
        mbar_wait_bounded(bar, j & 1u, kDrainPolls);
      }
      return;
    }
    // refill the box with the next tile once the decode phase has read it;
    // the barrier that ended the phase orders those generic-proxy reads
    // before the async-proxy writes
    auto refill = [&]() {
      if (threadIdx.x == 0 && tn < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, (uint32_t)T::box_bytes);
        tma_load_3d(box, &tmap, bar, (tn % ntz) * T::TZ - T::HZ, (tn / ntz) * T::TX - 2, 0);
      }
    };
    using Pull = SmemPullBox2D<CL, PR, AXI>;
    using Hook = decltype(refill);
    Pull pull{P, box, tz * T::TZ - T::HZ, tx * T::TX - 2};
    if (bulk) step_body<2, CL, PR, T::TZ, T::TX, 1, false, Pull, Hook, false, AXI>(P, body, pull, F, tz, tx, 0, refill);
    else step_body<2, CL, PR, T::TZ, T::TX, 1, true, Pull, Hook, false, AXI>(P, body, pull, F, tz, tx, 0, refill);
    __syncthreads();  // the records and E slots are free for the next tile
  }
}

}  // namespace lbp
