// Instantiation of the kernel table for one storage precision.
#pragma once

#include "lb_aux.cuh"
#include "lb_dispatch.h"
#include "lb_step_tma.cuh"

namespace lbp {

// Tiles of the plain step kernel.  1D: 64 nodes per CTA spreads the 2048-node
// run over 32 SMs.  3D: 32 x 4 x 4 keeps the decode halo at 2.4x the tile
// (512 threads, register budget 128; the rolled set loops fit it for both
// closures).
template <int DIM, int CL, int PR> struct Tile;
template <int CL, int PR> struct Tile<1, CL, PR> { static constexpr int TZ = 64, TX = 1, TY = 1; };
template <int CL, int PR> struct Tile<2, CL, PR> { static constexpr int TZ = 32, TX = 8, TY = 1; };
template <int CL, int PR> struct Tile<3, CL, PR> {
  static constexpr int TZ = 32, TX = 4, TY = 4;
};

// 3D marching columns (the automatic 3D kernel): 32 x 8 nodes per column,
// chunks of 32 planes.
struct March3D { static constexpr int TZ = 32, TX = 8, YC = 32; };

inline unsigned grid1(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <int DIM, int CL, int PR>
struct Impl {
  using T = Tile<DIM, CL, PR>;
  using Cfg = StepCfg<DIM, CL, PR, T::TZ, T::TX, T::TY>;
  using real = typename Prec<PR>::real;
  using store = typename Prec<PR>::store;

  static cudaError_t prepare() {
    return cudaFuncSetAttribute(lb_step_kernel<DIM, CL, PR, T::TZ, T::TX, T::TY>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem_bytes_gkeep);
  }
  static void step(const StepParams& P, dim3 grid, cudaStream_t s) {
    lb_step_kernel<DIM, CL, PR, T::TZ, T::TX, T::TY><<<grid, Cfg::NT, Cfg::smem_bytes_gkeep, s>>>(P);
  }
  using MC = StepCfg<3, CL, PR, March3D::TZ, March3D::TX, 1>;
  static constexpr bool kMarch = DIM == 3;
  static cudaError_t prepare_march() {
    if constexpr (kMarch)
      return cudaFuncSetAttribute(lb_step_march3d_kernel<CL, PR, March3D::TZ, March3D::TX, March3D::YC>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MC::smem_bytes);
    return cudaErrorNotSupported;
  }
  static void step_march(const StepParams& P, dim3 grid, cudaStream_t s) {
    if constexpr (kMarch)
      lb_step_march3d_kernel<CL, PR, March3D::TZ, March3D::TX, March3D::YC><<<grid, MC::NT, MC::smem_bytes, s>>>(P);
  }
  static void init_fields(const AuxParams& A, void* E, void* B, void* Elo, void* Blo, cudaStream_t s) {
    init_fields_kernel<DIM, real><<<grid1(A.ncell, 256), 256, 0, s>>>(A, (real*)E, (real*)B, (real*)Elo, (real*)Blo);
  }
  static void import_pops(const AuxParams& A, const double* src, void* dst, cudaStream_t s) {
    import_pops_kernel<DIM, CL, PR><<<grid1(A.ncell, 128), 128, 0, s>>>(A, src, (store*)dst);
  }
  static void export_pops(const AuxParams& A, const void* src, double* dst, cudaStream_t s) {
    export_pops_kernel<DIM, CL, PR><<<grid1(A.ncell, 128), 128, 0, s>>>(A, (const store*)src, dst);
  }
  static void advected(const AuxParams& A, const void* src, double* dst, cudaStream_t s) {
    advected_kernel<DIM, CL, PR><<<grid1(A.ncell, 128), 128, 0, s>>>(A, (const store*)src, dst);
  }
  static void moments(const AuxParams& A, const void* src, uint32_t mask, double* dst, cudaStream_t s) {
    moments_kernel<DIM, CL, PR><<<grid1(A.ncell, 128), 128, 0, s>>>(A, (const store*)src, mask, dst);
  }
  static void import_fields(const AuxParams& A, const double* E, const double* B, void* Ed, void* Bd, void* Elo,
                            void* Blo, cudaStream_t s) {
    import_fields_kernel<DIM, real><<<grid1(A.ncell, 256), 256, 0, s>>>(A, E, B, (real*)Ed, (real*)Bd, (real*)Elo,
                                                                         (real*)Blo);
  }
  static void export_fields(const AuxParams& A, const void* E, const void* B, const void* Elo, const void* Blo,
                            int ncomp, int4 comps, int4 isb, double* dst, cudaStream_t s) {
    export_fields_kernel<real><<<grid1(A.ncell, 256), 256, 0, s>>>(A, (const real*)E, (const real*)B,
                                                                    (const real*)Elo, (const real*)Blo, ncomp,
                                                                    comps, isb, dst);
  }
  static void reduce_partial(const AuxParams& A, const void* src, double* partial, int nblk, cudaStream_t s) {
    reduce_partial_kernel<DIM, CL, PR><<<nblk, 256, 0, s>>>(A, (const store*)src, partial);
  }
  static constexpr bool kAxi = DIM == 2;
  static cudaError_t prepare_axi() {
    if constexpr (kAxi)
      return cudaFuncSetAttribute(lb_step_axi_kernel<CL, PR, T::TZ, T::TX>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem_bytes_gkeep);
    return cudaErrorNotSupported;
  }
  static void step_axi(const StepParams& P, dim3 grid, cudaStream_t s) {
    if constexpr (kAxi) lb_step_axi_kernel<CL, PR, T::TZ, T::TX><<<grid, Cfg::NT, Cfg::smem_bytes_gkeep, s>>>(P);
  }
  using TC = TmaCfg2D<CL, PR>;
  static constexpr bool kTma = DIM == 2 && TC::enabled;
  static cudaError_t prepare_tma() {
    if constexpr (kTma)
      return cudaFuncSetAttribute(lb_step_tma2d_kernel<CL, PR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TC::smem_bytes);
    return cudaErrorNotSupported;
  }
  static void step_tma(const StepParams& P, const void* map, dim3 grid, cudaStream_t s) {
    if constexpr (kTma)
      lb_step_tma2d_kernel<CL, PR><<<grid, TC::TZ * TC::TX, TC::smem_bytes, s>>>(
          P, *reinterpret_cast<const CUtensorMap*>(map));
  }
  using PC = PersistCfg2D<CL, PR>;
  static constexpr bool kPersist = DIM == 2 && PC::enabled;
  static cudaError_t prepare_persist() {
    if constexpr (kPersist)
      return cudaFuncSetAttribute(lb_step_persist2d_kernel<CL, PR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)PC::smem_bytes);
    return cudaErrorNotSupported;
  }
  static void step_persist(const StepParams& P, const void* map, int grid, int ntz, int ntiles, cudaStream_t s) {
    if constexpr (kPersist)
      lb_step_persist2d_kernel<CL, PR><<<grid, PC::TZ * PC::TX, PC::smem_bytes, s>>>(
          P, *reinterpret_cast<const CUtensorMap*>(map), ntz, ntiles);
  }
  static cudaError_t prepare_persist_axi() {
    if constexpr (kPersist)
      return cudaFuncSetAttribute(lb_step_persist2d_kernel<CL, PR, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PC::smem_bytes);
    return cudaErrorNotSupported;
  }
  static void step_persist_axi(const StepParams& P, const void* map, int grid, int ntz, int ntiles,
                               cudaStream_t s) {
    if constexpr (kPersist)
      lb_step_persist2d_kernel<CL, PR, true><<<grid, PC::TZ * PC::TX, PC::smem_bytes, s>>>(
          P, *reinterpret_cast<const CUtensorMap*>(map), ntz, ntiles);
  }
  static void fill(KernelSet* ks) {
    ks->has_axi = kAxi;
    ks->prepare_axi = &prepare_axi;
    ks->step_axi = &step_axi;
    ks->has_march = kMarch;
    ks->march_tz = March3D::TZ;
    ks->march_tx = March3D::TX;
    ks->march_yc = March3D::YC;
    ks->prepare_march = &prepare_march;
    ks->step_march = &step_march;
    ks->has_persist = kPersist;
    ks->persist_auto = kPersist && PC::automatic;
    ks->per_tz = PC::TZ;
    ks->per_tx = PC::TX;
    ks->per_ctas = PC::MINB;
    ks->per_box[0] = PC::BZ;
    ks->per_box[1] = PC::BX;
    ks->per_box[2] = PC::BK;
    ks->per_smem = PC::smem_bytes;
    ks->prepare_persist = &prepare_persist;
    ks->step_persist = &step_persist;
    ks->prepare_persist_axi = &prepare_persist_axi;
    ks->step_persist_axi = &step_persist_axi;
    ks->has_tma = kTma;
    ks->tma_tz = TC::TZ;
    ks->tma_tx = TC::TX;
    ks->tma_box[0] = TC::BZ;
    ks->tma_box[1] = TC::BX;
    ks->tma_box[2] = TC::BK;
    ks->tma_halo_z = TC::HZ;
    ks->tma_elem_bytes = (int)sizeof(store);
    ks->tma_smem = TC::smem_bytes;
    ks->prepare_tma = &prepare_tma;
    ks->step_tma = &step_tma;
    ks->tz = T::TZ; ks->tx = T::TX; ks->ty = T::TY;
    ks->step_smem = Cfg::smem_bytes_gkeep;
    ks->prepare = &prepare;
    ks->step = &step;
    ks->init_fields = &init_fields;
    ks->import_pops = &import_pops;
    ks->export_pops = &export_pops;
    ks->advected = &advected;
    ks->moments = &moments;
    ks->import_fields = &import_fields;
    ks->export_fields = &export_fields;
    ks->reduce_partial = &reduce_partial;
  }
};

template <int PR>
bool kernels_for(int dim, int closure, KernelSet* ks) {
  if (dim == 1 && closure == CL_LEC) { Impl<1, CL_LEC, PR>::fill(ks); return true; }
  if (dim == 1 && closure == CL_WARMC) { Impl<1, CL_WARMC, PR>::fill(ks); return true; }
  if (dim == 2 && closure == CL_LEC) { Impl<2, CL_LEC, PR>::fill(ks); return true; }
  if (dim == 2 && closure == CL_WARMC) { Impl<2, CL_WARMC, PR>::fill(ks); return true; }
  if (dim == 3 && closure == CL_LEC) { Impl<3, CL_LEC, PR>::fill(ks); return true; }
  if (dim == 3 && closure == CL_WARMC) { Impl<3, CL_WARMC, PR>::fill(ks); return true; }
  return false;
}

}  // namespace lbp
