// Kernel table of one (dimension, closure, precision) combination; the
// runtime picks one at create time.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lbp {

struct StepParams;
struct AuxParams;

struct KernelSet {
  int tz, tx, ty;        // step tile
  size_t step_smem;      // dynamic shared memory of the step kernel
  cudaError_t (*prepare)();
  void (*step)(const StepParams&, dim3 grid, cudaStream_t);
  void (*init_fields)(const AuxParams&, void* E, void* B, void* Elo, void* Blo, cudaStream_t);
  void (*import_pops)(const AuxParams&, const double* src, void* dst, cudaStream_t);
  void (*export_pops)(const AuxParams&, const void* src, double* dst, cudaStream_t);
  void (*advected)(const AuxParams&, const void* src, double* dst, cudaStream_t);
  void (*moments)(const AuxParams&, const void* src, uint32_t mask, double* dst, cudaStream_t);
  // FP32 fields carry low parts (Elo, Blo); null in FP64
  void (*import_fields)(const AuxParams&, const double* E, const double* B, void* Ed, void* Bd, void* Elo,
                        void* Blo, cudaStream_t);
  void (*export_fields)(const AuxParams&, const void* E, const void* B, const void* Elo, const void* Blo, int ncomp,
                        int4 comps, int4 isb, double* dst, cudaStream_t);
  void (*reduce_partial)(const AuxParams&, const void* src, double* partial, int nblk, cudaStream_t);
  // TMA-staged 2D step (open boundaries); has_tma == false when not built
  bool has_tma;
  int tma_tz, tma_tx;            // tile
  int tma_box[3];                // box extent (z, x, planes) in elements
  int tma_halo_z;                // box starts this many elements before the tile
  int tma_elem_bytes;
  size_t tma_smem;
  cudaError_t (*prepare_tma)();
  void (*step_tma)(const StepParams&, const void* tensor_map, dim3 grid, cudaStream_t);
  // 2D axisymmetric (z, r) step on the plain kernel's tile; has_axi == false
  // outside 2D
  bool has_axi;
  cudaError_t (*prepare_axi)();
  void (*step_axi)(const StepParams&, dim3 grid, cudaStream_t);
  // 3D step marching columns of march_tz x march_tx nodes up chunks of
  // march_yc planes; has_march == false outside 3D
  bool has_march;
  int march_tz, march_tx, march_yc;
  cudaError_t (*prepare_march)();
  void (*step_march)(const StepParams&, dim3 grid, cudaStream_t);
  // persistent TMA 2D step (LEC), per_ctas CTAs per SM; has_persist == false when not built;
  // persist_auto: the automatic kernel choice takes it
  bool has_persist, persist_auto;
  int per_tz, per_tx, per_ctas;
  int per_box[3];
  size_t per_smem;
  cudaError_t (*prepare_persist)();
  void (*step_persist)(const StepParams&, const void* tensor_map, int grid, int ntz, int ntiles, cudaStream_t);
  // the same kernel with the axisymmetric rules (axisymmetric LEC runs)
  cudaError_t (*prepare_persist_axi)();
  void (*step_persist_axi)(const StepParams&, const void* tensor_map, int grid, int ntz, int ntiles, cudaStream_t);
};

bool kernels_f64(int dim, int closure, KernelSet* ks);
bool kernels_f32(int dim, int closure, KernelSet* ks);
bool kernels_f16s(int dim, int closure, KernelSet* ks);
bool kernels_f32c(int dim, int closure, KernelSet* ks);

}  // namespace lbp
