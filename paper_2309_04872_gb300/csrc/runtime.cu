// Host runtime of liblbpwfa.so: the C ABI declared in include/lbpwfa.h.
// It owns all device state of a run (double-buffered populations and fields,
// WARMC previous-step values, reduction partials), validates the problem
// statement and queues the kernels of lb_step.cuh / lb_aux.cuh on the
// handle's stream.  No compute happens on the host.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbpwfa.h"
#include "lb_aux.cuh"
#include "lb_batch_dispatch.h"
#include "lb_batch_types.cuh"
#include "lb_diag.cuh"
#include "lb_dispatch.h"
#include "lb_runtime.h"

using namespace lbp;
using namespace lbprt;

namespace {
constexpr int kReduceBlocks = 256;   // fixed: the FP64 sums do not depend on the GPU
constexpr float kF16Scale = 1024.0f; // binary16 deviations are stored times 2^10
}  // namespace

namespace lbprt {

int fail_cuda(lbpwfa_s* h, cudaError_t e, const char* what) {
  if (h) {
    h->err = std::string(what) + ": " + cudaGetErrorString(e);
  }
  return LBPWFA_ERR_CUDA;
}

int alloc(lbpwfa_s* h, Buf& b, size_t bytes) {
  if (bytes == 0) return LBPWFA_OK;
  const size_t cap = h->prm.device_bytes_cap;
  if (cap != 0 && (bytes > cap || h->device_bytes > cap - bytes)) {
    h->err = "device memory cap: " + std::to_string(h->device_bytes + bytes) + " bytes would pass the cap of " +
             std::to_string(cap);
    b.p = nullptr;
    return LBPWFA_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    b.p = nullptr;
    return LBPWFA_ERR_OOM;
  }
  b.bytes = bytes;
  h->device_bytes += bytes;
  return LBPWFA_OK;
}

void release(Buf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

int ensure_scratch(lbpwfa_s* h, size_t bytes) {
  if (h->scratch.bytes >= bytes) return LBPWFA_OK;
  if (h->scratch.p) {
    cudaStreamSynchronize(h->stream);
    h->device_bytes -= h->scratch.bytes;
    release(h->scratch);
  }
  return alloc(h, h->scratch, bytes);
}

int validate(const lbpwfa_params* p) {
  if (!p) return LBPWFA_ERR_INVALID;
  if (p->dim < 1 || p->dim > 3) return LBPWFA_ERR_INVALID;
  for (int a = 0; a < p->dim; ++a)
    if (p->n[a] < 3 || p->n[a] > (1 << 24)) return LBPWFA_ERR_INVALID;
  if (!(p->dx > 0.0) || !std::isfinite(p->dx)) return LBPWFA_ERR_INVALID;
  if (!(p->courant > 0.0) || p->courant > 1.0 / std::sqrt((double)p->dim) + 1e-12) return LBPWFA_ERR_INVALID;
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return LBPWFA_ERR_INVALID;
  if (p->closure != LBPWFA_LEC && p->closure != LBPWFA_WARMC) return LBPWFA_ERR_INVALID;
  if (p->dv != 1 && p->dv != 3) return LBPWFA_ERR_INVALID;
  if (!(p->mu >= 0.0) || !std::isfinite(p->mu)) return LBPWFA_ERR_INVALID;
  if (!std::isfinite(p->alpha) || !std::isfinite(p->z0)) return LBPWFA_ERR_INVALID;
  if (p->profile) {
    if (p->profile_len < 2 || !(p->profile_dz > 0.0)) return LBPWFA_ERR_INVALID;
  } else if (!(p->sigma_z > 0.0)) {
    return LBPWFA_ERR_INVALID;
  }
  if (p->dim >= 2 && !(p->sigma_r > 0.0)) return LBPWFA_ERR_INVALID;
  if (p->precision < LBPWFA_FP64 || p->precision > LBPWFA_FP32C) return LBPWFA_ERR_INVALID;
  if (p->boundary != LBPWFA_OPEN && p->boundary != LBPWFA_PERIODIC) return LBPWFA_ERR_INVALID;
  if (p->kernel_variant < 0 || p->kernel_variant > 4) return LBPWFA_ERR_INVALID;
  if (p->geometry != LBPWFA_CARTESIAN && p->geometry != LBPWFA_AXISYMMETRIC) return LBPWFA_ERR_INVALID;
  // axisymmetric (z, r): 2D, open boundaries, the plain (1) or persistent (3) kernel
  if (p->geometry == LBPWFA_AXISYMMETRIC &&
      (p->dim != 2 || p->boundary != LBPWFA_OPEN || p->kernel_variant == 2 || p->kernel_variant == 4))
    return LBPWFA_ERR_INVALID;
  // the tiled kernels launch (z tiles, x tiles, y tiles) with tiles at least
  // 4 nodes wide in x and y, and a grid's y and z extents are at most 65535
  if (p->dim >= 2 && p->n[1] > 4 * 65535) return LBPWFA_ERR_INVALID;
  if (p->dim >= 3 && p->n[2] > 4 * 65535) return LBPWFA_ERR_INVALID;
  long long cells = 1;
  for (int a = 0; a < p->dim; ++a) cells *= p->n[a];
  if (cells > (1LL << 34)) return LBPWFA_ERR_INVALID;
  if (p->record_tape < 0 || p->checkpoint_every < 0) return LBPWFA_ERR_INVALID;
  return LBPWFA_OK;
}

AuxParams aux_params(const lbpwfa_s* h) {
  AuxParams A{};
  for (int a = 0; a < 3; ++a) A.n[a] = h->n[a];
  A.nzp = h->nzp;
  A.plane = h->plane;
  A.ncell = h->ncell;
  A.periodic = h->prm.boundary == LBPWFA_PERIODIC;
  A.dx = h->prm.dx;
  A.dt = h->dt;
  A.mu = h->prm.mu;
  A.D = h->prm.dv;
  for (int k = 0; k < 11; ++k) {
    A.Arest[k] = h->Arest[k];
    A.scale[k] = h->scale[k];
    A.inv_scale[k] = h->inv_scale[k];
  }
  A.alpha = h->prm.alpha;
  A.inv2sz2 = h->prm.sigma_z > 0 ? 1.0 / (2.0 * h->prm.sigma_z * h->prm.sigma_z) : 0.0;
  A.sigma_r = h->prm.sigma_r;
  A.inv2sr2 = h->prm.sigma_r > 0 ? 1.0 / (2.0 * h->prm.sigma_r * h->prm.sigma_r) : 0.0;
  A.z0 = h->prm.z0;
  A.profile = h->profile_d;
  A.plen = (int)h->profile_h.size();
  A.pdz = h->prm.profile_dz;
  A.axi = h->use_axi ? 1 : 0;
  A.xoff = h->use_axi ? 0.0 : 0.5 * (h->n[1] - 1);  // axisymmetric: node j at r = j dx
  A.yoff = 0.5 * (h->n[2] - 1);
  A.t = h->step * h->dt;
  return A;
}

// Driver centre z0 + step dt, rounded like the batched kernel computes it
// (product, then sum; no fused multiply-add).
double zeta0_of(double z0, long long step, double dt) {
  volatile double t = (double)step * dt;
  return z0 + t;
}

template <typename real>
void fill_consts(const lbpwfa_s* h, StepConst<real>& c) {
  const double dx = h->prm.dx, dt = h->dt;
  c.dx = (real)dx;
  c.idx = (real)(1.0 / dx);
  c.i2dx = (real)(0.5 / dx);
  c.dt = (real)dt;
  c.idt = (real)(1.0 / dt);
  c.courant = (real)h->prm.courant;
  c.inv_tau = (real)(1.0 / h->prm.tau);
  c.mu = (real)h->prm.mu;
  c.cH = (real)((1.0 + 0.5 * h->prm.dv) * h->prm.mu);
  c.zeta0 = (real)zeta0_of(h->prm.z0, h->step, dt);
  c.alpha = (real)h->prm.alpha;
  c.inv2sz2 = (real)(h->prm.sigma_z > 0 ? 1.0 / (2.0 * h->prm.sigma_z * h->prm.sigma_z) : 0.0);
  c.inv2sr2 = (real)(h->prm.sigma_r > 0 ? 1.0 / (2.0 * h->prm.sigma_r * h->prm.sigma_r) : 0.0);
  c.xoff = (real)(h->use_axi ? 0.0 : 0.5 * (h->n[1] - 1));
  c.yoff = (real)(0.5 * (h->n[2] - 1));
  c.pdz_inv = (real)(h->prm.profile_dz > 0 ? 1.0 / h->prm.profile_dz : 0.0);
  c.phalf = (real)(0.5 * ((double)h->profile_h.size() - 1.0));
  for (int k = 0; k < 11; ++k) c.Arest[k] = (real)h->Arest[k];
  const int nth = h->prm.closure == LBPWFA_WARMC ? h->K - 2 - h->prm.dim : 0;
  c.ilam0 = (real)(h->prm.closure == LBPWFA_WARMC ? 1.0 / h->Arest[1] : 0.0);
  for (int j = 0; j < 6; ++j) c.threst[j] = (real)(j < nth ? h->Arest[2 + h->prm.dim + j] / h->Arest[1] : 0.0);
}

StepParams step_params(const lbpwfa_s* h) {
  StepParams P{};
  const int in = h->cur, out = 1 - h->cur;
  P.fin = h->f[in].p;
  P.fout = h->f[out].p;
  P.Ein = h->E[in].p;
  P.Eout = h->E[out].p;
  P.Bin = h->B[in].p;
  P.Bout = h->B[out].p;
  P.Ein_lo = lo_of(h, h->E[in]);
  P.Eout_lo = lo_of(h, h->E[out]);
  P.Bin_lo = lo_of(h, h->B[in]);
  P.Bout_lo = lo_of(h, h->B[out]);
  P.prev = h->prev.p;
  P.have_prev = h->have_prev;
  for (int a = 0; a < 3; ++a) P.n[a] = h->n[a];
  P.nzp = h->nzp;
  P.plane = h->plane;
  P.axis_stride[0] = 1;
  P.axis_stride[1] = h->nzp;
  P.axis_stride[2] = h->nzp * h->n[1];
  P.periodic = h->prm.boundary == LBPWFA_PERIODIC;
  P.D = h->prm.dv;
  P.profile = h->profile_d;
  P.plen = (int)h->profile_h.size();
  for (int k = 0; k < 11; ++k) {
    P.scale[k] = h->scale[k];
    P.inv_scale[k] = h->inv_scale[k];
  }
  P.err = h->err_d;
  P.wait_limit = h->wait_limit;
  fill_consts<float>(h, P.cf);
  fill_consts<double>(h, P.cd);
  return P;
}

dim3 step_grid(const lbpwfa_s* h) {
  return dim3((unsigned)((h->n[0] + h->ks.tz - 1) / h->ks.tz),
              (unsigned)((h->n[1] + h->ks.tx - 1) / h->ks.tx),
              (unsigned)((h->n[2] + h->ks.ty - 1) / h->ks.ty));
}

PFN_cuPointerGetAttribute_v4000 pointer_attr_fn() {
  static PFN_cuPointerGetAttribute_v4000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuPointerGetAttribute_v4000)p;
  }
  return fn;
}

// The device address of a caller's host buffer of `bytes` bytes that the
// device can read and write directly: page-locked memory mapped into the
// device's address space (cudaHostAlloc, cudaMallocHost, cudaHostRegister
// with mapping), aligned for the kernels' 8-byte accesses, the whole buffer
// inside the allocation CUDA reports for it.  Null otherwise (pageable
// memory, or a range CUDA cannot confirm), and the caller stages the copy.
// The import and export kernels then move the values over the host link
// themselves, without a staging copy.
void* mapped_host(const void* p, size_t bytes) {
  if (reinterpret_cast<uintptr_t>(p) % alignof(double) != 0) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const uintptr_t d = reinterpret_cast<uintptr_t>(at.devicePointer);
  if (at.type != cudaMemoryTypeHost || d == 0 || d % alignof(double) != 0) return nullptr;
  PFN_cuPointerGetAttribute_v4000 fn = pointer_attr_fn();
  CUdeviceptr start = 0;
  size_t size = 0;
  if (!fn || fn(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)d) != CUDA_SUCCESS ||
      fn(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)d) != CUDA_SUCCESS)
    return nullptr;
  if (d < start || bytes > size || d - start > size - bytes) return nullptr;
  return at.devicePointer;
}

// Copy device results to a caller buffer (host or device).
int deliver(lbpwfa_s* h, const void* src, void* dst, size_t bytes, int dst_is_device) {
  CK(h, cudaMemcpyAsync(dst, src, bytes, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        h->stream));
  if (!dst_is_device) CK(h, cudaStreamSynchronize(h->stream));
  return LBPWFA_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// Tensor map of one population buffer viewed as [NPL planes][nx rows][nzp]:
// the step's box is (z, x, planes) = ks.tma_box.
bool make_pop_map(lbpwfa_s* h, void* base, CUtensorMap* map, const int* boxdim) {
  auto enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t es = (cuuint64_t)h->ks.tma_elem_bytes;
  const CUtensorMapDataType dt = es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                               : (es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
  cuuint64_t dims[3] = {(cuuint64_t)h->nzp, (cuuint64_t)h->n[1], (cuuint64_t)h->NPL};
  cuuint64_t strides[2] = {(cuuint64_t)h->nzp * es, (cuuint64_t)h->plane * es};
  cuuint32_t box[3] = {(cuuint32_t)boxdim[0], (cuuint32_t)boxdim[1], (cuuint32_t)boxdim[2]};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// The state was replaced: a timeout flagged before no longer applies.
int clear_err_word(lbpwfa_s* h) {
  CK(h, cudaMemsetAsync(h->err_d, 0, sizeof(int), h->stream));
  return LBPWFA_OK;
}

int check_err_word(lbpwfa_s* h) {
  int v = 0;
  CK(h, cudaMemcpyAsync(&v, h->err_d, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  if (v != 0) {
    h->err = "a bounded device wait gave up";
    return LBPWFA_ERR_TIMEOUT;
  }
  return LBPWFA_OK;
}

// Rest state n = 1, u = 0 (all stored deviations zero: every storage format
// encodes 0 as zero bits), the initial driver field, step 0.
int init_rest_state(lbpwfa_s* h) {
  const size_t pop_bytes = h->f[0].bytes, fld_bytes = h->E[0].bytes;
  for (int j = 0; j < 2; ++j) {
    CK(h, cudaMemsetAsync(h->f[j].p, 0, pop_bytes, h->stream));
    CK(h, cudaMemsetAsync(h->E[j].p, 0, fld_bytes, h->stream));
    CK(h, cudaMemsetAsync(h->B[j].p, 0, fld_bytes, h->stream));
  }
  if (h->prev.p) CK(h, cudaMemsetAsync(h->prev.p, 0, h->prev.bytes, h->stream));
  if (h->prm.init_fields && h->prm.dim >= 2) {
    AuxParams A = aux_params(h);
    A.t = 0.0;
    h->ks.init_fields(A, h->E[0].p, h->B[0].p, lo_of(h, h->E[0]), lo_of(h, h->B[0]), h->stream);
    CK_LAUNCH(h, "init_fields");
  }
  h->fields_from_driver = h->prm.init_fields && h->prm.dim >= 2;
  h->cur = 0;
  h->step = 0;
  h->have_prev = 0;
  return LBPWFA_OK;
}

uint32_t crc32_update(uint32_t crc, const void* data, size_t len) {
  static uint32_t table[256];
  static bool init = false;
  if (!init) {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int j = 0; j < 8; ++j) c = (c & 1) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      table[i] = c;
    }
    init = true;
  }
  const unsigned char* p = (const unsigned char*)data;
  crc = ~crc;
  for (size_t i = 0; i < len; ++i) crc = table[(crc ^ p[i]) & 0xFF] ^ (crc >> 8);
  return ~crc;
}

// One step of the single-run kernel in use; tape != null records the step's
// adjoint inputs (lb_step.cuh).
int launch_step(lbpwfa_s* h, void* tape) {
  const dim3 grid = h->use_tma ? dim3((unsigned)((h->n[0] + h->ks.tma_tz - 1) / h->ks.tma_tz),
                                      (unsigned)((h->n[1] + h->ks.tma_tx - 1) / h->ks.tma_tx), 1)
                               : step_grid(h);
  StepParams P = step_params(h);
  P.tape = tape;
  if (h->use_persist) {
    const int ntz = (h->n[0] + h->ks.per_tz - 1) / h->ks.per_tz;
    const int ntiles = ntz * ((h->n[1] + h->ks.per_tx - 1) / h->ks.per_tx);
    const int slots = h->num_sms * h->ks.per_ctas;
    const int pgrid = ntiles < slots ? ntiles : slots;
    if (h->use_axi) h->ks.step_persist_axi(P, &h->maps[h->cur], pgrid, ntz, ntiles, h->stream);
    else h->ks.step_persist(P, &h->maps[h->cur], pgrid, ntz, ntiles, h->stream);
  } else if (h->use_axi) {
    h->ks.step_axi(P, grid, h->stream);
  } else if (h->use_march) {
    const dim3 mg((unsigned)((h->n[0] + h->ks.march_tz - 1) / h->ks.march_tz),
                  (unsigned)((h->n[1] + h->ks.march_tx - 1) / h->ks.march_tx),
                  (unsigned)((h->n[2] + h->ks.march_yc - 1) / h->ks.march_yc));
    h->ks.step_march(P, mg, h->stream);
  } else if (h->use_tma) {
    h->ks.step_tma(P, &h->maps[h->cur], grid, h->stream);
  } else {
    h->ks.step(P, grid, h->stream);
  }
  CK_LAUNCH(h, "lb_step_kernel launch");
  h->cur = 1 - h->cur;
  h->step += 1;
  if (h->NPREV) h->have_prev = 1;
  return LBPWFA_OK;
}

// The step kernel of a kernel variant (lbpwfa_params.kernel_variant; the
// axisymmetric geometry's own rules are set by lbpwfa_create).  A variant
// the run cannot take falls back to the plain kernel, which computes the
// same step.
void select_kernel(lbpwfa_s* h, int variant) {
  const int dim = h->prm.dim;
  // 3D: marching columns unless the tiled kernel is asked for (variant 1)
  h->use_march = dim == 3 && (variant == 0 || variant == 4) && h->ks.has_march;
  if (h->use_march && h->ks.prepare_march() != cudaSuccess) {
    cudaGetLastError();
    h->use_march = false;
  }
  const bool tma_ok = dim == 2 && h->prm.boundary == LBPWFA_OPEN;
  // automatic choice for LEC: the persistent refilling CTAs where the tile
  // table marks them faster, else one TMA box per CTA; WARMC's 72-plane box
  // leaves two CTAs per SM and the global-memory pull is faster there
  const bool persist_auto = variant == 0 && h->prm.closure == LBPWFA_LEC && h->ks.persist_auto;
  h->use_persist = (variant == 3 || persist_auto) && tma_ok && h->ks.has_persist && h->num_sms > 0;
  if (h->use_persist) {
    cudaError_t e = h->use_axi ? h->ks.prepare_persist_axi() : h->ks.prepare_persist();
    bool ok = e == cudaSuccess && make_pop_map(h, h->f[0].p, &h->maps[0], h->ks.per_box) &&
              make_pop_map(h, h->f[1].p, &h->maps[1], h->ks.per_box);
    if (!ok) {
      cudaGetLastError();
      h->use_persist = false;
    }
  }
  const bool tma_auto = variant == 0 && h->prm.closure == LBPWFA_LEC;
  h->use_tma = !h->use_persist && !h->use_axi && (tma_auto || variant == 2) && tma_ok && h->ks.has_tma;
  if (h->use_tma) {
    cudaError_t e = h->ks.prepare_tma();
    bool ok = e == cudaSuccess && make_pop_map(h, h->f[0].p, &h->maps[0], h->ks.tma_box) &&
              make_pop_map(h, h->f[1].p, &h->maps[1], h->ks.tma_box);
    if (!ok) {
      cudaGetLastError();
      h->use_tma = false;  // the plain kernel computes the same step
    }
  }
}

// The variant the run's step uses, as lbpwfa_info reports it.
int variant_in_use(const lbpwfa_s* h) {
  return h->use_persist ? 3 : (h->use_axi ? 5 : (h->use_march ? 4 : (h->use_tma ? 2 : 1)));
}

}  // namespace lbprt

extern "C" {

const char* lbpwfa_status_string(int s) {
  switch (s) {
    case LBPWFA_OK: return "ok";
    case LBPWFA_ERR_INVALID: return "invalid argument";
    case LBPWFA_ERR_OOM: return "out of memory";
    case LBPWFA_ERR_CUDA: return "CUDA error";
    case LBPWFA_ERR_NONFINITE: return "non-finite populations";
    case LBPWFA_ERR_TIMEOUT: return "device wait timed out";
    case LBPWFA_ERR_STATE: return "invalid state";
    case LBPWFA_ERR_IO: return "checkpoint I/O error";
    default: return "unknown status";
  }
}

const char* lbpwfa_last_error(lbpwfa_t h) { return h ? h->err.c_str() : ""; }

static void destroy_run(lbpwfa_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  adj_free(h);
  for (int j = 0; j < 2; ++j) { release(h->f[j]); release(h->E[j]); release(h->B[j]); }
  release(h->prev);
  release(h->partial);
  release(h->out3);
  release(h->scratch);
  if (h->err_d) cudaFree(h->err_d);
  if (h->profile_d) cudaFree(h->profile_d);
  if (h->owns_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

void lbpwfa_destroy(lbpwfa_t h) {
  if (!h || h->in_batch) return;
  destroy_run(h);
}

int lbpwfa_create(const lbpwfa_params* p, lbpwfa_t* out) {
  if (!out) return LBPWFA_ERR_INVALID;
  *out = nullptr;
  int st = validate(p);
  if (st != LBPWFA_OK) return st;
  lbpwfa_s* h = new lbpwfa_s();
  h->prm = *p;
  h->prm.profile = nullptr;
  if (p->profile) h->profile_h.assign(p->profile, p->profile + p->profile_len);
  const int dim = p->dim;
  bool ok = false;
  if (p->precision == LBPWFA_FP64) ok = kernels_f64(dim, p->closure, &h->ks);
  else if (p->precision == LBPWFA_FP32) ok = kernels_f32(dim, p->closure, &h->ks);
  else if (p->precision == LBPWFA_FP32C) ok = kernels_f32c(dim, p->closure, &h->ks);
  else ok = kernels_f16s(dim, p->closure, &h->ks);
  if (!ok) { delete h; return LBPWFA_ERR_INVALID; }

  h->Q = dim == 1 ? 3 : (dim == 2 ? 9 : 19);
  const int nth = p->closure == LBPWFA_WARMC ? (dim == 1 ? 1 : (dim == 2 ? 4 : 6)) : 0;
  h->K = p->closure == LBPWFA_LEC ? 1 + dim : 2 + dim + nth;
  h->NPREV = p->closure == LBPWFA_WARMC ? 1 + 2 * dim : 0;
  for (int a = 0; a < 3; ++a) h->n[a] = a < dim ? p->n[a] : 1;
  h->nzp = (h->n[0] + 31) / 32 * 32;
  h->plane = (long long)h->nzp * h->n[1] * h->n[2];
  h->ncell = (long long)h->n[0] * h->n[1] * h->n[2];
  if ((long long)h->Q * h->plane >= (1LL << 31)) { delete h; return LBPWFA_ERR_INVALID; }  // 32-bit plane offsets
  h->store_sz = p->precision == LBPWFA_FP64 ? 8 : (p->precision == LBPWFA_FP16S ? 2 : 4);
  h->real_sz = p->precision == LBPWFA_FP64 ? 8 : 4;
  h->dt = p->courant * p->dx;
  h->NPL = h->K * h->Q + (p->precision == LBPWFA_FP16S ? h->K : 0);
  if (p->device_bytes_cap != 0) {
    // the state's size against the cap, before any CUDA call
    const double need = 2.0 * h->NPL * (double)h->plane * h->store_sz +
                        4.0 * 3.0 * (double)h->plane * h->real_sz * (h->real_sz == 4 ? 2.0 : 1.0) +
                        (double)h->NPREV * h->plane * h->real_sz;
    if (need > (double)p->device_bytes_cap) { delete h; return LBPWFA_ERR_OOM; }
  }

  // Rest advected values.  WARMC: Eq. (traces3) at rest (theta^{00} = 0,
  // theta^{ij} = mu delta^{ij} over the D kinetic dimensions, n_0 = 1):
  // h^2 + D mu h - 1 = 0, lambda = 1/h.
  h->Arest[0] = 1.0;
  if (p->closure == LBPWFA_WARMC) {
    const double D = p->dv, mu = p->mu;
    const double h0 = 2.0 / (D * mu + std::sqrt(D * D * mu * mu + 4.0));
    const double lam0 = 1.0 / h0;
    h->Arest[1] = lam0;
    const int ta[6] = {0, 1, 2, 0, 0, 1}, tb[6] = {0, 1, 2, 1, 2, 2};
    for (int j = 0; j < nth; ++j) {
      const bool diag = ta[j] == tb[j];
      const double th = (diag && (p->dv == 3 || ta[j] == 0)) ? mu : 0.0;
      h->Arest[2 + dim + j] = lam0 * th;
    }
  }
  for (int k = 0; k < 11; ++k) {
    h->scale[k] = p->precision == LBPWFA_FP16S ? kF16Scale : 1.0f;
    h->inv_scale[k] = 1.0f / h->scale[k];
  }

  if (p->stream) {
    h->stream = (cudaStream_t)p->stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { int r = fail_cuda(h, e, "cudaStreamCreate"); lbpwfa_destroy(h); return r; }
    h->owns_stream = true;
  }
  cudaError_t pe = h->ks.prepare();
  if (pe != cudaSuccess) { fail_cuda(h, pe, "cudaFuncSetAttribute"); lbpwfa_destroy(h); return LBPWFA_ERR_CUDA; }

  // FP16S: one more plane per set for the rest population's low part (NPL)
  const size_t pop_bytes = (size_t)h->NPL * h->plane * h->store_sz;
  const size_t fld_bytes = 3 * (size_t)h->plane * h->real_sz * (h->real_sz == 4 ? 2 : 1);
  int r = LBPWFA_OK;
  for (int j = 0; j < 2 && r == LBPWFA_OK; ++j) {
    r = alloc(h, h->f[j], pop_bytes);
    if (r == LBPWFA_OK) r = alloc(h, h->E[j], fld_bytes);
    if (r == LBPWFA_OK) r = alloc(h, h->B[j], fld_bytes);
  }
  if (r == LBPWFA_OK && h->NPREV) r = alloc(h, h->prev, (size_t)h->NPREV * h->plane * h->real_sz);
  if (r == LBPWFA_OK) r = alloc(h, h->partial, (size_t)kReduceBlocks * 3 * sizeof(double));
  if (r == LBPWFA_OK) r = alloc(h, h->out3, 4 * sizeof(double));
  if (r != LBPWFA_OK) { lbpwfa_destroy(h); return r; }
  {
    cudaError_t e = cudaMalloc(&h->err_d, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err_d, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) { int rr = fail_cuda(h, e, "error word"); lbpwfa_destroy(h); return rr; }
  }
  {
    int dev = 0;
    cudaGetDevice(&dev);
    h->device = dev;
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  // axisymmetric (z, r) grids: the plain kernel with the axis rules
  h->use_axi = p->geometry == LBPWFA_AXISYMMETRIC;
  if (h->use_axi) {
    cudaError_t e = h->ks.has_axi ? h->ks.prepare_axi() : cudaErrorNotSupported;
    if (e != cudaSuccess) { fail_cuda(h, e, "cudaFuncSetAttribute"); lbpwfa_destroy(h); return LBPWFA_ERR_CUDA; }
  }
  select_kernel(h, p->kernel_variant);
  if (!h->profile_h.empty()) {
    cudaError_t e = cudaMalloc(&h->profile_d, h->profile_h.size() * sizeof(double));
    if (e != cudaSuccess) { lbpwfa_destroy(h); return LBPWFA_ERR_OOM; }
    e = cudaMemcpyAsync(h->profile_d, h->profile_h.data(), h->profile_h.size() * sizeof(double),
                        cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) { int rr = fail_cuda(h, e, "profile upload"); lbpwfa_destroy(h); return rr; }
  }
  r = init_rest_state(h);
  if (r != LBPWFA_OK) { lbpwfa_destroy(h); return r; }
  h->cur = 0;
  h->step = 0;
  h->have_prev = 0;
  if (p->record_tape > 0) {
    // the adjoint window the parameters ask for, from step 0
    const lbpwfa_record_params rp{p->record_tape, p->checkpoint_every};
    r = lbpwfa_record(h, &rp);
    if (r != LBPWFA_OK) { lbpwfa_destroy(h); return r; }
  }
  *out = h;
  return LBPWFA_OK;
}

int lbpwfa_step(lbpwfa_t h, int64_t nsteps) {
  if (!h || nsteps < 0) return LBPWFA_ERR_INVALID;
  if (h->in_batch) {
    h->err = "lbpwfa_step: this run belongs to a batch; use lbpwfa_batch_step";
    return LBPWFA_ERR_STATE;
  }
  for (int64_t s = 0; s < nsteps; ++s) {
    void* tape = nullptr;
    int r = adj_before_step(h, &tape);
    if (r != LBPWFA_OK) return r;
    r = launch_step(h, tape);
    if (r != LBPWFA_OK) return r;
  }
  return LBPWFA_OK;
}

int lbpwfa_advected(lbpwfa_t h, double* dst, size_t count, int dst_is_device) {
  if (!h || !dst) return LBPWFA_ERR_INVALID;
  const size_t need = (size_t)h->K * h->ncell;
  if (count < need) return LBPWFA_ERR_INVALID;
  AuxParams A = aux_params(h);
  double* out = dst;
  double* mapped = dst_is_device ? nullptr : (double*)mapped_host(dst, need * sizeof(double));
  if (mapped) {
    out = mapped;
  } else if (!dst_is_device) {
    int r = ensure_scratch(h, need * sizeof(double));
    if (r != LBPWFA_OK) return r;
    out = (double*)h->scratch.p;
  }
  h->ks.advected(A, h->f[h->cur].p, out, h->stream);
  CK_LAUNCH(h, "advected_kernel launch");
  if (mapped) CK(h, cudaStreamSynchronize(h->stream));
  else if (!dst_is_device) return deliver(h, out, dst, need * sizeof(double), 0);
  return LBPWFA_OK;
}

int lbpwfa_moments(lbpwfa_t h, uint32_t mask, double* dst, size_t count, int dst_is_device) {
  if (!h || !dst) return LBPWFA_ERR_INVALID;
  mask &= 0x3FFFFu;
  int nb = 0;
  for (int b = 0; b < 18; ++b) nb += (mask >> b) & 1u;
  const size_t need = (size_t)nb * h->ncell;
  if (nb == 0) return LBPWFA_OK;
  if (count < need) return LBPWFA_ERR_INVALID;
  AuxParams A = aux_params(h);
  double* out = dst;
  double* mapped = dst_is_device ? nullptr : (double*)mapped_host(dst, need * sizeof(double));
  if (mapped) {
    out = mapped;
  } else if (!dst_is_device) {
    int r = ensure_scratch(h, need * sizeof(double));
    if (r != LBPWFA_OK) return r;
    out = (double*)h->scratch.p;
  }
  h->ks.moments(A, h->f[h->cur].p, mask, out, h->stream);
  CK_LAUNCH(h, "moments_kernel launch");
  if (mapped) CK(h, cudaStreamSynchronize(h->stream));
  else if (!dst_is_device) return deliver(h, out, dst, need * sizeof(double), 0);
  return LBPWFA_OK;
}

int lbpwfa_fields(lbpwfa_t h, uint32_t mask, double* dst, size_t count, int dst_is_device) {
  if (!h || !dst) return LBPWFA_ERR_INVALID;
  mask &= 0x3Fu;
  // bits: E_x, E_y, E_z, B_x, B_y, B_z -> internal component (z=0, x=1, y=2)
  const int comp_of_bit[6] = {1, 2, 0, 1, 2, 0};
  int comps[6], isb[6], nb = 0;
  for (int b = 0; b < 6; ++b)
    if (mask & (1u << b)) { comps[nb] = comp_of_bit[b]; isb[nb] = b >= 3; ++nb; }
  if (nb == 0) return LBPWFA_OK;
  const size_t need = (size_t)nb * h->ncell;
  if (count < need) return LBPWFA_ERR_INVALID;
  AuxParams A = aux_params(h);
  double* out = dst;
  double* mapped = dst_is_device ? nullptr : (double*)mapped_host(dst, need * sizeof(double));
  if (mapped) {
    out = mapped;
  } else if (!dst_is_device) {
    int r = ensure_scratch(h, need * sizeof(double));
    if (r != LBPWFA_OK) return r;
    out = (double*)h->scratch.p;
  }
  for (int j0 = 0; j0 < nb; j0 += 4) {
    const int m = nb - j0 < 4 ? nb - j0 : 4;
    int c4[4] = {0, 0, 0, 0}, b4[4] = {0, 0, 0, 0};
    for (int j = 0; j < m; ++j) { c4[j] = comps[j0 + j]; b4[j] = isb[j0 + j]; }
    h->ks.export_fields(A, h->E[h->cur].p, h->B[h->cur].p, lo_of(h, h->E[h->cur]), lo_of(h, h->B[h->cur]), m,
                        make_int4(c4[0], c4[1], c4[2], c4[3]),
                        make_int4(b4[0], b4[1], b4[2], b4[3]), out + (size_t)j0 * h->ncell, h->stream);
    CK_LAUNCH(h, "export_fields_kernel launch");
  }
  if (mapped) CK(h, cudaStreamSynchronize(h->stream));
  else if (!dst_is_device) return deliver(h, out, dst, need * sizeof(double), 0);
  return LBPWFA_OK;
}

int lbpwfa_line_fit(lbpwfa_t h, const lbpwfa_fit_params* fp, double* out) {
  if (!h || !fp || !out) return LBPWFA_ERR_INVALID;
  if (fp->quantity != LBPWFA_FIT_EZ && fp->quantity != LBPWFA_FIT_N) return LBPWFA_ERR_INVALID;
  const int dim = h->prm.dim;
  const int ix = dim >= 2 ? fp->line[0] : 0, iy = dim >= 3 ? fp->line[1] : 0;
  if (ix < 0 || ix >= h->n[1] || iy < 0 || iy >= h->n[2]) return LBPWFA_ERR_INVALID;
  if (fp->nk < 3 || fp->nk > 65536) return LBPWFA_ERR_INVALID;
  if (!std::isfinite(fp->k_lo) || !std::isfinite(fp->k_hi) || !(fp->k_hi > fp->k_lo)) return LBPWFA_ERR_INVALID;
  if (!std::isfinite(fp->xi_lo) || !std::isfinite(fp->xi_hi) || !(fp->xi_hi > fp->xi_lo)) return LBPWFA_ERR_INVALID;
  const size_t nres = (size_t)fp->nk + 8;
  int r = ensure_scratch(h, ((size_t)h->ncell + nres) * sizeof(double));
  if (r != LBPWFA_OK) return r;
  double* q = (double*)h->scratch.p;
  double* res = q + h->ncell;
  AuxParams A = aux_params(h);
  if (fp->quantity == LBPWFA_FIT_N) {
    h->ks.moments(A, h->f[h->cur].p, 1u, q, h->stream);
  } else {
    h->ks.export_fields(A, h->E[h->cur].p, h->B[h->cur].p, lo_of(h, h->E[h->cur]), lo_of(h, h->B[h->cur]), 1,
                        make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0), q, h->stream);
  }
  CK_LAUNCH(h, "line_fit export");
  FitLine L{};
  L.q = q;
  L.base = (long long)h->n[0] * ((long long)ix + (long long)h->n[1] * iy);
  L.nz = h->n[0];
  // the populations are at t_n, the stored E at t_{n-1/2}
  const double t = fp->quantity == LBPWFA_FIT_N ? (double)h->step * h->dt : ((double)h->step - 0.5) * h->dt;
  L.zd = h->prm.z0 + t;
  L.dx = h->prm.dx;
  L.offset = fp->quantity == LBPWFA_FIT_N ? 1.0 : 0.0;
  L.xi_lo = fp->xi_lo;
  L.xi_hi = fp->xi_hi;
  L.k_lo = fp->k_lo;
  L.dk = (fp->k_hi - fp->k_lo) / (double)(fp->nk - 1);
  L.nk = fp->nk;
  fit_scan_kernel<<<fp->nk, kFitThreads, 0, h->stream>>>(L, res);
  CK_LAUNCH(h, "fit_scan_kernel");
  fit_pick_kernel<<<1, kFitThreads, 0, h->stream>>>(L, res, res + fp->nk);
  CK_LAUNCH(h, "fit_pick_kernel");
  return deliver(h, res + fp->nk, out, 5 * sizeof(double), 0);
}

int lbpwfa_gauss_residual(lbpwfa_t h, const int* lo, const int* hi, double* out) {
  if (!h || !lo || !hi || !out) return LBPWFA_ERR_INVALID;
  const int dim = h->prm.dim;
  GaussArgs G{};
  G.dim = dim;
  G.ncells = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      if (lo[a] < 0 || hi[a] > h->n[a] - 1 || lo[a] >= hi[a]) return LBPWFA_ERR_INVALID;
      G.lo[a] = lo[a];
      G.hi[a] = hi[a];
    } else {
      G.lo[a] = 0;
      G.hi[a] = 1;
    }
    G.ncells *= G.hi[a] - G.lo[a];
  }
  constexpr int nblk = 256;
  int r = ensure_scratch(h, (4 * (size_t)h->ncell + 2 * nblk + 4) * sizeof(double));
  if (r != LBPWFA_OK) return r;
  double* nbuf = (double*)h->scratch.p;
  double* Ebuf = nbuf + h->ncell;
  double* part = Ebuf + 3 * (size_t)h->ncell;
  double* res = part + 2 * nblk;
  AuxParams A = aux_params(h);
  h->ks.moments(A, h->f[h->cur].p, 1u, nbuf, h->stream);
  CK_LAUNCH(h, "gauss_residual density");
  h->ks.export_fields(A, h->E[h->cur].p, h->B[h->cur].p, lo_of(h, h->E[h->cur]), lo_of(h, h->B[h->cur]), 3,
                      make_int4(0, 1, 2, 0), make_int4(0, 0, 0, 0), Ebuf, h->stream);
  CK_LAUNCH(h, "gauss_residual fields");
  A.t = ((double)h->step - 0.5) * h->dt;  // the stored E is at t_{n-1/2}
  G.A = A;
  G.n = nbuf;
  G.E = Ebuf;
  gauss_partial_kernel<<<nblk, 256, 0, h->stream>>>(G, part);
  CK_LAUNCH(h, "gauss_partial_kernel");
  gauss_final_kernel<<<1, 32, 0, h->stream>>>(part, nblk, G.ncells, res);
  CK_LAUNCH(h, "gauss_final_kernel");
  return deliver(h, res, out, 3 * sizeof(double), 0);
}

int lbpwfa_set_state(lbpwfa_t h, const double* f, const double* E, const double* B, int src_is_device) {
  if (!h) return LBPWFA_ERR_INVALID;
  AuxParams A = aux_params(h);
  const size_t nf = (size_t)h->K * h->Q * h->ncell, nfl = 3 * (size_t)h->ncell;
  const double *fd = f, *Ed = E, *Bd = B;
  // page-locked host buffers mapped into the device are read in place
  bool mapped = !src_is_device;
  if (mapped) {
    const double* fm = f ? (const double*)mapped_host(f, nf * sizeof(double)) : nullptr;
    const double* Em = E ? (const double*)mapped_host(E, nfl * sizeof(double)) : nullptr;
    const double* Bm = B ? (const double*)mapped_host(B, nfl * sizeof(double)) : nullptr;
    mapped = (!f || fm) && (!E || Em) && (!B || Bm);
    if (mapped) { fd = fm; Ed = Em; Bd = Bm; }
  }
  size_t need = 0;
  if (!src_is_device && !mapped) need = (f ? nf : 0) + (E ? nfl : 0) + (B ? nfl : 0);
  if (need) {
    int r = ensure_scratch(h, need * sizeof(double));
    if (r != LBPWFA_OK) return r;
  }
  double* sp = (double*)h->scratch.p;
  if (!src_is_device && !mapped) {
    size_t o = 0;
    if (f) { CK(h, cudaMemcpyAsync(sp + o, f, nf * 8, cudaMemcpyHostToDevice, h->stream)); fd = sp + o; o += nf; }
    if (E) { CK(h, cudaMemcpyAsync(sp + o, E, nfl * 8, cudaMemcpyHostToDevice, h->stream)); Ed = sp + o; o += nfl; }
    if (B) { CK(h, cudaMemcpyAsync(sp + o, B, nfl * 8, cudaMemcpyHostToDevice, h->stream)); Bd = sp + o; o += nfl; }
  }
  if (fd) {
    h->ks.import_pops(A, fd, h->f[h->cur].p, h->stream);
    CK_LAUNCH(h, "import_pops_kernel launch");
  }
  if (Ed || Bd) {
    h->ks.import_fields(A, Ed, Bd, h->E[h->cur].p, h->B[h->cur].p, lo_of(h, h->E[h->cur]), lo_of(h, h->B[h->cur]),
                        h->stream);
    CK_LAUNCH(h, "import_fields_kernel launch");
    h->fields_from_driver = false;
  }
  adj_invalidate(h);
  h->have_prev = 0;
  {
    int r = clear_err_word(h);
    if (r != LBPWFA_OK) return r;
  }
  if (!src_is_device) CK(h, cudaStreamSynchronize(h->stream));
  return LBPWFA_OK;
}

int lbpwfa_get_state(lbpwfa_t h, double* f, double* E, double* B, int dst_is_device) {
  if (!h) return LBPWFA_ERR_INVALID;
  AuxParams A = aux_params(h);
  const size_t nf = (size_t)h->K * h->Q * h->ncell, nfl = 3 * (size_t)h->ncell;
  bool any_mapped = false;
  if (f) {
    double* out = f;
    double* mapped = dst_is_device ? nullptr : (double*)mapped_host(f, nf * 8);
    if (mapped) {
      out = mapped;
      any_mapped = true;
    } else if (!dst_is_device) {
      int r = ensure_scratch(h, nf * 8);
      if (r != LBPWFA_OK) return r;
      out = (double*)h->scratch.p;
    }
    h->ks.export_pops(A, h->f[h->cur].p, out, h->stream);
    CK_LAUNCH(h, "export_pops_kernel launch");
    if (!dst_is_device && !mapped) {
      int r = deliver(h, out, f, nf * 8, 0);
      if (r != LBPWFA_OK) return r;
    }
  }
  // E and B in the ABI's component order z, x, y
  for (int which = 0; which < 2; ++which) {
    double* dst = which == 0 ? E : B;
    if (!dst) continue;
    double* out = dst;
    double* mapped = dst_is_device ? nullptr : (double*)mapped_host(dst, nfl * 8);
    if (mapped) {
      out = mapped;
      any_mapped = true;
    } else if (!dst_is_device) {
      int r = ensure_scratch(h, nfl * 8);
      if (r != LBPWFA_OK) return r;
      out = (double*)h->scratch.p;
    }
    h->ks.export_fields(A, h->E[h->cur].p, h->B[h->cur].p, lo_of(h, h->E[h->cur]), lo_of(h, h->B[h->cur]), 3,
                        make_int4(0, 1, 2, 0),
                        make_int4(which, which, which, 0), out, h->stream);
    CK_LAUNCH(h, "export_fields_kernel launch");
    if (!dst_is_device && !mapped) {
      int r = deliver(h, out, dst, nfl * 8, 0);
      if (r != LBPWFA_OK) return r;
    }
  }
  if (any_mapped) CK(h, cudaStreamSynchronize(h->stream));
  return LBPWFA_OK;
}

int lbpwfa_reduce(lbpwfa_t h, double out[3]) {
  if (!h || !out) return LBPWFA_ERR_INVALID;
  AuxParams A = aux_params(h);
  h->ks.reduce_partial(A, h->f[h->cur].p, (double*)h->partial.p, kReduceBlocks, h->stream);
  CK_LAUNCH(h, "reduce_partial_kernel launch");
  reduce_final_kernel<<<1, 32, 0, h->stream>>>((const double*)h->partial.p, kReduceBlocks, (double*)h->out3.p);
  CK_LAUNCH(h, "reduce_final_kernel launch");
  CK(h, cudaMemcpyAsync(out, h->out3.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  int st = check_err_word(h);
  if (st != LBPWFA_OK) return st;
  return out[2] > 0 ? LBPWFA_ERR_NONFINITE : LBPWFA_OK;
}

int lbpwfa_info(lbpwfa_t h, lbpwfa_info_t* info) {
  if (!h || !info) return LBPWFA_ERR_INVALID;
  info->K = h->K;
  info->Q = h->Q;
  info->ncell = h->ncell;
  info->step = h->step;
  info->dt = h->dt;
  info->time = h->step * h->dt;
  info->device_bytes = h->device_bytes;
  const int dim = h->prm.dim;
  const int ne = dim == 1 ? 1 : (dim == 2 ? 2 : 3);
  const int nbf = dim == 1 ? 0 : (dim == 2 ? 1 : 3);
  // FP32 fields: high and low parts
  const double field_words = (ne + nbf) * (h->real_sz == 4 ? 2.0 : 1.0);
  info->bytes_per_update = 2.0 * h->NPL * h->store_sz + 2.0 * (field_words + h->NPREV) * h->real_sz;
  info->kernel_variant = variant_in_use(h);
  // the method's bytes: populations, one real per field component, and the
  // WARMC previous-step theta^{0 beta}, w^beta (beta = 0..dim)
  const int nalg_prev = h->prm.closure == LBPWFA_WARMC ? 2 * (1 + dim) : 0;
  info->algorithmic_bytes_per_update =
      2.0 * h->K * h->Q * h->store_sz + 2.0 * (ne + nbf) * h->real_sz + 2.0 * nalg_prev * h->real_sz;
  return LBPWFA_OK;
}

int lbpwfa_set_stream(lbpwfa_t h, void* stream) {
  if (!h) return LBPWFA_ERR_INVALID;
  CK(h, cudaStreamSynchronize(h->stream));
  if (stream) {
    if (h->owns_stream) { cudaStreamDestroy(h->stream); h->owns_stream = false; }
    h->stream = (cudaStream_t)stream;
  } else if (!h->owns_stream) {
    CK(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->owns_stream = true;
  }
  return LBPWFA_OK;
}

int lbpwfa_synchronize(lbpwfa_t h) {
  if (!h) return LBPWFA_ERR_INVALID;
  CK(h, cudaStreamSynchronize(h->stream));
  return check_err_word(h);
}

int lbpwfa_set_wait_limit(lbpwfa_t h, uint32_t polls) {
  if (!h) return LBPWFA_ERR_INVALID;
  h->wait_limit = polls;
  return LBPWFA_OK;
}

// ---------------------------------------------------------------------------
// Checkpoints.
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version;
  int32_t dim, n0, n1, n2, closure, dv, precision, boundary, K, Q, have_prev;
  int32_t from_driver;  // E, B still the driver's initial fields
  int32_t geometry;     // LBPWFA_CARTESIAN (0 in files written before it existed) or AXISYMMETRIC
  int64_t step;
  double dx, courant, tau, mu, alpha, sigma_z, sigma_r, z0;
  uint64_t pop_bytes, fld_bytes, prev_bytes;
};
}  // namespace

int lbpwfa_save(lbpwfa_t h, const char* path) {
  if (!h || !path) return LBPWFA_ERR_INVALID;
  CkptHeader H{};
  std::memcpy(H.magic, "LBPWFA02", 8);
  H.version = 1;
  H.dim = h->prm.dim; H.n0 = h->n[0]; H.n1 = h->n[1]; H.n2 = h->n[2];
  H.closure = h->prm.closure; H.dv = h->prm.dv; H.precision = h->prm.precision; H.boundary = h->prm.boundary;
  H.K = h->K; H.Q = h->Q; H.have_prev = h->have_prev; H.step = h->step;
  H.from_driver = h->fields_from_driver ? 1 : 0;
  H.geometry = h->prm.geometry;
  H.dx = h->prm.dx; H.courant = h->prm.courant; H.tau = h->prm.tau; H.mu = h->prm.mu;
  H.alpha = h->prm.alpha; H.sigma_z = h->prm.sigma_z; H.sigma_r = h->prm.sigma_r; H.z0 = h->prm.z0;
  H.pop_bytes = h->f[h->cur].bytes; H.fld_bytes = h->E[h->cur].bytes; H.prev_bytes = h->prev.bytes;
  std::vector<char> buf(H.pop_bytes + 2 * H.fld_bytes + H.prev_bytes);
  char* q = buf.data();
  CK(h, cudaMemcpyAsync(q, h->f[h->cur].p, H.pop_bytes, cudaMemcpyDeviceToHost, h->stream));
  q += H.pop_bytes;
  CK(h, cudaMemcpyAsync(q, h->E[h->cur].p, H.fld_bytes, cudaMemcpyDeviceToHost, h->stream));
  q += H.fld_bytes;
  CK(h, cudaMemcpyAsync(q, h->B[h->cur].p, H.fld_bytes, cudaMemcpyDeviceToHost, h->stream));
  q += H.fld_bytes;
  if (H.prev_bytes) CK(h, cudaMemcpyAsync(q, h->prev.p, H.prev_bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  uint32_t crc = crc32_update(0, &H, sizeof(H));
  crc = crc32_update(crc, buf.data(), buf.size());
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return LBPWFA_ERR_IO;
  bool ok = std::fwrite(&H, sizeof(H), 1, fp) == 1 && std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size() &&
            std::fwrite(&crc, sizeof(crc), 1, fp) == 1;
  ok = (std::fclose(fp) == 0) && ok;
  return ok ? LBPWFA_OK : LBPWFA_ERR_IO;
}

int lbpwfa_load(lbpwfa_t h, const char* path) {
  if (!h || !path) return LBPWFA_ERR_INVALID;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return LBPWFA_ERR_IO;
  CkptHeader H{};
  if (std::fread(&H, sizeof(H), 1, fp) != 1 || std::memcmp(H.magic, "LBPWFA02", 8) != 0) {
    std::fclose(fp);
    return LBPWFA_ERR_IO;
  }
  const bool match = H.dim == h->prm.dim && H.n0 == h->n[0] && H.n1 == h->n[1] && H.n2 == h->n[2] &&
                     H.closure == h->prm.closure && H.dv == h->prm.dv && H.precision == h->prm.precision &&
                     H.boundary == h->prm.boundary && H.geometry == h->prm.geometry && H.K == h->K && H.Q == h->Q &&
                     H.pop_bytes == h->f[0].bytes && H.fld_bytes == h->E[0].bytes && H.prev_bytes == h->prev.bytes &&
                     H.dx == h->prm.dx && H.courant == h->prm.courant && H.tau == h->prm.tau && H.mu == h->prm.mu;
  if (!match) { std::fclose(fp); return LBPWFA_ERR_IO; }
  std::vector<char> buf(H.pop_bytes + 2 * H.fld_bytes + H.prev_bytes);
  uint32_t crc_file = 0;
  bool ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size() && std::fread(&crc_file, sizeof(crc_file), 1, fp) == 1;
  std::fclose(fp);
  if (!ok) return LBPWFA_ERR_IO;
  uint32_t crc = crc32_update(0, &H, sizeof(H));
  crc = crc32_update(crc, buf.data(), buf.size());
  if (crc != crc_file) return LBPWFA_ERR_IO;
  const char* q = buf.data();
  CK(h, cudaMemcpyAsync(h->f[h->cur].p, q, H.pop_bytes, cudaMemcpyHostToDevice, h->stream));
  q += H.pop_bytes;
  CK(h, cudaMemcpyAsync(h->E[h->cur].p, q, H.fld_bytes, cudaMemcpyHostToDevice, h->stream));
  q += H.fld_bytes;
  CK(h, cudaMemcpyAsync(h->B[h->cur].p, q, H.fld_bytes, cudaMemcpyHostToDevice, h->stream));
  q += H.fld_bytes;
  if (H.prev_bytes) CK(h, cudaMemcpyAsync(h->prev.p, q, H.prev_bytes, cudaMemcpyHostToDevice, h->stream));
  {
    int r = clear_err_word(h);
    if (r != LBPWFA_OK) return r;
  }
  CK(h, cudaStreamSynchronize(h->stream));
  adj_invalidate(h);
  h->step = H.step;
  h->have_prev = H.have_prev;
  h->fields_from_driver = H.from_driver != 0;
  return LBPWFA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free FP64 reduction.
//
// Callers whose device memory is owned by another allocator (a framework's
// caching allocator, an embedding that reserves the whole device), or whose
// loop cannot afford the implicit device synchronisation that cudaMalloc /
// cudaFree may bring, get the diagnostic sums of lbpwfa_reduce without the
// library touching the allocator: the per-block partial sums live in the
// fixed array below instead of a buffer allocated by the handle.
//
// The array is sized for kNoallocMaxBlocks partials of kNoallocNodesPerBlock
// nodes each, so it serves runs of at most 2^25 nodes (the 256 x 256 x 512
// 3D grid); larger runs are rejected.  Every GPU that loads the library holds
// the array until the process exits.  All calls on a device share it and it
// keeps the last call's contents: each call overwrites every partial it later
// reads, so nothing has to start at zero, but calls whose work overlaps on
// the GPU (two streams, or two handles at once) race on it.
// ---------------------------------------------------------------------------
namespace {
constexpr int kNoallocMaxBlocks = 4096;
constexpr long long kNoallocNodesPerBlock = 8192;
constexpr long long kNoallocMaxNodes = (long long)kNoallocMaxBlocks * kNoallocNodesPerBlock;
constexpr int kNoallocDoubles = kNoallocMaxBlocks * 3 + 4;
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

namespace {
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[256] = {nullptr};

// Device address of the array on the handle's device; resolved by the first
// call on each device (host code may not use the symbol itself as an
// address: in host code it names a host-side stand-in).
int noalloc_scratch(lbpwfa_s* h, double** out) {
  int dev = -1;
  CK(h, cudaGetDevice(&dev));
  if (dev != h->device) {
    h->err = "lbpwfa_reduce_noalloc: device " + std::to_string(dev) + " is current, but the run lives on device " +
             std::to_string(h->device);
    return LBPWFA_ERR_INVALID;
  }
  if (dev < 0 || dev >= 256) {
    h->err = "lbpwfa_reduce_noalloc: device index " + std::to_string(dev) + " is outside 0..255";
    return LBPWFA_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail_cuda(h, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return LBPWFA_OK;
}
}  // namespace

extern "C" int lbpwfa_reduce_noalloc(lbpwfa_t h, double* out, int out_is_device) {
  if (!h || !out) return LBPWFA_ERR_INVALID;
  if (h->ncell > kNoallocMaxNodes) {
    h->err = "lbpwfa_reduce_noalloc: " + std::to_string(h->ncell) + " nodes exceed the static scratch limit of " +
             std::to_string(kNoallocMaxNodes) + " nodes";
    return LBPWFA_ERR_INVALID;
  }
  double* scratch = nullptr;
  int st = noalloc_scratch(h, &scratch);
  if (st != LBPWFA_OK) return st;
  const int nblk = (int)((h->ncell + kNoallocNodesPerBlock - 1) / kNoallocNodesPerBlock);
  double* result = scratch + (size_t)kNoallocMaxBlocks * 3;
  AuxParams A = aux_params(h);
  h->ks.reduce_partial(A, h->f[h->cur].p, scratch, nblk, h->stream);
  CK_LAUNCH(h, "reduce_partial_kernel launch (static scratch)");
  reduce_final_kernel<<<1, 32, 0, h->stream>>>(scratch, nblk, result);
  CK_LAUNCH(h, "reduce_final_kernel launch (static scratch)");
  CK(h, cudaMemcpyAsync(out, result, 3 * sizeof(double),
                        out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  if (out_is_device) return LBPWFA_OK;
  CK(h, cudaStreamSynchronize(h->stream));
  // a bounded device wait that gave up in an earlier step left a
  // half-updated state: report that before the sums (the error word is the
  // handle's own, allocated at create)
  st = check_err_word(h);
  if (st != LBPWFA_OK) return st;
  return out[2] > 0 ? LBPWFA_ERR_NONFINITE : LBPWFA_OK;
}

// ---------------------------------------------------------------------------
// FP64 fused multiply-add rate of the current GPU: the ALU roofline of the
// FP64 storage mode.  Every thread runs kFmaChains independent DFMA chains
// (enough independent work to keep the FP64 pipe busy at full occupancy);
// the result reaches memory only if it equals a value it never takes, so
// the chains are not removed and nothing is written.
// ---------------------------------------------------------------------------
namespace {
constexpr int kFmaChains = 8;
static __device__ double g_fp64_sink;

__global__ void __launch_bounds__(256) fp64_fma_kernel(int iters, double m, double c) {
  double a[kFmaChains];
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) a[j] = 1.0 + 1e-9 * (double)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) a[j] = fma(a[j], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) s += a[j];
  if (s == -1.0) g_fp64_sink = s;
}
}  // namespace

extern "C" int lbpwfa_measure_fp64_rate(double* flops) {
  if (!flops) return LBPWFA_ERR_INVALID;
  *flops = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBPWFA_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LBPWFA_ERR_CUDA;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return LBPWFA_ERR_CUDA;
  int r = LBPWFA_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = LBPWFA_ERR_CUDA;
  const int blocks = sms * 8, threads = 256, iters = 4096;
  double best_ms = 1e30;
  for (int rep = 0; rep < 4 && r == LBPWFA_OK; ++rep) {  // the first launch is a warm-up
    cudaEventRecord(e0, st);
    fp64_fma_kernel<<<blocks, threads, 0, st>>>(iters, 0.9999999, 1e-8);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      r = LBPWFA_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best_ms) best_ms = ms;
  }
  if (r == LBPWFA_OK)
    *flops = 2.0 * kFmaChains * (double)iters * blocks * threads / (best_ms * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return r;
}

// ---------------------------------------------------------------------------
// Batched sweeps.
// ---------------------------------------------------------------------------
// Per closure (index LBPWFA_LEC, LBPWFA_WARMC): its candidate tile, grid and
// (run, tile) work list; a step launches one persistent kernel per closure
// that has runs.
struct lbpwfa_batch_s {
  std::vector<lbpwfa_s*> runs;
  BatchKernelSet bk{};
  int cand[2] = {0, 0};
  int grid[2] = {0, 0};
  int precision = 0;
  std::vector<BatchRun> runs_h;
  BatchRun* runs_d = nullptr;
  int2* items_d[2] = {nullptr, nullptr};
  long long* step_d = nullptr;
  long long nitems[2] = {0, 0};
  long long step = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  // with runs of both closures the WARMC launch forks onto side_stream, so
  // the two persistent kernels fill each other's tails
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_steps = 32;
  double tuned_ms[2][4] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}};
  size_t device_bytes = 0;
  std::string err;
};

namespace {

int batch_fail(lbpwfa_batch_s* b, cudaError_t e, const char* what) {
  b->err = std::string(what) + ": " + cudaGetErrorString(e);
  return LBPWFA_ERR_CUDA;
}
#define BCK(b, call)                                            \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return batch_fail((b), e_, #call);   \
  } while (0)

void batch_free_lists(lbpwfa_batch_s* b) {
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->graph_exec = nullptr;
  b->graph = nullptr;
  if (b->runs_d) cudaFree(b->runs_d);
  b->runs_d = nullptr;
  for (int cl = 0; cl < 2; ++cl) {
    if (b->items_d[cl]) cudaFree(b->items_d[cl]);
    b->items_d[cl] = nullptr;
  }
}

// Launch records and the per-closure (run, tile) work lists for candidate
// tiles c[LBPWFA_LEC] and c[LBPWFA_WARMC].
int batch_build(lbpwfa_batch_s* b, const int* c) {
  batch_free_lists(b);
  b->runs_h.assign(b->runs.size(), BatchRun{});
  std::vector<int2> items[2];
  for (size_t i = 0; i < b->runs.size(); ++i) {
    lbpwfa_s* h = b->runs[i];
    BatchRun& R = b->runs_h[i];
    const int cl = h->prm.closure;
    const int tz = b->bk.tz[c[cl]], tx = b->bk.tx[c[cl]];
    const int cur = h->cur;
    for (int par = 0; par < 2; ++par) {
      h->cur = par;
      R.P[par] = step_params(h);
    }
    h->cur = cur;
    R.z0 = h->prm.z0;
    R.dt = h->dt;
    R.prev_from = h->have_prev ? -1 : b->step;
    R.closure = cl;
    R.axi = h->use_axi ? 1 : 0;
    R.ntz = (h->n[0] + tz - 1) / tz;
    R.ntx = (h->n[1] + tx - 1) / tx;
    for (int t = 0; t < R.ntz * R.ntx; ++t) items[cl].push_back(make_int2((int)i, t));
  }
  BCK(b, cudaMalloc(&b->runs_d, sizeof(BatchRun) * b->runs_h.size()));
  BCK(b, cudaMemcpyAsync(b->runs_d, b->runs_h.data(), sizeof(BatchRun) * b->runs_h.size(),
                         cudaMemcpyHostToDevice, b->stream));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int cl = 0; cl < 2; ++cl) {
    b->nitems[cl] = (long long)items[cl].size();
    b->cand[cl] = c[cl];
    b->grid[cl] = 0;
    if (items[cl].empty()) continue;
    BCK(b, cudaMalloc(&b->items_d[cl], sizeof(int2) * items[cl].size()));
    BCK(b, cudaMemcpyAsync(b->items_d[cl], items[cl].data(), sizeof(int2) * items[cl].size(), cudaMemcpyHostToDevice,
                           b->stream));
    BCK(b, b->bk.prepare[cl][c[cl]]());
    const int occ = b->bk.occupancy[cl][c[cl]]();
    const long long g = (long long)sms * (occ > 0 ? occ : 1);
    b->grid[cl] = (int)(g < b->nitems[cl] ? g : b->nitems[cl]);
  }
  BCK(b, cudaStreamSynchronize(b->stream));
  return LBPWFA_OK;
}

int batch_launch_one(lbpwfa_batch_s* b) {
  const bool fork = b->nitems[0] > 0 && b->nitems[1] > 0 && b->side_stream;
  if (fork) {
    BCK(b, cudaEventRecord(b->fork_ev, b->stream));
    BCK(b, cudaStreamWaitEvent(b->side_stream, b->fork_ev, 0));
  }
  for (int cl = 0; cl < 2; ++cl) {
    if (b->nitems[cl] == 0) continue;
    BatchArgs A{};
    A.runs = b->runs_d;
    A.items = b->items_d[cl];
    A.nitems = (int)b->nitems[cl];
    A.step = b->step_d;
    b->bk.launch[cl][b->cand[cl]](A, b->grid[cl], fork && cl == 1 ? b->side_stream : b->stream);
    BCK(b, cudaGetLastError());
  }
  if (fork) {
    BCK(b, cudaEventRecord(b->join_ev, b->side_stream));
    BCK(b, cudaStreamWaitEvent(b->stream, b->join_ev, 0));
  }
  batch_advance(b->step_d, b->stream);
  BCK(b, cudaGetLastError());
  return LBPWFA_OK;
}

// Restart from the rest state at step 0 (used after tuning).
int batch_reset(lbpwfa_batch_s* b) {
  for (lbpwfa_s* h : b->runs) {
    int r = init_rest_state(h);
    if (r != LBPWFA_OK) { b->err = h->err; return r; }
  }
  BCK(b, cudaMemsetAsync(b->step_d, 0, sizeof(long long), b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  b->step = 0;
  return LBPWFA_OK;
}

std::string batch_key(const lbpwfa_batch_s* b) {
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::string k = std::string(prop.name) + "|p" + std::to_string(b->precision);
  for (const lbpwfa_s* h : b->runs)
    k += "|" + std::to_string(h->prm.closure) + ":" + std::to_string(h->n[0]) + "x" + std::to_string(h->n[1]);
  char buf[32];
  std::snprintf(buf, sizeof(buf), "%016zx", std::hash<std::string>{}(k));
  return buf;
}

// Tuning cache: one line per entry, `"<key>": <candidate>`, inside a JSON object.
int cache_lookup(const std::string& key) {
  const char* path = std::getenv("LBPWFA_TUNE_CACHE");
  if (!path) return -1;
  FILE* fp = std::fopen(path, "r");
  if (!fp) return -1;
  char line[256];
  int found = -1;
  while (std::fgets(line, sizeof(line), fp)) {
    char k[64];
    int c;
    if (std::sscanf(line, " \"%63[0-9a-f]\": %d", k, &c) == 2 && key == k) found = c;
  }
  std::fclose(fp);
  return found;
}

void cache_store(const std::string& key, int c) {
  const char* path = std::getenv("LBPWFA_TUNE_CACHE");
  if (!path) return;
  std::vector<std::string> entries;
  if (FILE* fp = std::fopen(path, "r")) {
    char line[256];
    while (std::fgets(line, sizeof(line), fp)) {
      char k[64];
      int v;
      if (std::sscanf(line, " \"%63[0-9a-f]\": %d", k, &v) == 2 && key != k)
        entries.push_back(std::string("\"") + k + "\": " + std::to_string(v));
    }
    std::fclose(fp);
  }
  entries.push_back("\"" + key + "\": " + std::to_string(c));
  if (FILE* fp = std::fopen(path, "w")) {
    std::fprintf(fp, "{\n");
    for (size_t i = 0; i < entries.size(); ++i)
      std::fprintf(fp, "  %s%s\n", entries[i].c_str(), i + 1 < entries.size() ? "," : "");
    std::fprintf(fp, "}\n");
    std::fclose(fp);
  }
}

// Time each candidate tile over a few steps of the real batch, one closure
// at a time (the other closure's kernel is the same in every timing), keep
// the fastest, and return to the rest state.  The cache stores the pair as
// 4 * c[LEC] + c[WARMC].
int batch_autotune(lbpwfa_batch_s* b) {
  const std::string key = batch_key(b);
  const int cached = cache_lookup(key);
  if (cached >= 0 && cached / 4 < b->bk.ncand && cached % 4 < b->bk.ncand) {
    const int c[2] = {cached / 4, cached % 4};
    return batch_build(b, c);
  }
  bool present[2] = {false, false};
  for (const lbpwfa_s* h : b->runs) present[h->prm.closure] = true;
  cudaEvent_t e0, e1;
  BCK(b, cudaEventCreate(&e0));
  BCK(b, cudaEventCreate(&e1));
  int best[2] = {0, 0};
  for (int cl = 0; cl < 2; ++cl) {
    if (!present[cl]) continue;
    double best_ms = 1e30;
    for (int cc = 0; cc < b->bk.ncand; ++cc) {
      int c[2] = {best[0], best[1]};
      c[cl] = cc;
      int r = batch_build(b, c);
      for (int w = 0; w < 2 && r == LBPWFA_OK; ++w) r = batch_launch_one(b);
      if (r == LBPWFA_OK) cudaEventRecord(e0, b->stream);
      for (int w = 0; w < 4 && r == LBPWFA_OK; ++w) r = batch_launch_one(b);
      if (r == LBPWFA_OK) cudaEventRecord(e1, b->stream);
      if (r != LBPWFA_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return r; }
      BCK(b, cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      b->tuned_ms[cl][cc] = ms / 4.0;
      if (b->tuned_ms[cl][cc] < best_ms) { best_ms = b->tuned_ms[cl][cc]; best[cl] = cc; }
      r = batch_reset(b);
      if (r != LBPWFA_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return r; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cache_store(key, 4 * best[0] + best[1]);
  return batch_build(b, best);
}

}  // namespace

extern "C" {

void lbpwfa_batch_destroy(lbpwfa_batch_t b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->side_stream) cudaStreamSynchronize(b->side_stream);
  batch_free_lists(b);
  if (b->side_stream) cudaStreamDestroy(b->side_stream);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->join_ev) cudaEventDestroy(b->join_ev);
  if (b->step_d) cudaFree(b->step_d);
  for (lbpwfa_s* h : b->runs) destroy_run(h);
  if (b->owns_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int lbpwfa_batch_create(const lbpwfa_params* p, int nruns, int flags, lbpwfa_batch_t* out) {
  if (!out || !p || nruns < 1) return LBPWFA_ERR_INVALID;
  *out = nullptr;
  for (int i = 0; i < nruns; ++i) {
    int st = validate(&p[i]);
    if (st != LBPWFA_OK) return st;
    if (p[i].dim != 2 || p[i].precision != p[0].precision) return LBPWFA_ERR_INVALID;
    if (p[i].precision == LBPWFA_FP32C) return LBPWFA_ERR_INVALID;  // single runs only
    if (p[i].record_tape > 0) return LBPWFA_ERR_INVALID;           // no adjoint in batches
  }
  lbpwfa_batch_s* b = new lbpwfa_batch_s();
  b->precision = p[0].precision;
  const int bpr = b->precision == LBPWFA_FP64 ? PR_F64 : (b->precision == LBPWFA_FP32 ? PR_F32 : PR_F16S);
  if (!batch_kernels(bpr, &b->bk)) {
    delete b;
    return LBPWFA_ERR_INVALID;
  }
  if (p[0].stream) {
    b->stream = (cudaStream_t)p[0].stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return LBPWFA_ERR_CUDA; }
    b->owns_stream = true;
  }
  for (int i = 0; i < nruns; ++i) {
    lbpwfa_params q = p[i];
    q.stream = b->stream;
    q.kernel_variant = 1;
    lbpwfa_t h = nullptr;
    int st = lbpwfa_create(&q, &h);
    if (st != LBPWFA_OK) { lbpwfa_batch_destroy(b); return st; }
    h->in_batch = true;
    b->runs.push_back(h);
    b->device_bytes += h->device_bytes;
  }
  if (cudaMalloc(&b->step_d, sizeof(long long)) != cudaSuccess) { lbpwfa_batch_destroy(b); return LBPWFA_ERR_OOM; }
  if (cudaStreamCreateWithFlags(&b->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming) != cudaSuccess) {
    lbpwfa_batch_destroy(b);
    return LBPWFA_ERR_CUDA;
  }
  if (cudaMemsetAsync(b->step_d, 0, sizeof(long long), b->stream) != cudaSuccess) {
    lbpwfa_batch_destroy(b);
    return LBPWFA_ERR_CUDA;
  }
  const int first[2] = {0, 0};
  int st = (flags & 1) ? batch_build(b, first) : batch_autotune(b);
  if (st != LBPWFA_OK) { lbpwfa_batch_destroy(b); return st; }
  *out = b;
  return LBPWFA_OK;
}

int lbpwfa_create_batch(const lbpwfa_params* p, int nruns, lbpwfa_batch_t* out) {
  return lbpwfa_batch_create(p, nruns, 0, out);
}

int lbpwfa_batch_step(lbpwfa_batch_t b, int64_t nsteps) {
  if (!b || nsteps < 0) return LBPWFA_ERR_INVALID;
  if (nsteps == 0) return LBPWFA_OK;
  // a member whose state was replaced restarts its WARMC backward differences
  bool dirty = false;
  for (size_t i = 0; i < b->runs.size(); ++i) {
    lbpwfa_s* h = b->runs[i];
    if (h->prm.closure == LBPWFA_WARMC && !h->have_prev && b->runs_h[i].prev_from != b->step) {
      b->runs_h[i].prev_from = b->step;
      dirty = true;
    }
  }
  if (dirty)
    BCK(b, cudaMemcpyAsync(b->runs_d, b->runs_h.data(), sizeof(BatchRun) * b->runs_h.size(),
                           cudaMemcpyHostToDevice, b->stream));
  int64_t left = nsteps;
  if (left >= b->graph_steps && !b->graph_exec) {
    BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int r = LBPWFA_OK;
    for (int s = 0; s < b->graph_steps && r == LBPWFA_OK; ++s) r = batch_launch_one(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (r != LBPWFA_OK) return r;
    if (e != cudaSuccess) return batch_fail(b, e, "cudaStreamEndCapture");
    b->graph = g;
    BCK(b, cudaGraphInstantiate(&b->graph_exec, b->graph, 0));
  }
  while (b->graph_exec && left >= b->graph_steps) {
    BCK(b, cudaGraphLaunch(b->graph_exec, b->stream));
    left -= b->graph_steps;
  }
  for (; left > 0; --left) {
    int r = batch_launch_one(b);
    if (r != LBPWFA_OK) return r;
  }
  b->step += nsteps;
  for (lbpwfa_s* h : b->runs) {
    h->step = b->step;
    h->cur = (int)(b->step & 1);
    if (h->NPREV) h->have_prev = 1;
  }
  return LBPWFA_OK;
}

int lbpwfa_batch_member(lbpwfa_batch_t b, int i, lbpwfa_t* run) {
  if (!b || !run || i < 0 || i >= (int)b->runs.size()) return LBPWFA_ERR_INVALID;
  *run = b->runs[i];
  return LBPWFA_OK;
}

int lbpwfa_batch_info(lbpwfa_batch_t b, lbpwfa_batch_info_t* info) {
  if (!b || !info) return LBPWFA_ERR_INVALID;
  info->nruns = (int)b->runs.size();
  info->ncell = 0;
  info->bytes_per_step = 0.0;
  info->algorithmic_bytes_per_step = 0.0;
  for (lbpwfa_s* h : b->runs) {
    lbpwfa_info_t ri{};
    lbpwfa_info(h, &ri);
    info->ncell += ri.ncell;
    info->bytes_per_step += ri.bytes_per_update * (double)ri.ncell;
    info->algorithmic_bytes_per_step += ri.algorithmic_bytes_per_update * (double)ri.ncell;
  }
  info->nitems = b->nitems[0] + b->nitems[1];
  for (int cl = 0; cl < 2; ++cl) {
    info->tile[cl][0] = b->nitems[cl] ? b->bk.tz[b->cand[cl]] : 0;
    info->tile[cl][1] = b->nitems[cl] ? b->bk.tx[b->cand[cl]] : 0;
    info->grid[cl] = b->grid[cl];
    for (int c = 0; c < 4; ++c) info->tuned_ms[cl][c] = b->tuned_ms[cl][c];
  }
  info->graph_steps = b->graph_steps;
  info->step = b->step;
  info->device_bytes = b->device_bytes;
  return LBPWFA_OK;
}

int lbpwfa_autotune(lbpwfa_t h, double* ms_out) {
  if (!h) return LBPWFA_ERR_INVALID;
  if (ms_out)
    for (int v = 0; v < 5; ++v) ms_out[v] = -1.0;
  if (h->in_batch) {
    h->err = "lbpwfa_autotune: this run belongs to a batch (lbpwfa_batch_create tunes its tiles)";
    return LBPWFA_ERR_STATE;
  }
  // the candidates: the variants this run can take (axisymmetric runs report
  // their plain kernel as 5)
  auto takes = [&](int v) {
    select_kernel(h, v);
    const int u = variant_in_use(h);
    return u == v || (v == 1 && u == 5);
  };
  std::string key;
  {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, h->device);
    std::string k = std::string(prop.name) + "|run|" + std::to_string(h->prm.dim) + "|" +
                    std::to_string(h->prm.closure) + "|" + std::to_string(h->prm.precision) + "|" +
                    std::to_string(h->prm.boundary) + "|" + std::to_string(h->prm.geometry) + "|" +
                    std::to_string(h->n[0]) + "x" + std::to_string(h->n[1]) + "x" + std::to_string(h->n[2]);
    char buf[32];
    std::snprintf(buf, sizeof(buf), "%016zx", std::hash<std::string>{}(k));
    key = buf;
  }
  const int cached = cache_lookup(key);
  if (cached >= 1 && cached <= 4 && takes(cached)) return LBPWFA_OK;
  // keep the state while the candidates step it
  const size_t pb = h->f[0].bytes, fb = h->E[0].bytes, qb = h->prev.bytes;
  Buf snap;
  int st = alloc(h, snap, pb + 2 * fb + qb);
  if (st != LBPWFA_OK) {
    h->err = "lbpwfa_autotune: no room to keep the state while tuning (" + std::to_string(pb + 2 * fb + qb) + " bytes)";
    return st;
  }
  char* sp = (char*)snap.p;
  const int cur = h->cur, have_prev = h->have_prev;
  const long long step = h->step;
  auto keep = [&](bool back) -> int {
    char* dst[4] = {sp, sp + pb, sp + pb + fb, sp + pb + 2 * fb};
    char* src[4] = {(char*)h->f[cur].p, (char*)h->E[cur].p, (char*)h->B[cur].p, (char*)h->prev.p};
    const size_t n[4] = {pb, fb, fb, qb};
    for (int j = 0; j < 4; ++j)
      if (n[j]) CK(h, cudaMemcpyAsync(back ? src[j] : dst[j], back ? dst[j] : src[j], n[j], cudaMemcpyDeviceToDevice,
                                      h->stream));
    return LBPWFA_OK;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) st = fail_cuda(h, ce, "lbpwfa_autotune: events");
  const bool kept = st == LBPWFA_OK && (st = keep(false)) == LBPWFA_OK;
  int best = 0;
  double best_ms = 1e30;
  for (int v = 1; v <= 4 && st == LBPWFA_OK; ++v) {
    if (!takes(v)) continue;
    // two steps to warm up, five timed, then back to the kept state
    for (int w = 0; w < 2 && st == LBPWFA_OK; ++w) st = launch_step(h, nullptr);
    if (st == LBPWFA_OK && (ce = cudaEventRecord(e0, h->stream)) != cudaSuccess) st = fail_cuda(h, ce, "event");
    for (int w = 0; w < 5 && st == LBPWFA_OK; ++w) st = launch_step(h, nullptr);
    if (st == LBPWFA_OK && (ce = cudaEventRecord(e1, h->stream)) != cudaSuccess) st = fail_cuda(h, ce, "event");
    if (st == LBPWFA_OK && (ce = cudaEventSynchronize(e1)) != cudaSuccess) st = fail_cuda(h, ce, "event");
    if (st == LBPWFA_OK) st = check_err_word(h);
    float ms = 0.f;
    if (st == LBPWFA_OK) cudaEventElapsedTime(&ms, e0, e1);
    // back to the kept state, after a failed step as well
    h->cur = cur;
    h->step = step;
    h->have_prev = have_prev;
    const int back = kept ? keep(true) : LBPWFA_OK;
    if (st == LBPWFA_OK) st = back;
    if (st != LBPWFA_OK) break;
    const double per = ms / 5.0;
    if (ms_out) ms_out[v] = per;
    if (per < best_ms) { best_ms = per; best = v; }
  }
  ce = cudaStreamSynchronize(h->stream);  // the copies back read the kept state
  if (st == LBPWFA_OK && ce != cudaSuccess) st = fail_cuda(h, ce, "lbpwfa_autotune");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->device_bytes -= snap.bytes;
  release(snap);
  if (st != LBPWFA_OK) {
    select_kernel(h, h->prm.kernel_variant);
    return st;
  }
  takes(best);
  cache_store(key, best);
  return LBPWFA_OK;
}

}  // extern "C"
