// Internal host-side declarations shared by the runtime translation units:
// the run handle, device buffers and the helpers that queue a step.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/lbpwfa.h"
#include "lb_dispatch.h"

namespace lbp {
struct StepParams;
}

namespace lbprt {

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct AdjRec;  // adjoint recording of a run (adjoint_rt.cu)

}  // namespace lbprt

struct lbpwfa_s {
  lbpwfa_params prm{};
  std::vector<double> profile_h;
  double* profile_d = nullptr;
  lbp::KernelSet ks{};
  int K = 0, Q = 0, NPREV = 0;
  int NPL = 0;  // planes of a population buffer (K*Q, plus K low parts in FP16S)
  int n[3] = {1, 1, 1};
  int nzp = 0;
  long long plane = 0, ncell = 0;
  size_t store_sz = 0, real_sz = 0;
  double dt = 0.0;
  long long step = 0;
  int cur = 0;  // index of the buffers holding the current state
  lbprt::Buf f[2], E[2], B[2], prev, partial, out3, scratch;
  int have_prev = 0;
  bool fields_from_driver = false;  // E, B still the driver's initial fields (step 0)
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  double Arest[11] = {0};
  float scale[11], inv_scale[11];
  size_t device_bytes = 0;
  std::string err;
  bool use_tma = false;
  bool use_persist = false;
  bool use_march = false;  // 3D marching columns
  bool use_axi = false;    // 2D axisymmetric (z, r) kernel
  bool in_batch = false;  // owned by a batch: stepped only through lbpwfa_batch_step
  int num_sms = 0;
  int device = -1;  // the CUDA device current at lbpwfa_create (holds every buffer)
  unsigned wait_limit = LBPWFA_WAIT_POLLS;  // polls of a tile's first barrier wait
  alignas(64) CUtensorMap maps[2];
  int* err_d = nullptr;  // device error word written by bounded waits
  lbprt::AdjRec* adj = nullptr;
};

namespace lbprt {

// FP32 fields are kept as high + low parts: each E or B buffer holds the
// three high components followed by the three low ones (FP64: high only).
inline bool split_fields(const lbpwfa_s* h) { return h->real_sz == 4; }
inline void* lo_of(const lbpwfa_s* h, const Buf& b) {
  return split_fields(h) ? (char*)b.p + 3 * (size_t)h->plane * h->real_sz : nullptr;
}

int fail_cuda(lbpwfa_s* h, cudaError_t e, const char* what);
int alloc(lbpwfa_s* h, Buf& b, size_t bytes);
void release(Buf& b);
lbp::StepParams step_params(const lbpwfa_s* h);
double zeta0_of(double z0, long long step, double dt);
int launch_step(lbpwfa_s* h, void* tape);
int check_err_word(lbpwfa_s* h);
int clear_err_word(lbpwfa_s* h);

// adjoint recording hooks (adjoint_rt.cu)
int adj_before_step(lbpwfa_s* h, void** tape);  // checkpoint / tape slot of the next step
void adj_invalidate(lbpwfa_s* h);                // the state was replaced: recording ends
void adj_free(lbpwfa_s* h);

}  // namespace lbprt

#define CK(h, call)                                                   \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return lbprt::fail_cuda((h), e_, #call);   \
  } while (0)

#define CK_LAUNCH(h, what)                                            \
  do {                                                                \
    cudaError_t e_ = cudaGetLastError();                              \
    if (e_ != cudaSuccess) return lbprt::fail_cuda((h), e_, what);    \
  } while (0)
