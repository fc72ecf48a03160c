// Launch parameters of the adjoint kernels (lb_adjoint.cuh), shared with
// the host runtime.
#pragma once

#include "lb_common.cuh"

namespace lbp {

struct AdjParams {
  StepParams P;             // geometry and constants of the forward step
  const void* tape;         // this step's entry [NTAPE][plane] (real)
  const void* tape_prev;    // previous step's entry, or null (then prev0)
  const void* prev0;        // previous-step values [NPREV][plane] when tape_prev is null
  const void* lf_in;        // adjoint of f^{n+1} [K][Q][plane]
  void* lf_out;             // adjoint of f^n
  const void* lE_in;        // adjoint of E^{n+1/2} (next state) [3][plane]
  void* lE_out;             // adjoint of E^{n-1/2}
  const void* lB_in;        // adjoint of B^{n+1} [3][plane]
  void* lB_out;             // adjoint of B^n
  const void* lp_in;        // adjoint of the WARMC previous-step values written by this step
  void* lp_out;             // adjoint of those read by this step
  void* rA;                 // [K][plane]  decode adjoint of the node's local terms + collision
  void* rG;                 // [NG][plane] gradient-stencil coefficients
  void* rEn;                // [3][plane]  adjoint of the node-averaged E^{n+1/2}
  void* rBn;                // [3][plane]  adjoint of the node-averaged B^n
  // per node and set, from the gather of the next state's population
  // adjoints (adj_coll_kernel): the collision's adjoint of A_k, of dt F_k,
  // and A_k times its part of the adjoint of u
  void* cA;                 // [K][plane]
  void* cF;                 // [K][plane]
  void* cU;                 // [K][DIM][plane]
  void* lAf;                // [K][plane]  the node's adjoint of A_k after the field terms (adj_field_kernel)
  void* cW;                 // WARMC [2][DIM][plane]: the node's w = lambda u, and the previous step's (adj_coll_kernel)
  int band_rows;            // 2D, 7 or more nodes per axis: rows of adj_coll_kernel blocks (after the tiles' rows)
                            // that take the nodes within 3 of an edge, one per thread; 0: the tiles take every node
  double* rows;             // [2][gridDim.y][n0] partial row sums of this step
  const double* Tx;         // [2][n1]: T(x) and T(x) x^2 / sigma_r^3 at the E_z slots
};

// Row sets of the driver-parameter gradient (see grad_sets_kernel).
struct GradParams {
  int n0;
  int nsets, ntx;
  const double* rows;       // [nsets][2][ntx][n0]
  const double2* setp;      // [nsets] (zeta0, zoff)
  double dx, alpha, sigma_z, inv2sz2;
  const double* profile; int plen; double pdz;
  double* gpart;            // [nsets][3]
  double* g3;               // [3] accumulated
  double* gp;               // [plen] accumulated
};

}  // namespace lbp
