// On-GPU wake diagnostic: least-squares sinusoid fit along one line of the
// grid (the dispersion measurement of Sec. 6, Fig. 3: the wake's wavenumber
// k_w behind the driver).
//
// For a trial k the line's values q_j at xi_j = j dx - z_d inside the window
// are fitted by a cos(k xi) + b sin(k xi) (normal equations of the five sums
// below); R(k) = sum q^2 - (a sum q cos + b sum q sin) is the residual.  The
// scan evaluates R on a uniform k grid, one block per k; the pick takes the
// grid minimum, refines it by the parabola through it and its neighbours,
// and refits at the refined k.  All sums are FP64 with a fixed reduction
// order, so repeated calls return identical bits.
#pragma once

#include <cuda_runtime.h>

#include "lb_aux.cuh"

namespace lbp {

struct FitLine {
  const double* q;   // FP64 values of the grid, cell c = iz + nz (ix + nx iy)
  long long base;    // cell of iz = 0 on the line
  int nz;
  double zd, dx;     // xi_j = j dx - zd
  double offset;     // fitted value q - offset (1 for the density)
  double xi_lo, xi_hi;
  double k_lo, dk;
  int nk;
};

constexpr int kFitThreads = 256;

__device__ __forceinline__ bool fit_in_window(const FitLine& L, int j, double& xi) {
  xi = (double)j * L.dx - L.zd;
  return xi >= L.xi_lo && xi <= L.xi_hi;
}

// Block-wide fixed-order sum of v[0..N) per thread into s[0..N) on thread 0.
template <int N>
__device__ __forceinline__ void fit_block_sum(double* v, double (*sh)[kFitThreads]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int i = 0; i < N; ++i) sh[i][t] = v[i];
  __syncthreads();
  for (int w = kFitThreads / 2; w > 0; w >>= 1) {
    if (t < w) {
#pragma unroll
      for (int i = 0; i < N; ++i) sh[i][t] += sh[i][t + w];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = sh[i][0];
}

// sums: cc, cs, ss, qc, qs, qq, count
__device__ __forceinline__ void fit_sums(const FitLine& L, double k, double* s) {
  for (int i = 0; i < 7; ++i) s[i] = 0.0;
  for (int j = threadIdx.x; j < L.nz; j += kFitThreads) {
    double xi;
    if (!fit_in_window(L, j, xi)) continue;
    double sn, cs;
    sincos(k * xi, &sn, &cs);
    const double q = L.q[L.base + j] - L.offset;
    s[0] += cs * cs;
    s[1] += cs * sn;
    s[2] += sn * sn;
    s[3] += q * cs;
    s[4] += q * sn;
    s[5] += q * q;
    s[6] += 1.0;
  }
}

// (a, b, R) of the normal equations
__device__ __forceinline__ void fit_solve(const double* s, double& a, double& b, double& R) {
  const double det = s[0] * s[2] - s[1] * s[1];
  if (!(det > 0.0)) { a = b = 0.0; R = s[5]; return; }
  a = (s[3] * s[2] - s[4] * s[1]) / det;
  b = (s[4] * s[0] - s[3] * s[1]) / det;
  R = s[5] - (a * s[3] + b * s[4]);
}

// One block per trial k: res[m] = R(k_m).
__global__ void __launch_bounds__(kFitThreads) fit_scan_kernel(FitLine L, double* res) {
  __shared__ double sh[7][kFitThreads];
  const int m = blockIdx.x;
  double s[7];
  fit_sums(L, L.k_lo + (double)m * L.dk, s);
  fit_block_sum<7>(s, sh);
  if (threadIdx.x == 0) {
    double a, b, R;
    fit_solve(s, a, b, R);
    res[m] = R;
  }
}

// Grid minimum, parabolic refinement, refit: out = (k, amplitude sqrt(a^2 +
// b^2), phase phi with q ~ A cos(k xi + phi), rms residual, points).
__global__ void __launch_bounds__(kFitThreads) fit_pick_kernel(FitLine L, const double* res, double* out) {
  __shared__ double sh[7][kFitThreads];
  __shared__ double kstar;
  if (threadIdx.x == 0) {
    int mb = 0;
    for (int m = 1; m < L.nk; ++m)
      if (res[m] < res[mb]) mb = m;
    double d = 0.0;
    if (mb > 0 && mb < L.nk - 1) {
      const double rm = res[mb - 1], r0 = res[mb], rp = res[mb + 1];
      const double den = rm - 2.0 * r0 + rp;
      if (den > 0.0) d = 0.5 * (rm - rp) / den;
      d = d < -0.5 ? -0.5 : (d > 0.5 ? 0.5 : d);
    }
    kstar = L.k_lo + ((double)mb + d) * L.dk;
  }
  __syncthreads();
  const double k = kstar;
  double s[7];
  fit_sums(L, k, s);
  fit_block_sum<7>(s, sh);
  if (threadIdx.x == 0) {
    double a, b, R;
    fit_solve(s, a, b, R);
    out[0] = k;
    out[1] = sqrt(a * a + b * b);
    out[2] = -atan2(b, a);
    out[3] = s[6] > 0.0 ? sqrt((R > 0.0 ? R : 0.0) / s[6]) : 0.0;
    out[4] = s[6];
  }
}

// ---------------------------------------------------------------------------
// Gauss's law residual (the field check of Sec. 6: it is not imposed and
// holds up to the LB's numerical diffusion).  On the dual cells, centred at
// (z_{i+1/2}, x_{j+1/2}, y_{k+1/2}), the Yee slots give
//   div E = (E_z(i+1) - E_z(i)) / dx + (E_x(j+1) - E_x(j)) / dx + (E_y(k+1) - E_y(k)) / dx
// (axisymmetric: (r_{j+1} E_r(j+1) - r_j E_r(j)) / (r_{j+1/2} dx) for the
// radial term), and rho = -(nbar - 1) - n_b, nbar the mean density of the
// cell's corner nodes and n_b the driver at the centre at the time of the
// stored E (t_{n-1/2}).  Sums of (div E - rho)^2 and rho^2 over a range of
// cells, FP64, fixed block partition and tree.
// ---------------------------------------------------------------------------
struct GaussArgs {
  AuxParams A;         // grid and driver; A.t = time of the stored E
  const double* n;     // density at the nodes [ncell]
  const double* E;     // E_z, E_x, E_y slots [3][ncell]
  int dim;
  int lo[3], hi[3];    // cell-centre index ranges
  long long ncells;    // product of the range lengths
};

__global__ void __launch_bounds__(256) gauss_partial_kernel(GaussArgs G, double* partial) {
  __shared__ double sh[2][256];
  const AuxParams& A = G.A;
  const int w0 = G.hi[0] - G.lo[0], w1 = G.hi[1] - G.lo[1];
  const long long per_block = (G.ncells + gridDim.x - 1) / gridDim.x;
  const long long q0 = blockIdx.x * per_block;
  const long long q1 = min(G.ncells, q0 + per_block);
  const long long sx = A.n[0], sy = (long long)A.n[0] * A.n[1];
  double s_res = 0.0, s_rho = 0.0;
  for (long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const int i = G.lo[0] + (int)(q % w0);
    const long long r = q / w0;
    const int j = G.lo[1] + (int)(r % w1);
    const int k = G.lo[2] + (int)(r / w1);
    const long long c = i + sx * j + sy * k;
    const double idx = 1.0 / A.dx;
    double div = (G.E[c + 1] - G.E[c]) * idx;
    if (G.dim >= 2) {
      const double* Ex = G.E + A.ncell;
      if (A.axi) {
        const double rl = j * A.dx, rh = rl + A.dx, rm = rl + 0.5 * A.dx;
        div += (rh * Ex[c + sx] - rl * Ex[c]) / (rm * A.dx);
      } else {
        div += (Ex[c + sx] - Ex[c]) * idx;
      }
    }
    if (G.dim >= 3) {
      const double* Ey = G.E + 2 * A.ncell;
      div += (Ey[c + sy] - Ey[c]) * idx;
    }
    double nbar = 0.0;
    const int cz = 2, cxn = G.dim >= 2 ? 2 : 1, cyn = G.dim >= 3 ? 2 : 1;
    for (int b = 0; b < cyn; ++b)
      for (int a = 0; a < cxn; ++a)
        for (int d = 0; d < cz; ++d) nbar += G.n[c + d + sx * a + sy * b];
    nbar /= (double)(cz * cxn * cyn);
    const double zc = (i + 0.5) * A.dx;
    double nb = driver_long_d(A, zc - A.z0 - A.t);
    if (G.dim >= 2) {
      const double xc = (j + 0.5 - A.xoff) * A.dx;
      const double yc = G.dim >= 3 ? (k + 0.5 - A.yoff) * A.dx : 0.0;
      nb *= exp(-(xc * xc + yc * yc) * A.inv2sr2);
    }
    const double rho = -(nbar - 1.0) - nb;
    s_res += (div - rho) * (div - rho);
    s_rho += rho * rho;
  }
  sh[0][threadIdx.x] = s_res;
  sh[1][threadIdx.x] = s_rho;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sh[0][0];
    partial[2 * blockIdx.x + 1] = sh[1][0];
  }
}

__global__ void gauss_final_kernel(const double* partial, int nblk, long long ncells, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int q = 0; q < nblk; ++q) { a += partial[2 * q]; b += partial[2 * q + 1]; }
  out[0] = a;
  out[1] = b;
  out[2] = (double)ncells;
}

}  // namespace lbp
