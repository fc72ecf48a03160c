// Auxiliary kernels around the step: initial driver fields, state import
// (un-streaming) and export (pull), FP64 moments / advected scalars, field
// export and the deterministic FP64 reduction.
#pragma once

#include "lb_step.cuh"

namespace lbp {

struct AuxParams {
  int n[3];
  int nzp;
  long long plane;
  long long ncell;   // unpadded node count
  int periodic;
  double dx, dt, mu;
  int D;
  double Arest[11];
  float inv_scale[11], scale[11];
  double alpha, inv2sz2, sigma_r, inv2sr2, z0;
  const double* profile; int plen; double pdz;
  double xoff, yoff;
  double t;          // time of the stored populations
  int axi;           // 2D axisymmetric (z, r): x is r = j dx, xoff = 0
};

__device__ __forceinline__ void unflatten(const AuxParams& A, long long c, int* e) {
  e[0] = (int)(c % A.n[0]);
  long long r = c / A.n[0];
  e[1] = (int)(r % A.n[1]);
  e[2] = (int)(r / A.n[1]);
}
__device__ __forceinline__ long long padded(const AuxParams& A, const int* e) {
  return (long long)e[0] + (long long)A.nzp * ((long long)e[1] + (long long)A.n[1] * e[2]);
}

__device__ __forceinline__ double driver_long_d(const AuxParams& A, double zeta) {
  if (A.profile) {
    const double s = zeta / A.pdz + 0.5 * (A.plen - 1);
    if (!(s > -1.0 && s < (double)A.plen)) return 0.0;
    const int j = (int)floor(s);
    const double fr = s - j;
    const double a = j >= 0 ? A.profile[j] : 0.0, b = j + 1 < A.plen ? A.profile[j + 1] : 0.0;
    return (1.0 - fr) * a + fr * b;
  }
  return A.alpha * exp(-zeta * zeta * A.inv2sz2);
}

// radial factor (1 - exp(-s)) / (2 s), s = r^2 / 2 sigma_r^2; 1/2 at r = 0
__device__ __forceinline__ double radial_factor(double r2, double sr) {
  double s = r2 / (2.0 * sr * sr);
  return s > 0.0 ? -expm1(-s) / (2.0 * s) : 0.5;
}

// A field value into its slot: FP64 as is; FP32 as a high part and the
// rounding remainder in the low array (value = high + low).
template <typename real>
__device__ __forceinline__ void put_field(real* hi, real* lo, long long i, double v) {
  const real h = real(v);
  hi[i] = h;
  if (lo) lo[i] = real(v - (double)h);
}
template <typename real>
__device__ __forceinline__ double get_field(const real* hi, const real* lo, long long i) {
  return (double)hi[i] + (lo ? (double)lo[i] : 0.0);
}

// Initial fields: rigid bunch field in the v -> c limit (Sec. 6): E_z = 0,
// div_perp E_perp = -n_b, B = z x E; E at t = -dt/2, B at t = 0.
// Conducting-wall slots of E are zero.
template <int DIM, typename real>
__global__ void init_fields_kernel(AuxParams A, real* E, real* B, real* Elo, real* Blo) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= A.ncell) return;
  int e[3];
  unflatten(A, c, e);
  const long long p = padded(A, e);
  const double dx = A.dx, sr = A.sigma_r;
  const double z = e[0] * dx, x = (e[1] - A.xoff) * dx, y = (e[2] - A.yoff) * dx;
  const double tE = -0.5 * A.dt;
  double Ev[3] = {0, 0, 0}, Bv[3] = {0, 0, 0};
  if (DIM == 2 && A.axi) {
    // E_r = -L sr^2 (1 - exp(-r^2/2sr^2)) / r at the E_r slot (z + dx/2, r),
    // B_phi = E_r at the node; both 0 on the axis
    const double k = x * radial_factor(x * x, sr);
    Ev[1] = -driver_long_d(A, z + 0.5 * dx - A.z0 - tE) * k;
    Bv[2] = -driver_long_d(A, z - A.z0) * k;
  } else if (DIM == 2) {
    const double k = sr * sqrt(M_PI / 2.0) * erf(x / (sqrt(2.0) * sr));
    Ev[1] = -driver_long_d(A, z + 0.5 * dx - A.z0 - tE) * k;   // E_x slot: z + dx/2
    Bv[2] = -driver_long_d(A, z - A.z0) * k;                   // B_y at the node
  } else if (DIM == 3) {
    {  // E_x slot (x, y + dx/2, z + dx/2)
      double yy = y + 0.5 * dx;
      Ev[1] = -driver_long_d(A, z + 0.5 * dx - A.z0 - tE) * x * radial_factor(x * x + yy * yy, sr);
    }
    {  // E_y slot (x + dx/2, y, z + dx/2)
      double xx = x + 0.5 * dx;
      Ev[2] = -driver_long_d(A, z + 0.5 * dx - A.z0 - tE) * y * radial_factor(xx * xx + y * y, sr);
    }
    {  // B_x slot (x + dx/2, y, z): B_x = -E_y
      double xx = x + 0.5 * dx;
      Bv[1] = driver_long_d(A, z - A.z0) * y * radial_factor(xx * xx + y * y, sr);
    }
    {  // B_y slot (x, y + dx/2, z): B_y = E_x
      double yy = y + 0.5 * dx;
      Bv[2] = -driver_long_d(A, z - A.z0) * x * radial_factor(x * x + yy * yy, sr);
    }
  }
  if (!A.periodic) {
    for (int a = 0; a < 3; ++a) {
      const int b = (a + 1) % 3, d = (a + 2) % 3;
      bool wall = (b >= 1 && b < DIM && e[b] == A.n[b] - 1) || (d >= 1 && d < DIM && e[d] == A.n[d] - 1);
      if (wall) Ev[a] = 0.0;
    }
  }
  for (int a = 0; a < 3; ++a) {
    put_field(E, Elo, a * A.plane + p, Ev[a]);
    put_field(B, Blo, a * A.plane + p, Bv[a]);
  }
}

// Import populations f^n (FP64 [K][Q][ncell]) into post-collision storage
// f*^{n-1} such that the pull of the next step returns f^n: the stored value
// at y for velocity i is f^n_i(y + xi_i).  Entries never read by a pull (the
// source would not be a bulk node with open boundaries) take f^n_i(y).
template <int DIM, int CL, int PR>
__global__ void import_pops_kernel(AuxParams A, const double* fin, typename Prec<PR>::store* out) {
  using L = Lattice<DIM>;
  using M = Model<DIM, CL>;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= A.ncell) return;
  int e[3];
  unflatten(A, c, e);
  const long long p = padded(A, e);
  for (int k = 0; k < M::K; ++k) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      int s[3] = {e[0], e[1], e[2]};
      bool bulk = true;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        s[a] += L::c(i, a);
        if (A.periodic) s[a] = s[a] < 0 ? s[a] + A.n[a] : (s[a] >= A.n[a] ? s[a] - A.n[a] : s[a]);
        else bulk = bulk && s[a] >= 1 && s[a] <= A.n[a] - 2;
      }
      long long src = c;
      if (A.periodic || bulk) src = (long long)s[0] + (long long)A.n[0] * ((long long)s[1] + (long long)A.n[1] * s[2]);
      const double v = fin[((long long)k * L::Q + i) * A.ncell + src] - L::w(i) * A.Arest[k];
      if (i == 0)
        Codec<PR>::store0(out + (long long)k * L::Q * A.plane, p, out + ((long long)M::K * L::Q + k) * A.plane, p,
                          (typename Prec<PR>::real)v, A.scale[k]);
      else
        Codec<PR>::store(out + ((long long)k * L::Q + i) * A.plane, p, (typename Prec<PR>::real)v, A.scale[k]);
    }
  }
}

// Export f^n (FP64 [K][Q][ncell]) by pulling the stored post-collision values
// (on the axis of a (z, r) grid the odd sets take the mirrored velocity, as
// the step's pull does).
template <int DIM, int CL, int PR>
__global__ void export_pops_kernel(AuxParams A, const typename Prec<PR>::store* fs, double* out) {
  using L = Lattice<DIM>;
  using M = Model<DIM, CL>;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= A.ncell) return;
  int e[3];
  unflatten(A, c, e);
  int b[3] = {e[0], e[1], e[2]};
  if (!A.periodic)
    for (int a = 0; a < DIM; ++a) b[a] = min(max(e[a], 1), A.n[a] - 2);
  for (int k = 0; k < M::K; ++k) {
    bool mirror = false;
    if constexpr (DIM == 2) mirror = A.axi && e[1] == 0 && odd_in_r<CL>(k);
#pragma unroll
    for (int j = 0; j < L::Q; ++j) {
      // D2Q9 with x reversed: 3 <-> 4, 5 <-> 7, 6 <-> 8
      const int i = !mirror ? j : (j == 3 ? 4 : j == 4 ? 3 : j == 5 ? 7 : j == 7 ? 5 : j == 6 ? 8 : j == 8 ? 6 : j);
      int s[3] = {b[0], b[1], b[2]};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        s[a] -= L::c(i, a);
        if (A.periodic) s[a] = s[a] < 0 ? s[a] + A.n[a] : (s[a] >= A.n[a] ? s[a] - A.n[a] : s[a]);
      }
      const long long ps = padded(A, s);
      const double dv =
          i == 0 ? (double)Codec<PR>::load0(fs + (long long)k * L::Q * A.plane, ps,
                                            fs + ((long long)M::K * L::Q + k) * A.plane, ps, A.inv_scale[k])
                 : (double)Codec<PR>::load(fs + ((long long)k * L::Q + i) * A.plane, ps, A.inv_scale[k]);
      out[((long long)k * L::Q + j) * A.ncell + c] = L::w(i) * A.Arest[k] + dv;
    }
  }
}

// FP64 advected scalars of node e from the stored populations.
template <int DIM, int CL, int PR>
__device__ __forceinline__ void advected_d(const AuxParams& A, const typename Prec<PR>::store* fs,
                                           const int* e, double* Av, int nsets = Model<DIM, CL>::K) {
  using L = Lattice<DIM>;
  using M = Model<DIM, CL>;
  int b[3] = {e[0], e[1], e[2]};
  if (!A.periodic)
    for (int a = 0; a < DIM; ++a) b[a] = min(max(e[a], 1), A.n[a] - 2);
  for (int k = nsets; k < M::K; ++k) Av[k] = A.Arest[k];
  for (int k = 0; k < nsets; ++k) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      int q[3] = {b[0], b[1], b[2]};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        q[a] -= L::c(i, a);
        if (A.periodic) q[a] = q[a] < 0 ? q[a] + A.n[a] : (q[a] >= A.n[a] ? q[a] - A.n[a] : q[a]);
      }
      const long long pq = padded(A, q);
      s += i == 0 ? (double)Codec<PR>::load0(fs + (long long)k * L::Q * A.plane, pq,
                                             fs + ((long long)M::K * L::Q + k) * A.plane, pq, A.inv_scale[k])
                  : (double)Codec<PR>::load(fs + ((long long)k * L::Q + i) * A.plane, pq, A.inv_scale[k]);
    }
    Av[k] = A.Arest[k] + s;
  }
}

template <int DIM, int CL, int PR>
__global__ void advected_kernel(AuxParams A, const typename Prec<PR>::store* fs, double* out) {
  using M = Model<DIM, CL>;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= A.ncell) return;
  int e[3];
  unflatten(A, c, e);
  double Av[M::K];
  advected_d<DIM, CL, PR>(A, fs, e, Av);
  for (int k = 0; k < M::K; ++k) out[(long long)k * A.ncell + c] = Av[k];
}

// Macroscopic outputs decoded in FP64 (bits documented in lbpwfa.h).
template <int DIM, int CL, int PR>
__global__ void moments_kernel(AuxParams A, const typename Prec<PR>::store* fs, uint32_t mask, double* out) {
  using M = Model<DIM, CL>;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= A.ncell) return;
  int e[3];
  unflatten(A, c, e);
  // n alone needs only the density set and no decode
  const bool decode = (mask & ~1u) != 0;
  double Av[M::K];
  advected_d<DIM, CL, PR>(A, fs, e, Av, decode ? M::K : 1);
  double v[18];
  for (int j = 0; j < 18; ++j) v[j] = 0.0;
  const double n = Av[0];
  v[0] = n;
  if (!decode) {
    // v[0] = n is all the mask asks for
  } else if constexpr (CL == CL_LEC) {
    double Ap[DIM], u[DIM], Pi, g;
    for (int a = 0; a < DIM; ++a) Ap[a] = Av[1 + a];
    decode_lec<DIM, double>(n, Ap, (1.0 + 0.5 * A.D) * A.mu, A.D, u, Pi, &g);
    for (int a = 0; a < DIM; ++a) { v[1 + a] = u[a]; v[5 + a] = g * u[a]; }
    v[4] = g;
    v[8] = A.mu * Pi;
  } else {
    const double nl = Av[1];
    const double lam = nl / n;
    double u[3] = {0, 0, 0}, aw2 = 0.0;
    for (int a = 0; a < DIM; ++a) { u[a] = Av[2 + a] / nl; aw2 += Av[2 + a] * Av[2 + a]; }
    // gamma = A_1 / sqrt(A_1^2 - |A_w|^2), written without cancellation
    const double aw = sqrt(aw2);
    const double g = nl / sqrt((nl - aw) * (nl + aw));
    for (int a = 0; a < DIM; ++a) { v[1 + a] = u[a]; v[5 + a] = g * u[a]; }
    v[4] = g;
    v[9] = lam;
    // theta zz, xx, yy, zx, zy, xy -> bits 10..15
    const int ta[6] = {0, 1, 2, 0, 0, 1}, tb[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q) {
      const int j = M::thidx(ta[q], tb[q]);
      v[10 + q] = j >= 0 ? Av[2 + DIM + j] / lam : 0.0;
    }
    if constexpr (DIM == 2) {
      // rest-frame pressures (App. A inversion, r -> x, phi -> y, c = 1):
      // P_perp = theta^{yy}, P_par = [theta^{xx} + theta^{zz} - theta^{00}
      // u^2 - theta^{yy} (1 + u_x^2)] / (1 + u_z^2), theta^{00} = u_i u_j
      // theta^{ij} (mass-shell rows); theta^{xy} = theta^{zy} = 0 in 2D
      const double tzz = v[10], txx = v[11], tyy = v[12], tzx = v[13];
      const double t00 = u[0] * u[0] * tzz + u[1] * u[1] * txx + 2.0 * u[0] * u[1] * tzx;
      const double u2 = u[0] * u[0] + u[1] * u[1];
      v[16] = (txx + tzz - t00 * u2 - tyy * (1.0 + u[1] * u[1])) / (1.0 + u[0] * u[0]);
      v[17] = tyy;
    }
  }
  int o = 0;
  for (int bit = 0; bit < 18; ++bit) {
    if (!(mask & (1u << bit))) continue;
    out[(long long)o * A.ncell + c] = v[bit];
    ++o;
  }
}

// Field slots (real, padded) -> FP64 unpadded, for the selected components
// (comp[j] = internal component index z=0, x=1, y=2; is_b[j] picks B).
template <typename real>
__global__ void export_fields_kernel(AuxParams A, const real* E, const real* B, const real* Elo, const real* Blo,
                                     int ncomp, int4 comps, int4 isb, double* out) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= A.ncell) return;
  int e[3];
  unflatten(A, c, e);
  const long long p = padded(A, e);
  const int cc[4] = {comps.x, comps.y, comps.z, comps.w};
  const int bb[4] = {isb.x, isb.y, isb.z, isb.w};
  for (int j = 0; j < ncomp; ++j) {
    const real* src = bb[j] ? B : E;
    const real* lo = bb[j] ? Blo : Elo;
    out[(long long)j * A.ncell + c] = get_field(src, lo, cc[j] * A.plane + p);
  }
}

template <int DIM, typename real>
__global__ void import_fields_kernel(AuxParams A, const double* Ein, const double* Bin, real* E, real* B, real* Elo,
                                     real* Blo) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= A.ncell) return;
  int e[3];
  unflatten(A, c, e);
  const long long p = padded(A, e);
  for (int a = 0; a < 3; ++a) {
    if (Ein) {
      const int b = (a + 1) % 3, d = (a + 2) % 3;
      bool wall = !A.periodic &&
                  ((b >= 1 && b < DIM && e[b] == A.n[b] - 1) || (d >= 1 && d < DIM && e[d] == A.n[d] - 1));
      if (A.axi && a == 1 && e[1] == 0) wall = true;  // E_r on the axis
      put_field(E, Elo, a * A.plane + p, (e_present<DIM>(a) && !wall) ? Ein[a * A.ncell + c] : 0.0);
    }
    const bool axis_b = A.axi && a == 2 && e[1] == 0;  // B_phi on the axis
    if (Bin) put_field(B, Blo, a * A.plane + p, (b_present<DIM>(a) && !axis_b) ? Bin[a * A.ncell + c] : 0.0);
  }
}

// Deterministic FP64 reduction, pass 1: each block reduces a contiguous
// range of nodes with a fixed tree; partial[blk][0..2] = sum n, sum n_b,
// non-finite populations.
template <int DIM, int CL, int PR>
__global__ void reduce_partial_kernel(AuxParams A, const typename Prec<PR>::store* fs, double* partial) {
  using L = Lattice<DIM>;
  using M = Model<DIM, CL>;
  __shared__ double sh[3][256];
  const long long per_block = (A.ncell + gridDim.x - 1) / gridDim.x;
  const long long c0 = blockIdx.x * per_block;
  const long long c1 = min(A.ncell, c0 + per_block);
  double sn = 0.0, sb = 0.0, bad = 0.0;
  for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    int e[3];
    unflatten(A, c, e);
    double Av[M::K];
    advected_d<DIM, CL, PR>(A, fs, e, Av);
    sn += Av[0];
    const double z = e[0] * A.dx, x = (e[1] - A.xoff) * A.dx, y = (e[2] - A.yoff) * A.dx;
    double nbv = driver_long_d(A, z - A.z0 - A.t);
    if (DIM >= 2) nbv *= exp(-(x * x + (DIM >= 3 ? y * y : 0.0)) * A.inv2sr2);
    sb += nbv;
    const long long p = padded(A, e);
    for (int k = 0; k < M::K; ++k)
      for (int i = 0; i < L::Q; ++i) {
        const double v = (double)Codec<PR>::load(fs + ((long long)k * L::Q + i) * A.plane, p, 1.0f);
        if (!isfinite(v)) bad += 1.0;
      }
  }
  sh[0][threadIdx.x] = sn;
  sh[1][threadIdx.x] = sb;
  sh[2][threadIdx.x] = bad;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) partial[blockIdx.x * 3 + q] = sh[q][0];
}

// pass 2: one block sums the partials in index order.
static __global__ void reduce_final_kernel(const double* partial, int nblk, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < nblk; ++b)
    for (int q = 0; q < 3; ++q) s[q] += partial[b * 3 + q];
  for (int q = 0; q < 3; ++q) out[q] = s[q];
}

}  // namespace lbp
