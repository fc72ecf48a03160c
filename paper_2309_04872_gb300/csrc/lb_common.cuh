// Device-side building blocks of the GB300 lattice Boltzmann warm-plasma
// solver: lattice tables, model traits, launch parameters, storage codecs,
// closure decoders and the boundary index rules.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace lbp {

enum { CL_LEC = 0, CL_WARMC = 1 };
// PR_F32C: FP32 storage whose set moments and post-collision remainders are
// carried exactly (every rounding error of their sums kept, one rounding at
// the end), at a higher cost per step than PR_F32.
enum { PR_F64 = 0, PR_F32 = 1, PR_F16S = 2, PR_F32C = 3 };

// ---------------------------------------------------------------------------
// Lattices.  D3Q19 is the set of Fig. 1 (weights 1/3, 1/18, 1/36); D1Q3 and
// D2Q9 are its 1D and 2D members with the same nu^2 = 1/3 (Eq. ade-feq).
// Velocity order is part of the ABI (lbpwfa.h).  Component index 0 = z,
// 1 = x, 2 = y.
// ---------------------------------------------------------------------------
template <int DIM> struct Lattice;

template <> struct Lattice<1> {
  static constexpr int Q = 3;
  __host__ __device__ static constexpr int c(int i, int a) {
    return a != 0 ? 0 : (i == 1 ? 1 : (i == 2 ? -1 : 0));
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
};

template <> struct Lattice<2> {
  static constexpr int Q = 9;
  // 0 rest, 1 +z, 2 -z, 3 +x, 4 -x, 5 +z+x, 6 -z-x, 7 +z-x, 8 -z+x
  __host__ __device__ static constexpr int c(int i, int a) {
    return a == 0 ? ((i == 1 || i == 5 || i == 7) ? 1 : ((i == 2 || i == 6 || i == 8) ? -1 : 0))
         : a == 1 ? ((i == 3 || i == 5 || i == 8) ? 1 : ((i == 4 || i == 6 || i == 7) ? -1 : 0))
                  : 0;
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

template <> struct Lattice<3> {
  static constexpr int Q = 19;
  // 0 rest; faces 1..6: +z -z +x -x +y -y; edges 7..18:
  // (+z+x) (-z-x) (+z-x) (-z+x) (+z+y) (-z-y) (+z-y) (-z+y) (+x+y) (-x-y) (+x-y) (-x+y)
  __host__ __device__ static constexpr int c(int i, int a) {
    return a == 0 ? cz(i) : (a == 1 ? cx(i) : cy(i));
  }
  __host__ __device__ static constexpr int cz(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

// ---------------------------------------------------------------------------
// Model traits.  K advected scalars per closure (Sec. 4.1 LEC: n, n H p;
// Sec. 5.1 WARMC: n, n w^beta, n theta^{beta gamma} / h) and the record of
// decoded values each node publishes to its neighbours (shared memory).
//   LEC   record: n, u[DIM], Pi = (n/gamma)^(1+2/D)
//   WARMC record: n, lambda, u[DIM], theta pairs[NTH], theta^{0a}[DIM]
// WARMC theta pairs: 1D zz; 2D zz xx yy zx; 3D zz xx yy zx zy xy.
// ---------------------------------------------------------------------------
template <int DIM, int CL> struct Model {
  static constexpr int Q = Lattice<DIM>::Q;
  static constexpr int NTH = CL == CL_WARMC ? (DIM == 1 ? 1 : (DIM == 2 ? 4 : 6)) : 0;
  static constexpr int K = CL == CL_LEC ? 1 + DIM : 2 + DIM + NTH;
  static constexpr int NM = CL == CL_LEC ? 2 + DIM : 2 + 2 * DIM + NTH;
  static constexpr int NPREV = CL == CL_WARMC ? 1 + 2 * DIM : 0;  // th00, th0[DIM], w[DIM]
  // record slots
  static constexpr int R_N = 0;
  static constexpr int R_U = CL == CL_LEC ? 1 : 2;
  static constexpr int R_PI = 1 + DIM;          // LEC
  static constexpr int R_LAM = 1;               // WARMC
  static constexpr int R_TH = 2 + DIM;          // WARMC
  static constexpr int R_TH0 = 2 + DIM + NTH;   // WARMC
  __host__ __device__ static constexpr int tha(int j) {
    return j == 0 ? 0 : (j == 1 ? 1 : (j == 2 ? 2 : (j == 3 ? 0 : (j == 4 ? 0 : 1))));
  }
  __host__ __device__ static constexpr int thb(int j) {
    return j == 0 ? 0 : (j == 1 ? 1 : (j == 2 ? 2 : (j == 3 ? 1 : (j == 4 ? 2 : 2))));
  }
  // index of pair (a, b) in the stored list, -1 if not stored
  __host__ __device__ static constexpr int thidx(int a, int b) {
    return DIM == 1 ? ((a == 0 && b == 0) ? 0 : -1)
         : (a == b ? a
            : (((a == 0 && b == 1) || (a == 1 && b == 0)) ? (DIM >= 2 ? 3 : -1)
               : (((a == 0 && b == 2) || (a == 2 && b == 0)) ? (DIM == 3 ? 4 : -1)
                  : (DIM == 3 ? 5 : -1))));
  }
};

template <int PR> struct Prec;
template <> struct Prec<PR_F64> { using real = double; using store = double; };
template <> struct Prec<PR_F32> { using real = float; using store = float; };
template <> struct Prec<PR_F16S> { using real = float; using store = __half; };
template <> struct Prec<PR_F32C> { using real = float; using store = float; };
// whether a storage precision carries its set sums exactly
template <int PR> __host__ __device__ constexpr bool exact_sums() { return PR == PR_F32C; }

// Present field components on the dual Yee grid (component index z, x, y).
template <int DIM> __host__ __device__ constexpr bool e_present(int a) {
  return DIM == 1 ? a == 0 : (DIM == 2 ? (a == 0 || a == 1) : true);
}
template <int DIM> __host__ __device__ constexpr bool b_present(int a) {
  return DIM == 1 ? false : (DIM == 2 ? a == 2 : true);
}
template <int DIM> __host__ __device__ constexpr bool axis_present(int a) { return a < DIM; }

// ---------------------------------------------------------------------------
// Launch parameters of the step kernel (all derived on the host).  Every
// scalar the kernel computes with comes pre-converted in both precisions
// (StepConst), so no double -> float conversion runs on the device.
// ---------------------------------------------------------------------------
template <typename real>
struct StepConst {
  real dx, idx, i2dx;     // dx, 1/dx, 1/(2 dx)
  real dt, idt;           // dt, 1/dt
  real courant, inv_tau;  // C, 1/tau
  real mu, cH;            // mu, (1 + D/2) mu
  real zeta0;             // driver centre z0 + t_n
  real alpha, inv2sz2, inv2sr2;
  real xoff, yoff;        // (nx-1)/2, (ny-1)/2
  real pdz_inv, phalf;    // 1/profile_dz, (len-1)/2
  real Arest[11];
  real ilam0;             // WARMC 1 / lambda_0
  real threst[6];         // WARMC rest theta pairs A_rest,j / lambda_0
};

struct StepParams {
  const void* fin;       // populations, stored deviations, [K][Q][plane]
  void* fout;
  const void* Ein;       // E^{n-1/2} slots [3][plane] (real)
  void* Eout;            // E^{n+1/2}
  const void* Bin;       // B^n
  void* Bout;            // B^{n+1}
  // reduced precision: low parts of E and B (value = high + low, FP32 each;
  // null in FP64)
  const void* Ein_lo;
  void* Eout_lo;
  const void* Bin_lo;
  void* Bout_lo;
  void* prev;            // WARMC previous-step th00, th0[DIM], w[DIM]: [NPREV][plane]
  int have_prev;
  int n[3];              // nodes along z, x, y (1 for absent axes)
  int nzp;               // padded row pitch along z
  long long plane;       // nzp * nx * ny (Q * plane < 2^31 is enforced)
  int axis_stride[3];    // 1, nzp, nzp * nx
  int periodic;
  int D;
  const double* profile; int plen;
  float inv_scale[11];   // FP16S: 1/s_k
  float scale[11];       // FP16S: s_k
  int* err;              // device error word (bit 0: a bounded wait gave up)
  unsigned wait_limit;   // polls of a tile's first barrier wait before it gives up
  void* tape;            // adjoint recording (1D/2D), or null: this step's
                         // deviation moments dA [K], E^{n+1/2} [DIM] and
                         // B^n [present B] as [K + DIM + NB][plane] of real
  StepConst<float> cf;
  StepConst<double> cd;
};

template <typename real> __device__ __forceinline__ const StepConst<real>& consts(const StepParams& P);
template <> __device__ __forceinline__ const StepConst<float>& consts<float>(const StepParams& P) { return P.cf; }
template <> __device__ __forceinline__ const StepConst<double>& consts<double>(const StepParams& P) { return P.cd; }

// Storage codec: populations are kept as deviations from w_i A_rest,k.
// Global-memory access with the state space explicit: a store through a
// plain pointer could alias shared memory, so a kernel whose launch
// parameters live in shared memory (the batched step) would have to reload
// them after every store.
// gld is for data no thread writes during the kernel (the read-only path
// lets the compiler move it past stores); gldc for data the kernel also
// writes (the previous-step values, read and then overwritten in place).
template <typename T> __device__ __forceinline__ void gst(T* p, T v) { __stwb(p, v); }
template <typename T> __device__ __forceinline__ T gld(const T* p) { return __ldg(p); }
template <typename T> __device__ __forceinline__ T gldc(const T* p) { return __ldcg(p); }

template <int PR> struct Codec;
// store_q stores v and returns the value a later load reads back.
// load0 / store0 access the rest population (velocity 0) of a set: the
// reduced-precision format keeps a low part for it in plane K*Q + k of the
// buffer (lo, element j); the other formats ignore lo.
template <> struct Codec<PR_F64> {
  static constexpr int kLoPlanes = 0;  // extra planes per population set
  __device__ static double load(const double* p, long long i, float) { return __ldg(p + i); }
  __device__ static void store(double* p, long long i, double v, float) { gst(p + i, v); }
  __device__ static double store_q(double* p, long long i, double v, float, float) {
    gst(p + i, v);
    return v;
  }
  __device__ static double load0(const double* p, long long i, const double*, long long, float) {
    return __ldg(p + i);
  }
  __device__ static void store0(double* p, long long i, double*, long long, double v, float) { gst(p + i, v); }
  // storage units (the step's working units; scale 1 here)
  static constexpr bool kScaled = false;
  __device__ static double load_u(const double* p, long long i) { return __ldg(p + i); }
  __device__ static double load0_u(const double* p, long long i, const double*, long long) { return __ldg(p + i); }
  __device__ static double store_qu(double* p, long long i, double v) {
    gst(p + i, v);
    return v;
  }
  __device__ static void store0_u(double* p, long long i, double*, long long, double v) { gst(p + i, v); }
};
template <> struct Codec<PR_F32> {
  static constexpr int kLoPlanes = 0;
  __device__ static float load(const float* p, long long i, float) { return __ldg(p + i); }
  __device__ static void store(float* p, long long i, float v, float) { gst(p + i, v); }
  __device__ static float store_q(float* p, long long i, float v, float, float) {
    gst(p + i, v);
    return v;
  }
  __device__ static float load0(const float* p, long long i, const float*, long long, float) {
    return __ldg(p + i);
  }
  __device__ static void store0(float* p, long long i, float*, long long, float v, float) { gst(p + i, v); }
  static constexpr bool kScaled = false;
  __device__ static float load_u(const float* p, long long i) { return __ldg(p + i); }
  __device__ static float load0_u(const float* p, long long i, const float*, long long) { return __ldg(p + i); }
  __device__ static float store_qu(float* p, long long i, float v) {
    gst(p + i, v);
    return v;
  }
  __device__ static void store0_u(float* p, long long i, float*, long long, float v) { gst(p + i, v); }
};
template <> struct Codec<PR_F32C> : Codec<PR_F32> {};
// Binary16 of the scaled deviation.  The rest population takes the remainder
// of its set's moment in the collision, so its rounding is the one error of
// the node's moment that does not cancel; it carries a second binary16 with
// its rounding residual scaled by 2^11 (together about 22 significant bits).
template <> struct Codec<PR_F16S> {
  static constexpr int kLoPlanes = 1;
  static constexpr float kLoScale = 2048.0f, kLoInv = 1.0f / 2048.0f;
  __device__ static float load(const __half* p, long long i, float inv_s) {
    return __half2float(__ldg(p + i)) * inv_s;
  }
  __device__ static void store(__half* p, long long i, float v, float s) {
    gst(p + i, __float2half_rn(v * s));
  }
  __device__ static float store_q(__half* p, long long i, float v, float s, float inv_s) {
    const __half h = __float2half_rn(v * s);
    gst(p + i, h);
    return __half2float(h) * inv_s;
  }
  __device__ static float join(__half hi, __half lo, float inv_s) {
    return fmaf(__half2float(lo), kLoInv, __half2float(hi)) * inv_s;
  }
  __device__ static float load0(const __half* p, long long i, const __half* lo, long long j, float inv_s) {
    return join(__ldg(p + i), __ldg(lo + j), inv_s);
  }
  __device__ static void store0(__half* p, long long i, __half* lo, long long j, float v, float s) {
    const float x = v * s;
    const __half h = __float2half_rn(x);
    gst(p + i, h);
    // x - h is exact in FP32: h is x rounded to 11 significant bits, and the
    // difference holds the rest of x's bits
    gst(lo + j, __float2half_rn(__fsub_rn(x, __half2float(h)) * kLoScale));
  }
  // Storage units: the stored binary16 read as FP32 without the 1/s_k.  The
  // scale is a power of two, so working in these units and applying 1/s_k
  // once to a set's moment gives the same bits as scaling every population.
  static constexpr bool kScaled = true;
  __device__ static float load_u(const __half* p, long long i) { return __half2float(__ldg(p + i)); }
  __device__ static float join_u(__half hi, __half lo) {
    return fmaf(__half2float(lo), kLoInv, __half2float(hi));
  }
  __device__ static float load0_u(const __half* p, long long i, const __half* lo, long long j) {
    return join_u(__ldg(p + i), __ldg(lo + j));
  }
  __device__ static float store_qu(__half* p, long long i, float x) {
    const __half h = __float2half_rn(x);
    gst(p + i, h);
    return __half2float(h);
  }
  __device__ static void store0_u(__half* p, long long i, __half* lo, long long j, float x) {
    const __half h = __float2half_rn(x);
    gst(p + i, h);
    gst(lo + j, __float2half_rn(__fsub_rn(x, __half2float(h)) * kLoScale));
  }
};

// ---------------------------------------------------------------------------
// Index rules.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap_or_clamp(int v, int n, int periodic) {
  if (periodic) return v < 0 ? v + n : (v >= n ? v - n : v);
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}
__device__ __forceinline__ int cell_index32(const StepParams& P, int z, int x, int y) {
  return z + x * P.axis_stride[1] + y * P.axis_stride[2];
}

// Compensated (two-float) accumulation hi + lo += d: Knuth's two-sum of hi
// and d, its error folded into lo and renormalised, FP32 operations only.
__device__ __forceinline__ void two_float_add(float& hi, float& lo, float d) {
  const float s = __fadd_rn(hi, d);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
  const float l = __fadd_rn(lo, err);
  hi = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(hi, s));
}

// Knuth's TwoSum: s = fl(a + b) and e with s + e == a + b exactly (FP32
// operations only, uncontracted).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Uncontracted sums: the same rounding in every kernel that inlines them.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

__device__ __forceinline__ float rsqrt_t(float x) { return 1.0f / sqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }

// Power (n/gamma)^(2/D) of the LEC closure (Eq. temp-scaling).
template <typename real> __device__ __forceinline__ real pow_2_over_D(real x, int D);
template <> __device__ __forceinline__ double pow_2_over_D<double>(double x, int D) {
  return D == 1 ? x * x : (D == 3 ? cbrt(x * x) : x);
}
template <> __device__ __forceinline__ float pow_2_over_D<float>(float x, int D) {
  return D == 1 ? x * x : (D == 3 ? cbrtf(x * x) : x);
}

// Pi - 1 = (n/gamma)^(1+2/D) - 1 without cancellation near rest, from
// dn = n - 1, |p|^2 and gamma: x - 1 = (dn - (gamma - 1)) / gamma with
// gamma - 1 = |p|^2 / (gamma + 1); D = 1: x^3 - 1 = d (3 + 3 d + d^2);
// D = 3: x^(5/3) - 1 = d x^(2/3) + (x^(2/3) - 1), x^(2/3) - 1 =
// (x^2 - 1) / (x^(4/3) + x^(2/3) + 1).
template <typename real>
__device__ __forceinline__ real lec_pi_minus_1(real dn, real p2, real g, int D) {
  const real d = (dn - p2 / (g + real(1))) / g;
  if (D == 1) return d * (real(3) + d * (real(3) + d));
  const real x = real(1) + d;
  const real xe = pow_2_over_D<real>(x, D);
  return d * xe + d * (real(2) + d) / (xe * xe + xe + real(1));
}
// FP32 form: x^(2/3) enters only multiplied by d or in a denominator near 3,
// so the hardware log2/exp2 (a few ulp) keeps Pi - 1 to a few ulp; so do the
// hardware reciprocals (about 1 ulp), which replace correctly rounded ones.
__device__ __forceinline__ float lec_pi_minus_1_f32(float dn, float p2, float ig, float g, int D) {
  const float d = (dn - p2 * __fdividef(1.0f, g + 1.0f)) * ig;
  if (D == 1) return d * (3.0f + d * (3.0f + d));
  const float x = 1.0f + d;
  const float xe = exp2f((2.0f / 3.0f) * __log2f(x));
  return d * xe + d * (2.0f + d) * __fdividef(1.0f, fmaf(xe, xe, xe) + 1.0f);
}

// LEC transport velocity, Sec. 4.1: p^(0) = A_p / n, then
// gamma^(k) = sqrt(1 + |p^(k)|^2), p^(k+1) = p^(0) / (1 + (1 + D/2) mu (n/gamma^(k))^(2/D)),
// stopped when the largest change is within a few ulps of the largest |p|.
// cH = (1 + D/2) mu.
template <int DIM, typename real>
__device__ __forceinline__ void decode_lec(real n, const real* Ap, real cH, int D, real* u, real& Pi,
                                           real* gamma_out = nullptr, real dn = real(0),
                                           real* pim1_out = nullptr) {
  constexpr bool dbl = sizeof(real) == 8;
  const real tol = dbl ? real(1e-15) : real(4e-7);
  const int maxit = dbl ? 64 : 32;
  const real in_ = real(1) / n;
  real p0[DIM], p[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) { p0[a] = Ap[a] * in_; p[a] = p0[a]; }
  for (int it = 0; it < maxit; ++it) {
    real s = real(1);
#pragma unroll
    for (int a = 0; a < DIM; ++a) s += p[a] * p[a];
    const real ig = rsqrt_t(s);
    const real iH = real(1) / (real(1) + cH * pow_2_over_D<real>(n * ig, D));
    real d = 0, pm = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const real pn = p0[a] * iH;
      d = fmax(d, fabs(pn - p[a]));
      pm = fmax(pm, fabs(pn));
      p[a] = pn;
    }
    if (d <= tol * pm) break;
  }
  real s = real(1);
#pragma unroll
  for (int a = 0; a < DIM; ++a) s += p[a] * p[a];
  const real g = sqrt(s);
  const real ig = real(1) / g;
#pragma unroll
  for (int a = 0; a < DIM; ++a) u[a] = p[a] * ig;
  const real x = n * ig;
  Pi = x * pow_2_over_D<real>(x, D);
  if (gamma_out) *gamma_out = g;
  if (pim1_out) *pim1_out = lec_pi_minus_1<real>(dn, s - real(1), g, D);
}

// FP32 form of the same iteration for the reduced-precision modes.  The
// power is split as (n/gamma)^(2/D) = n^(2/D) s^(-1/D) with s = 1 + |p|^2,
// so log2 n leaves the loop and one iteration costs a log2, an exp2 and a
// hardware reciprocal (their error is scaled by (1 + D/2) mu in H: below
// 1e-8 for mu <= 5e-2).  1/gamma of the result is the hardware reciprocal
// square root (about 1 ulp); gamma = s / gamma.
template <int DIM>
__device__ __forceinline__ void decode_lec_f32(float n, const float* Ap, float cH, int D, float* u, float& Pi,
                                               float dn = 0.0f, float* pim1_out = nullptr) {
  const float in_ = __fdividef(1.0f, n);
  float p0[DIM], p[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) { p0[a] = Ap[a] * in_; p[a] = p0[a]; }
  const float e = 2.0f / (float)D;
  const float ln = e * __log2f(n);  // log2 n^(2/D)
  const float n2 = n * n;           // D = 1: (n/gamma)^2 = n^2 / s
  for (int it = 0; it < 32; ++it) {
    float s = 1.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) s = fmaf(p[a], p[a], s);
    const float pw = D == 1 ? n2 * __fdividef(1.0f, s) : exp2f(fmaf(-0.5f * e, __log2f(s), ln));
    const float iH = __fdividef(1.0f, fmaf(cH, pw, 1.0f));
    float d = 0.0f, pm = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const float pn = p0[a] * iH;
      d = fmaxf(d, fabsf(pn - p[a]));
      pm = fmaxf(pm, fabsf(pn));
      p[a] = pn;
    }
    if (d <= 4e-7f * pm) break;
  }
  float s = 1.0f;
#pragma unroll
  for (int a = 0; a < DIM; ++a) s = fmaf(p[a], p[a], s);
  const float ig = rsqrtf(s);
  const float g = s * ig;
#pragma unroll
  for (int a = 0; a < DIM; ++a) u[a] = p[a] * ig;
  if (pim1_out) {
    // only Pi - 1 is wanted (central differences)
    float p2 = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) p2 = fmaf(p[a], p[a], p2);
    *pim1_out = lec_pi_minus_1_f32(dn, p2, ig, g, D);
    Pi = 1.0f + *pim1_out;
  } else {
    const float x = n * ig;
    Pi = x * pow_2_over_D<float>(x, D);
  }
}

// Driver longitudinal factor L(zeta) (Eq. bunch-density, rms reading).  A
// sampled profile is interpolated linearly with zero samples just outside
// both ends, so L stays continuous.
template <typename real>
__device__ __forceinline__ real driver_long(const StepParams& P, const StepConst<real>& S, real zeta) {
  if (P.profile) {
    const real q = zeta * S.pdz_inv + S.phalf;
    if (!(q > real(-1) && q < real(P.plen))) return real(0);
    const int j = (int)floor(q);
    const real fr = q - real(j);
    const real a = j >= 0 ? real(gld(P.profile + j)) : real(0);
    const real b = j + 1 < P.plen ? real(gld(P.profile + j + 1)) : real(0);
    return (real(1) - fr) * a + fr * b;
  }
  return S.alpha * exp(-zeta * zeta * S.inv2sz2);
}

}  // namespace lbp
