// Fused time step of the moment-matching LB warm-plasma scheme (one launch
// per step).  A CTA owns a tile of TZ x TX x TY nodes and goes through
//   A. pull + moments + closure decode for the tile and a one-node halo
//      (Eq. disc-moments-ade; LEC Sec. 4.1 iteration or WARMC Sec. 5.1),
//      published as a record per node in shared memory;
//   B. E^{n+1/2} = E^{n-1/2} + dt (curl B^n + n u + n_b z) on the slots of
//      the tile and its low-side halo (dual Yee grid, Sec. 6);
//   C. per tile node: B^{n+1} = B^n - dt curl E^{n+1/2}; sources of Eq.
//      lb-ade-lec-comps-F / lb-ade-warmc-comps-F with E^{n+1/2}, B^n and
//      central differences of the neighbours' records; BGK relaxation to
//      Eq. ade-feq plus w_i dt F (Eq. lbe, lsource); store.
// Streaming is the pull in A/C of the next step: the stored array holds
// post-collision populations, and node x reads f*_i(x - xi_i) (with the
// open-boundary rule of Eq. open-bc: a boundary node reads as its nearest
// bulk node).  Populations are kept as deviations from w_i A_rest,k.
#pragma once

#include <type_traits>

#include "lb_common.cuh"

namespace lbp {

template <int DIM>
__host__ __device__ constexpr bool opposite_pairs() {
  using L = Lattice<DIM>;
  for (int i = 1; i + 1 < L::Q; i += 2)
    for (int a = 0; a < 3; ++a)
      if (L::c(i + 1, a) != -L::c(i, a) || L::w(i + 1) != L::w(i)) return false;
  return true;
}

__host__ __device__ constexpr int levi(int i, int j, int k) {
  return (i == j || j == k || i == k) ? 0
       : (((i == 0 && j == 1) || (i == 1 && j == 2) || (i == 2 && j == 0)) ? 1 : -1);
}

// Moment of one population set, A_k = sum_i f_ki (Eq. disc-moments-ade), with
// each pair of opposite velocities added first: the pair sum cancels the odd
// (momentum-flux) parts before they meet the set's total, which halves the
// rounding of the deviation moment in reduced precision.  Uncontracted, so
// every caller gets the same bits.
template <int Q, typename real>
__device__ __forceinline__ real set_moment(const real* df) {
  real s = df[0];
#pragma unroll
  for (int i = 1; i + 1 < Q; i += 2) s = add_rn(s, add_rn(df[i], df[i + 1]));
  return s;
}

// Deviation moment dA_k of a set pulled in storage units: the sum, times
// 1/s_k for the scaled binary16 format (a power of two: the same bits as
// summing the scaled-back populations).
// The set sum with every rounding error kept (TwoSum) and one final
// rounding (exact_sums precisions).
template <int Q>
__device__ __forceinline__ float set_moment_exact(const float* df) {
  float s = df[0], c = 0.0f;
#pragma unroll
  for (int i = 1; i + 1 < Q; i += 2) {
    float p, e1, e2;
    two_sum(df[i], df[i + 1], p, e1);
    two_sum(s, p, s, e2);
    c = __fadd_rn(c, __fadd_rn(e1, e2));
  }
  return __fadd_rn(s, c);
}

template <int Q, int PR, typename real>
__device__ __forceinline__ real set_dA(const real* df, float inv_s) {
  if constexpr (exact_sums<PR>()) return set_moment_exact<Q>(df);
  const real m = set_moment<Q>(df);
  if constexpr (Codec<PR>::kScaled) return m * inv_s;
  return m;
}

// Running sum of the stored moving populations of a set, and the rest
// population as the remainder (dA + dt F) - that sum: plainly, or with the
// rounding errors carried (exact_sums) so the remainder is rounded once.
template <int PR, typename real>
struct Remainder {
  static_assert(!exact_sums<PR>() || !Codec<PR>::kScaled, "the exact sums run in unscaled FP32");
  real s = 0, c = 0;
  __device__ __forceinline__ void add(real v) {
    if constexpr (exact_sums<PR>()) {
      float e;
      two_sum(s, v, s, e);
      c = __fadd_rn(c, e);
    } else {
      s = add_rn(s, v);
    }
  }
  // (dA + dtF) us - sum
  __device__ __forceinline__ real rest(real dA, real dtF, real us) const {
    if constexpr (exact_sums<PR>()) {
      float th, tl, dh, dl;
      two_sum(dA, dtF, th, tl);
      two_sum(th, -s, dh, dl);
      return __fadd_rn(dh, __fsub_rn(__fadd_rn(dl, tl), c));
    } else {
      return sub_rn(add_rn(dA, dtF) * us, s);
    }
  }
};

// 3D models keep the loops over population sets rolled: one 19-velocity body
// per loop instead of K (up to 11), so the step fits the instruction cache.
// 2D models unroll them (2D WARMC, 8 x 9 populations, runs faster unrolled at
// 110 registers than rolled at 63).
template <int DIM, int K> struct RollSets {
  static constexpr bool value = DIM == 3;
};

template <int DIM, int CL, int PR, int TZ, int TX, int TY>
struct StepCfg {
  using M = Model<DIM, CL>;
  using real = typename Prec<PR>::real;
  static constexpr int NT = TZ * TX * TY;
  static constexpr int RZ = TZ + 2;
  static constexpr int RX = DIM >= 2 ? TX + 2 : 1;
  static constexpr int RY = DIM >= 3 ? TY + 2 : 1;
  static constexpr int NR = RZ * RX * RY;
  // records, E slots, and the separable driver factors of the tile's slots
  static constexpr int NDRV = (TZ + 1) + (TX + 1) + (TY + 1);
  // FP32 fields are carried as high + low parts (compensated updates)
  static constexpr bool CF = sizeof(real) == 4;
  static constexpr int NEC = DIM;                   // present E components (z[, x[, y]])
  static constexpr int NE_SLOTS = CF ? 2 * NEC : NEC;
  // rolled set loops keep their per-set values (moments, sources) in a
  // per-thread shared-memory column [K][NT] instead of local memory
  static constexpr bool ROLL = RollSets<DIM, M::K>::value;
  static constexpr int NSCR = ROLL ? M::K * NT : 0;
  // 2D: fields of the low-side halo E slots, staged by asynchronous copies
  // (E_z, E_x, B_y and B_y one node up along x and z; FP32 also low parts)
  static constexpr int NHALO_E = DIM == 2 ? (TZ + 1) * (TX + 1) - TZ * TX : 0;
  static constexpr int NSTAGE = NHALO_E * (CF ? 10 : 5);
  // 3D marching: the set moments of the top plane's nodes beyond the first
  // NT, pulled one (node, set) per thread across the CTA
  // (2D WARMC: the decode ring's set moments, pulled the same way)
  static constexpr int NXTRA = (DIM == 3 && TY == 1 && RZ * RX > NT) ? RZ * RX - NT
                               : ((DIM == 2 && CL == CL_WARMC && NR > NT) ? NR - NT : 0);
  static constexpr int NSPLIT = NXTRA * M::K;
  static constexpr size_t smem_bytes =
      ((size_t)(M::NM + NE_SLOTS) * NR + NDRV + NSCR + NSTAGE + NSPLIT) * sizeof(real);
  // Sets too wide for registers (2D WARMC, K*Q = 72) could keep the own
  // node's populations in a shared-memory column [K*Q][NT] for the
  // collision instead of pulling them again (launch reserving
  // smem_bytes_gkeep).  Off: it holds the kernel to two CTAs per SM, and
  // three CTAs per SM that pull again measure faster (1024 x 512 FP32: 5.94
  // against 5.67 GLUPS; 4.2 with neither).
  static constexpr bool SKEEP_OK = false;
  static constexpr int NKEEP = SKEEP_OK ? M::K * M::Q * NT : 0;
  static constexpr size_t smem_bytes_gkeep = smem_bytes + (size_t)NKEEP * sizeof(real);
  __host__ __device__ static constexpr int stride(int a) { return a == 0 ? 1 : (a == 1 ? RZ : RZ * RX); }
};

// Axisymmetric (z, r) grids: whether set k changes sign under r -> -r (an odd
// number of r indices: n A_r; n lambda u_r and lambda theta^{rz}).
template <int CL>
__host__ __device__ constexpr bool odd_in_r(int k) {
  if constexpr (CL == CL_LEC) {
    return k == 2;
  } else {
    using M = Model<2, CL>;
    if (k == 3) return true;
    if (k >= 4) return (M::tha(k - 4) == 1) != (M::thb(k - 4) == 1);
    return false;
  }
}

// Deviations of the pulled populations f^n_ki - w_i A_rest,k at node
// (z, x, y) (already inside the domain), straight from global memory, in
// storage units (FP16S: times s_k; set_dA applies 1/s_k to the set's sum).
// AXI: (z, r) grid whose x = 0 row is the r = 0 boundary node; it takes the
// pulled populations of its bulk node as they are (Eq. open-bc) for the
// sets even under r -> -r and with the mirrored velocity (Eq. reflective-bc)
// for the odd ones.
template <int DIM, int CL, int PR, bool EDGE, bool AXI = false>
__device__ __forceinline__ void pulled_dev(const StepParams& P, int z, int x, int y, int k,
                                           typename Prec<PR>::real* df) {
  using L = Lattice<DIM>;
  using store = typename Prec<PR>::store;
  static_assert(!AXI || DIM == 2, "axisymmetric grids are (z, r)");
  const bool mirror = AXI && EDGE && x == 0 && odd_in_r<CL>(k);
  if (EDGE && !P.periodic) {
    z = min(max(z, 1), P.n[0] - 2);
    if (DIM >= 2) x = min(max(x, 1), P.n[1] - 2);
    if (DIM >= 3) y = min(max(y, 1), P.n[2] - 2);
  }
  const store* f = (const store*)P.fin + (size_t)k * L::Q * (size_t)P.plane;
  const int pl = (int)P.plane;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    int sz = z - L::c(i, 0), sx = x - L::c(i, 1), sy = y - L::c(i, 2);
    if (EDGE && P.periodic) {
      sz = sz < 0 ? sz + P.n[0] : (sz >= P.n[0] ? sz - P.n[0] : sz);
      if (DIM >= 2) sx = sx < 0 ? sx + P.n[1] : (sx >= P.n[1] ? sx - P.n[1] : sx);
      if (DIM >= 3) sy = sy < 0 ? sy + P.n[2] : (sy >= P.n[2] ? sy - P.n[2] : sy);
    }
    if (i == 0) {
      // rest population (with its low part in the reduced-precision format)
      const store* lo = (const store*)P.fin + ((size_t)Model<DIM, CL>::K * L::Q + k) * (size_t)P.plane;
      const int c0 = cell_index32(P, sz, sx, sy);
      df[0] = Codec<PR>::load0_u(f, c0, lo, c0);
    } else {
      df[i] = Codec<PR>::load_u(f, i * pl + cell_index32(P, sz, sx, sy));
    }
  }
  if constexpr (AXI) {
    if (mirror) {
      // D2Q9 order (0, +z, -z, +x, -x, +z+x, -z-x, +z-x, -z+x): x reversed
      typename Prec<PR>::real t;
      t = df[3]; df[3] = df[4]; df[4] = t;
      t = df[5]; df[5] = df[7]; df[7] = t;
      t = df[6]; df[6] = df[8]; df[8] = t;
    }
  }
}

// Population source reading the stored post-collision array in global memory
// (any boundary rule).
template <int DIM, int CL, int PR, bool SHARED_KEEP = false, bool AXI = false>
struct GlobalPull {
  // the step keeps the own node's populations in shared memory for the
  // collision (sets too wide for registers) instead of pulling them again
  static constexpr bool kSharedKeep = SHARED_KEEP;
  const StepParams& P;
  template <bool EDGE>
  __device__ __forceinline__ void get(int z, int x, int y, int k, typename Prec<PR>::real* df) const {
    pulled_dev<DIM, CL, PR, EDGE, AXI>(P, z, x, y, k, df);
  }
};

// Decode the record of one node from its deviation moments dA[K].  Values
// that only enter central differences are kept as deviations from rest
// (LEC: Pi - 1; WARMC: theta - theta_rest), so the differences of neighbours
// do not cancel against the rest value in reduced precision.
template <int DIM, int CL, typename real>
__device__ __forceinline__ void decode_record(const StepParams& P, const StepConst<real>& S, const real* dA,
                                              real* rec) {
  using M = Model<DIM, CL>;
  if constexpr (CL == CL_LEC) {
    real n = real(1) + dA[0];
    real Ap[DIM], u[DIM], Pi, Pim1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) Ap[a] = dA[1 + a];
    if constexpr (sizeof(real) == 4) decode_lec_f32<DIM>(n, Ap, S.cH, P.D, u, Pi, dA[0], &Pim1);
    else decode_lec<DIM, real>(n, Ap, S.cH, P.D, u, Pi, nullptr, dA[0], &Pim1);
    rec[M::R_N] = n;
#pragma unroll
    for (int a = 0; a < DIM; ++a) rec[M::R_U + a] = u[a];
    rec[M::R_PI] = Pim1;
  } else {
    const real n = real(1) + dA[0];
    const real nl = S.Arest[1] + dA[1];
    const real inl = real(1) / nl;
    const real lam = nl / n;
    const real ilam = n * inl;
    real u[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) u[a] = dA[2 + a] * inl;
    // theta_j - theta_rest,j = A_rest,j (n/nl - 1/lambda_0) + dA_j n/nl with
    // n/nl - 1/lambda_0 = (dA_0 - dA_1/lambda_0)/nl
    const real dil = (dA[0] - dA[1] * S.ilam0) * inl;
    real th[M::NTH], thd[M::NTH];
#pragma unroll
    for (int j = 0; j < M::NTH; ++j) {
      thd[j] = S.Arest[2 + DIM + j] * dil + dA[2 + DIM + j] * ilam;
      th[j] = S.threst[j] + thd[j];
    }
    rec[M::R_N] = n;
    rec[M::R_LAM] = lam;
#pragma unroll
    for (int a = 0; a < DIM; ++a) rec[M::R_U + a] = u[a];
#pragma unroll
    for (int j = 0; j < M::NTH; ++j) rec[M::R_TH + j] = thd[j];
    // theta^{0a} = u_b theta^{ab} (Eq. traces4, App. A mass-shell rows)
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      real s = 0;
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        const int j = M::thidx(a, b);
        if (j >= 0) s += u[b] * th[j];
      }
      rec[M::R_TH0 + a] = s;
    }
  }
}

// Field values around the own node, loaded at the start of the kernel so
// that their latency overlaps the population staging and the decode.
//   Ec[a]    = E_a^{n-1/2} at the node's slot
//   Bc[a]    = B_a^n at the node's slot
//   Bp[d][b] = B_d^n one node up along axis b (curl at the E slot)
//   Bm[a]    = B_a^n one node down along a (node average of B_a)
//   *_lo: low parts of the same values (FP32 fields; zero in FP64)
template <typename real>
struct FieldPF {
  real Ec[3], Bc[3], Bp[3][3], Bm[3];
  real Ec_lo[3], Bc_lo[3], Bp_lo[3][3], Bm_lo[3];
};

template <bool EDGE>
__device__ __forceinline__ int nb_offset(const StepParams& P, int e, int axis, int delta) {
  if (!EDGE) return delta * P.axis_stride[axis];
  const int v = wrap_or_clamp(e + delta, P.n[axis], P.periodic);
  return (v - e) * P.axis_stride[axis];
}

template <int DIM, typename real, bool EDGE>
__device__ __forceinline__ void load_fields(const StepParams& P, int e0, int e1, int e2, int id, FieldPF<real>& F) {
  constexpr bool CF = sizeof(real) == 4;
  const real* Ein = reinterpret_cast<const real*>(P.Ein);
  const real* Bin = reinterpret_cast<const real*>(P.Bin);
  const real* Elo = reinterpret_cast<const real*>(P.Ein_lo);
  const real* Blo = reinterpret_cast<const real*>(P.Bin_lo);
  const int pl = (int)P.plane;
  const int e[3] = {e0, e1, e2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    F.Ec_lo[a] = F.Bc_lo[a] = F.Bm_lo[a] = real(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) F.Bp_lo[a][b] = real(0);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (e_present<DIM>(a)) {
      F.Ec[a] = gld(Ein + a * pl + id);
      if (CF) F.Ec_lo[a] = gld(Elo + a * pl + id);
    }
    if (b_present<DIM>(a)) {
      F.Bc[a] = gld(Bin + a * pl + id);
      if (CF) F.Bc_lo[a] = gld(Blo + a * pl + id);
      if (axis_present<DIM>(a)) {
        const int o = a * pl + id + nb_offset<EDGE>(P, e[a], a, -1);
        F.Bm[a] = gld(Bin + o);
        if (CF) F.Bm_lo[a] = gld(Blo + o);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!e_present<DIM>(a)) continue;
    const int b = (a + 1) % 3, d = (a + 2) % 3;
    if (axis_present<DIM>(b) && b_present<DIM>(d)) {
      const int o = d * pl + id + nb_offset<EDGE>(P, e[b], b, +1);
      F.Bp[d][b] = gld(Bin + o);
      if (CF) F.Bp_lo[d][b] = gld(Blo + o);
    }
    if (axis_present<DIM>(d) && b_present<DIM>(b)) {
      const int o = b * pl + id + nb_offset<EDGE>(P, e[d], d, +1);
      F.Bp[b][d] = gld(Bin + o);
      if (CF) F.Bp_lo[b][d] = gld(Blo + o);
    }
  }
}

// Asynchronous 4- or 8-byte copy global -> shared (cp.async); each thread
// waits for its own copies with cp_async_wait_all.
template <typename real>
__device__ __forceinline__ void cp_async_el(real* dst, const real* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const size_t g = __cvta_generic_to_global(src);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(g), "n"(sizeof(real)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// 2D bulk node `id`: queue copies of the values load_fields reads (E_z, E_x,
// B_y, B_y at x + 1 and at z + 1, then the low parts in FP32) to dst[v * ns].
template <typename real>
__device__ __forceinline__ void stage_fields_2d(const StepParams& P, int id, real* dst, int ns) {
  constexpr bool CF = sizeof(real) == 4;
  const int pl = (int)P.plane;
  const int o[5] = {id, pl + id, 2 * pl + id, 2 * pl + id + P.axis_stride[1], 2 * pl + id + 1};
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    cp_async_el(dst + v * ns, (v < 2 ? reinterpret_cast<const real*>(P.Ein) : reinterpret_cast<const real*>(P.Bin)) + o[v]);
    if (CF)
      cp_async_el(dst + (5 + v) * ns,
                  (v < 2 ? reinterpret_cast<const real*>(P.Ein_lo) : reinterpret_cast<const real*>(P.Bin_lo)) + o[v]);
  }
}

// The staged values as load_fields<2> would have loaded them.
template <typename real>
__device__ __forceinline__ void fields_2d_from_stage(const real* src, int ns, FieldPF<real>& F) {
  constexpr bool CF = sizeof(real) == 4;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    F.Ec[a] = F.Bc[a] = F.Bm[a] = F.Ec_lo[a] = F.Bc_lo[a] = F.Bm_lo[a] = real(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) F.Bp[a][b] = F.Bp_lo[a][b] = real(0);
  }
  F.Ec[0] = src[0];
  F.Ec[1] = src[ns];
  F.Bc[2] = src[2 * ns];
  F.Bp[2][1] = src[3 * ns];
  F.Bp[2][0] = src[4 * ns];
  if (CF) {
    F.Ec_lo[0] = src[5 * ns];
    F.Ec_lo[1] = src[6 * ns];
    F.Bc_lo[2] = src[7 * ns];
    F.Bp_lo[2][1] = src[8 * ns];
    F.Bp_lo[2][0] = src[9 * ns];
  }
}

// Difference of two compensated values (high parts first: close values
// subtract exactly).
template <typename real>
__device__ __forceinline__ real diff2(real ah, real al, real bh, real bl) {
  return (ah - bh) + (al - bl);
}

// Driver current n_b at the E_z slot of node e: L(z - z0 - t) at the node's
// z, times the transverse Gaussians half a cell up along x and y.
template <int DIM, typename real>
__device__ __forceinline__ real driver_at(const StepParams& P, const StepConst<real>& S, int e0, int e1, int e2) {
  real nbv = driver_long<real>(P, S, real(e0) * S.dx - S.zeta0);
  if (DIM >= 2) {
    const real x = (real(e1) - S.xoff + real(0.5)) * S.dx;
    real r2 = x * x;
    if (DIM >= 3) {
      const real y = (real(e2) - S.yoff + real(0.5)) * S.dx;
      r2 += y * y;
    }
    nbv *= exp(-r2 * S.inv2sr2);
  }
  return nbv;
}

// E_a^{n+1/2} at the slot of node e (region index r): dual-grid curl of B^n,
// n u_a averaged over the nodes around the slot, driver current for a = z.
// AXI: (z, r) grid with node j at r = j dx: E_r vanishes on the axis and
// (curl B)_z = (1/r) d_r (r B_phi) at r_{j+1/2}, which is the Cartesian
// difference plus (B_{j+1} + B_j) / ((2j + 1) dx).
template <int DIM, int CL, int PR, int TZ, int TX, int TY, bool EDGE, bool AXI = false>
__device__ __forceinline__ void e_slot(const StepParams& P, const StepConst<typename Prec<PR>::real>& S,
                                       const typename Prec<PR>::real* smac, typename Prec<PR>::real* sE,
                                       const typename Prec<PR>::real* sdrv, int oz, int ox, int oy,
                                       int r, int e0, int e1, int e2,
                                       const FieldPF<typename Prec<PR>::real>& F) {
  using C = StepCfg<DIM, CL, PR, TZ, TX, TY>;
  using M = Model<DIM, CL>;
  using real = typename Prec<PR>::real;
  constexpr int NR = C::NR;
  const int e[3] = {e0, e1, e2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!e_present<DIM>(a)) continue;
    const int b = (a + 1) % 3, d = (a + 2) % 3;
    if (EDGE && !P.periodic) {
      bool wall = false;
      if (b >= 1 && axis_present<DIM>(b) && e[b] == P.n[b] - 1) wall = true;
      if (d >= 1 && axis_present<DIM>(d) && e[d] == P.n[d] - 1) wall = true;
      if (AXI && a == 1 && e1 == 0) wall = true;
      if (wall) {
        sE[a * NR + r] = real(0);
        if (C::CF) sE[(C::NEC + a) * NR + r] = real(0);
        continue;
      }
    }
    real curl = 0;
    if (axis_present<DIM>(b) && b_present<DIM>(d))
      curl += diff2(F.Bp[d][b], F.Bp_lo[d][b], F.Bc[d], F.Bc_lo[d]) * S.idx;
    if (axis_present<DIM>(d) && b_present<DIM>(b))
      curl -= diff2(F.Bp[b][d], F.Bp_lo[b][d], F.Bc[b], F.Bc_lo[b]) * S.idx;
    if constexpr (AXI) {
      if (a == 0)
        curl += ((F.Bp[2][1] + F.Bp_lo[2][1]) + (F.Bc[2] + F.Bc_lo[2])) * (S.idx / real(2 * e1 + 1));
    }
    real J = 0;
    if (a < DIM) {
      const bool ob = axis_present<DIM>(b), od = axis_present<DIM>(d);
      const int sb = ob ? C::stride(b) : 0, sd = od ? C::stride(d) : 0;
      const int nb = ob ? 2 : 1, nd = od ? 2 : 1;
#pragma unroll
      for (int jb = 0; jb < 2; ++jb)
#pragma unroll
        for (int jd = 0; jd < 2; ++jd) {
          if (jb < nb && jd < nd) {
            const int rr = r + jb * sb + jd * sd;
            J += smac[M::R_N * NR + rr] * smac[(M::R_U + a) * NR + rr];
          }
        }
      J *= real(1) / real(nb * nd);
    }
    if (a == 0) {
      real nbv;
      if (!EDGE) {
        // separable driver n_b = L(zeta) T(x) T(y) from the tile's tables
        nbv = sdrv[e0 - oz];
        if (DIM >= 2) nbv *= sdrv[(TZ + 1) + (e1 - ox)];
        if (DIM >= 3) nbv *= sdrv[(TZ + 1) + (TX + 1) + (e2 - oy)];
      } else {
        nbv = driver_at<DIM, real>(P, S, e0, e1, e2);
      }
      J += nbv;
    }
    if constexpr (C::CF) {
      real hi = F.Ec[a], lo = F.Ec_lo[a];
      two_float_add(hi, lo, S.dt * (curl + J));
      sE[a * NR + r] = hi;
      sE[(C::NEC + a) * NR + r] = lo;
    } else {
      sE[a * NR + r] = F.Ec[a] + S.dt * (curl + J);
    }
  }
}

// Decode one region node (z, x, y already inside the domain) into its record.
template <int DIM, int CL, int PR, bool EDGE, class Pull>
__device__ __forceinline__ void decode_node(const StepParams& P, const StepConst<typename Prec<PR>::real>& S,
                                            const Pull& pull, int z, int x, int y, typename Prec<PR>::real* smac,
                                            int NR, int r, typename Prec<PR>::real* scr, int NT) {
  using M = Model<DIM, CL>;
  using real = typename Prec<PR>::real;
  constexpr int K = M::K, Q = Lattice<DIM>::Q;
  real dA[K];
  if constexpr (RollSets<DIM, K>::value) {
    // scr: this thread's shared-memory column (stride NT)
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      real df[Q];
      pull.template get<EDGE>(z, x, y, k, df);
      scr[k * NT] = set_dA<Q, PR>(df, P.inv_scale[k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) dA[k] = scr[k * NT];
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      real df[Q];
      pull.template get<EDGE>(z, x, y, k, df);
      dA[k] = set_dA<Q, PR>(df, P.inv_scale[k]);
    }
  }
  real rec[M::NM];
  decode_record<DIM, CL, real>(P, S, dA, rec);
#pragma unroll
  for (int m = 0; m < M::NM; ++m) smac[m * NR + r] = rec[m];
}

// The three phases of one step for the CTA's tile; `pull` supplies the
// deviations of the pulled populations of a node (global memory or a staged
// shared-memory box).  `smem` holds the records and the E^{n+1/2} slots.
// EDGE = false promises that the tile and its halo lie in the bulk
// (1 <= index <= n-2 on every axis), so no boundary rule applies.
// In 1D and 2D the caller loads the own node's fields (FieldPF) before the
// populations arrive; in 3D, where registers are scarce, they are loaded here
// just before they are used.
// Node h of the 2D decode halo ring (region coordinates rz, rx).
template <int RZ, int RX>
__device__ __forceinline__ void ring_node_2d(int h, int& rz, int& rx) {
  if (h < RZ) { rz = h; rx = 0; }
  else if (h < 2 * RZ) { rz = h - RZ; rx = RX - 1; }
  else { const int j = h - 2 * RZ; rz = (j & 1) ? RZ - 1 : 0; rx = 1 + (j >> 1); }
}

// `after_decode` runs on every thread right after the barrier that ends the
// decode phase: when the own populations stay in registers (K*Q <= 32) the
// pull source is not read again, so a caller may start refilling it there.
template <int DIM> struct EarlyFields { static constexpr bool value = DIM <= 2; };

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// MARCH (3D, TY = 1): the tile is one plane of a column that the caller
// walks up in y, with a barrier after each call.  The region's planes ry =
// 0, 1, 2 are the planes below, at and above the tile.  On the first plane
// (first_plane) the whole region is decoded; on each later plane phase A
// moves the records of planes 1, 2 (and the E slots of plane 1) down one
// plane and decodes only the new top plane, and phase B skips the low face
// ry = 0 (it was the previous plane's own and low-face slots).  A node's
// values are moved and decoded by the same thread, so phase A needs no
// extra barrier.
// AXI (2D): the (z, r) grid of App. A, node j at r = j dx with j = 0 the
// r = 0 boundary node (see pulled_dev, e_slot): B_phi stays 0 on the axis,
// the E_z slot below the axis mirrors the one above it, and the 1/r terms
// of App. A join the sources at r > 0 (left out on the axis, where they
// are singular).
template <int DIM, int CL, int PR, int TZ, int TX, int TY, bool EDGE, class Pull, class Hook = NoHook,
          bool MARCH = false, bool AXI = false>
__device__ __forceinline__ void step_body(const StepParams& P, unsigned char* smem, const Pull& pull,
                                          FieldPF<typename Prec<PR>::real>& F, int tile_z, int tile_x,
                                          int tile_y, const Hook& after_decode = Hook(), bool first_plane = true) {
  static_assert(!MARCH || (DIM == 3 && TY == 1), "marching walks one-plane 3D tiles");
  static_assert(!AXI || DIM == 2, "axisymmetric grids are (z, r)");
  using C = StepCfg<DIM, CL, PR, TZ, TX, TY>;
  using M = Model<DIM, CL>;
  using L = Lattice<DIM>;
  using real = typename Prec<PR>::real;
  using store = typename Prec<PR>::store;
  constexpr int NT = C::NT, RZ = C::RZ, RX = C::RX, RY = C::RY, NR = C::NR;
  constexpr int K = M::K, Q = L::Q;
  constexpr bool KEEP = K * Q <= 32;  // own node's pulled populations stay in registers
  // ... or, for global pulls of wider sets, in shared memory
  constexpr bool SKEEP = C::SKEEP_OK && (std::is_same<Pull, GlobalPull<DIM, CL, PR, true>>::value ||
                                         std::is_same<Pull, GlobalPull<DIM, CL, PR, true, true>>::value);

  const StepConst<real>& S = consts<real>(P);
  real* smac = reinterpret_cast<real*>(smem);  // [NM][NR]
  real* sE = smac + M::NM * NR;                 // [DIM][NR] (+ [DIM][NR] low parts in FP32)
  real* sdrv = sE + C::NE_SLOTS * NR;           // [TZ+1 | TX+1 | TY+1] driver factors
  real* scr = sdrv + C::NDRV + threadIdx.x;     // rolled loops: this thread's column [K] (stride NT)

  const int tid = threadIdx.x;
  const int tz = tid % TZ, tx = (tid / TZ) % TX, ty = tid / (TZ * TX);
  const int gz0 = tile_z * TZ, gx0 = tile_x * TX, gy0 = tile_y * TY;
  const int oz = gz0 - 1, ox = gx0 - (DIM >= 2 ? 1 : 0), oy = gy0 - (DIM >= 3 ? 1 : 0);
  const int pl = (int)P.plane;

  if (!EDGE) {
    // separable driver factors of the slots [oz, oz + TZ] x [ox, ox + TX] x [oy, oy + TY]
    for (int t = tid; t < C::NDRV; t += NT) {
      real v;
      if (t <= TZ) {
        v = driver_long<real>(P, S, real(oz + t) * S.dx - S.zeta0);
      } else if (t <= TZ + 1 + TX) {
        const real x = (real(ox + t - (TZ + 1)) - S.xoff + real(0.5)) * S.dx;
        v = DIM >= 2 ? exp(-x * x * S.inv2sr2) : real(1);
      } else {
        const real y = (real(oy + t - (TZ + 1) - (TX + 1)) - S.yoff + real(0.5)) * S.dx;
        v = DIM >= 3 ? exp(-y * y * S.inv2sr2) : real(1);
      }
      sdrv[t] = v;
    }
  }

  const int gz = gz0 + tz, gx = DIM >= 2 ? gx0 + tx : 0, gy = DIM >= 3 ? gy0 + ty : 0;
  const bool own_inside = !EDGE || (gz < P.n[0] && (DIM < 2 || gx < P.n[1]) && (DIM < 3 || gy < P.n[2]));
  const int r_own = (tz + 1) + RZ * ((DIM >= 2 ? tx + 1 : 0) + RX * (DIM >= 3 ? ty + 1 : 0));

  // 2D bulk tiles: the fields of the low-side halo E slots are copied to
  // shared memory asynchronously now and used in phase B, so their global
  // latency overlaps the decode
  real* sH = sdrv + C::NDRV + C::NSCR;
  real* skeep = sH + C::NSTAGE + tid;  // SKEEP: this thread's column [K*Q] (stride NT)
  if constexpr (DIM == 2 && !EDGE) {
    static_assert(C::NHALO_E <= NT, "one halo slot per thread");
    if (tid < C::NHALO_E) {
      const int rz = tid <= TZ ? tid : 0, rx = tid <= TZ ? 0 : tid - TZ;
      stage_fields_2d<real>(P, cell_index32(P, oz + rz, ox + rx, 0), sH + tid, C::NHALO_E);
    }
    cp_async_commit();
  }

  // ---------------- A: pull + decode of the tile and its halo -------------
  real keep[KEEP ? K * Q : 1];
  real dA_own[K];
  const bool march_on = MARCH && !first_plane;  // continuing plane of a march
  if (!march_on) {
    const int ez = EDGE ? wrap_or_clamp(gz, P.n[0], P.periodic) : gz;
    const int ex = DIM >= 2 ? (EDGE ? wrap_or_clamp(gx, P.n[1], P.periodic) : gx) : 0;
    const int ey = DIM >= 3 ? (EDGE ? wrap_or_clamp(gy, P.n[2], P.periodic) : gy) : 0;
    if constexpr (RollSets<DIM, K>::value) {
      static_assert(!KEEP, "rolled set loops keep no populations in registers");
#pragma unroll 1
      for (int k = 0; k < K; ++k) {
        real df[Q];
        pull.template get<EDGE>(ez, ex, ey, k, df);
        scr[k * NT] = set_dA<Q, PR>(df, P.inv_scale[k]);
      }
#pragma unroll
      for (int k = 0; k < K; ++k) dA_own[k] = scr[k * NT];
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        real df[Q];
        pull.template get<EDGE>(ez, ex, ey, k, df);
        if constexpr (KEEP) {
#pragma unroll
          for (int i = 0; i < Q; ++i) keep[k * Q + i] = df[i];
        } else if constexpr (SKEEP) {
#pragma unroll
          for (int i = 0; i < Q; ++i) skeep[(k * Q + i) * NT] = df[i];
        }
        dA_own[k] = set_dA<Q, PR>(df, P.inv_scale[k]);
      }
    }
    real rec[M::NM];
    decode_record<DIM, CL, real>(P, S, dA_own, rec);
#pragma unroll
    for (int m = 0; m < M::NM; ++m) smac[m * NR + r_own] = rec[m];
    if constexpr (DIM <= 2) {
      // adjoint recording: the moments this step decodes and B^n
      if (P.tape != nullptr && own_inside) {
        real* tp = reinterpret_cast<real*>(P.tape);
        const int id_own = cell_index32(P, gz, gx, gy);
#pragma unroll
        for (int k = 0; k < K; ++k) gst(tp + k * pl + id_own, dA_own[k]);
        if constexpr (DIM == 2) gst(tp + (K + DIM) * pl + id_own, F.Bc[2] + F.Bc_lo[2]);
      }
    }
  }
  {
    // halo ring
    if constexpr (DIM == 2 && C::NXTRA > 0) {
      // 2D WARMC: the ring's set moments are pulled one (node, set) per
      // thread, consecutive threads on consecutive ring nodes of one set, so
      // the 72 pulls of a ring node do not all fall on one thread; the
      // records are decoded after a barrier
      constexpr int NRING = NR - NT;
      static_assert(C::NXTRA == NRING, "one ring split");
      real* ssplit = sH + C::NSTAGE;  // [NRING][K]
      auto ring = [&](int h, int& r, int& z, int& x) {
        int rz, rx;
        ring_node_2d<RZ, RX>(h, rz, rx);
        r = rz + RZ * rx;
        z = oz + rz;
        x = ox + rx;
        if (EDGE) {
          z = wrap_or_clamp(z, P.n[0], P.periodic);
          x = wrap_or_clamp(x, P.n[1], P.periodic);
        }
      };
      for (int u = tid; u < C::NSPLIT; u += NT) {
        const int h = u % NRING, k = u / NRING;
        int r, z, x;
        ring(h, r, z, x);
        real df[Q];
        pull.template get<EDGE>(z, x, 0, k, df);
        ssplit[h * K + k] = set_dA<Q, PR>(df, P.inv_scale[k]);
      }
      __syncthreads();
      for (int h = tid; h < NRING; h += NT) {
        int r, z, x;
        ring(h, r, z, x);
        real dA[K];
#pragma unroll
        for (int k = 0; k < K; ++k) dA[k] = ssplit[h * K + k];
        real rec[M::NM];
        decode_record<DIM, CL, real>(P, S, dA, rec);
#pragma unroll
        for (int m = 0; m < M::NM; ++m) smac[m * NR + r] = rec[m];
      }
    } else if constexpr (DIM <= 2) {
      constexpr int NRING = NR - NT;
      for (int h = tid; h < NRING; h += NT) {
        int rz, rx = 0;
        if constexpr (DIM == 1) rz = h == 0 ? 0 : RZ - 1;
        else ring_node_2d<RZ, RX>(h, rz, rx);
        const int r = rz + RZ * rx;
        int z = oz + rz, x = ox + rx;
        if (EDGE) {
          z = wrap_or_clamp(z, P.n[0], P.periodic);
          if (DIM >= 2) x = wrap_or_clamp(x, P.n[1], P.periodic);
        }
        decode_node<DIM, CL, PR, EDGE>(P, S, pull, z, x, 0, smac, NR, r, scr, NT);
      }
    } else if (march_on) {
      // marching: move the planes down, decode the new top plane.  Its first
      // NT nodes are pulled and decoded by one thread each; the set moments
      // of the rest are pulled one (node, set) per thread across the CTA and
      // decoded after a barrier, so no thread pulls two nodes' sets
      constexpr int PLN = RZ * RX;
      auto top = [&](int j, int& z, int& x, int& y) {
        z = oz + j % RZ, x = ox + j / RZ, y = oy + 2;
        if (EDGE) {
          z = wrap_or_clamp(z, P.n[0], P.periodic);
          x = wrap_or_clamp(x, P.n[1], P.periodic);
          y = wrap_or_clamp(y, P.n[2], P.periodic);
        }
      };
      for (int j = tid; j < PLN; j += NT) {
#pragma unroll 1
        for (int m = 0; m < M::NM; ++m) {
          smac[m * NR + j] = smac[m * NR + PLN + j];
          smac[m * NR + PLN + j] = smac[m * NR + 2 * PLN + j];
        }
#pragma unroll
        for (int a = 0; a < C::NE_SLOTS; ++a) sE[a * NR + j] = sE[a * NR + PLN + j];
        if (C::NXTRA == 0 || j < NT) {
          int z, x, y;
          top(j, z, x, y);
          decode_node<DIM, CL, PR, EDGE>(P, S, pull, z, x, y, smac, NR, 2 * PLN + j, scr, NT);
        }
      }
      if constexpr (C::NXTRA > 0) {
        real* ssplit = sH + C::NSTAGE;  // [NXTRA][K]
#pragma unroll 1
        for (int u = tid; u < C::NSPLIT; u += NT) {
          // consecutive threads take consecutive nodes of one set (coalesced)
          const int jj = u % C::NXTRA, k = u / C::NXTRA, j = NT + jj;
          int z, x, y;
          top(j, z, x, y);
          real df[Q];
          pull.template get<EDGE>(z, x, y, k, df);
          ssplit[jj * K + k] = set_dA<Q, PR>(df, P.inv_scale[k]);
        }
        __syncthreads();
        for (int j = NT + tid; j < PLN; j += NT) {
          real dA[K];
#pragma unroll
          for (int k = 0; k < K; ++k) dA[k] = ssplit[(j - NT) * K + k];
          real rec[M::NM];
          decode_record<DIM, CL, real>(P, S, dA, rec);
#pragma unroll
          for (int m = 0; m < M::NM; ++m) smac[m * NR + 2 * PLN + j] = rec[m];
        }
      }
    } else {
      // 3D: stride over the region and skip the interior
      for (int r = tid; r < NR; r += NT) {
        const int rz = r % RZ, rx = (r / RZ) % RX, ry = r / (RZ * RX);
        if (rz >= 1 && rz <= TZ && rx >= 1 && rx <= TX && ry >= 1 && ry <= TY) continue;
        int z = oz + rz, x = ox + rx, y = oy + ry;
        if (EDGE) {
          z = wrap_or_clamp(z, P.n[0], P.periodic);
          x = wrap_or_clamp(x, P.n[1], P.periodic);
          y = wrap_or_clamp(y, P.n[2], P.periodic);
        }
        decode_node<DIM, CL, PR, EDGE>(P, S, pull, z, x, y, smac, NR, r, scr, NT);
      }
    }
  }
  __syncthreads();
  after_decode();

  // ---------------- B: E^{n+1/2} on the slots of tile + low halo ----------
  if constexpr (!EarlyFields<DIM>::value) {
    if (own_inside) load_fields<DIM, real, EDGE>(P, gz, gx, gy, cell_index32(P, gz, gx, gy), F);
  }
  if (own_inside) e_slot<DIM, CL, PR, TZ, TX, TY, EDGE, AXI>(P, S, smac, sE, sdrv, oz, ox, oy, r_own, gz, gx, gy, F);
  {
    // low-side halo slots: region cells with rz = 0 (or rx = 0, ry = 0) in
    // [0, TZ] x [0, TX] x [0, TY]
    constexpr int SZ = TZ + 1, SX = DIM >= 2 ? TX + 1 : 1, SY = DIM >= 3 ? TY + 1 : 1;
    constexpr int NHALO = DIM == 3 ? SZ * SX * SY : SZ * SX * SY - TZ * (DIM >= 2 ? TX : 1);
    for (int h = tid; h < NHALO; h += NT) {
      int rz = 0, rx = 0, ry = 0;
      if constexpr (DIM == 1) {
        rz = 0;
      } else if constexpr (DIM == 2) {
        if (h < SZ) { rz = h; rx = 0; } else { rz = 0; rx = h - SZ + 1; }
      } else {
        // 3D: stride over the slot box and skip everything but the low faces
        rz = h % SZ; rx = (h / SZ) % SX; ry = h / (SZ * SX);
        if (rz != 0 && rx != 0 && ry != 0) continue;
        if (march_on && ry == 0) continue;  // carried over from the previous plane
      }
      const int r = rz + RZ * (rx + RX * ry);
      int e0 = oz + rz, e1 = ox + rx, e2 = oy + ry;
      int r_eff = r;
      if (EDGE) {
        if (P.periodic) {
          e0 = wrap_or_clamp(e0, P.n[0], 1);
          if (DIM >= 2) e1 = wrap_or_clamp(e1, P.n[1], 1);
          if (DIM >= 3) e2 = wrap_or_clamp(e2, P.n[2], 1);
        } else {
          // transverse ghost: conducting wall; z ghost: the nearest slot;
          // below the axis (AXI): the mirror image of the slot above it
          if (AXI && e1 < 0) { r_eff += RZ; e1 = 0; }
          const bool trans_out = (DIM >= 2 && (e1 < 0 || e1 >= P.n[1])) || (DIM >= 3 && (e2 < 0 || e2 >= P.n[2]));
          if (trans_out) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
              if (e_present<DIM>(a)) {
                sE[a * NR + r] = real(0);
                if (C::CF) sE[(C::NEC + a) * NR + r] = real(0);
              }
            continue;
          }
          if (e0 < 0) { r_eff += 1; e0 = 0; }
          if (e0 >= P.n[0]) continue;  // never read
        }
      }
      const int id = cell_index32(P, e0, e1, e2);
      FieldPF<real> G;
      if constexpr (DIM == 2 && !EDGE) {
        cp_async_wait_all();
        fields_2d_from_stage<real>(sH + h, C::NHALO_E, G);
      } else {
        load_fields<DIM, real, EDGE>(P, e0, e1, e2, id, G);
      }
      e_slot<DIM, CL, PR, TZ, TX, TY, EDGE, AXI>(P, S, smac, sE, sdrv, oz, ox, oy, r_eff, e0, e1, e2, G);
      if (r_eff != r) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (e_present<DIM>(a)) {
            // below the axis E_r (never read there) is zero
            const bool zero = AXI && a == 1 && r_eff - r >= RZ;
            sE[a * NR + r] = zero ? real(0) : sE[a * NR + r_eff];
            if (C::CF) sE[(C::NEC + a) * NR + r] = zero ? real(0) : sE[(C::NEC + a) * NR + r_eff];
          }
      }
    }
  }
  __syncthreads();

  // ---------------- C: per tile node ------------------------------------
  if (!own_inside) return;
  const int r = r_own;
  const int id = cell_index32(P, gz, gx, gy);
  const real dt = S.dt;

  real* Eout = reinterpret_cast<real*>(P.Eout);
  real* Bout = reinterpret_cast<real*>(P.Bout);
  real En[3] = {0, 0, 0}, Bn[3] = {0, 0, 0};
  real* tape = reinterpret_cast<real*>(P.tape);
  real* Eout_lo = reinterpret_cast<real*>(P.Eout_lo);
  real* Bout_lo = reinterpret_cast<real*>(P.Bout_lo);
  // E slot value (high + low in FP32)
  auto Ev = [&](int a, int rr) -> real { return C::CF ? sE[a * NR + rr] + sE[(C::NEC + a) * NR + rr] : sE[a * NR + rr]; };
  auto Ed = [&](int a, int r1, int r2) -> real {
    return C::CF ? diff2(sE[a * NR + r1], sE[(C::NEC + a) * NR + r1], sE[a * NR + r2], sE[(C::NEC + a) * NR + r2])
                 : sE[a * NR + r1] - sE[a * NR + r2];
  };
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (e_present<DIM>(a)) {
      gst(Eout + a * pl + id, sE[a * NR + r]);
      if (C::CF) gst(Eout_lo + a * pl + id, sE[(C::NEC + a) * NR + r]);
      if (DIM <= 2 && tape != nullptr) gst(tape + (K + a) * pl + id, Ev(a, r));
      const int b = (a + 1) % 3, d = (a + 2) % 3;
      const bool ob = axis_present<DIM>(b), od = axis_present<DIM>(d);
      const int sb = ob ? C::stride(b) : 0, sd = od ? C::stride(d) : 0;
      const int nb = ob ? 2 : 1, nd = od ? 2 : 1;
      real s = 0;
#pragma unroll
      for (int jb = 0; jb < 2; ++jb)
#pragma unroll
        for (int jd = 0; jd < 2; ++jd)
          if (jb < nb && jd < nd) s += Ev(a, r - jb * sb - jd * sd);
      En[a] = s * (real(1) / real(nb * nd));
    }
    if (b_present<DIM>(a)) {
      const real bo = F.Bc[a] + F.Bc_lo[a];
      Bn[a] = axis_present<DIM>(a) ? real(0.5) * (bo + (F.Bm[a] + F.Bm_lo[a])) : bo;
      const int b = (a + 1) % 3, d = (a + 2) % 3;
      real curl = 0;
      if (axis_present<DIM>(b) && e_present<DIM>(d)) curl += Ed(d, r, r - C::stride(b)) * S.idx;
      if (axis_present<DIM>(d) && e_present<DIM>(b)) curl -= Ed(b, r, r - C::stride(d)) * S.idx;
      if (AXI && gx == 0) {
        // B_phi vanishes on the axis
        gst(Bout + a * pl + id, real(0));
        if constexpr (C::CF) gst(Bout_lo + a * pl + id, real(0));
      } else if constexpr (C::CF) {
        real hi = F.Bc[a], lo = F.Bc_lo[a];
        two_float_add(hi, lo, -(dt * curl));
        gst(Bout + a * pl + id, hi);
        gst(Bout_lo + a * pl + id, lo);
      } else {
        gst(Bout + a * pl + id, F.Bc[a] - dt * curl);
      }
    }
  }

  const real n = smac[M::R_N * NR + r];
  real u[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < DIM; ++a) u[a] = smac[(M::R_U + a) * NR + r];
  real uxB[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    real s = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l)
        if (levi(a, k, l) != 0) s += real(levi(a, k, l)) * u[k] * Bn[l];
    uxB[a] = s;
  }

  // Sources of each advected scalar (Eq. lb-ade-lec-comps-F,
  // lb-ade-warmc-comps-F with App. A), evaluated per set inside the collide
  // loop so that only their inputs stay live.
  real th[3][3], th0[3] = {0, 0, 0}, gw[3][3], divth[3] = {0, 0, 0};
  real dth00 = 0, dth0[3] = {0, 0, 0}, dw[3] = {0, 0, 0}, divth0 = 0, Eu = 0;
  if constexpr (CL == CL_WARMC) {
    real* prev = reinterpret_cast<real*>(P.prev);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int j = M::thidx(a, b);
        th[a][b] = j >= 0 ? S.threst[j] + smac[(M::R_TH + j) * NR + r] : real(0);
      }
    real w[3] = {0, 0, 0};
    const real lam = smac[M::R_LAM * NR + r];
#pragma unroll
    for (int a = 0; a < DIM; ++a) { th0[a] = smac[(M::R_TH0 + a) * NR + r]; w[a] = lam * u[a]; }
    real th00 = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) th00 += u[a] * th0[a];
    // backward time differences (zero on the first step after a reset)
    if (P.have_prev) {
      const real idt = S.idt;
      dth00 = (th00 - gldc(prev + id)) * idt;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        dth0[a] = (th0[a] - gldc(prev + (1 + a) * pl + id)) * idt;
        dw[a] = (w[a] - gldc(prev + (1 + DIM + a) * pl + id)) * idt;
      }
    }
    gst(prev + id, th00);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      gst(prev + (1 + a) * pl + id, th0[a]);
      gst(prev + (1 + DIM + a) * pl + id, w[a]);
    }
    // spatial gradients from the neighbours' records; gw[a][k] = d_k w^a
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) gw[a][k] = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const int rp = r + C::stride(k), rm = r - C::stride(k);
      const real lp = smac[M::R_LAM * NR + rp], lm = smac[M::R_LAM * NR + rm];
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        gw[a][k] = (lp * smac[(M::R_U + a) * NR + rp] - lm * smac[(M::R_U + a) * NR + rm]) * S.i2dx;
      divth0 += (smac[(M::R_TH0 + k) * NR + rp] - smac[(M::R_TH0 + k) * NR + rm]) * S.i2dx;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int j = M::thidx(a, k);
        if (j >= 0) divth[a] += (smac[(M::R_TH + j) * NR + rp] - smac[(M::R_TH + j) * NR + rm]) * S.i2dx;
      }
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) Eu += En[a] * u[a];
  }
  auto source = [&](int k) -> real {
    if (k == 0) return real(0);
    if constexpr (CL == CL_LEC) {
      const int a = k - 1;
      const real gPi = (smac[M::R_PI * NR + r + C::stride(a)] - smac[M::R_PI * NR + r - C::stride(a)]) * S.i2dx;
      return -S.mu * gPi - n * (En[a] + uxB[a]);
    } else {
      if (k == 1) return -dth00 - divth0 - n * Eu;
      if (k < 2 + DIM) {
        const int a = k - 2;
        return -dth0[a] - divth[a] - n * (En[a] + uxB[a]);
      }
      const int j = k - 2 - DIM;
      const int a = M::tha(j), b = M::thb(j);
      real sv = -th0[b] * dw[a] - th0[a] * dw[b];
#pragma unroll
      for (int q = 0; q < DIM; ++q) sv -= th[b][q] * gw[a][q] + th[a][q] * gw[b][q];
      real em = En[a] * th0[b] + En[b] * th0[a];
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          if (levi(a, q, l) != 0) em += real(levi(a, q, l)) * th[b][q] * Bn[l];
          if (levi(b, q, l) != 0) em += real(levi(b, q, l)) * th[a][q] * Bn[l];
        }
      return sv - em;
    }
  };

  // AXI: the 1/r terms of the cylindrical divergence of App. A (r = x,
  // phi = y, c = 1), written with the set's advected value A_k: -A_k u_r / r
  // for every set (3 A_k u_r / r for lambda theta^{phi phi}), plus
  // theta^{0r} / r (n lambda), theta^{rz} / r (n lambda u_z) and
  // (theta^{rr} - theta^{phi phi}) / r (n lambda u_r); zero on the axis.
  real ir = 0;
  if constexpr (AXI) ir = gx > 0 ? S.idx / real(gx) : real(0);
  auto geo = [&](int k, real A) -> real {
    if constexpr (CL == CL_LEC) {
      return -u[1] * A * ir;
    } else {
      real cf = real(1), extra = real(0);
      if (k == 1) extra = th0[1];
      else if (k == 2) extra = th[0][1];
      else if (k == 3) extra = th[1][1] - th[2][2];
      else if (k >= 2 + DIM && M::tha(k - 2 - DIM) == 2 && M::thb(k - 2 - DIM) == 2) cf = real(3);
      return -(cf * A * u[1] + extra) * ir;
    }
  };

  // ---------------- collide + store (deviation form) ----------------------
  // f* - w A_rest = df (1 - 1/tau) + (f^eq - w A_rest)/tau + w dt F, with
  // f^eq - w A_rest = w (dA + A P_i), P_i = 3 cu + 9/2 cu^2 - 3/2 u^2 split
  // into its even and odd parts over each pair of opposite velocities.
  // The moving populations are stored first; the rest population takes the
  // remainder of the set's post-collision moment dA + dt F (Eq. lbe with
  // sum_i w_i = 1, sum_i w_i P_i = 0), summed over the values as stored.  In
  // reduced precision the rounded weights sum to 1 + O(eps), and the direct
  // form would scale every moment deviation by 1 + O(eps)/tau each step.
  static_assert(opposite_pairs<DIM>(), "lattice order must pair opposite velocities");
  real ul[3] = {0, 0, 0};
  real usq = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) { ul[a] = S.courant * u[a]; usq += ul[a] * ul[a]; }
  const real itau = S.inv_tau, omt = real(1) - S.inv_tau;
  const real base = real(-1.5) * usq;
  store* fout = reinterpret_cast<store*>(P.fout);
  // 1D/2D: the equilibrium's set-independent factors of each pair of
  // opposite velocities, with 1/tau folded in, formed once per node:
  // Ef = w (base + 9/2 cu^2) / tau, Of = 3 w cu / tau; then per set and pair
  // f*_i - w A_rest = df_i (1 - 1/tau) + w (dA/tau + dt F) + A Ef +- A Of.
  // 3D (rolled set loop, registers scarce) forms them per set.
  constexpr int NP = (Q - 1) / 2;
  constexpr bool PRE = DIM <= 2;
  real Ef[PRE ? NP : 1], Of[PRE ? NP : 1];
  if constexpr (PRE) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const int i = 1 + 2 * q;
      real cu = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) cu += real(L::c(i, a)) * ul[a];
      const real wi = real(L::w(i));
      Ef[q] = (wi * (base + real(4.5) * cu * cu)) * itau;
      Of[q] = ((real(3) * wi) * cu) * itau;
    }
  }
  // one population set: pull (or the kept values), relax, store; the source
  // dt F_k is evaluated after the pull (dtF_of), as in a plain loop body
  auto collide_set = [&](int k, real Arest_k, float sc, float isc, auto dtF_of) {
    real df[Q];
    real dA;
    if constexpr (KEEP) {
#pragma unroll
      for (int i = 0; i < Q; ++i) df[i] = keep[k * Q + i];
      dA = dA_own[k];
    } else if constexpr (SKEEP) {
#pragma unroll
      for (int i = 0; i < Q; ++i) df[i] = skeep[(k * Q + i) * NT];
      dA = dA_own[k];
    } else {
      pull.template get<EDGE>(gz, gx, gy, k, df);
      dA = set_dA<Q, PR>(df, isc);
    }
    const real A = Arest_k + dA;
    real dtF = dtF_of();
    if constexpr (AXI) dtF += dt * geo(k, A);
    store* fk = fout + (size_t)k * Q * (size_t)P.plane;
    // df and the stored values are in storage units; us = s_k (FP16S) scales
    // the equilibrium and source parts into them (exactly: a power of two)
    const real us = Codec<PR>::kScaled ? real(sc) : real(1);
    Remainder<PR, real> moved;
    if constexpr (PRE) {
      const real As = A * us;
      const real gs = (dA * itau + dtF) * us;
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const int i = 1 + 2 * q, j = i + 1;
        const real evw = As * Ef[q] + real(L::w(i)) * gs;
        const real odd = As * Of[q];
        moved.add(Codec<PR>::store_qu(fk, i * pl + id, df[i] * omt + (evw + odd)));
        moved.add(Codec<PR>::store_qu(fk, j * pl + id, df[j] * omt + (evw - odd)));
      }
    } else {
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const int i = 1 + 2 * q, j = i + 1;
        real cu = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) cu += real(L::c(i, a)) * ul[a];
        const real wi = real(L::w(i));
        const real even = (wi * (dA + A * (base + real(4.5) * cu * cu))) * us;
        const real odd = ((real(3) * wi) * A * cu) * us;
        const real wF = (wi * dtF) * us;
        moved.add(Codec<PR>::store_qu(fk, i * pl + id, df[i] * omt + (even + odd) * itau + wF));
        moved.add(Codec<PR>::store_qu(fk, j * pl + id, df[j] * omt + (even - odd) * itau + wF));
      }
    }
    Codec<PR>::store0_u(fk, id, fout + ((size_t)K * Q + k) * (size_t)P.plane, id, moved.rest(dA, dtF, us));
  };
  if constexpr (RollSets<DIM, K>::value) {
    // the sources first, into this thread's shared-memory column; the
    // rolled loop reads them, and the per-set constants from the launch
    // parameters (grid constants)
#pragma unroll
    for (int k = 0; k < K; ++k) scr[k * NT] = dt * source(k);
#pragma unroll 1
    for (int k = 0; k < K; ++k) collide_set(k, S.Arest[k], P.scale[k], P.inv_scale[k], [&] { return scr[k * NT]; });
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) collide_set(k, S.Arest[k], P.scale[k], P.inv_scale[k], [&] { return dt * source(k); });
  }
}

// 3D launch order of the tiles: z-tiles fastest, then the (x, y) tiles in
// strips W rows high in y (x, then y within a strip), so the CTAs resident at
// one time cover a compact patch and read their x and y neighbours' halos
// while those are still in L2 (row by row, the y-neighbours of a row of
// tiles came several waves later).
template <int W>
__device__ __forceinline__ void tile_order_3d(int& bz, int& bx, int& by) {
  const int ntz = gridDim.x, ntx = gridDim.y, nty = gridDim.z;
  const int lin = blockIdx.x + ntz * (blockIdx.y + ntx * blockIdx.z);
  bz = lin % ntz;
  const int rest = lin / ntz;
  const int strip = rest / (ntx * W);
  const int y0 = strip * W;
  const int h = min(W, nty - y0);
  const int q = rest - strip * ntx * W;
  bx = q / h;
  by = y0 + q % h;
}

// Whether the tile and its one-node halo lie in the bulk on every axis.
template <int DIM, int TZ, int TX, int TY>
__device__ __forceinline__ bool tile_is_bulk(const StepParams& P, int tile_z, int tile_x, int tile_y) {
  const int gz0 = tile_z * TZ, gx0 = tile_x * TX, gy0 = tile_y * TY;
  bool bulk = gz0 - 1 >= 1 && gz0 + TZ <= P.n[0] - 2;
  if (DIM >= 2) bulk = bulk && gx0 - 1 >= 1 && gx0 + TX <= P.n[1] - 2;
  if (DIM >= 3) bulk = bulk && gy0 - 1 >= 1 && gy0 + TY <= P.n[2] - 2;
  return bulk;
}

// Own node's field prefetch (coordinates of a ragged tile's idle threads are
// clamped so every load stays inside the arrays).
template <int DIM, typename real, bool EDGE, int TZ, int TX, int TY>
__device__ __forceinline__ void prefetch_own(const StepParams& P, FieldPF<real>& F, int tile_z, int tile_x,
                                             int tile_y) {
  const int tid = threadIdx.x;
  int gz = tile_z * TZ + tid % TZ;
  int gx = DIM >= 2 ? tile_x * TX + (tid / TZ) % TX : 0;
  int gy = DIM >= 3 ? tile_y * TY + tid / (TZ * TX) : 0;
  if (EDGE) {
    gz = min(gz, P.n[0] - 1);
    if (DIM >= 2) gx = min(gx, P.n[1] - 1);
    if (DIM >= 3) gy = min(gy, P.n[2] - 1);
  }
  load_fields<DIM, real, EDGE>(P, gz, gx, gy, cell_index32(P, gz, gx, gy), F);
}

// Plain variant: populations pulled straight from global memory (any
// dimension, open or periodic boundaries).
// Resident CTAs the register budget of the plain kernel is held to: the 2D
// WARMC in reduced precision runs three per SM (85 registers), which hides
// more of its pull latency than two with its 72 own populations kept in
// shared memory (1024 x 512, FP32: 5.94 against 5.67 GLUPS).  0 leaves the
// budget to the compiler, as a bound without a block count does (writing 1
// instead changes its register choice: FP64 2D WARMC 181 -> 255).
template <int DIM, int CL, int PR>
struct PlainMinBlocks {
  static constexpr int value = (DIM == 2 && CL == CL_WARMC && PR != PR_F64) ? 3 : 0;
};

template <int DIM, int CL, int PR, int TZ, int TX, int TY>
__global__ void __launch_bounds__(TZ* TX* TY, (PlainMinBlocks<DIM, CL, PR>::value))
lb_step_kernel(const __grid_constant__ StepParams P) {
  using real = typename Prec<PR>::real;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GlobalPull<DIM, CL, PR, StepCfg<DIM, CL, PR, TZ, TX, TY>::SKEEP_OK> pull{P};
  FieldPF<real> F;
  int bz = blockIdx.x, bx = blockIdx.y, by = blockIdx.z;
  if constexpr (DIM == 3) tile_order_3d<3>(bz, bx, by);
  if (tile_is_bulk<DIM, TZ, TX, TY>(P, bz, bx, by)) {
    if constexpr (EarlyFields<DIM>::value) prefetch_own<DIM, real, false, TZ, TX, TY>(P, F, bz, bx, by);
    step_body<DIM, CL, PR, TZ, TX, TY, false>(P, smem_raw, pull, F, bz, bx, by);
  } else {
    if constexpr (EarlyFields<DIM>::value) prefetch_own<DIM, real, true, TZ, TX, TY>(P, F, bz, bx, by);
    step_body<DIM, CL, PR, TZ, TX, TY, true>(P, smem_raw, pull, F, bz, bx, by);
  }
}

// Axisymmetric (z, r) step: the plain 2D kernel with the AXI rules of
// step_body (r = 0 boundary node, cylindrical curl and 1/r sources).
template <int CL, int PR, int TZ, int TX>
__global__ void __launch_bounds__(TZ* TX, (PlainMinBlocks<2, CL, PR>::value))
lb_step_axi_kernel(const __grid_constant__ StepParams P) {
  using real = typename Prec<PR>::real;
  using Pull = GlobalPull<2, CL, PR, StepCfg<2, CL, PR, TZ, TX, 1>::SKEEP_OK, true>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Pull pull{P};
  FieldPF<real> F;
  const int bz = blockIdx.x, bx = blockIdx.y;
  if (tile_is_bulk<2, TZ, TX, 1>(P, bz, bx, 0)) {
    prefetch_own<2, real, false, TZ, TX, 1>(P, F, bz, bx, 0);
    step_body<2, CL, PR, TZ, TX, 1, false, Pull, NoHook, false, true>(P, smem_raw, pull, F, bz, bx, 0);
  } else {
    prefetch_own<2, real, true, TZ, TX, 1>(P, F, bz, bx, 0);
    step_body<2, CL, PR, TZ, TX, 1, true, Pull, NoHook, false, true>(P, smem_raw, pull, F, bz, bx, 0);
  }
}

// 3D step marching a column of TZ x TX nodes up a chunk of YC planes (the
// MARCH mode of step_body): each node is decoded about (TZ + 2)(TX + 2) /
// (TZ TX) times, not the 2.4 times of a 32 x 4 x 4 tile, and the planes
// above and below come from shared memory instead of being pulled again by
// another tile.  Grid: (z tiles, x tiles, chunks of YC planes).
template <int CL, int PR, int TZ, int TX, int YC>
__global__ void __launch_bounds__(TZ* TX) lb_step_march3d_kernel(const __grid_constant__ StepParams P) {
  using real = typename Prec<PR>::real;
  using Pull = GlobalPull<3, CL, PR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Pull pull{P};
  FieldPF<real> F;
  const int bz = blockIdx.x, bx = blockIdx.y;
  const int y0 = blockIdx.z * YC, y1 = min(y0 + YC, P.n[2]);
  for (int y = y0; y < y1; ++y) {
    if (tile_is_bulk<3, TZ, TX, 1>(P, bz, bx, y))
      step_body<3, CL, PR, TZ, TX, 1, false, Pull, NoHook, true>(P, smem_raw, pull, F, bz, bx, y, NoHook(), y == y0);
    else
      step_body<3, CL, PR, TZ, TX, 1, true, Pull, NoHook, true>(P, smem_raw, pull, F, bz, bx, y, NoHook(), y == y0);
    __syncthreads();  // the next plane moves the records other threads read
  }
}

}  // namespace lbp
