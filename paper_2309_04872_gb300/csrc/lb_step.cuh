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

#include "lb_common.cuh"

namespace lbp {

__host__ __device__ constexpr int levi(int i, int j, int k) {
  return (i == j || j == k || i == k) ? 0
       : (((i == 0 && j == 1) || (i == 1 && j == 2) || (i == 2 && j == 0)) ? 1 : -1);
}

template <int DIM, int CL, int PR, int TZ, int TX, int TY>
struct StepCfg {
  using M = Model<DIM, CL>;
  using real = typename Prec<PR>::real;
  static constexpr int NT = TZ * TX * TY;
  static constexpr int RZ = TZ + 2;
  static constexpr int RX = DIM >= 2 ? TX + 2 : 1;
  static constexpr int RY = DIM >= 3 ? TY + 2 : 1;
  static constexpr int NR = RZ * RX * RY;
  static constexpr size_t smem_bytes = (size_t)(M::NM + 3) * NR * sizeof(real);
  __host__ __device__ static constexpr int stride(int a) { return a == 0 ? 1 : (a == 1 ? RZ : RZ * RX); }
};

// Deviations of the pulled populations f^n_ki - w_i A_rest,k at node
// (z, x, y) (already inside the domain), straight from global memory.
template <int DIM, int CL, int PR>
__device__ __forceinline__ void pulled_dev(const StepParams& P, int z, int x, int y, int k,
                                           typename Prec<PR>::real* df) {
  using L = Lattice<DIM>;
  using store = typename Prec<PR>::store;
  if (!P.periodic) {
    z = min(max(z, 1), P.n[0] - 2);
    if (DIM >= 2) x = min(max(x, 1), P.n[1] - 2);
    if (DIM >= 3) y = min(max(y, 1), P.n[2] - 2);
  }
  const store* f = (const store*)P.fin + (size_t)k * L::Q * (size_t)P.plane;
  const float is = P.inv_scale[k];
  const int pl = (int)P.plane;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    int sz = z - L::c(i, 0), sx = x - L::c(i, 1), sy = y - L::c(i, 2);
    if (P.periodic) {
      sz = sz < 0 ? sz + P.n[0] : (sz >= P.n[0] ? sz - P.n[0] : sz);
      if (DIM >= 2) sx = sx < 0 ? sx + P.n[1] : (sx >= P.n[1] ? sx - P.n[1] : sx);
      if (DIM >= 3) sy = sy < 0 ? sy + P.n[2] : (sy >= P.n[2] ? sy - P.n[2] : sy);
    }
    df[i] = Codec<PR>::load(f, i * pl + cell_index32(P, sz, sx, sy), is);
  }
}

// Population source reading the stored post-collision array in global memory
// (any boundary rule).
template <int DIM, int CL, int PR>
struct GlobalPull {
  const StepParams& P;
  __device__ __forceinline__ void operator()(int z, int x, int y, int k, typename Prec<PR>::real* df) const {
    pulled_dev<DIM, CL, PR>(P, z, x, y, k, df);
  }
};

// Decode the record of one node from its deviation moments dA[K].
template <int DIM, int CL, typename real>
__device__ __forceinline__ void decode_record(const StepParams& P, const StepConst<real>& S, const real* dA,
                                              real* rec) {
  using M = Model<DIM, CL>;
  if constexpr (CL == CL_LEC) {
    real n = real(1) + dA[0];
    real Ap[DIM], u[DIM], Pi;
#pragma unroll
    for (int a = 0; a < DIM; ++a) Ap[a] = dA[1 + a];
    decode_lec<DIM, real>(n, Ap, S.cH, P.D, u, Pi);
    rec[M::R_N] = n;
#pragma unroll
    for (int a = 0; a < DIM; ++a) rec[M::R_U + a] = u[a];
    rec[M::R_PI] = Pi;
  } else {
    const real n = real(1) + dA[0];
    const real nl = S.Arest[1] + dA[1];
    const real inl = real(1) / nl;
    const real lam = nl / n;
    const real ilam = n * inl;
    real u[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) u[a] = dA[2 + a] * inl;
    real th[M::NTH];
#pragma unroll
    for (int j = 0; j < M::NTH; ++j) th[j] = (S.Arest[2 + DIM + j] + dA[2 + DIM + j]) * ilam;
    rec[M::R_N] = n;
    rec[M::R_LAM] = lam;
#pragma unroll
    for (int a = 0; a < DIM; ++a) rec[M::R_U + a] = u[a];
#pragma unroll
    for (int j = 0; j < M::NTH; ++j) rec[M::R_TH + j] = th[j];
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

// The three phases of one step for the CTA's tile; `pull` supplies the
// deviations of the pulled populations of a node (global memory or a staged
// shared-memory box).  `smem` holds the records and the E^{n+1/2} slots.
template <int DIM, int CL, int PR, int TZ, int TX, int TY, class Pull>
__device__ __forceinline__ void step_body(const StepParams& P, unsigned char* smem, const Pull& pull) {
  using C = StepCfg<DIM, CL, PR, TZ, TX, TY>;
  using M = Model<DIM, CL>;
  using L = Lattice<DIM>;
  using real = typename Prec<PR>::real;
  using store = typename Prec<PR>::store;
  constexpr int NT = C::NT, RZ = C::RZ, RX = C::RX, NR = C::NR;
  constexpr int K = M::K, Q = L::Q;
  constexpr bool KEEP = K * Q <= 32;  // own node's pulled populations stay in registers

  const StepConst<real>& S = consts<real>(P);
  real* smac = reinterpret_cast<real*>(smem);  // [NM][NR]
  real* sE = smac + M::NM * NR;                 // [3][NR]

  const int tid = threadIdx.x;
  const int tz = tid % TZ, tx = (tid / TZ) % TX, ty = tid / (TZ * TX);
  const int gz0 = blockIdx.x * TZ, gx0 = blockIdx.y * TX, gy0 = blockIdx.z * TY;
  const int oz = gz0 - 1, ox = gx0 - (DIM >= 2 ? 1 : 0), oy = gy0 - (DIM >= 3 ? 1 : 0);
  const real dt = S.dt, idx_ = S.idx, i2dx = S.i2dx;
  const int pl = (int)P.plane;
  const real* Ein = reinterpret_cast<const real*>(P.Ein);
  const real* Bin = reinterpret_cast<const real*>(P.Bin);

  // own node (ragged tiles: nodes past the domain still decode a clamped copy)
  const int gz = gz0 + tz, gx = DIM >= 2 ? gx0 + tx : 0, gy = DIM >= 3 ? gy0 + ty : 0;
  const bool own_inside = gz < P.n[0] && (DIM < 2 || gx < P.n[1]) && (DIM < 3 || gy < P.n[2]);
  const int r_own = (tz + 1) + RZ * ((DIM >= 2 ? tx + 1 : 0) + RX * (DIM >= 3 ? ty + 1 : 0));

  // ---------------- A: pull + decode of the tile and its halo -------------
  real keep[KEEP ? K * Q : 1];
  real dA_own[K];
  {
    const int ez = wrap_or_clamp(gz, P.n[0], P.periodic);
    const int ex = DIM >= 2 ? wrap_or_clamp(gx, P.n[1], P.periodic) : 0;
    const int ey = DIM >= 3 ? wrap_or_clamp(gy, P.n[2], P.periodic) : 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      real df[Q];
      pull(ez, ex, ey, k, df);
      real s = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        s += df[i];
        if constexpr (KEEP) keep[k * Q + i] = df[i];
      }
      dA_own[k] = s;
    }
    real rec[M::NM];
    decode_record<DIM, CL, real>(P, S, dA_own, rec);
#pragma unroll
    for (int m = 0; m < M::NM; ++m) smac[m * NR + r_own] = rec[m];
  }
  for (int r = tid; r < NR; r += NT) {
    const int rz = r % RZ, rx = (r / RZ) % RX, ry = r / (RZ * RX);
    const bool interior = rz >= 1 && rz <= TZ && (DIM < 2 || (rx >= 1 && rx <= TX)) &&
                          (DIM < 3 || (ry >= 1 && ry <= TY));
    if (interior) continue;
    const int ez = wrap_or_clamp(oz + rz, P.n[0], P.periodic);
    const int ex = DIM >= 2 ? wrap_or_clamp(ox + rx, P.n[1], P.periodic) : 0;
    const int ey = DIM >= 3 ? wrap_or_clamp(oy + ry, P.n[2], P.periodic) : 0;
    real dA[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      real df[Q];
      pull(ez, ex, ey, k, df);
      real s = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) s += df[i];
      dA[k] = s;
    }
    real rec[M::NM];
    decode_record<DIM, CL, real>(P, S, dA, rec);
#pragma unroll
    for (int m = 0; m < M::NM; ++m) smac[m * NR + r] = rec[m];
  }
  __syncthreads();

  // ---------------- B: E^{n+1/2} on the slots of tile + low halo ----------
  {
    constexpr int SZ = TZ + 1, SX = DIM >= 2 ? TX + 1 : 1, SY = DIM >= 3 ? TY + 1 : 1;
    for (int q = tid; q < SZ * SX * SY; q += NT) {
      const int rz = q % SZ, rx = (q / SZ) % SX, ry = q / (SZ * SX);
      const int r = rz + RZ * (rx + RX * ry);
      const int g0 = oz + rz, g1 = ox + rx, g2 = oy + ry;
      const bool inside = g0 >= 0 && g0 < P.n[0] && (DIM < 2 || (g1 >= 0 && g1 < P.n[1])) &&
                          (DIM < 3 || (g2 >= 0 && g2 < P.n[2]));
      if (!inside && !P.periodic) continue;  // ghost, filled below
      const int e0 = wrap_or_clamp(g0, P.n[0], 1);
      const int e1 = DIM >= 2 ? wrap_or_clamp(g1, P.n[1], 1) : 0;
      const int e2 = DIM >= 3 ? wrap_or_clamp(g2, P.n[2], 1) : 0;
      const int e[3] = {e0, e1, e2};
      const int id = cell_index32(P, e0, e1, e2);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (!e_present<DIM>(a)) continue;
        const int b = (a + 1) % 3, d = (a + 2) % 3;
        bool wall = false;
        if (!P.periodic) {
          if (b >= 1 && axis_present<DIM>(b) && e[b] == P.n[b] - 1) wall = true;
          if (d >= 1 && axis_present<DIM>(d) && e[d] == P.n[d] - 1) wall = true;
        }
        if (wall) { sE[a * NR + r] = real(0); continue; }
        real curl = 0;
        if (axis_present<DIM>(b) && b_present<DIM>(d)) {
          const int nb = wrap_or_clamp(e[b] + 1, P.n[b], P.periodic);
          const int id2 = id + (nb - e[b]) * P.axis_stride[b];
          curl += (Bin[d * pl + id2] - Bin[d * pl + id]) * idx_;
        }
        if (axis_present<DIM>(d) && b_present<DIM>(b)) {
          const int nb = wrap_or_clamp(e[d] + 1, P.n[d], P.periodic);
          const int id2 = id + (nb - e[d]) * P.axis_stride[d];
          curl -= (Bin[b * pl + id2] - Bin[b * pl + id]) * idx_;
        }
        // n u_a averaged over the nodes around the slot
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
          const real zeta = real(e0) * S.dx - S.zeta0;
          real nbv = driver_long<real>(P, S, zeta);
          if (DIM >= 2) {
            const real x = (real(e1) - S.xoff + real(0.5)) * S.dx;
            real r2 = x * x;
            if (DIM >= 3) {
              const real y = (real(e2) - S.yoff + real(0.5)) * S.dx;
              r2 += y * y;
            }
            nbv *= exp(-r2 * S.inv2sr2);
          }
          J += nbv;
        }
        sE[a * NR + r] = Ein[a * pl + id] + dt * (curl + J);
      }
    }
  }
  __syncthreads();
  if (!P.periodic) {
    // low-side ghosts: transverse -> conducting wall (0); z -> nearest slot
    constexpr int SZ = TZ + 1, SX = DIM >= 2 ? TX + 1 : 1, SY = DIM >= 3 ? TY + 1 : 1;
    for (int q = tid; q < SZ * SX * SY; q += NT) {
      const int rz = q % SZ, rx = (q / SZ) % SX, ry = q / (SZ * SX);
      const int r = rz + RZ * (rx + RX * ry);
      const int g0 = oz + rz, g1 = ox + rx, g2 = oy + ry;
      bool trans_out = false;
      if (DIM >= 2) trans_out = trans_out || g1 < 0 || g1 >= P.n[1];
      if (DIM >= 3) trans_out = trans_out || g2 < 0 || g2 >= P.n[2];
      if (trans_out) {
#pragma unroll
        for (int a = 0; a < 3; ++a) if (e_present<DIM>(a)) sE[a * NR + r] = real(0);
      } else if (g0 < 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) if (e_present<DIM>(a)) sE[a * NR + r] = sE[a * NR + r + 1];
      }
    }
    __syncthreads();
  }

  // ---------------- C: per tile node ------------------------------------
  if (!own_inside) return;
  const int r = r_own;
  const int id = cell_index32(P, gz, gx, gy);
  const int e[3] = {gz, gx, gy};

  real* Eout = reinterpret_cast<real*>(P.Eout);
  real* Bout = reinterpret_cast<real*>(P.Bout);
  real En[3] = {0, 0, 0}, Bn[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (e_present<DIM>(a)) {
      Eout[a * pl + id] = sE[a * NR + r];
      const int b = (a + 1) % 3, d = (a + 2) % 3;
      const bool ob = axis_present<DIM>(b), od = axis_present<DIM>(d);
      const int sb = ob ? C::stride(b) : 0, sd = od ? C::stride(d) : 0;
      const int nb = ob ? 2 : 1, nd = od ? 2 : 1;
      real s = 0;
#pragma unroll
      for (int jb = 0; jb < 2; ++jb)
#pragma unroll
        for (int jd = 0; jd < 2; ++jd)
          if (jb < nb && jd < nd) s += sE[a * NR + r - jb * sb - jd * sd];
      En[a] = s * (real(1) / real(nb * nd));
    }
    if (b_present<DIM>(a)) {
      const real bo = Bin[a * pl + id];
      if (axis_present<DIM>(a)) {
        const int nm = wrap_or_clamp(e[a] - 1, P.n[a], P.periodic);
        Bn[a] = real(0.5) * (bo + Bin[a * pl + id + (nm - e[a]) * P.axis_stride[a]]);
      } else {
        Bn[a] = bo;
      }
      const int b = (a + 1) % 3, d = (a + 2) % 3;
      real curl = 0;
      if (axis_present<DIM>(b) && e_present<DIM>(d))
        curl += (sE[d * NR + r] - sE[d * NR + r - C::stride(b)]) * idx_;
      if (axis_present<DIM>(d) && e_present<DIM>(b))
        curl -= (sE[b * NR + r] - sE[b * NR + r - C::stride(d)]) * idx_;
      Bout[a * pl + id] = bo - dt * curl;
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

  real F[K];
  if constexpr (CL == CL_LEC) {
    F[0] = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const real gPi = (smac[M::R_PI * NR + r + C::stride(a)] - smac[M::R_PI * NR + r - C::stride(a)]) * i2dx;
      F[1 + a] = -S.mu * gPi - n * (En[a] + uxB[a]);
    }
  } else {
    real* prev = reinterpret_cast<real*>(P.prev);
    real th[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int j = M::thidx(a, b);
        th[a][b] = j >= 0 ? smac[(M::R_TH + j) * NR + r] : real(0);
      }
    real th0[3] = {0, 0, 0}, w[3] = {0, 0, 0};
    const real lam = smac[M::R_LAM * NR + r];
#pragma unroll
    for (int a = 0; a < DIM; ++a) { th0[a] = smac[(M::R_TH0 + a) * NR + r]; w[a] = lam * u[a]; }
    real th00 = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) th00 += u[a] * th0[a];
    // backward time differences (zero on the first step after a reset)
    real dth00 = 0, dth0[3] = {0, 0, 0}, dw[3] = {0, 0, 0};
    if (P.have_prev) {
      const real idt = S.idt;
      dth00 = (th00 - prev[id]) * idt;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        dth0[a] = (th0[a] - prev[(1 + a) * pl + id]) * idt;
        dw[a] = (w[a] - prev[(1 + DIM + a) * pl + id]) * idt;
      }
    }
    prev[id] = th00;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      prev[(1 + a) * pl + id] = th0[a];
      prev[(1 + DIM + a) * pl + id] = w[a];
    }
    // spatial gradients from the neighbours' records
    real gw[3][3];  // gw[a][k] = d_k w^a
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) gw[a][k] = 0;
    real divth[3] = {0, 0, 0}, divth0 = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const int rp = r + C::stride(k), rm = r - C::stride(k);
      const real lp = smac[M::R_LAM * NR + rp], lm = smac[M::R_LAM * NR + rm];
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        gw[a][k] = (lp * smac[(M::R_U + a) * NR + rp] - lm * smac[(M::R_U + a) * NR + rm]) * i2dx;
      divth0 += (smac[(M::R_TH0 + k) * NR + rp] - smac[(M::R_TH0 + k) * NR + rm]) * i2dx;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int j = M::thidx(a, k);
        if (j >= 0) divth[a] += (smac[(M::R_TH + j) * NR + rp] - smac[(M::R_TH + j) * NR + rm]) * i2dx;
      }
    }
    real Eu = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) Eu += En[a] * u[a];
    F[0] = 0;
    F[1] = -dth00 - divth0 - n * Eu;
#pragma unroll
    for (int a = 0; a < DIM; ++a) F[2 + a] = -dth0[a] - divth[a] - n * (En[a] + uxB[a]);
#pragma unroll
    for (int j = 0; j < M::NTH; ++j) {
      const int a = M::tha(j), b = M::thb(j);
      real s = -th0[b] * dw[a] - th0[a] * dw[b];
#pragma unroll
      for (int k = 0; k < DIM; ++k) s -= th[b][k] * gw[a][k] + th[a][k] * gw[b][k];
      real em = En[a] * th0[b] + En[b] * th0[a];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          if (levi(a, k, l) != 0) em += real(levi(a, k, l)) * th[b][k] * Bn[l];
          if (levi(b, k, l) != 0) em += real(levi(b, k, l)) * th[a][k] * Bn[l];
        }
      F[2 + DIM + j] = s - em;
    }
  }

  // ---------------- collide + store (deviation form) ----------------------
  real ul[3] = {0, 0, 0};
  real usq = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) { ul[a] = S.courant * u[a]; usq += ul[a] * ul[a]; }
  const real itau = S.inv_tau;
  store* fout = reinterpret_cast<store*>(P.fout);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    real df[Q];
    real dA;
    if constexpr (KEEP) {
#pragma unroll
      for (int i = 0; i < Q; ++i) df[i] = keep[k * Q + i];
      dA = dA_own[k];
    } else {
      pull(gz, gx, gy, k, df);
      dA = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) dA += df[i];
    }
    const real A = S.Arest[k] + dA;
    const real dtF = dt * F[k];
    const float s = P.scale[k];
    store* fk = fout + (size_t)k * Q * (size_t)P.plane;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      real cu = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) cu += real(L::c(i, a)) * ul[a];
      const real wi = real(L::w(i));
      const real Pi = real(3) * cu + real(4.5) * cu * cu - real(1.5) * usq;
      const real dfeq = wi * (dA + A * Pi);
      const real v = df[i] - (df[i] - dfeq) * itau + wi * dtF;
      Codec<PR>::store(fk, i * pl + id, v, s);
    }
  }
}

// Plain variant: populations pulled straight from global memory (any
// dimension, open or periodic boundaries).
template <int DIM, int CL, int PR, int TZ, int TX, int TY>
__global__ void __launch_bounds__(TZ* TX* TY)
lb_step_kernel(const StepParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GlobalPull<DIM, CL, PR> pull{P};
  step_body<DIM, CL, PR, TZ, TX, TY>(P, smem_raw, pull);
}

}  // namespace lbp
