// Discrete adjoint of one coupled time step (1D and 2D), for gradients of a
// field value with respect to the driver parameters (Eq. bunch-density:
// alpha, sigma_z, sigma_r or the sampled profile).
//
// The forward step (lb_step.cuh) is, per node: moments and closure decode
// (Eq. disc-moments-ade, Sec. 4.1 / 5.1), E^{n+1/2} = E^{n-1/2} + dt (curl B
// + n u + n_b z), B^{n+1} = B^n - dt curl E^{n+1/2}, sources (Eq.
// lb-ade-lec-comps-F / lb-ade-warmc-comps-F with App. A) from E^{n+1/2},
// B^n and central differences of the neighbours, BGK + w_i dt F (Eq. lbe,
// lsource), pull streaming with the open-boundary copy (Eq. open-bc).  The
// reverse step applies the transpose of each stage in the opposite order.
// Every transposed stencil is written in gather ("pull") form, so each node
// computes its own adjoint without atomics:
//   adj_coll_kernel   - per node and set: the gather of the next state's
//     population adjoints (folding the boundary copies), formed as they are
//     read from the values the previous reverse step's gather left and its
//     adjoint of A_k: lambda_f^{n+1} = (1 - 1/tau) lambda_fs^{n+1} +
//     lambda_A^{n+1}; then the adjoint of streaming and collision for that
//     set.  One thread per (node, set), so the gathers run in parallel
//     instead of on each node's chain; the gathered values are kept for the
//     next reverse step, and no kernel writes lambda_f itself.
//   adj_local_kernel  - per node: the collision adjoints summed over the
//     sets, and the adjoint of the sources' local terms; publishes small
//     records for the neighbours: the decode adjoint of its local part, the
//     coefficients of its gradient stencils, and the adjoints of its
//     node-averaged E^{n+1/2} and B^n.
//   adj_field_kernel  - per node: adjoint of E^{n+1/2} at the slots around
//     the node (next-state E, B update, node averages), of B^n (E update,
//     node average), of the decoded values (neighbours' gradient records,
//     the current n u) and the decode adjoint, giving lambda_A; plus per-row
//     partial sums of dt lambda(E_z) times the driver's transverse factor,
//     from which the driver-parameter gradients are formed.
// The step's forward values come from the tape the step kernel wrote while
// recording: its deviation moments dA^n (decoded here exactly as the step
// decoded them), E^{n+1/2} and B^n; the previous step's values of the WARMC
// backward differences come from the previous tape entry.
#pragma once

#include "lb_adjoint_types.cuh"
#include "lb_step.cuh"

namespace lbp {

template <int DIM, int CL>
struct AdjModel {
  using M = Model<DIM, CL>;
  static constexpr int K = M::K;
  static constexpr int NE = DIM;                                // present E components z[, x]
  static constexpr int NB = DIM == 2 ? 1 : 0;                   // present B components [y]
  static constexpr int NTAPE = K + NE + NB;
  static constexpr int NG = CL == CL_LEC ? DIM : 1 + DIM + DIM * DIM;
  static constexpr int NPREV = M::NPREV;
};


// ---------------------------------------------------------------------------
// Index helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int aidx(const StepParams& P, int z, int x) { return z + x * P.nzp; }

// Nodes m with wrap_or_clamp(m + delta) == c along an axis of n nodes.
struct Pre {
  int v[2];
  int cnt;
};
__device__ __forceinline__ Pre preimage(int c, int n, int delta, int periodic) {
  Pre r;
  r.cnt = 0;
  const int m = c - delta;
  if (periodic) {
    r.v[r.cnt++] = m < 0 ? m + n : (m >= n ? m - n : m);
  } else {
    if (m >= 0 && m < n) r.v[r.cnt++] = m;
    if ((delta > 0 && c == n - 1) || (delta < 0 && c == 0)) r.v[r.cnt++] = c;
  }
  return r;
}

// Adjoints of the post-collision populations of set k at node (z, x): for
// velocity i, the sum of the next state's population adjoints of every node
// that pulls it.  Node y pulls f*_i(bulk(y) - xi_i); with open boundaries the
// boundary nodes copy their nearest bulk node, so a bulk target also
// collects their adjoints.  EDGE = false promises that (z, x) lies at least
// three nodes inside the grid, so no boundary rule applies and the Q loads
// are issued back to back.
// The next state's population adjoints formed where they are gathered:
// lambda_f^{n+1}_i(m) = (1 - 1/tau) lambda_fs_i(m) + lambda_A_k(m), from the
// values the previous reverse step's gather left at node m (lam, [K][Q]
// planes) and its adjoint of A_k (lA, [K] planes), so that no kernel writes
// lambda_f itself.
template <int DIM, bool EDGE, typename real>
struct NextLSrc {
  const StepParams& P;
  const real* lam;
  const real* lA;
  real omt;
  __device__ __forceinline__ void load(int k, int z, int x, real (&l)[Lattice<DIM>::Q]) const {
    using L = Lattice<DIM>;
    constexpr int Q = L::Q;
    const int pl = (int)P.plane;
    const real* lk = lam + (size_t)k * Q * pl;
    const real* ak = lA + (size_t)k * pl;
    auto v = [&](int i, int m) { return omt * gld(lk + i * pl + m) + gld(ak + m); };
    if constexpr (!EDGE) {
      const int b = aidx(P, z, x);
#pragma unroll
      for (int i = 0; i < Q; ++i) l[i] = v(i, b + L::c(i, 0) + (DIM >= 2 ? L::c(i, 1) * P.nzp : 0));
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        int yz = z + L::c(i, 0), yx = DIM >= 2 ? x + L::c(i, 1) : 0;
        if (P.periodic) {
          yz = wrap_or_clamp(yz, P.n[0], 1);
          if (DIM >= 2) yx = wrap_or_clamp(yx, P.n[1], 1);
          l[i] = v(i, aidx(P, yz, yx));
          continue;
        }
        real s = 0;
        const bool in = yz >= 1 && yz <= P.n[0] - 2 && (DIM < 2 || (yx >= 1 && yx <= P.n[1] - 2));
        if (in) {
          int cz[3] = {yz, -1, -1}, cx[3] = {yx, -1, -1};
          if (yz == 1) cz[1] = 0;
          if (yz == P.n[0] - 2) cz[2] = P.n[0] - 1;
          if (DIM >= 2) {
            if (yx == 1) cx[1] = 0;
            if (yx == P.n[1] - 2) cx[2] = P.n[1] - 1;
          }
#pragma unroll
          for (int qz = 0; qz < 3; ++qz) {
            if (cz[qz] < 0) continue;
#pragma unroll
            for (int qx = 0; qx < (DIM >= 2 ? 3 : 1); ++qx) {
              if (cx[qx] < 0) continue;
              s += v(i, aidx(P, cz[qz], cx[qx]));
            }
          }
        }
        l[i] = s;
      }
    }
  }
};

// Programmatic dependent launch: the reverse step's kernels are launched
// so that the next one's CTAs may be scheduled while this one's last CTAs
// run; each kernel lets its dependents launch on entry and waits for its
// predecessor's completion (and memory) before it reads anything.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Whether every node of the calling warp lies three or more nodes inside
// the grid (a warp is 32 consecutive z of one x row of the tile).
template <int DIM, int TZ, int TX>
__device__ __forceinline__ bool warp_interior(const StepParams& P) {
  static_assert(TZ % 32 == 0, "a warp spans 32 consecutive z");
  const int w = (int)threadIdx.x / 32;
  const int z0 = blockIdx.x * TZ + (w % (TZ / 32)) * 32, x = DIM >= 2 ? blockIdx.y * TX + w / (TZ / 32) : 0;
  bool in = z0 >= 3 && z0 + 31 <= P.n[0] - 4;
  if (DIM >= 2) in = in && x >= 3 && x <= P.n[1] - 4;
  return in;
}

// Whether every node of the block's tile lies three or more nodes inside
// the grid (no boundary rule in the population gather).
template <int DIM, int TZ, int TX>
__device__ __forceinline__ bool block_interior(const StepParams& P) {
  const int z0 = blockIdx.x * TZ, x0 = blockIdx.y * TX;
  bool in = z0 >= 3 && z0 + TZ - 1 <= P.n[0] - 4;
  if (DIM >= 2) in = in && x0 >= 3 && x0 + TX - 1 <= P.n[1] - 4;
  return in;
}

// ---------------------------------------------------------------------------
// Decoded values of a node, from its tape moments (the step's decode).
// ---------------------------------------------------------------------------
template <int DIM, int CL, typename real>
struct Node {
  real dA[Model<DIM, CL>::K];
  real rec[Model<DIM, CL>::NM];
};

template <int DIM, int CL, typename real>
__device__ __forceinline__ void load_node(const StepParams& P, const real* tp, int id, Node<DIM, CL, real>& N) {
  constexpr int K = Model<DIM, CL>::K;
  const int pl = (int)P.plane;
#pragma unroll
  for (int k = 0; k < K; ++k) N.dA[k] = gld(tp + k * pl + id);
  decode_record<DIM, CL, real>(P, consts<real>(P), N.dA, N.rec);
}

// WARMC theta^{ab} from the record (stored pairs as deviations from rest,
// symmetric; 0 elsewhere).
template <int DIM, typename real>
__device__ __forceinline__ real th_of(const StepConst<real>& S, const real* rec, int a, int b) {
  using M = Model<DIM, CL_WARMC>;
  const int j = M::thidx(a, b);
  return j >= 0 ? S.threst[j] + rec[M::R_TH + j] : real(0);
}

// Adjoint of the decoded values of one node.
template <typename real>
struct LMac {
  real n, lam, Pi, th00;
  real u[3], th0[3], w[3];
  real th[3][3];
  __device__ __forceinline__ void zero() {
    n = lam = Pi = th00 = real(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      u[a] = th0[a] = w[a] = real(0);
#pragma unroll
      for (int b = 0; b < 3; ++b) th[a][b] = real(0);
    }
  }
};

// Transposed decode: adds d(decoded)/d(dA)^T lm to lA.
//  LEC (Sec. 4.1): n = A_0; p solves n H(n/gamma) p = A_p with
//    gamma = sqrt(1 + p^2), H = 1 + (1 + D/2) mu (n/gamma)^(2/D); u = p/gamma,
//    Pi = (n/gamma)^(1+2/D).  At the fixed point the implicit function
//    theorem gives dp = M^-1 (dA_p - p (H + cH e x^e) dn) with
//    M = n (H I - beta p p^T), beta = cH e x^e / gamma^2 (x = n/gamma,
//    e = 2/D), inverted by the Sherman-Morrison formula.
//  WARMC (Eq. lb-ade-warmc-comps-A, traces4): the record n, lambda = nl/n,
//    u = A_u / nl, theta_j = A_j n / nl, theta^{0a} = u_b theta^{ab}, and
//    the step's theta^{00} = u_a theta^{0a}, w^a = lambda u^a.
template <int DIM, int CL, typename real>
__device__ __forceinline__ void decode_adjoint(const StepParams& P, const StepConst<real>& S,
                                               const Node<DIM, CL, real>& N, LMac<real> lm, real* lA) {
  using M = Model<DIM, CL>;
  if constexpr (CL == CL_LEC) {
    const real n = N.rec[M::R_N];
    real u[DIM], p[DIM], uu = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) { u[a] = N.rec[M::R_U + a]; uu += u[a] * u[a]; }
    const real g = real(1) / sqrt(real(1) - uu);
    const real ig = real(1) / g;
#pragma unroll
    for (int a = 0; a < DIM; ++a) p[a] = g * u[a];
    const real D = real(P.D), e = real(2) / D;
    const real x = n * ig;
    const real xe = pow_2_over_D<real>(x, P.D);
    const real Pi = x * xe;
    const real H = real(1) + S.cH * xe;
    real lp[DIM], pl = 0, pp = 0;
    real ud = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) ud += lm.u[a] * p[a];
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      lp[b] = lm.u[b] * ig - ud * p[b] * ig * ig * ig - lm.Pi * (real(1) + e) * Pi * p[b] * ig * ig;
      pl += p[b] * lp[b];
      pp += p[b] * p[b];
    }
    real ln = lm.n + lm.Pi * (real(1) + e) * xe * ig;
    const real beta = S.cH * e * xe * ig * ig;
    const real c = beta * pl / (H - beta * pp);
    const real inH = real(1) / (n * H);
    const real dn_coef = H + S.cH * e * xe;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const real mu_a = (lp[a] + c * p[a]) * inH;
      lA[1 + a] += mu_a;
      ln -= mu_a * p[a] * dn_coef;
    }
    lA[0] += ln;
  } else {
    const real n = real(1) + N.dA[0];
    const real nl = S.Arest[1] + N.dA[1];
    const real inl = real(1) / nl;
    const real lam = N.rec[M::R_LAM];
    real u[3] = {0, 0, 0}, th0[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) { u[a] = N.rec[M::R_U + a]; th0[a] = N.rec[M::R_TH0 + a]; }
    // theta^{00} = u_a theta^{0a}
#pragma unroll
    for (int a = 0; a < DIM; ++a) { lm.u[a] += lm.th00 * th0[a]; lm.th0[a] += lm.th00 * u[a]; }
    // theta^{0a} = u_b theta^{ab}
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        if (M::thidx(a, b) < 0) continue;
        lm.u[b] += lm.th0[a] * th_of<DIM>(S, N.rec, a, b);
        lm.th[a][b] += lm.th0[a] * u[b];
      }
    // w^a = lambda u^a
#pragma unroll
    for (int a = 0; a < DIM; ++a) { lm.lam += lm.w[a] * u[a]; lm.u[a] += lm.w[a] * lam; }
    // theta_j = A_j n / nl
    real lilam = 0;
    const real ilam = n * inl;
#pragma unroll
    for (int j = 0; j < M::NTH; ++j) {
      const int a = M::tha(j), b = M::thb(j);
      const real l = a == b ? lm.th[a][a] : lm.th[a][b] + lm.th[b][a];
      lA[2 + DIM + j] += l * ilam;
      lilam += l * (S.Arest[2 + DIM + j] + N.dA[2 + DIM + j]);
    }
    real ln = lm.n + lilam * inl;
    real linl = lilam * n;
    // u_a = A_{2+a} / nl
#pragma unroll
    for (int a = 0; a < DIM; ++a) { lA[2 + a] += lm.u[a] * inl; linl += lm.u[a] * N.dA[2 + a]; }
    // lambda = nl / n
    real lnl = lm.lam / n;
    ln -= lm.lam * lam / n;
    lnl -= linl * inl * inl;
    lA[1] += lnl;
    lA[0] += ln;
  }
}

// ---------------------------------------------------------------------------
// Kernel 2: collision adjoints summed over the sets, local source adjoints.
// ---------------------------------------------------------------------------
template <int DIM, int CL, typename real>
__device__ __forceinline__ void adj_local_node(const AdjParams& A, int z, int x) {
  using M = Model<DIM, CL>;
  using AM = AdjModel<DIM, CL>;
  using L = Lattice<DIM>;
  constexpr int K = M::K, Q = L::Q;
  const StepParams& P = A.P;
  const StepConst<real>& S = consts<real>(P);
  const int pl = (int)P.plane;
  const int id = aidx(P, z, x);
  const real* tp = reinterpret_cast<const real*>(A.tape);

  Node<DIM, CL, real> N;
  load_node<DIM, CL, real>(P, tp, id, N);
  const real n = N.rec[M::R_N];
  real u[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < DIM; ++a) u[a] = N.rec[M::R_U + a];

  LMac<real> lm;
  lm.zero();

  // ---- fields at the node (E^{n+1/2}, B^n from the tape) -------------------
  const real* tE = tp + K * pl;
  real En[3] = {0, 0, 0}, Bn[3] = {0, 0, 0};
  if constexpr (DIM == 1) {
    En[0] = gld(tE + id);
  } else {
    // E_z: slots (z, x) and (z, x - 1) (conducting-wall ghost below x = 0)
    real ez = gld(tE + id);
    if (x >= 1) ez += gld(tE + aidx(P, z, x - 1));
    else if (P.periodic) ez += tE[aidx(P, z, P.n[1] - 1)];
    En[0] = real(0.5) * ez;
    // E_x: slots (z, x) and (z - 1, x) (z clamps)
    const int zm = z >= 1 ? z - 1 : (P.periodic ? P.n[0] - 1 : 0);
    En[1] = real(0.5) * (gld(tE + pl + id) + gld(tE + pl + aidx(P, zm, x)));
    Bn[2] = gld(tp + (K + DIM) * pl + id);
  }

  // ---- WARMC: values of the sources' time and space derivatives ------------
  const int hp = P.have_prev;
  real th0[3] = {0, 0, 0}, w[3] = {0, 0, 0}, dw[3] = {0, 0, 0};
  real gw[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  if constexpr (CL == CL_WARMC) {
    const real lam = N.rec[M::R_LAM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) { th0[a] = N.rec[M::R_TH0 + a]; w[a] = lam * u[a]; }
    // w = lambda u of this node's previous step and of its neighbours, as
    // their records give it (formed once per node by adj_coll_kernel)
    const real* cW = reinterpret_cast<const real*>(A.cW);
    // previous-step w (backward time difference)
    if (hp) {
#pragma unroll
      for (int a = 0; a < DIM; ++a) dw[a] = (w[a] - gld(cW + (DIM + a) * pl + id)) * S.idt;
    }
    // gradients of w from the neighbours' decode
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const int ck = k == 0 ? z : x;
      const int cp = wrap_or_clamp(ck + 1, P.n[k], P.periodic), cm = wrap_or_clamp(ck - 1, P.n[k], P.periodic);
      const int idp = k == 0 ? aidx(P, cp, x) : aidx(P, z, cp);
      const int idm = k == 0 ? aidx(P, cm, x) : aidx(P, z, cm);
#pragma unroll
      for (int a = 0; a < DIM; ++a) gw[a][k] = (gld(cW + a * pl + idp) - gld(cW + a * pl + idm)) * S.i2dx;
    }
    // adjoints of the previous-step values this step wrote
    if (A.lp_in) {
      const real* lpi = reinterpret_cast<const real*>(A.lp_in);
      lm.th00 += gld(lpi + id);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        lm.th0[a] += gld(lpi + (1 + a) * pl + id);
        lm.w[a] += gld(lpi + (1 + DIM + a) * pl + id);
      }
    }
  }

  // ---- streaming + collision adjoint (per set, adj_coll_kernel) -----------
  real lA[K], lF[K], lu_c[3] = {0, 0, 0};
  {
    const real* cA = reinterpret_cast<const real*>(A.cA);
    const real* cF = reinterpret_cast<const real*>(A.cF);
    const real* cU = reinterpret_cast<const real*>(A.cU);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      lA[k] = gld(cA + k * pl + id);
      lF[k] = gld(cF + k * pl + id);
#pragma unroll
      for (int a = 0; a < DIM; ++a) lu_c[a] += gld(cU + (k * DIM + a) * pl + id);
    }
  }
#pragma unroll
  for (int a = 0; a < DIM; ++a) lm.u[a] += lu_c[a] * S.courant * S.inv_tau;

  // ---- source adjoint, local terms ----------------------------------------
  real lEn[3] = {0, 0, 0}, lBn[3] = {0, 0, 0};
  real G[AM::NG];
  real lpo[AM::NPREV > 0 ? AM::NPREV : 1];
#pragma unroll
  for (int j = 0; j < (AM::NPREV > 0 ? AM::NPREV : 1); ++j) lpo[j] = real(0);
  // -n (E + u x B)_a and its adjoint, shared by both closures
  auto lorentz = [&](int a, real l) {
    real uxB = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int e3 = levi(a, k, q);
        if (e3 == 0) continue;
        uxB += real(e3) * u[k] * Bn[q];
        lm.u[k] -= n * real(e3) * Bn[q] * l;
        lBn[q] -= n * real(e3) * u[k] * l;
      }
    lm.n -= (En[a] + uxB) * l;
    lEn[a] -= n * l;
  };
  if constexpr (CL == CL_LEC) {
    // F_p = -mu grad Pi - n (E + u x B)
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      G[a] = lF[1 + a];
      lorentz(a, lF[1 + a]);
    }
  } else {
    // F_{n lambda} = -d_t th00 - d_k th0k - n E.u
    {
      const real l = lF[1];
      G[0] = l;
      if (hp) { lm.th00 -= l * S.idt; lpo[0] += l * S.idt; }
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        lm.n -= En[a] * u[a] * l;
        lEn[a] -= n * u[a] * l;
        lm.u[a] -= n * En[a] * l;
      }
    }
    // F_{n lambda u_a} = -d_t th0a - d_b th_ab - n (E + u x B)_a
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const real l = lF[2 + a];
      G[1 + a] = l;
      if (hp) { lm.th0[a] -= l * S.idt; lpo[1 + a] += l * S.idt; }
      lorentz(a, l);
    }
    // F_{lambda th_ab}: time and space derivatives of w, EM terms
    real ldw[3] = {0, 0, 0}, lgw[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int j = 0; j < M::NTH; ++j) {
      const real l = lF[2 + DIM + j];
      const int a = M::tha(j), b = M::thb(j);
      lm.th0[b] -= dw[a] * l;
      ldw[a] -= th0[b] * l;
      lm.th0[a] -= dw[b] * l;
      ldw[b] -= th0[a] * l;
#pragma unroll
      for (int q = 0; q < DIM; ++q) {
        lm.th[b][q] -= gw[a][q] * l;
        lgw[a][q] -= th_of<DIM>(S, N.rec, b, q) * l;
        lm.th[a][q] -= gw[b][q] * l;
        lgw[b][q] -= th_of<DIM>(S, N.rec, a, q) * l;
      }
      lEn[a] -= th0[b] * l;
      lm.th0[b] -= En[a] * l;
      lEn[b] -= th0[a] * l;
      lm.th0[a] -= En[b] * l;
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int ea = levi(a, q, r), eb = levi(b, q, r);
          if (ea != 0) {
            lm.th[b][q] -= real(ea) * Bn[r] * l;
            lBn[r] -= real(ea) * th_of<DIM>(S, N.rec, b, q) * l;
          }
          if (eb != 0) {
            lm.th[a][q] -= real(eb) * Bn[r] * l;
            lBn[r] -= real(eb) * th_of<DIM>(S, N.rec, a, q) * l;
          }
        }
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (hp) { lm.w[a] += ldw[a] * S.idt; lpo[1 + DIM + a] -= ldw[a] * S.idt; }
#pragma unroll
      for (int k = 0; k < DIM; ++k) G[1 + DIM + a * DIM + k] = lgw[a][k];
    }
  }

  decode_adjoint<DIM, CL, real>(P, S, N, lm, lA);

  real* rA = reinterpret_cast<real*>(A.rA);
#pragma unroll
  for (int k = 0; k < K; ++k) rA[k * pl + id] = lA[k];
  real* rG = reinterpret_cast<real*>(A.rG);
#pragma unroll
  for (int j = 0; j < AM::NG; ++j) rG[j * pl + id] = G[j];
  real* rEn = reinterpret_cast<real*>(A.rEn);
#pragma unroll
  for (int a = 0; a < DIM; ++a) rEn[a * pl + id] = lEn[a];
  if constexpr (DIM == 2) reinterpret_cast<real*>(A.rBn)[2 * pl + id] = lBn[2];
  if constexpr (AM::NPREV > 0) {
    real* lpo_g = reinterpret_cast<real*>(A.lp_out);
#pragma unroll
    for (int j = 0; j < AM::NPREV; ++j) lpo_g[j * pl + id] = lpo[j];
  }
}

template <int DIM, int CL, typename real, int TZ, int TX, int MINB>
__global__ void __launch_bounds__(TZ* TX, MINB) adj_local_kernel(const AdjParams A) {
  pdl_enter();
  const StepParams& P = A.P;
  const int z = blockIdx.x * TZ + threadIdx.x % TZ;
  const int x = DIM >= 2 ? blockIdx.y * TX + threadIdx.x / TZ : 0;
  if (z >= P.n[0] || (DIM >= 2 && x >= P.n[1])) return;
  adj_local_node<DIM, CL, real>(A, z, x);
}

// ---------------------------------------------------------------------------
// Kernel 1 (launched first): streaming and collision adjoints per set.
// ---------------------------------------------------------------------------

// Streaming + collision adjoint of one set k at one node, the gather of the
// next state's population adjoints kept off the per-node kernels' chains:
// fs = f (1 - 1/tau) + f^eq(A, C u)/tau + w dt F with
// f^eq = w A (1 + 3 cu + 9/2 cu^2 - 3/2 u^2) gives
//   lambda_A += sum_i w_i (1 + P_i) lambda_fs / tau
//   lambda_u += sum_i w_i A C (3 xi + 9 cu xi - 3 u) lambda_fs / tau
//   lambda_F  = dt sum_i w_i lambda_fs.
// Written: cA = the first, cF = the third, cU = A_k times the sum of the
// second (adj_local adds C/tau times its sum over the sets, in set order).
// Sets per thread of the per-(node, set) kernels (2D WARMC FP32, cost ratio
// of the 1000-step sweep with the whole tape: one set 3.13-3.14, two 3.36-3.37,
// four 3.81-3.82: the gathers want threads, not longer threads).
constexpr int kAdjSetsPerThread = 1;

template <int DIM, int CL, typename real, class LSrc>
__device__ __forceinline__ void adj_coll_node(const AdjParams& A, const LSrc& src, int z, int x, int k0) {
  using L = Lattice<DIM>;
  constexpr int Q = L::Q;
  const StepParams& P = A.P;
  const StepConst<real>& S = consts<real>(P);
  const int pl = (int)P.plane;
  const int id = aidx(P, z, x);
  const real* tp = reinterpret_cast<const real*>(A.tape);
  // the node's u as the step decoded it (WARMC: only the moments it needs)
  real u[3] = {0, 0, 0};
  if constexpr (CL == CL_WARMC) {
    const real nl = S.Arest[1] + gld(tp + pl + id);
    const real inl = real(1) / nl;
#pragma unroll
    for (int a = 0; a < DIM; ++a) u[a] = gld(tp + (2 + a) * pl + id) * inl;
    if (k0 == 0) {
      // w = lambda u of this step and of the previous one, for adj_local's
      // backward time difference and its neighbours' central differences
      real* cW = reinterpret_cast<real*>(A.cW);
      const real lam = nl / (real(1) + gld(tp + id));
#pragma unroll
      for (int a = 0; a < DIM; ++a) cW[a * pl + id] = lam * u[a];
      if (P.have_prev) {
        real wp[3] = {0, 0, 0};
        if (A.tape_prev) {
          const real* tq = reinterpret_cast<const real*>(A.tape_prev);
          const real nlq = S.Arest[1] + gld(tq + pl + id);
          const real inlq = real(1) / nlq;
          const real lamq = nlq / (real(1) + gld(tq + id));
#pragma unroll
          for (int a = 0; a < DIM; ++a) wp[a] = lamq * (gld(tq + (2 + a) * pl + id) * inlq);
        } else {
          const real* p0 = reinterpret_cast<const real*>(A.prev0);
#pragma unroll
          for (int a = 0; a < DIM; ++a) wp[a] = gld(p0 + (1 + DIM + a) * pl + id);
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) cW[(DIM + a) * pl + id] = wp[a];
      }
    }
  } else {
    Node<DIM, CL, real> N;
    load_node<DIM, CL, real>(P, tp, id, N);
#pragma unroll
    for (int a = 0; a < DIM; ++a) u[a] = N.rec[Model<DIM, CL>::R_U + a];
  }
  real ul[3] = {0, 0, 0}, usq = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    ul[a] = S.courant * u[a];
    usq += ul[a] * ul[a];
  }
  // opposite velocities (i, i + 1) share w_i and |cu|: with s = l_i + l_j and
  // d = l_i - l_j the even part carries 1 + 9/2 cu^2 - 3/2 u^2, the odd 3 cu
  static_assert(opposite_pairs<DIM>(), "lattice order must pair opposite velocities");
  const real even0 = real(1) - real(1.5) * usq;
#pragma unroll
  for (int ks = 0; ks < kAdjSetsPerThread; ++ks) {
  const int k = k0 + ks;
  if (k >= Model<DIM, CL>::K) break;
  real lk[Q];
  src.load(k, z, x, lk);
  // the gathered values, from which the next reverse step forms this step's
  // population adjoints (NextLSrc)
  {
    real* lo = reinterpret_cast<real*>(A.lf_out) + (size_t)k * Q * pl + id;
#pragma unroll
    for (int i = 0; i < Q; ++i) lo[i * pl] = lk[i];
  }
  const real w0l = real(L::w(0)) * lk[0];
  real m0 = w0l, mA = w0l * even0, mu_[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < DIM; ++a) mu_[a] = -real(3) * ul[a] * w0l;
#pragma unroll
  for (int q = 0; q < (Q - 1) / 2; ++q) {
    const int i = 1 + 2 * q;
    const real wi = real(L::w(i));
    const real sp = wi * (lk[i] + lk[i + 1]), dm = wi * (lk[i] - lk[i + 1]);
    real cu = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) cu += real(L::c(i, a)) * ul[a];
    m0 += sp;
    mA += sp * (even0 + real(4.5) * cu * cu) + real(3) * cu * dm;
    const real t = real(3) * dm + real(9) * cu * sp;
#pragma unroll
    for (int a = 0; a < DIM; ++a) mu_[a] += real(L::c(i, a)) * t - real(3) * ul[a] * sp;
  }
  const real Ak = S.Arest[k] + gld(tp + k * pl + id);
  reinterpret_cast<real*>(A.cA)[k * pl + id] = mA * S.inv_tau;
  reinterpret_cast<real*>(A.cF)[k * pl + id] = S.dt * m0;
  real* cU = reinterpret_cast<real*>(A.cU);
#pragma unroll
  for (int a = 0; a < DIM; ++a) cU[(k * DIM + a) * pl + id] = Ak * mu_[a];
  }
}

// Resident threads per SM the gather kernel's register budget is held to
// in FP32: 2048 (32 registers, 32 bytes of spills; the sweep's cost ratio
// 3.03 against 3.05-3.06 at 1536 threads and 40 registers); the FP64 kernels
// are left to the compiler (held to 32 registers they spill 330 bytes).
template <typename real, int NT> struct AdjGatherBlocks { static constexpr int value = 1; };
template <int NT> struct AdjGatherBlocks<float, NT> { static constexpr int value = 2048 / NT; };

// grid: (z tiles, x tiles, K)
template <int DIM, int CL, typename real, int TZ, int TX>
__global__ void __launch_bounds__(TZ* TX, (AdjGatherBlocks<real, TZ * TX>::value)) adj_coll_kernel(const AdjParams A) {
  pdl_enter();
  const StepParams& P = A.P;
  const int k = blockIdx.z * kAdjSetsPerThread;
  const real* lam = reinterpret_cast<const real*>(A.lf_in);
  const real* lA = reinterpret_cast<const real*>(A.lAf);
  const real omt = real(1) - consts<real>(P).inv_tau;
  if (DIM == 2 && A.band_rows > 0) {
    // 2D: the nodes within 3 of an edge (the band, whose gathers fold the
    // boundary copies) are taken by the last band_rows rows of blocks, one
    // band node per thread; the tiles' threads skip them, so no warp mixes
    // the two gathers
    const int n0 = P.n[0], n1 = P.n[1];
    const int ntiles_x = (int)gridDim.y - A.band_rows;
    if ((int)blockIdx.y < ntiles_x) {
      const int z = blockIdx.x * TZ + threadIdx.x % TZ, x = blockIdx.y * TX + threadIdx.x / TZ;
      if (z < 3 || z >= n0 - 3 || x < 3 || x >= n1 - 3) return;
      adj_coll_node<DIM, CL, real>(A, NextLSrc<DIM, false, real>{P, lam, lA, omt}, z, x, k);
    } else {
      const int t = ((blockIdx.y - ntiles_x) * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
      int z, x;
      if (t < 3 * n0) { x = t / n0; z = t - x * n0; }
      else if (t < 6 * n0) { const int u = t - 3 * n0; x = n1 - 3 + u / n0; z = u % n0; }
      else if (t < 6 * n0 + 6 * (n1 - 6)) { const int u = t - 6 * n0, j = u % 6; x = 3 + u / 6; z = j < 3 ? j : n0 - 6 + j; }
      else return;
      adj_coll_node<DIM, CL, real>(A, NextLSrc<DIM, true, real>{P, lam, lA, omt}, z, x, k);
    }
    return;
  }
  const int z = blockIdx.x * TZ + threadIdx.x % TZ;
  const int x = DIM >= 2 ? blockIdx.y * TX + threadIdx.x / TZ : 0;
  if (warp_interior<DIM, TZ, TX>(P)) {
    adj_coll_node<DIM, CL, real>(A, NextLSrc<DIM, false, real>{P, lam, lA, omt}, z, x, k);
  } else {
    if (z >= P.n[0] || (DIM >= 2 && x >= P.n[1])) return;
    adj_coll_node<DIM, CL, real>(A, NextLSrc<DIM, true, real>{P, lam, lA, omt}, z, x, k);
  }
}

// ---------------------------------------------------------------------------
// Kernel 3: field adjoints, gradient-stencil gathers, decode adjoint and the
// population adjoint of the previous state.
// ---------------------------------------------------------------------------

// Adjoint of E_a^{n+1/2} at slot (sz, sx): as the next state's E, through
// the node averages of the sources and through B^{n+1}; zero on walls.
template <int DIM, typename real>
__device__ __forceinline__ real lEn_slot(const AdjParams& A, int a, int sz, int sx) {
  const StepParams& P = A.P;
  const StepConst<real>& S = consts<real>(P);
  const int pl = (int)P.plane;
  const real* lE = reinterpret_cast<const real*>(A.lE_in);
  const real* rEn = reinterpret_cast<const real*>(A.rEn);
  const int id = aidx(P, sz, sx);
  if constexpr (DIM == 1) {
    return gld(lE + id) + gld(rEn + id);
  } else {
    const real* lB = reinterpret_cast<const real*>(A.lB_in) + 2 * pl;  // B_y
    const real* rE = rEn + a * pl;
    const real cdt = S.dt * S.idx;
    if (a == 0) {
      if (!P.periodic && sx == P.n[1] - 1) return real(0);  // conducting wall
      real v = gld(lE + id) + real(0.5) * gld(rE + id) + cdt * gld(lB + id);
      int xp = sx + 1;
      if (xp >= P.n[1]) xp = P.periodic ? 0 : -1;
      if (xp >= 0) {
        const int idp = aidx(P, sz, xp);
        v += real(0.5) * gld(rE + idp) - cdt * gld(lB + idp);
      }
      return v;
    } else {
      real v = gld(lE + pl + id) + real(0.5) * gld(rE + id) - cdt * gld(lB + id);
      int zp = sz + 1;
      if (zp >= P.n[0]) zp = P.periodic ? 0 : -1;
      if (zp >= 0) {
        const int idp = aidx(P, zp, sx);
        v += real(0.5) * gld(rE + idp) + cdt * gld(lB + idp);
      }
      if (!P.periodic && sz == 0) v += real(0.5) * gld(rE + id) + cdt * gld(lB + id);
      return v;
    }
  }
}

// Per-row partial sums of the driver-gradient weights of the block's tile.
template <int TZ, int TX>
__device__ __forceinline__ void row_partials(const AdjParams& A, double (&red)[2][TX][TZ], int tzi, int txi, int z,
                                             double r0, double r2) {
  red[0][txi][tzi] = r0;
  red[1][txi][tzi] = r2;
  __syncthreads();
  if (txi == 0 && z < A.P.n[0]) {
    double s0 = 0.0, s2 = 0.0;
#pragma unroll
    for (int t = 0; t < TX; ++t) { s0 += red[0][t][tzi]; s2 += red[1][t][tzi]; }
    const int ntx = gridDim.y;
    A.rows[(size_t)blockIdx.y * A.P.n[0] + z] = s0;
    A.rows[((size_t)ntx + blockIdx.y) * A.P.n[0] + z] = s2;
  }
}

template <int DIM, int CL, typename real>
__device__ __forceinline__ void adj_field_node(const AdjParams& A, int z, int x, double& r0, double& r2) {
  using M = Model<DIM, CL>;
  using L = Lattice<DIM>;
  constexpr int K = M::K, Q = L::Q;
  const StepParams& P = A.P;
  const StepConst<real>& S = consts<real>(P);
  {
    const int pl = (int)P.plane;
    const int id = aidx(P, z, x);
    const real* tp = reinterpret_cast<const real*>(A.tape);
    Node<DIM, CL, real> N;
    load_node<DIM, CL, real>(P, tp, id, N);
    const real n = N.rec[M::R_N];
    real u[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) u[a] = N.rec[M::R_U + a];

    LMac<real> lm;
    lm.zero();
    const real dt = S.dt;
    // ---- E^{n+1/2} slots: own (E_a at this node) and the ones below --------
    // J_a at slot s averages n u_a over s and s + e_b (b the slot's offset
    // axis; 1D: the node itself); the B_y curl at this node reads the same
    // slots.
    real* lEo = reinterpret_cast<real*>(A.lE_out);
    if constexpr (DIM == 1) {
      const real l = lEn_slot<DIM, real>(A, 0, z, 0);
      lEo[id] = l;
      lm.n += dt * l * u[0];
      lm.u[0] += dt * l * n;
      r0 = (double)(dt * l);
      r2 = 0.0;
    } else {
      const real cdt = dt * S.idx;
      real lBy = gld(reinterpret_cast<const real*>(A.lB_in) + 2 * pl + id) +
                 gld(reinterpret_cast<const real*>(A.rBn) + 2 * pl + id);
      // E_z: offset axis x
      {
        const real lc = lEn_slot<DIM, real>(A, 0, z, x);
        lEo[id] = lc;
        r0 = (double)(dt * lc) * gld(A.Tx + x);
        r2 = (double)(dt * lc) * gld(A.Tx + P.n[1] + x);
        real jsum = real(0.5) * lc;   // slot s = this node
        lBy -= cdt * lc;
        const Pre pr = preimage(x, P.n[1], +1, P.periodic);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q >= pr.cnt) break;
          const real ls = pr.v[q] == x ? lc : lEn_slot<DIM, real>(A, 0, z, pr.v[q]);
          jsum += real(0.5) * ls;
          lBy += cdt * ls;
        }
        lm.n += dt * jsum * u[0];
        lm.u[0] += dt * jsum * n;
      }
      // E_x: offset axis z
      {
        const real lc = lEn_slot<DIM, real>(A, 1, z, x);
        lEo[pl + id] = lc;
        real jsum = real(0.5) * lc;
        lBy += cdt * lc;
        const Pre pr = preimage(z, P.n[0], +1, P.periodic);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q >= pr.cnt) break;
          const real ls = pr.v[q] == z ? lc : lEn_slot<DIM, real>(A, 1, pr.v[q], x);
          jsum += real(0.5) * ls;
          lBy -= cdt * ls;
        }
        lm.n += dt * jsum * u[1];
        lm.u[1] += dt * jsum * n;
      }
      reinterpret_cast<real*>(A.lB_out)[2 * pl + id] = lBy;
    }

    // ---- gradient stencils of the neighbours that read this node -----------
    const real* rG = reinterpret_cast<const real*>(A.rG);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const int ck = k == 0 ? z : x;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        // side 0: m + e_k = this node (coefficient -1/2dx); side 1: m - e_k
        const Pre pr = preimage(ck, P.n[k], side == 0 ? +1 : -1, P.periodic);
        const real sgn = side == 0 ? real(-1) : real(1);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q >= pr.cnt) break;
          const int m = k == 0 ? aidx(P, pr.v[q], x) : aidx(P, z, pr.v[q]);
          const real c = sgn * S.i2dx;
          if constexpr (CL == CL_LEC) {
            lm.Pi += c * S.mu * gld(rG + k * pl + m);
          } else {
            lm.th0[k] += c * gld(rG + m);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
              lm.th[a][k] += c * gld(rG + (1 + a) * pl + m);
              lm.w[a] -= c * gld(rG + (1 + DIM + a * DIM + k) * pl + m);
            }
          }
        }
      }
    }

    real lA[K];
    const real* rA = reinterpret_cast<const real*>(A.rA);
#pragma unroll
    for (int k = 0; k < K; ++k) lA[k] = gld(rA + k * pl + id);
    decode_adjoint<DIM, CL, real>(P, S, N, lm, lA);

    // the population adjoint of the previous state adds lA (formed by the
    // next reverse step's gather, NextLSrc)
    real* lAf = reinterpret_cast<real*>(A.lAf);
#pragma unroll
    for (int k = 0; k < K; ++k) lAf[k * pl + id] = lA[k];
  }
}

template <int DIM, int CL, typename real, int TZ, int TX, int MINB>
__global__ void __launch_bounds__(TZ* TX, MINB) adj_field_kernel(const AdjParams A) {
  pdl_enter();
  const StepParams& P = A.P;
  __shared__ double red[2][TX][TZ];
  const int tzi = threadIdx.x % TZ, txi = threadIdx.x / TZ;
  const int z = blockIdx.x * TZ + tzi;
  const int x = DIM >= 2 ? blockIdx.y * TX + txi : 0;
  double r0 = 0.0, r2 = 0.0;
  if (z < P.n[0] && (DIM < 2 || x < P.n[1])) adj_field_node<DIM, CL, real>(A, z, x, r0, r2);
  row_partials<TZ, TX>(A, red, tzi, txi, z, r0, r2);
}

// ---------------------------------------------------------------------------
// Driver-parameter gradients from the row sums.
//
// A row set j holds, per z, R0 = sum_x c(x) and R2 = sum_x c2(x) for a
// quantity whose forward value is n_b-like: v(z, x) = L(zeta) T(x) with
// zeta = z dx + zoff_j - zeta0_j.  Then
//   dJ/dalpha   += sum R0 exp(-zeta^2 / 2 sigma_z^2)      (Gaussian L)
//   dJ/dsigma_z += sum R0 L zeta^2 / sigma_z^3           (Gaussian L)
//   dJ/dsigma_r += sum R2 L
//   dJ/dprofile_j += sum R0 (interpolation weight of sample j at zeta).
// ---------------------------------------------------------------------------

__device__ __forceinline__ double row_sum(const GradParams& G, int j, int q, int z) {
  const double* r = G.rows + ((size_t)j * 2 + q) * (size_t)G.ntx * G.n0;
  double s = 0.0;
  for (int t = 0; t < G.ntx; ++t) s += r[(size_t)t * G.n0 + z];
  return s;
}

__device__ __forceinline__ double glong(const GradParams& G, double zeta) {
  if (G.profile) {
    const double s = zeta / G.pdz + 0.5 * (G.plen - 1);
    if (!(s > -1.0 && s < (double)G.plen)) return 0.0;
    const int j = (int)floor(s);
    const double fr = s - j;
    const double a = j >= 0 ? G.profile[j] : 0.0, b = j + 1 < G.plen ? G.profile[j + 1] : 0.0;
    return (1.0 - fr) * a + fr * b;
  }
  return G.alpha * exp(-zeta * zeta * G.inv2sz2);
}

// one block of 256 threads per row set: fixed-order tree over z
__global__ void __launch_bounds__(256) grad_sets_kernel(const GradParams G) {
  __shared__ double red[3][256];
  const int j = blockIdx.x;
  const double zeta0 = G.setp[j].x, zoff = G.setp[j].y;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int z = threadIdx.x; z < G.n0; z += 256) {
    const double R0 = row_sum(G, j, 0, z), R2 = row_sum(G, j, 1, z);
    const double zeta = z * G.dx + zoff - zeta0;
    const double L = glong(G, zeta);
    if (!G.profile) {
      const double g = exp(-zeta * zeta * G.inv2sz2);
      a0 += R0 * g;
      a1 += R0 * L * zeta * zeta / (G.sigma_z * G.sigma_z * G.sigma_z);
    }
    a2 += R2 * L;
  }
  red[0][threadIdx.x] = a0;
  red[1][threadIdx.x] = a1;
  red[2][threadIdx.x] = a2;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 3) G.gpart[j * 3 + threadIdx.x] = red[threadIdx.x][0];
}

// sets summed in order into the running gradient (one thread per output)
__global__ void grad_accum_kernel(const GradParams G) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 3) {
    double s = G.g3[q];
    for (int j = 0; j < G.nsets; ++j) s += G.gpart[j * 3 + q];
    G.g3[q] = s;
  }
  if (G.profile && q < G.plen) {
    // sample q collects the rows whose zeta interpolates between q-1..q+1
    double s = G.gp[q];
    for (int j = 0; j < G.nsets; ++j) {
      const double zeta0 = G.setp[j].x, zoff = G.setp[j].y;
      const double zc = ((q - 0.5 * (G.plen - 1)) * G.pdz + zeta0 - zoff) / G.dx;
      const double span = G.pdz / G.dx + 2.0;
      int zlo = (int)floor(zc - span), zhi = (int)ceil(zc + span);
      zlo = zlo < 0 ? 0 : zlo;
      zhi = zhi > G.n0 - 1 ? G.n0 - 1 : zhi;
      for (int z = zlo; z <= zhi; ++z) {
        const double zeta = z * G.dx + zoff - zeta0;
        const double sv = zeta / G.pdz + 0.5 * (G.plen - 1);
        if (!(sv > -1.0 && sv < (double)G.plen)) continue;
        const int jj = (int)floor(sv);
        const double fr = sv - jj;
        double wgt = 0.0;
        if (jj == q) wgt = 1.0 - fr;
        else if (jj + 1 == q) wgt = fr;
        if (wgt != 0.0) s += row_sum(G, j, 0, z) * wgt;
      }
    }
    G.gp[q] = s;
  }
}

// Initial driver field (2D, v -> c limit): E_x = -L(zeta_E) k(x) at the E_x
// slot (z + dx/2, t = -dt/2), B_y = -L(zeta_B) k(x) at the node (t = 0),
// k(x) = sigma_r sqrt(pi/2) erf(x / (sqrt(2) sigma_r)).  Row sets 0 (E) and
// 1 (B): R0 = sum_x lambda (-k), R2 = sum_x lambda (-dk/dsigma_r).
template <typename real, int TZ, int TX>
__global__ void __launch_bounds__(TZ* TX) adj_init_rows_kernel(StepParams P, const real* lE, const real* lB,
                                                                const double* Kx, double* rows) {
  __shared__ double red[4][TX][TZ];
  const int tzi = threadIdx.x % TZ, txi = threadIdx.x / TZ;
  const int z = blockIdx.x * TZ + tzi, x = blockIdx.y * TX + txi;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (z < P.n[0] && x < P.n[1]) {
    const int pl = (int)P.plane;
    const int id = aidx(P, z, x);
    const double le = (double)lE[pl + id], lb = (double)lB[2 * pl + id];
    v[0] = le * Kx[x];
    v[1] = le * Kx[P.n[1] + x];
    v[2] = lb * Kx[x];
    v[3] = lb * Kx[P.n[1] + x];
  }
  for (int q = 0; q < 4; ++q) red[q][txi][tzi] = v[q];
  __syncthreads();
  if (txi == 0 && z < P.n[0]) {
    const int ntx = gridDim.y;
    for (int q = 0; q < 4; ++q) {
      double s = 0.0;
      for (int t = 0; t < TX; ++t) s += red[q][t][tzi];
      // set (q / 2), component (q % 2)
      rows[(((size_t)(q / 2) * 2 + (q % 2)) * ntx + blockIdx.y) * P.n[0] + z] = s;
    }
  }
}

template <typename real>
__global__ void adj_seed_kernel(real* lE, long long idx, double v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) lE[idx] = real(v);
}

template <typename real>
__global__ void read_slot_kernel(const real* E, const real* Elo, long long idx, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = (double)E[idx] + (Elo ? (double)Elo[idx] : 0.0);
}

}  // namespace lbp
