/*
 * FP64 CPU oracle for the moment-matching lattice Boltzmann (LB) warm-plasma
 * wakefield scheme of arXiv 2309.04872 (Simeoni et al., "Lattice Boltzmann
 * method for warm fluid simulations of plasma wakefield acceleration").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is read by tests/, by the smoke check
 * and by the CPU-baseline leg of bench.py.  The product path (the CUDA
 * library) never includes, links or calls it, and it shares no source with
 * the CUDA path: the stencil tables, the closures, the field update and the
 * driver are all restated here on their own.
 *
 * It is deliberately plain: triple loops over cells, one array per stage,
 * streaming as a full-array pull, everything in double precision.  Each
 * function names the passage of the paper it restates.
 *
 * Units (the paper's normalisation, Sec. 6): length k_p^-1, time omega_p^-1,
 * density n_i, momentum m c, E in m c omega_p / e, B in E/c; so c = m = e = 1
 * and the electron charge is -1.
 *
 * Spatial component index: 0 = z (driver axis), 1 = x, 2 = y.  (z, x, y) is
 * a cyclic permutation of (x, y, z), so the Levi-Civita symbol and the cross
 * product keep their usual form in this index order.
 *
 * Readings of the paper that it fixes (each one is listed with its reason in
 * the design notes of the repository):
 *  - Eq. (ade-feq): the quadratic term is (u.xi)^2 / (2 nu^4), the standard
 *    second-order form; the printed form without the 1/2 does not conserve A.
 *  - Sec. 2.2: source S_i = w_i F with no (1 - 1/2tau) factor; A = sum f.
 *  - Eq. (open-bc): after streaming, every boundary node takes the
 *    populations of its nearest bulk node (corner -> diagonal bulk node).
 *  - Sec. 4.1 iteration: p^(0) = A_p / n, fixed point until the largest
 *    change is <= 1e-15 times the largest |p| (64 iterations at most).
 *  - Eq. (bunch-density): Gaussians written with 2 sigma^2 (rms sizes), the
 *    driver moves towards +z.
 *  - Time levels of the fluid-Maxwell coupling (Sec. 4.1, left to the
 *    companion paper): fluid at integer steps, E at half steps, B at integer
 *    steps on a dual Yee grid; see orc_step_once.
 *  - App. A time derivatives: backward differences of the previous step's
 *    decoded quantities (zero on the first step after a state is set).
 *  - App. A spatial derivatives: second-order central differences; at the
 *    open boundary the missing neighbour is the nearest in-domain node.
 *  - Axisymmetric geometry (Sec. 2.2 end, App. A): the 2D grid is (z, r) with
 *    node j at r = j dx; j = 0 is the r = 0 boundary node.  After streaming
 *    it takes the populations of node j = 1: as they are (Eq. open-bc) for
 *    the sets even under r -> -r, with the mirrored direction (Eq.
 *    reflective-bc) for the odd ones (n A_r; n lambda u_r, lambda theta^{rz}).
 *    The 1/r terms of App. A are added to the sources at r > 0 and left out
 *    at r = 0.  Yee slots as in 2D (E_z at r + dx/2, E_r and B_phi at r);
 *    on the axis E_r = B_phi = 0, and the E_z slot below the axis mirrors
 *    the one above it; (curl B)_z = d_r(r B_phi)/r.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lbpwfa_oracle.h"

/* Planted mistakes, for the test that the pins catch each of them (tests/
 * test_oracle_mutants.py builds the oracle once per mistake with
 * -DORC_PLANT=n).  Without that define PLANTED(n, right, wrong) is `right`
 * and the oracle is exactly the scheme as written. */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif
#define PLANTED(n, right, wrong) (ORC_PLANT == (n) ? (wrong) : (right))

#define ORC_MAXQ 19

typedef struct {
  double n, u[3], gamma;
  double Pi;                       /* LEC: (n/gamma)^(1+2/D) */
  double lam;                      /* WARMC: lambda = n/h = w^0 */
  double th[3][3], th0[3], th00;   /* WARMC: theta^{ab}, theta^{0a}, theta^{00} */
  double w[3];                     /* WARMC: w^a = lambda u^a */
} orc_macro;

struct orc_state {
  orc_params p;
  int Ds, Q, K, ntheta;
  int n[3];           /* cells along z, x, y (1 for absent axes) */
  long ncell;
  double dt;
  int xi[ORC_MAXQ][3];
  double w[ORC_MAXQ];
  int thpair[6][2];
  int mir[ORC_MAXQ];  /* velocity mirrored in x (r -> -r) */
  double Arest[11];
  double *f;          /* [K][Q][ncell] populations at time n (after streaming) */
  double *E, *B;      /* [3][ncell]: E at t_{n-1/2}, B at t_n */
  double *prev;       /* [7][ncell]: theta00, theta0[3], w[3] of the previous step */
  int have_prev;
  int fields_from_driver;  /* E, B still the driver's initial fields */
  long step;
  /* stage arrays */
  orc_macro *mac;
  double *F;          /* [K][ncell] */
  double *fs;         /* [K][Q][ncell] post-collision */
  double *En, *Bn;
};

/* ------------------------------------------------------------------------ */
/* Velocity sets.  Fig. 1 prints D3Q19 (weights 1/3, 1/18, 1/36); the 1D and
 * 2D sets are the D1Q3 and D2Q9 members of the same family with
 * nu^2 = 1/3 (Eq. ade-feq).  Component order of xi: (z, x, y).            */
/* ------------------------------------------------------------------------ */
int orc_stencil(int dim, int* xi /* [Q][3] */, double* w)
{
  int q = 0;
  if (dim == 1) {
    int t[3] = {0, 1, -1};
    for (int i = 0; i < 3; ++i) {
      xi[3 * i] = t[i]; xi[3 * i + 1] = 0; xi[3 * i + 2] = 0;
      w[i] = (i == 0) ? 2.0 / 3.0 : 1.0 / 6.0;
    }
    return 3;
  }
  if (dim == 2) {
    int t[9][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1},
                   {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
    for (int i = 0; i < 9; ++i) {
      xi[3 * i] = t[i][0]; xi[3 * i + 1] = t[i][1]; xi[3 * i + 2] = 0;
      int m = abs(t[i][0]) + abs(t[i][1]);
      w[i] = (m == 0) ? 4.0 / 9.0 : (m == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    return 9;
  }
  if (dim == 3) {
    int t[19][3] = {{0, 0, 0},
                    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
                    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
                    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    for (int i = 0; i < 19; ++i) {
      for (int a = 0; a < 3; ++a) xi[3 * i + a] = t[i][a];
      int m = abs(t[i][0]) + abs(t[i][1]) + abs(t[i][2]);
      w[i] = (m == 0) ? 1.0 / 3.0 : (m == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    return 19;
  }
  return q;
}

/* ------------------------------------------------------------------------ */
/* Eq. (ade-feq) with the 1/2 on the quadratic term; u is the lattice
 * velocity (C times the physical velocity), nu^2 = 1/3.                    */
/* ------------------------------------------------------------------------ */
static double feq_one(double wi, double A, const int* xi, const double* ul)
{
  double cu = xi[0] * ul[0] + xi[1] * ul[1] + xi[2] * ul[2];
  double usq = ul[0] * ul[0] + ul[1] * ul[1] + ul[2] * ul[2];
  double nu2 = 1.0 / 3.0;
  return wi * A * (1.0 + cu / nu2 + (cu * cu) / PLANTED(1, 2.0 * nu2 * nu2, nu2 * nu2) - usq / (2.0 * nu2));
}

void orc_equilibrium(int dim, double A, const double* u_phys, double courant, double* feq)
{
  int xi[ORC_MAXQ * 3]; double w[ORC_MAXQ];
  int Q = orc_stencil(dim, xi, w);
  double ul[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) ul[a] = courant * u_phys[a];
  for (int i = 0; i < Q; ++i) feq[i] = feq_one(w[i], A, &xi[3 * i], ul);
}

/* ------------------------------------------------------------------------ */
/* LEC decode, Sec. 4.1 (Eq. lb-ade-lec-comps-A and the iteration after it). */
/* A = (n, [1 + (1 + D/2) mu (n/gamma)^(2/D)] n p).                          */
/* ------------------------------------------------------------------------ */
int orc_decode_lec(int Ds, int D, double mu, const double* A,
                   double* n_out, double* u_out, double* gamma_out, double* Pi_out)
{
  double n = A[0];
  double p0[3] = {0, 0, 0}, p[3] = {0, 0, 0};
  for (int a = 0; a < Ds; ++a) { p0[a] = A[1 + a] / n; p[a] = p0[a]; }
  double e = 2.0 / (double)D;
  int it;
  for (it = 0; it < 64; ++it) {
    double g = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double H = 1.0 + PLANTED(8, 1.0 + 0.5 * D, 1.0 + 2.0 / D) * mu * pow(n / g, e);
    double dmax = 0.0, pmax = 0.0;
    for (int a = 0; a < 3; ++a) {
      double pn = p0[a] / H;
      double d = fabs(pn - p[a]);
      if (d > dmax) dmax = d;
      p[a] = pn;
      if (fabs(pn) > pmax) pmax = fabs(pn);
    }
    if (dmax <= 1e-15 * pmax) break;
  }
  double g = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  *n_out = n;
  for (int a = 0; a < 3; ++a) u_out[a] = p[a] / g;
  *gamma_out = g;
  *Pi_out = pow(n / g, 1.0 + e);
  return it + 1;
}

/* ------------------------------------------------------------------------ */
/* WARMC decode, Sec. 5.1 (Eq. lb-ade-warmc-comps-A) and App. A:
 * A = (n, n lambda, n lambda u^a, lambda theta^{ab}); lambda = n/h = w^0;
 * theta^{0a} and theta^{00} from U_nu theta^{mu nu} = 0 (Eq. traces4).      */
/* ------------------------------------------------------------------------ */
static void warmc_pairs(int dim, int pairs[6][2], int* np)
{
  static const int p1[1][2] = {{0, 0}};
  static const int p2[4][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}};
  static const int p3[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  const int (*src)[2] = dim == 1 ? p1 : (dim == 2 ? p2 : p3);
  *np = dim == 1 ? 1 : (dim == 2 ? 4 : 6);
  for (int j = 0; j < *np; ++j) { pairs[j][0] = src[j][0]; pairs[j][1] = src[j][1]; }
}

void orc_decode_warmc(int dim, const double* A, double* out /* see header */)
{
  int pairs[6][2], np;
  warmc_pairs(dim, pairs, &np);
  int Ds = dim;
  double n = A[0], nl = A[1];
  double lam = nl / n;
  double u[3] = {0, 0, 0};
  for (int a = 0; a < Ds; ++a) u[a] = A[2 + a] / PLANTED(15, nl, n);
  double th[3][3] = {{0}};
  for (int j = 0; j < np; ++j) {
    double v = A[2 + Ds + j] / lam;
    th[pairs[j][0]][pairs[j][1]] = v;
    th[pairs[j][1]][pairs[j][0]] = v;
  }
  double th0[3];
  for (int a = 0; a < 3; ++a) th0[a] = u[0] * th[a][0] + u[1] * th[a][1] + u[2] * th[a][2];
  double th00 = u[0] * th0[0] + u[1] * th0[1] + u[2] * th0[2];
  /* out layout: n, lam, u[3], gamma, th[3][3] (9), th0[3], th00, w[3] */
  out[0] = n; out[1] = lam;
  for (int a = 0; a < 3; ++a) out[2 + a] = u[a];
  out[5] = 1.0 / sqrt(1.0 - (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[6 + 3 * a + b] = th[a][b];
  for (int a = 0; a < 3; ++a) out[15 + a] = th0[a];
  out[18] = th00;
  for (int a = 0; a < 3; ++a) out[19 + a] = lam * u[a];
}

/* ------------------------------------------------------------------------ */
/* Sources.                                                                 */
/* ------------------------------------------------------------------------ */
static int eps3(int i, int j, int k)
{
  if (i == j || j == k || i == k) return 0;
  /* even permutations of (0,1,2) */
  if ((i == 0 && j == 1 && k == 2) || (i == 1 && j == 2 && k == 0) || (i == 2 && j == 0 && k == 1))
    return 1;
  return -1;
}

/* Eq. (lb-ade-lec-comps-F), q = -1: F_p = -mu grad Pi - n (E + u x B). */
void orc_lec_source(double mu, double n, const double* u, const double* gradPi,
                    const double* E, const double* B, double* Fp)
{
  for (int a = 0; a < 3; ++a) {
    double uxB = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) uxB += eps3(a, k, l) * u[k] * B[l];
    Fp[a] = -mu * gradPi[a] - n * (E[a] + PLANTED(5, uxB, -uxB));
  }
}

/* Eq. (lb-ade-warmc-comps-F) with c = 1, q = -1, written in Cartesian form
 * (App. A without the 1/r terms):
 *   F_{n lambda}    = -d_t th00 - d_k th0k - n E.u
 *   F_{n lambda u_a}= -d_t th0a - d_b th_ab - n (E + u x B)_a
 *   F_{lambda th_ab}= -th0b d_t w_a - th_bk d_k w_a - th0a d_t w_b - th_ak d_k w_b
 *                     - [E_a th0b + E_b th0a + eps_akl th_bk B_l + eps_bkl th_ak B_l]
 * All derivative arrays are supplied by the caller.                        */
void orc_warmc_source(double n, const double* u, const double* th /*[3][3]*/,
                      const double* th0, double dth00_dt, const double* dth0_dt,
                      const double* dw_dt, const double* dth /*[a][b][k]*/,
                      const double* dth0 /*[a][k]*/, const double* dw /*[a][k]*/,
                      const double* E, const double* B,
                      double* F_nl, double* F_nlu /*[3]*/, double* F_th /*[3][3]*/)
{
  double Eu = E[0] * u[0] + E[1] * u[1] + E[2] * u[2];
  *F_nl = -dth00_dt - (dth0[0 * 3 + 0] + dth0[1 * 3 + 1] + dth0[2 * 3 + 2]) - n * Eu;
  for (int a = 0; a < 3; ++a) {
    double uxB = 0.0, divth = 0.0;
    for (int k = 0; k < 3; ++k) {
      for (int l = 0; l < 3; ++l) uxB += eps3(a, k, l) * u[k] * B[l];
      divth += dth[(a * 3 + k) * 3 + k];
    }
    F_nlu[a] = -dth0_dt[a] - divth - n * (E[a] + uxB);
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = -th0[b] * dw_dt[a] - th0[a] * dw_dt[b];
      for (int k = 0; k < 3; ++k)
        s -= th[b * 3 + k] * dw[a * 3 + k] + th[a * 3 + k] * dw[b * 3 + k];
      double em = E[a] * th0[b] + E[b] * th0[a];
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l)
          em += eps3(a, k, l) * th[b * 3 + k] * B[l] + PLANTED(6, eps3(b, k, l) * th[a * 3 + k] * B[l], 0.0);
      F_th[a * 3 + b] = s - em;
    }
}

/* ------------------------------------------------------------------------ */
/* Driver, Eq. (bunch-density) read with rms sizes: n_b = L(zeta) T(r),
 * zeta = z - z0 - t (moves towards +z at c), L = alpha exp(-zeta^2/2sz^2)
 * or a sampled profile with linear interpolation, T = exp(-r^2 / 2 sr^2).  */
/* ------------------------------------------------------------------------ */
/* Sampled profile: sample j sits at zeta_j = (j - (len-1)/2) dz; linear
 * interpolation between samples, with zero samples just outside both ends
 * (so L is continuous and falls to 0 one sample beyond the ends). */
static double profile_sample(const orc_params* p, int j)
{
  return (j >= 0 && j < p->profile_len) ? p->profile[j] : 0.0;
}

static double driver_long(const orc_params* p, double zeta)
{
  if (p->profile && p->profile_len >= 2) {
    double s = zeta / p->profile_dz + 0.5 * (p->profile_len - 1);
    if (!(s > -1.0 && s < (double)p->profile_len)) return 0.0;
    int j = (int)floor(s);
    double fr = s - j;
    return (1.0 - fr) * profile_sample(p, j) + fr * profile_sample(p, j + 1);
  }
  return p->alpha * exp(-zeta * zeta / (2.0 * p->sigma_z * p->sigma_z));
}

static double driver_density(const orc_params* p, double z, double x, double y, double t)
{
  double L = driver_long(p, z - p->z0 + PLANTED(14, -t, t));
  double r2 = 0.0;
  if (p->dim >= 2) r2 += x * x;
  if (p->dim >= 3) r2 += y * y;
  if (p->dim == 1) return L;
  return L * exp(-r2 / (2.0 * p->sigma_r * p->sigma_r));
}

double orc_driver_density(const orc_params* p, double z, double x, double y, double t)
{
  return driver_density(p, z, x, y, t);
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers.                                                        */
/* ------------------------------------------------------------------------ */
static void coords(const orc_state* S, long c, int* i)
{
  i[0] = (int)(c % S->n[0]);
  long r = c / S->n[0];
  i[1] = (int)(r % S->n[1]);
  i[2] = (int)(r / S->n[1]);
}

static long index_of(const orc_state* S, const int* i)
{
  return i[0] + (long)S->n[0] * (i[1] + (long)S->n[1] * i[2]);
}

static int present(const orc_state* S, int axis) { return axis < S->p.dim; }

static int axi(const orc_state* S) { return S->p.geometry == ORC_AXISYMMETRIC; }

/* Axisymmetric: whether set k changes sign under r -> -r (an odd number of
 * r indices: n A_r; n lambda u_r and lambda theta^{rz}). */
static int odd_in_r(const orc_state* S, int k)
{
  if (S->p.closure == ORC_LEC) return k == 2;
  if (k == 3) return 1;
  if (k >= 2 + S->Ds) {
    int j = k - 2 - S->Ds;
    return (S->thpair[j][0] == 1) != (S->thpair[j][1] == 1);
  }
  return 0;
}

/* Node-quantity neighbour (macros, J, B): wrap (periodic) or clamp (open). */
static long nb_node(const orc_state* S, long c, int axis, int delta)
{
  int i[3]; coords(S, c, i);
  int v = i[axis] + delta, n = S->n[axis];
  if (S->p.boundary == ORC_PERIODIC) v = ((v % n) + n) % n;
  else v = v < 0 ? 0 : (v >= n ? n - 1 : v);
  i[axis] = v;
  return index_of(S, i);
}

/* E neighbour: transverse (x, y) out-of-range slots are conducting walls
 * (tangential E = 0) -> returns -1; z clamps; periodic wraps.              */
static long nb_E(const orc_state* S, long c, int axis, int delta)
{
  int i[3]; coords(S, c, i);
  int v = i[axis] + delta, n = S->n[axis];
  if (S->p.boundary == ORC_PERIODIC) v = ((v % n) + n) % n;
  else if (v < 0 || v >= n) {
    if (axis != 0) return -1;
    v = v < 0 ? 0 : n - 1;
  }
  i[axis] = v;
  return index_of(S, i);
}

/* Dual Yee grid: E_a sits half a cell up along both axes other than a,
 * B_a half a cell up along a.  Present E components: 1D {z}; 2D {z, x};
 * 3D all.  Present B: 1D none; 2D {y}; 3D all.                            */
static int E_present(const orc_state* S, int a)
{
  if (S->p.dim == 1) return a == 0;
  if (S->p.dim == 2) return a == 0 || a == 1;
  return 1;
}
static int B_present(const orc_state* S, int a)
{
  if (S->p.dim == 1) return 0;
  if (S->p.dim == 2) return a == 2;
  return 1;
}

/* A slot of E_a on a conducting wall: offset along a transverse axis b and
 * sitting at index n_b - 1 (position n_b - 1/2).                           */
static int E_wall(const orc_state* S, long c, int a)
{
  if (S->p.boundary == ORC_PERIODIC) return 0;
  int i[3]; coords(S, c, i);
  for (int b = 1; b < 3; ++b)
    if (b != a && present(S, b) && i[b] == S->n[b] - 1) return 1;
  /* axisymmetric: E_r vanishes on the axis (odd under r -> -r) */
  if (axi(S) && a == 1 && i[1] == 0) return 1;
  return 0;
}

/* Axisymmetric: B_phi vanishes on the axis. */
static int B_axis(const orc_state* S, long c, int a)
{
  if (!axi(S) || a != 2) return 0;
  int i[3]; coords(S, c, i);
  return i[1] == 0;
}

static void node_pos(const orc_state* S, const int* i, double* pos /* z, x, y */)
{
  double dx = S->p.dx;
  pos[0] = i[0] * dx;
  pos[1] = axi(S) ? i[1] * dx : (i[1] - 0.5 * (S->n[1] - 1)) * dx;
  pos[2] = (i[2] - 0.5 * (S->n[2] - 1)) * dx;
}

static double Eget(const orc_state* S, const double* E, int a, long idx)
{
  (void)S;
  return idx < 0 ? 0.0 : E[(long)a * S->ncell + idx];
}

/* ------------------------------------------------------------------------ */
/* Creation and state.                                                      */
/* ------------------------------------------------------------------------ */
static double warmc_h0(int D, double mu)
{
  /* Eq. (traces3) at rest (theta^{00} = 0, theta^{ij} = mu delta^{ij} over
   * the D kinetic dimensions, n0 = 1): h^2 + D mu h - 1 = 0, positive root. */
  return 2.0 / (D * mu + sqrt(D * D * mu * mu + 4.0));
}

static void init_fields(orc_state* S);

orc_state* orc_create(const orc_params* p, int* status)
{
  *status = -1;
  if (p->dim < 1 || p->dim > 3) return NULL;
  int nn[3] = {p->nz, p->dim >= 2 ? p->nx : 1, p->dim >= 3 ? p->ny : 1};
  for (int a = 0; a < p->dim; ++a) if (nn[a] < 3) return NULL;
  if (!(p->dx > 0) || !(p->courant > 0) || !(p->tau > 0.5)) return NULL;
  if (p->closure != ORC_LEC && p->closure != ORC_WARMC) return NULL;
  if (p->dv != 1 && p->dv != 3) return NULL;
  if (!(p->mu >= 0)) return NULL;
  if (p->dim >= 2 && !(p->sigma_r > 0)) return NULL;
  if (!p->profile && !(p->sigma_z > 0)) return NULL;
  if (p->geometry != ORC_CARTESIAN && p->geometry != ORC_AXISYMMETRIC) return NULL;
  if (p->geometry == ORC_AXISYMMETRIC && (p->dim != 2 || p->boundary != ORC_OPEN)) return NULL;

  orc_state* S = (orc_state*)calloc(1, sizeof(orc_state));
  S->p = *p;
  if (p->profile && p->profile_len > 0) {
    double* pr = (double*)malloc(sizeof(double) * p->profile_len);
    memcpy(pr, p->profile, sizeof(double) * p->profile_len);
    S->p.profile = pr;
  } else {
    S->p.profile = NULL;
  }
  for (int a = 0; a < 3; ++a) S->n[a] = nn[a];
  S->ncell = (long)nn[0] * nn[1] * nn[2];
  S->Ds = p->dim;
  S->dt = p->courant * p->dx;
  int xi[ORC_MAXQ * 3];
  S->Q = orc_stencil(p->dim, xi, S->w);
  for (int i = 0; i < S->Q; ++i)
    for (int a = 0; a < 3; ++a) S->xi[i][a] = xi[3 * i + a];
  for (int i = 0; i < S->Q; ++i)
    for (int j = 0; j < S->Q; ++j)
      if (S->xi[j][0] == S->xi[i][0] && S->xi[j][1] == -S->xi[i][1] && S->xi[j][2] == S->xi[i][2]) S->mir[i] = j;
  if (p->closure == ORC_LEC) {
    S->K = 1 + S->Ds;
    S->ntheta = 0;
    S->Arest[0] = 1.0;
    for (int a = 0; a < S->Ds; ++a) S->Arest[1 + a] = 0.0;
  } else {
    warmc_pairs(p->dim, S->thpair, &S->ntheta);
    S->K = 2 + S->Ds + S->ntheta;
    double lam0 = 1.0 / warmc_h0(p->dv, p->mu);
    S->Arest[0] = 1.0;
    S->Arest[1] = lam0;
    for (int a = 0; a < S->Ds; ++a) S->Arest[2 + a] = 0.0;
    for (int j = 0; j < S->ntheta; ++j) {
      int a = S->thpair[j][0], b = S->thpair[j][1];
      double th = (a == b && (p->dv == 3 || a == 0)) ? p->mu : 0.0;
      S->Arest[2 + S->Ds + j] = lam0 * th;
    }
  }
  long nc = S->ncell;
  S->f = (double*)calloc((size_t)S->K * S->Q * nc, sizeof(double));
  S->fs = (double*)calloc((size_t)S->K * S->Q * nc, sizeof(double));
  S->E = (double*)calloc(3 * (size_t)nc, sizeof(double));
  S->B = (double*)calloc(3 * (size_t)nc, sizeof(double));
  S->En = (double*)calloc(3 * (size_t)nc, sizeof(double));
  S->Bn = (double*)calloc(3 * (size_t)nc, sizeof(double));
  S->prev = (double*)calloc(7 * (size_t)nc, sizeof(double));
  S->mac = (orc_macro*)calloc((size_t)nc, sizeof(orc_macro));
  S->F = (double*)calloc((size_t)S->K * nc, sizeof(double));
  if (!S->f || !S->fs || !S->E || !S->B || !S->En || !S->Bn || !S->prev || !S->mac || !S->F) {
    orc_destroy(S);
    *status = -2;
    return NULL;
  }
  /* rest state: f = f^eq(A_rest, u = 0) = w_i A_rest */
  for (int k = 0; k < S->K; ++k)
    for (int i = 0; i < S->Q; ++i)
      for (long c = 0; c < nc; ++c)
        S->f[((size_t)k * S->Q + i) * nc + c] = S->w[i] * S->Arest[k];
  if (p->init_fields) init_fields(S);
  S->fields_from_driver = p->init_fields && p->dim >= 2;
  S->have_prev = 0;
  S->step = 0;
  *status = 0;
  return S;
}

void orc_destroy(orc_state* S)
{
  if (!S) return;
  free((void*)S->p.profile);
  free(S->f); free(S->fs); free(S->E); free(S->B); free(S->En); free(S->Bn);
  free(S->prev); free(S->mac); free(S->F);
  free(S);
}

void orc_sizes(const orc_state* S, int* K, int* Q, long* ncell)
{
  *K = S->K; *Q = S->Q; *ncell = S->ncell;
}

long orc_get_step(const orc_state* S) { return S->step; }
double orc_get_dt(const orc_state* S) { return S->dt; }
void orc_rest_advected(const orc_state* S, double* A) { for (int k = 0; k < S->K; ++k) A[k] = S->Arest[k]; }

/* Initial fields, Sec. 6 (rigid bunch solved in its rest frame and boosted):
 * the v -> c limit, E_z = 0, E_perp = -grad_perp psi with
 * div_perp E_perp = -n_b, B = z x E.  E is taken at t = -dt/2, B at t = 0. */
static void init_fields(orc_state* S)
{
  const orc_params* p = &S->p;
  long nc = S->ncell;
  memset(S->E, 0, sizeof(double) * 3 * nc);
  memset(S->B, 0, sizeof(double) * 3 * nc);
  if (p->dim == 1) return;
  double sr = p->sigma_r, dx = p->dx;
  for (long c = 0; c < nc; ++c) {
    int i[3]; coords(S, c, i);
    double pos[3]; node_pos(S, i, pos);
    if (p->dim == 2 && axi(S)) {
      /* E_r = -L sr^2 (1 - exp(-r^2/2sr^2)) / r at the E_r slot (z + dx/2, r),
       * B_phi = E_r at the node (z, r), t = 0. */
      double tE = -0.5 * S->dt, r = pos[1];
      double s = r * r / (2.0 * sr * sr);
      double fr = s > 0 ? -expm1(-s) / (2.0 * s) : 0.5;
      S->E[1 * nc + c] = -driver_long(p, pos[0] + 0.5 * dx - p->z0 - tE) * r * fr;
      S->B[2 * nc + c] = -driver_long(p, pos[0] - p->z0) * r * fr;
    } else if (p->dim == 2) {
      /* E_x slot: (z + dx/2, x);  B_y at the node. */
      double tE = -0.5 * S->dt;
      double Lx = driver_long(p, pos[0] + 0.5 * dx - p->z0 - tE);
      double Ex = -Lx * sr * sqrt(M_PI / 2.0) * erf(pos[1] / (sqrt(2.0) * sr));
      S->E[1 * nc + c] = Ex;
      double LB = driver_long(p, pos[0] - p->z0);
      S->B[2 * nc + c] = -LB * sr * sqrt(M_PI / 2.0) * erf(pos[1] / (sqrt(2.0) * sr));
    } else {
      /* E_r = -L sr^2 (1 - exp(-r^2/2sr^2)) / r; E_a = E_r x_a / r. */
      double tE = -0.5 * S->dt;
      /* E_x slot at (x, y + dx/2, z + dx/2) */
      {
        double z = pos[0] + PLANTED(18, 0.5 * dx, 0.0), x = pos[1], y = pos[2] + 0.5 * dx;
        double s = (x * x + y * y) / (2.0 * sr * sr);
        double fr = s > 0 ? -expm1(-s) / (2.0 * s) : 0.5;
        S->E[1 * nc + c] = -driver_long(p, z - p->z0 - tE) * x * fr;
      }
      /* E_y slot at (x + dx/2, y, z + dx/2) */
      {
        double z = pos[0] + 0.5 * dx, x = pos[1] + 0.5 * dx, y = pos[2];
        double s = (x * x + y * y) / (2.0 * sr * sr);
        double fr = s > 0 ? -expm1(-s) / (2.0 * s) : 0.5;
        S->E[2 * nc + c] = -driver_long(p, z - p->z0 - tE) * y * fr;
      }
      /* B_x slot at (x + dx/2, y, z): B_x = -E_y there, t = 0 */
      {
        double z = pos[0], x = pos[1] + 0.5 * dx, y = pos[2];
        double s = (x * x + y * y) / (2.0 * sr * sr);
        double fr = s > 0 ? -expm1(-s) / (2.0 * s) : 0.5;
        S->B[1 * nc + c] = driver_long(p, z - p->z0) * y * fr;
      }
      /* B_y slot at (x, y + dx/2, z): B_y = E_x there, t = 0 */
      {
        double z = pos[0], x = pos[1], y = pos[2] + 0.5 * dx;
        double s = (x * x + y * y) / (2.0 * sr * sr);
        double fr = s > 0 ? -expm1(-s) / (2.0 * s) : 0.5;
        S->B[2 * nc + c] = -driver_long(p, z - p->z0) * x * fr;
      }
    }
  }
  for (long c = 0; c < nc; ++c)
    for (int a = 0; a < 3; ++a) {
      if (E_wall(S, c, a)) S->E[(long)a * nc + c] = 0.0;
      if (B_axis(S, c, a)) S->B[(long)a * nc + c] = 0.0;
    }
}

/* Nearest bulk node of c (Eq. open-bc); identity for periodic domains. */
static long bulk_of(const orc_state* S, long c)
{
  if (S->p.boundary == ORC_PERIODIC) return c;
  int i[3]; coords(S, c, i);
  for (int a = 0; a < S->p.dim; ++a) {
    if (i[a] < 1) i[a] = 1;
    if (i[a] > S->n[a] - 2) i[a] = S->n[a] - 2;
  }
  return index_of(S, i);
}

/* Velocity whose population a boundary node c takes from its bulk node for
 * set k: i itself (Eq. open-bc), or on the axis of an axisymmetric domain
 * the mirrored velocity for sets odd under r -> -r (Eq. reflective-bc). */
static int boundary_dir(const orc_state* S, long c, int k, int i)
{
  if (!axi(S) || !odd_in_r(S, k)) return i;
  int ic[3]; coords(S, c, ic);
  return ic[1] == 0 ? S->mir[i] : i;
}

void orc_set_state(orc_state* S, const double* f, const double* E, const double* B)
{
  long nc = S->ncell;
  if (f) {
    for (int k = 0; k < S->K; ++k)
      for (int i = 0; i < S->Q; ++i)
        for (long c = 0; c < nc; ++c) {
          size_t src = ((size_t)k * S->Q + boundary_dir(S, c, k, i)) * nc;
          S->f[((size_t)k * S->Q + i) * nc + c] = f[src + bulk_of(S, c)];
        }
  }
  if (E || B) S->fields_from_driver = 0;
  if (E) {
    memcpy(S->E, E, sizeof(double) * 3 * nc);
    for (long c = 0; c < nc; ++c)
      for (int a = 0; a < 3; ++a)
        if (!E_present(S, a) || E_wall(S, c, a)) S->E[(long)a * nc + c] = 0.0;
  }
  if (B) {
    memcpy(S->B, B, sizeof(double) * 3 * nc);
    for (long c = 0; c < nc; ++c)
      for (int a = 0; a < 3; ++a)
        if (!B_present(S, a) || B_axis(S, c, a)) S->B[(long)a * nc + c] = 0.0;
  }
  S->have_prev = 0;
}

void orc_get_state(const orc_state* S, double* f, double* E, double* B)
{
  long nc = S->ncell;
  if (f) memcpy(f, S->f, sizeof(double) * (size_t)S->K * S->Q * nc);
  if (E) memcpy(E, S->E, sizeof(double) * 3 * nc);
  if (B) memcpy(B, S->B, sizeof(double) * 3 * nc);
}

/* ------------------------------------------------------------------------ */
/* One time step (Sec. 2.1 algorithm: source/collision, streaming, moments;
 * Sec. 4.1 coupling to the FDTD Maxwell solver).  State at entry: f^n, E at
 * t_{n-1/2}, B at t_n.
 *  (1) decode every node: A_k = sum_i f_ki (Eq. disc-moments-ade), closure
 *  (2) E^{n+1/2} = E^{n-1/2} + dt (curl B^n + n u + n_b(t_n) z)
 *  (3) B^{n+1}   = B^n - dt curl E^{n+1/2}
 *  (4) sources F^n with E^{n+1/2}, B^n averaged to the node
 *  (5) BGK relaxation + source w_i dt F (Eq. lbe, lsource), then pull
 *      streaming and the open-boundary copy (Eq. open-bc)
 *  (6) keep this step's theta^{0b}, w^a for the next backward difference.  */
/* ------------------------------------------------------------------------ */
static void decode_node(const orc_state* S, long c, orc_macro* m)
{
  long nc = S->ncell;
  double A[11];
  for (int k = 0; k < S->K; ++k) {
    double s = 0.0;
    for (int i = 0; i < S->Q; ++i) s += S->f[((size_t)k * S->Q + i) * nc + c];
    A[k] = s;
  }
  memset(m, 0, sizeof(*m));
  if (S->p.closure == ORC_LEC) {
    orc_decode_lec(S->Ds, S->p.dv, S->p.mu, A, &m->n, m->u, &m->gamma, &m->Pi);
  } else {
    double o[22];
    orc_decode_warmc(S->p.dim, A, o);
    m->n = o[0]; m->lam = o[1];
    for (int a = 0; a < 3; ++a) m->u[a] = o[2 + a];
    m->gamma = o[5];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) m->th[a][b] = o[6 + 3 * a + b];
    for (int a = 0; a < 3; ++a) m->th0[a] = o[15 + a];
    m->th00 = o[18];
    for (int a = 0; a < 3; ++a) m->w[a] = o[19 + a];
  }
}

/* E^{n+1/2} (S->En) and B^n (S->B) averaged to node c. */
static void node_fields(const orc_state* S, long c, double* En, double* Bn)
{
  long nc = S->ncell;
  for (int a = 0; a < 3; ++a) {
    En[a] = 0.0;
    Bn[a] = 0.0;
    if (E_present(S, a)) {
      int b = (a + 1) % 3, d = (a + 2) % 3;
      int off[2], no = 0;
      if (present(S, b)) off[no++] = b;
      if (present(S, d)) off[no++] = d;
      double s = 0.0;
      for (int q = 0; q < (1 << no); ++q) {
        long cc = c;
        for (int j = 0; j < no && cc >= 0; ++j)
          if (q & (1 << j)) {
            long nb = nb_E(S, cc, off[j], -1);
            /* axisymmetric: the E_z slot below the axis mirrors the one above */
            if (nb < 0 && axi(S) && a == 0 && off[j] == 1) nb = cc;
            cc = nb;
          }
        s += Eget(S, S->En, a, cc);
      }
      En[a] = s / (double)(1 << no);
    }
    if (B_present(S, a)) {
      if (present(S, a))
        Bn[a] = 0.5 * (S->B[(long)a * nc + c] + S->B[(long)a * nc + nb_node(S, c, a, -1)]);
      else
        Bn[a] = S->B[(long)a * nc + c];
    }
  }
}

/* Stages (1)-(5a) of a step: decoded macros, E^{n+1/2} (En), B^{n+1} (Bn),
 * sources (F) and post-collision populations (fs); the state is unchanged. */
static void forward_stages(orc_state* S)
{
  const orc_params* p = &S->p;
  long nc = S->ncell;
  double dt = S->dt, dx = p->dx;
  double t = S->step * dt;
  int K = S->K, Q = S->Q;

  /* (1) decode */
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) decode_node(S, c, &S->mac[c]);

  /* (2) E^{n+1/2} */
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    int i[3]; coords(S, c, i);
    double pos[3]; node_pos(S, i, pos);
    for (int a = 0; a < 3; ++a) {
      long ia = (long)a * nc + c;
      if (!E_present(S, a)) { S->En[ia] = 0.0; continue; }
      if (E_wall(S, c, a)) { S->En[ia] = 0.0; continue; }
      int b = (a + 1) % 3, d = (a + 2) % 3;
      /* (curl B)_a = d_b B_d - d_d B_b at the E_a slot */
      double curl = 0.0;
      if (a == 0 && axi(S)) {
        /* (curl B)_z = (1/r) d_r (r B_phi) at r_{j+1/2}, B_phi at r_j, r_{j+1} */
        double rl = i[1] * dx, rh = rl + dx, rm = rl + 0.5 * dx;
        curl += PLANTED(9, (rh * S->B[(long)d * nc + nb_node(S, c, b, +1)] - rl * S->B[(long)d * nc + c]) / (rm * dx),
                        (S->B[(long)d * nc + nb_node(S, c, b, +1)] - S->B[(long)d * nc + c]) / dx);
      } else if (present(S, b) && B_present(S, d))
        curl += (S->B[(long)d * nc + nb_node(S, c, b, +1)] - S->B[(long)d * nc + c]) / dx;
      if (present(S, d) && B_present(S, b))
        curl -= (S->B[(long)b * nc + nb_node(S, c, d, +1)] - S->B[(long)b * nc + c]) / dx;
      /* n u_a averaged over the nodes around the slot */
      int off[2], no = 0;
      if (present(S, b)) off[no++] = b;
      if (present(S, d)) off[no++] = d;
      double J = 0.0;
      for (int s = 0; s < (1 << no); ++s) {
        long cc = c;
        for (int j = 0; j < no; ++j)
          if (s & (1 << j)) cc = nb_node(S, cc, off[j], +1);
        J += S->mac[cc].n * S->mac[cc].u[a];
      }
      J /= (double)(1 << no);
      if (a == 0) {
        double q[3] = {pos[0], pos[1], pos[2]};
        for (int j = 0; j < no; ++j) q[off[j]] += 0.5 * dx;
        J += driver_density(p, q[0], q[1], q[2], t);
      }
      S->En[ia] = S->E[ia] + dt * PLANTED(3, curl + J, curl - J);
    }
  }

  /* (3) B^{n+1} */
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    for (int a = 0; a < 3; ++a) {
      long ia = (long)a * nc + c;
      if (!B_present(S, a) || B_axis(S, c, a)) { S->Bn[ia] = 0.0; continue; }
      int b = (a + 1) % 3, d = (a + 2) % 3;
      /* (curl E)_a = d_b E_d - d_d E_b at the B_a slot */
      double curl = 0.0;
      if (present(S, b) && E_present(S, d))
        curl += (Eget(S, S->En, d, c) - Eget(S, S->En, d, nb_E(S, c, b, -1))) / dx;
      if (present(S, d) && E_present(S, b))
        curl -= (Eget(S, S->En, b, c) - Eget(S, S->En, b, nb_E(S, c, d, -1))) / dx;
      S->Bn[ia] = S->B[ia] + PLANTED(4, -dt, dt) * curl;
    }
  }

  /* (4) sources */
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    const orc_macro* m = &S->mac[c];
    double En[3], Bn[3];
    node_fields(S, c, En, Bn);
    double Fk[11] = {0};
    if (p->closure == ORC_LEC) {
      double gPi[3] = {0, 0, 0};
      for (int a = 0; a < S->Ds; ++a)
        gPi[a] = (S->mac[nb_node(S, c, a, +1)].Pi - S->mac[nb_node(S, c, a, -1)].Pi) / (2.0 * dx);
      double Fp[3];
      orc_lec_source(p->mu, m->n, m->u, gPi, En, Bn, Fp);
      Fk[0] = 0.0;
      for (int a = 0; a < S->Ds; ++a) Fk[1 + a] = Fp[a];
    } else {
      double dth[27] = {0}, dth0[9] = {0}, dw[9] = {0};
      for (int k = 0; k < S->Ds; ++k) {
        const orc_macro* mp = &S->mac[nb_node(S, c, k, +1)];
        const orc_macro* mm = &S->mac[nb_node(S, c, k, -1)];
        for (int a = 0; a < 3; ++a) {
          for (int b = 0; b < 3; ++b)
            dth[(a * 3 + b) * 3 + k] = (mp->th[a][b] - mm->th[a][b]) / (2.0 * dx);
          dth0[a * 3 + k] = (mp->th0[a] - mm->th0[a]) / (2.0 * dx);
          dw[a * 3 + k] = (mp->w[a] - mm->w[a]) / (2.0 * dx);
        }
      }
      double dth00_dt = 0.0, dth0_dt[3] = {0, 0, 0}, dw_dt[3] = {0, 0, 0};
      if (S->have_prev) {
        dth00_dt = (m->th00 - S->prev[0 * nc + c]) / dt;
        for (int a = 0; a < 3; ++a) {
          dth0_dt[a] = PLANTED(17, (m->th0[a] - S->prev[(long)(1 + a) * nc + c]) / dt, 0.0);
          dw_dt[a] = (m->w[a] - S->prev[(long)(4 + a) * nc + c]) / dt;
        }
      }
      double Fnl, Fnlu[3], Fth[9];
      orc_warmc_source(m->n, m->u, &m->th[0][0], m->th0, dth00_dt, dth0_dt, dw_dt,
                       dth, dth0, dw, En, Bn, &Fnl, Fnlu, Fth);
      Fk[0] = 0.0;
      Fk[1] = Fnl;
      for (int a = 0; a < S->Ds; ++a) Fk[2 + a] = Fnlu[a];
      for (int j = 0; j < S->ntheta; ++j)
        Fk[2 + S->Ds + j] = Fth[S->thpair[j][0] * 3 + S->thpair[j][1]];
    }
    if (axi(S)) {
      int ic[3]; coords(S, c, ic);
      if (ic[1] > 0) {
        /* App. A: the 1/r terms of the cylindrical divergence (index 1 = r,
         * 2 = phi, 0 = z; c = 1) */
        double r = ic[1] * dx, ur = m->u[1];
        if (p->closure == ORC_LEC) {
          /* D(n) = -u_r n / r;  D(n A_a) = -u_r (n A_a) / r */
          double A[3] = {0, 0, 0};
          for (int k = 0; k < K; ++k)
            for (int i = 0; i < Q; ++i) A[k] += S->f[((size_t)k * Q + i) * nc + c];
          for (int k = 0; k < K; ++k) Fk[k] += PLANTED(11, -ur, ur) * A[k] / r;
        } else {
          double n = m->n, nl = m->n * m->lam;
          Fk[0] += -n * ur / r;
          Fk[1] += -nl * ur / r - m->th0[1] / r;
          Fk[2] += -nl * m->u[0] * ur / r - m->th[0][1] / r;        /* n lambda u_z */
          Fk[3] += -nl * ur * ur / r - PLANTED(10, m->th[1][1] - m->th[2][2], m->th[1][1] + m->th[2][2]) / r;  /* n lambda u_r */
          for (int j = 0; j < S->ntheta; ++j) {
            int a = S->thpair[j][0], b = S->thpair[j][1];
            double coef = (a == 2 && b == 2) ? 3.0 : 1.0;  /* lambda theta^{phi phi}: 3 */
            Fk[2 + S->Ds + j] += -coef * m->lam * m->th[a][b] * ur / r;
          }
        }
      }
    }
    for (int k = 0; k < K; ++k) S->F[(long)k * nc + c] = Fk[k];
  }

  /* (5a) BGK + source */
  double C = p->courant, tau = p->tau;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    const orc_macro* m = &S->mac[c];
    double ul[3] = {0, 0, 0};
    for (int a = 0; a < S->Ds; ++a) ul[a] = C * m->u[a];
    for (int k = 0; k < K; ++k) {
      double A = 0.0;
      for (int i = 0; i < Q; ++i) A += S->f[((size_t)k * Q + i) * nc + c];
      for (int i = 0; i < Q; ++i) {
        size_t ix = ((size_t)k * Q + i) * nc + c;
        double fe = feq_one(S->w[i], A, S->xi[i], ul);
        S->fs[ix] = S->f[ix] - (S->f[ix] - fe) / tau + S->w[i] * PLANTED(7, dt, 1.0) * S->F[(long)k * nc + c];
      }
    }
  }

}

/* Stages (5b) and (6): pull streaming into the state and the time advance. */
static void finish_step(orc_state* S)
{
  const orc_params* p = &S->p;
  long nc = S->ncell;
  int K = S->K, Q = S->Q;
  /* (5b) pull streaming with the open-boundary copy */
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    long cb = bulk_of(S, c);
    int ib[3]; coords(S, cb, ib);
    for (int k = 0; k < K; ++k)
      for (int i = 0; i < Q; ++i) {
        int ii = boundary_dir(S, c, k, i);
        int src[3] = {ib[0], ib[1], ib[2]};
        for (int a = 0; a < S->p.dim; ++a) {
          int v = PLANTED(2, src[a] - S->xi[ii][a], src[a] + S->xi[ii][a]), n = S->n[a];
          if (p->boundary == ORC_PERIODIC) v = ((v % n) + n) % n;
          src[a] = v;
        }
        long cs = index_of(S, src);
        S->f[((size_t)k * Q + i) * nc + c] = S->fs[((size_t)k * Q + ii) * nc + cs];
      }
  }

  /* (6) */
  if (p->closure == ORC_WARMC) {
    for (long c = 0; c < nc; ++c) {
      const orc_macro* m = &S->mac[c];
      S->prev[0 * nc + c] = m->th00;
      for (int a = 0; a < 3; ++a) {
        S->prev[(long)(1 + a) * nc + c] = m->th0[a];
        S->prev[(long)(4 + a) * nc + c] = m->w[a];
      }
    }
    S->have_prev = 1;
  }
  memcpy(S->E, S->En, sizeof(double) * 3 * nc);
  memcpy(S->B, S->Bn, sizeof(double) * 3 * nc);
  S->step += 1;
}

static void step_once(orc_state* S)
{
  forward_stages(S);
  finish_step(S);
}

void orc_step(orc_state* S, long nsteps)
{
  for (long s = 0; s < nsteps; ++s) step_once(S);
}

/* ------------------------------------------------------------------------ */
/* Outputs.                                                                 */
/* ------------------------------------------------------------------------ */
void orc_advected(const orc_state* S, double* A)
{
  long nc = S->ncell;
  for (int k = 0; k < S->K; ++k)
    for (long c = 0; c < nc; ++c) {
      double s = 0.0;
      for (int i = 0; i < S->Q; ++i) s += S->f[((size_t)k * S->Q + i) * nc + c];
      A[(long)k * nc + c] = s;
    }
}

/* Rest-frame pressures of the WARMC tensor (App. A, the axisymmetric
 * inversion, read with r -> x and phi -> y, c = 1): P_perp = theta^{yy} and
 * P_par = [theta^{xx} + theta^{zz} - theta^{00} u^2 - theta^{yy} (1 + u_x^2)]
 * / (1 + u_z^2), with theta^{00} = u_i u_j theta^{ij} (the mass-shell rows).
 * th is [3][3] in the order z, x, y; u = (u_z, u_x, u_y); out = {P_par,
 * P_perp}.                                                                 */
void orc_rest_pressures(const double* th, const double* u, double* out)
{
  double t00 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) t00 += u[i] * u[j] * th[3 * i + j];
  const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  out[1] = th[8];
  out[0] = (th[4] + th[0] - t00 * u2 - th[8] * (1.0 + u[1] * u[1])) / (1.0 + u[0] * u[0]);
}

/* Bits: 0 n, 1 u_z, 2 u_x, 3 u_y, 4 gamma, 5 p_z, 6 p_x, 7 p_y (gamma u),
 * 8 LEC rest-frame pressure P0 = mu (n/gamma)^(1+2/D), 9 lambda (WARMC),
 * 10..15 theta zz, xx, yy, zx, zy, xy (WARMC), 16 P_par and 17 P_perp
 * (WARMC in 2D: orc_rest_pressures; 0 otherwise).  Output [bit][cell] in
 * increasing bit order.                                                    */
int orc_moments(const orc_state* S, unsigned mask, double* dst)
{
  long nc = S->ncell;
  int nout = 0;
  for (int b = 0; b < 18; ++b) {
    if (!(mask & (1u << b))) continue;
    for (long c = 0; c < nc; ++c) {
      orc_macro m; decode_node(S, c, &m);
      double v = 0.0;
      switch (b) {
        case 0: v = m.n; break;
        case 1: v = m.u[0]; break;
        case 2: v = m.u[1]; break;
        case 3: v = m.u[2]; break;
        case 4: v = m.gamma; break;
        case 5: v = m.gamma * m.u[0]; break;
        case 6: v = m.gamma * m.u[1]; break;
        case 7: v = m.gamma * m.u[2]; break;
        case 8: v = S->p.closure == ORC_LEC ? S->p.mu * m.Pi : 0.0; break;
        case 9: v = m.lam; break;
        case 10: v = m.th[0][0]; break;
        case 11: v = m.th[1][1]; break;
        case 12: v = m.th[2][2]; break;
        case 13: v = m.th[0][1]; break;
        case 14: v = m.th[0][2]; break;
        case 15: v = m.th[1][2]; break;
        case 16:
        case 17:
          if (S->p.closure == ORC_WARMC && S->p.dim == 2) {
            double th9[9], pr[2];
            for (int i = 0; i < 3; ++i)
              for (int j = 0; j < 3; ++j) th9[3 * i + j] = m.th[i][j];
            orc_rest_pressures(th9, m.u, pr);
            v = pr[b - 16];
          }
          break;
      }
      dst[(long)nout * nc + c] = v;
    }
    ++nout;
  }
  return nout;
}

/* out[0] = sum n, out[1] = sum n_b(t_n) over nodes, out[2] = number of
 * non-finite populations.                                                  */
void orc_reduce(const orc_state* S, double* out)
{
  long nc = S->ncell;
  double sn = 0.0, sb = 0.0, bad = 0.0;
  double t = S->step * S->dt;
  for (long c = 0; c < nc; ++c) {
    double n = 0.0;
    for (int i = 0; i < S->Q; ++i) {
      double v = S->f[(size_t)i * nc + c];
      n += v;
    }
    sn += n;
    int ii[3]; coords(S, c, ii);
    double pos[3]; node_pos(S, ii, pos);
    sb += driver_density(&S->p, pos[0], pos[1], pos[2], t);
  }
  for (size_t j = 0; j < (size_t)S->K * S->Q * nc; ++j)
    if (!isfinite(S->f[j])) bad += 1.0;
  out[0] = sn; out[1] = sb; out[2] = bad;
}

/* ======================================================================== */
/* Discrete adjoint (FP64), 1D and 2D.                                        */
/*                                                                          */
/* J = E_z at one slot after N steps from the current state.  The driver     */
/* parameters enter a step only through n_b in the E_z update (step 2) and  */
/* the initial fields; every other stage is transposed one by one, in       */
/* reverse order: streaming (a push), collision, sources (their gradient     */
/* stencils become scatters to the neighbours), the node averages of E and  */
/* B, the B and E updates, and the closure decode (LEC: implicit            */
/* differentiation of the converged fixed point, Sec. 4.1; WARMC: chain     */
/* rule through Eq. lb-ade-warmc-comps-A and the mass-shell components).    */
/* ======================================================================== */
typedef struct {
  double *lf, *lE, *lB, *lprev;     /* adjoint of the state (f^n, E, B, prev) */
  double *lfs, *lA, *lF, *lEn;      /* adjoint of stage quantities */
  orc_macro *lm;                    /* adjoint of the decoded quantities */
} orc_adj;

/* ∂n_b/∂theta at (z, x, y, t): theta = (alpha, sigma_z, sigma_r) Gaussian, or
 * the profile samples (gp, weights added) and sigma_r. */
static void driver_grad(const orc_params* p, double z, double x, double y, double t, double scale,
                        double* g3, double* gp)
{
  double zeta = z - p->z0 - t;
  double T = 1.0, r2 = 0.0;
  if (p->dim >= 2) {
    r2 = x * x + (p->dim >= 3 ? y * y : 0.0);
    T = exp(-r2 / (2.0 * p->sigma_r * p->sigma_r));
  }
  double L = driver_long(p, zeta);
  if (p->profile && p->profile_len >= 2) {
    double s = zeta / p->profile_dz + 0.5 * (p->profile_len - 1);
    if (s > -1.0 && s < (double)p->profile_len) {
      int j = (int)floor(s);
      double fr = s - j;
      if (j >= 0) gp[j] += scale * T * (1.0 - fr);
      if (j + 1 < p->profile_len) gp[j + 1] += scale * T * fr;
    }
  } else {
    double sz = p->sigma_z;
    g3[0] += scale * T * exp(-zeta * zeta / (2.0 * sz * sz));
    g3[1] += scale * L * T * zeta * zeta / (sz * sz * sz);
  }
  if (p->dim >= 2) {
    double sr = p->sigma_r;
    g3[2] += scale * L * T * r2 / (sr * sr * sr);
  }
}

/* LEC decode transposed (implicit function theorem at the fixed point
 * n H(n, gamma(p)) p = A_p; H = 1 + (1 + D/2) mu (n/gamma)^(2/D)). */
static void adj_decode_lec(const orc_state* S, long c, const double* A, const orc_macro* m,
                           const orc_macro* lm, double* lA)
{
  int Ds = S->Ds;
  double D = S->p.dv, e = 2.0 / D, cH = (1.0 + 0.5 * D) * S->p.mu;
  double n = A[0], g = m->gamma, x = n / g;
  double p[3] = {0, 0, 0};
  for (int a = 0; a < Ds; ++a) p[a] = g * m->u[a];
  double xe = pow(x, e), H = 1.0 + cH * xe;
  double lp[3] = {0, 0, 0};
  for (int b = 0; b < Ds; ++b) {
    double s = 0.0;
    for (int a = 0; a < Ds; ++a) s += lm->u[a] * ((a == b ? 1.0 / g : 0.0) - p[a] * p[b] / (g * g * g));
    lp[b] = s - lm->Pi * (1.0 + e) * m->Pi * p[b] / (g * g);
  }
  double ln = lm->n + lm->Pi * (1.0 + e) * xe / g;
  double beta = cH * e * xe / (g * g), pp = 0.0, pl = 0.0;
  for (int a = 0; a < Ds; ++a) { pp += p[a] * p[a]; pl += p[a] * lp[a]; }
  for (int a = 0; a < Ds; ++a) {
    double mu_a = (lp[a] + beta * p[a] * pl / (H - beta * pp)) / (n * H);
    lA[(long)(1 + a) * S->ncell + c] += mu_a;
    ln -= mu_a * p[a] * (H + cH * e * xe);
  }
  lA[c] += ln;
}

/* WARMC decode transposed (Eq. lb-ade-warmc-comps-A, traces4). */
static void adj_decode_warmc(const orc_state* S, long c, const double* A, const orc_macro* m,
                             orc_macro* lm, double* lA)
{
  long nc = S->ncell;
  int Ds = S->Ds;
  double n = A[0], nl = A[1];
  /* theta00 = u . theta0 */
  for (int a = 0; a < 3; ++a) { lm->u[a] += lm->th00 * m->th0[a]; lm->th0[a] += lm->th00 * m->u[a]; }
  /* theta0_a = sum_b u_b theta_ab */
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      lm->u[b] += lm->th0[a] * m->th[a][b];
      lm->th[a][b] += lm->th0[a] * m->u[b];
    }
  /* w_a = A_{2+a} / n */
  for (int a = 0; a < Ds; ++a) {
    lA[(long)(2 + a) * nc + c] += lm->w[a] / n;
    lA[c] -= lm->w[a] * A[2 + a] / (n * n);
  }
  /* u_a = A_{2+a} / A_1 */
  for (int a = 0; a < Ds; ++a) {
    lA[(long)(2 + a) * nc + c] += lm->u[a] / nl;
    lA[1 * nc + c] -= lm->u[a] * A[2 + a] / (nl * nl);
  }
  /* theta_pair = A_theta n / A_1 */
  for (int j = 0; j < S->ntheta; ++j) {
    int a = S->thpair[j][0], b = S->thpair[j][1];
    double l = lm->th[a][b] + (a != b ? PLANTED(16, lm->th[b][a], 0.0) : 0.0);
    double At = A[2 + Ds + j];
    lA[(long)(2 + Ds + j) * nc + c] += l * n / nl;
    lA[c] += l * At / nl;
    lA[1 * nc + c] -= l * At * n / (nl * nl);
  }
  /* lambda = A_1 / n */
  lA[1 * nc + c] += lm->lam / n;
  lA[c] -= lm->lam * nl / (n * n);
  lA[c] += lm->n;
}

/* One reverse step.  On entry S holds the forward state X_n with its stage
 * arrays recomputed (forward_stages) and J holds the adjoint of X_{n+1}; on
 * exit J holds the adjoint of X_n; g3/gp accumulate dJ/dtheta of step n. */
static void adj_step(orc_state* S, orc_adj* J, double* g3, double* gp)
{
  const orc_params* p = &S->p;
  long nc = S->ncell;
  int K = S->K, Q = S->Q, Ds = S->Ds;
  double dt = S->dt, dx = p->dx, C = p->courant, tau = p->tau;
  double t = S->step * dt;
  size_t fsz = (size_t)K * Q * nc;
  memset(J->lfs, 0, sizeof(double) * fsz);
  memset(J->lA, 0, sizeof(double) * (size_t)K * nc);
  memset(J->lF, 0, sizeof(double) * (size_t)K * nc);
  memset(J->lEn, 0, sizeof(double) * 3 * nc);
  memset(J->lm, 0, sizeof(orc_macro) * (size_t)nc);
  double* lf_old = (double*)calloc(fsz, sizeof(double));
  double* lE_old = (double*)calloc(3 * (size_t)nc, sizeof(double));
  double* lB_old = (double*)calloc(3 * (size_t)nc, sizeof(double));
  double* lprev_old = (double*)calloc(7 * (size_t)nc, sizeof(double));

  /* (6)^T prev_{n+1} = (th00, th0, w) of this step */
  if (p->closure == ORC_WARMC) {
    for (long c = 0; c < nc; ++c) {
      J->lm[c].th00 += J->lprev[c];
      for (int a = 0; a < 3; ++a) {
        J->lm[c].th0[a] += J->lprev[(long)(1 + a) * nc + c];
        J->lm[c].w[a] += J->lprev[(long)(4 + a) * nc + c];
      }
    }
  }
  /* (5b)^T streaming: f_new(x)_i = fs(bulk(x) - xi_i)_i */
  for (long c = 0; c < nc; ++c) {
    long cb = bulk_of(S, c);
    int ib[3]; coords(S, cb, ib);
    for (int i = 0; i < Q; ++i) {
      int src[3] = {ib[0], ib[1], ib[2]};
      for (int a = 0; a < p->dim; ++a) {
        int v = src[a] - S->xi[i][a], n = S->n[a];
        if (p->boundary == ORC_PERIODIC) v = ((v % n) + n) % n;
        src[a] = v;
      }
      long cs = index_of(S, src);
      for (int k = 0; k < K; ++k)
        J->lfs[((size_t)k * Q + i) * nc + cs] += J->lf[((size_t)k * Q + i) * nc + c];
    }
  }
  /* (5a)^T collision: fs = f (1 - 1/tau) + feq(A, u)/tau + w dt F */
  for (long c = 0; c < nc; ++c) {
    const orc_macro* m = &S->mac[c];
    double ul[3] = {0, 0, 0};
    for (int a = 0; a < Ds; ++a) ul[a] = C * m->u[a];
    for (int k = 0; k < K; ++k) {
      double A = 0.0;
      for (int i = 0; i < Q; ++i) A += S->f[((size_t)k * Q + i) * nc + c];
      for (int i = 0; i < Q; ++i) {
        size_t ix = ((size_t)k * Q + i) * nc + c;
        double l = J->lfs[ix];
        if (l == 0.0) continue;
        double cu = S->xi[i][0] * ul[0] + S->xi[i][1] * ul[1] + S->xi[i][2] * ul[2];
        double usq = ul[0] * ul[0] + ul[1] * ul[1] + ul[2] * ul[2];
        double P = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq;
        lf_old[ix] += (1.0 - 1.0 / tau) * l;
        J->lA[(long)k * nc + c] += S->w[i] * (1.0 + P) / tau * l;
        for (int a = 0; a < Ds; ++a)
          J->lm[c].u[a] += S->w[i] * A / tau * C * (3.0 * S->xi[i][a] + 9.0 * cu * S->xi[i][a] - 3.0 * ul[a]) * l;
        J->lF[(long)k * nc + c] += S->w[i] * dt * l;
      }
    }
  }
  /* (4)^T sources */
  for (long c = 0; c < nc; ++c) {
    const orc_macro* m = &S->mac[c];
    orc_macro* lm = &J->lm[c];
    double En[3], Bn[3], lEn[3] = {0, 0, 0}, lBn[3] = {0, 0, 0};
    node_fields(S, c, En, Bn);
    if (p->closure == ORC_LEC) {
      for (int a = 0; a < Ds; ++a) {
        double l = J->lF[(long)(1 + a) * nc + c];
        if (l == 0.0) continue;
        long cp = nb_node(S, c, a, +1), cm = nb_node(S, c, a, -1);
        J->lm[cp].Pi -= PLANTED(12, 1.0, -1.0) * p->mu * l / (2.0 * dx);
        J->lm[cm].Pi += p->mu * l / (2.0 * dx);
        double uxB = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int q = 0; q < 3; ++q) {
            int e3 = eps3(a, k, q);
            if (!e3) continue;
            uxB += e3 * m->u[k] * Bn[q];
            lm->u[k] -= m->n * e3 * Bn[q] * l;
            lBn[q] -= m->n * e3 * m->u[k] * l;
          }
        lm->n -= (En[a] + uxB) * l;
        lEn[a] -= PLANTED(13, m->n, 0.0) * l;
      }
    } else {
      double lnl = J->lF[1 * nc + c];
      double hp = S->have_prev ? 1.0 : 0.0;
      double lnlu[3] = {0, 0, 0}, lth[3][3] = {{0}};
      for (int a = 0; a < Ds; ++a) lnlu[a] = J->lF[(long)(2 + a) * nc + c];
      for (int j = 0; j < S->ntheta; ++j) {
        int a = S->thpair[j][0], b = S->thpair[j][1];
        lth[a][b] = J->lF[(long)(2 + Ds + j) * nc + c];
      }
      /* F_nl = -d_t th00 - d_k th0_k - n E.u */
      if (lnl != 0.0) {
        lm->th00 -= hp * lnl / dt;
        lprev_old[c] += hp * lnl / dt;
        for (int k = 0; k < Ds; ++k) {
          J->lm[nb_node(S, c, k, +1)].th0[k] -= lnl / (2.0 * dx);
          J->lm[nb_node(S, c, k, -1)].th0[k] += lnl / (2.0 * dx);
        }
        for (int a = 0; a < 3; ++a) {
          lm->n -= En[a] * m->u[a] * lnl;
          lEn[a] -= m->n * m->u[a] * lnl;
          lm->u[a] -= m->n * En[a] * lnl;
        }
      }
      /* F_nlu_a = -d_t th0_a - d_b th_ab - n (E + u x B)_a */
      for (int a = 0; a < Ds; ++a) {
        double l = lnlu[a];
        if (l == 0.0) continue;
        lm->th0[a] -= hp * l / dt;
        lprev_old[(long)(1 + a) * nc + c] += hp * l / dt;
        for (int b = 0; b < Ds; ++b) {
          J->lm[nb_node(S, c, b, +1)].th[a][b] -= l / (2.0 * dx);
          J->lm[nb_node(S, c, b, -1)].th[a][b] += l / (2.0 * dx);
        }
        double uxB = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int q = 0; q < 3; ++q) {
            int e3 = eps3(a, k, q);
            if (!e3) continue;
            uxB += e3 * m->u[k] * Bn[q];
            lm->u[k] -= m->n * e3 * Bn[q] * l;
            lBn[q] -= m->n * e3 * m->u[k] * l;
          }
        lm->n -= (En[a] + uxB) * l;
        lEn[a] -= m->n * l;
      }
      /* F_th_ab; time derivatives of w against prev */
      double dw_dt[3] = {0, 0, 0};
      if (S->have_prev)
        for (int a = 0; a < 3; ++a) dw_dt[a] = (m->w[a] - S->prev[(long)(4 + a) * nc + c]) / dt;
      double gw[3][3] = {{0}};
      for (int k = 0; k < Ds; ++k) {
        const orc_macro* mp = &S->mac[nb_node(S, c, k, +1)];
        const orc_macro* mm = &S->mac[nb_node(S, c, k, -1)];
        for (int a = 0; a < 3; ++a) gw[a][k] = (mp->w[a] - mm->w[a]) / (2.0 * dx);
      }
      double ldw[3] = {0, 0, 0}, lgw[3][3] = {{0}};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double l = lth[a][b];
          if (l == 0.0) continue;
          /* s = -th0_b dw_a - th0_a dw_b - th_bk gw_ak - th_ak gw_bk */
          lm->th0[b] -= dw_dt[a] * l;
          ldw[a] -= m->th0[b] * l;
          lm->th0[a] -= dw_dt[b] * l;
          ldw[b] -= m->th0[a] * l;
          for (int k = 0; k < 3; ++k) {
            lm->th[b][k] -= gw[a][k] * l;
            lgw[a][k] -= m->th[b][k] * l;
            lm->th[a][k] -= gw[b][k] * l;
            lgw[b][k] -= m->th[a][k] * l;
          }
          /* em = E_a th0_b + E_b th0_a + eps_akq th_bk B_q + eps_bkq th_ak B_q */
          lEn[a] -= m->th0[b] * l;
          lm->th0[b] -= En[a] * l;
          lEn[b] -= m->th0[a] * l;
          lm->th0[a] -= En[b] * l;
          for (int k = 0; k < 3; ++k)
            for (int q = 0; q < 3; ++q) {
              int ea = eps3(a, k, q), eb = eps3(b, k, q);
              if (ea) { lm->th[b][k] -= ea * Bn[q] * l; lBn[q] -= ea * m->th[b][k] * l; }
              if (eb) { lm->th[a][k] -= eb * Bn[q] * l; lBn[q] -= eb * m->th[a][k] * l; }
            }
        }
      for (int a = 0; a < 3; ++a) {
        lm->w[a] += hp * ldw[a] / dt;
        lprev_old[(long)(4 + a) * nc + c] -= hp * ldw[a] / dt;
        for (int k = 0; k < Ds; ++k) {
          J->lm[nb_node(S, c, k, +1)].w[a] += lgw[a][k] / (2.0 * dx);
          J->lm[nb_node(S, c, k, -1)].w[a] -= lgw[a][k] / (2.0 * dx);
        }
      }
    }
    /* node averages of E^{n+1/2} and B^n */
    for (int a = 0; a < 3; ++a) {
      if (E_present(S, a) && lEn[a] != 0.0) {
        int b = (a + 1) % 3, d = (a + 2) % 3;
        int off[2], no = 0;
        if (present(S, b)) off[no++] = b;
        if (present(S, d)) off[no++] = d;
        for (int q = 0; q < (1 << no); ++q) {
          long cc = c;
          for (int j = 0; j < no && cc >= 0; ++j)
            if (q & (1 << j)) cc = nb_E(S, cc, off[j], -1);
          if (cc >= 0) J->lEn[(long)a * nc + cc] += lEn[a] / (double)(1 << no);
        }
      }
      if (B_present(S, a) && lBn[a] != 0.0) {
        if (present(S, a)) {
          lB_old[(long)a * nc + c] += 0.5 * lBn[a];
          lB_old[(long)a * nc + nb_node(S, c, a, -1)] += 0.5 * lBn[a];
        } else {
          lB_old[(long)a * nc + c] += lBn[a];
        }
      }
    }
  }
  /* lambda of E^{n+1/2}: as next state's E, through the sources, through B^{n+1} */
  for (size_t q = 0; q < 3 * (size_t)nc; ++q) J->lEn[q] += J->lE[q];
  for (long c = 0; c < nc; ++c)
    for (int a = 0; a < 3; ++a) {
      if (!B_present(S, a)) continue;
      double l = J->lB[(long)a * nc + c];
      lB_old[(long)a * nc + c] += l;
      int b = (a + 1) % 3, d = (a + 2) % 3;
      if (present(S, b) && E_present(S, d)) {
        J->lEn[(long)d * nc + c] -= dt * l / dx;
        long cm = nb_E(S, c, b, -1);
        if (cm >= 0) J->lEn[(long)d * nc + cm] += dt * l / dx;
      }
      if (present(S, d) && E_present(S, b)) {
        J->lEn[(long)b * nc + c] += dt * l / dx;
        long cm = nb_E(S, c, d, -1);
        if (cm >= 0) J->lEn[(long)b * nc + cm] -= dt * l / dx;
      }
    }
  /* (2)^T E^{n+1/2} = E + dt (curl B + avg(n u) + n_b) */
  for (long c = 0; c < nc; ++c) {
    int i[3]; coords(S, c, i);
    double pos[3]; node_pos(S, i, pos);
    for (int a = 0; a < 3; ++a) {
      if (!E_present(S, a) || E_wall(S, c, a)) continue;
      double l = J->lEn[(long)a * nc + c];
      if (l == 0.0) continue;
      lE_old[(long)a * nc + c] += l;
      int b = (a + 1) % 3, d = (a + 2) % 3;
      if (present(S, b) && B_present(S, d)) {
        lB_old[(long)d * nc + nb_node(S, c, b, +1)] += dt * l / dx;
        lB_old[(long)d * nc + c] -= dt * l / dx;
      }
      if (present(S, d) && B_present(S, b)) {
        lB_old[(long)b * nc + nb_node(S, c, d, +1)] -= dt * l / dx;
        lB_old[(long)b * nc + c] += dt * l / dx;
      }
      int off[2], no = 0;
      if (present(S, b)) off[no++] = b;
      if (present(S, d)) off[no++] = d;
      for (int s = 0; s < (1 << no); ++s) {
        long cc = c;
        for (int j = 0; j < no; ++j)
          if (s & (1 << j)) cc = nb_node(S, cc, off[j], +1);
        double w = dt * l / (double)(1 << no);
        J->lm[cc].n += w * S->mac[cc].u[a];
        J->lm[cc].u[a] += w * S->mac[cc].n;
      }
      if (a == 0) {
        double q[3] = {pos[0], pos[1], pos[2]};
        for (int j = 0; j < no; ++j) q[off[j]] += 0.5 * dx;
        driver_grad(p, q[0], q[1], q[2], t, dt * l, g3, gp);
      }
    }
  }
  /* (1)^T decode, then moments */
  for (long c = 0; c < nc; ++c) {
    double A[11];
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int i = 0; i < Q; ++i) s += S->f[((size_t)k * Q + i) * nc + c];
      A[k] = s;
    }
    if (p->closure == ORC_LEC) adj_decode_lec(S, c, A, &S->mac[c], &J->lm[c], J->lA);
    else adj_decode_warmc(S, c, A, &S->mac[c], &J->lm[c], J->lA);
    for (int k = 0; k < K; ++k)
      for (int i = 0; i < Q; ++i) lf_old[((size_t)k * Q + i) * nc + c] += J->lA[(long)k * nc + c];
  }
  memcpy(J->lf, lf_old, sizeof(double) * fsz);
  memcpy(J->lE, lE_old, sizeof(double) * 3 * nc);
  memcpy(J->lB, lB_old, sizeof(double) * 3 * nc);
  memcpy(J->lprev, lprev_old, sizeof(double) * 7 * nc);
  free(lf_old); free(lE_old); free(lB_old); free(lprev_old);
}

/* Initial driver field (init_fields) differentiated with respect to theta,
 * contracted with the adjoint of E^{-1/2} and B^0. */
static void adj_init_fields(const orc_state* S, const double* lE, const double* lB, double* g3, double* gp)
{
  const orc_params* p = &S->p;
  if (p->dim != 2 || !p->init_fields) return;
  long nc = S->ncell;
  double sr = p->sigma_r, dx = p->dx;
  for (long c = 0; c < nc; ++c) {
    int i[3]; coords(S, c, i);
    double pos[3]; node_pos(S, i, pos);
    double x = pos[1];
    double er = erf(x / (sqrt(2.0) * sr));
    double k = sr * sqrt(M_PI / 2.0) * er;
    double dk_dsr = sqrt(M_PI / 2.0) * er - x / sr * exp(-x * x / (2.0 * sr * sr));
    for (int which = 0; which < 2; ++which) {
      double l = which == 0 ? (E_wall(S, c, 1) ? 0.0 : lE[1 * nc + c]) : lB[2 * nc + c];
      if (l == 0.0) continue;
      double z = which == 0 ? pos[0] + 0.5 * dx : pos[0];
      double t = which == 0 ? -0.5 * S->dt : 0.0;
      double zeta = z - p->z0 - t;
      /* field = -L(zeta) k(x): d/dL = -k, d/dsr = -L dk/dsr */
      orc_params q = *p;
      q.dim = 1;  /* longitudinal factor only */
      driver_grad(&q, z, 0.0, 0.0, t, -k * l, g3, gp);
      g3[2] += -driver_long(p, zeta) * dk_dsr * l;
    }
  }
}

double orc_adjoint_run(orc_state* S, long N, long witness, double* g3, double* gp,
                       double* lf0, double* lE0, double* lB0)
{
  if (S->p.dim > 2 || axi(S)) return NAN;
  long nc = S->ncell;
  int K = S->K, Q = S->Q;
  size_t fsz = (size_t)K * Q * nc, esz = 3 * (size_t)nc, psz = 7 * (size_t)nc;
  size_t ssz = fsz + 2 * esz + psz;
  double* X = (double*)malloc(sizeof(double) * ssz * (size_t)(N + 1));
  int* hp = (int*)malloc(sizeof(int) * (size_t)(N + 1));
  long step0 = S->step;
  for (long n = 0; n <= N; ++n) {
    double* x = X + ssz * (size_t)n;
    memcpy(x, S->f, sizeof(double) * fsz);
    memcpy(x + fsz, S->E, sizeof(double) * esz);
    memcpy(x + fsz + esz, S->B, sizeof(double) * esz);
    memcpy(x + fsz + 2 * esz, S->prev, sizeof(double) * psz);
    hp[n] = S->have_prev;
    if (n < N) step_once(S);
  }
  double Jv = S->E[witness];
  orc_adj J;
  J.lf = (double*)calloc(fsz, sizeof(double));
  J.lE = (double*)calloc(esz, sizeof(double));
  J.lB = (double*)calloc(esz, sizeof(double));
  J.lprev = (double*)calloc(psz, sizeof(double));
  J.lfs = (double*)calloc(fsz, sizeof(double));
  J.lA = (double*)calloc((size_t)K * nc, sizeof(double));
  J.lF = (double*)calloc((size_t)K * nc, sizeof(double));
  J.lEn = (double*)calloc(esz, sizeof(double));
  J.lm = (orc_macro*)calloc((size_t)nc, sizeof(orc_macro));
  J.lE[witness] = 1.0;
  for (long n = N - 1; n >= 0; --n) {
    double* x = X + ssz * (size_t)n;
    memcpy(S->f, x, sizeof(double) * fsz);
    memcpy(S->E, x + fsz, sizeof(double) * esz);
    memcpy(S->B, x + fsz + esz, sizeof(double) * esz);
    memcpy(S->prev, x + fsz + 2 * esz, sizeof(double) * psz);
    S->have_prev = hp[n];
    S->step = step0 + n;
    forward_stages(S);
    adj_step(S, &J, g3, gp);
  }
  if (step0 == 0 && S->fields_from_driver) adj_init_fields(S, J.lE, J.lB, g3, gp);
  if (lf0) memcpy(lf0, J.lf, sizeof(double) * fsz);
  if (lE0) memcpy(lE0, J.lE, sizeof(double) * esz);
  if (lB0) memcpy(lB0, J.lB, sizeof(double) * esz);
  /* leave the final state in S */
  double* x = X + ssz * (size_t)N;
  memcpy(S->f, x, sizeof(double) * fsz);
  memcpy(S->E, x + fsz, sizeof(double) * esz);
  memcpy(S->B, x + fsz + esz, sizeof(double) * esz);
  memcpy(S->prev, x + fsz + 2 * esz, sizeof(double) * psz);
  S->have_prev = hp[N];
  S->step = step0 + N;
  free(J.lf); free(J.lE); free(J.lB); free(J.lprev); free(J.lfs); free(J.lA); free(J.lF); free(J.lEn); free(J.lm);
  free(X); free(hp);
  return Jv;
}
