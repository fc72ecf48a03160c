/*
 * FP64 CPU oracle for the moment-matching LB warm-plasma wakefield scheme
 * (arXiv 2309.04872).  TEST INFRASTRUCTURE ONLY: used by tests/, the smoke
 * check and bench.py's CPU baseline; never by the CUDA library, with which it
 * shares no source.
 *
 * Layouts: cell index c = iz + nz * (ix + nx * iy) (z fastest);
 * populations f[k][i][c] (advected scalar k, velocity i, cell c);
 * fields E[a][c], B[a][c] with a = 0 z, 1 x, 2 y on a dual Yee grid
 * (E_a half a cell up along the two axes other than a, B_a half a cell up
 * along a).
 */
#ifndef LBPWFA_ORACLE_H
#define LBPWFA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_LEC = 0, ORC_WARMC = 1 };
enum { ORC_OPEN = 0, ORC_PERIODIC = 1 };
enum { ORC_CARTESIAN = 0, ORC_AXISYMMETRIC = 1 };

typedef struct {
  int dim;                 /* 1, 2, 3 */
  int nz, nx, ny;          /* nodes along z, x, y (absent axes ignored) */
  double dx;               /* k_p^-1 */
  double courant;          /* C = c dt / dx */
  double tau;              /* BGK relaxation time in units of dt (> 1/2) */
  int closure;             /* ORC_LEC or ORC_WARMC */
  int dv;                  /* kinetic momentum dimensions D: 1 or 3 */
  double mu;               /* k_B T_i / m c^2 */
  double alpha;            /* driver peak n_b / n_i */
  double sigma_z, sigma_r; /* rms sizes, k_p^-1 */
  double z0;               /* driver centre at t = 0 */
  const double* profile;   /* optional longitudinal profile samples (copied):
                              sample j at zeta_j = (j - (len-1)/2) profile_dz,
                              linear between samples, zero samples just
                              outside both ends */
  int profile_len;
  double profile_dz;
  int boundary;            /* ORC_OPEN or ORC_PERIODIC */
  int init_fields;         /* 1: v -> c driver field at t = 0 (2D, 3D) */
  int geometry;            /* ORC_CARTESIAN, or ORC_AXISYMMETRIC (dim 2, open
                              boundaries): the x axis is r >= 0, node j at
                              r = j dx, y is the azimuth phi (Sec. 2.2, App. A) */
} orc_params;

typedef struct orc_state orc_state;

orc_state* orc_create(const orc_params* p, int* status);
void orc_destroy(orc_state* S);
void orc_sizes(const orc_state* S, int* K, int* Q, long* ncell);
long orc_get_step(const orc_state* S);
double orc_get_dt(const orc_state* S);
void orc_rest_advected(const orc_state* S, double* A);
void orc_set_state(orc_state* S, const double* f, const double* E, const double* B);
void orc_get_state(const orc_state* S, double* f, double* E, double* B);
void orc_step(orc_state* S, long nsteps);
void orc_advected(const orc_state* S, double* A);
int orc_moments(const orc_state* S, unsigned mask, double* dst);
void orc_rest_pressures(const double* th, const double* u, double* out);
void orc_reduce(const orc_state* S, double* out);

/* pieces exposed for the pins */
int orc_stencil(int dim, int* xi, double* w);
void orc_equilibrium(int dim, double A, const double* u_phys, double courant, double* feq);
int orc_decode_lec(int Ds, int D, double mu, const double* A,
                   double* n, double* u, double* gamma, double* Pi);
void orc_decode_warmc(int dim, const double* A, double* out);
void orc_lec_source(double mu, double n, const double* u, const double* gradPi,
                    const double* E, const double* B, double* Fp);
void orc_warmc_source(double n, const double* u, const double* th, const double* th0,
                      double dth00_dt, const double* dth0_dt, const double* dw_dt,
                      const double* dth, const double* dth0, const double* dw,
                      const double* E, const double* B,
                      double* F_nl, double* F_nlu, double* F_th);
double orc_driver_density(const orc_params* p, double z, double x, double y, double t);

/* Discrete adjoint (1D, 2D): runs N steps from the current state, returns
 * J = E[witness] after them (an index into E[3][ncell]; the E_z slot of cell c
 * is c), and adds dJ/d(alpha, sigma_z, sigma_r) to g3 (Gaussian driver; with a
 * profile g3[0..1] stay 0) and dJ/d(profile samples) to gp.  When the run
 * starts at step 0 from the driver's initial fields, their dependence on the
 * driver parameters is included.  S is left in the final state.  Returns NaN
 * for 3D.  Memory: N + 1 stored states.  lf0, lE0, lB0 (each may be NULL)
 * receive dJ/d(f, E, B) of the starting state, layouts as orc_get_state. */
double orc_adjoint_run(orc_state* S, long N, long witness, double* g3, double* gp,
                       double* lf0, double* lE0, double* lB0);

#ifdef __cplusplus
}
#endif
#endif
