/*
 * lbpwfa: lattice Boltzmann warm-plasma wakefield solver for NVIDIA GB300
 * (sm_103a).  C ABI of the CUDA library liblbpwfa.so.
 *
 * The method is the moment-matching lattice Boltzmann (LB) scheme of
 * arXiv 2309.04872 (Simeoni et al.): every advected scalar A_k of a warm
 * relativistic electron fluid is carried by its own set of populations f_ki
 * on a D1Q3 / D2Q9 / D3Q19 lattice (Sec. 2.2, Eq. ade-feq, lbe), the fluid is
 * closed either by the local-equilibrium closure LEC (Sec. 4, Eq.
 * lb-ade-lec-comps-A/F) or by the warm-plasma closure WARMC (Sec. 5, Eq.
 * lb-ade-warmc-comps-A/F, App. A), and it is coupled to an FDTD Maxwell
 * solver driven by a rigid Gaussian bunch moving at c (Sec. 6, Eq.
 * bunch-density).
 *
 * Units (Sec. 6): length k_p^-1, time omega_p^-1, density n_i, momentum m c,
 * velocity c, E in m c omega_p / e, B in E/c.
 *
 * Common conventions
 *  - Spatial axes: z (driver direction), x, y.  A 1D run uses z; 2D uses
 *    (z, x) with fields (E_z, E_x, B_y); 3D uses (z, x, y).
 *  - Cell index c = iz + nz * (ix + nx * iy) (z fastest) for every host or
 *    device array crossing this interface (unpadded).
 *  - Node positions: z = iz dx, x = (ix - (nx-1)/2) dx, y = (iy - (ny-1)/2) dx.
 *  - Fields live on a dual Yee grid: E_a half a cell up along the two axes
 *    other than a, B_a half a cell up along a.  E is stored at t_{n-1/2},
 *    B at t_n, populations at t_n.  Transverse boundaries are conducting
 *    walls half a cell outside the outermost nodes.
 *  - Populations f[k][i][c]: k = advected scalar, i = lattice velocity in the
 *    order below, c = cell.  Advected scalars:
 *      LEC  : n, n H p_z, (n H p_x), (n H p_y),
 *             H = 1 + (1 + D/2) mu (n/gamma)^(2/D)
 *      WARMC: n, n lambda, n lambda u_z, (n lambda u_x), (n lambda u_y),
 *             lambda theta^{ab} for the pairs
 *             1D: zz;  2D: zz, xx, yy, zx;  3D: zz, xx, yy, zx, zy, xy.
 *  - Velocity order (components z, x, y):
 *      D1Q3 : 0, +z, -z
 *      D2Q9 : 0, +z, -z, +x, -x, (+z+x), (-z-x), (+z-x), (-z+x)
 *      D3Q19: 0, +z, -z, +x, -x, +y, -y, (+z+x), (-z-x), (+z-x), (-z+x),
 *             (+z+y), (-z-y), (+z-y), (-z+y), (+x+y), (-x-y), (+x-y), (-x+y)
 *  - Every function returns an lbpwfa_status; nothing else crosses the ABI
 *    (no exceptions, no exit).  A handle must not be used from two host
 *    threads at once.  Work is queued on the handle's stream; functions that
 *    return host data synchronise that stream.
 */
#ifndef LBPWFA_H
#define LBPWFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbpwfa_s* lbpwfa_t;

typedef enum {
  LBPWFA_OK = 0,
  LBPWFA_ERR_INVALID = -1,    /* bad argument or parameter */
  LBPWFA_ERR_OOM = -2,        /* device or host allocation failed */
  LBPWFA_ERR_CUDA = -3,       /* a CUDA call failed; see lbpwfa_last_error */
  LBPWFA_ERR_NONFINITE = -4,  /* a NaN/Inf population was found */
  LBPWFA_ERR_TIMEOUT = -5,    /* a bounded device wait gave up */
  LBPWFA_ERR_STATE = -6,      /* call not valid in the handle's state */
  LBPWFA_ERR_IO = -7          /* checkpoint file error or CRC mismatch */
} lbpwfa_status;

enum { LBPWFA_LEC = 0, LBPWFA_WARMC = 1 };
enum { LBPWFA_FP64 = 0, LBPWFA_FP32 = 1, LBPWFA_FP16S = 2, LBPWFA_FP32C = 3 };
enum { LBPWFA_OPEN = 0, LBPWFA_PERIODIC = 1 };
enum { LBPWFA_CARTESIAN = 0, LBPWFA_AXISYMMETRIC = 1 };

/* Problem statement (Sec. 6, Eq. bunch-density and Qtilde). */
typedef struct {
  int dim;                 /* 1, 2 or 3 */
  int n[3];                /* nodes along z, x, y; absent axes ignored; >= 3;
                              x and y at most 262 140 (4 x 65 535 tiles) */
  double dx;               /* lattice spacing, k_p^-1 */
  double courant;          /* C = c dt / dx; dt = C dx. 0 < C <= 1/sqrt(dim) */
  double tau;              /* BGK relaxation time in units of dt, > 1/2
                              (Eq. diff-coeff: kappa = nu^2 (tau - 1/2)) */
  int closure;             /* LBPWFA_LEC or LBPWFA_WARMC */
  int dv;                  /* kinetic momentum dimensions D: 1 or 3 */
  double mu;               /* k_B T_i / (m c^2) >= 0 */
  double alpha;            /* driver peak n_b / n_i */
  double sigma_z;          /* rms length of the driver, k_p^-1 (> 0) */
  double sigma_r;          /* rms radius of the driver, k_p^-1 (> 0, 2D/3D) */
  double z0;               /* driver centre at t = 0, k_p^-1 */
  const double* profile;   /* optional longitudinal profile L(zeta) sampled at
                              zeta_j = (j - (len-1)/2) profile_dz about the
                              driver centre, linearly interpolated with zero
                              samples just outside both ends (continuous,
                              0 from one sample beyond the ends); replaces
                              alpha exp(-zeta^2/2 sigma_z^2).
                              Copied at create; NULL for the Gaussian. */
  int profile_len;         /* >= 2 when profile != NULL */
  double profile_dz;       /* > 0 when profile != NULL */
  int precision;           /* population storage: FP64, FP32 (deviation from
                              w_i A_rest), FP16S (binary16 deviation, scaled;
                              the rest population of each set keeps a
                              second binary16 with its rounding residual),
                              FP32C (FP32 storage whose set moments and
                              post-collision remainders carry every rounding
                              error of their sums and round once: about half
                              the FP32 error of n - 1 at a higher step cost;
                              single runs and the adjoint, not batches) */
  int boundary;            /* LBPWFA_OPEN (Eq. open-bc; conducting transverse
                              walls) or LBPWFA_PERIODIC (all axes) */
  int init_fields;         /* 1: start from the v -> c field of the driver
                              (2D, 3D); 0: zero fields */
  void* stream;            /* cudaStream_t to queue work on; NULL = a stream
                              owned by the library */
  int kernel_variant;      /* 0: automatic (2D open-boundary LEC runs stage
                              each tile's populations in shared memory by
                              TMA bulk-tensor loads: FP32 and FP16S with
                              persistent refilling CTAs (variant 3), FP64
                              with one box per CTA (variant 2); the rest,
                              WARMC included, pull from global memory, which
                              measures faster for its 72 population planes);
                              1: plain global-memory pull; 2: one TMA box per
                              CTA (2D open boundaries);
                              3: LEC 2D with persistent CTAs, each refilling
                              its TMA box with its next tile as soon as the
                              decode phase has read it; 4: 3D columns of
                              32 x 8 nodes marching up chunks of 32 planes,
                              each plane decoded once per column (the
                              automatic 3D choice; 1 gives 32 x 4 x 4 tiles).
                              All compute the same step.  Axisymmetric runs
                              take 0, 1 or 3: LEC in FP32 and FP16S runs the
                              persistent kernel with the axis rules (3,
                              automatic), the rest the plain kernel with
                              them (reported as 5). */
  int geometry;            /* LBPWFA_CARTESIAN, or LBPWFA_AXISYMMETRIC: the
                              3D3V axisymmetric (z, r) geometry of Sec. 2.2
                              and App. A on a 2D grid (dim 2, open
                              boundaries); x is r, node j at r = j dx, and
                              j = 0 is the r = 0 boundary node, which takes
                              the populations of node 1 as they are (Eq.
                              open-bc) for the sets even under r -> -r and
                              with the mirrored velocity (Eq. reflective-bc)
                              for the odd ones (n A_r; n lambda u_r,
                              lambda theta^{rz}).  Fields: E_z, E_r, B_phi
                              in the slots of E_z, E_x, B_y; E_r = B_phi = 0
                              on the axis; (curl B)_z = d_r(r B_phi)/r.  The
                              1/r terms of App. A are added to the sources
                              at r > 0.  Batches may mix both geometries;
                              the adjoint takes Cartesian runs only
                              (LBPWFA_ERR_INVALID). */
  size_t device_bytes_cap; /* 0: no cap.  Else the most device memory the
                              handle may hold (state, diagnostics scratch,
                              adjoint tape and checkpoints together): a
                              create or a later allocation that would pass
                              it returns LBPWFA_ERR_OOM, before any device
                              memory is touched.  lbpwfa_create checks the
                              state's size first, before any CUDA call. */
  int64_t record_tape;     /* > 0: lbpwfa_create also starts an adjoint
                              recording window of this many steps at step 0
                              (lbpwfa_record with max_steps = record_tape);
                              0: none.  Not for batches. */
  int64_t checkpoint_every;/* the window's checkpoint interval C (0: keep
                              every step's tape), as lbpwfa_record */
} lbpwfa_params;

typedef struct {
  int K;                   /* advected scalars */
  int Q;                   /* lattice velocities */
  int64_t ncell;           /* nodes */
  int64_t step;            /* steps taken */
  double dt;               /* time step, omega_p^-1 */
  double time;             /* step * dt */
  size_t device_bytes;     /* device memory held by the handle */
  double bytes_per_update; /* stored HBM bytes one node update of the step
                              kernel reads and writes in this design:
                              populations (with the FP16S low planes),
                              fields (FP32 modes: high and low parts) and the
                              WARMC previous-step values */
  int kernel_variant;      /* step kernel in use: 1 plain, 2 TMA box per CTA,
                              3 persistent TMA, 4 3D marching columns,
                              5 axisymmetric plain */
  double algorithmic_bytes_per_update; /* the method's bytes per node update,
                              independent of this design's extra storage:
                              2 K Q s (populations read and written, s the
                              stored population size) + 2 F r (the F field
                              components, r the real size: 8 in FP64, 4
                              otherwise) + 2 (2 (1 + dim)) r for WARMC (the
                              previous step's theta^{0 beta} and w^beta).
                              2D LEC: 480 / 240 / 132 B in FP64 / FP32 /
                              FP16S; 2D WARMC FP32 648; 3D WARMC FP32 1784 */
} lbpwfa_info_t;

/* Create a run: validates *p, allocates all device state on the handle's
 * stream and sets the rest state n = 1, u = 0 (f = f^eq, Eq. ade-feq) with
 * the initial fields.  The library owns all device memory; *out receives the
 * handle.  Errors: INVALID (bad parameters, out == NULL), OOM, CUDA. */
int lbpwfa_create(const lbpwfa_params* p, lbpwfa_t* out);

/* Advance nsteps >= 0 time steps (Sec. 2.1 algorithm with the Sec. 4.1
 * coupling): decode, E^{n+1/2} = E^{n-1/2} + dt (curl B^n + n u + n_b z),
 * B^{n+1} = B^n - dt curl E^{n+1/2}, sources with E^{n+1/2} and B^n,
 * BGK + w_i dt F, pull streaming with the open-boundary copy.
 * One fused kernel launch per step; asynchronous.  Errors: INVALID, CUDA. */
int lbpwfa_step(lbpwfa_t h, int64_t nsteps);

/* Macroscopic fields decoded in FP64 from the current populations.
 * mask bits (output blocks in increasing bit order, each ncell doubles):
 *   0 n, 1 u_z, 2 u_x, 3 u_y, 4 gamma, 5 p_z, 6 p_x, 7 p_y (gamma u),
 *   8 LEC rest-frame pressure P0 = mu (n/gamma)^(1+2/D) (0 for WARMC),
 *   9 lambda = n/h (WARMC; 0 for LEC),
 *   10..15 theta zz, xx, yy, zx, zy, xy (WARMC; 0 for LEC),
 *   16 P_par, 17 P_perp: rest-frame pressures along and across z (App. A's
 *   inversion of theta with r -> x, phi -> y: P_perp = theta_yy, P_par =
 *   [theta_xx + theta_zz - theta^00 u^2 - theta_yy (1 + u_x^2)] /
 *   (1 + u_z^2), theta^00 = u_i u_j theta_ij; 2D WARMC only, else 0).
 * dst holds count >= popcount(mask & 0x3FFFF) * ncell doubles, on the device
 * when dst_is_device, else on the host.  A page-locked host buffer that CUDA
 * maps into the device (cudaHostAlloc, cudaMallocHost), 8-byte aligned and
 * lying inside the allocation CUDA reports for it, is written in place by
 * the kernel; other host memory through a device staging buffer.  Host
 * outputs are complete on return.  Errors: INVALID, CUDA. */
int lbpwfa_moments(lbpwfa_t h, uint32_t mask, double* dst, size_t count, int dst_is_device);

/* Raw field slots (FP64), mask bits 0 E_x, 1 E_y, 2 E_z, 3 B_x, 4 B_y, 5 B_z;
 * E at t_{n-1/2}, B at t_n, on the dual Yee grid described above.  Host
 * buffers as for lbpwfa_moments. */
int lbpwfa_fields(lbpwfa_t h, uint32_t mask, double* dst, size_t count, int dst_is_device);

/* Wake diagnostic on the device (the dispersion measurement of Sec. 6,
 * Fig. 3): least-squares fit of q = A cos(k xi + phi) along one grid line in
 * z, over the co-moving window xi_lo <= xi <= xi_hi with xi = z - z_d(t),
 * z_d = z0 + t the driver centre (t = t_n for the density, t_{n-1/2} for the
 * stored E).  q is E_z (LBPWFA_FIT_EZ, the slots of the line) or n - 1
 * (LBPWFA_FIT_N).  For each k of the uniform grid k_lo .. k_hi (nk points)
 * the residual R(k) of the best a cos + b sin is formed from FP64 sums in a
 * fixed order; the grid minimum is refined by the parabola through it and
 * its neighbours and refitted there.
 * line: transverse indices (x, y) of the line (ignored for absent axes).
 * out (host, 5 doubles): k, A, phi, rms residual, points in the window.
 * Uses the handle's device scratch buffer; LBPWFA_ERR_INVALID for a line
 * outside the grid, nk outside [3, 65536] or an empty k or xi range. */
enum { LBPWFA_FIT_EZ = 0, LBPWFA_FIT_N = 1 };
typedef struct {
  int quantity;
  int line[2];
  double xi_lo, xi_hi;
  double k_lo, k_hi;
  int nk;
} lbpwfa_fit_params;
int lbpwfa_line_fit(lbpwfa_t h, const lbpwfa_fit_params* fp, double* out);

/* Gauss's law residual (Sec. 6: not imposed; it holds up to the LB's
 * numerical diffusion), FP64 on the device.  On the dual cells centred at
 * (z_{i+1/2}, x_{j+1/2}, y_{k+1/2}) the Yee slots give div E (axisymmetric:
 * the radial term (r_{j+1} E_r(j+1) - r_j E_r(j)) / (r_{j+1/2} dx)); rho =
 * -(nbar - 1) - n_b with nbar the mean density of the cell's corner nodes
 * (at t_n) and n_b the driver at the centre at t_{n-1/2}, the time of the
 * stored E.  lo[a] <= i < hi[a] per present axis, 0 <= lo < hi <= n[a] - 1.
 * out (host, 3 doubles): sum (div E - rho)^2, sum rho^2, cells.  Fixed
 * block partition and tree: repeated calls return identical bits.  Uses the
 * handle's device scratch buffer. */
int lbpwfa_gauss_residual(lbpwfa_t h, const int* lo, const int* hi, double* out);

/* Advected scalars A_k = sum_i f_ki (Eq. disc-moments-ade), FP64,
 * [K][ncell]; count >= K * ncell.  Host buffers as for lbpwfa_moments. */
int lbpwfa_advected(lbpwfa_t h, double* dst, size_t count, int dst_is_device);

/* Replace the state: f = populations at t_n after streaming, FP64
 * [K][Q][ncell]; E [3][ncell] (z, x, y) at t_{n-1/2}; B [3][ncell] at t_n.
 * Any pointer may be NULL to keep that part.  With open boundaries the
 * boundary nodes take the populations of their nearest bulk node
 * (Eq. open-bc) and wall slots of E are zeroed.  The backward time
 * differences of WARMC restart (zero on the next step).  Mapped page-locked
 * host buffers (all given ones) are read in place by the import kernels,
 * other host memory through a device staging buffer; host inputs may be
 * reused on return.  Errors: INVALID, OOM, CUDA. */
int lbpwfa_set_state(lbpwfa_t h, const double* f, const double* E, const double* B,
                     int src_is_device);

/* Read the state in the layout of lbpwfa_set_state (FP64).  Host buffers as
 * for lbpwfa_moments. */
int lbpwfa_get_state(lbpwfa_t h, double* f, double* E, double* B, int dst_is_device);

/* FP64 global sums over nodes, in a fixed order (deterministic):
 * out[0] = sum n, out[1] = sum n_b(t_n), out[2] = number of non-finite
 * populations.  Synchronises.  Returns NONFINITE when out[2] > 0. */
int lbpwfa_reduce(lbpwfa_t h, double out[3]);

int lbpwfa_info(lbpwfa_t h, lbpwfa_info_t* info);

/* Choose the run's step kernel by timing: every kernel variant the run can
 * take (1 plain, 2 TMA box per CTA, 3 persistent, 4 3D marching; the step
 * of lbpwfa_step, Sec. 2.1 algorithm, which they all compute) steps the
 * current state twice to warm up and five times under CUDA events, the
 * state is put back exactly (a device copy of f, E, B and the previous-step
 * values, allocated for the call), and the fastest is kept for the run's
 * later steps (lbpwfa_info reports it).  With LBPWFA_TUNE_CACHE naming a
 * JSON file, the choice is stored there under a key of the device name,
 * dim, closure, precision, boundary, geometry and grid, and read back by
 * later calls for the same key, which then time nothing.  ms_out (host,
 * 5 doubles, may be NULL): per variant the mean step time in ms, -1 where
 * not timed.  The run's step count and recording are unchanged.
 * Synchronises.  Errors: INVALID, STATE (a batch member), OOM (no room for
 * the copy of the state), TIMEOUT, CUDA. */
int lbpwfa_autotune(lbpwfa_t h, double* ms_out);

/* The sums of lbpwfa_reduce for callers that cannot allocate device memory:
 * code whose device memory belongs to another allocator (a framework's
 * caching allocator, an embedding that reserves the whole device) or whose
 * loop cannot take the implicit synchronisation of cudaMalloc / cudaFree.
 * It allocates nothing.  The paper has no counterpart; this is plumbing
 * around its FP64 diagnostics.
 *  - Scratch: the per-block partial sums live in one fixed device array of
 *    4096 x 3 + 4 doubles inside the library (about 96 KB, held on every GPU
 *    that loads the library until the process exits).  It serves runs of at
 *    most 2^25 = 33,554,432 nodes; larger runs return LBPWFA_ERR_INVALID
 *    with the limit in lbpwfa_last_error.
 *  - The first call on a device resolves the array's device address; make
 *    that first call before any stream capture on that device.
 *  - All calls on a device share the array and it keeps the last call's
 *    contents; each call overwrites every partial it reads, but calls whose
 *    work overlaps on the GPU race on it.
 *  - out: 3 doubles (sum n, sum n_b, non-finite populations) on the device
 *    when out_is_device (asynchronous), else on the host.  The host form
 *    synchronises and then, like lbpwfa_reduce, returns TIMEOUT when a
 *    bounded device wait of an earlier step gave up, else NONFINITE when
 *    out[2] > 0.  The device form reports neither: read out[2], and call
 *    lbpwfa_synchronize for the timeout status.
 *  - Call with the handle's device current; another current device returns
 *    INVALID with the reason in lbpwfa_last_error.  The summation order
 *    differs from lbpwfa_reduce (more, smaller blocks), so the two agree to
 *    FP64 round-off, not bitwise. */
int lbpwfa_reduce_noalloc(lbpwfa_t h, double* out, int out_is_device);

/* Checkpoint: binary file with a header (parameters, step, precision), the
 * stored populations, fields and WARMC previous-step values, and a CRC32.
 * Resume is bitwise.  lbpwfa_load requires a handle created with the same
 * parameters.  Errors: IO (open/short read/CRC/header mismatch), CUDA. */
int lbpwfa_save(lbpwfa_t h, const char* path);
int lbpwfa_load(lbpwfa_t h, const char* path);

/* Queue subsequent work on another stream (NULL = the library stream). */
int lbpwfa_set_stream(lbpwfa_t h, void* stream);
/* Wait for the handle's queued work; returns TIMEOUT when a bounded device
 * wait gave up (the step is then incomplete).  The timeout status sticks
 * (lbpwfa_reduce and lbpwfa_synchronize keep returning it) until the state
 * is replaced by lbpwfa_set_state or lbpwfa_load. */
int lbpwfa_synchronize(lbpwfa_t h);

/* The FP64 fused multiply-add rate of the current device, in FLOP/s (two
 * per DFMA), measured by a kernel of independent register-resident DFMA
 * chains timed with CUDA events on a stream of its own (best of three
 * launches after a warm-up).  It is the ALU roofline of the FP64 storage
 * mode: on GB300 the FP64 step is bound by FP64 arithmetic, not by HBM.
 * Changes no device setting and allocates nothing.  The paper has no
 * counterpart.  Errors: INVALID (flops NULL), CUDA. */
int lbpwfa_measure_fp64_rate(double* flops);

/* Failure-detection hook: the number of polls the first wait of each tile
 * (the TMA-staged step kernels wait on an mbarrier for their population box)
 * makes before it gives up, flags LBPWFA_ERR_TIMEOUT in the handle's device
 * error word, lets the copy in flight land, and ends the CTA.  lbpwfa_create
 * sets LBPWFA_WAIT_POLLS; 0 gives up at once, so a test can reach the
 * timeout path without a fault.  The step is then incomplete.  The kernels
 * that pull from global memory do not wait.  Errors: INVALID (h NULL). */
#define LBPWFA_WAIT_POLLS (1u << 24)
int lbpwfa_set_wait_limit(lbpwfa_t h, uint32_t polls);

/* ------------------------------------------------------------------------
 * Gradients by the discrete adjoint (1D and 2D; FP64 or FP32 storage).
 * The quantity differentiated is J = E_z at one slot after a window of steps
 * (the accelerating field at a witness position behind the driver, Sec. 6);
 * the parameters are those of the driver in Eq. (bunch-density): alpha,
 * sigma_z, sigma_r, or the sampled profile values.  The reverse sweep
 * applies, per step and in reverse order, the transpose of every stage of
 * lbpwfa_step (streaming with the open-boundary copy, BGK collision, the
 * LEC / WARMC sources with their central differences, the closure decode by
 * implicit differentiation, the Yee updates and the driver current), on the
 * forward values the step kernel saved while recording.  The paper has no
 * adjoint; this is the exact gradient of the discrete scheme it defines.
 * ------------------------------------------------------------------------ */
typedef struct {
  int64_t max_steps;        /* steps the window may hold (>= 1) */
  int64_t checkpoint_every; /* C > 0: keep the full state every C steps and
                               recompute each C-step segment (recording its
                               tape) during the reverse sweep; 0: keep the
                               tape of every step (no recomputation):
                               (K + dim + (dim == 2)) values per node per step */
} lbpwfa_record_params;

/* Start recording at the current step: the next up-to-max_steps calls of
 * lbpwfa_step form the window.  Replaces an earlier recording.  Stepping past
 * max_steps returns STATE; lbpwfa_set_state and lbpwfa_load end the
 * recording.  Errors: INVALID (3D, FP16S storage, a batch member, bad
 * arguments, a grid of more than 2^31 / max(K + E and B components, K dim,
 * Q) cells, beyond the reverse kernels' 32-bit offsets), OOM, CUDA. */
int lbpwfa_record(lbpwfa_t h, const lbpwfa_record_params* rp);

typedef struct {
  int witness[3];           /* node (z, x, y) of the E_z slot defining J */
  double seed;              /* dL/dJ; the outputs are dL/dtheta = seed dJ/dtheta */
  double J;                 /* out: E_z at the witness slot after the window */
  double grad_driver[3];    /* out: dL/d(alpha, sigma_z, sigma_r); with a
                               profile the first two are 0 */
  double* grad_profile;     /* out: dL/d(profile sample j), profile_len host
                               doubles, or NULL */
} lbpwfa_adjoint_io;

/* Reverse sweep over the recorded window (at least one step).  When the
 * window starts at step 0 from the driver's initial fields
 * (init_fields = 1, 2D), their dependence on the parameters is included.
 * The run's state stays (or is put back) at the end of the window and the
 * recording ends.  Synchronises.  Errors: INVALID (witness outside the grid),
 * STATE (nothing recorded), OOM, CUDA. */
int lbpwfa_adjoint_step(lbpwfa_t h, lbpwfa_adjoint_io* io);

/* ------------------------------------------------------------------------
 * Batched sweeps (uneven 2D grids, mixed closures, one launch per step).
 * The paper runs each parameter point as a separate simulation (Sec. 6:
 * temperature and driver scans, Figs. 3 and 6); a batch advances many such
 * runs together: every step is one persistent kernel per closure over that
 * closure's work list of (run, tile) items, and runs of lbpwfa_batch_step
 * are replayed from a captured CUDA graph.  A device-side step counter supplies each step's time
 * and buffer parity, so the graph is valid from any step.
 * ------------------------------------------------------------------------ */
typedef struct lbpwfa_batch_s* lbpwfa_batch_t;

typedef struct {
  int nruns;
  int64_t ncell;           /* nodes over all runs */
  int64_t nitems;          /* (run, tile) work items per step, both closures */
  int tile[2][2];          /* per closure [LBPWFA_LEC, LBPWFA_WARMC]: tile (z, x)
                              chosen by the autotuner; 0 without such runs */
  int grid[2];             /* per closure: CTAs of its persistent launch */
  int graph_steps;         /* steps per captured graph */
  int64_t step;
  size_t device_bytes;
  double bytes_per_step;   /* stored HBM bytes of one batch step (the runs'
                              bytes_per_update times their nodes) */
  double tuned_ms[2][4];   /* per closure: autotuner step time per candidate
                              tile (-1 unused) */
  double algorithmic_bytes_per_step; /* the runs' algorithmic_bytes_per_update
                              times their nodes */
} lbpwfa_batch_info_t;

/* Create nruns >= 1 runs from p[0..nruns-1], each validated as by
 * lbpwfa_create.  Every run must be 2D with the same precision (FP64, FP32
 * or FP16S storage); closures, geometries, grids and driver parameters may
 * differ.  flags bit 0: skip the autotuner
 * (use the first candidate tile).  The autotuner times each candidate tile,
 * closure by closure, over a few steps and restores the rest state; when the environment
 * variable LBPWFA_TUNE_CACHE names a JSON file, choices are read from and
 * written to it.  p[i].stream of run 0 is the batch's stream.
 * Errors: INVALID, OOM, CUDA. */
int lbpwfa_batch_create(const lbpwfa_params* p, int nruns, int flags, lbpwfa_batch_t* out);
/* lbpwfa_batch_create with flags = 0 (autotuned), under the name the
 * problem statement's interface gives it. */
int lbpwfa_create_batch(const lbpwfa_params* p, int nruns, lbpwfa_batch_t* out);

/* Advance every run by nsteps >= 0 steps. */
int lbpwfa_batch_step(lbpwfa_batch_t b, int64_t nsteps);

/* Handle of run i for lbpwfa_moments, lbpwfa_fields, lbpwfa_advected,
 * lbpwfa_get_state, lbpwfa_set_state, lbpwfa_reduce, lbpwfa_info and
 * lbpwfa_save.  It stays owned by the batch; lbpwfa_step on it returns
 * LBPWFA_ERR_STATE, and lbpwfa_destroy on it does nothing. */
int lbpwfa_batch_member(lbpwfa_batch_t b, int i, lbpwfa_t* run);

int lbpwfa_batch_info(lbpwfa_batch_t b, lbpwfa_batch_info_t* info);
void lbpwfa_batch_destroy(lbpwfa_batch_t b);

void lbpwfa_destroy(lbpwfa_t h);
const char* lbpwfa_status_string(int status);
/* Text of the last CUDA error seen by this handle ("" if none). */
const char* lbpwfa_last_error(lbpwfa_t h);

#ifdef __cplusplus
}
#endif
#endif /* LBPWFA_H */
