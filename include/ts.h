/*
 * ts.h -- C ABI of the GB300 library for one time step of the 6-D spectral
 * transport method of Bonazzola, Vasset & Peres (A&A 2011, "Solving the
 * transport equation by the use of 6D spectral methods in spherical
 * coordinates").
 *
 * The step advances the distribution function F(r, theta, phi, Theta, Phi)
 * of one or more independent energy groups under
 *     dF/dt + L_sph F = CT                                   (Eq. Transpfpsph, Sect. 4.1)
 *     L_sph = cos(Th) d_r + (1/r)[ sin(Th)cos(Ph) d_th + sin(Th)sin(Ph)/sin(th) d_ph
 *                                  - sin(Th) d_Th - sin(Th)sin(Ph) cot(th) d_Ph ]
 *                                                            (Eq. Liouvsph, Sect. 4.1)
 *     CT = eta - kappa F + kappa_s (J + b omega.H + c omega.M~.omega - F)
 *          (Eq. Transp, Sect. 2.2, coherent scattering Eq. sigmadif so that groups
 *           decouple, kernel (kappa_s/4pi)(1 + b mu + c (mu^2 - 1/3)), mu =
 *           omega.omega'; J, H, M~ the zeroth, first and traceless second angular
 *           moments; b = c = 0 (isotropic, Eq. sigman with B = 0) unless set by
 *           ts_set_scattering_anisotropy / ts_set_scattering_quadrupole)
 * with spectral derivatives on every axis (Sect. 5.1): Chebyshev in r on
 * Gauss-Lobatto nodes, double-Fourier-sphere parity Fourier series on the
 * pole-free nodes th_j = pi (j+1/2)/N_theta and Th_k = pi (k+1/2)/N_Theta,
 * Fourier in phi and Phi; inflow boundaries by the Tau method (Sect. 5.1;
 * inflow at R1 where cos Theta > 0, at R2 where cos Theta < 0, Sect. 4.2);
 * classical RK4 or second-order Adams-Bashforth (Sect. 5.1) in time.
 *
 * Conventions shared by every entry point
 *  - Layout of a field F: F[g][i_r][j_theta][l_phi][k_Theta][m_Phi], row-major,
 *    Phi fastest. Coefficient fields (kappa, eta, kappa_s, gradients, moments):
 *    [g][i_r][j_theta][l_phi]. Inflow data: g_R1[g][j][l][k < NTheta/2][m]
 *    (cos Theta > 0), g_R2[g][j][l][k - NTheta/2][m] (cos Theta < 0).
 *  - Element type: double for TS_FP64 grids; float for every other precision.
 *    Coefficient fields, gradients and moments are always double.
 *  - Pointers are DEVICE pointers unless the name ends in _host. The caller
 *    owns every pointer it passes; the library owns the grid (tables and
 *    workspace) from ts_create_grid to ts_destroy_grid. Device fields (F, K,
 *    LF, lambda, lambda_prev, x0) must be 16-byte aligned (every cudaMalloc
 *    and PyTorch allocation is; the passes use 16-byte vector accesses);
 *    otherwise TS_ERR_ARG.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Calls are asynchronous on that stream unless stated otherwise.
 *  - Argument errors are returned synchronously and leave the device state
 *    untouched. Launch errors are returned as TS_ERR_CUDA. The text of the
 *    last error of the calling thread is returned by ts_last_error().
 *  - Supported sizes: 3 <= Nr <= 129; 2 <= Ntheta <= 64; Nphi, NTheta, NPhi
 *    even and 2..64; groups >= 1. Otherwise TS_ERR_UNSUPPORTED.
 */
#ifndef TS_H_
#define TS_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TS_OK = 0,
  TS_ERR_ARG = 1,          /* null pointer, non-finite dt, wrong size */
  TS_ERR_UNSUPPORTED = 2,  /* valid request this build does not offer */
  TS_ERR_OOM = 3,          /* device allocation failed */
  TS_ERR_CUDA = 4,         /* a CUDA call or launch failed */
  TS_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
  TS_ERR_STATE = 6         /* call order violated (e.g. step before coefficients) */
} ts_status;

typedef enum {
  TS_FP64 = 0,     /* double storage, double arithmetic */
  TS_FP32 = 1,     /* float storage, float arithmetic */
  TS_FP32_R64 = 2, /* float storage and angular arithmetic; the two radial
                      derivative rows nearest each of r = R1 and r = R2 (the rows
                      with the largest entries) accumulated in double, and the
                      split scheme's implicit collision step in double */
  TS_TF32X3 = 3,   /* float storage; the radial derivative on the tensor cores
                      (tcgen05, operands split into TF32 hi + lo, three products
                      hi*hi + hi*lo + lo*hi accumulated in FP32) for N_r <= 81,
                      angular passes as TS_FP32 (with the environment variable
                      TS_TC_ANGULAR=1 at grid creation, 16 x 16 direction blocks
                      and the isotropic kernel, the Theta and Phi contractions of
                      the angular pass also run on the tensor cores, same split) */
  TS_BF16X3 = 4    /* float storage; the radial derivative on the tensor cores
                      with operands split into three bf16 terms b0 + b1 + b2 and
                      the six products of total order <= 2 accumulated in FP32,
                      for N_r <= 81; angular passes as TS_FP32 */
} ts_precision;

typedef enum {
  TS_RK4 = 0,                 /* classical RK4 on -L F + CT */
  TS_RK4_SPLIT_IMPLICIT = 1,  /* RK4 on -L F, then backward-Euler collision step
                                 (closed form), then F = inflow data at inflow nodes
                                 (implicit first-order source step of App. B) */
  TS_AB2 = 2                  /* second-order Adams-Bashforth on -L F + CT (Sect. 5.1):
                                 F + dt (3/2 K_n - 1/2 K_{n-1}), one stage derivative
                                 per step. The grid keeps K_{n-1} between calls; the
                                 first step after a restart is F + dt K_n. Restarts:
                                 grid creation, ts_set_coeffs,
                                 ts_set_scattering_anisotropy, ts_apply_inflow,
                                 ts_reset_history, and a ts_step on a different F
                                 pointer than the last one. In batches whose
                                 problems are all TS_AB2; its adjoint is
                                 ts_adjoint_step_ab2. */
} ts_scheme;

typedef enum {
  TS_BC_TAU_INFLOW = 0,  /* Tau inflow condition on every stage derivative */
  TS_BC_NONE = 1         /* no boundary rows (operator tests, closed domains) */
} ts_bc;

typedef enum {
  TS_RADIAL_CHEBYSHEV = 0,  /* Chebyshev-Gauss-Lobatto nodes, spectral d_r (Sect. 5.1) */
  TS_RADIAL_UPWIND_FD = 1,  /* the hybrid grid of Sect. 5.3: N_r uniform nodes
                               r_i = R1 + i (R2-R1)/(N_r-1), first-order one-sided
                               differences upstream of each direction (cos Theta > 0:
                               (F_i - F_{i-1})/dr, cos Theta < 0: (F_{i+1} - F_i)/dr);
                               with TS_BC_TAU_INFLOW the inflow nodes hold their data
                               (zero rate) in place of the Tau rows; radial integrals by
                               the trapezoid rule; no radial filter. TS_FP64 and
                               TS_FP32 only; no adjoint, no batches, no
                               ts_moments_noalloc (TS_ERR_UNSUPPORTED). */
  TS_RADIAL_ZONED = 2       /* the three radial zones of App. B: zone_nodes uniform
                               nodes with first-order upwind differences in each edge
                               zone of width zone_width (R2-R1), and Chebyshev-Gauss-
                               Lobatto differentiation on the Nr - 2 (zone_nodes - 1)
                               nodes of the central zone [R1 + w, R2 - w] (the zones
                               share their interface node; Nr counts every node). The
                               rate at an interface node is the upstream zone's (the
                               zone the direction comes from); the central zone takes
                               it at its inflow interface by the Tau method (its top
                               Chebyshev coefficient replaced so that its rate there
                               equals the upstream one). The outer inflow nodes hold
                               their data (zero rate). Radial integrals: trapezoid in
                               the edge zones, Clenshaw-Curtis in the central one. The
                               paper advances the central zone with an implicit
                               radial update; here every zone is explicit (the grid's
                               scheme). TS_FP64 and TS_FP32; no adjoint, no batches,
                               no ts_moments_noalloc (TS_ERR_UNSUPPORTED). */
} ts_radial;

typedef enum {
  TS_FORM_ADVECTIVE = 0,    /* the state is F; the streaming operator is Eq. Liouvsph
                               (coefficient x derivative on every axis) */
  TS_FORM_CONSERVATIVE = 1  /* App. A, Eq. Cohercons: the state is Fhat = r^2 sin(theta)
                               sin(Theta) F (inflow data and ts_apply_inflow too) and
                               the streaming operator its flux divergence:
                                 d_r(cos Th Fhat) + d_th(sin Th cos Ph Fhat / r)
                                 + d_ph(sin Th sin Ph Fhat / (r sin th))
                                 - d_Th(sin Th Fhat / r) - d_Ph(sin Th sin Ph cot th Fhat / r).
                               Fhat is odd under the double-Fourier-sphere reflections
                               (its theta and Theta derivatives continue it with a minus
                               sign at the partner node); the Theta flux is taken as
                               sin Th d_Th Fhat + cos Th Fhat with the Nyquist bin of the
                               doubled Theta circle removed from the second product, the
                               Phi flux as the derivative of sin Ph Fhat; the collision
                               term is r^2 sin th sin Th CT(F) at F = Fhat / (r^2 sin th
                               sin Th). Every flux but the theta one then integrates
                               exactly to its boundary value (ts_number_balance), the
                               theta one to spectral accuracy. Every precision (the float
                               ones compute the angular pass in float);
                               TS_RADIAL_CHEBYSHEV, TS_RK4 or TS_AB2, no filter; no adjoint,
                               moments, flux weights, batches (TS_ERR_UNSUPPORTED). */
} ts_form;

typedef struct {
  double R1, R2;                            /* shell radii, 0 < R1 < R2 */
  int Nr, Ntheta, Nphi, NTheta, NPhi;       /* nodes per axis */
  int groups;                               /* independent energy groups */
  int precision;                            /* ts_precision */
  int scheme;                               /* ts_scheme */
  int bc;                                   /* ts_bc */
  int filter_on;                            /* 1: exponential filter after each step */
  double filter_alpha;                      /* sigma(k) = exp(-alpha (k/kmax)^order) */
  int filter_order;
  int radial;                               /* ts_radial (0: Chebyshev) */
  int zone_nodes;                           /* TS_RADIAL_ZONED: nodes per edge zone (>= 2) */
  double zone_width;                        /* TS_RADIAL_ZONED: edge-zone width / (R2-R1),
                                               in (0, 1/2) */
  int form;                                 /* ts_form (0: advective, the state is F) */
} ts_grid_desc;

typedef struct ts_grid ts_grid;             /* opaque, library-owned */

/* Create a grid: builds the node, differentiation, quadrature and filter
 * tables on the host (Sect. 5.1 bases), uploads them, and allocates the
 * workspace (three fields of the grid's element type plus small buffers) on
 * the current device. Synchronous. *out is NULL on failure. */
ts_status ts_create_grid(const ts_grid_desc* desc, ts_grid** out);

/* Free the grid's tables and workspace. Synchronizes the device first. */
ts_status ts_destroy_grid(ts_grid* grid);

/* Host copies of the nodes: r[Nr] (Chebyshev-Gauss-Lobatto on [R1,R2], or
 * uniform for TS_RADIAL_UPWIND_FD; ascending), theta[Ntheta], phi[Nphi],
 * Theta[NTheta], Phi[NPhi]. Any pointer
 * may be NULL. Synchronous, host memory only. */
ts_status ts_grid_nodes(const ts_grid* grid, double* r_host, double* theta_host,
                        double* phi_host, double* Theta_host, double* Phi_host);

/* Number of elements of one field (groups * Nr * Ntheta * Nphi * NTheta * NPhi). */
size_t ts_field_elems(const ts_grid* grid);

/* Set the absorption kappa, emissivity eta and isotropic scattering kappa_s
 * (Eq. Transp with the density folded in), each [G][Nr][Ntheta][Nphi]
 * double, and the static inflow data g_R1, g_R2 (layout above, element type
 * of the grid). Any pointer may be NULL, meaning zero. Values are copied into
 * the grid (device to device on `stream`). */
ts_status ts_set_coeffs(ts_grid* grid, const double* kappa, const double* eta,
                        const double* kappa_s, const void* inflow_R1,
                        const void* inflow_R2, void* stream);

/* Make the scattering linearly anisotropic (Eqs. sigmadif, crossnun, crossnup,
 * Sect. 3.1 and 6): the kernel becomes (kappa_s/4pi)(1 + b omega.omega'), so
 *   CT = eta - kappa F + kappa_s (J + b omega.H - F),  H = (1/4pi) int omega F dOmega.
 * b: [G][Nr][Ntheta][Nphi] double, DEVICE, copied into the grid on `stream`;
 * b = -1/3 for neutrino-neutron and -1/10 for neutrino-proton scattering, and
 * b = -(A_n/3 + A_p/10)/(A_n + A_p) with kappa_s = 4 pi (A_n + A_p) for their
 * mixture (Eq. cross). The kernel is non-negative for |b| <= 1; values are not
 * checked. NULL restores isotropic scattering (the default). Applies to every
 * later ts_step (every scheme), ts_rhs, ts_adjoint_step and batched step of the
 * grid. TS_ERR_UNSUPPORTED if NTheta < 3 or NPhi < 3 (the split scheme's
 * closed form relies on the direction quadrature integrating omega_i omega_j
 * exactly). The first call allocates one coefficient field on the device. */
ts_status ts_set_scattering_anisotropy(ts_grid* grid, const double* b, void* stream);

/* Add a mu^2 term to the scattering kernel (mu = omega.omega'): with it and
 * ts_set_scattering_anisotropy the kernel is
 *   (kappa_s/4pi)(1 + b mu + c (mu^2 - 1/3)),
 *   CT = eta - kappa F + kappa_s (J + b omega.H + c omega.M~.omega - F),
 * M~ = M - J I/3 the traceless second moment, M = (1/4pi) int omega omega F dOmega.
 * Thomson scattering (3/16pi)(1 + mu^2) per unit sigma_t (Eq. sigmaTh) is c = 3/4,
 * b = 0. c: [G][Nr][Ntheta][Nphi] double, DEVICE, copied into the grid on
 * `stream`; NULL removes the term (the default). The kernel is non-negative
 * when 1 - |b| - c/3 >= 0 and 1 + 2c/3 - |b| >= 0; values are not checked.
 * Applies like ts_set_scattering_anisotropy. TS_ERR_UNSUPPORTED for the split
 * scheme with NTheta < 6 or NPhi < 6 (its closed form relies on the direction
 * quadrature integrating products of four components of omega exactly). The
 * first call allocates one coefficient field on the device. */
ts_status ts_set_scattering_quadrupole(ts_grid* grid, const double* c, void* stream);

/* Set F = inflow data at the inflow nodes (r = R1 with cos Theta > 0, r = R2
 * with cos Theta < 0). Call once on initial data: the Tau rows of ts_step
 * then keep those values fixed. */
ts_status ts_apply_inflow(ts_grid* grid, void* F, void* stream);

/* Forget the TS_AB2 history of the grid: its next step is a forward-Euler
 * starting step. No effect on the other schemes. */
ts_status ts_reset_history(ts_grid* grid);

/* Advance F (in place) by `nsteps` steps of size dt with the grid's scheme,
 * boundary rows, scattering kernel and filter. Requires ts_set_coeffs first
 * (TS_ERR_STATE). Uses the grid's workspace: calls on one grid must not
 * overlap. Launches per step: 12 for TS_RK4 (three passes per stage), 13 for
 * TS_RK4_SPLIT_IMPLICIT, 3 for TS_AB2, plus the filter's when it is on. */
ts_status ts_step(ts_grid* grid, void* F, double dt, int nsteps, void* stream);

/* As ts_step, and also times every kernel launch with CUDA events recorded on
 * `stream` around it. On return (the stream is synchronized):
 *   pass_ms[0..3]  = summed device time in ms of the angular-block passes,
 *                    the (theta,phi)-plane passes, the radial passes (with
 *                    the Tau rows and the stage update), and all other kernels;
 *   launches[0..3] = the number of launches of each.
 * Host arrays of 4 elements; either may be NULL. The events serialize
 * nothing that the plain call does not, but add a small per-launch cost. */
ts_status ts_step_profile(ts_grid* grid, void* F, double dt, int nsteps, double* pass_ms_host,
                          int* launches_host, void* stream);

/* As ts_step, with F in HOST memory: copies F to the device, steps, copies
 * back, and synchronizes `stream` before returning. Float grids with more than
 * one group (and a scheme other than TS_AB2) are pipelined in two chunks of
 * groups: chunk k is stepped on `stream` while chunk k+1 is copied in and chunk
 * k-1 copied out on two copy streams of the grid (one cudaMemcpyAsync per chunk
 * and direction), so only the first chunk's copy in and the last chunk's copy
 * out add to the step's time; the copies are ordered after earlier work on
 * `stream`. Double grids (whose step time dwarfs the copies) and TS_AB2 (whose
 * history covers every group, and follows the host pointer: stepping another
 * F_host restarts it) copy the whole field each way. Allocates a device field
 * on first use. F_host should be pinned for full copy bandwidth. */
ts_status ts_step_host(ts_grid* grid, void* F_host, double dt, int nsteps, void* stream);

/* One stage derivative K = Tau(-L_sph F + CT) (the right-hand side of
 * Eq. Transpfpsph with the grid's boundary rows) written to K. */
ts_status ts_rhs(ts_grid* grid, const void* F, void* K, void* stream);

/* L_sph F alone (Eq. Liouvsph), no collision, no boundary rows. */
ts_status ts_liouville(ts_grid* grid, const void* F, void* LF, void* stream);

/* Discrete adjoint of one ts_step step (TS_RK4 scheme, filter off).
 * Given F_n (the state the step started from) and lambda = dObj/dF_{n+1},
 * overwrites lambda with dObj/dF_n and ADDS this step's contributions to
 * grad_kappa and grad_eta ([G][Nr][Ntheta][Nphi], double):
 *   dObj/dkappa = -sum_stages b_s sum_(Theta,Phi) lambda~_s U_s,
 *   dObj/deta   =  sum_stages b_s sum_(Theta,Phi) lambda~_s,
 * lambda~_s being the stage adjoint after the transposed Tau rows. kappa_s
 * receives no gradient. The paper has no adjoint: this is the exact transpose
 * of the discrete step. Uses the grid's workspace. */
ts_status ts_adjoint_step(ts_grid* grid, const void* F_n, void* lambda,
                          double* grad_kappa, double* grad_eta, double dt, void* stream);

/* Discrete adjoint of one TS_AB2 step (filter off). The marching F_{n+1} =
 * F_n + dt (3/2 K_n - 1/2 K_{n-1}) (Sect. 5.1), started by F_1 = F_0 + dt K_0,
 * uses K_n = K(F_n) in step n (weight 3/2 dt; dt in the starting step) and in
 * step n+1 (weight -1/2 dt). Given F_n, lambda = dObj/dF_{n+1} and lambda_prev =
 * dObj/dF_{n+2} (zeros for the last step), with mu = dt (w lambda -
 * lambda_prev/2), w = 1 if `first` (n = 0) else 3/2: overwrites lambda_prev with
 * lambda and lambda with dObj/dF_n = lambda + A^T Tau^T mu (A the linear part of
 * the stage derivative), and ADDS to grad_kappa and grad_eta ([G][Nr][Ntheta][Nphi])
 * -sum_(Theta,Phi) (Tau^T mu) F_n and sum_(Theta,Phi) Tau^T mu. Walking n = N-1
 * .. 0 with the recomputed states gives the gradients of an objective of F_N.
 * The paper has no adjoint: this is the exact transpose of the discrete AB2
 * step. Uses the grid's adjoint workspace. */
ts_status ts_adjoint_step_ab2(ts_grid* grid, const void* F_n, void* lambda, void* lambda_prev,
                              double* grad_kappa, double* grad_eta, double dt, int first,
                              void* stream);

/* Set the TS_AB2 history: the grid's next ts_step on the field F (the same device
 * pointer) takes K_prev (device, the grid's element type and the layout of F) as
 * K_{n-1} instead of starting with a forward-Euler step. Lets a caller resume
 * AB2 from a saved state F_n and K_{n-1} = K(F_{n-1}) (ts_rhs), e.g. to
 * recompute a checkpointed segment. TS_ERR_UNSUPPORTED for other schemes. */
ts_status ts_set_history(ts_grid* grid, const void* F, const void* K_prev, void* stream);

/* The number balance of App. A (Eqs. Cons, Npho, Flux) of the grid's operator at
 * the state F, per group g: out[5 g + 0..4] = (N, J_R1, J_R2, dN/dt, S) with
 *   N     = int F dV (TS_FORM_ADVECTIVE: int r^2 dr sin th dth dph sin Th dTh dPh F;
 *           TS_FORM_CONSERVATIVE: int dr dth dph dTh dPh Fhat),
 *   J_R   = the radial flux through R (Eq. Flux; int cos Th Fhat(R) for Fhat),
 *   dN/dt = N of the stage derivative WITHOUT Tau rows (the operator itself, with
 *           the grid's collision term),
 *   S     = N of the absorption and emission part, eta - kappa F (times r^2 sin th
 *           sin Th for Fhat), zero for pure scattering,
 * so that dN/dt + J_R2 - J_R1 - S is the operator's balance error: zero to rounding
 * for TS_FORM_CONSERVATIVE up to the theta flux's integral, and for the advective
 * form zero only to spectral accuracy. Quadrature: Clenshaw-Curtis in r, Fejer's
 * first rule in cos theta, cos Theta (on Fhat / sin: int h dth of h = sin th g is
 * Fejer on g), trapezoid in phi, Phi, and the grid's radial rule (Clenshaw-Curtis
 * on Chebyshev nodes, trapezoid on the uniform ones, both on the zoned grid); the
 * sums run in a fixed order. Any precision. out: HOST array of 5 G doubles; the call returns
 * after the result is copied (it synchronises the stream). Allocates and frees one
 * field-sized scratch buffer. */
ts_status ts_number_balance(ts_grid* grid, const void* F, double* out, void* stream);

/* Weights w[Ntheta][Nphi][NTheta][NPhi] (device, double) such that the
 * outgoing radial flux J_R2 of Eq. (Flux), App. A, for group g is
 * sum w * F[g][Nr-1][...]. */
ts_status ts_flux_weights(ts_grid* grid, double* w, void* stream);

/* Outgoing radial flux through R2 per group (Eq. Flux, App. A):
 *   J_R2[g] = sum_{j,l,k,m} w[j][l][k][m] F[g][Nr-1][j][l][k][m]
 * with the weights of ts_flux_weights (the quadrature of ts_moments restricted
 * to the r = R2 slab; equal to ts_moments' J_R2 up to summation order).
 * F: the grid's element type; J_R2: [G] device doubles. Reads only the r = R2
 * slab. Deterministic (fixed summation order). Uses a small scratch buffer of
 * the grid: calls on one grid must not overlap. */
ts_status ts_outgoing_flux(ts_grid* grid, const void* F, double* J_R2, void* stream);

/* Gradient of sum_g gJ[g] J_R2[g] with respect to F (the adjoint seed of the
 * outgoing-flux objective): writes lambda[g][i][...] = gJ[g] w[...] for
 * i = Nr-1 and 0 for every other radial node. gJ: [G] device doubles; lambda:
 * the grid's element type and the layout of F (overwritten entirely). */
ts_status ts_outgoing_flux_adjoint(ts_grid* grid, const double* gJ, void* lambda, void* stream);

/* Angular moments and balances (App. A and App. C), all double:
 *   F0[G][Nr][Nth][Nph] = (1/4pi) int F dOmega,
 *   F1[3][G][Nr][Nth][Nph] = (1/4pi) int F omega dOmega (Cartesian x,y,z,
 *                            Eqs. omegax-omegaz; F = F0 + 3 F1.omega, Eq. Fmom0),
 *   N[G]   = particle number (Eq. Npho, with d Theta),
 *   J_R1[G], J_R2[G] = radial fluxes through R1, R2 (Eq. Flux).
 * Quadrature: Clenshaw-Curtis (r), Fejer's first rule (theta, Theta),
 * trapezoid (phi, Phi). Any output pointer may be NULL. */
ts_status ts_moments(ts_grid* grid, const void* F, double* F0, double* F1, double* N,
                     double* J_R1, double* J_R2, void* stream);

/* The same outputs as ts_moments, for callers that cannot allocate device
 * memory: a process whose device memory is held by another allocator's pool,
 * a deployment with a fixed device-memory budget, or a tight loop that cannot
 * afford an allocation's implicit synchronisation. The paper has no
 * counterpart; this is a property of the library only.
 *  - Takes the grid description instead of a ts_grid (creating a grid
 *    allocates) and computes its node and quadrature tables in the kernel.
 *    Precision selects the element type of F (double for TS_FP64, float for
 *    every other precision).
 *  - Allocates nothing: its per-block partial sums live in a static device
 *    array of 2^21 doubles (16 MiB) that every GPU loading the library holds
 *    until the process exits. Grids needing more than
 *    groups*Nr*Ntheta*Nphi + 2*groups*Ntheta*Nphi > 2^21 doubles are
 *    rejected with TS_ERR_UNSUPPORTED (text in ts_last_error()).
 *  - The first call on a device (with that device current) looks up the
 *    array's device address and caches it; make that first call before any
 *    stream capture. Calls on a stream that is not capturing look it up again,
 *    so a device reset that moves the array is followed; calls during a
 *    capture use the cached address.
 *  - Every call shares the array and it keeps the last call's contents. Each
 *    call writes every slot it reads, so nothing needs clearing, but calls
 *    whose kernels overlap on the GPU (other streams, other host threads)
 *    race on it. */
ts_status ts_moments_noalloc(const ts_grid_desc* desc, const void* F, double* F0, double* F1,
                             double* N, double* J_R1, double* J_R2, void* stream);

/* ---------------------------------------------------------------- tuning
 * Time the candidate tile shapes of the three forward passes of this grid
 * (angular blocks per CTA, Phi column pairs per plane tile, columns per radial
 * tile) with CUDA events and keep the fastest for later calls on this grid.
 * Results are cached per (precision, Nr, Ntheta, Nphi, NTheta, NPhi) for the
 * process and, if the environment variable TS_AUTOTUNE_CACHE names a file,
 * appended to / read from that file. Overwrites the grid's workspace.
 * Synchronous. Tile shapes change results at most at the rounding level: every
 * element is computed by the same operations in any tile, but some shapes
 * select a form of a pass compiled for the grid's sizes. (No counterpart in the
 * paper.) */
ts_status ts_autotune(ts_grid* grid, void* stream);

/* The tile shapes the grid's forward passes use (after ts_autotune, or the
 * built-in choice). Host ints; any pointer may be NULL. */
ts_status ts_tile_shape(const ts_grid* grid, int* angular_blocks, int* plane_pairs,
                        int* radial_columns);

/* ---------------------------------------------------------------- batches
 * Many independent problems of uneven sizes (each with its own grid
 * description, energy groups, scheme and coefficients; one precision for the
 * whole batch) stepped together. Problems of fewer than 2^22 points share one
 * persistent launch per pass of a stage, whose CTAs take tiles of every such
 * problem from an atomic work queue (the run-time-size form of each pass);
 * larger problems, which fill the GPU on their own, are stepped by their
 * grid's own passes (the compiled line-length forms where the sizes have them).
 * A step is captured into a CUDA graph and replayed (captured again when a
 * field pointer, a dt or a problem's coefficients change). A batch runs the
 * RK4 schemes (TS_RK4, TS_RK4_SPLIT_IMPLICIT, mixed freely) or TS_AB2 on every
 * problem; an AB2 batch keeps its history between calls like a grid does (a
 * restart -- new fields, steps or coefficients, or a grid's own history reset
 * -- makes the next step forward Euler for every problem). Results equal those
 * of ts_step on each problem's grid to rounding (bit for bit for the large
 * problems: the same launches), and replaying the graph reproduces them bit for
 * bit. (The paper steps one problem at a time;
 * batching is a property of this library.) */
typedef struct ts_batch ts_batch;

/* Create grids for descs[0..n-1] (as ts_create_grid) and, if autotune != 0,
 * run ts_autotune on each. Synchronous. */
ts_status ts_batch_create(const ts_grid_desc* descs, int n, int autotune, ts_batch** out);

/* Destroy the batch and its grids. Synchronizes the device. */
ts_status ts_batch_destroy(ts_batch* batch);

/* Borrow problem `problem`'s grid (owned by the batch) for ts_set_coeffs,
 * ts_grid_nodes, ts_apply_inflow, ts_moments, ts_step. */
ts_status ts_batch_grid(ts_batch* batch, int problem, ts_grid** grid);

/* Advance every problem by nsteps steps: F_host_array[q] is the DEVICE
 * pointer of problem q's field and dt_host[q] its time step (host arrays of n
 * entries). Every problem needs ts_set_coeffs first (TS_ERR_STATE). Work runs
 * on the batch's own stream, ordered after prior work on `stream` and before
 * later work on `stream`. */
ts_status ts_batch_step(ts_batch* batch, void* const* F_host_array, const double* dt_host,
                        int nsteps, void* stream);

/* ------------------------------------------------- conservative 2-D variant
 * The spherically symmetric problem F(r, Theta) of App. B written for the
 * conservative variable Fhat = r^2 sin(Theta) F (App. B, Eq. flux), with
 * coherent scattering of kernel (kappa_s/4pi)(1 + c (mu^2 - 1/3)):
 *   dFhat/dt = - cos Th dFhat/dr + (1/r) (sin Th dFhat/dTh + cos Th P Fhat)
 *              + kappa_s [ - Fhat + sin Th int_0^pi k_c(Th, Th') Fhat(Th') dTh' ],
 *   k_c = (1/2)(1 + c (cos^2 Th cos^2 Th' + (1/2) sin^2 Th sin^2 Th' - 1/3))
 * (Eq. speccons; c = 3/4 is the Thomson form printed there, c = 0 isotropic
 * scattering). r: Chebyshev-Gauss-Lobatto nodes and differentiation; Theta:
 * the pole-free nodes pi (k+1/2)/NTheta with Fhat odd on the doubled circle;
 * P drops the Nyquist sine mode of Fhat so that the Theta term integrates to
 * zero exactly; Theta' integrals by Fejer's first rule on Fhat / sin Th'. With
 * N = 8 pi^2 int dr int dTh Fhat and J_R = 8 pi^2 int cos Th Fhat(R, Th) dTh
 * (Eqs. Npho, Flux with the theta, phi, Phi integrals done), the discrete
 * operator without boundary rows satisfies dN/dt + J_R2 - J_R1 = 0 (Eq. Cons)
 * to rounding for every Fhat. Time: classical RK4; boundaries: Tau inflow rows
 * (TS_BC_TAU_INFLOW: the rate at each direction's inflow node is zero) or none.
 * FP64. Fields: Fhat[P][Nr][NTheta] (device doubles), P independent problems
 * stepped together, each by one CTA holding its whole grid in shared memory
 * (TS_ERR_UNSUPPORTED if a problem's working set exceeds it). radial =
 * TS_RADIAL_ZONED puts the problem on the three-zone radial grid of App. B (as
 * for ts_grid_desc: zone_nodes uniform nodes with upwind differences in each edge
 * zone of width zone_width (R2-R1), Chebyshev in the central zone, the interface
 * Tau correction; the outer inflow nodes hold their data in place of the Tau
 * rows; radial integrals trapezoid + Clenshaw-Curtis), the configuration the
 * paper runs this problem on; the balance is then exact only up to the edge
 * zones' first-order differences. The paper's own 2-D time scheme (an implicit
 * radial update) is not this one. */
typedef struct {
  double R1, R2;        /* shell radii, 0 < R1 < R2 */
  int Nr, NTheta;       /* 3 <= Nr <= 129; NTheta even, 2..64 */
  int problems;         /* independent problems */
  double scatter_c;     /* kernel parameter c */
  int bc;               /* ts_bc */
  int radial;           /* TS_RADIAL_CHEBYSHEV (0) or TS_RADIAL_ZONED */
  int zone_nodes;       /* TS_RADIAL_ZONED: nodes per edge zone (>= 2) */
  double zone_width;    /* TS_RADIAL_ZONED: edge-zone width / (R2-R1), in (0, 1/2) */
} ts_cons2d_desc;

typedef struct ts_cons2d ts_cons2d;   /* opaque, library-owned */

/* Create: node and differentiation tables (closed forms), uploaded; kappa_s and
 * inflow data zero until set. Synchronous. */
ts_status ts_cons2d_create(const ts_cons2d_desc* desc, ts_cons2d** out);
ts_status ts_cons2d_destroy(ts_cons2d* grid);
/* Host copies of r[Nr] (ascending) and Theta[NTheta]; either may be NULL. */
ts_status ts_cons2d_nodes(const ts_cons2d* grid, double* r_host, double* Theta_host);
/* kappa_s[P][Nr] (device), inflow Fhat data inflow_R1[P][NTheta/2] at R1 for the
 * directions cos Th > 0 and inflow_R2[P][NTheta/2] at R2 for cos Th < 0
 * (device); NULL means zero. Copied on `stream`. */
ts_status ts_cons2d_set_coeffs(ts_cons2d* grid, const double* kappa_s, const double* inflow_R1,
                               const double* inflow_R2, void* stream);
/* Fhat = inflow data at the inflow nodes. */
ts_status ts_cons2d_apply_inflow(ts_cons2d* grid, double* Fhat, void* stream);
/* K = the right-hand side (with the grid's boundary rows) of Fhat. */
ts_status ts_cons2d_rhs(ts_cons2d* grid, const double* Fhat, double* K, void* stream);
/* nsteps classical RK4 steps of size dt, in place, every stage and step in
 * shared memory (one launch per call). */
ts_status ts_cons2d_step(ts_cons2d* grid, double* Fhat, double dt, int nsteps, void* stream);
/* Per problem p: NJ[3p..3p+2] = N, J_R1, J_R2 of Fhat, and residual[p] =
 * dN/dt + J_R2 - J_R1 of the operator without boundary rows (zero to rounding:
 * the discrete form of Eq. Cons). Device doubles. */
ts_status ts_cons2d_balance(ts_cons2d* grid, const double* Fhat, double* NJ, double* residual,
                            void* stream);

/* Measured fused multiply-add rate of the current device in TFLOP/s (2 flops
 * per FMA), for precision TS_FP64 or TS_FP32 (else TS_ERR_UNSUPPORTED): a loop
 * of 8 independent FMA chains per thread, 8 CTAs of 256 threads per SM, best
 * of three timed launches after one warm-up, CUDA events on `stream`.
 * Allocates and frees a small device buffer and synchronizes `stream`. The
 * paper has no counterpart: this is the measured denominator of the roofline of
 * the FP64 passes, which are bound by the FP64 arithmetic units. */
ts_status ts_probe_fma_rate(int precision, double* tflops, void* stream);

/* out[i] = in[i] widened from float to double (device arrays of n elements)
 * by the integer-unit widening the TS_FP32_R64 end rows use (exact: the IEEE-754
 * binary32 fields moved into binary64 ones; subnormals, infinities and NaNs by
 * the conversion instruction), so that tests can compare it bit for bit with the
 * hardware conversion. Asynchronous on `stream`. No counterpart in the paper. */
ts_status ts_probe_widen(const float* in, double* out, size_t n, void* stream);

/* Time-step limit of the grid's explicit stage operator (the Courant limits of
 * Sect. 5.4, every axis included, taken from the discrete operator itself):
 * power iteration on the linear part A x = K(x) - K(0) of the stage derivative
 * K of ts_rhs (the grid's coefficients, scattering kernel and boundary rows),
 * from the start field x0 (device; the grid's element type and the layout of
 * F; any field with a component along the dominant eigenvectors, e.g. seeded
 * random numbers; not modified): x <- A x / |A x| for `iters` iterations
 * (2..100000); rho = the geometric mean of the growth factors |A x| / |x| over
 * the last half of them (Gelfand's formula: it settles even when the largest
 * eigenvalues are a complex pair). dt_max = 2.6 / rho keeps dt A inside
 * classical RK4's stability region (which reaches 2 sqrt 2 on the imaginary
 * axis and 2.79 on the negative real axis). Host outputs, either may be NULL.
 * Overwrites the grid's workspace and restarts the TS_AB2 history; allocates a
 * small scratch buffer on first use; synchronizes `stream`. */
ts_status ts_stable_dt(ts_grid* grid, const void* x0, int iters, double* rho_host,
                       double* dt_max_host, void* stream);

/* Failure-detection hook: bound the tensor-core radial pass's (TS_TF32X3,
 * TS_BF16X3) wait for its operand copy to `operand_wait_iterations` spins of
 * mbarrier.try_wait. 0 restores the default bound (2^24); a negative value
 * makes that wait give up at once, so that every CTA of the pass takes its
 * timeout path: it issues no products, latches the grid's error flag
 * (ts_sync_status then returns TS_ERR_TIMEOUT), waits with the full bound for
 * its own copy to land, frees its tensor memory and returns; that pass's
 * outputs are not written. Only this wait changes: the waits that drain work
 * in flight keep their full bound. Host-side; takes effect at the next
 * launch. (No counterpart in the paper: a test hook of the bounded waits.) */
ts_status ts_set_wait_limit(ts_grid* grid, long long operand_wait_iterations);

/* Status of device-side checks latched since the last call (bounded waits).
 * Synchronizes `stream`. */
ts_status ts_sync_status(ts_grid* grid, void* stream);

/* Text of the last error raised on the calling thread ("" if none). */
const char* ts_last_error(void);

/* Library version string. */
const char* ts_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TS_H_ */
