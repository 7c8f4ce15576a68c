/*
 * dgw.h -- C ABI of the GB300 (sm_103a) DG wall-model operator library (libdgw.so).
 *
 * The library evaluates, matrix-free and by sum factorisation, the spatial DG operators of the
 * function-enrichment wall model of Krank, Kronbichler & Wall (arXiv 1705.08813) on hexahedral
 * Q_k cells, and solves the pressure Poisson problem built on them:
 *   - SIPG pressure Laplacian                 Sec. 4.2, pressure Laplace term, eq. (ipflux)
 *   - velocity divergence (Poisson rhs)       Sec. 4.2, velocity divergence; eq. (poissonspat)
 *   - Lax-Friedrichs convective term          Sec. 4.2, convective term
 *   - multiscale interior-penalty viscous     Sec. 4.2, eq. (viscous_multiscale), (harmweights),
 *     term with the clipped viscosity         Sec. 4.3, eq. (minvt)
 *   - eddy viscosity of the enrichment        Sec. 2.2, eq. (mix), (lmix), (ydes)
 *   - enrichment u~ = psi(y+) sum N_B u~_B     Sec. 3.1 eq. (enrichment), Sec. 3.2 eq. (psi)
 *
 * Conventions (all entry points):
 *   - Vectors are CALLER-OWNED device buffers (e.g. torch tensors). Meshes, metric tables, wall
 *     tables, multigrid hierarchies and solver workspaces are LIBRARY-OWNED.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Applies are
 *     asynchronous on it; dgw_mesh_create, dgw_mesh_info and dgw_pressure_solve synchronise it.
 *   - Every call returns a dgw_status; on error dgw_last_error() returns a thread-local message.
 *     Errors of asynchronous work surface on a later synchronising call.
 *   - Nothing falls back to the CPU: without a CUDA device every compute call fails with
 *     DGW_ECUDA.
 *
 * Canonical layouts (ABI level):
 *   - cells lexicographic: c = i + nx*(j + ny*kz) (x fastest, then y, then z); j = 0 is the
 *     bottom wall row.
 *   - pressure p[c][(k+1)^3], local index a + (k+1)*(b + (k+1)*c3) over the Gauss-Lobatto
 *     nodes (x fastest).
 *   - velocity: standard part u[c][3][(k+1)^3], followed by the enrichment coefficients
 *     u~[e][3][8] (enrich_l = 1, Q1 vertex v = vx + 2 vy + 4 vz) or u~[e][3] (enrich_l = 0,
 *     a constant weight, Sec. 5.1) of the enriched cells; enriched cells are
 *     numbered bottom layer(s) first, then top layer(s), lexicographic (x fastest, then z)
 *     within a layer.
 *   - prec: DGW_FP64 -> buffers are double*, DGW_FP32 -> float*; DGW_DF64 -> buffers are
 *     double*, arithmetic in double-float (pairs of FP32 numbers with error-free
 *     transformations, about 48 significant bits) on the FP32 units, which GB300 runs at 64 times
 *     its FP64 rate; the result agrees with the FP64 apply to about 1e-14 relative to the
 *     magnitude of the summed terms. Only the applies that say so accept DGW_DF64.
 */
#ifndef DGW_H
#define DGW_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgw_mesh *dgw_mesh_t;
typedef struct dgw_server *dgw_server_t;

typedef enum {
  DGW_OK = 0,
  DGW_EINVAL = -1,    /* invalid argument (sizes, degree, null pointers, unsupported option) */
  DGW_ENOMEM = -2,    /* device or host allocation failed / HBM budget exceeded */
  DGW_ENOTCONV = -3,  /* solver reached max_iter before rtol */
  DGW_ETIMEOUT = -4,  /* a bounded wait ran out (serving loop) */
  DGW_EBUSY = -5,     /* job not finished yet (dgw_poll) */
  DGW_ECUDA = -6,     /* CUDA runtime error (no device, launch failure, ...) */
  DGW_EDEVICE = -7    /* a kernel set its device-side error word */
} dgw_status;

enum { DGW_FP64 = 0, DGW_FP32 = 1, DGW_DF64 = 2 };

/* Mesh and discretisation parameters.
 * Channel (geometry 0): [0,lx] x [-ly/2, ly/2] x [0,lz], periodic in x and z, no-slip walls at
 * y = +-ly/2; vertex rows y_j = (ly/2) tanh(gamma (2j/ny - 1)) / tanh(gamma) (Sec. 5.1).
 * Bump (geometry 1; the periodic-hill setting of Sec. 5.2): x in [0,lx], lower wall
 * y_w(x) = 0.3 cos^2(pi (x - lx/2)/2) for |x - lx/2| < 1 (else 0), upper wall y = ly, z in [0,lz],
 * periodic in x and z; the logical point (a0, a1, a2) maps to x = lx a0/nx, z = lz a2/nz,
 * y = y_w + (ly - y_w)(1 + f(a1/ny))/2 with f the tanh grading above, and every cell is the
 * isoparametric Q_k image of its Gauss-Lobatto nodes (J^-1 and det J stored per quadrature point).
 * Enriched cells: the n_layers cell rows next to each wall (Sec. 3.1, eq. enrichment).
 * Wall distance y_B of each Q1 vertex = distance to the closest wall node (vertex for the bump);
 * tau_w,B = tau_w (Sec. 3.2). psi: Spalding's law (wall_law 0, kappa 0.41, B 5.17) or van Driest's law
 * (wall_law 1, eq. psi, evaluated as in Appendix A). */
typedef struct {
  int nx, ny, nz;      /* cells per direction (>= 1; ny >= 2*n_layers when enriched) */
  int degree;          /* k in 1..5 */
  int enrich_l;        /* 1: trilinear weights N^1 (24 coefficients per cell); 0: constant weight (3) */
  int q_wall;          /* Gauss points in the wall-normal direction of enriched cells (1..10) */
  int geometry;        /* 0: channel of boxes, 1: curved bump channel */
  int wall_law;        /* 0 Spalding, 1 van Driest */
  int n_layers;        /* enriched layers per wall (0 = no enrichment) */
  double lx, ly, lz;   /* domain lengths */
  double stretch_gamma;/* tanh grading (> 0) */
  double nu;           /* kinematic viscosity */
  double tau_w;        /* wall shear stress (rho = 1) */
  int precision_mask;  /* bit 0: FP64 tables, bit 1: FP32 tables (for DGW_FP32 applies) */
  int full_quadrature; /* 1: enriched cells take q_wall Gauss points in every direction and faces
                          touching them q_wall per tangential direction (the paper's 8^3 to 12^3
                          rule, Sec. 4.4); 0: q_wall wall-normal only. Both geometries (curved
                          meshes then also tabulate their metric at the q_wall^2 in-plane points). */
} dgw_mesh_params;

/* Build a mesh: geometry, penalty parameters tau_IP (Sec. 4.2: (k+1)^2 A(dK)/V(K), interior
 * faces weighted 1/2, max over both sides; x10 on walls for the viscous term; curved cells
 * integrate A and V with k+2 Gauss points), wall tables
 * (y_h, y+, psi, grad psi at every enriched quadrature point, Sec. 3.2 and Appendix A) and the
 * operator diagonal. Synchronises `stream`. *out receives a library-owned handle. */
dgw_status dgw_mesh_create(const dgw_mesh_params *params, void *stream, dgw_mesh_t *out);
/* Free a mesh and everything the library holds for it (solver, Helmholtz and projection workspaces).
 * Waits for the device; NULL is accepted. Handles, not paper operations: no passage defines these. */
dgw_status dgw_mesh_destroy(dgw_mesh_t mesh);
/* Sizes of the discrete spaces (Sec. 3.1 enrichment, Sec. 4.2 spaces): n_p = nc (k+1)^3,
 * n_u = 3 n_p + 24 n_enriched (enrich_l = 1) or 3 n_p + 3 n_enriched (enrich_l = 0);
 * hbm_bytes = device memory the mesh holds. */
dgw_status dgw_mesh_info(dgw_mesh_t mesh, long *n_p, long *n_u, long *n_enriched, size_t *hbm_bytes);
/* Physical positions of the pressure/velocity nodes (the Gauss-Lobatto nodal points of the Q_k basis,
 * Sec. 4.4; on curved cells the isoparametric map of Sec. 5.2), host buffer of 3*n_p doubles,
 * layout [c][(k+1)^3][xyz]. */
dgw_status dgw_mesh_node_coords(dgw_mesh_t mesh, double *xyz_host);

/* Evaluate nu_t = l_mix^2 |eps(u~)| (Sec. 2.2, eq. mix/lmix/ydes; kappa 0.41, A+ 26,
 * C_DES 0.85, beta 6, h = dy_e/(k+1)) at every quadrature point of the enriched cells and faces
 * from the enrichment part of u_dev (FP64, n_u doubles). The values stay frozen for all later
 * viscous applies until the next call. Before the first call nu_t = 0. */
dgw_status dgw_update_eddy_viscosity(dgw_mesh_t mesh, const double *u_dev, void *stream);

/* Wall shear stress on the linear wall nodes (Sec. 3.2):
 *   tau_w,B = | int_wall N_B rho nu (grad u_h) n dA | / int_wall N_B dA,  rho = 1,
 * the numerator integrated per component before the norm; N_B are the continuous bilinear
 * functions of the wall vertices (periodic in x and z) and u_h = ubar + utilde with the mesh's
 * current enrichment; k+1 Gauss points per tangential direction on each wall face.
 * u_dev: n_u doubles (device). tau_nodes_dev: 2 nx nz doubles (device, caller-owned), node
 * index wall * nx * nz + i + nx * k (wall 0 = bottom). Does not change the mesh. Asynchronous. */
dgw_status dgw_wall_shear_stress(dgw_mesh_t mesh, const double *u_dev, double *tau_nodes_dev, void *stream);

/* Set the nodal wall shear stress (same layout, device buffer) and rebuild the wall tables: the
 * enriched-cell vertices on a wall take their node's value, vertices off the wall the value of
 * the wall node that defines their wall distance y_B; tau_w,h, y+, psi and grad psi follow at every
 * enriched point (Sec. 3.2; the enrichment space changes). nu_t keeps its values until the next
 * dgw_update_eddy_viscosity. Every value must be finite and > 0 (DGW_EINVAL otherwise); the
 * check reads the buffer back, so the call synchronises `stream`. */
dgw_status dgw_set_wall_shear_stress(dgw_mesh_t mesh, const double *tau_nodes_dev, void *stream);

/* Move the velocity into the space of a new nodal wall shear stress (Sec. 3.2, eq. l2): sets
 * tau_nodes_dev as dgw_set_wall_shear_stress does and writes the cell-wise L2 projection of u_old
 * (a vector of the space before the call) onto the new space into u_new: in every enriched cell
 * (v, u_new) = (v, u_old) for all v of the new space, per component, with the velocity point set
 * (k+1 Gauss points in-plane, q_w wall-normal); other cells are copied. The cell systems are
 * solved by Cholesky factorisation in FP64. u_old, u_new: n_u doubles (device, caller-owned; they
 * may be the same buffer). The first call allocates scratch of n_enriched ((k+1)^3 + nef)^2
 * doubles. Synchronises `stream`. DGW_EINVAL for a non-positive or non-finite nodal value or for
 * q_wall < k+3 (l = 1) / k+2 (l = 0), where the wall-normal factor of a wall cell's space has more
 * functions than points and the cell mass matrix is singular;
 * DGW_EDEVICE if a cell matrix is not numerically positive definite (the enrichment and the
 * polynomials are too close to independent there: switch the enrichment off). */
dgw_status dgw_project_velocity(dgw_mesh_t mesh, const double *tau_nodes_dev, const double *u_old_dev,
                                double *u_new_dev, void *stream);

/* Operators of the projection step (Sec. 4.2, eq. projectionspat), FP64, device buffers:
 * pressure gradient y = P(v, p) = -(div v, p)_K + (v, {{p}} n)_dK with {{p}} = p^- on walls, for every
 * velocity test function (standard and enriched). p: n_p doubles, y: n_u doubles. */
dgw_status dgw_apply_gradient(dgw_mesh_t mesh, const double *p, double *y, void *stream);
/* tau_D per cell (eq. tauD): tau_D = |u|_K h dt / Cr with |u|_K the volume average of the velocity
 * magnitude over the cell and h the cube root of the cell volume. u: n_u doubles, tau_d: nc
 * doubles (cells lexicographic). */
dgw_status dgw_tau_divdiv(dgw_mesh_t mesh, const double *u, double dt, double cr, double *tau_d, void *stream);
/* div-div penalty y = D(v, u) = (div v, tau_D div u)_K (eq. div-div), cell-local; u, y: n_u doubles. */
dgw_status dgw_apply_divdiv(dgw_mesh_t mesh, const double *tau_d, const double *u, double *y, void *stream);
/* y = (v, curl u)_K for every velocity test function (standard and enriched), the right-hand side of
 * the vorticity's L2 projection omega_h = M^-1 y (Sec. 4.2, pressure Laplace term). u, y: n_u doubles. */
dgw_status dgw_apply_curl(dgw_mesh_t mesh, const double *u, double *y, void *stream);
/* High-order pressure Neumann data (Sec. 4.1 eq. bc_d_pres, Sec. 4.2 eq. ipflux): adds to the pressure
 * vector b (n_p doubles) the wall integrals (q, g) with
 *   g = -(beta0 (div(u0 x u0) + nu curl w0) + beta1 (div(u1 x u1) + nu curl w1) - f) . n,
 * interior traces at k+1 Gauss points per tangential direction of every wall face; w0, w1 are the
 * vorticities of u0, u1 (dgw_apply_curl then dgw_apply_inverse_mass); beta1 = 0 ignores u1, w1
 * (may be NULL). force: 3 doubles (host). */
dgw_status dgw_add_pressure_neumann(dgw_mesh_t mesh, const double *u0, const double *w0, double beta0,
                                    const double *u1, const double *w1, double beta1, const double *force, double *b,
                                    void *stream);
/* x = M^-1 r (Sec. 4.2 mass term), exactly: cells without switched-on enrichment by the collocation
 * inverse S^-1 W^-1 S^-T, the others by the Cholesky factor of the cell mass matrix (computed on the
 * first call after every change of the space, then kept). r, x: n_u doubles, distinct buffers.
 * Synchronises `stream` when it factorises. */
dgw_status dgw_apply_inverse_mass(dgw_mesh_t mesh, const double *r, double *x, void *stream);

/* Switch-off of the wall model (Sec. 3.2): from now on, and again after every change of tau_w, a
 * wall column is switched off when every point of the velocity point set of its wall-nearest
 * enriched cell has y+ < yplus_off (y+ from the linear y_h and tau_w,h); the paper takes 30 and
 * reports 20 to 30 as equivalent; 0 (the default) never switches off. A switched-off cell is a
 * standard cell for every operator (point sets and face classes included) and its enrichment
 * coefficients keep their slots in the vector: applies and solves write zeros there, and inputs
 * there are ignored. To move a velocity between spaces with different switched-off cells use
 * dgw_project_velocity (whose new space follows the threshold). Asynchronous. */
dgw_status dgw_set_enrichment_switch(dgw_mesh_t mesh, double yplus_off, void *stream);

/* Which enriched cells have the wall model switched on (the switch-off of Sec. 3.2): active_host[e]
 * (n_enriched ints, may be NULL) and their count *n_active (may be NULL). Synchronises `stream`. */
dgw_status dgw_enrichment_active(dgw_mesh_t mesh, int *active_host, int *n_active, void *stream);

/* y = -L(q, p) (Sec. 4.2, SIPG Laplace term with the flux of eq. ipflux on interior and
 * periodic faces; homogeneous Neumann on walls). p, y: n_p values of type `prec`; DGW_DF64 is
 * accepted on the channel (box cells), DGW_EINVAL on curved meshes. */
dgw_status dgw_apply_laplace(dgw_mesh_t mesh, int prec, const void *p, void *y, void *stream);

/* b = -C(q, u) = (grad q, u) - (q, {{u}}.n) with {{u}} = u^- on walls (Sec. 4.2, velocity
 * divergence; boundary rule below eq. poissonspat). u: n_u doubles, b: n_p doubles. */
dgw_status dgw_apply_divergence(dgw_mesh_t mesh, const double *u, double *b, void *stream);

/* The same divergence (Sec. 4.2, velocity divergence item) with a precision: DGW_FP64 (as
 * dgw_apply_divergence) or DGW_DF64 (double
 * vectors, double-float arithmetic on the box rows whose cells and neighbours are standard cells;
 * the rows of and next to the enriched layers are computed in FP64; box cells only, DGW_EINVAL on
 * curved meshes). u: n_u doubles, b: n_p doubles. */
dgw_status dgw_apply_divergence_prec(dgw_mesh_t mesh, int prec, const double *u, double *b, void *stream);

/* y = F^c(v, u) = -(grad v, u x u) + (v, F^c*.n), local Lax-Friedrichs flux with
 * Lambda = max(2|u^-.n|, 2|u^+.n|), mirror state u^+ = -u^- on walls (Sec. 4.2). Over-integrated
 * with floor(3k/2)+1 Gauss points per direction, q_wall wall-normal points in enriched cells
 * (Sec. 4.4). u, y: n_u values of type `prec`; DGW_DF64 as for dgw_apply_divergence_prec. */
dgw_status dgw_apply_convective(dgw_mesh_t mesh, int prec, const void *u, void *y, void *stream);

/* y = -F^nu(vbar, v~; ubar, u~), eq. (viscous_multiscale), with the frozen nu_t of the last
 * dgw_update_eddy_viscosity, harmonic weights eq. (harmweights), clipped viscosity eq. (minvt),
 * penalty with nu only, mirror state on walls. u, y: n_u values of type `prec`; DGW_DF64 as for
 * dgw_apply_divergence_prec. */
dgw_status dgw_apply_viscous(dgw_mesh_t mesh, int prec, const void *u, void *y, void *stream);

typedef struct {
  double rtol;        /* relative residual ||b - A p||_2 / ||b||_2 target (e.g. 1e-10) */
  int max_iter;       /* limit on CG iterations (mode 1: inner iterations summed over refinement steps) */
  int mode;           /* 0: FP64 CG + FP64 multigrid; 1 (mixed): FP64 iterative refinement (p, b - A p
                         and its norm in FP64) around FP32 CG + FP32 multigrid, each inner solve
                         reducing the unit-scaled residual by 1e-5 or to what the target still needs,
                         dot products accumulated in FP64; 2: FP64 CG + Jacobi */
  int cheb_degree;    /* Chebyshev smoother degree (e.g. 5) */
} dgw_solve_opts;

typedef struct {
  int iterations;      /* CG iterations (mode 1: inner FP32 iterations, all refinement steps) */
  double rel_residual; /* true residual of the returned p, recomputed in FP64 */
  float ms;            /* device time of the solve */
  double dof_applies;  /* operator DoF applications inside the solve (all levels, both precisions) */
} dgw_solve_info;

/* Solve -L p = b (Sec. 4.1 eq. poisson, Sec. 4.2 eq. poissonspat) by preconditioned CG on the
 * zero-mean subspace: b is projected to 1^T b = 0 internally (b itself is not modified), p is
 * returned with 1^T p = 0. b, p: n_p doubles. Synchronises `stream`. Returns DGW_ENOTCONV (with
 * p and info filled) when max_iter is reached first. */
dgw_status dgw_pressure_solve(dgw_mesh_t mesh, const double *b, double *p, const dgw_solve_opts *opts,
                              dgw_solve_info *info, void *stream);

/* Mixed-precision solves (mode 1 of dgw_pressure_solve; Sec. 4.1 eq. poisson) of ncols right-hand
 * sides on one mesh, run
 * as one block: up to 8 columns share every launch (the FP32 operator, one captured V-cycle over the
 * block, the FP64 operator of the refinement), dot products are kept per column in a fixed order, so
 * each column's result does not depend on the other columns (the same bits alone or in any block).
 * When ncols > 8, further columns join the block as columns finish (between refinement rounds).
 * b[c], p[c]: device pointers to n_p doubles each (host arrays of ncols pointers); b is projected to
 * zero mean internally, p is returned with zero mean; infos[c] per column (iterations: inner FP32
 * iterations of that column; ms: host time from the column's admission to its completion;
 * dof_applies: the block's applications divided evenly). opts->mode must be 1. Box cells only
 * (geometry 0) and meshes whose coarsest multigrid level is solved densely; otherwise DGW_EINVAL.
 * The block workspace (8 columns) is allocated on first use and kept with the mesh; a call that
 * fails with DGW_ECUDA releases it (the next call starts a new block). Synchronises `stream`.
 * DGW_ENOTCONV if some column reached max_iter. */
dgw_status dgw_pressure_solve_batch(dgw_mesh_t mesh, int ncols, const double *const *b, double *const *p,
                                    const dgw_solve_opts *opts, dgw_solve_info *infos, void *stream);

/* Pressure solve that allocates nothing, for callers that cannot let a library allocate device
 * memory at solve time: code whose device memory belongs to a framework's caching allocator or
 * to a budget fixed at start-up (an allocation outside that pool can fail or exhaust it), and
 * latency-critical loops where cudaMalloc/cudaFree would synchronise the device and stall other
 * streams. The paper has no counterpart; this is a service of the library.
 * Solves -L p = b like dgw_pressure_solve with mode 2 (FP64 CG, Jacobi preconditioner, zero-mean
 * b and p) on `stream`, with all scratch vectors in one file-scope device array of fixed size:
 * 5 * 131072 + 312 doubles (about 5.2 MB), which every GPU that loads the library holds until the
 * process exits. Meshes with n_p > 131072 are rejected with DGW_EINVAL. The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and keeps it for later calls; make
 * that first call before any stream capture, and do not reset the device (cudaDeviceReset)
 * between calls, which would leave the kept address stale. Every call shares the one array and
 * clears what must start at zero; calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller. The solve reads the residual norm
 * back every iteration, so it synchronises `stream` once per iteration and cannot be recorded into a
 * CUDA graph: a stream that is being captured is refused with DGW_EINVAL before any work. info->ms is
 * host wall time. */
dgw_status dgw_pressure_solve_jacobi_noalloc(dgw_mesh_t mesh, const double *b, double *p, double rtol, int max_iter,
                                             dgw_solve_info *info, void *stream);

/* ---- Viscous step of the dual-splitting scheme ------------------------------------------- */

/* y = M(v, u) = (v, u) over every cell (Sec. 4.2 mass term) for the velocity space: standard test
 * functions and, in enriched cells, the enriched ones psi N_B e_a, with the linear-term points
 * (q_wall wall-normal in enriched cells). No face terms. u, y: n_u values of type `prec`. */
dgw_status dgw_apply_mass(dgw_mesh_t mesh, int prec, const void *u, void *y, void *stream);

typedef struct {
  double rtol;        /* relative residual ||rhs - H u||_2 / ||rhs||_2 target */
  int max_iter;       /* limit on GMRES iterations (Krylov vectors built, all restarts) */
  int restart;        /* Krylov vectors per restart cycle (1..64; 0: 30) */
} dgw_helmholtz_opts;

/* Solve the viscous Helmholtz problem of the dual-splitting step (eq. helmholtzspat),
 *   H u = gamma M u - F^nu(vbar, v~; ubar, u~) = rhs,   gamma = gamma_0 / dt > 0,
 * with the nu_t frozen by the last dgw_update_eddy_viscosity (the paper's right-hand side is
 * gamma M u^^ of the projected velocity). u: on entry the initial guess, on exit the solution
 * (n_u doubles, device); rhs: n_u doubles. Restarted GMRES with right preconditioning by the
 * inverse of gamma times the block-diagonal mass (the collocation inverse S^-1 W^-1 S^-T of each
 * cell's standard block, exact off the wall cells, and the inverted enriched blocks), FP64;
 * the workspace ((restart + 1) + restart vectors of n_u doubles) is allocated on first use and kept
 * with the mesh. info->iterations = Krylov vectors built, rel_residual = the true relative residual
 * of the returned u, ms = host wall time. Synchronises `stream`. Returns DGW_ENOTCONV (u and info
 * filled) when max_iter is reached first. */
dgw_status dgw_helmholtz_solve(dgw_mesh_t mesh, double gamma, const double *rhs, double *u,
                               const dgw_helmholtz_opts *opts, dgw_solve_info *info, void *stream);

/* Rate of the adaptive time step (Sec. 4.1: the step follows a CFL condition with the Courant number
 * Cr, whose exact form the paper takes from its reference; reading: rate = the largest Euclidean norm
 * of J^-1 (ubar + u~), the velocity in reference-cell lengths per unit time, over the volume points of
 * the linear point set of every cell (k+1 Gauss points per direction, q_wall wall-normal in enriched
 * cells), and dt = Cr / (k^1.5 rate)). u: n_u doubles (device); *rate: host double. FP64, needs the
 * mesh's FP64 tables. Synchronises `stream`. */
dgw_status dgw_cfl_rate(dgw_mesh_t mesh, const double *u, double *rate, void *stream);

/* ---- Dual-splitting time step ------------------------------------------------------------- */

typedef struct dgw_ns *dgw_ns_t;

typedef struct {
  double dt;              /* constant time step */
  double cr;              /* Courant number of tau_D (eq. tauD; the paper takes 0.14) */
  double force[3];        /* constant body force f (e.g. the mean pressure gradient driving a channel) */
  double rtol_pressure;   /* relative residual of the pressure solve */
  double rtol_projection; /* relative residual of the (M + D) solve of the projection step */
  double rtol_viscous;    /* relative residual of the Helmholtz solve */
  int max_iter;           /* limit on iterations of every solve */
  int pressure_mode;      /* dgw_solve_opts.mode of the pressure solve */
  int update_wall_model;  /* 1: at the start of every step tau_w,B from u^n, the velocity history
                             L2-projected onto the new space, the convective history recomputed */
  int pressure_bc;        /* 0: homogeneous Neumann data for the pressure; 1: the high-order data of
                             eq. bc_d_pres from u^{n-i} and their vorticities */
  int adaptive_dt;        /* 0: constant step dt; 1: dt_n = min(dt, Cr / (k^1.5 dgw_cfl_rate(u^n)))
                             (Sec. 4.1, Cr = cr) with the BDF2 and extrapolation constants of the
                             step ratio w = dt_n / dt_{n-1}: gamma_0 = (1 + 2w) / (1 + w),
                             alpha_0 = 1 + w, alpha_1 = -w^2 / (1 + w), beta_0 = 1 + w, beta_1 = -w */
} dgw_ns_params;

typedef struct {
  int pressure_iterations, projection_iterations, viscous_iterations;
  double ms;              /* host wall time of the step */
  double dt;              /* the step size taken */
} dgw_ns_step_info;

/* A time integrator of the dual-splitting scheme (Sec. 4.1, Galerkin forms of Sec. 4.2) on `mesh`,
 * starting from the velocity u0 (n_u doubles, device, copied). The integrator owns its vectors;
 * the mesh must outlive it. Synchronises `stream`. */
dgw_status dgw_ns_create(dgw_mesh_t mesh, const dgw_ns_params *params, const double *u0, void *stream, dgw_ns_t *out);
/* Free the integrator's vectors (not the mesh); NULL is accepted. A handle of the Sec. 4.1 scheme,
 * not an operation of the paper. */
dgw_status dgw_ns_destroy(dgw_ns_t ns);
/* One time step, BDF2 with second-order extrapolation (first order in the first step), constant dt
 * or (adaptive_dt) the CFL step of dgw_cfl_rate with the variable-step constants:
 *   u^  = (sum alpha_i u^{n-i} + dt f - dt M^-1 sum beta_i F^c(u^{n-i})) / gamma_0 (eq. convstepspat)
 *   A p = (gamma_0 / dt)(-C u^) + (q, g)_walls (eq. poissonspat), g = 0 or the high-order data of
 *         eq. bc_d_pres (pressure_bc = 1) from u^n, u^{n-1} and their vorticities
 *   (M + D) u^^ = M u^ - (dt / gamma_0) P(v, p)                      (eq. projectionspat)
 *   (gamma_0 / dt) M u^{n+1} - F^nu(u^{n+1}) = (gamma_0 / dt) M u^^   (eq. helmholtzspat)
 * with tau_D and nu_t from u^n, CG with the exact inverse mass for the projection and GMRES for the
 * viscous step. Synchronises `stream`. DGW_ENOTCONV if a solve reaches max_iter. */
dgw_status dgw_ns_step(dgw_ns_t ns, dgw_ns_step_info *info, void *stream);
/* Device pointers of the current velocity u^n and pressure p^n of the Sec. 4.1 scheme (owned by the
 * integrator, valid until the next step) and the number of steps taken. */
dgw_status dgw_ns_state(dgw_ns_t ns, const double **u_dev, const double **p_dev, int *steps);
/* Copy the current velocity (n_u doubles) and/or pressure (n_p doubles) of the Sec. 4.1 scheme into
 * caller-owned device buffers (either may be NULL). Asynchronous on `stream`. */
dgw_status dgw_ns_copy_state(dgw_ns_t ns, double *u_dev, double *p_dev, void *stream);

/* Describe (building it if needed) the multigrid hierarchy of `mode` (0 FP64, 1 FP32) that
 * preconditions the pressure solve (Sec. 4.4 names a multigrid-preconditioned CG; the hierarchy is
 * this library's own design): number of
 * levels, the estimated largest eigenvalue of D^-1 A per level (the Chebyshev smoother works on
 * [1.1 lmax / 45, 1.1 lmax]) and the cell count per level, finest first; at most max_levels
 * entries are written. Synchronises the library's solver stream. */
dgw_status dgw_solver_describe(dgw_mesh_t mesh, int mode, int *n_levels, double *lmax, int *cells, int max_levels,
                               void *stream);

/* ---- Request loop (serving) --------------------------------------------------------------
 * No counterpart in the paper: a service for running many independent jobs. Jobs of any mesh size
 * and degree are admitted as worker slots and device memory free up; each job runs on a resident
 * mesh with its parameters (created on first use, kept for later jobs, at most one job per mesh
 * instance at a time, idle meshes evicted least-recently-used when the HBM budget is short), and
 * each worker has its own CUDA stream, so concurrent jobs overlap on the device. Mixed-precision
 * solves (opts.mode 1) on channel meshes are batched continuously: the worker that takes one runs it
 * as a block solve (dgw_pressure_solve_batch's engine) and, between refinement rounds, admits queued
 * solves with the same mesh parameters and Chebyshev degree into free columns (up to 8); a column
 * that converges is reported at once and frees its column. Results do not depend on the mix (jobs
 * share no scratch; all kernels and reductions are deterministic and per column). */
enum { DGW_JOB_SOLVE = 0, DGW_JOB_LAPLACE = 1, DGW_JOB_DIVERGENCE = 2, DGW_JOB_CONVECTIVE = 3, DGW_JOB_VISCOUS = 4 };

typedef struct {
  int kind;               /* DGW_JOB_* */
  int prec;               /* applies: DGW_FP64 or DGW_FP32 (divergence and solves are FP64) */
  dgw_mesh_params mesh;   /* mesh of the job (meshes are cached by these parameters) */
  const void *in;         /* caller-owned device input: b (solve), p (Laplace), u (other applies) */
  void *out;              /* caller-owned device output: p (solve) or y */
  const double *aux;      /* viscous only: FP64 velocity (n_u) that freezes nu_t before the apply;
                             NULL keeps the mesh's current nu_t */
  dgw_solve_opts opts;    /* solves only */
} dgw_job;

/* Serving (no counterpart in the paper; a service of the library around the solve of Sec. 4.1).
 * Start a request loop with `max_inflight` worker slots (1..64) and a device-memory budget for
 * resident meshes and solver state. */
dgw_status dgw_server_create(size_t hbm_budget, int max_inflight, dgw_server_t *out);
/* Queue a job. Its input must be complete on the device when submitted (synchronise the stream
 * that produced it); in, out and aux must stay valid until dgw_poll reports completion. A viscous
 * job with aux != NULL first freezes nu_t from aux (dgw_update_eddy_viscosity), then applies. */
dgw_status dgw_submit(dgw_server_t server, const dgw_job *job, long *ticket);
/* Non-blocking. Returns DGW_EBUSY (and *job_status = DGW_EBUSY) while the job is queued or running;
 * otherwise DGW_OK with the job's own status (DGW_ENOMEM if it can never fit the budget), the solve
 * info (solves) and the submit-to-completion latency. A completed ticket is reported once. */
dgw_status dgw_poll(dgw_server_t server, long ticket, dgw_status *job_status, dgw_solve_info *info, double *latency_ms);
/* Queue depth, running jobs, resident meshes and reserved device bytes (request loop; no counterpart
 * in the paper). */
dgw_status dgw_server_stats(dgw_server_t server, int *queued, int *running, int *resident_meshes, size_t *reserved_bytes);
/* Cancel queued jobs and wait up to timeout_ms for running ones; on DGW_ETIMEOUT the server stays
 * alive (running jobs still own their streams) and may be destroyed again later. */
dgw_status dgw_server_destroy(dgw_server_t server, int timeout_ms);

/* Thread-local description of the last error. */
const char *dgw_last_error(void);

/* Process-wide counters since the library was loaded (no counterpart in the paper): kernels the
 * library launched, and operator DoF applications (the output DoFs of every operator apply,
 * including those inside solves). */
void dgw_counters(unsigned long long *kernel_launches, unsigned long long *dof_applies);

#ifdef __cplusplus
}
#endif

#endif /* DGW_H */
