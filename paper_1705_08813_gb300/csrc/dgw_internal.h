// Internal data structures of libdgw (host and device). Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/dgw.h"

namespace dgw {

constexpr int NMAX = 6;    // max nodes per direction (k <= 5)
constexpr int QMAX = 10;   // max quadrature points per direction
constexpr int QW_MAX = 10; // max wall-normal points in enriched cells

// Quadrature sets: 0 = k+1 Gauss points (linear terms), 1 = floor(3k/2)+1 (convective term),
// 2 = q_wall points (wall-normal direction of enriched cells), Sec. 4.4.
enum { QSET_LIN = 0, QSET_CONV = 1, QSET_WALL = 2, NQSET = 3 };

// Gauss-Lobatto nodal basis tabulated at Gauss points, for one degree. S[s][q*n1+j] = l_j(x_q),
// D[s][q*n1+j] = l_j'(x_q); dend[side][j] = l_j'(side); x, w: Gauss points/weights on [0,1].
template <typename T>
struct Basis {
  int n1;
  int q[NQSET];
  T S[NQSET][QMAX * NMAX];
  T D[NQSET][QMAX * NMAX];
  T x[NQSET][QMAX];
  T w[NQSET][QMAX];
  T dend[2][NMAX];
  T mass[NMAX * NMAX];   // 1-D reference mass matrix sum_q w_q l_a(x_q) l_b(x_q)
  // h-multigrid embedding: P[o][i*n1+j] = l_j((o + xhat_i)/2), child offset o in {0,1}
  T P[2][NMAX * NMAX];
};

// Per-point wall-table record of an enriched cell: psi and its physical gradient.
constexpr int WT = 4;

// Cell geometry: axis-aligned boxes (channel) or isoparametric curved cells (bump).
enum { GEO_BOX = 0, GEO_CURVED = 1 };

// Metric record of a curved cell at one point: J^-1 row-major ([r*3+c] = d xi_r / d x_c), det J.
constexpr int MREC = 10;
// Volume metric tables by (x-set, y-set): (lin, lin), (conv, conv), (lin, wall), (conv, wall) and,
// for the q_w^3 rule in enriched cells (full_quadrature), (wall, wall).
constexpr int NMVOL = 5;
constexpr int MVOL_WALL_WALL = 4;

// Device-side view of a mesh in precision T.
template <typename T>
struct MeshView {
  int nx, ny, nz, n1, nc, ne;
  int q[NQSET];       // point counts of the quadrature sets (host-visible copy)
  long np, nu;
  int nef;            // enrichment coefficients per component and wall cell: 8 (l = 1) or 1 (l = 0)
  int full_q;         // 1: enriched cells use the q_wall set in every direction (faces: both tangential)
  int geo;            // GEO_BOX or GEO_CURVED
  // rows [plain_lo, plain_hi) hold standard box cells (no enrichment slot in the row; with the q_w^3
  // rule none in the rows above and below either): the degree-specialised kernels of box_ops.cu take
  // them, adding an enriched y-neighbour's u~ on the faces between; the general kernel the other rows
  // (plain_lo = plain_hi = ny: all general)
  int plain_lo = 0, plain_hi = 0;
  // rows [std_lo, std_hi) hold no enrichment slot: the volume-only operators (mass, div-div) take
  // them with box kernels whatever the neighbours (std_lo = std_hi = ny: all general)
  int std_lo = 0, std_hi = 0;
  T hx, hz;
  const T *hy;        // [ny] row heights (boxes)
  const T *tau;       // [nc] penalty tau_IP per cell
  const T *rowops;    // [ny][24] per-row scalars of the factorised Laplace operator (boxes)
  // curved metric tables per metric column m = i + nx*j (the map is an extrusion along z):
  // mvol[pair]: [m][a1][a0][MREC]; mxf[y-set]: [m][side][a1][MREC] (faces xi_0 = side);
  // myf[x-set]: [m][side][a0][MREC] (faces xi_1 = side); faces xi_2 = side use mvol. The tables of
  // the (wall, wall) pair and myf[QSET_WALL] exist only on meshes with the q_w^3 rule.
  const T *mvol[NMVOL];
  const T *mxf[NQSET];
  const T *myf[NQSET];
  // curved SIPG Laplacian tables per metric column (k+1 Gauss points): lvol [m][(k+1)^3][6] =
  // |det J| w J^-1 J^-T (xx yy zz xy xz yz); lface [m][6][(k+1)^2][7] = dA, dA J^-1 n of the own
  // side, dA J^-1 n of the neighbour at the shared point (n the own outward normal; zero on walls)
  const T *lvol;
  const T *lface;
  const int *enr;     // [nc] enriched index or -1 (-1 also where the wall model is switched off)
  const int *slot;    // [nc] enriched index whether switched on or off, -1 off the wall layers
  T visc;             // kinematic viscosity nu
  const Basis<T> *basis;
  // wall tables [qset lin/conv]: volume [ne][nvol][WT], faces [ne][6][fpmax][WT]
  const T *wt_vol[2];
  const T *wt_face[2];
  int nvol[2], fpmax[2];
  // frozen eddy viscosity (linear quadrature set): [ne][nvol[0]], [ne][6][fpmax[0]]
  const T *tau_d = nullptr;   // [nc] div-div penalty per cell (OP_DIVDIV; set per call)
  const T *nut_vol;
  const T *nut_face;
};

// One multigrid level (a nested coarser channel mesh with the same degree).
struct Level;
struct Batch;

struct MeshHost;

}  // namespace dgw

// Opaque handle behind dgw_mesh_t.
struct dgw_mesh {
  dgw_mesh_params P;
  int n1, nc, ne;
  int nef = 8;                  // 8 (l = 1) or 1 (l = 0)
  long np, nu;
  size_t hbm_bytes = 0;
  std::vector<double> yv;       // vertex rows
  std::vector<double> hy;       // row heights
  std::vector<double> tau;      // per cell tau_IP
  std::vector<int> enr;         // cell -> enriched index
  std::vector<int> enr_cell;    // enriched index -> cell
  std::vector<double> ywall;    // [ne][8] vertex wall distances
  std::vector<double> tauv;     // [ne][8] vertex wall shear stresses
  std::vector<int> tsrc;        // [ne][8] wall node that defines the vertex's wall distance
  std::vector<double> dye;      // [ne] wall-normal width
  std::vector<double> cxn, cyn; // curved: nodal (x, y) per metric column [nx*ny][n*n]
  dgw::Basis<double> basis64;   // host copies of the basis tables
  dgw::Basis<float> basis32;
  // device allocations (owned)
  std::vector<void *> allocs;
  dgw::MeshView<double> v64;
  dgw::MeshView<float> v32;
  bool has32 = false;
  double *hy_dev64 = nullptr;
  int *enr_cell_dev = nullptr;
  double *wall_ywall_dev = nullptr, *wall_tauv_dev = nullptr;
  int *tsrc_dev = nullptr;
  int *slot_dev = nullptr;          // [nc] enriched index (layout), constant
  int *wslot_dev = nullptr;         // [ne] enriched index of the wall-nearest cell of the column
  double yp_off = 0.0;              // switch-off threshold on y+ (0: never)
  double *wall_mom_dev = nullptr;   // [2 nx nz][16] per-wall-face moments of the tau_w update
  double *proj_A = nullptr;         // L2 projection scratch: [ne][N][N] cell matrices (lazily allocated)
  double *proj_P = nullptr;         // [ne][points][3] old field at the points
  int *proj_err = nullptr;
  int proj_nvec = 0;                // vectors proj_P has room for
  bool mass_factor_valid = false;   // proj_A holds the Cholesky factors of the current space
  double *aux_vol = nullptr, *aux_face = nullptr;   // (y_h, y+, l_mix^2) at linear-set points
  double *dye_dev = nullptr;
  double *diag64 = nullptr;     // Jacobi diagonal of the Laplace operator
  float *diag32 = nullptr;
  struct dgw_solver *solver = nullptr;   // lazily built solver workspace and multigrid hierarchy
  struct dgw_helm *helm = nullptr;       // lazily built Helmholtz (GMRES) workspace
  dgw::Batch *batch = nullptr;           // lazily built block solver (batched mixed-precision solves)
  double *rate_dev = nullptr;            // device scalar of dgw_cfl_rate (allocated on first use)
  int batch_cheb = 0;                    // its Chebyshev degree
};

namespace dgw {

// process-wide counters: kernel launches and operator DoF applications (output DoFs of every
// operator apply, including the applies inside solves)
void note_launch();
void note_launches(unsigned long long n);
void note_dofs(long long n);
unsigned long long dof_counter();
unsigned long long launch_counter();

// error reporting (thread-local message)
dgw_status set_error(dgw_status s, const std::string &msg);
dgw_status cuda_check(cudaError_t e, const char *what);

// host-side 1-D rules (Gauss-Legendre, Gauss-Lobatto, barycentric Lagrange)
void gauss_rule(int n, double *x, double *w);
void lobatto_nodes(int n, double *x);
template <typename T>
void fill_basis(int k, int q_conv, int q_wall, Basis<T> *b);
void embed_matrix(int n, double a, double b, double *P);
// Lagrange basis on the nodes z[0..n-1] at s: values l_j(s) and derivatives l_j'(s).
void lagrange_row(int n, const double *z, double s, double *val, double *der);

// Geometry of a channel of boxes: uniform x and z spacing, graded rows in y.
struct BoxGeometry {
  int nx, ny, nz, k;
  double hx, hz;
  std::vector<double> yv, hy, tau;
};
// Row heights and penalty tau_IP = (k+1)^2 A(dK)/V(K) (interior faces weighted 1/2, walls 1).
void box_geometry(int k, int nx, int ny, int nz, double lx, double lz, const std::vector<double> &yv, BoxGeometry &g);
// Diagonal of the SIPG Laplacian (Jacobi), from the 1-D mass and stiffness diagonals.
void laplace_diagonal(const BoxGeometry &g, const Basis<double> &B, std::vector<double> &dg);
// Per-row 1-D operators of the factorised SIPG Laplacian on boxes (full matrices, host use).
void box_rowops(const BoxGeometry &g, const Basis<double> &B, std::vector<double> &R);
// Per-row scalars of the same operator for the device kernel ([ny][24]).
void box_rowscal(const BoxGeometry &g, std::vector<double> &R);
// Degree tables of the box kernel in constant memory (once per device; host-synchronous).
cudaError_t box_constants_init();
// Host evaluation of the same factorised operator (small coarse-level matrices).
void host_box_apply(const BoxGeometry &g, const Basis<double> &B, const std::vector<double> &R, const double *x,
                    double *y);

// Curved bump channel (geometry 1), host side: metric tables, penalty and wall data of a mesh
// with nx x ny x nz cells of degree k over the bump map of the parameters.
struct CurvedHost {
  int nx, ny, nz, k;
  std::vector<double> mvol[NMVOL], mxf[NQSET], myf[NQSET];   // layouts as in MeshView
  std::vector<double> tau;                               // [nx*ny] per metric column
  std::vector<double> lvol, lface;                       // Laplace tables (layout as in MeshView)
  std::vector<double> xn, yn;                            // [nx*ny][n*n] nodal (x, y), x-node fastest
};
void curved_geometry(const dgw_mesh_params &P, int nx, int ny, int nz, int k, const Basis<double> &B, CurvedHost &G);
// Physical (x, y) of the logical coordinates (a0, a1) of the bump map (z is lz a2 / nz).
void bump_point(const dgw_mesh_params &P, int nx, int ny, double a0, double a1, double *x, double *y);

// Elementwise epilogue of a Laplace apply t = A x, fused into the operator kernel:
//   LAP_PLAIN y = t; LAP_RESIDUAL y = b - t;
//   LAP_CHEB  Chebyshev step d = (first ? 0 : c1 d) + c2 D^-1 (b - t), xout = x + d (xout != x:
//             neighbouring cells still read x; y is not written).
enum { LAP_PLAIN = 0, LAP_RESIDUAL = 1, LAP_CHEB = 2 };
//   ncols > 1 (boxes): the vectors hold ncols columns of np values each (dinv is shared), one
//             launch applies the operator to every column (gridDim.y = ncols).
template <typename T>
struct LapEpi {
  int mode;
  const T *b;
  T *d;
  const T *dinv;
  T *xout;
  T c1, c2;
  int first;
  int ncols;
};

// kernels (launched by api.cu)
template <typename T>
cudaError_t launch_laplace(const MeshView<T> &m, const T *p, T *y, cudaStream_t s);
template <typename T>
cudaError_t launch_laplace_epi(const MeshView<T> &m, const T *p, T *y, const LapEpi<T> &epi, cudaStream_t s);
// y = A_L p with double vectors in double-float arithmetic on the FP32 units (box cells only)
cudaError_t launch_laplace_df(const MeshView<double> &m, const double *p, double *y, cudaStream_t s);
// Jacobi diagonal of the SIPG Laplacian of a curved mesh (FP64, one thread per DoF)
cudaError_t launch_curved_diagonal(const MeshView<double> &m, double *dg, cudaStream_t s);
// SIPG Laplacian on curved cells from the lvol/lface tables (degree-specialised line passes)
template <typename T>
cudaError_t launch_curved_laplace(const MeshView<T> &m, const T *p, T *y, const LapEpi<T> &epi, cudaStream_t s);
// Degree tables of the curved Laplace kernel in constant memory (once per device; host-synchronous)
cudaError_t curved_constants_init();
template <typename T>
cudaError_t launch_vector_op(int op, const MeshView<T> &m, const T *u, T *y, cudaStream_t s,
                             const LapEpi<T> *epi = nullptr);
// the same operator with double vectors and double-float arithmetic on the box rows the
// specialised kernels take (the general kernel computes the other rows in FP64); OP_DIV, OP_VISC,
// OP_CONV
cudaError_t launch_vector_op_df(int op, const MeshView<double> &m, const double *u, double *y, cudaStream_t s);
struct df64;
// degree-specialised box-cell kernels on rows [j0, j0 + nrows) (box_ops.cu); R = compute type
template <typename T, typename R>
cudaError_t launch_box_vec_rows(int op, const MeshView<T> &m, const T *u, T *y, int j0, int nrows, cudaStream_t s);
cudaError_t launch_wall_tables(dgw_mesh *M, cudaStream_t s);
cudaError_t launch_wall_shear(dgw_mesh *M, const double *u, double *tau_nodes, cudaStream_t s);
cudaError_t launch_set_tau_nodes(dgw_mesh *M, const double *tau_nodes, cudaStream_t s);
cudaError_t launch_switch(dgw_mesh *M, cudaStream_t s);
cudaError_t launch_projection(dgw_mesh *M, const double *tau_new, int nvec, const double *const *u_old,
                              double *const *u_new, cudaStream_t s, int *bad_cell);
cudaError_t launch_inverse_mass_cells(dgw_mesh *M, const double *r, double *x, cudaStream_t s);
cudaError_t launch_collocation_inverse_mass(dgw_mesh *M, const double *r, double *x, cudaStream_t s);
// modes of the projection-step kernel: pressure gradient P(v, p), tau_D per cell, (v, curl u)
enum { NS_GRAD = 0, NS_TAU = 2, NS_CURL = 3 };
cudaError_t launch_ns_op(int mode, dgw_mesh *M, const double *in, double dt_over_cr, double *y, cudaStream_t s);
cudaError_t launch_pressure_neumann(dgw_mesh *M, const double *u0, const double *w0, double b0, const double *u1,
                                    const double *w1, double b1, const double *f, double *y, cudaStream_t s);
cudaError_t launch_eddy_viscosity(dgw_mesh *M, const double *u, cudaStream_t s);
cudaError_t launch_to_float(const double *a, float *b, size_t n, cudaStream_t s);

enum { OP_DIV = 0, OP_CONV = 1, OP_VISC = 2, OP_LAP = 3, OP_MASS = 4, OP_DIVDIV = 5, OP_CFL = 6 };
// max over cells and the linear volume point set of |J^-1 (ubar + u~)|_2 into *rate (a device double,
// zeroed by the caller; FP64 only): the speed that sets the adaptive time step
cudaError_t launch_cfl_rate(const MeshView<double> &m, const double *u, double *rate, cudaStream_t s);

}  // namespace dgw
