// Internal declarations of libmhde (host setup, device kernels, solver).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <tuple>
#include <utility>
#include <string>
#include <vector>

#include "../../include/mhde.h"

namespace mhde {

constexpr int NQ = 7;        // quadrature points per triangle (degree-5 rule)
constexpr int NLOC = 6;      // P2 nodes per triangle
constexpr int MAX_J = 64;    // members per ensemble handled by the small dense kernels
constexpr int KIN_MAX = 16;  // longest inner GMRES on F
constexpr int IG_PMAX = 512;  // largest grid of the persistent inner GMRES

// ----------------------------------------------------------------- host FE data
struct HostCsr {
  int nrows = 0, ncols = 0;
  std::vector<int> rowptr, col;
  std::vector<double> val;
  long long nnz() const { return (long long)col.size(); }
};

struct AmgLevelHost {
  HostCsr A;                  // level operator
  std::vector<double> dinv;   // 1 / diag(A)
  double omega = 0.0;         // Jacobi damping 4 / (3 rho(D^-1 A))
  HostCsr P, R;               // prolongation to this level from the next, R = P^T
  // block-Jacobi smoother instead of point Jacobi (level 0 of the
  // discontinuous pressure): bs > 0 gives blocks of bs dofs
  // blk_idx[b*bs + i] with dense inverses of A's diagonal blocks
  // blk_inv[b][bs][bs] and damping blk_omega = 1.6 / rho(Binv A)
  int bs = 0;
  std::vector<int> blk_idx;
  std::vector<double> blk_inv;
  double blk_omega = 0.0;
};

struct AmgHost {
  std::vector<AmgLevelHost> levels;   // levels[0] = fine pressure Laplacian (pinned)
  int nc = 0;                         // coarsest size
  std::vector<double> coarse_inv;     // dense inverse of the coarsest operator [nc][nc]
};

struct FeHost {
  int nv = 0, nt = 0, ne = 0, n2 = 0, np = 0;
  int element = 0;                        // 0 continuous P1 pressure, 1 discontinuous (3 dofs per triangle)
  std::vector<double> xy;                 // [nv][2]
  std::vector<int> tri;                   // [nt][3]
  std::vector<long long> edges;           // sorted keys a * nv + b, a < b
  std::vector<int> edge_count;            // triangles per edge
  std::vector<int> dofs;                  // [nt][6]
  std::vector<unsigned char> is_bnd;      // [n2]
  std::vector<int> bnd_nodes;             // boundary P2 nodes, ascending
  std::vector<double> node_xy;            // [n2][2]
  std::vector<double> geom;               // [nt][8]: grad lambda_0..2 (x, y), det, pad

  // scalar P2 pattern F (n2 x n2) and its element scatter map
  HostCsr F;                              // pattern only
  std::vector<int> f_slot_nnz;            // [nt*36] nnz index of element slot (a, b)
  std::vector<int> f_gather_ptr;          // [nnzF + 1]
  std::vector<int> f_gather_slot;         // [nt*36] slots sorted by nnz then slot id
  std::vector<int> f_diag;                // [n2] nnz index of the diagonal

  // divergence pattern B (np x n2) with scatter map, and its transpose
  HostCsr B;                              // pattern only
  std::vector<int> b_gather_ptr;          // [nnzB + 1]
  std::vector<int> b_gather_slot;         // [nt*18] element slots e*18 + i*6 + a
  HostCsr BT;                             // pattern (n2 x np)
  std::vector<int> bt_src;                // [nnzB] index into B's values

  // node -> element-local slot lists (e*6 + a) for node-wise gathers
  std::vector<int> node_ptr;              // [n2 + 1]
  std::vector<int> node_slot;             // [nt*6]

  // pressure Laplacian (dof 0 pinned) and lumped pressure mass.  Either the
  // P1 stiffness of the continuous pressure, whose element -> nnz map (slots
  // e*9 + 3i + k) also assembles the pressure convection matrix of the PCD
  // Schur approximation, or the algebraic B D^{-1} B^T (build_algebraic_laplacian)
  HostCsr Kp;
  std::vector<int> p1_gather_ptr;         // [nnzKp + 1] (P1 stiffness only)
  std::vector<int> p1_gather_slot;        // [nt*9]
  std::vector<double> mp_lumped;          // [np]
  std::vector<double> lsc_dinv;           // [n2] 1/D on interior P2 nodes, 0 on Dirichlet nodes
  AmgHost amg;
};

// Builds everything above but Kp for element 1 (see below); returns an empty
// string or an error message.  element: 0 continuous P1 pressure
// (Taylor-Hood), 1 discontinuous P1 pressure (Scott-Vogelius).
std::string build_fe(const mhde_mesh* mesh, FeHost& fe, int element);
// Replaces Kp by L = sum_d B_d D^{-1} B_d^T over the interior P2 nodes (D the
// diagonal of the P2 mass matrix scaled to the element areas), dof 0 pinned:
// the pressure Laplacian of the discontinuous pressure and of the
// least-squares commutator.  Fills lsc_dinv.
std::string build_algebraic_laplacian(FeHost& fe);
std::string build_amg(FeHost& fe, int coarse_max);

// ----------------------------------------------------------------- small dense (host, FP64)
// Symmetric eigen-decomposition of an n x n matrix (row-major, copied):
// eigenvalues descending in w, eigenvectors in the columns of U (row-major).
void eig_sym(int n, const double* A, double* w, double* U);

// Cholesky QR factors T = R^{-1}, S = R of a Gram matrix G = R^T R (r x r,
// row-major), only when full rank is certain (every eigenvalue above
// 100 thresh lambda_max); false otherwise (callers then use the eigen form).
bool cholqr_factors(int r, const std::vector<double>& G, double thresh, std::vector<double>& Tm,
                    std::vector<double>& Sm);

// Incremental least squares for block GMRES: block upper Hessenberg H with
// block width r and the right-hand side E1 S0 (S0 is r x J).
struct BlockLS {
  int r = 0, J = 0, m = 0, k = 0;
  int ldr = 0;                 // m r: row length of R
  std::vector<double> R;       // (m r) x (m r), row-major, upper triangular
  std::vector<double> hv;      // Householder vectors, 2r per reflector
  std::vector<double> htau;    // [m r]
  std::vector<double> g;       // ((m+1) r) x J, row-major: the rotated right-hand sides
  std::vector<double> c, s;    // work: the new block column, dot products
  void init(int r_, int J_, int m_, const double* S0 /* r x J row-major */);
  // h: ((k+2) r) x r row-major = the new block column [H_0; ...; H_k; S_{k+1}].
  // Returns false on a (numerically) singular diagonal.
  bool add(const double* h);
  // residual norm of right-hand-side column j after the last add
  double resid(int j) const;
  // solve R Y = g[0:(k r)] -> Y ((k r) x J) row-major
  void solve(std::vector<double>& Y) const;
};

// ----------------------------------------------------------------- device data
struct DevCsr {
  int nrows = 0, ncols = 0;
  long long nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  float* valf = nullptr;
  double* dinv = nullptr;
  float* dinvf = nullptr;
};

struct DevAmgLevel {
  DevCsr A, P, R;
  double omega = 0.0;
  int bs = 0, nb = 0;                           // block-Jacobi smoother (bs > 0): nb blocks of bs dofs
  int* blk_idx = nullptr;                       // [nb][bs]
  double* blk_inv = nullptr;  float* blk_invf = nullptr;   // [nb][bs][bs]
  double blk_omega = 0.0;
  double* x = nullptr;  float* xf = nullptr;   // [n][Jp] work vectors
  double* b = nullptr;  float* bf = nullptr;
  double* r = nullptr;  float* rf = nullptr;
};

struct Sub {                       // one subproblem (v: which = 0, w: which = 1)
  int which = 0;
  BlockLS ls;                      // block least-squares state of the current GMRES cycle
  cudaStream_t stream = nullptr;
  double* Fval = nullptr;          // [nnzF]
  float* Fvalf = nullptr;
  double* Fdinv = nullptr;         // [n2]
  float* Fdinvf = nullptr;
  double* FD = nullptr;            // [nnzF] F[k] * dinv[col[k]]: the inner solve's operator F D^{-1}
  float* FDf = nullptr;
  double* Floc = nullptr;          // [nt][36] element slot buffer
  double* Cloc = nullptr;          // [nt][6][2][Jp] convection slot buffer of the RHS
  double* Bv = nullptr;            // right-hand sides [n_rows][Jp]
  double* X = nullptr;             // next state [n_rows][Jp]
  double* S = nullptr;             // current state [n_rows][Jp]
  double* Sprev = nullptr;         // previous state (initial-guess extrapolation)
  double* Res = nullptr;           // FP64 residual [n_rows][Jp]
  void* basis = nullptr;           // (m+1) blocks [n_rows][Jp] in the Krylov precision
  void* Wk = nullptr;              // work blocks of the Krylov precision
  void* Zk = nullptr;
  void* Uk = nullptr;
  void* Tk = nullptr;              // preconditioner temps [n_rows][Jp]
  void* Pk = nullptr;
  void* Rk = nullptr;              // scaled residual of the correction equation
  void* Dk = nullptr;              // correction
  double* dscale = nullptr;        // [2 Jp]: 1/||res_j||, ||res_j||
  int* d_err = nullptr;            // bounded-wait failure word of this subproblem's staged kernels
  void* hcoef = nullptr;           // pinned host staging of coefficients [(m+1) J J] doubles
  double* part = nullptr;          // gram partial sums [nchunk][m+1][MAX_J*MAX_J]
  double* gram = nullptr;          // reduced gram [m+1][J][J]
  void* coef = nullptr;            // coefficients for block combines [m+1][J][J] (Krylov precision)
  double* colsq = nullptr;         // per-chunk column sums of squares [nchunk][Jp]
  double* hbuf = nullptr;          // pinned host mirror of gram [m+1][J][J]
  double* hcol = nullptr;          // pinned host column norms [nchunk][Jp]
  std::vector<DevAmgLevel> amg;    // per-subproblem AMG work vectors (shared operators)
  double* Np = nullptr;            // pressure convection matrix values (P1 pattern) [nnzKp]
  float* Npf = nullptr;
  void* ibasis = nullptr;          // inner GMRES basis (kin+1) x [n2][2 Jp] (Krylov precision)
  double* ipart = nullptr;         // inner dot partial sums [nchunk][kin+2][2 Jp]
  double* idot = nullptr;          // reduced inner dots [kin+2][2 Jp]
  double* ih = nullptr;            // inner Hessenberg [kin+1][kin][2 Jp]
  double* ibeta = nullptr;         // [2 Jp] initial norms, then [2 Jp] inverse norms
  double* iy = nullptr;            // inner least-squares solutions [kin][2 Jp]
  unsigned* ibar = nullptr;        // grid-barrier counters of the persistent inner GMRES [2]
  void* zbasis = nullptr;          // flexible GMRES: preconditioned basis m x [n_rows][Jp]
  // captured preconditioner graphs keyed by (input, output) device pointers
  std::map<std::tuple<const void*, const void*, int>, std::pair<cudaGraphExec_t, long long>> prec_graphs;
  // stats
  int iters = 0, refine = 0;
  int graphs_built = 0;
  bool graphs_off = false;         // a capture failed: the preconditioner runs uncaptured from then on
  double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // MHDE_TRACE: assemble, residual, precond, spmm, cgs, normalise
  double relres = 0.0;
  int status = 0;
  std::string err;
};

}  // namespace mhde

struct mhde_ctx {
  mhde::FeHost fe;
  mhde_options opt{};
  int J = 0, Jp = 0;
  int n_rows = 0;
  double s = 0.0, rs = 0.0, dt = 0.0;
  std::vector<double> nu, nu_m;
  double nubar = 0.0, nubar_m = 0.0;
  std::vector<double> c_cross, c_same;   // (nu_j - nu_m,j), (nu'_j + nu'_m,j)
  std::string err;
  bool bound = false, have_initial = false;
  bool have_prev = false;              // Sprev holds the state of the previous step
  long long steps = 0;
  mhde_stats stats{};
  int nchunk = 0;
  int nchunk_in = 0;                   // row chunks of the inner (velocity-block) dot products
  int amg_levels = 0;

  // device workspace
  char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t sv = nullptr, sw = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // constant device tables
  int* d_dofs = nullptr;
  double* d_geom = nullptr;
  unsigned char* d_isbnd = nullptr;
  int* d_bnd = nullptr;                // [n2] boundary index of a node, -1 inside
  mhde::DevCsr F;                      // pattern (rowptr, col) shared by both F's
  int* d_fslot_ptr = nullptr;
  int* d_fslot = nullptr;
  int* d_fdiag = nullptr;
  double* d_M = nullptr;               // [nnzF]
  double* d_K = nullptr;
  mhde::DevCsr B;                      // np x n2, values as pairs (x, y): val has 2*nnzB
  int* d_bslot_ptr = nullptr;
  int* d_bslot = nullptr;
  mhde::DevCsr BT;                     // n2 x np, values as pairs
  int* d_btsrc = nullptr;
  int* d_p1slot_ptr = nullptr;
  int* d_p1slot = nullptr;
  int* d_node_ptr = nullptr;
  int* d_node_slot = nullptr;
  double* d_lsc_dinv = nullptr;        // [n2] 1/D of the least-squares commutator (0 on Dirichlet nodes)
  float* d_lsc_dinvf = nullptr;
  double* d_mp = nullptr;              // lumped pressure mass [np]
  float* d_mpf = nullptr;
  double* d_Mloc = nullptr;            // scratch for the constant assembly [nt][36]
  double* d_Kloc = nullptr;
  double* d_Bloc = nullptr;            // [nt][18][2]
  std::vector<mhde::DevAmgLevel> amg_ops;  // shared level operators
  double* d_coarse_inv = nullptr;
  float* d_coarse_invf = nullptr;

  // state and inputs
  double* d_F1 = nullptr;              // Elsaesser forcing [n2][2][Jp]
  double* d_F2 = nullptr;
  bool have_forcing = false;
  double* d_Gv = nullptr;              // Dirichlet values [nbnd][2][Jp]
  double* d_Gw = nullptr;
  double* d_mean_v = nullptr;          // [n2][2]
  double* d_mean_w = nullptr;
  double* d_l2_v = nullptr;            // [nt][7]
  double* d_l2_w = nullptr;
  double* d_ccross = nullptr;          // [Jp] nu_j - nu_m,j
  double* d_csame = nullptr;           // [Jp] nu'_j + nu'_m,j
  int device = 0;
  bool trace = false;                  // MHDE_TRACE=1: per-sweep residuals on stderr
  bool use_graphs = true;              // MHDE_GRAPHS=0 disables graph capture
  bool serial = false;                 // MHDE_SERIAL=1: solve the two subproblems one after the other
  bool spmm_rows = false;              // MHDE_SPMM=rows: row-per-thread saddle SpMM variant
  int spmm_block = 256;                // CTA size of the chunked saddle SpMM (autotuned at bind)
  bool spmm_forced = false;            // MHDE_SPMM set: skip the autotuner
  double spmm_tuned_us[3] = {0, 0, 0}; // autotuner timings for CTA sizes 128, 256, 512
  // FP32 block Gram and combination: tensor-core (tcgen05) or CUDA-core
  // kernels, picked at bind by timing both on this context's sizes
  bool gram_tc = false, comb_tc = false;
  double gram_tuned_us[2] = {0, 0};    // CUDA cores, tensor cores
  double comb_tuned_us[2] = {0, 0};
  // mixed-path inner GMRES: persistent cooperative kernel (ig_P CTAs, row
  // ranges d_ig_rows; 0 CTAs where it does not apply) or the launch chain,
  // picked at bind by timing both
  bool inner_grid = false;
  int ig_P = 0;
  int* d_ig_rows = nullptr;            // [IG_PMAX + 1]
  double inner_tuned_us[2] = {0, 0};   // launch chain, persistent
  mhde::Sub sub[2];
  std::vector<int> h_bidx;             // boundary index of every P2 node (host copy)
  std::vector<double> h_M;             // mass matrix values (host copy, for the energy)
};
