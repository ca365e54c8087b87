// Launch wrappers of the libmhde device kernels.  All multi-vectors are
// row-major [rows][Jp] with J real columns (the rest zero).  Velocity rows
// are ordered node-major: row 2a + c is component c of P2 node a; pressure
// row i of a saddle multi-vector is row 2 n2 + i.
#pragma once

#include <cuda_runtime.h>

#include "mhde_internal.h"

namespace mhde {

// Kernel launches issued by this library (all contexts), for the
// benchmark's launch count.
long long launch_count();
void count_launch(long long n = 1);
void set_capturing(bool on);   // launches issued while capturing a graph are not counted

// Programmatic dependent launch.  The solver's kernels form long chains of
// small dependent launches on one stream; a kernel launched through
// launch_pdl may be scheduled while its predecessor drains, and overlaps its
// launch and CTA start-up with that tail.  Every kernel launched this way
// executes pdl_wait() before its first global memory access: it blocks until
// the preceding grid has completed and its writes are visible (without the
// launch attribute it returns at once), so results do not depend on the
// overlap.  pdl_trigger() lets the next launch be scheduled once every CTA of
// this grid has started.  MHDE_PDL=0 turns the attribute off.
bool pdl_enabled();
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

struct QuadTables {             // degree-5 rule and P2 basis tables (host copy)
  double lam[NQ][3];
  double w[NQ];                 // reference weights, sum 1/2
  double phi[NQ][NLOC];
  double dphi[NQ][NLOC][3];     // d phi_a / d lambda_k
};
void quad_tables(QuadTables& q);
cudaError_t upload_quad_tables();
cudaError_t upload_adjoint_tables();

// ---- finite element kernels (FP64) ----------------------------------------
void launch_const_local(int nt, const double* geom, double* Mloc, double* Kloc, double* Bloc,
                        cudaStream_t st);
void launch_gather_const(const mhde_ctx* c, cudaStream_t st);
void launch_means(int n2, int J, int Jp, const double* Sv, const double* Sw, double* mv, double* mw,
                  cudaStream_t st);
void launch_l2(int nt, int J, int Jp, const int* dofs, const double* Sv, const double* Sw,
               const double* mv, const double* mw, double* l2v, double* l2w, cudaStream_t st);
void launch_F_local(int nt, const int* dofs, const double* geom, const double* mean_conv,
                    const double* l2, double coef_eddy, int conv_form, double* Floc,
                    cudaStream_t st);
void launch_F_gather(const mhde_ctx* c, const double* Floc, double inv_dt, double nu_hat,
                     double* Fval, float* Fvalf, double* Fdinv, float* Fdinvf, cudaStream_t st);
void launch_rhs_conv_local(int nt, int J, int Jp, const int* dofs, const double* geom,
                           const double* S_self, const double* S_other, const double* mean_other,
                           int conv_form, double* Cloc, cudaStream_t st);
void launch_rhs_assemble(const mhde_ctx* c, const double* S_self, const double* S_other,
                         const double* Fz, const double* G, const double* Cloc,
                         const double* c_cross, const double* c_same, double* Bv, cudaStream_t st);

// ---- linear algebra kernels (T = double or float) -------------------------
// Y = A X (mode 0) or Y = Bvec - A X (mode 1) for the saddle matrix.
// (ld = row stride of X, Y and Bvec, a multiple of 4)
template <typename T>
void launch_saddle_spmm(const mhde_ctx* c, const T* Fval, const T* Bval, const T* BTval, const T* X,
                        const double* Bvec, T* Y, int mode, int ld, cudaStream_t st);
// generic CSR: mode 0 y = A x; 1 y = b - A x; 2 y = x + omega dinv (b - A x);
// 3 y = omega dinv b; 4 y += A x; 5 y = b + A x
template <typename T>
void launch_csr(int nrows, const int* rowptr, const int* col, const T* val, const T* dinv, T omega,
                const T* x, const T* b, T* y, int mode, int Jp, cudaStream_t st);
template <typename T>
void launch_dense_apply(int n, const T* Ainv, const T* x, T* y, int Jp, cudaStream_t st);
// velocity rows: z = dinv r (first) or z_out = z_in + omega dinv (r - F z_in); identity rows copy r
template <typename T>
void launch_jacobi_F(const mhde_ctx* c, const T* Fval, const T* Fdinv, T omega, const T* r,
                     const T* zin, T* zout, int ld, cudaStream_t st);
// pressure part of the block preconditioner:
//   zp = -(1/dt) x - nu_hat rp / mp, zp[0] = rp[0]
//   (PCD adds - (N_p x) / mp when Np is not null; N_p has the P1 pattern rp/col)
template <typename T>
void launch_precond_p(int np, int Jp, const T* x, const T* rp, const T* mp, T inv_dt, T nu_hat,
                      const int* nrp, const int* ncol, const T* Np, T* zp, cudaStream_t st);
// tu = ru - B^T zp (velocity rows; Dirichlet rows keep ru)
template <typename T>
void launch_bt_apply(const mhde_ctx* c, const T* BTval, const T* ru, const T* zp, T* tu, int ld,
                     cudaStream_t st);
// block-Jacobi sweep x_out = x_in + omega Binv r over nb blocks of bs dofs
// (idx [nb][bs], inv [nb][bs][bs]); x_in null means zero; x_out may be x_in
template <typename T>
void launch_block_jacobi(int nb, int bs, const int* idx, const T* inv, T omega, const T* x_in, const T* r,
                         T* x_out, int Jp, cudaStream_t st);
// least-squares commutator middle product z = B D^{-1} F D^{-1} B^T y:
// t = D^{-1} B^T y and s = D^{-1} F t (velocity rows, D^{-1} = dinv, zero on
// Dirichlet rows), z = B s (pressure rows); y's dof 0 is taken as zero and
// z_0 = 0 (the pinned dof)
template <typename T>
void launch_lsc_middle(const mhde_ctx* c, const T* Fval, const T* BTval, const T* Bval, const T* dinv,
                       const T* y, T* t, T* s, T* z, int ld, cudaStream_t st);
// Gram partial sums: part[chunk][i][p][q] = sum_rows V_i[row][p] W[row][q].
// err: the calling subproblem's device error word; with it the FP32 Gram may
// take the TMA-staged kernel, which sets *err = 1 when a stage never lands
// (nullptr: the unstaged kernels only)
// allow_tc: the FP32 Gram may run on the tensor cores (tcgen05, split TF32)
template <typename T>
void launch_gram(const T* V, size_t vstride, int kblocks, const T* W, int n_rows, int Jp, int r,
                 int nchunk, double* part, double* gram, cudaStream_t st, bool reduce = true,
                 int* err = nullptr, bool allow_tc = false);
// partial sums of the FP32 block Gram on the tensor cores (kernels_tc.cu):
// one partial per CTA (at most max_parts) in part[nparts][kblocks][r][r].
// false (nothing launched) when the sizes or the device do not fit the
// kernel; err as for launch_gram (required)
struct TcGramPlan {
  int nch = 0, N = 0, mtiles = 0, TR = 0, kgroup = 0, ngroups = 0, nst = 0, nl = 0, per_sm = 1;
  unsigned ncols = 0, stage_bytes = 0, off_lay = 0, lay_bytes = 0;
  size_t smem = 0;
};
bool gram_tc_plan(int kblocks, int ld, int r, TcGramPlan& plan);
bool tc_gram_available();
bool launch_gram_tc(const float* V, size_t vstride, int kblocks, const float* W, int n_rows, int ld, int r,
                    int max_parts, double* part, cudaStream_t st, int* err, int& nparts);
void launch_gram_reduce(int nparts, int total, const double* part, double* gram, cudaStream_t st);
// block combination of launch_block_combine on the tensor cores (kernels_tc.cu,
// FP32 only): false (nothing launched) when the sizes, alignment or device do
// not fit
struct TcCombinePlan {
  int N = 0, KC = 0, MT = 0, rows_per_cta = 0, nctas = 0, nst = 0, nl = 0;
  unsigned ncols = 0, stage_bytes = 0, a_bytes = 0, b_bytes = 0, off_a = 0, off_b = 0;
  size_t smem = 0;
};
bool combine_tc_plan(int n_rows, int ldv, int r_in, int r_out, int nsm, TcCombinePlan& plan);
bool launch_combine_tc(float* out, const float* in, float alpha, const float* V, size_t vstride, int kblocks,
                       int r_in, const float* C, int r_out, int n_rows, int ldv, int ldo, cudaStream_t st, int* err);
// G = [H_0 .. H_k, W^T W] (r x r blocks) -> block k+2 := W^T W - sum_i H_i^T H_i
void launch_proj_gram(double* G, int k, int r, cudaStream_t st);
// 1 if a staged Gram or combine launch of the subproblem owning d_err gave
// up waiting for a TMA stage since the last call (the word is then cleared
// on st), 0 if not, -1 on a CUDA error
int take_async_error(int* d_err, cudaStream_t st);
// C_i = -H_i T (i <= k), C_{k+1} = T, converted to the Krylov precision
template <typename T>
void launch_make_coef(const double* G, const double* Tm, int k, int r, T* C, cudaStream_t st);
// out[row][q] = alpha in[row][q] + sum_i sum_p V_i[row][p] C_i[p][q], q < r_out; 0 beyond
// (V rows have stride ldv, in/out rows stride Jp); err as for launch_gram;
// allow_tc: the FP32 combination may run on the tensor cores
template <typename T>
void launch_block_combine(T* out, const T* in, T alpha, const T* V, size_t vstride, int kblocks,
                          int r_in, const T* C, int r_out, int n_rows, int ldv, int Jp, cudaStream_t st,
                          int* err = nullptr, bool allow_tc = false);
// out[row][q] = (T) sum_p X[row][p] C[p][q], q < r (0 beyond); X, C (J x r) in FP64;
// X rows have stride Jp, out rows stride ldo
template <typename T>
void launch_combine_from_f64(T* out, const double* X, const double* C, int J, int r, int n_rows, int Jp,
                             int ldo, cudaStream_t st);
// per-chunk column sums of squares (FP64)
template <typename T>
void launch_colsq(const T* X, int n_rows, int Jp, int nchunk, double* out, cudaStream_t st);
// y[:, j] = (T)(x[:, j] * scale[j])   (FP64 -> T with per-column scaling)
template <typename T>
void launch_scale_to(const double* x, const double* scale, T* y, size_t n, int Jp, cudaStream_t st);
// x[:, j] += (double) d[:, j] * scale[j]
template <typename T>
void launch_axpy_from(const T* d, const double* scale, double* x, size_t n, int Jp, cudaStream_t st);
// out = a x + b y (elementwise, n entries)
template <typename T>
void launch_axpby(T* out, T a, const T* x, T b, const T* y, size_t n, cudaStream_t st);
void launch_d2f(const double* x, float* y, size_t n, cudaStream_t st);

// pressure convection matrix N_p(a) of the PCD Schur approximation (P1,
// standard form (a . grad psi_k, psi_i), a = mean convecting field)
void launch_Np(const mhde_ctx* c, const double* mean_conv, double* slots, double* Np, float* Npf,
               cudaStream_t st);
// inner per-column GMRES(k) on F (velocity block), z ~ F^{-1} r; with
// allow_half and options.inner_fp16 the FP32 path keeps its basis in FP16
template <typename T>
void launch_inner_gmres(const mhde_ctx* c, const Sub& s, const T* FDv, const T* dinv, const T* r, T* z, int ld,
                        int kin, cudaStream_t st, bool allow_half = true);
// the persistent form (kernels_inner_grid.cu) on the FP32 path: grid size
// and row ranges for a context (0: not applicable), and the launch (false:
// not launched, use the chain)
int inner_grid_plan(const mhde_ctx* c, std::vector<int>& row_start);
bool launch_inner_grid(const mhde_ctx* c, const Sub& s, const float* FDv, const float* dinv, const float* r,
                       float* z, int ld, int kin, cudaStream_t st);
// shared-memory limits of the inner and block kernels (set once, before any capture)
cudaError_t init_inner_attributes();
cudaError_t init_inner_grid_attributes();
cudaError_t init_la_attributes();
// solver entry points (solver.cu)
int assemble_sub(mhde_ctx* c, int which);
// zero_guess: start from X = 0 (transposed adjoint solves) instead of the
// extrapolation of the last two states
int solve_sub(mhde_ctx* c, int which, bool zero_guess = false);

// discrete adjoint (kernels_adj.cu)
void launch_fd_values(const mhde_ctx* c, Sub& s, cudaStream_t st);
void launch_transpose_values(long long nnz, const int* tpos, const double* F, double* FT, float* FTf,
                             cudaStream_t st);
void launch_scale_pair(long long n, double s, double* x, float* xf, cudaStream_t st);
void launch_energy_seed(const mhde_ctx* c, const double* mean, double* seed, cudaStream_t st);
void launch_adj_rhs(const mhde_ctx* c, const double* seed, double* B, cudaStream_t st);
void launch_adj_contract(const mhde_ctx* c, const double* Z, const double* Y, const double* meanY,
                         const double* X, const double* Yh, double* slotZ, double* slotY, double* slotM,
                         int* kstar, double* kap, double* lamZ, double* lamY, double* tmp, double* prod,
                         int nchunk, double* part, cudaStream_t st);
// benchmark helpers in the context's Krylov precision
void precond_apply_any(mhde_ctx* c, int which, const void* in, void* out);
void gram_any(mhde_ctx* c, int which, const void* V, size_t vstride, int k, const void* W, bool reduce = true);
void combine_any(mhde_ctx* c, int which, const void* V, size_t vstride, int k, void* out);

}  // namespace mhde
