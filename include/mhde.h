/*
 * mhde.h — C ABI of libmhde: one time step of the decoupled ensemble scheme
 * for J parameterized MHD flows in Elsaesser variables (Algorithm 1, eq.
 * weaknew1 and weaknew2), run on one GPU.
 *
 * Problem statement (Section 1, eq. gov1-gov5): J members share a mesh and
 * differ in viscosity nu_j, magnetic diffusivity nu_m,j, body force f_j,
 * curl g_j, initial data u_j^0, B_j^0 and Dirichlet data.  The library works
 * in the Elsaesser variables v = u + sqrt(s) B, w = u - sqrt(s) B with
 * f1 = f + sqrt(s) curl g and f2 = f - sqrt(s) curl g (Section 1) and converts
 * at the boundary of every call.
 *
 * Discretisation: P2 velocity on the given triangulation with either a
 * continuous P1 pressure (Taylor-Hood; Section 2, eq. infsup: any inf-sup
 * stable pair) or a discontinuous P1 pressure (Scott-Vogelius P2/P1disc, the
 * paper's element: Section 2 and Section 4, stable on barycenter-refined
 * meshes, velocities divergence-free at every point); options.element picks
 * one.  A 7-point degree-5 quadrature, Dirichlet data by identity rows,
 * pressure dof 0 pinned and pressures reported with mean zero (Q = L^2_0,
 * Section 2).
 *
 * Numbering: P2 node k < nv is mesh vertex k; node nv + e is the midpoint of
 * edge e, the edges being the distinct unordered vertex pairs sorted
 * lexicographically by (smaller vertex, larger vertex).  Continuous P1
 * pressure node i = vertex i; discontinuous P1 pressure dof 3t + i = the
 * barycentric coordinate of local vertex i of triangle t.
 * Nodal arrays are row-major: [J][n2][2] for member vector fields,
 * [n2][2] for one field, [J][np] for member pressures.
 *
 * Ownership: every host array is owned by the caller; the library copies
 * in or out during the call and keeps no pointer.  Device memory is one
 * workspace the caller allocates (e.g. a torch uint8 tensor) of the size
 * mhde_workspace_size() reports and hands over with mhde_bind(); after bind
 * the library allocates no device memory.  The two CUDA streams passed to
 * mhde_bind carry the v and w subproblems; the library synchronizes them
 * before every call returns.
 *
 * Errors: every int-returning call returns MHDE_OK (0) or a negative code;
 * mhde_last_error() describes the last failure on a context.
 */
#ifndef MHDE_H
#define MHDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MHDE_OK 0
#define MHDE_EINVAL -1      /* bad argument: J < 1, dt <= 0, s < 0, bad mesh, NULL ... */
#define MHDE_ESTAB -2       /* alpha_j <= 0 or mu <= 1/2 with options.strict = 1 (Section 3.1) */
#define MHDE_ENOCONV -3     /* solver hit its iteration cap; state left unchanged */
#define MHDE_ENAN -4        /* non-finite residual; state left unchanged */
#define MHDE_ECUDA -5       /* a CUDA call failed */
#define MHDE_EWORKSPACE -6  /* workspace missing, too small or misaligned */
#define MHDE_ESTATE -7      /* call out of order (e.g. step before bind / initial data) */

/* Precision of the Krylov iterations (Section 1 block solve; the FP64
 * refinement reading is the library's). */
#define MHDE_PREC_FP64 0    /* block GMRES, SpMM and preconditioner in FP64 */
#define MHDE_PREC_MIXED 1   /* FP32 block GMRES/SpMM/preconditioner, FP64 refinement */

typedef struct mhde_ctx mhde_ctx;   /* opaque, owned by the library */

/* Triangulation: nv vertices, nt counter-clockwise triangles, 0-based. */
typedef struct {
  int nv, nt;
  const double* xy;   /* [nv][2] */
  const int* tri;     /* [nt][3] */
} mhde_mesh;

typedef struct {
  double mu;            /* mixing-length tuning parameter (Section 1, nu_T = mu dt l^2); default 1 */
  int conv_form;        /* 0: skew-symmetric b (default), 1: standard b(u,v,w) = (u.grad v, w) */
  int precision;        /* MHDE_PREC_FP64 or MHDE_PREC_MIXED (default) */
  double rtol;          /* target FP64 relative residual ||b_j - A x_j|| / ||b_j|| per member;
                           default 0 = by precision: 1e-13 on the FP64 path, 1e-12 on the mixed
                           path (per-step residuals accumulate over a run; these keep the FP64
                           and mixed solutions within 1e-10 and 1e-8 of the oracle over 100
                           steps of the 32x32 cavity ensemble) */
  double inner_rtol;    /* mixed: FP32 inner relative tolerance per refinement sweep; default 1e-3
                           (shorter Krylov cycles, cheaper block Gram-Schmidt per iteration: on the
                           128x128 cavity ensemble 100.2 against 110.8 ms/step for 1e-5 at the same
                           block-iteration count; the FP64 rtol alone decides the accuracy) */
  int restart;          /* block GMRES restart length m (blocks); default 30 */
  int max_iter;         /* cap on block GMRES iterations per subproblem solve; default 2000 */
  int max_refine;       /* cap on FP64 refinement sweeps (one block GMRES cycle each); default 60 */
  int jacobi_sweeps;    /* damped Jacobi sweeps approximating F^{-1}; default 3 */
  double jacobi_omega;  /* damping of those sweeps; default 0.3 */
  int amg_sweeps;       /* Jacobi sweeps per level in the pressure-Laplacian V-cycle; default 1 */
  int amg_cycles;       /* V-cycles per application of the pressure-Laplacian inverse; default 1 */
  int inner_iters;      /* k of the inner per-column GMRES(k) on F (flexible outer GMRES);
                           0 = damped Jacobi sweeps instead; default 6
                           (on the 128x128 cavity ensemble 6 inner steps and one smoothing
                           sweep per AMG level cost more outer iterations than 8 and 2 but
                           less time per step) */
  int schur;            /* pressure Schur approximation: 0 Cahouet-Chabard, 1 pressure
                           convection-diffusion (adds the mean-field P1 convection; continuous
                           pressure only), 2 least-squares commutator
                           (L^{-1} B D^{-1} F D^{-1} B^T L^{-1} with L = B D^{-1} B^T, D the
                           diagonal of the P2 mass on interior nodes); default 1.  With the
                           discontinuous pressure the Laplacian is always B D^{-1} B^T (0 or 2;
                           1 is rejected with MHDE_EINVAL) */
  int strict;           /* 1: reject alpha_j <= 0 or mu <= 1/2 with MHDE_ESTAB; default 0 */
  int inner_fp16;       /* 1: the mixed path keeps the inner GMRES basis in FP16 (scaled by
                           sqrt(n2); arithmetic stays FP32), halving the basis traffic of the
                           inner solve; ignored on the FP64 path; default 0 (on the 128x128
                           cavity ensemble the inner solve is bound by its chain of dependent
                           launches, not by traffic: 283 vs 286 us per application) */
  int element;          /* 0 Taylor-Hood P2/P1 (default); 1 Scott-Vogelius P2/P1disc (give a
                           barycenter-refined mesh; on other meshes the pair need not be
                           inf-sup stable and the solve may fail).  Element 1 needs schur 0 or
                           2; schur 0 with amg_sweeps 2 was the fastest measured (64x64
                           refined cavity, J = 20: 240 ms per step against 275 ms with one
                           sweep and 400 ms for schur 2) and is what the Python binding sets
                           for this element unless told otherwise */
} mhde_options;

typedef struct {
  int nv, nt, ne, n2, np;   /* vertices, triangles, edges, P2 nodes, pressure dofs (nv for
                               Taylor-Hood, 3 nt for Scott-Vogelius) */
  int n_rows;               /* rows of one saddle system: 2 n2 + np */
  int J, J_pad;             /* members, padded row width of the device multi-vectors */
  long long nnz_F;          /* nonzeros of the scalar P2 block F */
  long long nnz_B;          /* nonzeros of the divergence block (per component) */
  long long nnz_saddle;     /* nonzeros of the full saddle matrix (2 nnz_F + 4 nnz_B + 1) */
  int n_boundary;           /* Dirichlet P2 nodes */
  int amg_levels;           /* levels of the pressure-Laplacian hierarchy */
  long long nnz_L;          /* nonzeros of its finest operator (P1 stiffness or B D^{-1} B^T) */
  int smoother_block;       /* smoother of that finest level: 0 point Jacobi, 3 block Jacobi
                               over the dofs of each triangle, 9 over each macro triangle of a
                               barycenter refinement (discontinuous pressure) */
} mhde_sizes;

typedef struct {
  long long steps;            /* steps taken */
  int last_iters[2];          /* block GMRES iterations of the last step (v, w) */
  int last_refine[2];         /* refinement sweeps of the last step (v, w); 1 on the FP64 path */
  double last_relres[2];      /* max_j FP64 relative residual after the last step (v, w) */
  long long total_iters;      /* sum of block GMRES iterations over all steps and both subproblems */
  double last_step_ms;        /* wall time of the last mhde_step (host clock) */
  long long launches;         /* kernel launches issued by all steps so far */
  int spmm_block;             /* CTA size the bind-time autotuner chose for the
                                 saddle SpMM (128, 256 or 512; results do not
                                 depend on it) */
  double spmm_tuned_us[3];    /* its timings of one SpMM at 128, 256, 512 */
  int gram_tensor_cores;      /* 1 if the FP32 block Gram of the mixed path runs on the tensor
                                 cores (tcgen05, split TF32: about 2^-21 relative against FP32's
                                 2^-24), 0 on the CUDA cores; tensor cores for J > 32, so that
                                 the choice never depends on a timing */
  int combine_tensor_cores;   /* the same for the FP32 block combination */
  double gram_tuned_us[2];    /* its timings of one Gram of restart/2 + 1 blocks: CUDA cores,
                                 tensor cores (0 where not timed) */
  double combine_tuned_us[2]; /* the same for one combination of restart/2 blocks */
  int inner_persistent;       /* 1 if the mixed path's inner GMRES on F runs as the persistent
                                 form (one cooperative launch, grid barriers; chosen only through
                                 the environment, MHDE_INNER_GRID=1), 0 the chain of per-phase
                                 launches (the default) */
  double inner_tuned_us[2];   /* its timings of one inner solve: launch chain, persistent
                                 (0 where not timed) */
} mhde_stats;

/* Default options (listed above). */
void mhde_default_options(mhde_options* opt);

/* Build the discrete problem for a mesh and J members (host only, no GPU
 * work).  nu, nu_m: [J].  Checks J >= 1, dt > 0, s >= 0, a valid CCW mesh.
 * alpha_j = nubar + nubar_m - |nu_j - nu_m,j| - |nu'_j + nu'_m,j| > 0 and
 * mu > 1/2 are the stability conditions of Section 3.1; they are errors
 * (MHDE_ESTAB) only with opt->strict = 1.  opt may be NULL (defaults). */
int mhde_create(const mhde_mesh* mesh, int J, const double* nu, const double* nu_m, double s,
                double dt, const mhde_options* opt, mhde_ctx** out);

int mhde_get_sizes(const mhde_ctx* ctx, mhde_sizes* sizes);

/* Bytes of device workspace mhde_bind needs (256-byte aligned base). */
int mhde_workspace_size(const mhde_ctx* ctx, size_t* bytes);

/* Hand over the caller-allocated device workspace and the two streams
 * (cudaStream_t as void*, may be NULL for the legacy default stream).
 * Uploads the mesh tables and assembles the constant matrices M, K, B and the
 * pressure-Laplacian hierarchy.  The workspace must stay allocated until
 * mhde_destroy. */
int mhde_bind(mhde_ctx* ctx, void* dev_workspace, size_t bytes, void* stream_v, void* stream_w);

/* P2 node coordinates [n2][2] and Dirichlet flags [n2] (1 = boundary node);
 * either pointer may be NULL. */
int mhde_p2_nodes(const mhde_ctx* ctx, double* xy, unsigned char* is_boundary);

/* Initial data u_j^0, B_j^0 as P2 nodal values [J][n2][2] (host).  Resets the
 * step counter and the pressures to 0. */
int mhde_set_initial(mhde_ctx* ctx, const double* u0, const double* B0);

/* Replace the member viscosities nu_j, nu_m,j ([J] each, > 0; host) of a
 * context, with the derived means and splits (Section 1: nubar, nu'_j).  The
 * stability condition of Section 3.1 is checked as in mhde_create.  The
 * state is kept.  Errors: MHDE_EINVAL, MHDE_ESTAB (strict only). */
int mhde_set_viscosity(mhde_ctx* ctx, const double* nu, const double* nu_m);

/* Body force f_j and curl g_j at t^{n+1} as P2 nodal values [J][n2][2]
 * (host); the discrete forcing is M times the nodal interpolant.  NULL means
 * zero.  Values persist for later steps until set again. */
int mhde_set_forcing(mhde_ctx* ctx, const double* f, const double* curl_g);

/* Dirichlet data u_j, B_j at t^{n+1} as P2 nodal values [J][n2][2] (host);
 * only boundary nodes are read.  NULL means zero.  Values persist. */
int mhde_set_dirichlet(mhde_ctx* ctx, const double* u_bc, const double* B_bc);

/* One step n -> n+1 of Algorithm 1 for all members: ensemble means and
 * mixing-length field, the two shared matrices, the batched right-hand
 * sides, and the two block solves on the two streams.  On MHDE_ENOCONV or
 * MHDE_ENAN the state is left at step n. */
int mhde_step(mhde_ctx* ctx);

/* nsteps calls of mhde_step with the forcing and Dirichlet data held fixed. */
int mhde_advance(mhde_ctx* ctx, int nsteps);

/* Batched uneven ensembles: advance `count` independent, bound contexts
 * (any meshes and member counts) by nsteps steps each, from a pool of
 * nthreads host threads; every ensemble keeps its own two streams, so the
 * ensembles' kernels run concurrently on the device.  step_ms (optional,
 * [count][nsteps]) receives each step's wall time for latency statistics.
 * Returns the first failing context's error code. */
int mhde_advance_many(mhde_ctx** ctxs, int count, int nsteps, int nthreads, double* step_ms);

/* Ensemble means <u> = (<v>+<w>)/2 and <B> = (<v>-<w>)/(2 sqrt s) at the
 * current step as [n2][2] (host).  B_mean may be NULL; with s = 0 a non-NULL
 * B_mean is MHDE_EINVAL (B is not recoverable). */
int mhde_read_mean(mhde_ctx* ctx, double* u_mean, double* B_mean);

/* Elsaesser state: v, w [J][n2][2] and pressures q, r [J][np] (mean zero);
 * any pointer may be NULL. */
int mhde_read_state(mhde_ctx* ctx, double* v, double* w, double* q, double* r);

/* Primitive fields of member j: u, B [n2][2]; p = (q+r)/2 and
 * lambda = (q-r)/(2 sqrt s) [np]; any pointer may be NULL (B, lambda must be
 * NULL when s = 0). */
int mhde_read_member(mhde_ctx* ctx, int j, double* u, double* B, double* p, double* lambda);

/* E_h^n = 1/2 (||<v_h>^n||^2 + ||<w_h>^n||^2) (Section 4.2). */
int mhde_energy(mhde_ctx* ctx, double* E);

int mhde_get_stats(const mhde_ctx* ctx, mhde_stats* stats);

/* Copy of the full time-stepping state (step counter, the Elsaesser fields
 * with pressures of the current and of the previous step; the previous one
 * seeds the solver's initial guess) to / from a caller buffer of
 * mhde_state_bytes() bytes (host).  Loading reproduces an uninterrupted run
 * bit for bit. */
int mhde_state_bytes(const mhde_ctx* ctx, size_t* bytes);
int mhde_save_state(mhde_ctx* ctx, void* host_buffer);
int mhde_load_state(mhde_ctx* ctx, const void* host_buffer);

/* ------------------------------------------------------------------------
 * Discrete adjoint (gradient of the ensemble-mean energy).
 *
 * L = E_h^K = 1/2 (||<v_h>^K||^2 + ||<w_h>^K||^2) (Section 4.2) after K =
 * nsteps steps of Algorithm 1 from the context's current state, with the
 * forcing and Dirichlet data currently set held fixed over the K steps.
 * mhde_energy_adjoint runs the K steps (the context ends at step +K, as after
 * mhde_advance), returns L, and by the discrete adjoint of the step its
 * gradient with respect to nu_j and nu_m,j ([J] each, host, may be NULL) and
 * to the starting fields u_j, B_j as P2 nodal values ([J][n2][2] each, host,
 * may be NULL; at the start v = u + sqrt(s) B, w = u - sqrt(s) B).  The
 * reverse sweep keeps a checkpoint of the state every checkpoint_every steps
 * and recomputes each segment from it.  Each reverse step solves the
 * transposed shared matrix of both subproblems for all members with the
 * block solver of the forward step (same precision and tolerance).  The
 * gradient of the max in the mixing length l^2 = max_j |z'_j|^2 is taken at
 * the member attaining it.
 * Workspace: mhde_adjoint_workspace_size() bytes of device memory from the
 * caller (any alignment; the library aligns it), used only during the call.
 * Errors: MHDE_EINVAL, MHDE_ESTATE (not bound / no initial state),
 * MHDE_EWORKSPACE, MHDE_ENOCONV (a forward or adjoint solve failed; the
 * context is then left mid-run), MHDE_ECUDA. */
int mhde_adjoint_workspace_size(const mhde_ctx* ctx, int nsteps, int checkpoint_every, size_t* bytes);
int mhde_energy_adjoint(mhde_ctx* ctx, int nsteps, int checkpoint_every, void* workspace, size_t workspace_bytes,
                        double* loss, double* grad_nu, double* grad_nu_m, double* grad_u0, double* grad_B0);

const char* mhde_last_error(const mhde_ctx* ctx);
void mhde_destroy(mhde_ctx* ctx);

/* ------------------------------------------------------------------------
 * Probes: intermediate results of the current step for parity tests.  They
 * run the named kernels on the current state without advancing it.
 * which = 0 for the v subproblem, 1 for the w subproblem.
 * ---------------------------------------------------------------------- */

/* Ensemble means (Section 1) [n2][2] and the mixing-length field
 * l^2 = max_j |z'_j|^2 at the quadrature points [nt][7] for z = v and w. */
int mhde_probe_mean_l2(mhde_ctx* ctx, double* mean_v, double* mean_w, double* l2_v, double* l2_w);

/* Shared matrix F of eq. weaknew1 (which = 0) or weaknew2 (which = 1) with
 * Dirichlet identity rows, in CSR: rowptr [n2+1], col [nnz_F], val [nnz_F]. */
int mhde_probe_matrix_F(mhde_ctx* ctx, int which, int* rowptr, int* col, double* val);

/* Finest operator L of the pressure-Laplacian hierarchy, host data (callable
 * before bind): the P1 stiffness of the continuous pressure, or
 * L = sum_d B_d D^{-1} B_d^T over the interior P2 nodes (D the P2 mass
 * diagonal scaled to the element areas) for the discontinuous pressure and
 * the least-squares commutator; dof 0 pinned (identity row and column).
 * CSR: rowptr [np+1], col [nnz_L], val [nnz_L]; any pointer may be NULL. */
int mhde_probe_laplacian(const mhde_ctx* ctx, int* rowptr, int* col, double* val);

/* Level `level` (0 = finest) of the pressure-Laplacian hierarchy, host data
 * (callable before bind).  counts[6] receives: rows n, nnz(A), nnz(P),
 * nnz(R), the smoother's block size bs (0: damped point Jacobi) and the
 * number of levels; scal[2] the Jacobi damping (0 on a level smoothed by
 * blocks, where it is not used) and the block damping.  Each
 * non-NULL array receives a copy: A in CSR (a_rowptr [n+1], a_col, a_val),
 * the prolongation from the next level P (n x n_next) and the restriction
 * R = P^T in CSR, the blocks (blk_idx [n], blk_inv [n/bs][bs][bs]).  The
 * coarsest level has no P, R or blocks (it is solved by a dense inverse).
 * MHDE_EINVAL for a NULL ctx or counts, or a level out of range. */
int mhde_probe_amg_level(const mhde_ctx* ctx, int level, long long* counts, double* scal, int* a_rowptr,
                         int* a_col, double* a_val, int* p_rowptr, int* p_col, double* p_val, int* r_rowptr,
                         int* r_col, double* r_val, int* blk_idx, double* blk_inv);

/* Right-hand sides of eq. weaknew1 / weaknew2 for all members:
 * velocity part [J][n2][2] (boundary rows hold the Dirichlet values). */
int mhde_probe_rhs(mhde_ctx* ctx, int which, double* rhs);

/* Y = A X for the saddle matrix of subproblem `which` at the current step,
 * X and Y host arrays in the oracle's block order [J][2 n2 + np]
 * (x-components, y-components, pressures).  precision: 0 FP64 kernel,
 * 1 FP32 kernel (inputs rounded to float). */
int mhde_probe_spmm(mhde_ctx* ctx, int which, int precision, const double* X, double* Y);

/* Z ~ F^{-1} R by the mixed path's inner solve of the velocity block (the
 * preconditioner's per-column GMRES(k) on F D^{-1}, k = options.inner_iters,
 * zero start, FP32; Section 1 block solvers) for subproblem `which` at the
 * current step.  R and Z: host [J][2][n2] (member, component, node), R
 * rounded to float.  form: 0 the chain of per-phase launches, 1 the
 * persistent cooperative kernel.  MHDE_EINVAL on the FP64 path, with
 * inner_iters = 0, or for form 1 where the persistent kernel is not
 * available on this device or size. */
int mhde_probe_inner(mhde_ctx* ctx, int which, int form, const double* R, double* Z);

/* Average device time in milliseconds of one launch of a hot-path kernel
 * group on the current state of subproblem `which`, from CUDA events on that
 * subproblem's stream around `reps` back-to-back launches (benchmark
 * support; the time-stepping state is not changed, scratch buffers are).
 * kernel: 0 saddle SpMM (FP64), 1 saddle SpMM (FP32), 2 shared-matrix
 * assembly (element kernel + nnz gather), 3 batched right-hand sides
 * (element kernel + node gather), 4 ensemble means + mixing-length field,
 * 5 block preconditioner (Krylov precision), 6 block Gram of restart/2
 * basis blocks against one block (Krylov precision), 7 block combination
 * sum_i V_i C_i of restart/2 basis blocks (Krylov precision), 8 the partial
 * sums of kernel 6 alone (its dominant launch, without the final reduction),
 * 9 the residual b - L x of the pressure Laplacian on the finest level of
 * the V-cycle (Krylov precision; nnz(L) = sizes.nnz_L). */
int mhde_time_kernel(mhde_ctx* ctx, int which, int kernel, int reps, double* ms);

/* ------------------------------------------------------------------------
 * Batched block Gram reduction of the block Krylov solve (Section 1: one
 * shared matrix, all J right-hand sides solved together with block linear
 * solvers).  Context-free, FP64, device pointers, asynchronous on `stream`
 * (cudaStream_t as void*, NULL = legacy default stream).
 * ---------------------------------------------------------------------- */

/* Scratch bytes mhde_block_gram needs for n_rows rows, r columns and
 * kblocks basis blocks. */
int mhde_block_gram_scratch_bytes(int n_rows, int r, int kblocks, size_t* bytes);

/* G[i][p][q] = sum_rows V_i[row][p] W[row][q] for i < kblocks, p, q < r.
 * V_i = V + i * v_stride (elements); V_i and W are row-major [n_rows][ld]
 * with ld a multiple of 4, r <= ld <= 64 (columns r..ld-1 are read but do
 * not enter G), 1 <= kblocks <= 65535.  G: device [kblocks][r][r].  scratch: device, at least
 * mhde_block_gram_scratch_bytes() bytes, owned by the caller; fully
 * rewritten by every call.  The summation order is fixed (deterministic).
 * Errors: MHDE_EINVAL (bad sizes / NULL), MHDE_EWORKSPACE (scratch too
 * small), MHDE_ECUDA (launch failed). */
int mhde_block_gram(const double* V, size_t v_stride, int kblocks, const double* W, int n_rows, int ld,
                    int r, double* G, void* scratch, size_t scratch_bytes, void* stream);

/* FP32 block Gram, the Krylov precision of the mixed path: the same G (in
 * FP64) from FP32 V_i and W, same layout and limits as mhde_block_gram.
 * use_tensor_cores = 1 runs the tensor-core kernel (tcgen05, TF32 on split
 * operands: x = hi + lo with hi exact in TF32, products hi*hi + hi*lo + lo*hi
 * accumulated in FP32, relative error about 2^-21 per product; needs r <= 64,
 * ld <= 64, 16-byte aligned V and W and v_stride a multiple of 4, else
 * MHDE_EINVAL); 0 runs the CUDA-core kernels.  scratch: device, at least
 * mhde_block_gram_f32_scratch_bytes() bytes, owned by the caller.  The call
 * synchronizes `stream` and returns MHDE_ECUDA if a kernel's bounded wait for
 * its shared-memory stages gave up (G is then not valid). */
int mhde_block_gram_f32_scratch_bytes(int n_rows, int r, int kblocks, size_t* bytes);
int mhde_block_gram_f32(const float* V, size_t v_stride, int kblocks, const float* W, int n_rows, int ld, int r,
                        double* G, void* scratch, size_t scratch_bytes, int use_tensor_cores, void* stream);

/* Block combination of the block Krylov solve in FP32 (the new basis block
 * and the solution update, Section 1 block solvers):
 *   out[row][q] = alpha in[row][q] + sum_{i < kblocks} sum_{p < r_in} V_i[row][p] C_i[p][q]
 * for q < r_out, and 0 for r_out <= q < ldo.  V_i = V + i * v_stride
 * (elements), rows of stride ldv; in (may be NULL: alpha ignored) and out
 * rows of stride ldo; C: device [kblocks][r_in][r_out].  out may alias in or
 * one of the V_i (every row is read before it is written).  use_tensor_cores
 * = 1 runs the tensor-core kernel (tcgen05, TF32 on split operands as in
 * mhde_block_gram_f32; r_out <= 64 and the shared-memory plan must fit,
 * 16-byte aligned out, in and V, else MHDE_EINVAL); 0 the CUDA-core kernel.
 * scratch: device, >= 256 bytes (error word).  The call synchronizes
 * `stream`; MHDE_ECUDA if a bounded wait gave up. */
int mhde_block_combine_f32(float* out, const float* in, float alpha, const float* V, size_t v_stride, int kblocks,
                           int r_in, const float* C, int r_out, int n_rows, int ldv, int ldo, void* scratch,
                           size_t scratch_bytes, int use_tensor_cores, void* stream);

/* Allocation-free variant of mhde_block_gram, for callers that must not
 * allocate device memory (hosts that own the whole device through their own
 * pool, latency-critical loops that cannot afford cudaMalloc).  The paper has
 * no counterpart: this is a property of the library, not of the method.
 * Same arguments and result as mhde_block_gram without the scratch buffer:
 * the partial sums live in one fixed 2 MiB __device__ array that every GPU
 * loading the library holds until the process exits.  Sizes whose partials
 * for one row chunk exceed it (kblocks * r * r > 262144) are rejected with
 * MHDE_EWORKSPACE; larger n_rows are handled with fewer, longer chunks.
 * kblocks > 65535 is MHDE_EINVAL, as for mhde_block_gram.
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture, and do not call again on a device after a
 * cudaDeviceReset of it in the same process (the kept address is then stale).  All
 * calls share the array, so calls that overlap on the GPU (different streams
 * without ordering) race; order them on one stream.  Every call rewrites the
 * partials it uses, so no clearing is needed.  Allocates nothing: no
 * cudaMalloc, cudaFree or allocating library routine. */
int mhde_block_gram_noalloc(const double* V, size_t v_stride, int kblocks, const double* W, int n_rows,
                            int ld, int r, double* G, void* stream);

/* Measured rate of independent FP64 fused multiply-adds on the current
 * device in TFLOP/s (dependent chains, 8 per thread, 8 CTAs of 256 threads
 * per SM, CUDA events on `stream`): the roofline denominator of the
 * library's FP64 kernels.  The paper has no counterpart; this measures the
 * hardware the library runs on.  Synchronizes `stream`. */
int mhde_fp64_fma_rate(void* stream, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* MHDE_H */
