// One subproblem of a time step (eq. weaknew1 or weaknew2 for all J members):
// shared-matrix assembly, batched right-hand sides, and the block solve
// A [x_1 | ... | x_J] = [b_1 | ... | b_J] (Section 1) by FP64 iterative
// refinement around a right-preconditioned block GMRES(m) in the Krylov
// precision T (double on the FP64 path, float on the mixed path).
//
// Preconditioner (block upper triangular, fixed and linear):
//   z_p = -(1/dt) L_p^{-1} r_p - nu_hat M_p^{-1} r_p      (pressure Schur part)
//   z_u = Jacobi_k(F, r_u - B^T z_p)                     (velocity part)
// with L_p the P1 pressure Laplacian (one smoothed-aggregation V-cycle) and
// M_p the lumped pressure mass.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <chrono>
#include <cstdio>
#include <cstring>

#include "kernels.h"

namespace mhde {

#define SCU(call)                                                        \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                             \
      s.err = std::string(#call) + ": " + cudaGetErrorString(e_);        \
      return MHDE_ECUDA;                                                 \
    }                                                                    \
  } while (0)

// Phase timing for MHDE_TRACE=1 runs: synchronizes the stream at phase
// boundaries (diagnostics only; off by default).
struct PhaseClock {
  const mhde_ctx* c;
  Sub& s;
  std::chrono::steady_clock::time_point t0;
  PhaseClock(const mhde_ctx* c_, Sub& s_) : c(c_), s(s_) {
    if (c->trace) {
      cudaStreamSynchronize(s.stream);
      t0 = std::chrono::steady_clock::now();
    }
  }
  void stop(int phase) {
    if (!c->trace) return;
    cudaStreamSynchronize(s.stream);
    s.phase_ms[phase] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

template <typename T> struct Prec;
template <> struct Prec<double> {
  static const double* F(const Sub& s) { return s.Fval; }
  static const double* Fd(const Sub& s) { return s.Fdinv; }
  static const double* FD(const Sub& s) { return s.FD; }
  static const double* B(const mhde_ctx* c) { return c->B.val; }
  static const double* BT(const mhde_ctx* c) { return c->BT.val; }
  static const double* mp(const mhde_ctx* c) { return c->d_mp; }
  static const double* lscd(const mhde_ctx* c) { return c->d_lsc_dinv; }
  static const double* Aval(const DevCsr& A) { return A.val; }
  static const double* Adinv(const DevCsr& A) { return A.dinv; }
  static double* x(DevAmgLevel& L) { return L.x; }
  static const double* blkinv(const DevAmgLevel& L) { return L.blk_inv; }
  static double* b(DevAmgLevel& L) { return L.b; }
  static double* r(DevAmgLevel& L) { return L.r; }
  static const double* cinv(const mhde_ctx* c) { return c->d_coarse_inv; }
  static const double* Np(const Sub& s) { return s.Np; }
  static constexpr double thresh = 1e-22;
};
template <> struct Prec<float> {
  static const float* F(const Sub& s) { return s.Fvalf; }
  static const float* Fd(const Sub& s) { return s.Fdinvf; }
  static const float* FD(const Sub& s) { return s.FDf; }
  static const float* B(const mhde_ctx* c) { return c->B.valf; }
  static const float* BT(const mhde_ctx* c) { return c->BT.valf; }
  static const float* mp(const mhde_ctx* c) { return c->d_mpf; }
  static const float* lscd(const mhde_ctx* c) { return c->d_lsc_dinvf; }
  static const float* Aval(const DevCsr& A) { return A.valf; }
  static const float* Adinv(const DevCsr& A) { return A.dinvf; }
  static float* x(DevAmgLevel& L) { return L.xf; }
  static const float* blkinv(const DevAmgLevel& L) { return L.blk_invf; }
  static float* b(DevAmgLevel& L) { return L.bf; }
  static float* r(DevAmgLevel& L) { return L.rf; }
  static const float* cinv(const mhde_ctx* c) { return c->d_coarse_invf; }
  static const float* Np(const Sub& s) { return s.Npf; }
  static constexpr double thresh = 1e-9;
};

// ------------------------------------------------------------------ preconditioner
template <typename T>
static void vcycle(const mhde_ctx* c, Sub& s, int l, const T* b, T* x, int Jp) {
  const int L = (int)c->amg_ops.size();
  cudaStream_t st = s.stream;
  if (l == L - 1) {
    launch_dense_apply<T>(c->fe.amg.nc, Prec<T>::cinv(c), b, x, Jp, st);
    return;
  }
  const DevAmgLevel& op = c->amg_ops[l];
  DevAmgLevel& w = s.amg[l];
  const DevCsr& A = op.A;
  const T om = (T)op.omega;
  const int nsw = std::max(1, c->opt.amg_sweeps);
  if (op.bs > 0) {
    // block-Jacobi smoothing in place on x; residuals are staged in this
    // level's right-hand-side buffer, which the finest level (the only one
    // with blocks; its right-hand side comes from the caller) leaves unused
    T* tmp = Prec<T>::b(w);
    const T bom = (T)op.blk_omega;
    launch_block_jacobi<T>(op.nb, op.bs, op.blk_idx, Prec<T>::blkinv(op), bom, nullptr, b, x, Jp, st);
    for (int k = 1; k < nsw; ++k) {
      launch_csr<T>(A.nrows, A.rowptr, A.col, Prec<T>::Aval(A), nullptr, T(0), x, b, tmp, 1, Jp, st);
      launch_block_jacobi<T>(op.nb, op.bs, op.blk_idx, Prec<T>::blkinv(op), bom, x, tmp, x, Jp, st);
    }
    DevAmgLevel& wn = s.amg[l + 1];
    launch_csr<T>(A.nrows, A.rowptr, A.col, Prec<T>::Aval(A), nullptr, T(0), x, b, tmp, 1, Jp, st);
    launch_csr<T>(op.R.nrows, op.R.rowptr, op.R.col, Prec<T>::Aval(op.R), nullptr, T(0), tmp, nullptr,
                  Prec<T>::b(wn), 0, Jp, st);
    vcycle<T>(c, s, l + 1, Prec<T>::b(wn), Prec<T>::x(wn), Jp);
    launch_csr<T>(op.P.nrows, op.P.rowptr, op.P.col, Prec<T>::Aval(op.P), nullptr, T(0), Prec<T>::x(wn), nullptr, x,
                  4, Jp, st);
    for (int k = 0; k < nsw; ++k) {
      launch_csr<T>(A.nrows, A.rowptr, A.col, Prec<T>::Aval(A), nullptr, T(0), x, b, tmp, 1, Jp, st);
      launch_block_jacobi<T>(op.nb, op.bs, op.blk_idx, Prec<T>::blkinv(op), bom, x, tmp, x, Jp, st);
    }
    return;
  }
  T* cur = x;
  T* other = Prec<T>::r(w);
  // pre-smoothing from zero
  launch_csr<T>(A.nrows, A.rowptr, A.col, Prec<T>::Aval(A), Prec<T>::Adinv(A), om, nullptr, b, cur, 3,
                Jp, st);
  for (int k = 1; k < nsw; ++k) {
    launch_csr<T>(A.nrows, A.rowptr, A.col, Prec<T>::Aval(A), Prec<T>::Adinv(A), om, cur, b, other, 2,
                  Jp, st);
    std::swap(cur, other);
  }
  // residual, restriction, coarse correction
  DevAmgLevel& wn = s.amg[l + 1];
  launch_csr<T>(A.nrows, A.rowptr, A.col, Prec<T>::Aval(A), nullptr, T(0), cur, b, other, 1, Jp, st);
  const DevCsr& R = op.R;
  launch_csr<T>(R.nrows, R.rowptr, R.col, Prec<T>::Aval(R), nullptr, T(0), other, nullptr,
                Prec<T>::b(wn), 0, Jp, st);
  vcycle<T>(c, s, l + 1, Prec<T>::b(wn), Prec<T>::x(wn), Jp);
  // prolongation into the buffer from which the nsw post-smoothing sweeps
  // (each writing the other buffer) end in x: no copy closes the level (the
  // residual in `other` has been restricted already, so it may be overwritten)
  const DevCsr& P = op.P;
  T* post = (nsw % 2 == 1) ? (x == cur ? other : cur) : x;
  if (post == cur) {
    launch_csr<T>(P.nrows, P.rowptr, P.col, Prec<T>::Aval(P), nullptr, T(0), Prec<T>::x(wn), nullptr, cur, 4,
                  Jp, st);
  } else {
    launch_csr<T>(P.nrows, P.rowptr, P.col, Prec<T>::Aval(P), nullptr, T(0), Prec<T>::x(wn), cur, post, 5,
                  Jp, st);
    other = cur;
    cur = post;
  }
  for (int k = 0; k < nsw; ++k) {
    launch_csr<T>(A.nrows, A.rowptr, A.col, Prec<T>::Aval(A), Prec<T>::Adinv(A), om, cur, b, other, 2,
                  Jp, st);
    std::swap(cur, other);
  }
  if (cur != x)    // not reached: the parity above ends the sweeps in x
    cudaMemcpyAsync(x, cur, (size_t)A.nrows * Jp * sizeof(T), cudaMemcpyDeviceToDevice, st);
}

// x0 = L^{-1} rhs approximated by amg_cycles V-cycles on the pressure
// Laplacian; further cycles work on the residual, x0 += V(rhs - L x0),
// staged in the pressure parts of the preconditioner temporaries Tk / Pk
template <typename T>
static void amg_solve(const mhde_ctx* c, Sub& s, const T* rhs, T* x0, int Jp) {
  const size_t poff = (size_t)2 * c->fe.n2 * Jp;
  cudaStream_t st = s.stream;
  vcycle<T>(c, s, 0, rhs, x0, Jp);
  for (int cyc = 1; cyc < c->opt.amg_cycles; ++cyc) {
    const DevCsr& A0 = c->amg_ops[0].A;
    T* res = (T*)s.Tk + poff;
    T* corr = (T*)s.Pk + poff;
    launch_csr<T>(A0.nrows, A0.rowptr, A0.col, Prec<T>::Aval(A0), nullptr, T(0), x0, rhs, res, 1, Jp, st);
    vcycle<T>(c, s, 0, res, corr, Jp);
    launch_axpby<T>(x0, T(1), x0, T(1), corr, (size_t)A0.nrows * Jp, st);
  }
}

template <typename T>
static void apply_prec_raw(const mhde_ctx* c, Sub& s, const T* in, T* out, int Jp) {
  const size_t poff = (size_t)2 * c->fe.n2 * Jp;
  cudaStream_t st = s.stream;
  T* tk = (T*)s.Tk;
  T* pk = (T*)s.Pk;
  const T* rp = in + poff;
  T* x0 = Prec<T>::x(s.amg[0]);
  const DevCsr& Kp = c->amg_ops[0].A;
  amg_solve<T>(c, s, rp, x0, Jp);
  if (c->opt.schur == 2) {
    // least-squares commutator: x0 = L^{-1} (B D^{-1} F D^{-1} B^T) L^{-1} rp,
    // zp = -x0; the middle product passes through the velocity parts of
    // Tk / Pk (free until the B^T apply below) and the pressure part of out
    T* zmid = out + poff;
    launch_lsc_middle<T>(c, Prec<T>::F(s), Prec<T>::BT(c), Prec<T>::B(c), Prec<T>::lscd(c), x0, tk, pk, zmid, Jp,
                         st);
    amg_solve<T>(c, s, zmid, x0, Jp);
    launch_precond_p<T>(c->fe.np, Jp, x0, rp, Prec<T>::mp(c), T(1), T(0), Kp.rowptr, Kp.col, (const T*)nullptr,
                        out + poff, st);
  } else {
    const double nu_hat = 0.5 * (c->nubar + c->nubar_m);
    launch_precond_p<T>(c->fe.np, Jp, x0, rp, Prec<T>::mp(c), (T)(1.0 / c->dt), (T)nu_hat, Kp.rowptr, Kp.col,
                        c->opt.schur == 1 ? Prec<T>::Np(s) : (const T*)nullptr, out + poff, st);
  }
  launch_bt_apply<T>(c, Prec<T>::BT(c), in, out + poff, tk, Jp, st);
  if (c->opt.inner_iters > 0) {
    launch_inner_gmres<T>(c, s, Prec<T>::FD(s), Prec<T>::Fd(s), tk, out, Jp, c->opt.inner_iters, st);
    return;
  }
  const int nsw = std::max(1, c->opt.jacobi_sweeps);
  const T om = (T)c->opt.jacobi_omega;
  T* cur = out;
  T* other = pk;
  launch_jacobi_F<T>(c, Prec<T>::F(s), Prec<T>::Fd(s), om, tk, nullptr, cur, Jp, st);
  for (int k = 1; k < nsw; ++k) {
    launch_jacobi_F<T>(c, Prec<T>::F(s), Prec<T>::Fd(s), om, tk, cur, other, Jp, st);
    std::swap(cur, other);
  }
  if (cur != out) cudaMemcpyAsync(out, cur, poff * sizeof(T), cudaMemcpyDeviceToDevice, st);
}

// The preconditioner is a fixed sequence of ~30 small kernels whose pointers
// and scalars do not change for the lifetime of the context (matrix values are
// read at execution time), so each (in, out) pair is captured once into a
// CUDA graph and replayed.
static std::mutex g_capture_mutex;

template <typename T>
static void apply_prec(const mhde_ctx* c, Sub& s, const T* in, T* out, int ld) {
  if (!c->use_graphs || s.graphs_off) {
    apply_prec_raw<T>(c, s, in, out, ld);
    return;
  }
  auto key = std::make_tuple((const void*)in, (const void*)out, ld);
  auto it = s.prec_graphs.find(key);
  if (it == s.prec_graphs.end()) {
    // one capture at a time in the process: many contexts stepped from many
    // host threads (mhde_advance_many) otherwise capture concurrently
    std::lock_guard<std::mutex> lock(g_capture_mutex);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      apply_prec_raw<T>(c, s, in, out, ld);
      return;
    }
    set_capturing(true);
    apply_prec_raw<T>(c, s, in, out, ld);
    set_capturing(false);
    size_t nodes = 0;
    if (cudaStreamEndCapture(s.stream, &g) != cudaSuccess || cudaGraphGetNodes(g, nullptr, &nodes) != cudaSuccess ||
        cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      s.graphs_off = true;   // do not retry a capture that failed once
      apply_prec_raw<T>(c, s, in, out, ld);
      return;
    }
    cudaGraphDestroy(g);
    s.graphs_built++;
    it = s.prec_graphs.emplace(key, std::make_pair(ge, (long long)nodes)).first;
  }
  cudaGraphLaunch(it->second.first, s.stream);
  count_launch(it->second.second);
}

// ------------------------------------------------------------------ small helpers
// Column norms (sqrt of the column sums of squares) of a [n_rows][Jp] vector.
template <typename T>
static int col_norms(const mhde_ctx* c, Sub& s, const T* X, std::vector<double>& nrm) {
  launch_colsq<T>(X, c->n_rows, c->Jp, c->nchunk, s.colsq, s.stream);
  SCU(cudaMemcpyAsync(s.hcol, s.colsq, sizeof(double) * c->nchunk * c->Jp, cudaMemcpyDeviceToHost,
                      s.stream));
  SCU(cudaStreamSynchronize(s.stream));
  nrm.assign(c->J, 0.0);
  for (int ch = 0; ch < c->nchunk; ++ch)
    for (int j = 0; j < c->J; ++j) nrm[j] += s.hcol[(size_t)ch * c->Jp + j];
  for (auto& v : nrm) v = std::sqrt(v);
  return MHDE_OK;
}

// Row chunks of a block Gram: as many as the partial-sum buffer holds (up to
// 8 per SM), so that small blocks still fill the GPU.
static int gram_chunks(const mhde_ctx* c, int k, int r) {
  const size_t cap = (size_t)c->nchunk * (c->opt.restart + 1) * c->J * c->J;
  const size_t per = (size_t)k * r * r;
  return (int)std::max<size_t>(1, std::min<size_t>({cap / per, (size_t)1216, (size_t)((c->n_rows + 63) / 64)}));
}

// Gram of V_0..V_{k-1} against W (r columns) -> host array [k][r][r].
template <typename T>
static int gram_host(const mhde_ctx* c, Sub& s, const T* V, size_t vstride, int k, const T* W, int r,
                     std::vector<double>& out, int ld) {
  launch_gram<T>(V, vstride, k, W, c->n_rows, ld, r, gram_chunks(c, k, r), s.part, s.gram, s.stream, true, s.d_err,
                 c->gram_tc);
  SCU(cudaMemcpyAsync(s.hbuf, s.gram, sizeof(double) * k * r * r, cudaMemcpyDeviceToHost, s.stream));
  SCU(cudaStreamSynchronize(s.stream));
  out.assign(s.hbuf, s.hbuf + (size_t)k * r * r);
  return MHDE_OK;
}

// Gram of V_0..V_k and W against W (k + 2 blocks), then the projected Gram
// W^T W - sum_i H_i^T H_i as block k + 2 -> host array of (k + 3) r r values.
template <typename T>
static int gram_proj_host(const mhde_ctx* c, Sub& s, const T* V, size_t vstride, int k, const T* W, int r, int ld,
                          std::vector<double>& out) {
  launch_gram<T>(V, vstride, k + 2, W, c->n_rows, ld, r, gram_chunks(c, k + 2, r), s.part, s.gram, s.stream, true,
                 s.d_err, c->gram_tc);
  launch_proj_gram(s.gram, k, r, s.stream);
  const size_t n = (size_t)(k + 3) * r * r;
  SCU(cudaMemcpyAsync(s.hbuf, s.gram, sizeof(double) * n, cudaMemcpyDeviceToHost, s.stream));
  SCU(cudaStreamSynchronize(s.stream));
  out.assign(s.hbuf, s.hbuf + n);
  return MHDE_OK;
}

// Upload coefficients (host doubles, converted to T) into staging slot
// `slot` (0..3) of the pinned host buffer and of the device coefficient
// buffer, without synchronizing: a slot is rewritten only after a later
// host synchronization (gram_host / col_norms) has drained the stream.
template <typename T>
static T* upload_coef(const mhde_ctx* c, Sub& s, const std::vector<double>& h, int slot) {
  const size_t cap = (size_t)(c->opt.restart + 1) * c->J * c->J;
  T* hc = reinterpret_cast<T*>(reinterpret_cast<double*>(s.hcoef) + (size_t)slot * cap);
  T* dc = reinterpret_cast<T*>(reinterpret_cast<char*>(s.coef) + (size_t)slot * cap * sizeof(double));
  for (size_t i = 0; i < h.size(); ++i) hc[i] = (T)h[i];
  cudaMemcpyAsync(dc, hc, sizeof(T) * h.size(), cudaMemcpyHostToDevice, s.stream);
  return dc;
}

// SVQB normalisation of an r-column Gram matrix G: keeps eigen-directions
// above thresh * lambda_max.  T_ = U_k Lambda_k^{-1/2} (r x k),
// S_ = Lambda_k^{1/2} U_k^T (k x r).  Returns the kept rank k.
static int svqb(int r, const std::vector<double>& G, double thresh, std::vector<double>& Tm,
                std::vector<double>& Sm) {
  std::vector<double> w(r), U((size_t)r * r);
  eig_sym(r, G.data(), w.data(), U.data());
  double lmax = std::max(w[0], 0.0);
  int k = 0;
  while (k < r && w[k] > thresh * lmax && w[k] > 0.0) ++k;
  Tm.assign((size_t)r * k, 0.0);
  Sm.assign((size_t)k * r, 0.0);
  for (int i = 0; i < r; ++i)
    for (int t = 0; t < k; ++t) {
      double sq = std::sqrt(w[t]);
      Tm[(size_t)i * k + t] = U[(size_t)i * r + t] / sq;
      Sm[(size_t)t * r + i] = U[(size_t)i * r + t] * sq;
    }
  return k;
}

// ------------------------------------------------------------------ block GMRES
// One cycle of right-preconditioned block GMRES for A D = R, where the first
// basis block V_0 = Res C0 is built from the FP64 residual (C0: J x r, FP64)
// and R = V_0 S0 (S0: r x J) are the unit-scaled columns of the residual.
// Stops when every column's residual estimate is <= tol, at m blocks, at a
// (numerically) rank-deficient new block, or after maxit iterations.  The
// correction D = P^{-1} V Y is left in s.Dk (Krylov precision).
template <typename T>
static int gmres_cycle(mhde_ctx* c, Sub& s, const std::vector<double>& C0, const std::vector<double>& S0,
                       int r, double tol, int maxit, int& used) {
  const int J = c->J, Jp = c->Jp, m = c->opt.restart;
  const size_t vs = (size_t)c->n_rows * Jp;
  cudaStream_t st = s.stream;
  T* Vb = (T*)s.basis;
  T* D = (T*)s.Dk;
  T* Wk = (T*)s.Wk;
  T* Zk = (T*)s.Zk;
  const double thresh = Prec<T>::thresh;
  used = 0;
  int rc;
  // the Krylov blocks carry only the r kept directions: rows of stride Rp
  const int Rp = (r + 3) / 4 * 4;
  double* dC0 = upload_coef<double>(c, s, C0, 3);
  launch_combine_from_f64<T>(Vb, s.Res, dC0, J, r, c->n_rows, Jp, Rp, st);
  BlockLS& ls = s.ls;                            // kept in the subproblem: no reallocation per cycle
  ls.init(r, J, m, S0.data());
  std::vector<double> G, H, Y, Hsum, Gp;
  int k = 0;
  T* Zb = (T*)s.zbasis;
  T* dcoef = (T*)s.coef;                         // combination coefficients (staging slot 0)
  bool ahead = false;                            // this block's preconditioner and operator are queued
  for (; k < m && used < maxit; ++k) {
    T* Vk = Vb + (size_t)k * vs;
    T* Zk_ = Zb + (size_t)k * vs;                 // flexible GMRES keeps every preconditioned block
    T* Wn = Vb + (size_t)(k + 1) * vs;            // W = A Z_k is built in the next basis slot
    if (!ahead) {
      PhaseClock pc1(c, s);
      apply_prec<T>(c, s, Vk, Zk_, Rp);
      pc1.stop(2);
      PhaseClock pc2(c, s);
      launch_saddle_spmm<T>(c, Prec<T>::F(s), Prec<T>::B(c), Prec<T>::BT(c), Zk_, nullptr, Wn, 0, Rp, st);
      pc2.stop(3);
    }
    ahead = false;
    PhaseClock pc3(c, s);
    // one reduction: [V_0 .. V_k, W]^T W gives the projections H_i = V_i^T W
    // and W^T W; the projected block's Gram W^T W - H^T H is formed on the
    // device, so the host receives H, the projected Gram and both traces
    if ((rc = gram_proj_host<T>(c, s, Vb, vs, k, Wn, r, Rp, G))) return rc;
    const size_t rr = (size_t)r * r;
    Hsum.assign(G.begin(), G.begin() + (size_t)(k + 1) * rr);
    Gp.assign(G.begin() + (size_t)(k + 2) * rr, G.begin() + (size_t)(k + 3) * rr);
    double trW = 0.0, trP = 0.0;
    for (int p = 0; p < r; ++p) {
      trW += G[(size_t)(k + 1) * rr + (size_t)p * r + p];
      trP += Gp[(size_t)p * r + p];
    }
    std::vector<double> Tn, Sn;
    int rk;
    if (trP > 1e-3 * trW) {
      rk = cholqr_factors(r, Gp, thresh, Tn, Sn) ? r : svqb(r, Gp, thresh, Tn, Sn);
      if (rk == r) {
        // V_{k+1} = (W - sum_i V_i H_i) T  in one pass, in place; the
        // coefficients -H_i T and T are formed on the device
        const double* dT = upload_coef<double>(c, s, Tn, 1);
        launch_make_coef<T>(s.gram, dT, k, r, dcoef, st);
        launch_block_combine<T>(Wn, nullptr, T(0), Vb, vs, k + 2, r, dcoef, r, c->n_rows, Rp, Rp, st, s.d_err, c->comb_tc);
      }
    } else {
      // strong cancellation: explicit two-pass Gram-Schmidt for this block
      H.assign(Hsum.begin(), Hsum.end());
      for (auto& v : H) v = -v;
      T* dc = upload_coef<T>(c, s, H, 0);
      launch_block_combine<T>(Wn, Wn, T(1), Vb, vs, k + 1, r, dc, r, c->n_rows, Rp, Rp, st, s.d_err, c->comb_tc);
      if ((rc = gram_host<T>(c, s, Vb, vs, k + 1, Wn, r, H, Rp))) return rc;
      for (size_t t2 = 0; t2 < H.size(); ++t2) Hsum[t2] += H[t2];
      for (auto& v : H) v = -v;
      dc = upload_coef<T>(c, s, H, 1);
      launch_block_combine<T>(Wn, Wn, T(1), Vb, vs, k + 1, r, dc, r, c->n_rows, Rp, Rp, st, s.d_err, c->comb_tc);
      if ((rc = gram_host<T>(c, s, Wn, 0, 1, Wn, r, G, Rp))) return rc;
      rk = svqb(r, G, thresh, Tn, Sn);
      if (rk == r) {
        dc = upload_coef<T>(c, s, Tn, 2);
        launch_block_combine<T>(Wn, nullptr, T(0), Wn, 0, 1, r, dc, r, c->n_rows, Rp, Rp, st, s.d_err, c->comb_tc);
      }
    }
    pc3.stop(4);
    const bool breakdown = rk < r;
    // queue the next block's preconditioner and operator before the host
    // updates the least-squares problem, so that the two overlap; if this
    // block turns out to be the last, that work is simply not used
    if (!breakdown && k + 1 < m && used + 1 < maxit && !c->trace) {
      T* Vn = Wn;
      T* Zn = Zb + (size_t)(k + 1) * vs;
      apply_prec<T>(c, s, Vn, Zn, Rp);
      launch_saddle_spmm<T>(c, Prec<T>::F(s), Prec<T>::B(c), Prec<T>::BT(c), Zn, nullptr,
                            Vb + (size_t)(k + 2) * vs, 0, Rp, st);
      ahead = true;
    }
    PhaseClock pc4(c, s);
    // new block column of the Hessenberg matrix, row-major: [H_0; ...; H_k; S]
    std::vector<double> hblk((size_t)(k + 2) * rr, 0.0);
    std::copy(Hsum.begin(), Hsum.begin() + (size_t)(k + 1) * rr, hblk.begin());
    // at a breakdown the rk significant directions of the projected block
    // (rows of Sn) still enter the least-squares problem: the cycle ends, but
    // its correction must minimise the true residual, not one that takes the
    // whole new block to lie in the basis
    if (!breakdown)
      std::copy(Sn.begin(), Sn.begin() + rr, hblk.begin() + (size_t)(k + 1) * rr);
    else
      std::copy(Sn.begin(), Sn.begin() + (size_t)rk * r, hblk.begin() + (size_t)(k + 1) * rr);
    bool ok = ls.add(hblk.data());
    pc4.stop(5);
    used++;
    double worst = 0.0;
    for (int j = 0; j < J; ++j) worst = std::max(worst, ls.resid(j));
    if (!std::isfinite(worst)) {
      s.err = "non-finite Krylov residual";
      return MHDE_ENAN;
    }
    if (worst <= tol || breakdown || !ok) {
      k++;
      break;
    }
  }
  ls.solve(Y);
  T* dc = upload_coef<T>(c, s, Y, 3);
  launch_block_combine<T>(D, nullptr, T(0), Zb, vs, k, r, dc, J, c->n_rows, Rp, Jp, st, s.d_err, c->comb_tc);
  return MHDE_OK;
}

// ------------------------------------------------------------------ subproblem
int assemble_sub(mhde_ctx* c, int which) {
  Sub& s = c->sub[which];
  cudaStream_t st = s.stream;
  PhaseClock pa(c, s);
  const Sub& o = c->sub[1 - which];
  const double* mean_conv = which == 0 ? c->d_mean_w : c->d_mean_v;
  const double* l2 = which == 0 ? c->d_l2_w : c->d_l2_v;
  const double nu_hat = 0.5 * (c->nubar + c->nubar_m);
  launch_F_local(c->fe.nt, c->d_dofs, c->d_geom, mean_conv, l2, 2.0 * c->opt.mu * c->dt,
                 c->opt.conv_form, s.Floc, st);
  launch_F_gather(c, s.Floc, 1.0 / c->dt, nu_hat, s.Fval, s.Fvalf, s.Fdinv, s.Fdinvf, st);
  launch_fd_values(c, s, st);
  if (c->opt.schur == 1) launch_Np(c, mean_conv, s.Floc, s.Np, s.Npf, st);   // slots reuse Floc
  launch_rhs_conv_local(c->fe.nt, c->J, c->Jp, c->d_dofs, c->d_geom, s.S, o.S, mean_conv,
                        c->opt.conv_form, s.Cloc, st);
  launch_rhs_assemble(c, s.S, o.S, c->have_forcing ? (which == 0 ? c->d_F1 : c->d_F2) : nullptr,
                      which == 0 ? c->d_Gv : c->d_Gw, s.Cloc, c->d_ccross, c->d_csame, s.Bv, st);
  SCU(cudaGetLastError());
  pa.stop(0);
  return MHDE_OK;
}

template <typename T>
static int solve_sub_t(mhde_ctx* c, int which, bool zero_guess) {
  Sub& s = c->sub[which];
  cudaStream_t st = s.stream;
  const int J = c->J;
  const size_t vs = (size_t)c->n_rows * c->Jp;
  int rc;
  // initial guess: linear extrapolation in time of the last two states
  if (zero_guess)
    SCU(cudaMemsetAsync(s.X, 0, vs * sizeof(double), st));
  else if (c->have_prev)
    launch_axpby<double>(s.X, 2.0, s.S, -1.0, s.Sprev, vs, st);
  else
    SCU(cudaMemcpyAsync(s.X, s.S, vs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  std::vector<double> bn, G, Gs, Tm, Sm, C0;
  if ((rc = col_norms<double>(c, s, s.Bv, bn))) return rc;
  s.iters = 0;
  s.refine = 0;
  const bool fp64 = std::is_same<T, double>::value;
  std::vector<double> rn(J), sc(J), unscale(c->Jp, 0.0);
  for (;;) {
    // FP64 residual and its Gram matrix (column norms on the diagonal)
    PhaseClock pc0(c, s);
    launch_saddle_spmm<double>(c, s.Fval, c->B.val, c->BT.val, s.X, s.Bv, s.Res, 1, c->Jp, st);
    if ((rc = gram_host<double>(c, s, s.Res, 0, 1, s.Res, J, G, c->Jp))) return rc;
    double worst = 0.0, min_target = 1.0;
    for (int j = 0; j < J; ++j) {
      rn[j] = std::sqrt(std::max(G[(size_t)j * J + j], 0.0));
      double ref = bn[j] > 0.0 ? bn[j] : 1.0;
      double rel = rn[j] / ref;
      if (!std::isfinite(rel)) {
        s.err = "non-finite residual";
        return MHDE_ENAN;
      }
      worst = std::max(worst, rel);
      if (rn[j] > 0.0) min_target = std::min(min_target, c->opt.rtol * ref / rn[j]);
    }
    s.relres = worst;
    pc0.stop(1);
    if (c->trace)
      std::fprintf(stderr, "[mhde] sub %d sweep %d iters %d relres %.3e\n", which, s.refine, s.iters, worst);
    if (worst <= c->opt.rtol) return MHDE_OK;
    if (s.refine >= c->opt.max_refine || s.iters >= c->opt.max_iter) {
      s.err = "solver did not reach rtol (relres " + std::to_string(worst) + ")";
      return MHDE_ENOCONV;
    }
    const double tol_in =
        fp64 ? std::max(0.3 * min_target, 1e-15) : std::max(c->opt.inner_rtol, 0.3 * min_target);
    // unit-scaled Gram, deflated below the inner tolerance, SVQB
    for (int j = 0; j < J; ++j) sc[j] = rn[j] > 0.0 ? 1.0 / rn[j] : 0.0;
    Gs.assign((size_t)J * J, 0.0);
    for (int i = 0; i < J; ++i)
      for (int j = 0; j < J; ++j) Gs[(size_t)i * J + j] = G[(size_t)i * J + j] * sc[i] * sc[j];
    // directions of the unit-scaled residual block below tau start in a later
    // sweep; on the FP64 path tau has a floor, because nearly parallel member
    // residuals kept down to rounding make the Krylov blocks rank-deficient
    // after a few iterations and end every cycle early
    const double tau = 0.1 * (fp64 ? std::max(tol_in, 1e-10) : tol_in) / std::sqrt((double)J);
    const int r = svqb(J, Gs, std::max(tau * tau, 1e-30), Tm, Sm);
    if (r == 0) return MHDE_OK;
    if (c->trace) std::fprintf(stderr, "[mhde] sub %d sweep %d block width %d\n", which, s.refine, r);
    C0.assign((size_t)J * r, 0.0);
    for (int p = 0; p < J; ++p)
      for (int t = 0; t < r; ++t) C0[(size_t)p * r + t] = sc[p] * Tm[(size_t)p * r + t];
    int used = 0;
    if ((rc = gmres_cycle<T>(c, s, C0, Sm, r, tol_in, c->opt.max_iter - s.iters, used))) return rc;
    s.iters += used;
    for (int j = 0; j < J; ++j) unscale[j] = rn[j];
    SCU(cudaMemcpyAsync(s.dscale, unscale.data(), sizeof(double) * c->Jp, cudaMemcpyHostToDevice, st));
    launch_axpy_from<T>((const T*)s.Dk, s.dscale, s.X, vs, c->Jp, st);
    SCU(cudaStreamSynchronize(st));
    s.refine++;
  }
}

void precond_apply_any(mhde_ctx* c, int which, const void* in, void* out) {
  Sub& s = c->sub[which];
  if (c->opt.precision == MHDE_PREC_FP64)
    apply_prec<double>(c, s, (const double*)in, (double*)out, c->Jp);
  else
    apply_prec<float>(c, s, (const float*)in, (float*)out, c->Jp);
}

void gram_any(mhde_ctx* c, int which, const void* V, size_t vstride, int k, const void* W, bool reduce) {
  Sub& s = c->sub[which];
  const int nchunk = gram_chunks(c, k, c->J);
  if (c->opt.precision == MHDE_PREC_FP64)
    launch_gram<double>((const double*)V, vstride, k, (const double*)W, c->n_rows, c->Jp, c->J, nchunk, s.part,
                        s.gram, s.stream, reduce, s.d_err, c->gram_tc);
  else
    launch_gram<float>((const float*)V, vstride, k, (const float*)W, c->n_rows, c->Jp, c->J, nchunk, s.part,
                       s.gram, s.stream, reduce, s.d_err, c->gram_tc);
}

// out = sum_i V_i C_i over k blocks of J columns with the coefficients in
// staging slot 0 (kernel timing)
void combine_any(mhde_ctx* c, int which, const void* V, size_t vstride, int k, void* out) {
  Sub& s = c->sub[which];
  if (c->opt.precision == MHDE_PREC_FP64)
    launch_block_combine<double>((double*)out, nullptr, 0.0, (const double*)V, vstride, k, c->J,
                                 (const double*)s.coef, c->J, c->n_rows, c->Jp, c->Jp, s.stream, s.d_err,
                                c->comb_tc);
  else
    launch_block_combine<float>((float*)out, nullptr, 0.f, (const float*)V, vstride, k, c->J, (const float*)s.coef,
                                c->J, c->n_rows, c->Jp, c->Jp, s.stream, s.d_err,
                                c->comb_tc);
}

int solve_sub(mhde_ctx* c, int which, bool zero_guess) {
  if (c->opt.precision == MHDE_PREC_FP64) return solve_sub_t<double>(c, which, zero_guess);
  return solve_sub_t<float>(c, which, zero_guess);
}

}  // namespace mhde
