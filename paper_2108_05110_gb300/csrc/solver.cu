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

template <typename T> struct Prec;
template <> struct Prec<double> {
  static const double* F(const Sub& s) { return s.Fval; }
  static const double* Fd(const Sub& s) { return s.Fdinv; }
  static const double* B(const mhde_ctx* c) { return c->B.val; }
  static const double* BT(const mhde_ctx* c) { return c->BT.val; }
  static const double* mp(const mhde_ctx* c) { return c->d_mp; }
  static const double* Aval(const DevCsr& A) { return A.val; }
  static const double* Adinv(const DevCsr& A) { return A.dinv; }
  static double* x(DevAmgLevel& L) { return L.x; }
  static double* b(DevAmgLevel& L) { return L.b; }
  static double* r(DevAmgLevel& L) { return L.r; }
  static const double* cinv(const mhde_ctx* c) { return c->d_coarse_inv; }
  static constexpr double thresh = 1e-26;
};
template <> struct Prec<float> {
  static const float* F(const Sub& s) { return s.Fvalf; }
  static const float* Fd(const Sub& s) { return s.Fdinvf; }
  static const float* B(const mhde_ctx* c) { return c->B.valf; }
  static const float* BT(const mhde_ctx* c) { return c->BT.valf; }
  static const float* mp(const mhde_ctx* c) { return c->d_mpf; }
  static const float* Aval(const DevCsr& A) { return A.valf; }
  static const float* Adinv(const DevCsr& A) { return A.dinvf; }
  static float* x(DevAmgLevel& L) { return L.xf; }
  static float* b(DevAmgLevel& L) { return L.bf; }
  static float* r(DevAmgLevel& L) { return L.rf; }
  static const float* cinv(const mhde_ctx* c) { return c->d_coarse_invf; }
  static constexpr double thresh = 1e-11;
};

// ------------------------------------------------------------------ preconditioner
template <typename T>
static void vcycle(const mhde_ctx* c, Sub& s, int l, const T* b, T* x) {
  const int L = (int)c->amg_ops.size();
  const int Jp = c->Jp;
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
  vcycle<T>(c, s, l + 1, Prec<T>::b(wn), Prec<T>::x(wn));
  const DevCsr& P = op.P;
  launch_csr<T>(P.nrows, P.rowptr, P.col, Prec<T>::Aval(P), nullptr, T(0), Prec<T>::x(wn), nullptr, cur, 4,
                Jp, st);
  for (int k = 0; k < nsw; ++k) {
    launch_csr<T>(A.nrows, A.rowptr, A.col, Prec<T>::Aval(A), Prec<T>::Adinv(A), om, cur, b, other, 2,
                  Jp, st);
    std::swap(cur, other);
  }
  if (cur != x)
    cudaMemcpyAsync(x, cur, (size_t)A.nrows * Jp * sizeof(T), cudaMemcpyDeviceToDevice, st);
}

template <typename T>
static void apply_prec(const mhde_ctx* c, Sub& s, const T* in, T* out) {
  const int Jp = c->Jp;
  const size_t poff = (size_t)2 * c->fe.n2 * Jp;
  cudaStream_t st = s.stream;
  T* tk = (T*)s.Tk;
  T* pk = (T*)s.Pk;
  const T* rp = in + poff;
  T* x0 = Prec<T>::x(s.amg[0]);
  vcycle<T>(c, s, 0, rp, x0);
  const double nu_hat = 0.5 * (c->nubar + c->nubar_m);
  launch_precond_p<T>(c->fe.np, Jp, x0, rp, Prec<T>::mp(c), (T)(1.0 / c->dt), (T)nu_hat, out + poff, st);
  launch_bt_apply<T>(c, Prec<T>::BT(c), in, out + poff, tk, st);
  const int nsw = std::max(1, c->opt.jacobi_sweeps);
  const T om = (T)c->opt.jacobi_omega;
  T* cur = out;
  T* other = pk;
  launch_jacobi_F<T>(c, Prec<T>::F(s), Prec<T>::Fd(s), om, tk, nullptr, cur, st);
  for (int k = 1; k < nsw; ++k) {
    launch_jacobi_F<T>(c, Prec<T>::F(s), Prec<T>::Fd(s), om, tk, cur, other, st);
    std::swap(cur, other);
  }
  if (cur != out) cudaMemcpyAsync(out, cur, poff * sizeof(T), cudaMemcpyDeviceToDevice, st);
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

// Gram of V_0..V_{k-1} against W (r columns) -> host array [k][r][r].
template <typename T>
static int gram_host(const mhde_ctx* c, Sub& s, const T* V, size_t vstride, int k, const T* W, int r,
                     std::vector<double>& out) {
  launch_gram<T>(V, vstride, k, W, c->n_rows, c->Jp, r, c->nchunk, s.part, s.gram, s.stream);
  SCU(cudaMemcpyAsync(s.hbuf, s.gram, sizeof(double) * k * r * r, cudaMemcpyDeviceToHost, s.stream));
  SCU(cudaStreamSynchronize(s.stream));
  out.assign(s.hbuf, s.hbuf + (size_t)k * r * r);
  return MHDE_OK;
}

// Upload coefficients (host doubles) to the device coefficient buffer in T.
template <typename T>
static int upload_coef(const mhde_ctx* c, Sub& s, const std::vector<double>& h, T** dev) {
  T* hc = (T*)s.hcoef;
  for (size_t i = 0; i < h.size(); ++i) hc[i] = (T)h[i];
  SCU(cudaMemcpyAsync(s.coef, hc, sizeof(T) * h.size(), cudaMemcpyHostToDevice, s.stream));
  // the host staging buffer is reused by the next upload: wait for this copy
  SCU(cudaStreamSynchronize(s.stream));
  *dev = (T*)s.coef;
  return MHDE_OK;
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
// Solves A D = R0 (both [n_rows][Jp] in T, J columns) to relative residual
// tol per column (columns of R0 have unit norm or are zero); D in s.Dk.
template <typename T>
static int block_gmres(mhde_ctx* c, Sub& s, double tol, int maxit, int& used) {
  const int J = c->J, Jp = c->Jp, m = c->opt.restart;
  const size_t vs = (size_t)c->n_rows * Jp;
  cudaStream_t st = s.stream;
  T* Vb = (T*)s.basis;
  T* R0 = (T*)s.Rk;
  T* D = (T*)s.Dk;
  T* Wk = (T*)s.Wk;
  T* Zk = (T*)s.Zk;
  T* Uk = (T*)s.Uk;
  const double thresh = Prec<T>::thresh;
  SCU(cudaMemsetAsync(D, 0, vs * sizeof(T), st));
  // Rcur = R0 initially, kept in Uk between cycles
  SCU(cudaMemcpyAsync(Uk, R0, vs * sizeof(T), cudaMemcpyDeviceToDevice, st));
  used = 0;
  std::vector<double> G, Tm, Sm, H, Y;
  BlockLS ls;
  int rc;
  while (used < maxit) {
    // block normalisation of the current residual
    if ((rc = gram_host<T>(c, s, Uk, 0, 1, Uk, J, G))) return rc;
    int r = svqb(J, G, thresh, Tm, Sm);
    if (r == 0) return MHDE_OK;          // zero residual
    // early exit if the current residual already meets the tolerance
    {
      double worst = 0.0;
      for (int j = 0; j < J; ++j) worst = std::max(worst, std::sqrt(std::max(G[(size_t)j * J + j], 0.0)));
      if (worst <= tol) return MHDE_OK;
    }
    T* dc;
    if ((rc = upload_coef<T>(c, s, Tm, &dc))) return rc;
    launch_block_combine<T>(Vb, nullptr, T(0), Uk, 0, 1, J, dc, r, c->n_rows, Jp, st);
    ls.init(r, J, m, Sm.data());
    int k = 0;
    bool done = false;
    for (; k < m && used < maxit; ++k) {
      T* Vk = Vb + (size_t)k * vs;
      apply_prec<T>(c, s, Vk, Zk);
      launch_saddle_spmm<T>(c, Prec<T>::F(s), Prec<T>::B(c), Prec<T>::BT(c), Zk, nullptr, Wk, 0, st);
      // block classical Gram-Schmidt, twice
      std::vector<double> Hsum((size_t)(k + 1) * r * r, 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        if ((rc = gram_host<T>(c, s, Vb, vs, k + 1, Wk, r, H))) return rc;
        for (size_t t = 0; t < H.size(); ++t) Hsum[t] += H[t];
        for (auto& v : H) v = -v;
        if ((rc = upload_coef<T>(c, s, H, &dc))) return rc;
        launch_block_combine<T>(Wk, Wk, T(1), Vb, vs, k + 1, r, dc, r, c->n_rows, Jp, st);
      }
      // normalise the new block
      if ((rc = gram_host<T>(c, s, Wk, 0, 1, Wk, r, G))) return rc;
      std::vector<double> Tn, Sn;
      int rk = svqb(r, G, thresh, Tn, Sn);
      bool breakdown = rk < r;
      // block column of the Hessenberg matrix, column-major ((k+2) r) x r
      const int rows = (k + 2) * r;
      std::vector<double> hcol((size_t)rows * r, 0.0);
      for (int i = 0; i <= k; ++i)
        for (int p = 0; p < r; ++p)
          for (int q = 0; q < r; ++q)
            hcol[(size_t)q * rows + i * r + p] = Hsum[(size_t)i * r * r + (size_t)p * r + q];
      if (!breakdown) {
        for (int p = 0; p < r; ++p)
          for (int q = 0; q < r; ++q) hcol[(size_t)q * rows + (k + 1) * r + p] = Sn[(size_t)p * r + q];
        if ((rc = upload_coef<T>(c, s, Tn, &dc))) return rc;
        launch_block_combine<T>(Vb + (size_t)(k + 1) * vs, nullptr, T(0), Wk, 0, 1, r, dc, r, c->n_rows,
                                Jp, st);
      }
      bool ok = ls.add(hcol.data());
      used++;
      double worst = 0.0;
      for (int j = 0; j < J; ++j) worst = std::max(worst, ls.resid(j));
      if (!std::isfinite(worst)) {
        s.err = "non-finite Krylov residual";
        return MHDE_ENAN;
      }
      if (worst <= tol || breakdown || !ok) {
        done = worst <= tol || breakdown;
        k++;
        break;
      }
    }
    // solution of this cycle: D += P^{-1} (V Y)
    ls.solve(Y);
    // Y is (k r) x J row-major: block i is rows i r .. (i+1) r - 1
    if ((rc = upload_coef<T>(c, s, Y, &dc))) return rc;
    launch_block_combine<T>(Wk, nullptr, T(0), Vb, vs, k, r, dc, J, c->n_rows, Jp, st);
    apply_prec<T>(c, s, Wk, Zk);
    launch_axpby<T>(D, T(1), D, T(1), Zk, vs, st);          // D += P^{-1} V Y
    if (done) return MHDE_OK;
    // restart from the true residual of the correction equation: R0 - A D
    launch_saddle_spmm<T>(c, Prec<T>::F(s), Prec<T>::B(c), Prec<T>::BT(c), D, nullptr, Wk, 0, st);
    launch_axpby<T>(Uk, T(1), R0, T(-1), Wk, vs, st);
  }
  return MHDE_OK;
}

// ------------------------------------------------------------------ subproblem
int assemble_sub(mhde_ctx* c, int which) {
  Sub& s = c->sub[which];
  cudaStream_t st = s.stream;
  const Sub& o = c->sub[1 - which];
  const double* mean_conv = which == 0 ? c->d_mean_w : c->d_mean_v;
  const double* l2 = which == 0 ? c->d_l2_w : c->d_l2_v;
  const double nu_hat = 0.5 * (c->nubar + c->nubar_m);
  launch_F_local(c->fe.nt, c->d_dofs, c->d_geom, mean_conv, l2, 2.0 * c->opt.mu * c->dt,
                 c->opt.conv_form, s.Floc, st);
  launch_F_gather(c, s.Floc, 1.0 / c->dt, nu_hat, s.Fval, s.Fvalf, s.Fdinv, s.Fdinvf, st);
  launch_rhs_conv_local(c->fe.nt, c->J, c->Jp, c->d_dofs, c->d_geom, s.S, o.S, mean_conv,
                        c->opt.conv_form, s.Cloc, st);
  launch_rhs_assemble(c, s.S, o.S, c->have_forcing ? (which == 0 ? c->d_F1 : c->d_F2) : nullptr,
                      which == 0 ? c->d_Gv : c->d_Gw, s.Cloc, c->d_ccross, c->d_csame, s.Bv, st);
  SCU(cudaGetLastError());
  return MHDE_OK;
}

template <typename T>
static int solve_sub_t(mhde_ctx* c, int which) {
  Sub& s = c->sub[which];
  cudaStream_t st = s.stream;
  const size_t vs = (size_t)c->n_rows * c->Jp;
  int rc;
  SCU(cudaMemcpyAsync(s.X, s.S, vs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  std::vector<double> bn, rn;
  if ((rc = col_norms<double>(c, s, s.Bv, bn))) return rc;
  s.iters = 0;
  s.refine = 0;
  const bool fp64 = std::is_same<T, double>::value;
  std::vector<double> scale(c->Jp, 0.0), unscale(c->Jp, 0.0);
  for (;;) {
    launch_saddle_spmm<double>(c, s.Fval, c->B.val, c->BT.val, s.X, s.Bv, s.Res, 1, st);
    if ((rc = col_norms<double>(c, s, s.Res, rn))) return rc;
    double worst = 0.0, min_target = 1.0;
    for (int j = 0; j < c->J; ++j) {
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
    if (worst <= c->opt.rtol) return MHDE_OK;
    if (s.refine >= (fp64 ? std::max(c->opt.max_refine, 4) : c->opt.max_refine) ||
        s.iters >= c->opt.max_iter) {
      s.err = "solver did not reach rtol (relres " + std::to_string(worst) + ")";
      return MHDE_ENOCONV;
    }
    double tol_in = fp64 ? std::max(0.3 * min_target, 1e-15) : std::max(c->opt.inner_rtol, 0.3 * min_target);
    for (int j = 0; j < c->Jp; ++j) {
      scale[j] = (j < c->J && rn[j] > 0.0) ? 1.0 / rn[j] : 0.0;
      unscale[j] = (j < c->J) ? rn[j] : 0.0;
    }
    SCU(cudaMemcpyAsync(s.dscale, scale.data(), sizeof(double) * c->Jp, cudaMemcpyHostToDevice, st));
    SCU(cudaMemcpyAsync(s.dscale + c->Jp, unscale.data(), sizeof(double) * c->Jp, cudaMemcpyHostToDevice,
                        st));
    launch_scale_to<T>(s.Res, s.dscale, (T*)s.Rk, vs, c->Jp, st);
    int used = 0;
    if ((rc = block_gmres<T>(c, s, tol_in, c->opt.max_iter - s.iters, used))) return rc;
    s.iters += used;
    launch_axpy_from<T>((const T*)s.Dk, s.dscale + c->Jp, s.X, vs, c->Jp, st);
    SCU(cudaStreamSynchronize(st));
    s.refine++;
  }
}

void precond_apply_any(mhde_ctx* c, int which, const void* in, void* out) {
  Sub& s = c->sub[which];
  if (c->opt.precision == MHDE_PREC_FP64)
    apply_prec<double>(c, s, (const double*)in, (double*)out);
  else
    apply_prec<float>(c, s, (const float*)in, (float*)out);
}

void gram_any(mhde_ctx* c, int which, const void* V, size_t vstride, int k, const void* W) {
  Sub& s = c->sub[which];
  if (c->opt.precision == MHDE_PREC_FP64)
    launch_gram<double>((const double*)V, vstride, k, (const double*)W, c->n_rows, c->Jp, c->J, c->nchunk,
                        s.part, s.gram, s.stream);
  else
    launch_gram<float>((const float*)V, vstride, k, (const float*)W, c->n_rows, c->Jp, c->J, c->nchunk,
                       s.part, s.gram, s.stream);
}

int solve_sub(mhde_ctx* c, int which) {
  if (c->opt.precision == MHDE_PREC_FP64) return solve_sub_t<double>(c, which);
  return solve_sub_t<float>(c, which);
}

}  // namespace mhde
