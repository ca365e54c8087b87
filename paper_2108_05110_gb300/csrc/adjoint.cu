// Gradient of the final-step ensemble energy E_h^K (Section 4.2) with
// respect to the member viscosities nu_j, nu_m,j and the initial fields, by
// the discrete adjoint of Algorithm 1: a forward run that keeps a checkpoint
// every C steps, then a reverse sweep that recomputes each segment of C steps
// from its checkpoint and walks it backwards.  Each reverse step assembles
// both shared matrices from the stored state, solves the transposed systems
// for all members with the block solver (F's values transposed on F's
// structurally symmetric pattern), and contracts the adjoint solutions with
// the derivatives of the right-hand sides and of the shared matrices
// (kernels_adj.cu).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"

using namespace mhde;

namespace {

int adj_fail(mhde_ctx* c, int code, const std::string& msg) {
  c->err = msg;
  return code;
}

#define ACU(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return adj_fail(c, MHDE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct AdjCarver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

struct AdjBuffers {
  double* ckpt = nullptr;     // [nck][4][vs]: S_v, S_w, Sprev_v, Sprev_w
  double* seg = nullptr;      // [C + 1][2][vs]: states of one segment
  double* fin = nullptr;      // [4][vs]: the final state, restored at the end
  double* lamV = nullptr;     // seeds being accumulated for the step's inputs
  double* lamW = nullptr;
  double* seedV = nullptr;    // seeds on the step's outputs
  double* seedW = nullptr;
  double* tmp = nullptr;      // [vs]
  double* prod = nullptr;     // [3][2 n2 Jp]
  double* slotZ = nullptr;    // [nt 6][2][Jp]
  double* slotY = nullptr;
  double* slotM = nullptr;    // [nt 6][2]
  int* kstar = nullptr;       // [nt][NQ]
  double* kap = nullptr;      // [nt][NQ][2]
  double* FT = nullptr;       // [nnz_F]
  float* FTf = nullptr;
  int* tpos = nullptr;        // [nnz_F]
  double* part = nullptr;     // [nchunk][3][Jp]
};

size_t adj_layout(const mhde_ctx* c, int nck, int C, char* base, AdjBuffers& b) {
  AdjCarver w{base};
  const size_t vs = (size_t)c->n_rows * c->Jp;
  const size_t nt = c->fe.nt, n2 = c->fe.n2, Jp = c->Jp, nnz = c->fe.F.nnz();
  b.ckpt = w.take<double>((size_t)std::max(nck, 1) * 4 * vs);
  b.seg = w.take<double>((size_t)(C + 1) * 2 * vs);
  b.fin = w.take<double>(4 * vs);
  b.lamV = w.take<double>(vs);
  b.lamW = w.take<double>(vs);
  b.seedV = w.take<double>(vs);
  b.seedW = w.take<double>(vs);
  b.tmp = w.take<double>(vs);
  b.prod = w.take<double>(3 * 2 * n2 * Jp);
  b.slotZ = w.take<double>(nt * 6 * 2 * Jp);
  b.slotY = w.take<double>(nt * 6 * 2 * Jp);
  b.slotM = w.take<double>(nt * 6 * 2);
  b.kstar = w.take<int>(nt * NQ);
  b.kap = w.take<double>(nt * NQ * 2);
  b.FT = w.take<double>(nnz);
  b.FTf = w.take<float>(nnz);
  b.tpos = w.take<int>(nnz);
  b.part = w.take<double>((size_t)c->nchunk * 3 * Jp);
  return w.off + 256;
}

// position of entry (r, a) for every entry (a, r) of F's pattern
bool transpose_positions(const HostCsr& F, std::vector<int>& tpos) {
  const int n = (int)F.rowptr.size() - 1;
  tpos.assign(F.col.size(), -1);
  for (int a = 0; a < n; ++a)
    for (int k = F.rowptr[a]; k < F.rowptr[a + 1]; ++k) {
      const int r = F.col[k];
      for (int t = F.rowptr[r]; t < F.rowptr[r + 1]; ++t)
        if (F.col[t] == a) {
          tpos[k] = t;
          break;
        }
      if (tpos[k] < 0) return false;
    }
  return true;
}

// One reverse step: the stored state (Sv, Sw) at step n and its successor
// (Xv, Xw); seeds on the successor in b.seedV / b.seedW; the seeds on
// (Sv, Sw) end up in b.lamV / b.lamW; parameter partials added to the host sums.
int reverse_step(mhde_ctx* c, AdjBuffers& b, const double* Sv, const double* Sw, const double* Xv,
                 const double* Xw, std::vector<double>& g_same, std::vector<double>& g_cross, double& g_c1) {
  const size_t vs = (size_t)c->n_rows * c->Jp;
  const int J = c->J, Jp = c->Jp;
  cudaStream_t st = c->sv;
  ACU(cudaMemcpyAsync(c->sub[0].S, Sv, vs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  ACU(cudaMemcpyAsync(c->sub[1].S, Sw, vs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  ACU(cudaMemsetAsync(b.lamV, 0, vs * sizeof(double), st));
  ACU(cudaMemsetAsync(b.lamW, 0, vs * sizeof(double), st));
  launch_means(c->fe.n2, J, Jp, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w, st);
  launch_l2(c->fe.nt, J, Jp, c->d_dofs, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w, c->d_l2_v, c->d_l2_w,
            st);
  ACU(cudaGetLastError());
  ACU(cudaStreamSynchronize(st));
  const long long nnz = (long long)c->fe.F.nnz();
  for (int which = 0; which < 2; ++which) {
    Sub& s = c->sub[which];
    int rc = assemble_sub(c, which);
    if (rc) return adj_fail(c, rc, s.err);
    // transposed shared matrix (and transposed pressure convection of the
    // PCD preconditioner: the skew form's N_p^T = -N_p)
    launch_transpose_values(nnz, b.tpos, s.Fval, b.FT, b.FTf, s.stream);
    ACU(cudaMemcpyAsync(s.Fval, b.FT, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s.stream));
    ACU(cudaMemcpyAsync(s.Fvalf, b.FTf, nnz * sizeof(float), cudaMemcpyDeviceToDevice, s.stream));
    launch_fd_values(c, s, s.stream);               // the inner solve's F^T D^{-1}
    if (c->opt.schur == 1) launch_scale_pair((long long)c->fe.Kp.nnz(), -1.0, s.Np, s.Npf, s.stream);
    launch_adj_rhs(c, which == 0 ? b.seedV : b.seedW, s.Bv, s.stream);
    ACU(cudaGetLastError());
    rc = solve_sub(c, which, true);
    if (rc) return adj_fail(c, rc, std::string(which == 0 ? "v" : "w") + " adjoint solve: " + s.err);
    const double* Z = which == 0 ? Sv : Sw;
    const double* Y = which == 0 ? Sw : Sv;
    const double* meanY = which == 0 ? c->d_mean_w : c->d_mean_v;
    const double* X = which == 0 ? Xv : Xw;
    double* lamZ = which == 0 ? b.lamV : b.lamW;
    double* lamY = which == 0 ? b.lamW : b.lamV;
    launch_adj_contract(c, Z, Y, meanY, X, s.X, b.slotZ, b.slotY, b.slotM, b.kstar, b.kap, lamZ, lamY, b.tmp,
                        b.prod, c->nchunk, b.part, s.stream);
    ACU(cudaGetLastError());
    std::vector<double> part((size_t)c->nchunk * 3 * Jp);
    ACU(cudaMemcpyAsync(part.data(), b.part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
    ACU(cudaStreamSynchronize(s.stream));
    for (int ch = 0; ch < c->nchunk; ++ch)
      for (int j = 0; j < J; ++j) {
        g_same[j] += -0.5 * part[((size_t)ch * 3 + 0) * Jp + j];
        g_cross[j] += -0.5 * part[((size_t)ch * 3 + 1) * Jp + j];
        g_c1 += -part[((size_t)ch * 3 + 2) * Jp + j];
      }
  }
  return MHDE_OK;
}

int copy4(mhde_ctx* c, double* dst, bool save) {
  const size_t vs = (size_t)c->n_rows * c->Jp;
  double* p[4] = {c->sub[0].S, c->sub[1].S, c->sub[0].Sprev, c->sub[1].Sprev};
  for (int i = 0; i < 4; ++i) {
    if (save)
      ACU(cudaMemcpyAsync(dst + i * vs, p[i], vs * sizeof(double), cudaMemcpyDeviceToDevice, c->sv));
    else
      ACU(cudaMemcpyAsync(p[i], dst + i * vs, vs * sizeof(double), cudaMemcpyDeviceToDevice, c->sv));
  }
  ACU(cudaStreamSynchronize(c->sv));
  return MHDE_OK;
}

}  // namespace

extern "C" {

int mhde_adjoint_workspace_size(const mhde_ctx* c, int nsteps, int checkpoint_every, size_t* bytes) {
  if (!c || !bytes || nsteps < 0 || checkpoint_every < 1) return MHDE_EINVAL;
  AdjBuffers b;
  const int nck = (nsteps + checkpoint_every - 1) / checkpoint_every;
  *bytes = adj_layout(c, nck, checkpoint_every, nullptr, b);
  return MHDE_OK;
}

int mhde_energy_adjoint(mhde_ctx* c, int nsteps, int checkpoint_every, void* ws, size_t ws_bytes, double* loss,
                        double* grad_nu, double* grad_nu_m, double* grad_u0, double* grad_B0) {
  if (!c) return MHDE_EINVAL;
  if (!c->bound || !c->have_initial) return adj_fail(c, MHDE_ESTATE, "context not bound or no initial state");
  if (nsteps < 0 || checkpoint_every < 1 || !loss) return adj_fail(c, MHDE_EINVAL, "bad nsteps, checkpoint or loss");
  const int C = checkpoint_every, K = nsteps, J = c->J, Jp = c->Jp;
  const int nck = (K + C - 1) / C;
  AdjBuffers b;
  const size_t need = adj_layout(c, nck, C, nullptr, b);
  if (!ws || ws_bytes < need) return adj_fail(c, MHDE_EWORKSPACE, "adjoint workspace missing or too small");
  char* base = reinterpret_cast<char*>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  adj_layout(c, nck, C, base, b);
  std::vector<int> tpos;
  if (!transpose_positions(c->fe.F, tpos)) return adj_fail(c, MHDE_EINVAL, "velocity pattern is not symmetric");
  ACU(cudaMemcpy(b.tpos, tpos.data(), tpos.size() * sizeof(int), cudaMemcpyHostToDevice));
  const size_t vs = (size_t)c->n_rows * Jp;
  const long long steps0 = c->steps;
  const mhde_stats stats0 = c->stats;
  std::vector<bool> prev_ck(std::max(nck, 1), false);
  int rc;
  // forward run with a checkpoint every C steps
  for (int n = 0; n < K; ++n) {
    if (n % C == 0) {
      if ((rc = copy4(c, b.ckpt + (size_t)(n / C) * 4 * vs, true))) return rc;
      prev_ck[n / C] = c->have_prev;
    }
    if ((rc = mhde_step(c))) return rc;
  }
  if ((rc = mhde_energy(c, loss))) return rc;
  const bool prev_fin = c->have_prev;
  const long long steps_fin = c->steps;
  if ((rc = copy4(c, b.fin, true))) return rc;
  // seeds of the final-step energy
  launch_means(c->fe.n2, J, Jp, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w, c->sv);
  launch_energy_seed(c, c->d_mean_v, b.seedV, c->sv);
  launch_energy_seed(c, c->d_mean_w, b.seedW, c->sv);
  ACU(cudaGetLastError());
  ACU(cudaStreamSynchronize(c->sv));
  std::vector<double> g_same(J, 0.0), g_cross(J, 0.0);
  double g_c1 = 0.0;
  for (int sgi = nck - 1; sgi >= 0; --sgi) {
    const int n0 = sgi * C, n1 = std::min(K, n0 + C);
    if ((rc = copy4(c, b.ckpt + (size_t)sgi * 4 * vs, false))) return rc;
    c->have_prev = prev_ck[sgi];
    for (int i = 0; i <= n1 - n0; ++i) {
      if (i > 0 && (rc = mhde_step(c))) return rc;
      ACU(cudaMemcpyAsync(b.seg + (size_t)(2 * i) * vs, c->sub[0].S, vs * sizeof(double), cudaMemcpyDeviceToDevice,
                          c->sv));
      ACU(cudaMemcpyAsync(b.seg + (size_t)(2 * i + 1) * vs, c->sub[1].S, vs * sizeof(double),
                          cudaMemcpyDeviceToDevice, c->sv));
    }
    ACU(cudaStreamSynchronize(c->sv));
    for (int n = n1 - 1; n >= n0; --n) {
      const int i = n - n0;
      const double* Sv = b.seg + (size_t)(2 * i) * vs;
      const double* Sw = Sv + vs;
      const double* Xv = b.seg + (size_t)(2 * i + 2) * vs;
      const double* Xw = Xv + vs;
      if ((rc = reverse_step(c, b, Sv, Sw, Xv, Xw, g_same, g_cross, g_c1))) return rc;
      std::swap(b.seedV, b.lamV);
      std::swap(b.seedW, b.lamW);
    }
  }
  // parameters: same_j = nu'_j + nu'_m,j, cross_j = nu_j - nu_m,j, c1 = (nubar + nubar_m)/2
  double mean_same = 0.0;
  for (int j = 0; j < J; ++j) mean_same += g_same[j];
  mean_same /= J;
  for (int j = 0; j < J; ++j) {
    if (grad_nu) grad_nu[j] = g_same[j] - mean_same + g_cross[j] + g_c1 / (2.0 * J);
    if (grad_nu_m) grad_nu_m[j] = g_same[j] - mean_same - g_cross[j] + g_c1 / (2.0 * J);
  }
  // initial fields: v = u + sqrt(s) B, w = u - sqrt(s) B
  if (grad_u0 || grad_B0) {
    const int n2 = c->fe.n2;
    std::vector<double> lv(2 * (size_t)n2 * Jp), lw(2 * (size_t)n2 * Jp);
    ACU(cudaMemcpy(lv.data(), b.seedV, lv.size() * sizeof(double), cudaMemcpyDeviceToHost));
    ACU(cudaMemcpy(lw.data(), b.seedW, lw.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int j = 0; j < J; ++j)
      for (int a = 0; a < n2; ++a)
        for (int d = 0; d < 2; ++d) {
          const size_t o = ((size_t)(2 * a + d)) * Jp + j;
          const size_t h = ((size_t)j * n2 + a) * 2 + d;
          if (grad_u0) grad_u0[h] = lv[o] + lw[o];
          if (grad_B0) grad_B0[h] = c->rs * (lv[o] - lw[o]);
        }
  }
  // leave the context at the final step, as mhde_advance(nsteps) would
  if ((rc = copy4(c, b.fin, false))) return rc;
  c->have_prev = prev_fin;
  c->steps = steps_fin;
  c->stats = stats0;
  c->stats.steps = steps_fin;
  (void)steps0;
  return MHDE_OK;
}

}  // extern "C"
