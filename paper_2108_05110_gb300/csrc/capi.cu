// C ABI of libmhde (declared in include/mhde.h): context life cycle,
// workspace layout, input conversion to Elsaesser variables (Section 1),
// the time step of Algorithm 1 on two streams, read-outs and parity probes.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <thread>

#include "kernels.h"

using namespace mhde;

namespace {

int fail(mhde_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CU(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(c, MHDE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

struct Carver {
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

size_t ksize(const mhde_ctx* c) { return c->opt.precision == MHDE_PREC_FP64 ? 8 : 4; }

// Assigns every device pointer inside the workspace (base may be nullptr to
// measure).  Returns the total bytes.
size_t layout(mhde_ctx* c, char* base) {
  Carver w{base};
  const FeHost& fe = c->fe;
  const size_t nt = fe.nt, n2 = fe.n2, np = fe.np, Jp = c->Jp;
  const size_t nf = fe.F.nnz(), nb = fe.B.nnz();
  const size_t vs = (size_t)c->n_rows * Jp;
  const int m = c->opt.restart;
  c->d_dofs = w.take<int>(nt * 6);
  c->d_geom = w.take<double>(nt * 8);
  c->d_isbnd = w.take<unsigned char>(n2);
  c->d_bnd = w.take<int>(n2);
  c->F.nrows = (int)n2;
  c->F.ncols = (int)n2;
  c->F.nnz = (long long)nf;
  c->F.rowptr = w.take<int>(n2 + 1);
  c->F.col = w.take<int>(nf);
  c->d_fslot_ptr = w.take<int>(nf + 1);
  c->d_fslot = w.take<int>(nt * 36);
  c->d_fdiag = w.take<int>(n2);
  c->d_M = w.take<double>(nf);
  c->d_K = w.take<double>(nf);
  c->B.nrows = (int)np;
  c->B.ncols = (int)n2;
  c->B.nnz = (long long)nb;
  c->B.rowptr = w.take<int>(np + 1);
  c->B.col = w.take<int>(nb);
  c->B.val = w.take<double>(2 * nb);
  c->B.valf = w.take<float>(2 * nb);
  c->d_bslot_ptr = w.take<int>(nb + 1);
  c->d_bslot = w.take<int>(nt * 18);
  c->BT.nrows = (int)n2;
  c->BT.ncols = (int)np;
  c->BT.nnz = (long long)nb;
  c->BT.rowptr = w.take<int>(n2 + 1);
  c->BT.col = w.take<int>(nb);
  c->BT.val = w.take<double>(2 * nb);
  c->BT.valf = w.take<float>(2 * nb);
  c->d_btsrc = w.take<int>(nb);
  c->d_p1slot_ptr = w.take<int>(fe.p1_gather_ptr.size());
  c->d_p1slot = w.take<int>(fe.p1_gather_slot.size());
  c->d_lsc_dinv = w.take<double>(n2);
  c->d_lsc_dinvf = w.take<float>(n2);
  c->d_node_ptr = w.take<int>(n2 + 1);
  c->d_node_slot = w.take<int>(nt * 6);
  c->d_mp = w.take<double>(np);
  c->d_mpf = w.take<float>(np);
  // AMG operators
  const AmgHost& amg = fe.amg;
  c->amg_ops.assign(amg.levels.size(), DevAmgLevel());
  for (size_t l = 0; l < amg.levels.size(); ++l) {
    const AmgLevelHost& H = amg.levels[l];
    DevAmgLevel& D = c->amg_ops[l];
    D.omega = H.omega;
    auto mk = [&](const HostCsr& A, DevCsr& d, bool diag) {
      d.nrows = A.nrows;
      d.ncols = A.ncols;
      d.nnz = A.nnz();
      d.rowptr = w.take<int>(A.nrows + 1);
      d.col = w.take<int>(A.nnz());
      d.val = w.take<double>(A.nnz());
      d.valf = w.take<float>(A.nnz());
      if (diag) {
        d.dinv = w.take<double>(A.nrows);
        d.dinvf = w.take<float>(A.nrows);
      }
    };
    mk(H.A, D.A, true);
    if (l + 1 < amg.levels.size()) {
      mk(H.P, D.P, false);
      mk(H.R, D.R, false);
      if (H.bs > 0) {
        D.bs = H.bs;
        D.nb = H.A.nrows / H.bs;
        D.blk_omega = H.blk_omega;
        D.blk_idx = w.take<int>(H.blk_idx.size());
        D.blk_inv = w.take<double>(H.blk_inv.size());
        D.blk_invf = w.take<float>(H.blk_inv.size());
      }
    }
  }
  c->d_ig_rows = w.take<int>(IG_PMAX + 1);
  c->d_coarse_inv = w.take<double>((size_t)amg.nc * amg.nc);
  c->d_coarse_invf = w.take<float>((size_t)amg.nc * amg.nc);
  c->d_ccross = w.take<double>(Jp);
  c->d_csame = w.take<double>(Jp);
  // inputs and ensemble quantities
  c->d_F1 = w.take<double>(n2 * 2 * Jp);
  c->d_F2 = w.take<double>(n2 * 2 * Jp);
  c->d_Gv = w.take<double>(fe.bnd_nodes.size() * 2 * Jp + 1);
  c->d_Gw = w.take<double>(fe.bnd_nodes.size() * 2 * Jp + 1);
  c->d_mean_v = w.take<double>(2 * n2);
  c->d_mean_w = w.take<double>(2 * n2);
  c->d_l2_v = w.take<double>(nt * NQ);
  c->d_l2_w = w.take<double>(nt * NQ);
  const size_t ks = ksize(c);
  for (int which = 0; which < 2; ++which) {
    Sub& s = c->sub[which];
    s.which = which;
    s.Fval = w.take<double>(nf);
    s.Fvalf = w.take<float>(nf);
    s.Fdinv = w.take<double>(n2);
    s.Fdinvf = w.take<float>(n2);
    s.FD = w.take<double>(fe.F.nnz());
    s.FDf = w.take<float>(fe.F.nnz());
    s.Floc = w.take<double>(nt * 36);
    s.Cloc = w.take<double>(nt * 6 * 2 * Jp);
    s.Bv = w.take<double>(vs);
    s.X = w.take<double>(vs);
    s.S = w.take<double>(vs);
    s.Sprev = w.take<double>(vs);
    s.Res = w.take<double>(vs);
    s.basis = w.take<char>((size_t)(m + 1) * vs * ks);
    s.Wk = w.take<char>(vs * ks);
    s.Zk = w.take<char>(vs * ks);
    s.Uk = w.take<char>(vs * ks);
    s.Tk = w.take<char>(vs * ks);
    s.Pk = w.take<char>(vs * ks);
    s.Rk = w.take<char>(vs * ks);
    s.Dk = w.take<char>(vs * ks);
    s.part = w.take<double>((size_t)c->nchunk * (m + 1) * c->J * c->J);
    s.gram = w.take<double>((size_t)(m + 2) * c->J * c->J);       // m + 1 blocks, then the projected Gram
    s.coef = w.take<char>(4 * (size_t)(m + 1) * c->J * c->J * 8);
    s.colsq = w.take<double>((size_t)c->nchunk * Jp);
    s.dscale = w.take<double>(2 * Jp);
    s.d_err = w.take<int>(1);                 // zeroed with the workspace at bind
    const size_t nnp = c->opt.schur == 1 ? (size_t)fe.Kp.nnz() : 0;   // PCD's pressure convection
    s.Np = w.take<double>(nnp);
    s.Npf = w.take<float>(nnp);
    {
      const int kin = std::max(1, c->opt.inner_iters);
      const size_t C2 = 2 * Jp;
      s.ibasis = w.take<char>((size_t)(kin + 1) * n2 * C2 * ks);
      s.ipart = w.take<double>((size_t)c->nchunk_in * (KIN_MAX + 2) * C2);
      s.idot = w.take<double>((size_t)(KIN_MAX + 2) * C2 * 2);      // doubles, then a float copy
      s.ih = w.take<double>((size_t)(kin + 1) * kin * C2);
      s.ibeta = w.take<double>(4 * C2);                              // beta, 1/norm, float copy of 1/norm
      s.iy = w.take<double>((size_t)kin * C2 * 2);                   // doubles, then a float copy
      s.ibar = w.take<unsigned>(2);                                  // zero between launches
      s.zbasis = w.take<char>((size_t)m * vs * ks);
    }
    s.amg.assign(amg.levels.size(), DevAmgLevel());
    for (size_t l = 0; l < amg.levels.size(); ++l) {
      size_t n = (size_t)amg.levels[l].A.nrows * Jp;
      DevAmgLevel& L = s.amg[l];
      if (ks == 8) {
        L.x = w.take<double>(n);
        L.b = w.take<double>(n);
        L.r = w.take<double>(n);
      } else {
        L.xf = w.take<float>(n);
        L.bf = w.take<float>(n);
        L.rf = w.take<float>(n);
      }
    }
  }
  return w.off + 256;
}

template <class T>
cudaError_t up(T* dst, const std::vector<T>& src, cudaStream_t st) {
  if (src.empty()) return cudaSuccess;
  return cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

// [J][n2][2] host (two fields a, b combined as a + sgn b) -> [n2][2][Jp] rows
void to_rows(const mhde_ctx* c, const double* a, const double* b, double sgn, double* out) {
  const int n2 = c->fe.n2, J = c->J, Jp = c->Jp;
  std::fill(out, out + (size_t)n2 * 2 * Jp, 0.0);
  for (int j = 0; j < J; ++j)
    for (int k = 0; k < n2; ++k)
      for (int d = 0; d < 2; ++d) {
        double v = a ? a[((size_t)j * n2 + k) * 2 + d] : 0.0;
        if (b) v += sgn * b[((size_t)j * n2 + k) * 2 + d];
        out[((size_t)k * 2 + d) * Jp + j] = v;
      }
}

// Block-size autotuner for the chunked saddle SpMM: times CTA sizes 128, 256
// and 512 in the Krylov precision on this context's matrix pattern and member
// width and keeps the fastest.  Every thread computes the same sums in the same
// order whatever the CTA size, so the choice never changes a result bit (a
// resumed run stays bit-identical to an uninterrupted one).  F's values are
// still zero at bind time; the access pattern and traffic are the real ones.
// FP32 block Gram and block combination of the mixed path: the CUDA-core
// and the tensor-core kernels are timed on this context's sizes (restart/2
// basis blocks of the zeroed workspace; values do not change the timing) and
// the timings reported in the stats, but the choice follows the member
// count alone, so that two contexts given the same data always compute the
// same bits: tensor cores for more than 32 members (12.5 FMA per byte at
// J = 50, where they were 4x faster), CUDA cores up to 32.  At J = 20 the
// tensor-core Gram was 1.15x faster, but its split-TF32 products (about
// 2^-21 relative against FP32's 2^-24) feed the Cholesky QR of the
// projected Gram and raised the block iterations per step on the 128 x 128
// cavity ensemble from 328 to 352.  MHDE_GRAM_TC / MHDE_COMB_TC = 0 or 1
// force the choice.
static int autotune_blockops(mhde_ctx* c) {
  c->gram_tc = c->comb_tc = false;
  if (c->opt.precision != MHDE_PREC_MIXED) return MHDE_OK;
  Sub& s = c->sub[0];
  cudaStream_t st = c->sv;
  const size_t vs = (size_t)c->n_rows * c->Jp;
  const int kb = std::max(1, c->opt.restart / 2);
  const float* Vb = (const float*)s.basis;
  float* Wn = (float*)s.basis + (size_t)kb * vs;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(c, MHDE_ECUDA, "cudaEventCreate failed in the block-operation autotuner");
  }
  const long long launches0 = launch_count();
  auto time = [&](auto&& once) -> double {
    once();
    cudaEventRecord(e0, st);
    for (int r = 0; r < 5; ++r) once();
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0;
    return 1000.0 * ms / 5;
  };
  const int nchunk = std::max(1, std::min(1216, (c->n_rows + 63) / 64));
  const size_t cap = (size_t)c->nchunk * (c->opt.restart + 1) * c->J * c->J;
  const int gchunks = (int)std::max<size_t>(1, std::min<size_t>(cap / ((size_t)(kb + 1) * c->J * c->J), nchunk));
  for (int tc = 0; tc < 2; ++tc) {
    c->gram_tuned_us[tc] = time([&] {
      launch_gram<float>(Vb, vs, kb + 1, Wn, c->n_rows, c->Jp, c->J, gchunks, s.part, s.gram, st, false, s.d_err,
                         tc == 1);
    });
    CU(cudaMemsetAsync(s.coef, 0, (size_t)kb * c->J * c->J * sizeof(float), st));
    c->comb_tuned_us[tc] = time([&] {
      launch_block_combine<float>((float*)s.Zk, nullptr, 0.f, Vb, vs, kb, c->J, (const float*)s.coef, c->J, c->n_rows,
                                  c->Jp, c->Jp, st, s.d_err, tc == 1);
    });
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  count_launch(launch_count() - launches0 > 0 ? -(launch_count() - launches0) : 0);   // not part of any step
  if (take_async_error(s.d_err, st) != 0 || cudaGetLastError() != cudaSuccess)
    return fail(c, MHDE_ECUDA, "block-operation autotuner: a kernel failed");
  auto pick = [c](const double us[2], const char* env) {
    if (const char* e = std::getenv(env)) return e[0] == '1' && us[1] > 0.0;
    return us[1] > 0.0 && c->J > 32;
  };
  c->gram_tc = pick(c->gram_tuned_us, "MHDE_GRAM_TC");
  c->comb_tc = pick(c->comb_tuned_us, "MHDE_COMB_TC");
  return MHDE_OK;
}

// Inner GMRES on F of the mixed path: the persistent form (one cooperative
// launch, grid barriers) and the launch chain, timed on this context's
// sizes (subproblem v's buffers and current operator values) for the stats.
// Both compute the same method with the same step count but round
// differently, so the choice is fixed rather than timed (two contexts given
// the same data compute the same bits): the launch chain, which was the
// faster on every workload measured; MHDE_INNER_GRID = 1 selects the
// persistent form, 0 skips it.
int autotune_inner(mhde_ctx* c) {
  c->inner_grid = false;
  c->ig_P = 0;
  c->inner_tuned_us[0] = c->inner_tuned_us[1] = 0.0;
  const char* env = std::getenv("MHDE_INNER_GRID");
  if (c->opt.precision != MHDE_PREC_MIXED || c->opt.inner_iters < 1 || c->opt.inner_fp16 || (env && env[0] == '0'))
    return MHDE_OK;
  std::vector<int> rows;
  const int P = inner_grid_plan(c, rows);
  if (P <= 0) return MHDE_OK;
  Sub& s = c->sub[0];
  cudaStream_t st = c->sv;
  CU(cudaMemcpyAsync(c->d_ig_rows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));
  c->ig_P = P;
  const float* r = (const float*)s.Tk;
  float* z = (float*)s.Pk;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(c, MHDE_ECUDA, "cudaEventCreate failed in the inner-solve autotuner");
  }
  const long long launches0 = launch_count();
  bool launched = true;
  for (int form = 0; form < 2; ++form) {
    c->inner_grid = form == 1;
    auto once = [&]() {
      launch_inner_gmres<float>(c, s, s.FDf, s.Fdinvf, r, z, c->Jp, c->opt.inner_iters, st, false);
    };
    once();
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 5; ++rep) once();
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) launched = false;
    c->inner_tuned_us[form] = 1000.0 * ms / 5;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  count_launch(-(launch_count() - launches0));   // not part of any step
  const int aerr = take_async_error(s.d_err, st);
  if (!launched || aerr != 0 || cudaGetLastError() != cudaSuccess) {
    // the persistent form did not run (or gave up at a barrier): keep the chain
    c->inner_grid = false;
    c->ig_P = 0;
    c->inner_tuned_us[1] = 0.0;
    return MHDE_OK;
  }
  c->inner_grid = env && env[0] == '1';
  return MHDE_OK;
}

int autotune_spmm(mhde_ctx* c) {
  Sub& s = c->sub[0];
  cudaStream_t st = c->sv;
  const bool f32 = c->opt.precision == MHDE_PREC_MIXED;
  const int blocks[3] = {128, 256, 512};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(c, MHDE_ECUDA, "cudaEventCreate failed in the SpMM autotuner");
  }
  auto once = [&]() {
    if (f32)
      launch_saddle_spmm<float>(c, s.Fvalf, c->B.valf, c->BT.valf, (const float*)s.Wk, nullptr, (float*)s.Zk, 0,
                                c->Jp, st);
    else
      launch_saddle_spmm<double>(c, s.Fval, c->B.val, c->BT.val, (const double*)s.Wk, nullptr, (double*)s.Zk, 0,
                                 c->Jp, st);
  };
  double best = 1e30;
  int best_block = 256;
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < 3 && err == cudaSuccess; ++i) {
    c->spmm_block = blocks[i];
    once();
    cudaEventRecord(e0, st);
    for (int r = 0; r < 5; ++r) once();
    cudaEventRecord(e1, st);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    c->spmm_tuned_us[i] = 1000.0 * ms / 5;
    if (err == cudaSuccess && c->spmm_tuned_us[i] < best) {
      best = c->spmm_tuned_us[i];
      best_block = blocks[i];
    }
  }
  c->spmm_block = best_block;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  count_launch(-18);  // tuning launches are not part of any step
  if (err != cudaSuccess) return fail(c, MHDE_ECUDA, std::string("SpMM autotuner: ") + cudaGetErrorString(err));
  return MHDE_OK;
}

int check_ready(mhde_ctx* c, bool need_initial) {
  if (!c) return MHDE_EINVAL;
  if (!c->bound) return fail(c, MHDE_ESTATE, "mhde_bind has not been called");
  if (need_initial && !c->have_initial) return fail(c, MHDE_ESTATE, "mhde_set_initial has not been called");
  return MHDE_OK;
}

}  // namespace

extern "C" {

void mhde_default_options(mhde_options* o) {
  if (!o) return;
  o->mu = 1.0;
  o->conv_form = 0;
  o->precision = MHDE_PREC_MIXED;
  o->rtol = 0.0;                 // resolved by precision at create
  o->inner_rtol = 1e-3;
  o->restart = 30;
  o->max_iter = 2000;
  o->max_refine = 60;
  o->jacobi_sweeps = 3;
  o->jacobi_omega = 0.3;
  o->amg_sweeps = 1;
  o->amg_cycles = 1;
  o->inner_iters = 6;
  o->schur = 1;
  o->strict = 0;
  o->inner_fp16 = 0;
  o->element = 0;
}

int mhde_create(const mhde_mesh* mesh, int J, const double* nu, const double* nu_m, double s, double dt,
                const mhde_options* opt, mhde_ctx** out) {
  if (!out) return MHDE_EINVAL;
  *out = nullptr;
  if (J < 1 || J > MAX_J || !nu || !nu_m || !(dt > 0.0) || !(s >= 0.0) || !mesh) return MHDE_EINVAL;
  mhde_ctx* c = new mhde_ctx();
  if (opt)
    c->opt = *opt;
  else
    mhde_default_options(&c->opt);
  // rtol 0 picks the precision's default: per-step residuals accumulate over
  // a run, and the FP64 path keeps rel L2 <= 1e-10 against the oracle over
  // 100 steps with 1e-13 (1e-12 gave 1.4e-10); the mixed path's 1e-8 holds
  // with 1e-12
  if (c->opt.rtol == 0.0) c->opt.rtol = c->opt.precision == MHDE_PREC_FP64 ? 1e-13 : 1e-12;
  if (c->opt.restart < 1 || c->opt.restart > 200 || c->opt.max_iter < 1 || !(c->opt.rtol > 0) ||
      (c->opt.precision != MHDE_PREC_FP64 && c->opt.precision != MHDE_PREC_MIXED) ||
      (c->opt.conv_form != 0 && c->opt.conv_form != 1) || c->opt.inner_iters < 0 ||
      c->opt.amg_cycles < 1 ||
      c->opt.inner_iters > mhde::KIN_MAX || c->opt.schur < 0 || c->opt.schur > 2 ||
      (c->opt.inner_fp16 != 0 && c->opt.inner_fp16 != 1) ||
      (c->opt.element != 0 && c->opt.element != 1) ||
      (c->opt.element == 1 && c->opt.schur == 1)) {   // PCD needs a continuous pressure
    delete c;
    return MHDE_EINVAL;
  }
  std::string e = build_fe(mesh, c->fe, c->opt.element);
  if (e.empty() && (c->opt.element == 1 || c->opt.schur == 2)) e = build_algebraic_laplacian(c->fe);
  if (e.empty()) e = build_amg(c->fe, 512);
  if (!e.empty()) {
    // keep the message reachable through a NULL-safe path
    delete c;
    return MHDE_EINVAL;
  }
  c->J = J;
  c->Jp = (J + 3) / 4 * 4;
  c->n_rows = 2 * c->fe.n2 + c->fe.np;
  c->s = s;
  c->rs = std::sqrt(s);
  c->dt = dt;
  c->nu.assign(nu, nu + J);
  c->nu_m.assign(nu_m, nu_m + J);
  for (int j = 0; j < J; ++j) {
    if (!(nu[j] > 0.0) || !(nu_m[j] > 0.0)) {
      delete c;
      return MHDE_EINVAL;
    }
    c->nubar += nu[j];
    c->nubar_m += nu_m[j];
  }
  c->nubar /= J;
  c->nubar_m /= J;
  c->c_cross.resize(J);
  c->c_same.resize(J);
  bool stable = c->opt.mu > 0.5;
  for (int j = 0; j < J; ++j) {
    c->c_cross[j] = nu[j] - nu_m[j];
    c->c_same[j] = (nu[j] - c->nubar) + (nu_m[j] - c->nubar_m);
    double alpha = c->nubar + c->nubar_m - std::fabs(c->c_cross[j]) - std::fabs(c->c_same[j]);
    if (!(alpha > 0.0)) stable = false;
  }
  if (!stable && c->opt.strict) {
    delete c;
    return MHDE_ESTAB;
  }
  c->nchunk = std::max(1, std::min(304, (c->n_rows + 255) / 256));
  // rows per partial-sum chunk of the inner dot products (MHDE_INNER_ROWS to experiment)
  int inner_rows = 128;
  if (const char* ir = std::getenv("MHDE_INNER_ROWS")) inner_rows = std::max(16, std::atoi(ir));
  c->nchunk_in = std::max(1, std::min(1024, (c->fe.n2 + inner_rows - 1) / inner_rows));
  const char* se = std::getenv("MHDE_SERIAL");
  c->serial = se && se[0] == '1';
  const char* tr = std::getenv("MHDE_TRACE");
  c->trace = tr && tr[0] == '1';
  const char* gr = std::getenv("MHDE_GRAPHS");
  c->use_graphs = !(gr && gr[0] == '0');
  const char* sv = std::getenv("MHDE_SPMM");
  c->spmm_rows = sv && std::string(sv) == "rows";
  c->spmm_forced = sv && sv[0] != 0;
  c->amg_levels = (int)c->fe.amg.levels.size();
  *out = c;
  return MHDE_OK;
}

int mhde_get_sizes(const mhde_ctx* c, mhde_sizes* z) {
  if (!c || !z) return MHDE_EINVAL;
  z->nv = c->fe.nv;
  z->nt = c->fe.nt;
  z->ne = c->fe.ne;
  z->n2 = c->fe.n2;
  z->np = c->fe.np;
  z->n_rows = c->n_rows;
  z->J = c->J;
  z->J_pad = c->Jp;
  z->nnz_F = c->fe.F.nnz();
  z->nnz_B = c->fe.B.nnz();
  z->nnz_saddle = 2 * z->nnz_F + 4 * z->nnz_B + 1;
  z->n_boundary = (int)c->fe.bnd_nodes.size();
  z->amg_levels = c->amg_levels;
  z->nnz_L = c->fe.Kp.nnz();
  z->smoother_block = c->fe.amg.levels.empty() ? 0 : c->fe.amg.levels[0].bs;
  return MHDE_OK;
}

int mhde_workspace_size(const mhde_ctx* c0, size_t* bytes) {
  if (!c0 || !bytes) return MHDE_EINVAL;
  mhde_ctx* c = const_cast<mhde_ctx*>(c0);
  // measuring does not change the bound pointers
  if (c->bound) {
    *bytes = c->ws_bytes;
    return MHDE_OK;
  }
  *bytes = layout(c, nullptr);
  return MHDE_OK;
}

int mhde_bind(mhde_ctx* c, void* ws, size_t bytes, void* stream_v, void* stream_w) {
  if (!c) return MHDE_EINVAL;
  if (c->bound) return fail(c, MHDE_ESTATE, "context is already bound");
  size_t need = layout(c, nullptr);
  if (!ws || bytes < need) return fail(c, MHDE_EWORKSPACE, "workspace missing or smaller than mhde_workspace_size");
  if (((uintptr_t)ws) & 255) return fail(c, MHDE_EWORKSPACE, "workspace must be 256-byte aligned");
  c->ws = (char*)ws;
  c->ws_bytes = bytes;
  layout(c, c->ws);
  CU(cudaGetDevice(&c->device));
  c->sv = (cudaStream_t)stream_v;
  c->sw = (cudaStream_t)stream_w;
  c->sub[0].stream = c->sv;
  c->sub[1].stream = c->sw;
  CU(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  CU(upload_quad_tables());
  CU(upload_adjoint_tables());
  CU(init_inner_attributes());
  CU(init_inner_grid_attributes());
  CU(init_la_attributes());
  const FeHost& fe = c->fe;
  cudaStream_t st = c->sv;
  CU(cudaMemsetAsync(c->ws, 0, need, st));
  CU(up(c->d_dofs, fe.dofs, st));
  CU(up(c->d_geom, fe.geom, st));
  CU(up(c->d_isbnd, fe.is_bnd, st));
  std::vector<int> bidx(fe.n2, -1);
  for (size_t i = 0; i < fe.bnd_nodes.size(); ++i) bidx[fe.bnd_nodes[i]] = (int)i;
  c->h_bidx = bidx;
  CU(up(c->d_bnd, bidx, st));
  CU(up(c->F.rowptr, fe.F.rowptr, st));
  CU(up(c->F.col, fe.F.col, st));
  CU(up(c->d_fslot_ptr, fe.f_gather_ptr, st));
  CU(up(c->d_fslot, fe.f_gather_slot, st));
  CU(up(c->d_fdiag, fe.f_diag, st));
  CU(up(c->B.rowptr, fe.B.rowptr, st));
  CU(up(c->B.col, fe.B.col, st));
  CU(up(c->d_bslot_ptr, fe.b_gather_ptr, st));
  CU(up(c->d_bslot, fe.b_gather_slot, st));
  CU(up(c->BT.rowptr, fe.BT.rowptr, st));
  CU(up(c->BT.col, fe.BT.col, st));
  CU(up(c->d_btsrc, fe.bt_src, st));
  CU(up(c->d_p1slot_ptr, fe.p1_gather_ptr, st));
  CU(up(c->d_p1slot, fe.p1_gather_slot, st));
  CU(up(c->d_node_ptr, fe.node_ptr, st));
  CU(up(c->d_node_slot, fe.node_slot, st));
  CU(up(c->d_mp, fe.mp_lumped, st));
  {
    std::vector<double> di = fe.lsc_dinv;
    di.resize(fe.n2, 0.0);
    std::vector<float> dif(di.begin(), di.end());
    CU(up(c->d_lsc_dinv, di, st));
    CU(up(c->d_lsc_dinvf, dif, st));
  }
  std::vector<float> mpf(fe.mp_lumped.begin(), fe.mp_lumped.end());
  CU(up(c->d_mpf, mpf, st));
  std::vector<double> cc(c->Jp, 0.0), cs(c->Jp, 0.0);
  for (int j = 0; j < c->J; ++j) {
    cc[j] = c->c_cross[j];
    cs[j] = c->c_same[j];
  }
  CU(up(c->d_ccross, cc, st));
  CU(up(c->d_csame, cs, st));
  // AMG operators
  std::vector<std::vector<float>> keep_f;   // host float copies alive until the sync below
  for (size_t l = 0; l < fe.amg.levels.size(); ++l) {
    const AmgLevelHost& H = fe.amg.levels[l];
    DevAmgLevel& D = c->amg_ops[l];
    auto put = [&](const HostCsr& A, DevCsr& d, const std::vector<double>* dinv) -> cudaError_t {
      cudaError_t e;
      if ((e = up(d.rowptr, A.rowptr, st))) return e;
      if ((e = up(d.col, A.col, st))) return e;
      if ((e = up(d.val, A.val, st))) return e;
      keep_f.emplace_back(A.val.begin(), A.val.end());
      if ((e = up(d.valf, keep_f.back(), st))) return e;
      if (dinv) {
        if ((e = up(d.dinv, *dinv, st))) return e;
        keep_f.emplace_back(dinv->begin(), dinv->end());
        if ((e = up(d.dinvf, keep_f.back(), st))) return e;
      }
      return cudaSuccess;
    };
    CU(put(H.A, D.A, &H.dinv));
    if (l + 1 < fe.amg.levels.size()) {
      CU(put(H.P, D.P, nullptr));
      CU(put(H.R, D.R, nullptr));
      if (D.bs > 0) {
        CU(up(D.blk_idx, H.blk_idx, st));
        CU(up(D.blk_inv, H.blk_inv, st));
        keep_f.emplace_back(H.blk_inv.begin(), H.blk_inv.end());
        CU(up(D.blk_invf, keep_f.back(), st));
      }
    }
  }
  CU(up(c->d_coarse_inv, fe.amg.coarse_inv, st));
  std::vector<float> cif(fe.amg.coarse_inv.begin(), fe.amg.coarse_inv.end());
  CU(up(c->d_coarse_invf, cif, st));
  // constant matrices: element scratch aliases the F slot buffers of the subproblems
  c->d_Mloc = c->sub[0].Floc;
  c->d_Kloc = c->sub[1].Floc;
  c->d_Bloc = c->sub[0].Cloc;
  launch_const_local(fe.nt, c->d_geom, c->d_Mloc, c->d_Kloc, c->d_Bloc, st);
  launch_gather_const(c, st);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  c->h_M.resize(fe.F.nnz());
  CU(cudaMemcpy(c->h_M.data(), c->d_M, sizeof(double) * fe.F.nnz(), cudaMemcpyDeviceToHost));
  // pinned host staging
  const size_t small = (size_t)(c->opt.restart + 2) * c->J * c->J;
  for (int which = 0; which < 2; ++which) {
    Sub& s = c->sub[which];
    CU(cudaMallocHost((void**)&s.hbuf, sizeof(double) * small));
    CU(cudaMallocHost((void**)&s.hcol, sizeof(double) * c->nchunk * c->Jp));
    CU(cudaMallocHost(&s.hcoef, 4 * sizeof(double) * small));
  }
  c->bound = true;
  if (!c->spmm_forced) {
    int rc = autotune_spmm(c);
    if (rc) return rc;
  }
  {
    int rc = autotune_blockops(c);
    if (rc) return rc;
  }
  {
    int rc = autotune_inner(c);
    if (rc) return rc;
  }
  return MHDE_OK;
}

int mhde_p2_nodes(const mhde_ctx* c, double* xy, unsigned char* isb) {
  if (!c) return MHDE_EINVAL;
  if (xy) std::copy(c->fe.node_xy.begin(), c->fe.node_xy.end(), xy);
  if (isb) std::copy(c->fe.is_bnd.begin(), c->fe.is_bnd.end(), isb);
  return MHDE_OK;
}

int mhde_set_initial(mhde_ctx* c, const double* u0, const double* B0) {
  int rc = check_ready(c, false);
  if (rc) return rc;
  if (!u0) return fail(c, MHDE_EINVAL, "u0 is NULL");
  if (B0 && c->s == 0.0) {
    // B does not enter the Elsaesser fields when s = 0
  }
  const size_t vs = (size_t)c->n_rows * c->Jp;
  std::vector<double> buf(vs, 0.0);
  for (int which = 0; which < 2; ++which) {
    std::fill(buf.begin(), buf.end(), 0.0);
    to_rows(c, u0, B0 ? B0 : nullptr, which == 0 ? c->rs : -c->rs, buf.data());
    CU(cudaMemcpy(c->sub[which].S, buf.data(), vs * sizeof(double), cudaMemcpyHostToDevice));
  }
  c->have_initial = true;
  c->have_prev = false;
  c->steps = 0;
  c->stats = mhde_stats();
  return MHDE_OK;
}

int mhde_set_viscosity(mhde_ctx* c, const double* nu, const double* nu_m) {
  if (!c) return MHDE_EINVAL;
  if (!nu || !nu_m) return fail(c, MHDE_EINVAL, "nu or nu_m is NULL");
  const int J = c->J;
  for (int j = 0; j < J; ++j)
    if (!(nu[j] > 0.0) || !(nu_m[j] > 0.0)) return fail(c, MHDE_EINVAL, "viscosities must be positive");
  double nb = 0.0, nbm = 0.0;
  for (int j = 0; j < J; ++j) {
    nb += nu[j];
    nbm += nu_m[j];
  }
  nb /= J;
  nbm /= J;
  std::vector<double> cc(c->Jp, 0.0), cs(c->Jp, 0.0);
  bool stable = c->opt.mu > 0.5;
  for (int j = 0; j < J; ++j) {
    cc[j] = nu[j] - nu_m[j];
    cs[j] = (nu[j] - nb) + (nu_m[j] - nbm);
    if (!(nb + nbm - std::fabs(cc[j]) - std::fabs(cs[j]) > 0.0)) stable = false;
  }
  if (!stable && c->opt.strict) return fail(c, MHDE_ESTAB, "alpha_j <= 0 or mu <= 1/2");
  c->nu.assign(nu, nu + J);
  c->nu_m.assign(nu_m, nu_m + J);
  c->nubar = nb;
  c->nubar_m = nbm;
  for (int j = 0; j < J; ++j) {
    c->c_cross[j] = cc[j];
    c->c_same[j] = cs[j];
  }
  if (c->bound) {
    CU(cudaStreamSynchronize(c->sv));
    CU(cudaStreamSynchronize(c->sw));
    CU(cudaMemcpy(c->d_ccross, cc.data(), cc.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->d_csame, cs.data(), cs.size() * sizeof(double), cudaMemcpyHostToDevice));
    // the captured preconditioner graphs carry (nubar + nubar_m)/2 as a launch argument
    for (int which = 0; which < 2; ++which) {
      for (auto& kv : c->sub[which].prec_graphs) cudaGraphExecDestroy(kv.second.first);
      c->sub[which].prec_graphs.clear();
    }
  }
  return MHDE_OK;
}

int mhde_set_forcing(mhde_ctx* c, const double* f, const double* cg) {
  int rc = check_ready(c, false);
  if (rc) return rc;
  if (!f && !cg) {
    c->have_forcing = false;
    return MHDE_OK;
  }
  const size_t n = (size_t)c->fe.n2 * 2 * c->Jp;
  std::vector<double> buf(n);
  to_rows(c, f, cg, c->rs, buf.data());
  CU(cudaMemcpy(c->d_F1, buf.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  to_rows(c, f, cg, -c->rs, buf.data());
  CU(cudaMemcpy(c->d_F2, buf.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  c->have_forcing = true;
  return MHDE_OK;
}

int mhde_set_dirichlet(mhde_ctx* c, const double* ub, const double* Bb) {
  int rc = check_ready(c, false);
  if (rc) return rc;
  const int nb = (int)c->fe.bnd_nodes.size(), J = c->J, Jp = c->Jp, n2 = c->fe.n2;
  std::vector<double> gv((size_t)nb * 2 * Jp, 0.0), gw((size_t)nb * 2 * Jp, 0.0);
  for (int i = 0; i < nb; ++i) {
    int k = c->fe.bnd_nodes[i];
    for (int j = 0; j < J; ++j)
      for (int d = 0; d < 2; ++d) {
        double u = ub ? ub[((size_t)j * n2 + k) * 2 + d] : 0.0;
        double b = Bb ? Bb[((size_t)j * n2 + k) * 2 + d] : 0.0;
        gv[((size_t)i * 2 + d) * Jp + j] = u + c->rs * b;
        gw[((size_t)i * 2 + d) * Jp + j] = u - c->rs * b;
      }
  }
  if (nb > 0) {
    CU(cudaMemcpy(c->d_Gv, gv.data(), gv.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->d_Gw, gw.data(), gw.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  return MHDE_OK;
}

static int run_sub(mhde_ctx* c, int which) {
  cudaSetDevice(c->device);
  Sub& s = c->sub[which];
  s.err.clear();
  int rc = assemble_sub(c, which);
  if (rc == MHDE_OK) rc = solve_sub(c, which);
  if (rc == MHDE_OK) {
    cudaError_t e = cudaStreamSynchronize(s.stream);
    if (e != cudaSuccess) {
      s.err = std::string("stream: ") + cudaGetErrorString(e);
      rc = MHDE_ECUDA;
    } else if (take_async_error(s.d_err, s.stream) != 0) {
      // a Gram launch gave up waiting for a TMA stage (bounded wait): the
      // solve used incomplete projections, so the step is not accepted
      s.err = "a bounded wait gave up (a block Gram or combination waiting for its shared-memory stage, "
              "or a grid barrier of the inner solve)";
      rc = MHDE_ECUDA;
    }
  }
  s.status = rc;
  return rc;
}

int mhde_step(mhde_ctx* c) {
  int rc = check_ready(c, true);
  if (rc) return rc;
  auto t0 = std::chrono::steady_clock::now();
  const long long launches0 = launch_count();
  // ensemble means and mixing-length fields of both variables (Section 1)
  launch_means(c->fe.n2, c->J, c->Jp, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w, c->sv);
  launch_l2(c->fe.nt, c->J, c->Jp, c->d_dofs, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w,
            c->d_l2_v, c->d_l2_w, c->sv);
  CU(cudaGetLastError());
  CU(cudaEventRecord(c->ev_fork, c->sv));
  CU(cudaStreamWaitEvent(c->sw, c->ev_fork, 0));
  // the two subproblems run concurrently on their own streams (one after the
  // other with MHDE_SERIAL=1, for per-phase timing without interference)
  if (c->serial) {
    run_sub(c, 0);
    run_sub(c, 1);
  } else {
    std::thread tw([c]() { run_sub(c, 1); });
    run_sub(c, 0);
    tw.join();
  }
  for (int which = 0; which < 2; ++which) {
    if (c->sub[which].status != MHDE_OK) {
      c->err = std::string(which == 0 ? "v" : "w") + " subproblem: " + c->sub[which].err;
      return c->sub[which].status;
    }
  }
  for (int which = 0; which < 2; ++which) {
    Sub& s = c->sub[which];
    double* old_prev = s.Sprev;
    s.Sprev = s.S;
    s.S = s.X;
    s.X = old_prev;
  }
  c->have_prev = true;
  c->steps++;
  c->stats.steps = c->steps;
  for (int which = 0; which < 2; ++which) {
    c->stats.last_iters[which] = c->sub[which].iters;
    c->stats.last_refine[which] = c->sub[which].refine;
    c->stats.last_relres[which] = c->sub[which].relres;
    c->stats.total_iters += c->sub[which].iters;
  }
  c->stats.launches += launch_count() - launches0;
  c->stats.last_step_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (c->trace) {
    for (int which = 0; which < 2; ++which) {
      Sub& s = c->sub[which];
      std::fprintf(stderr,
                   "[mhde] step %lld sub %d ms: assemble %.2f residual %.2f precond %.2f spmm %.2f cgs %.2f "
                   "normalise %.2f | graphs built %d\n",
                   c->steps, which, s.phase_ms[0], s.phase_ms[1], s.phase_ms[2], s.phase_ms[3], s.phase_ms[4],
                   s.phase_ms[5], s.graphs_built);
      for (double& v : s.phase_ms) v = 0.0;
    }
  }
  return MHDE_OK;
}

int mhde_advance_many(mhde_ctx** ctxs, int count, int nsteps, int nthreads, double* step_ms) {
  if (!ctxs || count < 1 || nsteps < 0 || nthreads < 1) return MHDE_EINVAL;
  for (int i = 0; i < count; ++i) {
    int rc = check_ready(ctxs[i], true);
    if (rc) return rc;
  }
  std::atomic<int> next{0};
  std::vector<int> status(count, MHDE_OK);
  auto worker = [&]() {
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) return;
      cudaSetDevice(ctxs[i]->device);
      for (int n = 0; n < nsteps; ++n) {
        auto t0 = std::chrono::steady_clock::now();
        int rc = mhde_step(ctxs[i]);
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (step_ms) step_ms[(size_t)i * nsteps + n] = ms;
        if (rc) {
          status[i] = rc;
          break;
        }
      }
    }
  };
  std::vector<std::thread> pool;
  const int nt = std::min(nthreads, count);
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (status[i] != MHDE_OK) return status[i];
  return MHDE_OK;
}

int mhde_advance(mhde_ctx* c, int nsteps) {
  if (nsteps < 0) return fail(c, MHDE_EINVAL, "nsteps < 0");
  for (int i = 0; i < nsteps; ++i) {
    int rc = mhde_step(c);
    if (rc) return rc;
  }
  return MHDE_OK;
}

int mhde_read_mean(mhde_ctx* c, double* u, double* B) {
  int rc = check_ready(c, true);
  if (rc) return rc;
  if (B && c->s == 0.0) return fail(c, MHDE_EINVAL, "B is not recoverable when s = 0");
  const int n2 = c->fe.n2;
  launch_means(n2, c->J, c->Jp, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w, c->sv);
  std::vector<double> mv(2 * (size_t)n2), mw(2 * (size_t)n2);
  CU(cudaMemcpyAsync(mv.data(), c->d_mean_v, mv.size() * sizeof(double), cudaMemcpyDeviceToHost, c->sv));
  CU(cudaMemcpyAsync(mw.data(), c->d_mean_w, mw.size() * sizeof(double), cudaMemcpyDeviceToHost, c->sv));
  CU(cudaStreamSynchronize(c->sv));
  for (size_t i = 0; i < mv.size(); ++i) {
    if (u) u[i] = 0.5 * (mv[i] + mw[i]);
    if (B) B[i] = 0.5 * (mv[i] - mw[i]) / c->rs;
  }
  return MHDE_OK;
}

// Reads the states into [J][n2][2] velocity arrays and mean-zero pressures [J][np].
static int read_state_host(mhde_ctx* c, std::vector<double>& v, std::vector<double>& w,
                           std::vector<double>& q, std::vector<double>& r) {
  const int n2 = c->fe.n2, np = c->fe.np, J = c->J, Jp = c->Jp;
  const size_t vs = (size_t)c->n_rows * Jp;
  std::vector<double> buf(vs);
  std::vector<double>* outs[2][2] = {{&v, &q}, {&w, &r}};
  double area = 0.0;
  for (double m : c->fe.mp_lumped) area += m;
  for (int which = 0; which < 2; ++which) {
    CU(cudaMemcpy(buf.data(), c->sub[which].S, vs * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double>& z = *outs[which][0];
    std::vector<double>& p = *outs[which][1];
    z.assign((size_t)J * n2 * 2, 0.0);
    p.assign((size_t)J * np, 0.0);
    for (int j = 0; j < J; ++j) {
      for (int k = 0; k < n2; ++k)
        for (int d = 0; d < 2; ++d) z[((size_t)j * n2 + k) * 2 + d] = buf[((size_t)k * 2 + d) * Jp + j];
      double mean = 0.0;
      for (int i = 0; i < np; ++i) {
        double val = buf[((size_t)2 * n2 + i) * Jp + j];
        p[(size_t)j * np + i] = val;
        mean += c->fe.mp_lumped[i] * val;
      }
      mean /= area;
      for (int i = 0; i < np; ++i) p[(size_t)j * np + i] -= mean;
    }
  }
  return MHDE_OK;
}

int mhde_read_state(mhde_ctx* c, double* v, double* w, double* q, double* r) {
  int rc = check_ready(c, true);
  if (rc) return rc;
  std::vector<double> hv, hw, hq, hr;
  if ((rc = read_state_host(c, hv, hw, hq, hr))) return rc;
  if (v) std::copy(hv.begin(), hv.end(), v);
  if (w) std::copy(hw.begin(), hw.end(), w);
  if (q) std::copy(hq.begin(), hq.end(), q);
  if (r) std::copy(hr.begin(), hr.end(), r);
  return MHDE_OK;
}

int mhde_read_member(mhde_ctx* c, int j, double* u, double* B, double* p, double* lam) {
  int rc = check_ready(c, true);
  if (rc) return rc;
  if (j < 0 || j >= c->J) return fail(c, MHDE_EINVAL, "member index out of range");
  if ((B || lam) && c->s == 0.0) return fail(c, MHDE_EINVAL, "B, lambda are not recoverable when s = 0");
  std::vector<double> hv, hw, hq, hr;
  if ((rc = read_state_host(c, hv, hw, hq, hr))) return rc;
  const int n2 = c->fe.n2, np = c->fe.np;
  for (size_t i = 0; i < (size_t)n2 * 2; ++i) {
    double a = hv[(size_t)j * n2 * 2 + i], b = hw[(size_t)j * n2 * 2 + i];
    if (u) u[i] = 0.5 * (a + b);
    if (B) B[i] = 0.5 * (a - b) / c->rs;
  }
  for (int i = 0; i < np; ++i) {
    double a = hq[(size_t)j * np + i], b = hr[(size_t)j * np + i];
    if (p) p[i] = 0.5 * (a + b);
    if (lam) lam[i] = 0.5 * (a - b) / c->rs;
  }
  return MHDE_OK;
}

int mhde_energy(mhde_ctx* c, double* E) {
  int rc = check_ready(c, true);
  if (rc) return rc;
  if (!E) return fail(c, MHDE_EINVAL, "E is NULL");
  const int n2 = c->fe.n2;
  launch_means(n2, c->J, c->Jp, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w, c->sv);
  std::vector<double> mv(2 * (size_t)n2), mw(2 * (size_t)n2);
  CU(cudaMemcpyAsync(mv.data(), c->d_mean_v, mv.size() * sizeof(double), cudaMemcpyDeviceToHost, c->sv));
  CU(cudaMemcpyAsync(mw.data(), c->d_mean_w, mw.size() * sizeof(double), cudaMemcpyDeviceToHost, c->sv));
  CU(cudaStreamSynchronize(c->sv));
  const HostCsr& F = c->fe.F;
  double e = 0.0;
  for (int r = 0; r < n2; ++r)
    for (int k = F.rowptr[r]; k < F.rowptr[r + 1]; ++k) {
      int col = F.col[k];
      double m = c->h_M[k];
      for (int d = 0; d < 2; ++d) e += m * (mv[2 * r + d] * mv[2 * col + d] + mw[2 * r + d] * mw[2 * col + d]);
    }
  *E = 0.5 * e;
  return MHDE_OK;
}

int mhde_get_stats(const mhde_ctx* c, mhde_stats* st) {
  if (!c || !st) return MHDE_EINVAL;
  *st = c->stats;
  st->spmm_block = c->spmm_block;
  for (int i = 0; i < 3; ++i) st->spmm_tuned_us[i] = c->spmm_tuned_us[i];
  st->gram_tensor_cores = c->gram_tc ? 1 : 0;
  st->combine_tensor_cores = c->comb_tc ? 1 : 0;
  for (int i = 0; i < 2; ++i) {
    st->gram_tuned_us[i] = c->gram_tuned_us[i];
    st->combine_tuned_us[i] = c->comb_tuned_us[i];
    st->inner_tuned_us[i] = c->inner_tuned_us[i];
  }
  st->inner_persistent = c->inner_grid ? 1 : 0;
  return MHDE_OK;
}

int mhde_state_bytes(const mhde_ctx* c, size_t* bytes) {
  if (!c || !bytes) return MHDE_EINVAL;
  *bytes = 2 * sizeof(long long) + 4 * (size_t)c->n_rows * c->Jp * sizeof(double);
  return MHDE_OK;
}

int mhde_save_state(mhde_ctx* c, void* buf) {
  int rc = check_ready(c, true);
  if (rc) return rc;
  if (!buf) return fail(c, MHDE_EINVAL, "buffer is NULL");
  char* p = (char*)buf;
  long long hdr[2] = {c->steps, c->have_prev ? 1 : 0};
  std::memcpy(p, hdr, sizeof(hdr));
  const size_t vs = (size_t)c->n_rows * c->Jp * sizeof(double);
  for (int which = 0; which < 2; ++which) {
    CU(cudaMemcpy(p + sizeof(hdr) + (2 * which) * vs, c->sub[which].S, vs, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(p + sizeof(hdr) + (2 * which + 1) * vs, c->sub[which].Sprev, vs, cudaMemcpyDeviceToHost));
  }
  return MHDE_OK;
}

int mhde_load_state(mhde_ctx* c, const void* buf) {
  int rc = check_ready(c, false);
  if (rc) return rc;
  if (!buf) return fail(c, MHDE_EINVAL, "buffer is NULL");
  const char* p = (const char*)buf;
  long long hdr[2];
  std::memcpy(hdr, p, sizeof(hdr));
  c->steps = hdr[0];
  c->have_prev = hdr[1] != 0;
  const size_t vs = (size_t)c->n_rows * c->Jp * sizeof(double);
  for (int which = 0; which < 2; ++which) {
    CU(cudaMemcpy(c->sub[which].S, p + sizeof(hdr) + (2 * which) * vs, vs, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->sub[which].Sprev, p + sizeof(hdr) + (2 * which + 1) * vs, vs, cudaMemcpyHostToDevice));
  }
  c->have_initial = true;
  c->stats.steps = c->steps;
  return MHDE_OK;
}

const char* mhde_last_error(const mhde_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

void mhde_destroy(mhde_ctx* c) {
  if (!c) return;
  if (c->bound) {
    cudaStreamSynchronize(c->sv);
    cudaStreamSynchronize(c->sw);
    for (int which = 0; which < 2; ++which) {
      for (auto& kv : c->sub[which].prec_graphs) cudaGraphExecDestroy(kv.second.first);
      if (c->sub[which].hbuf) cudaFreeHost(c->sub[which].hbuf);
      if (c->sub[which].hcol) cudaFreeHost(c->sub[which].hcol);
      if (c->sub[which].hcoef) cudaFreeHost(c->sub[which].hcoef);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
  }
  delete c;
}

// ------------------------------------------------------------------ probes
static int prepare_means(mhde_ctx* c) {
  launch_means(c->fe.n2, c->J, c->Jp, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w, c->sv);
  launch_l2(c->fe.nt, c->J, c->Jp, c->d_dofs, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w,
            c->d_l2_v, c->d_l2_w, c->sv);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(c->sv));
  return MHDE_OK;
}

int mhde_probe_mean_l2(mhde_ctx* c, double* mv, double* mw, double* l2v, double* l2w) {
  int rc = check_ready(c, true);
  if (rc) return rc;
  if ((rc = prepare_means(c))) return rc;
  const size_t n2 = c->fe.n2, nt = c->fe.nt;
  if (mv) CU(cudaMemcpy(mv, c->d_mean_v, 2 * n2 * sizeof(double), cudaMemcpyDeviceToHost));
  if (mw) CU(cudaMemcpy(mw, c->d_mean_w, 2 * n2 * sizeof(double), cudaMemcpyDeviceToHost));
  if (l2v) CU(cudaMemcpy(l2v, c->d_l2_v, nt * NQ * sizeof(double), cudaMemcpyDeviceToHost));
  if (l2w) CU(cudaMemcpy(l2w, c->d_l2_w, nt * NQ * sizeof(double), cudaMemcpyDeviceToHost));
  return MHDE_OK;
}

static int probe_assemble(mhde_ctx* c, int which) {
  int rc = check_ready(c, true);
  if (rc) return rc;
  if (which != 0 && which != 1) return fail(c, MHDE_EINVAL, "which must be 0 or 1");
  if ((rc = prepare_means(c))) return rc;
  cudaStream_t keep = c->sub[which].stream;
  c->sub[which].stream = c->sv;
  rc = assemble_sub(c, which);
  c->sub[which].stream = keep;
  if (rc) return fail(c, rc, c->sub[which].err);
  CU(cudaStreamSynchronize(c->sv));
  return MHDE_OK;
}

int mhde_probe_matrix_F(mhde_ctx* c, int which, int* rowptr, int* col, double* val) {
  int rc = probe_assemble(c, which);
  if (rc) return rc;
  const HostCsr& F = c->fe.F;
  if (rowptr) std::copy(F.rowptr.begin(), F.rowptr.end(), rowptr);
  if (col) std::copy(F.col.begin(), F.col.end(), col);
  if (val) CU(cudaMemcpy(val, c->sub[which].Fval, F.nnz() * sizeof(double), cudaMemcpyDeviceToHost));
  return MHDE_OK;
}

int mhde_probe_laplacian(const mhde_ctx* c, int* rowptr, int* col, double* val) {
  if (!c) return MHDE_EINVAL;
  const HostCsr& L = c->fe.Kp;
  if (rowptr) std::copy(L.rowptr.begin(), L.rowptr.end(), rowptr);
  if (col) std::copy(L.col.begin(), L.col.end(), col);
  if (val) std::copy(L.val.begin(), L.val.end(), val);
  return MHDE_OK;
}

int mhde_probe_amg_level(const mhde_ctx* c, int level, long long* counts, double* scal, int* a_rowptr,
                         int* a_col, double* a_val, int* p_rowptr, int* p_col, double* p_val, int* r_rowptr,
                         int* r_col, double* r_val, int* blk_idx, double* blk_inv) {
  if (!c || !counts) return MHDE_EINVAL;
  const auto& levels = c->fe.amg.levels;
  if (level < 0 || level >= (int)levels.size()) return MHDE_EINVAL;
  const AmgLevelHost& L = levels[level];
  counts[0] = L.A.nrows;
  counts[1] = L.A.nnz();
  counts[2] = L.P.nnz();
  counts[3] = L.R.nnz();
  counts[4] = L.bs;
  counts[5] = (long long)levels.size();
  if (scal) {
    scal[0] = L.omega;
    scal[1] = L.blk_omega;
  }
  auto put = [](const HostCsr& M, int* rp, int* col, double* val) {
    if (rp && !M.rowptr.empty()) std::copy(M.rowptr.begin(), M.rowptr.end(), rp);
    if (col) std::copy(M.col.begin(), M.col.end(), col);
    if (val) std::copy(M.val.begin(), M.val.end(), val);
  };
  put(L.A, a_rowptr, a_col, a_val);
  put(L.P, p_rowptr, p_col, p_val);
  put(L.R, r_rowptr, r_col, r_val);
  if (blk_idx) std::copy(L.blk_idx.begin(), L.blk_idx.end(), blk_idx);
  if (blk_inv) std::copy(L.blk_inv.begin(), L.blk_inv.end(), blk_inv);
  return MHDE_OK;
}

int mhde_probe_rhs(mhde_ctx* c, int which, double* rhs) {
  int rc = probe_assemble(c, which);
  if (rc) return rc;
  if (!rhs) return fail(c, MHDE_EINVAL, "rhs is NULL");
  const int n2 = c->fe.n2, J = c->J, Jp = c->Jp;
  std::vector<double> buf((size_t)2 * n2 * Jp);
  CU(cudaMemcpy(buf.data(), c->sub[which].Bv, buf.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int j = 0; j < J; ++j)
    for (int k = 0; k < n2; ++k)
      for (int d = 0; d < 2; ++d) rhs[((size_t)j * n2 + k) * 2 + d] = buf[((size_t)k * 2 + d) * Jp + j];
  return MHDE_OK;
}

int mhde_probe_inner(mhde_ctx* c, int which, int form, const double* R, double* Z) {
  int rc = probe_assemble(c, which);
  if (rc) return rc;
  if (!R || !Z || (form != 0 && form != 1)) return fail(c, MHDE_EINVAL, "R or Z is NULL, or form not 0/1");
  if (c->opt.precision != MHDE_PREC_MIXED || c->opt.inner_iters < 1)
    return fail(c, MHDE_EINVAL, "the inner solve probe needs the mixed path with inner_iters >= 1");
  if (form == 1 && c->ig_P <= 0) return fail(c, MHDE_EINVAL, "the persistent inner solve is not available here");
  const int n2 = c->fe.n2, J = c->J, Jp = c->Jp;
  const size_t nv = (size_t)2 * n2 * Jp;
  std::vector<float> buf(nv, 0.f);
  for (int j = 0; j < J; ++j)
    for (int d = 0; d < 2; ++d)
      for (int k = 0; k < n2; ++k) buf[((size_t)k * 2 + d) * Jp + j] = (float)R[((size_t)j * 2 + d) * n2 + k];
  Sub& s = c->sub[which];
  float* dr = (float*)s.Tk;
  float* dz = (float*)s.Pk;
  CU(cudaStreamSynchronize(c->sv));
  CU(cudaStreamSynchronize(s.stream));
  CU(cudaMemcpy(dr, buf.data(), nv * sizeof(float), cudaMemcpyHostToDevice));
  const bool keep = c->inner_grid;
  c->inner_grid = form == 1;
  launch_inner_gmres<float>(c, s, s.FDf, s.Fdinvf, dr, dz, Jp, c->opt.inner_iters, s.stream, false);
  c->inner_grid = keep;
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s.stream));
  if (take_async_error(s.d_err, s.stream) != 0) return fail(c, MHDE_ECUDA, "inner solve probe: a bounded wait gave up");
  CU(cudaMemcpy(buf.data(), dz, nv * sizeof(float), cudaMemcpyDeviceToHost));
  for (int j = 0; j < J; ++j)
    for (int d = 0; d < 2; ++d)
      for (int k = 0; k < n2; ++k) Z[((size_t)j * 2 + d) * n2 + k] = buf[((size_t)k * 2 + d) * Jp + j];
  return MHDE_OK;
}

int mhde_probe_spmm(mhde_ctx* c, int which, int precision, const double* X, double* Y) {
  int rc = probe_assemble(c, which);
  if (rc) return rc;
  if (!X || !Y) return fail(c, MHDE_EINVAL, "X or Y is NULL");
  const int n2 = c->fe.n2, np = c->fe.np, J = c->J, Jp = c->Jp, nr = c->n_rows;
  const size_t vs = (size_t)nr * Jp;
  std::vector<double> buf(vs, 0.0);
  for (int j = 0; j < J; ++j) {
    const double* x = X + (size_t)j * nr;
    for (int k = 0; k < n2; ++k)
      for (int d = 0; d < 2; ++d) buf[((size_t)k * 2 + d) * Jp + j] = x[(size_t)d * n2 + k];
    for (int i = 0; i < np; ++i) buf[((size_t)2 * n2 + i) * Jp + j] = x[(size_t)2 * n2 + i];
  }
  Sub& s = c->sub[which];
  double* dx = s.Res;   // FP64 scratch: the probe runs outside a step
  double* dy = s.X;
  CU(cudaStreamSynchronize(c->sv));
  CU(cudaMemcpy(dx, buf.data(), vs * sizeof(double), cudaMemcpyHostToDevice));
  if (precision == 0) {
    launch_saddle_spmm<double>(c, s.Fval, c->B.val, c->BT.val, dx, nullptr, dy, 0, c->Jp, c->sv);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->sv));
    CU(cudaMemcpy(buf.data(), dy, vs * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    float* fx = (float*)s.Wk;
    float* fy = (float*)s.Zk;
    if (ksize(c) != 4) {
      // FP64 Krylov buffers are twice as large: reuse them as float storage
    }
    launch_d2f(dx, fx, vs, c->sv);
    launch_saddle_spmm<float>(c, s.Fvalf, c->B.valf, c->BT.valf, fx, nullptr, fy, 0, c->Jp, c->sv);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->sv));
    std::vector<float> fb(vs);
    CU(cudaMemcpy(fb.data(), fy, vs * sizeof(float), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < vs; ++i) buf[i] = fb[i];
  }
  for (int j = 0; j < J; ++j) {
    double* y = Y + (size_t)j * nr;
    for (int k = 0; k < n2; ++k)
      for (int d = 0; d < 2; ++d) y[(size_t)d * n2 + k] = buf[((size_t)k * 2 + d) * Jp + j];
    for (int i = 0; i < np; ++i) y[(size_t)2 * n2 + i] = buf[((size_t)2 * n2 + i) * Jp + j];
  }
  return MHDE_OK;
}

int mhde_time_kernel(mhde_ctx* c, int which, int kernel, int reps, double* ms) {
  int rc = probe_assemble(c, which);
  if (rc) return rc;
  if (!ms || reps < 1 || kernel < 0 || kernel > 9) return fail(c, MHDE_EINVAL, "bad kernel id, reps or ms");
  Sub& s = c->sub[which];
  cudaStream_t st = s.stream;
  const size_t vs = (size_t)c->n_rows * c->Jp;
  CU(cudaStreamSynchronize(c->sv));
  // inputs: the current state as a saddle multi-vector
  double* xd = s.Res;
  double* yd = s.X;
  CU(cudaMemcpyAsync(xd, s.S, vs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const bool fp64 = c->opt.precision == MHDE_PREC_FP64;
  const bool block_input = kernel == 5 || kernel == 6 || kernel == 7 || kernel == 8 || kernel == 9;
  if (kernel == 1 || (!fp64 && block_input)) launch_d2f(xd, (float*)s.Wk, vs, st);
  if (fp64 && block_input)
    CU(cudaMemcpyAsync(s.Wk, xd, vs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const int kb = std::max(1, c->opt.restart / 2);
  if (kernel == 6 || kernel == 7 || kernel == 8) {
    // fill kb basis blocks with copies of the input
    for (int i = 0; i < kb; ++i)
      CU(cudaMemcpyAsync((char*)s.basis + (size_t)i * vs * ksize(c), s.Wk, vs * ksize(c),
                         cudaMemcpyDeviceToDevice, st));
  }
  if (kernel == 7) CU(cudaMemsetAsync(s.coef, 0, (size_t)kb * c->J * c->J * sizeof(double), st));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  auto once = [&]() {
    switch (kernel) {
      case 0:
        launch_saddle_spmm<double>(c, s.Fval, c->B.val, c->BT.val, xd, nullptr, yd, 0, c->Jp, st);
        break;
      case 1:
        launch_saddle_spmm<float>(c, s.Fvalf, c->B.valf, c->BT.valf, (const float*)s.Wk, nullptr,
                                  (float*)s.Zk, 0, c->Jp, st);
        break;
      case 2: {
        const double* mean_conv = which == 0 ? c->d_mean_w : c->d_mean_v;
        const double* l2 = which == 0 ? c->d_l2_w : c->d_l2_v;
        launch_F_local(c->fe.nt, c->d_dofs, c->d_geom, mean_conv, l2, 2.0 * c->opt.mu * c->dt,
                       c->opt.conv_form, s.Floc, st);
        launch_F_gather(c, s.Floc, 1.0 / c->dt, 0.5 * (c->nubar + c->nubar_m), s.Fval, s.Fvalf, s.Fdinv,
                        s.Fdinvf, st);
        launch_fd_values(c, s, st);
        break;
      }
      case 3: {
        const Sub& o = c->sub[1 - which];
        const double* mean_other = which == 0 ? c->d_mean_w : c->d_mean_v;
        launch_rhs_conv_local(c->fe.nt, c->J, c->Jp, c->d_dofs, c->d_geom, s.S, o.S, mean_other,
                              c->opt.conv_form, s.Cloc, st);
        launch_rhs_assemble(c, s.S, o.S, c->have_forcing ? (which == 0 ? c->d_F1 : c->d_F2) : nullptr,
                            which == 0 ? c->d_Gv : c->d_Gw, s.Cloc, c->d_ccross, c->d_csame, s.Bv, st);
        break;
      }
      case 4:
        launch_means(c->fe.n2, c->J, c->Jp, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w, st);
        launch_l2(c->fe.nt, c->J, c->Jp, c->d_dofs, c->sub[0].S, c->sub[1].S, c->d_mean_v, c->d_mean_w,
                  c->d_l2_v, c->d_l2_w, st);
        break;
      case 5:
        precond_apply_any(c, which, s.Wk, s.Zk);
        break;
      case 6:
        gram_any(c, which, s.basis, vs, kb, s.Wk);
        break;
      case 7:
        combine_any(c, which, s.basis, vs, kb, s.Zk);
        break;
      case 8:
        gram_any(c, which, s.basis, vs, kb, s.Wk, false);
        break;
      case 9: {
        // residual b - L x on the finest pressure level (pressure parts of
        // the block input and output)
        const size_t poff = (size_t)2 * c->fe.n2 * c->Jp;
        const DevCsr& L = c->amg_ops[0].A;
        if (fp64)
          launch_csr<double>(L.nrows, L.rowptr, L.col, L.val, nullptr, 0.0, (const double*)s.Wk + poff,
                             (const double*)s.Wk + poff, (double*)s.Zk + poff, 1, c->Jp, st);
        else
          launch_csr<float>(L.nrows, L.rowptr, L.col, L.valf, nullptr, 0.f, (const float*)s.Wk + poff,
                            (const float*)s.Wk + poff, (float*)s.Zk + poff, 1, c->Jp, st);
        break;
      }
    }
  };
  once();
  CU(cudaEventRecord(e0, st));
  for (int i = 0; i < reps; ++i) once();
  CU(cudaEventRecord(e1, st));
  CU(cudaEventSynchronize(e1));
  float t = 0.f;
  CU(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CU(cudaGetLastError());
  *ms = (double)t / reps;
  return MHDE_OK;
}

}  // extern "C"
