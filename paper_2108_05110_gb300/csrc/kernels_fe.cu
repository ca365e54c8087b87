// Finite element kernels of one ensemble time step (Algorithm 1), FP64.
//
// * constant element matrices M, K, B (once, at bind);
// * ensemble means <v>, <w> and the mixing-length field
//   l^2(x_q) = max_j |z'_j(x_q)|^2 at the quadrature points (Section 1);
// * element contributions of the shared matrix
//   F = M/dt + N(<z>) + (nubar + nubar_m)/2 K + K_T(2 mu dt l^2)
//   (left-hand sides of eq. weaknew1 / weaknew2) and their nnz-parallel
//   gather through the element -> nonzero map (no atomics);
// * the batched right-hand sides of eq. weaknew1 / weaknew2.
#include <atomic>
#include <cmath>

#include <cstdlib>

#include "kernels.h"

namespace mhde {

static std::atomic<long long> g_launches{0};
static thread_local bool g_capturing = false;
long long launch_count() { return g_launches.load(); }
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("MHDE_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}
void count_launch(long long n) {
  if (!g_capturing) g_launches += n;
}
void set_capturing(bool on) { g_capturing = on; }

__constant__ double c_lam[NQ][3];
__constant__ double c_w[NQ];
__constant__ double c_phi[NQ][NLOC];
__constant__ double c_dphi[NQ][NLOC][3];

// Radon's 7-point degree-5 rule on the reference triangle (weights sum to
// 1/2): the centroid, then the orbits (1-2a, a, a) and (1-2b, b, b) with
// a = (6 - sqrt 15)/21, b = (6 + sqrt 15)/21 and weights (155 -+ sqrt 15)/2400.
void quad_tables(QuadTables& q) {
  const double r15 = std::sqrt(15.0);
  const double orb[2] = {(6.0 - r15) / 21.0, (6.0 + r15) / 21.0};
  const double wo[2] = {(155.0 - r15) / 2400.0, (155.0 + r15) / 2400.0};
  q.lam[0][0] = q.lam[0][1] = q.lam[0][2] = 1.0 / 3.0;
  q.w[0] = 9.0 / 80.0;
  for (int o = 0; o < 2; ++o)
    for (int p = 0; p < 3; ++p) {
      int idx = 1 + 3 * o + p;
      for (int k = 0; k < 3; ++k) q.lam[idx][k] = (k == p) ? 1.0 - 2.0 * orb[o] : orb[o];
      q.w[idx] = wo[o];
    }
  // P2 Lagrange basis in barycentric coordinates: vertex k: l_k (2 l_k - 1);
  // edge (k0, k1) in the order (0,1), (1,2), (2,0): 4 l_k0 l_k1.
  const int E[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  for (int i = 0; i < NQ; ++i) {
    const double* l = q.lam[i];
    for (int a = 0; a < NLOC; ++a)
      for (int k = 0; k < 3; ++k) q.dphi[i][a][k] = 0.0;
    for (int k = 0; k < 3; ++k) {
      q.phi[i][k] = l[k] * (2.0 * l[k] - 1.0);
      q.dphi[i][k][k] = 4.0 * l[k] - 1.0;
    }
    for (int e = 0; e < 3; ++e) {
      int k0 = E[e][0], k1 = E[e][1];
      q.phi[i][3 + e] = 4.0 * l[k0] * l[k1];
      q.dphi[i][3 + e][k0] = 4.0 * l[k1];
      q.dphi[i][3 + e][k1] = 4.0 * l[k0];
    }
  }
}

cudaError_t upload_quad_tables() {
  QuadTables q;
  quad_tables(q);
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_lam, q.lam, sizeof(q.lam))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_w, q.w, sizeof(q.w))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_phi, q.phi, sizeof(q.phi))) != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_dphi, q.dphi, sizeof(q.dphi));
}

// physical gradients of the 6 P2 basis functions at quadrature point q
__device__ __forceinline__ void p2_grads(const double gl[3][2], int q, double gr[NLOC][2]) {
#pragma unroll
  for (int a = 0; a < NLOC; ++a) {
    gr[a][0] = c_dphi[q][a][0] * gl[0][0] + c_dphi[q][a][1] * gl[1][0] + c_dphi[q][a][2] * gl[2][0];
    gr[a][1] = c_dphi[q][a][0] * gl[0][1] + c_dphi[q][a][1] * gl[1][1] + c_dphi[q][a][2] * gl[2][1];
  }
}

__device__ __forceinline__ void load_geom(const double* geom, int e, double gl[3][2], double& det) {
  const double* g = geom + 8 * (size_t)e;
  gl[0][0] = g[0]; gl[0][1] = g[1];
  gl[1][0] = g[2]; gl[1][1] = g[3];
  gl[2][0] = g[4]; gl[2][1] = g[5];
  det = g[6];
}

// ------------------------------------------------------------ constant matrices
__global__ void k_const_local(int nt, const double* __restrict__ geom, double* __restrict__ Mloc,
                              double* __restrict__ Kloc, double* __restrict__ Bloc) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  double gl[3][2], det;
  load_geom(geom, e, gl, det);
  for (int a = 0; a < NLOC; ++a)
    for (int b = 0; b < NLOC; ++b) {
      double m = 0.0, k = 0.0;
      for (int q = 0; q < NQ; ++q) {
        double gr[NLOC][2];
        p2_grads(gl, q, gr);
        double wq = c_w[q] * det;
        m += wq * c_phi[q][a] * c_phi[q][b];
        k += wq * (gr[a][0] * gr[b][0] + gr[a][1] * gr[b][1]);
      }
      Mloc[36 * (size_t)e + 6 * a + b] = m;
      Kloc[36 * (size_t)e + 6 * a + b] = k;
    }
  // B_ia = -(d phi_a / dx_d, psi_i), psi_i = lambda_i
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < NLOC; ++a) {
      double bx = 0.0, by = 0.0;
      for (int q = 0; q < NQ; ++q) {
        double gr[NLOC][2];
        p2_grads(gl, q, gr);
        double wq = c_w[q] * det;
        bx -= wq * c_lam[q][i] * gr[a][0];
        by -= wq * c_lam[q][i] * gr[a][1];
      }
      Bloc[2 * (18 * (size_t)e + 6 * i + a)] = bx;
      Bloc[2 * (18 * (size_t)e + 6 * i + a) + 1] = by;
    }
}

void launch_const_local(int nt, const double* geom, double* Mloc, double* Kloc, double* Bloc,
                        cudaStream_t st) {
  count_launch();
  k_const_local<<<(nt + 127) / 128, 128, 0, st>>>(nt, geom, Mloc, Kloc, Bloc);
}

__global__ void k_gather_MK(long long nnz, const int* __restrict__ ptr, const int* __restrict__ slot,
                            const double* __restrict__ Mloc, const double* __restrict__ Kloc,
                            double* __restrict__ M, double* __restrict__ K) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  double m = 0.0, kk = 0.0;
  for (int t = ptr[k]; t < ptr[k + 1]; ++t) {
    m += Mloc[slot[t]];
    kk += Kloc[slot[t]];
  }
  M[k] = m;
  K[k] = kk;
}

__global__ void k_gather_B(long long nnz, const int* __restrict__ ptr, const int* __restrict__ slot,
                           const double* __restrict__ Bloc, double* __restrict__ B) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  double bx = 0.0, by = 0.0;
  for (int t = ptr[k]; t < ptr[k + 1]; ++t) {
    bx += Bloc[2 * (size_t)slot[t]];
    by += Bloc[2 * (size_t)slot[t] + 1];
  }
  B[2 * k] = bx;
  B[2 * k + 1] = by;
}

__global__ void k_transpose_pairs(long long nnz, const int* __restrict__ src, const double* __restrict__ B,
                                  double* __restrict__ BT, float* __restrict__ Bf,
                                  float* __restrict__ BTf) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  int s = src[k];
  BT[2 * k] = B[2 * (size_t)s];
  BT[2 * k + 1] = B[2 * (size_t)s + 1];
  BTf[2 * k] = (float)B[2 * (size_t)s];
  BTf[2 * k + 1] = (float)B[2 * (size_t)s + 1];
  Bf[2 * k] = (float)B[2 * k];
  Bf[2 * k + 1] = (float)B[2 * k + 1];
}

void launch_gather_const(const mhde_ctx* c, cudaStream_t st) {
  count_launch(3);
  long long nf = c->F.nnz, nb = c->B.nnz;
  k_gather_MK<<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(nf, c->d_fslot_ptr, c->d_fslot,
                                                             c->d_Mloc, c->d_Kloc, c->d_M, c->d_K);
  k_gather_B<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(nb, c->d_bslot_ptr, c->d_bslot,
                                                            c->d_Bloc, c->B.val);
  k_transpose_pairs<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(nb, c->d_btsrc, c->B.val,
                                                                  c->BT.val, c->B.valf, c->BT.valf);
}

// ------------------------------------------------------------ ensemble mean
// <z>(a, c) = (1/J) sum_j z_j(a, c) for z = v and w; rows 2a + c of the states.
__global__ void k_means(int nrows, int J, int Jp, const double* __restrict__ Sv,
                        const double* __restrict__ Sw, double* __restrict__ mv, double* __restrict__ mw) {
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrows) return;
  const double* a = Sv + (size_t)row * Jp;
  const double* b = Sw + (size_t)row * Jp;
  double sa = 0.0, sb = 0.0;
  for (int j = 0; j < J; ++j) {
    sa += a[j];
    sb += b[j];
  }
  mv[row] = sa / J;
  mw[row] = sb / J;
}

void launch_means(int n2, int J, int Jp, const double* Sv, const double* Sw, double* mv, double* mw,
                  cudaStream_t st) {
  count_launch();
  int nrows = 2 * n2;
  k_means<<<(nrows + 255) / 256, 256, 0, st>>>(nrows, J, Jp, Sv, Sw, mv, mw);
}

// l^2(e, q) = max_j |sum_a phi_a(q) (z_j - <z>)(dof_a)|^2 for z = v and w
__global__ void k_l2(int nt, int J, int Jp, const int* __restrict__ dofs, const double* __restrict__ Sv,
                     const double* __restrict__ Sw, const double* __restrict__ mv,
                     const double* __restrict__ mw, double* __restrict__ l2v, double* __restrict__ l2w) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int field = blockIdx.y;
  if (e >= nt) return;
  const double* S = field == 0 ? Sv : Sw;
  const double* m = field == 0 ? mv : mw;
  double* out = field == 0 ? l2v : l2w;
  int d[NLOC];
  double mean[NLOC][2];
  for (int a = 0; a < NLOC; ++a) {
    d[a] = dofs[6 * (size_t)e + a];
    mean[a][0] = m[2 * (size_t)d[a]];
    mean[a][1] = m[2 * (size_t)d[a] + 1];
  }
  double best[NQ];
  for (int q = 0; q < NQ; ++q) best[q] = 0.0;
  for (int j = 0; j < J; ++j) {
    double z[NLOC][2];
    for (int a = 0; a < NLOC; ++a) {
      z[a][0] = S[(size_t)(2 * d[a]) * Jp + j] - mean[a][0];
      z[a][1] = S[(size_t)(2 * d[a] + 1) * Jp + j] - mean[a][1];
    }
    for (int q = 0; q < NQ; ++q) {
      double zx = 0.0, zy = 0.0;
      for (int a = 0; a < NLOC; ++a) {
        zx += c_phi[q][a] * z[a][0];
        zy += c_phi[q][a] * z[a][1];
      }
      double s = zx * zx + zy * zy;
      best[q] = s > best[q] ? s : best[q];
    }
  }
  for (int q = 0; q < NQ; ++q) out[NQ * (size_t)e + q] = best[q];
}

void launch_l2(int nt, int J, int Jp, const int* dofs, const double* Sv, const double* Sw,
               const double* mv, const double* mw, double* l2v, double* l2w, cudaStream_t st) {
  count_launch();
  dim3 grid((nt + 127) / 128, 2);
  k_l2<<<grid, 128, 0, st>>>(nt, J, Jp, dofs, Sv, Sw, mv, mw, l2v, l2w);
}

// ------------------------------------------------------------ shared matrix F
// Element contribution N(a) + K_T(coef_eddy * l^2) (rows = test functions).
__global__ void k_F_local(int nt, const int* __restrict__ dofs, const double* __restrict__ geom,
                          const double* __restrict__ mconv, const double* __restrict__ l2,
                          double coef_eddy, int conv_form, double* __restrict__ Floc) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  double gl[3][2], det;
  load_geom(geom, e, gl, det);
  double an[NLOC][2];
  for (int a = 0; a < NLOC; ++a) {
    int d = dofs[6 * (size_t)e + a];
    an[a][0] = mconv[2 * (size_t)d];
    an[a][1] = mconv[2 * (size_t)d + 1];
  }
  double loc[36];
#pragma unroll
  for (int t = 0; t < 36; ++t) loc[t] = 0.0;
  for (int q = 0; q < NQ; ++q) {
    double gr[NLOC][2];
    p2_grads(gl, q, gr);
    double wq = c_w[q] * det;
    double ax = 0.0, ay = 0.0;
    for (int a = 0; a < NLOC; ++a) {
      ax += c_phi[q][a] * an[a][0];
      ay += c_phi[q][a] * an[a][1];
    }
    double cq = coef_eddy * l2[NQ * (size_t)e + q];
    double adg[NLOC];
    for (int a = 0; a < NLOC; ++a) adg[a] = ax * gr[a][0] + ay * gr[a][1];
#pragma unroll
    for (int a = 0; a < NLOC; ++a)
#pragma unroll
      for (int b = 0; b < NLOC; ++b) {
        double conv = (conv_form == 0)
                          ? 0.5 * (adg[b] * c_phi[q][a] - adg[a] * c_phi[q][b])
                          : adg[b] * c_phi[q][a];
        loc[6 * a + b] += wq * (conv + cq * (gr[a][0] * gr[b][0] + gr[a][1] * gr[b][1]));
      }
  }
#pragma unroll
  for (int t = 0; t < 36; ++t) Floc[36 * (size_t)e + t] = loc[t];
}

void launch_F_local(int nt, const int* dofs, const double* geom, const double* mean_conv,
                    const double* l2, double coef_eddy, int conv_form, double* Floc,
                    cudaStream_t st) {
  count_launch();
  k_F_local<<<(nt + 127) / 128, 128, 0, st>>>(nt, dofs, geom, mean_conv, l2, coef_eddy, conv_form,
                                              Floc);
}

// F[k] = M[k]/dt + nu_hat K[k] + sum of element slots; identity on Dirichlet rows.
__global__ void k_F_gather(int n2, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const int* __restrict__ ptr, const int* __restrict__ slot,
                           const double* __restrict__ Floc, const double* __restrict__ M,
                           const double* __restrict__ K, const unsigned char* __restrict__ isbnd,
                           double inv_dt, double nu_hat, double* __restrict__ F, float* __restrict__ Ff,
                           double* __restrict__ dinv, float* __restrict__ dinvf) {
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= n2) return;
  bool bnd = isbnd[row] != 0;
  for (int k = rowptr[row] + lane; k < rowptr[row + 1]; k += 32) {
    double v;
    if (bnd) {
      v = (col[k] == row) ? 1.0 : 0.0;
    } else {
      double s = 0.0;
      for (int t = ptr[k]; t < ptr[k + 1]; ++t) s += Floc[slot[t]];
      v = M[k] * inv_dt + nu_hat * K[k] + s;
    }
    F[k] = v;
    Ff[k] = (float)v;
    if (col[k] == row) {
      dinv[row] = 1.0 / v;
      dinvf[row] = (float)(1.0 / v);
    }
  }
}

void launch_F_gather(const mhde_ctx* c, const double* Floc, double inv_dt, double nu_hat,
                     double* Fval, float* Fvalf, double* Fdinv, float* Fdinvf, cudaStream_t st) {
  count_launch();
  int n2 = c->fe.n2;
  k_F_gather<<<(n2 + 7) / 8, 256, 0, st>>>(n2, c->F.rowptr, c->F.col, c->d_fslot_ptr, c->d_fslot, Floc,
                                           c->d_M, c->d_K, c->d_isbnd, inv_dt, nu_hat, Fval, Fvalf,
                                           Fdinv, Fdinvf);
}

// FD[k] = F[k] dinv[col[k]] (the inner solve's right-preconditioned operator
// F D^{-1}, formed once per assembly instead of per application); the float
// copy is the product of the float values, as the inner kernels formed it.
__global__ void k_fd_values(long long nnz, const int* __restrict__ col, const double* __restrict__ F,
                            const float* __restrict__ Ff, const double* __restrict__ dinv,
                            const float* __restrict__ dinvf, double* __restrict__ FD, float* __restrict__ FDf) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const int c = col[k];
  FD[k] = F[k] * dinv[c];
  FDf[k] = Ff[k] * dinvf[c];
}

void launch_fd_values(const mhde_ctx* c, Sub& s, cudaStream_t st) {
  count_launch();
  const long long nnz = c->F.nnz;
  k_fd_values<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(nnz, c->F.col, s.Fval, s.Fvalf, s.Fdinv, s.Fdinvf,
                                                             s.FD, s.FDf);
}

// ------------------------------------------------------------ PCD pressure convection
// Element slots [e][3][3]: (a . grad psi_k, psi_i) with psi = lambda (P1).
__global__ void k_Np_local(int nt, const int* __restrict__ dofs, const double* __restrict__ geom,
                           const double* __restrict__ mconv, double* __restrict__ slots) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  double gl[3][2], det;
  load_geom(geom, e, gl, det);
  double an[NLOC][2];
  for (int a = 0; a < NLOC; ++a) {
    int d = dofs[6 * (size_t)e + a];
    an[a][0] = mconv[2 * (size_t)d];
    an[a][1] = mconv[2 * (size_t)d + 1];
  }
  double loc[9];
  for (int t = 0; t < 9; ++t) loc[t] = 0.0;
  for (int q = 0; q < NQ; ++q) {
    double ax = 0.0, ay = 0.0;
    for (int a = 0; a < NLOC; ++a) {
      ax += c_phi[q][a] * an[a][0];
      ay += c_phi[q][a] * an[a][1];
    }
    double wq = c_w[q] * det;
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) loc[3 * i + k] += wq * (ax * gl[k][0] + ay * gl[k][1]) * c_lam[q][i];
  }
  for (int t = 0; t < 9; ++t) slots[9 * (size_t)e + t] = loc[t];
}

__global__ void k_Np_gather(long long nnz, const int* __restrict__ ptr, const int* __restrict__ slot,
                            const double* __restrict__ slots, double* __restrict__ Np, float* __restrict__ Npf) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  double s = 0.0;
  for (int t = ptr[k]; t < ptr[k + 1]; ++t) s += slots[slot[t]];
  Np[k] = s;
  Npf[k] = (float)s;
}

void launch_Np(const mhde_ctx* c, const double* mean_conv, double* slots, double* Np, float* Npf,
               cudaStream_t st) {
  count_launch(2);
  int nt = c->fe.nt;
  long long nnz = c->fe.Kp.nnz();
  k_Np_local<<<(nt + 127) / 128, 128, 0, st>>>(nt, c->d_dofs, c->d_geom, mean_conv, slots);
  k_Np_gather<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(nnz, c->d_p1slot_ptr, c->d_p1slot, slots, Np, Npf);
}

// ------------------------------------------------------------ right-hand sides
// Element vectors of b*(a_j, u_j, phi) for a_j = fluctuation of the other
// field and u_j = member j of this field (skew form 1/2[(a.grad u, phi) -
// (a.grad phi, u)] or standard (a.grad u, phi)), per member:
// Cloc[e][a][c][j].
__global__ void k_rhs_conv_local(int nt, int J, int Jp, const int* __restrict__ dofs,
                                 const double* __restrict__ geom, const double* __restrict__ Sself,
                                 const double* __restrict__ Sother, const double* __restrict__ mother,
                                 int conv_form, double* __restrict__ Cloc) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)nt * J) return;
  int e = (int)(tid / J), j = (int)(tid % J);
  double gl[3][2], det;
  load_geom(geom, e, gl, det);
  double u[NLOC][2], a[NLOC][2];
  for (int t = 0; t < NLOC; ++t) {
    size_t d = (size_t)dofs[6 * (size_t)e + t];
    u[t][0] = Sself[(2 * d) * Jp + j];
    u[t][1] = Sself[(2 * d + 1) * Jp + j];
    a[t][0] = Sother[(2 * d) * Jp + j] - mother[2 * d];
    a[t][1] = Sother[(2 * d + 1) * Jp + j] - mother[2 * d + 1];
  }
  double out[NLOC][2];
  for (int t = 0; t < NLOC; ++t) out[t][0] = out[t][1] = 0.0;
  for (int q = 0; q < NQ; ++q) {
    double gr[NLOC][2];
    p2_grads(gl, q, gr);
    double wq = c_w[q] * det;
    double ax = 0.0, ay = 0.0, ux = 0.0, uy = 0.0;
    double gux = 0.0, guy = 0.0, gvx = 0.0, gvy = 0.0;   // d u_x/dx, d u_x/dy, d u_y/dx, d u_y/dy
    for (int t = 0; t < NLOC; ++t) {
      double p = c_phi[q][t];
      ax += p * a[t][0];
      ay += p * a[t][1];
      ux += p * u[t][0];
      uy += p * u[t][1];
      gux += u[t][0] * gr[t][0];
      guy += u[t][0] * gr[t][1];
      gvx += u[t][1] * gr[t][0];
      gvy += u[t][1] * gr[t][1];
    }
    double adu0 = ax * gux + ay * guy;      // (a . grad) u, component x
    double adu1 = ax * gvx + ay * gvy;      // component y
    for (int t = 0; t < NLOC; ++t) {
      double p = c_phi[q][t];
      if (conv_form == 0) {
        double adp = ax * gr[t][0] + ay * gr[t][1];
        out[t][0] += wq * 0.5 * (adu0 * p - adp * ux);
        out[t][1] += wq * 0.5 * (adu1 * p - adp * uy);
      } else {
        out[t][0] += wq * adu0 * p;
        out[t][1] += wq * adu1 * p;
      }
    }
  }
  for (int t = 0; t < NLOC; ++t) {
    size_t base = ((size_t)(6 * (size_t)e + t) * 2) * Jp + j;
    Cloc[base] = out[t][0];
    Cloc[base + Jp] = out[t][1];
  }
}

void launch_rhs_conv_local(int nt, int J, int Jp, const int* dofs, const double* geom,
                           const double* S_self, const double* S_other, const double* mean_other,
                           int conv_form, double* Cloc, cudaStream_t st) {
  count_launch();
  long long n = (long long)nt * J;
  k_rhs_conv_local<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(nt, J, Jp, dofs, geom, S_self, S_other,
                                                                mean_other, conv_form, Cloc);
}

// b_j(a, c) = sum_k M_ak (f_j + z_j/dt)(k, c) - K_ak (c_cross_j y_j + c_same_j z_j)(k, c) / 2
//             - sum over element slots of node a of Cloc;
// Dirichlet rows take the boundary values, pressure rows are zero.
__global__ void k_rhs_assemble(int n2, int np, int J, int Jp, const int* __restrict__ rowptr,
                               const int* __restrict__ col, const double* __restrict__ M,
                               const double* __restrict__ K, double inv_dt,
                               const double* __restrict__ Sself, const double* __restrict__ Sother,
                               const double* __restrict__ Fz, const int* __restrict__ node_ptr,
                               const int* __restrict__ node_slot, const double* __restrict__ Cloc,
                               const unsigned char* __restrict__ isbnd, const int* __restrict__ bidx,
                               const double* __restrict__ G, const double* __restrict__ ccross,
                               const double* __restrict__ csame, double* __restrict__ Bv) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nvel = (long long)2 * n2 * Jp;
  if (tid >= nvel + (long long)np * Jp) return;
  if (tid >= nvel) {
    Bv[tid] = 0.0;
    return;
  }
  int j = (int)(tid % Jp);
  int row = (int)(tid / Jp);
  int a = row >> 1, c = row & 1;
  if (j >= J) {
    Bv[tid] = 0.0;
    return;
  }
  if (isbnd[a]) {
    Bv[tid] = G[((size_t)bidx[a] * 2 + c) * Jp + j];
    return;
  }
  double hc = 0.5 * ccross[j], hs = 0.5 * csame[j];
  double s = 0.0;
  for (int k = rowptr[a]; k < rowptr[a + 1]; ++k) {
    size_t x = ((size_t)col[k] * 2 + c) * Jp + j;
    double z = Sself[x];
    double mz = (Fz ? Fz[x] : 0.0) + z * inv_dt;
    s += M[k] * mz - K[k] * (hc * Sother[x] + hs * z);
  }
  for (int t = node_ptr[a]; t < node_ptr[a + 1]; ++t)
    s -= Cloc[((size_t)node_slot[t] * 2 + c) * Jp + j];
  Bv[tid] = s;
}

void launch_rhs_assemble(const mhde_ctx* c, const double* S_self, const double* S_other,
                         const double* Fz, const double* G, const double* Cloc,
                         const double* c_cross, const double* c_same, double* Bv, cudaStream_t st) {
  count_launch();
  long long n = (long long)c->n_rows * c->Jp;
  k_rhs_assemble<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      c->fe.n2, c->fe.np, c->J, c->Jp, c->F.rowptr, c->F.col, c->d_M, c->d_K, 1.0 / c->dt, S_self,
      S_other, Fz, c->d_node_ptr, c->d_node_slot, Cloc, c->d_isbnd, c->d_bnd, G, c_cross, c_same,
      Bv);
}

}  // namespace mhde
