// Discrete adjoint of the ensemble step (reverse sweep of Algorithm 1 for
// the final-step energy E_h of Section 4.2), FP64 throughout.
//
// For subproblem z (z = v, other field y = w, and the mirror), member j, the
// step solves A_z(<y>, l_z^2) x_j = b_j with
//   F_z = M/dt + N(<y>) + c1 K + K_T(2 mu dt l_z^2),   l_z^2 = max_k |y'_k|^2,
//   b_j = M f_j + M z_j/dt - N(y'_j) z_j - (cross_j/2) K y_j - (same_j/2) K z_j
// (left- and right-hand sides of eq. weaknew1 / weaknew2).  With yh_j the
// solution of A_z^T yh_j = seed_j (Dirichlet and pinned rows zero), the seed
// of the step's inputs receives yh_j^T (d b_j - dF_z x_j):
//   z_j:  M yh_j/dt - N(y'_j)^T yh_j - (same_j/2) K yh_j
//   y_j:  -(cross_j/2) K yh_j - G(z_j, yh_j) + (1/J) sum_k G(z_k, yh_k)
//         - (1/J) sum_k G(x_k, yh_k) + [eddy term on the member attaining
//         the max, minus its mean over members]
// with G(u, y) = d/da [y^T N(a) u].  The kernels below form these terms; the
// transposed solve reuses the block solver with F's values transposed.
#include "kernels.h"

namespace mhde {

// this file's copy of the degree-5 rule and the P2 basis tables (filled from
// the same host tables as the forward kernels' copy)
__constant__ double a_w[NQ];
__constant__ double a_phi[NQ][NLOC];
__constant__ double a_dphi[NQ][NLOC][3];

cudaError_t upload_adjoint_tables() {
  QuadTables q;
  quad_tables(q);
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(a_w, q.w, sizeof(q.w))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(a_phi, q.phi, sizeof(q.phi))) != cudaSuccess) return e;
  return cudaMemcpyToSymbol(a_dphi, q.dphi, sizeof(q.dphi));
}

namespace {

__device__ __forceinline__ void adj_p2_grads(const double gl[3][2], int q, double gr[NLOC][2]) {
#pragma unroll
  for (int a = 0; a < NLOC; ++a) {
    gr[a][0] = a_dphi[q][a][0] * gl[0][0] + a_dphi[q][a][1] * gl[1][0] + a_dphi[q][a][2] * gl[2][0];
    gr[a][1] = a_dphi[q][a][0] * gl[0][1] + a_dphi[q][a][1] * gl[1][1] + a_dphi[q][a][2] * gl[2][1];
  }
}

inline unsigned nblk_adj(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// F^T on F's own (structurally symmetric) pattern: entry k = (a, r) takes the
// value of entry tpos[k] = (r, a).  The diagonal is unchanged.
__global__ void k_transpose_values(long long nnz, const int* __restrict__ tpos, const double* __restrict__ F,
                                   double* __restrict__ FT, float* __restrict__ FTf) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const double v = F[tpos[k]];
  FT[k] = v;
  FTf[k] = (float)v;
}

__global__ void k_scale_pair(long long n, double s, double* __restrict__ x, float* __restrict__ xf) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  x[k] *= s;
  if (xf) xf[k] = (float)x[k];
}

// Seed of the final-step energy on the velocity rows: (1/J) (M <z>)(a, c) for
// every member; other rows and padding columns zero.
__global__ void k_energy_seed(int n2, int n_rows, int J, int Jp, const int* __restrict__ rowptr,
                              const int* __restrict__ col, const double* __restrict__ M,
                              const double* __restrict__ mean, double* __restrict__ seed) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n_rows) return;
  const int row = (int)tid;
  double s = 0.0;
  if (row < 2 * n2) {
    const int a = row >> 1, c = row & 1;
    for (int k = rowptr[a]; k < rowptr[a + 1]; ++k) s += M[k] * mean[2 * (size_t)col[k] + c];
    s /= J;
  }
  for (int j = 0; j < Jp; ++j) seed[(size_t)row * Jp + j] = (j < J) ? s : 0.0;
}

// Right-hand side of the transposed solve: the seed on the velocity rows of
// unconstrained nodes, zero on Dirichlet rows, pressure rows and padding.
__global__ void k_adj_rhs(int n2, int n_rows, int J, int Jp, const unsigned char* __restrict__ isbnd,
                          const double* __restrict__ seed, double* __restrict__ B) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n_rows * Jp) return;
  const int row = (int)(tid / Jp), j = (int)(tid % Jp);
  double v = 0.0;
  if (row < 2 * n2 && j < J && !isbnd[row >> 1]) v = seed[tid];
  B[tid] = v;
}

// Element part of the contraction, one thread per element, members in turn:
//   slotZ[e,t][c][j] = -(N(y'_j)^T yh_j)_t,c          (seed of z_j)
//   slotY[e,t][c][j] = -G(z_j, yh_j)_t,c             (seed of y'_j)
//   slotM[e,t][c]    = -sum_j G(x_j, yh_j)_t,c        (seed of <y>, before 1/J)
//   kstar[e][q], kap[e][q][c] = w_q (-2 mu dt H(q)) 2 y'_{k*}(q)_c with
//   H(q) = sum_j grad yh_j : grad x_j and k* the member attaining l^2(q).
// yh is read as zero on Dirichlet nodes.
__global__ void k_adj_elem(int nt, int J, int Jp, const int* __restrict__ dofs, const double* __restrict__ geom,
                           const double* __restrict__ Z, const double* __restrict__ Y,
                           const double* __restrict__ meanY, const double* __restrict__ X,
                           const double* __restrict__ Yh, const unsigned char* __restrict__ isbnd,
                           int conv_form, double coef_eddy, double* __restrict__ slotZ,
                           double* __restrict__ slotY, double* __restrict__ slotM, int* __restrict__ kstar,
                           double* __restrict__ kap) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  double gl[3][2];
  const double* g = geom + 8 * (size_t)e;
  gl[0][0] = g[0]; gl[0][1] = g[1];
  gl[1][0] = g[2]; gl[1][1] = g[3];
  gl[2][0] = g[4]; gl[2][1] = g[5];
  const double det = g[6];
  int d[NLOC];
  bool bnd[NLOC];
  double my[NLOC][2];
  for (int t = 0; t < NLOC; ++t) {
    d[t] = dofs[6 * (size_t)e + t];
    bnd[t] = isbnd[d[t]] != 0;
    my[t][0] = meanY[2 * (size_t)d[t]];
    my[t][1] = meanY[2 * (size_t)d[t] + 1];
  }
  double best[NQ], bestv[NQ][2], H[NQ];
  int kb[NQ];
  for (int q = 0; q < NQ; ++q) {
    best[q] = -1.0;
    bestv[q][0] = bestv[q][1] = 0.0;
    H[q] = 0.0;
    kb[q] = 0;
  }
  double sm[NLOC][2];
  for (int t = 0; t < NLOC; ++t) sm[t][0] = sm[t][1] = 0.0;
  const bool skew = conv_form == 0;
  for (int j = 0; j < J; ++j) {
    double z[NLOC][2], yp[NLOC][2], x[NLOC][2], yh[NLOC][2];
    for (int t = 0; t < NLOC; ++t)
      for (int c = 0; c < 2; ++c) {
        const size_t o = (size_t)(2 * d[t] + c) * Jp + j;
        z[t][c] = Z[o];
        yp[t][c] = Y[o] - my[t][c];
        x[t][c] = X[o];
        yh[t][c] = bnd[t] ? 0.0 : Yh[o];
      }
    double oz[NLOC][2], oy[NLOC][2];
    for (int t = 0; t < NLOC; ++t) oz[t][0] = oz[t][1] = oy[t][0] = oy[t][1] = 0.0;
    for (int q = 0; q < NQ; ++q) {
      double gr[NLOC][2];
      adj_p2_grads(gl, q, gr);
      const double wq = a_w[q] * det;
      double a[2] = {0.0, 0.0}, zq[2] = {0.0, 0.0}, yq[2] = {0.0, 0.0};
      double gz[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, gx[2][2] = {{0.0, 0.0}, {0.0, 0.0}},
             gy[2][2] = {{0.0, 0.0}, {0.0, 0.0}};      // [component][direction]
      for (int t = 0; t < NLOC; ++t) {
        const double p = a_phi[q][t];
        for (int c = 0; c < 2; ++c) {
          a[c] += p * yp[t][c];
          zq[c] += p * z[t][c];
          yq[c] += p * yh[t][c];
          for (int dd = 0; dd < 2; ++dd) {
            gz[c][dd] += z[t][c] * gr[t][dd];
            gx[c][dd] += x[t][c] * gr[t][dd];
            gy[c][dd] += yh[t][c] * gr[t][dd];
          }
        }
      }
      // eddy coefficient: H(q) and the member attaining max |y'|^2
      H[q] += gy[0][0] * gx[0][0] + gy[0][1] * gx[0][1] + gy[1][0] * gx[1][0] + gy[1][1] * gx[1][1];
      const double l2 = a[0] * a[0] + a[1] * a[1];
      if (l2 > best[q]) {
        best[q] = l2;
        bestv[q][0] = a[0];
        bestv[q][1] = a[1];
        kb[q] = j;
      }
      // (a . grad) yh per component
      const double agy[2] = {a[0] * gy[0][0] + a[1] * gy[0][1], a[0] * gy[1][0] + a[1] * gy[1][1]};
      // G(u, yh) integrand per direction dd: sum_c d_dd u_c yh_c (- d_dd yh_c u_c for skew)
      double gzv[2], gxv[2];
      for (int dd = 0; dd < 2; ++dd) {
        gzv[dd] = gz[0][dd] * yq[0] + gz[1][dd] * yq[1];
        gxv[dd] = 0.0;
      }
      double xq[2] = {0.0, 0.0};
      for (int t = 0; t < NLOC; ++t) {
        xq[0] += a_phi[q][t] * x[t][0];
        xq[1] += a_phi[q][t] * x[t][1];
      }
      for (int dd = 0; dd < 2; ++dd) gxv[dd] = gx[0][dd] * yq[0] + gx[1][dd] * yq[1];
      if (skew) {
        for (int dd = 0; dd < 2; ++dd) {
          gzv[dd] = 0.5 * (gzv[dd] - (gy[0][dd] * zq[0] + gy[1][dd] * zq[1]));
          gxv[dd] = 0.5 * (gxv[dd] - (gy[0][dd] * xq[0] + gy[1][dd] * xq[1]));
        }
      }
      for (int t = 0; t < NLOC; ++t) {
        const double p = a_phi[q][t];
        const double adp = a[0] * gr[t][0] + a[1] * gr[t][1];
        for (int c = 0; c < 2; ++c) {
          // (N(a)^T yh)_t,c: skew 1/2[(a.grad phi_t) yh_c - (a.grad yh_c) phi_t], standard (a.grad phi_t) yh_c
          const double nt_ = skew ? 0.5 * (adp * yq[c] - agy[c] * p) : adp * yq[c];
          oz[t][c] -= wq * nt_;
          oy[t][c] -= wq * p * gzv[c];
          sm[t][c] -= wq * p * gxv[c];
        }
      }
    }
    for (int t = 0; t < NLOC; ++t)
      for (int c = 0; c < 2; ++c) {
        const size_t o = ((size_t)(6 * (size_t)e + t) * 2 + c) * Jp + j;
        slotZ[o] = oz[t][c];
        slotY[o] = oy[t][c];
      }
  }
  for (int t = 0; t < NLOC; ++t)
    for (int c = 0; c < 2; ++c) slotM[(6 * (size_t)e + t) * 2 + c] = sm[t][c];
  for (int q = 0; q < NQ; ++q) {
    const double wq = a_w[q] * det;
    const double s = wq * (-coef_eddy * H[q]) * 2.0;
    kstar[NQ * (size_t)e + q] = kb[q];
    kap[(NQ * (size_t)e + q) * 2] = s * bestv[q][0];
    kap[(NQ * (size_t)e + q) * 2 + 1] = s * bestv[q][1];
  }
}

// Node part, one thread per (velocity row 2a + c, member j):
//   lamZ += M yh/dt - (same_j/2) K yh + gathered slotZ
//   lamY += -(cross_j/2) K yh + py,  py = gathered slotY + eddy term of member j
//   tmp   = py (its mean over members is removed by k_adj_node_mean)
//   prod[0..2] = yh (K z_j), yh (K y_j), yh (K x_j) at this row (parameter partials)
__global__ void k_adj_node(int n2, int J, int Jp, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const double* __restrict__ M, const double* __restrict__ K, double inv_dt,
                           const unsigned char* __restrict__ isbnd, const double* __restrict__ Z,
                           const double* __restrict__ Y, const double* __restrict__ X,
                           const double* __restrict__ Yh, const int* __restrict__ node_ptr,
                           const int* __restrict__ node_slot, const double* __restrict__ slotZ,
                           const double* __restrict__ slotY, const int* __restrict__ kstar,
                           const double* __restrict__ kap, const double* __restrict__ ccross,
                           const double* __restrict__ csame, double* __restrict__ lamZ,
                           double* __restrict__ lamY, double* __restrict__ tmp, double* __restrict__ prod) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nv = (long long)2 * n2 * Jp;
  if (tid >= nv) return;
  const int row = (int)(tid / Jp), j = (int)(tid % Jp);
  const int a = row >> 1, c = row & 1;
  if (j >= J) {
    tmp[tid] = 0.0;
    prod[tid] = prod[nv + tid] = prod[2 * nv + tid] = 0.0;
    return;
  }
  double myh = 0.0, kyh = 0.0, kz = 0.0, ky = 0.0, kx = 0.0;
  for (int k = rowptr[a]; k < rowptr[a + 1]; ++k) {
    const int r = col[k];
    const size_t o = ((size_t)r * 2 + c) * Jp + j;
    const double yh = isbnd[r] ? 0.0 : Yh[o];
    myh += M[k] * yh;
    kyh += K[k] * yh;
    kz += K[k] * Z[o];
    ky += K[k] * Y[o];
    kx += K[k] * X[o];
  }
  double pz = 0.0, py = 0.0;
  for (int t = node_ptr[a]; t < node_ptr[a + 1]; ++t) {
    const int sl = node_slot[t];
    pz += slotZ[((size_t)sl * 2 + c) * Jp + j];
    py += slotY[((size_t)sl * 2 + c) * Jp + j];
    const int e = sl / 6, loc = sl % 6;
    for (int q = 0; q < NQ; ++q)
      if (kstar[NQ * (size_t)e + q] == j) py += kap[(NQ * (size_t)e + q) * 2 + c] * a_phi[q][loc];
  }
  lamZ[tid] += myh * inv_dt - 0.5 * csame[j] * kyh + pz;
  lamY[tid] += -0.5 * ccross[j] * kyh + py;
  tmp[tid] = py;
  const double yh_here = isbnd[a] ? 0.0 : Yh[tid];
  prod[tid] = yh_here * kz;
  prod[nv + tid] = yh_here * ky;
  prod[2 * nv + tid] = yh_here * kx;
}

// Member-mean parts of the y seed, one thread per velocity row 2a + c:
// lamY_j -= (1/J) sum_k tmp_k, and += (1/J) gathered slotM (matrix convection).
__global__ void k_adj_node_mean(int n2, int J, int Jp, const int* __restrict__ node_ptr,
                                const int* __restrict__ node_slot, const double* __restrict__ slotM,
                                const double* __restrict__ tmp, double* __restrict__ lamY) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= 2 * n2) return;
  const int a = row >> 1, c = row & 1;
  double s = 0.0;
  for (int j = 0; j < J; ++j) s += tmp[(size_t)row * Jp + j];
  double m = 0.0;
  for (int t = node_ptr[a]; t < node_ptr[a + 1]; ++t) m += slotM[(size_t)node_slot[t] * 2 + c];
  const double add = (m - s) / J;
  for (int j = 0; j < J; ++j) lamY[(size_t)row * Jp + j] += add;
}

// Column sums of three [rows][Jp] arrays in fixed-size row chunks:
// part[chunk][a][j] (a = 0..2); the host adds the chunks in order.
__global__ void k_colsum3(int rows, int Jp, int rows_per_chunk, const double* __restrict__ P, long long stride,
                          double* __restrict__ part) {
  const int j = threadIdx.x % Jp, a = threadIdx.x / Jp;
  if (a >= 3) return;
  const int r0 = blockIdx.x * rows_per_chunk, r1 = min(rows, r0 + rows_per_chunk);
  double s = 0.0;
  for (int r = r0; r < r1; ++r) s += P[a * stride + (size_t)r * Jp + j];
  part[((size_t)blockIdx.x * 3 + a) * Jp + j] = s;
}

void launch_transpose_values(long long nnz, const int* tpos, const double* F, double* FT, float* FTf,
                             cudaStream_t st) {
  count_launch();
  k_transpose_values<<<nblk_adj(nnz, 256), 256, 0, st>>>(nnz, tpos, F, FT, FTf);
}

void launch_scale_pair(long long n, double s, double* x, float* xf, cudaStream_t st) {
  count_launch();
  k_scale_pair<<<nblk_adj(n, 256), 256, 0, st>>>(n, s, x, xf);
}

void launch_energy_seed(const mhde_ctx* c, const double* mean, double* seed, cudaStream_t st) {
  count_launch();
  k_energy_seed<<<nblk_adj(c->n_rows, 128), 128, 0, st>>>(c->fe.n2, c->n_rows, c->J, c->Jp, c->F.rowptr,
                                                          c->F.col, c->d_M, mean, seed);
}

void launch_adj_rhs(const mhde_ctx* c, const double* seed, double* B, cudaStream_t st) {
  count_launch();
  long long n = (long long)c->n_rows * c->Jp;
  k_adj_rhs<<<nblk_adj(n, 256), 256, 0, st>>>(c->fe.n2, c->n_rows, c->J, c->Jp, c->d_isbnd, seed, B);
}

void launch_adj_contract(const mhde_ctx* c, const double* Z, const double* Y, const double* meanY,
                         const double* X, const double* Yh, double* slotZ, double* slotY, double* slotM,
                         int* kstar, double* kap, double* lamZ, double* lamY, double* tmp, double* prod,
                         int nchunk, double* part, cudaStream_t st) {
  count_launch(4);
  const int nt = c->fe.nt, n2 = c->fe.n2;
  k_adj_elem<<<nblk_adj(nt, 64), 64, 0, st>>>(nt, c->J, c->Jp, c->d_dofs, c->d_geom, Z, Y, meanY, X, Yh, c->d_isbnd,
                                             c->opt.conv_form, 2.0 * c->opt.mu * c->dt, slotZ, slotY, slotM, kstar,
                                             kap);
  const long long nv = (long long)2 * n2 * c->Jp;
  k_adj_node<<<nblk_adj(nv, 128), 128, 0, st>>>(n2, c->J, c->Jp, c->F.rowptr, c->F.col, c->d_M, c->d_K,
                                               1.0 / c->dt, c->d_isbnd, Z, Y, X, Yh, c->d_node_ptr, c->d_node_slot,
                                               slotZ, slotY, kstar, kap, c->d_ccross, c->d_csame, lamZ, lamY, tmp,
                                               prod);
  k_adj_node_mean<<<nblk_adj(2 * n2, 128), 128, 0, st>>>(n2, c->J, c->Jp, c->d_node_ptr, c->d_node_slot, slotM,
                                                        tmp, lamY);
  const int rows = 2 * n2;
  const int rpc = (rows + nchunk - 1) / nchunk;
  k_colsum3<<<nchunk, 3 * c->Jp, 0, st>>>(rows, c->Jp, rpc, prod, nv, part);
}

}  // namespace mhde
