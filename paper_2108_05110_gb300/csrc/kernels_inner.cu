// Inner solver of the velocity block F (one matrix for both components and
// all members): per-column GMRES(k) with Jacobi right preconditioning, run
// entirely on the device with a fixed iteration count so that it can sit
// inside the captured preconditioner graph.  The velocity part of a saddle
// multi-vector is [n2][C] with C = 2 J_pad columns (component, member).
//
// One inner iteration i:  w = F D^{-1} v_i;  one classical Gram-Schmidt
// pass against v_0..v_i per column (norm from the Pythagorean identity);
// v_{i+1} = w / ||w||.  After k steps
// the per-column least-squares problems min || beta e_1 - H y || are solved
// by Givens rotations and z = D^{-1} sum_l v_l y_l.
#include <cmath>

#include "kernels.h"

namespace mhde {

template <typename T> struct IVec;
template <> struct IVec<double> { using type = double2; static constexpr int W = 2; };
template <> struct IVec<float> { using type = float4; static constexpr int W = 4; };

__device__ __forceinline__ void ifma(double2& a, double s, const double2& x) {
  a.x = fma(s, x.x, a.x);
  a.y = fma(s, x.y, a.y);
}
__device__ __forceinline__ void ifma(float4& a, float s, const float4& x) {
  a.x = fmaf(s, x.x, a.x);
  a.y = fmaf(s, x.y, a.y);
  a.z = fmaf(s, x.z, a.z);
  a.w = fmaf(s, x.w, a.w);
}
__device__ __forceinline__ double2 izero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float4 izero(float4) { return make_float4(0.f, 0.f, 0.f, 0.f); }

static inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// w[a][:] = sum_k F_ak dinv_k v[col_k][:]
template <typename T>
__global__ void k_fd_spmm(int n2, int nch, const int* __restrict__ rp, const int* __restrict__ col,
                          const T* __restrict__ F, const T* __restrict__ dinv, const T* __restrict__ v,
                          T* __restrict__ w) {
  using V = typename IVec<T>::type;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n2 * nch) return;
  int a = (int)(tid / nch), ch = (int)(tid % nch);
  const V* vv = reinterpret_cast<const V*>(v);
  V acc = izero(V());
  for (int k = rp[a]; k < rp[a + 1]; ++k) {
    int c = col[k];
    ifma(acc, F[k] * dinv[c], vv[(size_t)c * nch + ch]);
  }
  reinterpret_cast<V*>(w)[(size_t)a * nch + ch] = acc;
}

// Partial column dots: part[chunk][l][col] = sum_rows V_l[row][col] w[row][col]
// (l < nl), and part[chunk][nl][col] = sum_rows w^2 when with_norm.
template <typename T>
__global__ void __launch_bounds__(256) k_col_dots(int n_rows, int C, int nl, const T* V, size_t vstride,
                                                  const T* w, int rows_per_chunk, int with_norm,
                                                  double* __restrict__ part) {
  extern __shared__ double red[];
  const int G = blockDim.x / C;
  const int c = threadIdx.x % C, g = threadIdx.x / C;
  const int r0 = blockIdx.x * rows_per_chunk, r1 = min(n_rows, r0 + rows_per_chunk);
  T acc[KIN_MAX + 2];
#pragma unroll
  for (int l = 0; l < KIN_MAX + 2; ++l) acc[l] = T(0);
  if (g < G) {
    for (int row = r0 + g; row < r1; row += G) {
      const size_t o = (size_t)row * C + c;
      const T wv = w[o];
#pragma unroll
      for (int l = 0; l < KIN_MAX + 1; ++l)
        if (l < nl) acc[l] += V[(size_t)l * vstride + o] * wv;
      acc[KIN_MAX + 1] += wv * wv;
    }
  }
#pragma unroll
  for (int l = 0; l < KIN_MAX + 2; ++l) {
    const bool active = (l < nl) || (l == KIN_MAX + 1 && with_norm);   // uniform over the block
    if (!active) continue;
    const int slot = (l < nl) ? l : nl;
    if (g < G) red[g * C + c] = (double)acc[l];
    __syncthreads();
    if (threadIdx.x < C) {
      double sum = 0.0;
      for (int h = 0; h < G; ++h) sum += red[h * C + threadIdx.x];
      part[((size_t)blockIdx.x * (KIN_MAX + 2) + slot) * C + threadIdx.x] = sum;
    }
    __syncthreads();
  }
}

// Reduce the partial dots over chunks and update the Hessenberg column i.
// One CTA per column; its threads stride over the chunks and a fixed-shape
// shared-memory tree finishes the sums (deterministic).  mode 0: first
// Gram-Schmidt pass, H[l][i] = h; mode 1: second pass, H[l][i] += h, norm
// from the Pythagorean identity, H[i+1][i] = norm, inv[col] = 1/norm;
// mode 2: initial norms beta[col], inv[col] = 1/beta; mode 3: single pass,
// H[l][i] = h and the norm as in mode 1.
constexpr int RED_T = 128;

__global__ void __launch_bounds__(RED_T) k_col_reduce(int nchunk, int C, int nl, int kin,
                                                      const double* __restrict__ part, double* __restrict__ dots,
                                                      int mode, int i, double* __restrict__ H,
                                                      double* __restrict__ beta, double* __restrict__ inv) {
  __shared__ double sh[KIN_MAX + 2][RED_T];
  const int c = blockIdx.x;
  const int nout = nl + ((mode == 1 || mode == 3) ? 1 : 0);
  for (int l = 0; l < nout; ++l) {
    double s = 0.0;
    for (int ch = threadIdx.x; ch < nchunk; ch += RED_T) s += part[((size_t)ch * (KIN_MAX + 2) + l) * C + c];
    sh[l][threadIdx.x] = s;
  }
  __syncthreads();
  for (int w = RED_T / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int l = 0; l < nout; ++l) sh[l][threadIdx.x] += sh[l][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double ss = 0.0;
  for (int l = 0; l < nl; ++l) {
    const double s = sh[l][0];
    dots[(size_t)l * C + c] = s;
    ss += s * s;
    if (mode == 0 || mode == 3) H[((size_t)l * kin + i) * C + c] = s;
    if (mode == 1) H[((size_t)l * kin + i) * C + c] += s;
  }
  if (mode == 1 || mode == 3) {
    const double n2v = sh[nl][0] - ss;
    const double nrm = n2v > 0.0 ? sqrt(n2v) : 0.0;
    H[((size_t)(i + 1) * kin + i) * C + c] = nrm;
    inv[c] = nrm > 0.0 ? 1.0 / nrm : 0.0;
  } else if (mode == 2) {
    const double b = sh[0][0] > 0.0 ? sqrt(sh[0][0]) : 0.0;
    beta[c] = b;
    inv[c] = b > 0.0 ? 1.0 / b : 0.0;
  }
}

// out[row][col] = (in[row][col] - sum_l V_l[row][col] dots[l][col]) * scale[col]
// (in and out may alias; nl may be 0)
template <typename T>
__global__ void k_col_update(int n_rows, int C, int nl, const T* V, size_t vstride, const double* __restrict__ dots,
                             const T* in, T* out, const double* __restrict__ scale) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n_rows * C) return;
  const int c = (int)(tid % C);
  T acc = in[tid];
  for (int l = 0; l < nl; ++l) acc -= V[(size_t)l * vstride + tid] * (T)dots[(size_t)l * C + c];
  if (scale) acc *= (T)scale[c];
  out[tid] = acc;
}

// Per-column least squares min || beta e_1 - H y || by Givens rotations.
__global__ void k_col_lsq(int C, int kin, const double* __restrict__ H, const double* __restrict__ beta,
                          double* __restrict__ y) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double h[KIN_MAX + 1][KIN_MAX];
  double g[KIN_MAX + 1];
  for (int l = 0; l <= kin; ++l) {
    g[l] = 0.0;
    for (int i = 0; i < kin; ++i) h[l][i] = (l <= i + 1) ? H[((size_t)l * kin + i) * C + c] : 0.0;
  }
  g[0] = beta[c];
  for (int i = 0; i < kin; ++i) {
    double a = h[i][i], b = h[i + 1][i];
    double r = sqrt(a * a + b * b);
    double cs = r > 0.0 ? a / r : 1.0, sn = r > 0.0 ? b / r : 0.0;
    for (int j = i; j < kin; ++j) {
      double t1 = h[i][j], t2 = h[i + 1][j];
      h[i][j] = cs * t1 + sn * t2;
      h[i + 1][j] = -sn * t1 + cs * t2;
    }
    double t1 = g[i], t2 = g[i + 1];
    g[i] = cs * t1 + sn * t2;
    g[i + 1] = -sn * t1 + cs * t2;
  }
  for (int i = kin - 1; i >= 0; --i) {
    double s = g[i];
    for (int j = i + 1; j < kin; ++j) s -= h[i][j] * y[(size_t)j * C + c];
    y[(size_t)i * C + c] = h[i][i] != 0.0 ? s / h[i][i] : 0.0;
  }
}

// z[row][col] = dinv[row] * sum_l V_l[row][col] y[l][col]
template <typename T>
__global__ void k_col_final(int n_rows, int C, int kin, const T* __restrict__ V, size_t vstride,
                            const double* __restrict__ y, const T* __restrict__ dinv, T* __restrict__ z) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n_rows * C) return;
  const int c = (int)(tid % C);
  const int row = (int)(tid / C);
  T acc = T(0);
  for (int l = 0; l < kin; ++l) acc += V[(size_t)l * vstride + tid] * (T)y[(size_t)l * C + c];
  z[tid] = acc * dinv[row];
}

template <typename T>
void launch_inner_gmres(const mhde_ctx* c, const Sub& s, const T* Fv, const T* dinv, const T* r, T* z, int ld,
                        cudaStream_t st) {
  const int n2 = c->fe.n2, C = 2 * ld, kin = c->opt.inner_iters;
  const int nch = C / IVec<T>::W;
  const size_t vstride = (size_t)n2 * C;
  const int nchunk = c->nchunk_in;
  const int rows_per_chunk = (n2 + nchunk - 1) / nchunk;
  const int threads = (256 / C) * C;
  const size_t shm = (size_t)threads * sizeof(double);
  T* Vb = (T*)s.ibasis;
  const long long nel = (long long)n2 * C;
  count_launch(3 + 4 * kin + 2);
  // beta = ||r||, v_0 = r / beta
  k_col_dots<T><<<nchunk, threads, shm, st>>>(n2, C, 1, r, 0, r, rows_per_chunk, 0, s.ipart);
  k_col_reduce<<<C, RED_T, 0, st>>>(nchunk, C, 1, kin, s.ipart, s.idot, 2, 0, s.ih, s.ibeta,
                                         s.ibeta + C);
  k_col_update<T><<<nb(nel, 256), 256, 0, st>>>(n2, C, 0, Vb, vstride, s.idot, r, Vb, s.ibeta + C);
  for (int i = 0; i < kin; ++i) {
    T* vi = Vb + (size_t)i * vstride;
    T* w = Vb + (size_t)(i + 1) * vstride;
    k_fd_spmm<T><<<nb((long long)n2 * nch, 256), 256, 0, st>>>(n2, nch, c->F.rowptr, c->F.col, Fv, dinv, vi, w);
    // one classical Gram-Schmidt pass: dots against v_0..v_i and ||w||^2 in a
    // single sweep; the projected norm follows from the Pythagorean identity
    k_col_dots<T><<<nchunk, threads, shm, st>>>(n2, C, i + 1, Vb, vstride, w, rows_per_chunk, 1, s.ipart);
    k_col_reduce<<<C, RED_T, 0, st>>>(nchunk, C, i + 1, kin, s.ipart, s.idot, 3, i, s.ih, s.ibeta,
                                      s.ibeta + C);
    k_col_update<T><<<nb(nel, 256), 256, 0, st>>>(n2, C, i + 1, Vb, vstride, s.idot, w, w, s.ibeta + C);
  }
  k_col_lsq<<<nb(C, 64), 64, 0, st>>>(C, kin, s.ih, s.ibeta, s.iy);
  k_col_final<T><<<nb(nel, 256), 256, 0, st>>>(n2, C, kin, Vb, vstride, s.iy, dinv, z);
}

template void launch_inner_gmres<double>(const mhde_ctx*, const Sub&, const double*, const double*,
                                         const double*, double*, int, cudaStream_t);
template void launch_inner_gmres<float>(const mhde_ctx*, const Sub&, const float*, const float*, const float*,
                                        float*, int, cudaStream_t);

}  // namespace mhde
