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
//
// Storage: w (the operator output) is kept in the arithmetic type T; the basis
// v_0..v_{k-1} is kept in a storage type S, either T or, on the FP32 path with
// options.inner_fp16, FP16 scaled by sqrt(n2) (a unit column then has entries
// of order one, well inside FP16's normal range).  Arithmetic is always in T.
// The FP16 basis halves the traffic of the dot, update and final passes and
// of the gathers; on the 128 x 128 cavity ensemble that left the time of an
// application unchanged (the chain of dependent launches sets it), so it is
// an option, not the default.
#include <cmath>

#include <cuda_fp16.h>

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

// four consecutive entries (16-byte aligned for float, 32-byte for double)
__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// basis storage: four consecutive entries of S, returned (or given) in T; the
// FP16 form carries the scale sc (stored = sc * value, isc = 1 / sc)
__device__ __forceinline__ void lds4(const float* p, float, float v[4]) { ld4(p, v); }
__device__ __forceinline__ void lds4(const double* p, double, double v[4]) { ld4(p, v); }
__device__ __forceinline__ void lds4(const __half* p, float isc, float v[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  v[0] = a.x * isc; v[1] = a.y * isc; v[2] = b.x * isc; v[3] = b.y * isc;
}
__device__ __forceinline__ void sts4(float* p, float, const float v[4]) { st4(p, v); }
__device__ __forceinline__ void sts4(double* p, double, const double v[4]) { st4(p, v); }
__device__ __forceinline__ void sts4(__half* p, float sc, const float v[4]) {
  const __half2 a = __floats2half2_rn(v[0] * sc, v[1] * sc), b = __floats2half2_rn(v[2] * sc, v[3] * sc);
  uint2 u;
  u.x = *reinterpret_cast<const unsigned*>(&a);
  u.y = *reinterpret_cast<const unsigned*>(&b);
  *reinterpret_cast<uint2*>(p) = u;
}

// one IVec-wide chunk (index i in chunks) of a basis row, in T
template <typename T, typename S> struct Gather;
template <> struct Gather<float, float> {
  static __device__ __forceinline__ float4 ld(const float* p, size_t i, float) {
    return reinterpret_cast<const float4*>(p)[i];
  }
};
template <> struct Gather<double, double> {
  static __device__ __forceinline__ double2 ld(const double* p, size_t i, double) {
    return reinterpret_cast<const double2*>(p)[i];
  }
};
template <> struct Gather<float, __half> {
  static __device__ __forceinline__ float4 ld(const __half* p, size_t i, float isc) {
    float v[4];
    lds4(p + 4 * i, isc, v);
    return make_float4(v[0], v[1], v[2], v[3]);
  }
};

// w[a][:] = sum_k FD_ak v[col_k][:], FD = F D^{-1} (formed at assembly); two
// nonzeros per iteration keep two gathers in flight
template <typename T, typename S>
__global__ void k_fd_spmm(int n2, int nch, const int* __restrict__ rp, const int* __restrict__ col,
                          const T* __restrict__ FD, const S* __restrict__ v, T isc, T* __restrict__ w) {
  pdl_wait();
  pdl_trigger();
  using V = typename IVec<T>::type;
  using G = Gather<T, S>;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n2 * nch) return;
  int a = (int)(tid / nch), ch = (int)(tid % nch);
  V acc = izero(V());
  int k = rp[a];
  const int e = rp[a + 1];
  for (; k + 1 < e; k += 2) {
    const int c0 = col[k], c1 = col[k + 1];
    const T f0 = FD[k], f1 = FD[k + 1];
    const V x0 = G::ld(v, (size_t)c0 * nch + ch, isc), x1 = G::ld(v, (size_t)c1 * nch + ch, isc);
    ifma(acc, f0, x0);
    ifma(acc, f1, x1);
  }
  if (k < e) ifma(acc, FD[k], G::ld(v, (size_t)col[k] * nch + ch, isc));
  reinterpret_cast<V*>(w)[(size_t)a * nch + ch] = acc;
}

// Partial column dots: part[l][col][chunk] = sum_rows V_l[row][col] w[row][col]
// (l < nl), and part[nl][col][chunk] = sum_rows w^2 when with_norm.  A thread
// owns 4 consecutive columns of a row (one 16-byte load per vector for FP32),
// so many rows are in flight per CTA.
template <typename T, typename S, int NLM>
__global__ void __launch_bounds__(256) k_col_dots(int n_rows, int C, int nl, const S* V, size_t vstride, T isc,
                                                  const T* w, int rows_per_chunk, int with_norm,
                                                  double* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double red[];
  const int C4 = C / 4;
  const int G = blockDim.x / C4;
  const int c4 = threadIdx.x % C4, g = threadIdx.x / C4;
  const int r0 = blockIdx.x * rows_per_chunk, r1 = min(n_rows, r0 + rows_per_chunk);
  // acc[0..NLM-2]: dots with V_l; acc[NLM-1]: ||w||^2
  T acc[NLM][4];
#pragma unroll
  for (int l = 0; l < NLM; ++l)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[l][q] = T(0);
  if (g < G) {
    for (int row = r0 + g; row < r1; row += G) {
      const size_t o = (size_t)row * C + 4 * c4;
      T wv[4];
      ld4(w + o, wv);
#pragma unroll
      for (int l = 0; l < NLM - 1; ++l)
        if (l < nl) {
          T vv[4];
          lds4(V + (size_t)l * vstride + o, isc, vv);
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[l][q] += vv[q] * wv[q];
        }
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[NLM - 1][q] += wv[q] * wv[q];
    }
  }
  // stage every group's partial sums, then one thread per (output, column)
  // adds the G groups in a fixed order (deterministic); the chunk's partial
  // goes to part[(slot C + col) nchunk + chunk], chunk-contiguous so that the
  // reduction over chunks reads coalesced
  const int nout = nl + (with_norm ? 1 : 0);
  float* redf = reinterpret_cast<float*>(red);
  if (g < G) {
#pragma unroll
    for (int l = 0; l < NLM; ++l) {
      const bool active = (l < nl) || (l == NLM - 1 && with_norm);
      if (!active) continue;
      const int slot = (l < nl) ? l : nl;
#pragma unroll
      for (int q = 0; q < 4; ++q) redf[((size_t)slot * G + g) * C + 4 * c4 + q] = (float)acc[l][q];
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nout * C; o += blockDim.x) {
    const int slot = o / C, c = o - slot * C;
    float sum = 0.f;
    for (int h = 0; h < G; ++h) sum += redf[((size_t)slot * G + h) * C + c];
    part[(size_t)o * gridDim.x + blockIdx.x] = (double)sum;
  }
}

// Per-column least squares min || beta e_1 - H y || by Givens rotations
// (one thread; h: the column's (kin+1) x kin Hessenberg matrix, already in
// shared memory; g, yl: shared scratch of KIN_MAX+1 doubles).  y is written
// as doubles, then a float copy; nothing is read back from global memory.
__device__ void col_lsq(int C, int kin, int c, double (*h)[KIN_MAX], double beta, double* g, double* yl,
                        double* __restrict__ y) {
  for (int l = 0; l <= kin; ++l) g[l] = 0.0;
  g[0] = beta;
  for (int i = 0; i < kin; ++i) {
    const double a = h[i][i], b = h[i + 1][i];
    const double rr = sqrt(a * a + b * b);
    const double cs = rr > 0.0 ? a / rr : 1.0, sn = rr > 0.0 ? b / rr : 0.0;
    for (int j = i; j < kin; ++j) {
      const double t1 = h[i][j], t2 = h[i + 1][j];
      h[i][j] = cs * t1 + sn * t2;
      h[i + 1][j] = -sn * t1 + cs * t2;
    }
    const double t1 = g[i], t2 = g[i + 1];
    g[i] = cs * t1 + sn * t2;
    g[i + 1] = -sn * t1 + cs * t2;
  }
  for (int i = kin - 1; i >= 0; --i) {
    double sum = g[i];
    for (int j = i + 1; j < kin; ++j) sum -= h[i][j] * yl[j];
    yl[i] = h[i][i] != 0.0 ? sum / h[i][i] : 0.0;
  }
  float* yf = reinterpret_cast<float*>(y + (size_t)kin * C);
  for (int i = 0; i < kin; ++i) {
    y[(size_t)i * C + c] = yl[i];
    yf[(size_t)i * C + c] = (float)yl[i];
  }
}

// Reduce the partial dots over chunks and update the Hessenberg column i.
// One CTA per column; its threads stride over the chunks and a fixed-shape
// shared-memory tree finishes the sums (deterministic).  mode 0: first
// Gram-Schmidt pass, H[l][i] = h; mode 1: second pass, H[l][i] += h, norm
// from the Pythagorean identity, H[i+1][i] = norm, inv[col] = 1/norm;
// mode 2: initial norms beta[col], inv[col] = 1/beta; mode 3: single pass,
// H[l][i] = h and the norm as in mode 1.  With y given, the launch of the last
// step (i = kin - 1) also solves the column's least-squares problem into y:
// the earlier Hessenberg columns are staged into shared memory by all threads
// while the partial sums are reduced, so the serial part touches no global
// memory it has to wait for.
constexpr int RED_T = 32 * (KIN_MAX + 2);

__global__ void __launch_bounds__(RED_T) k_col_reduce(int nchunk, int C, int nl, int kin,
                                                      const double* __restrict__ part, double* __restrict__ dots,
                                                      int mode, int i, double* __restrict__ H,
                                                      double* __restrict__ beta, double* __restrict__ inv,
                                                      double* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[KIN_MAX + 2];
  __shared__ double lh[KIN_MAX + 1][KIN_MAX];
  __shared__ double lg[KIN_MAX + 1];
  __shared__ double ly[KIN_MAX + 1];
  const int c = blockIdx.x;
  const int nout = nl + ((mode == 1 || mode == 3) ? 1 : 0);
  const bool solve = y && i == kin - 1 && (mode == 1 || mode == 3);
  if (solve) {
    // H as the earlier launches left it (column i too, for the mode-1 sum);
    // entries below the subdiagonal are zero
    for (int e = threadIdx.x; e < (kin + 1) * kin; e += blockDim.x) {
      const int l = e / kin, j = e - l * kin;
      lh[l][j] = (l <= j + 1 && j <= i) ? H[((size_t)l * kin + j) * C + c] : 0.0;
    }
  }
  // every warp takes a share of one output's chunks: warp l sums output
  // l % nout over the chunk slices l / nout, l / nout + wpo, ...; the slices
  // are then added in slice order (a fixed order for given nout)
  __shared__ double shw[RED_T / 32];
  const int lane = threadIdx.x & 31, l = threadIdx.x >> 5;
  const int wpo = nout > 0 ? (RED_T / 32) / nout : 1;
  if (l < nout * wpo) {
    const int ot = l % nout, sl = l / nout;
    double s = 0.0;
    const double* pl = part + ((size_t)ot * C + c) * nchunk;
#pragma unroll 8
    for (int ch = lane + 32 * sl; ch < nchunk; ch += 32 * wpo) s += pl[ch];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) shw[l] = s;
  }
  __syncthreads();
  if (threadIdx.x < nout) {
    double s = 0.0;
    for (int sl = 0; sl < wpo; ++sl) s += shw[sl * nout + threadIdx.x];
    sh[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double ss = 0.0;
  float* dotsf = reinterpret_cast<float*>(dots + (size_t)(KIN_MAX + 2) * C);
  for (int t = 0; t < nl; ++t) {
    const double sv = sh[t];
    dots[(size_t)t * C + c] = sv;
    dotsf[(size_t)t * C + c] = (float)sv;
    ss += sv * sv;
    if (mode == 0 || mode == 3) H[((size_t)t * kin + i) * C + c] = sv;
    if (mode == 1) H[((size_t)t * kin + i) * C + c] += sv;
    if (solve) lh[t][i] = (mode == 3) ? sv : lh[t][i] + sv;
  }
  if (mode == 1 || mode == 3) {
    const double n2v = sh[nl] - ss;
    const double nrm = n2v > 0.0 ? sqrt(n2v) : 0.0;
    H[((size_t)(i + 1) * kin + i) * C + c] = nrm;
    inv[c] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    reinterpret_cast<float*>(inv + C)[c] = (float)inv[c];
    // after the last Arnoldi step, this column's least-squares problem
    if (solve) {
      lh[i + 1][i] = nrm;
      col_lsq(C, kin, c, lh, beta[c], lg, ly, y);
    }
  } else if (mode == 2) {
    const double b = sh[0] > 0.0 ? sqrt(sh[0]) : 0.0;
    beta[c] = b;
    inv[c] = b > 0.0 ? 1.0 / b : 0.0;
    reinterpret_cast<float*>(inv + C)[c] = (float)inv[c];
  }
}

// out[row][col] = (in[row][col] - sum_l V_l[row][col] dots[l][col]) * scale[col]
// (nl may be 0); in is in T, the basis V and out in the storage type S (out
// stored with scale osc); 4 consecutive entries per thread
template <typename T, typename S>
__global__ void k_col_update(int n_rows, int C, int nl, const S* __restrict__ V, size_t vstride, T isc,
                             const T* __restrict__ dots, const T* __restrict__ in, S* __restrict__ out, T osc,
                             const T* __restrict__ scale) {
  pdl_wait();
  pdl_trigger();
  long long t4 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)n_rows * C;
  if (4 * t4 >= n) return;
  const size_t o = (size_t)(4 * t4);
  const int c0 = (int)(o % C);
  T acc[4];
  ld4(in + o, acc);
  for (int l = 0; l < nl; ++l) {
    T vv[4];
    lds4(V + (size_t)l * vstride + o, isc, vv);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] -= vv[q] * dots[(size_t)l * C + c0 + q];
  }
  if (scale)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] *= scale[c0 + q];
  sts4(out + o, osc, acc);
}

// z[row][col] = dinv[row] * sum_l V_l[row][col] y[l][col]; 4 entries per thread
template <typename T, typename S>
__global__ void k_col_final(int n_rows, int C, int kin, const S* __restrict__ V, size_t vstride, T isc,
                            const T* __restrict__ y, const T* __restrict__ dinv, T* __restrict__ z) {
  pdl_wait();
  pdl_trigger();
  long long t4 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)n_rows * C;
  if (4 * t4 >= n) return;
  const size_t o = (size_t)(4 * t4);
  const int c0 = (int)(o % C);
  const int row = (int)(o / C);
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int l = 0; l < kin; ++l) {
    T vv[4];
    lds4(V + (size_t)l * vstride + o, isc, vv);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += vv[q] * y[(size_t)l * C + c0 + q];
  }
  const T d = dinv[row];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] *= d;
  st4(z + o, acc);
}

template <typename T, typename S>
static void col_dots(int nchunk, int threads, size_t shm, cudaStream_t st, int n_rows, int C, int nl, const S* V,
                     size_t vstride, T isc, const T* w, int rows_per_chunk, int with_norm, double* part) {
  if (nl + 1 <= 2)
    launch_pdl(k_col_dots<T, S, 2>, dim3(nchunk), dim3(threads), shm, st, n_rows, C, nl, V, vstride, isc, w,
               rows_per_chunk, with_norm, part);
  else if (nl + 1 <= 4)
    launch_pdl(k_col_dots<T, S, 4>, dim3(nchunk), dim3(threads), shm, st, n_rows, C, nl, V, vstride, isc, w,
               rows_per_chunk, with_norm, part);
  else if (nl + 1 <= 8)
    launch_pdl(k_col_dots<T, S, 8>, dim3(nchunk), dim3(threads), shm, st, n_rows, C, nl, V, vstride, isc, w,
               rows_per_chunk, with_norm, part);
  else if (nl + 1 <= 12)
    launch_pdl(k_col_dots<T, S, 12>, dim3(nchunk), dim3(threads), shm, st, n_rows, C, nl, V, vstride, isc, w,
               rows_per_chunk, with_norm, part);
  else
    launch_pdl(k_col_dots<T, S, KIN_MAX + 2>, dim3(nchunk), dim3(threads), shm, st, n_rows, C, nl, V, vstride, isc, w,
               rows_per_chunk, with_norm, part);
}

template <typename T, typename S>
static cudaError_t dots_attr() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  };
  set((const void*)k_col_dots<T, S, 2>);
  set((const void*)k_col_dots<T, S, 4>);
  set((const void*)k_col_dots<T, S, 8>);
  set((const void*)k_col_dots<T, S, 12>);
  set((const void*)k_col_dots<T, S, KIN_MAX + 2>);
  return e;
}

cudaError_t init_inner_attributes() {
  cudaError_t e = dots_attr<float, float>();
  if (e == cudaSuccess) e = dots_attr<float, __half>();
  if (e == cudaSuccess) e = dots_attr<double, double>();
  return e;
}

// Workspace s.ibasis: w ([n2][C] in T) first, then the basis v_0..v_{kin-1}
// ([n2][C] each in S); both fit the (kin + 1) T-vectors the workspace holds.
template <typename T, typename S>
static void inner_gmres(const mhde_ctx* c, const Sub& s, const T* FDv, const T* dinv, const T* r, T* z, int ld,
                        int kin, cudaStream_t st) {
  const int n2 = c->fe.n2, C = 2 * ld;
  const int nch = C / IVec<T>::W;
  const size_t vstride = (size_t)n2 * C;
  const int nchunk = c->nchunk_in;
  const int rows_per_chunk = (n2 + nchunk - 1) / nchunk;
  const int threads = (256 / (C / 4)) * (C / 4);          // whole row groups of C/4 threads
  const size_t shm = (size_t)(kin + 2) * (threads / (C / 4)) * C * sizeof(float);
  // FP16 basis: stored = sqrt(n2) * value, so unit columns have entries of order one
  const bool half = sizeof(S) < sizeof(T);
  const T sc = half ? (T)std::sqrt((double)n2) : T(1), isc = half ? T(1) / sc : T(1);

  T* w = (T*)s.ibasis;
  S* Vb = reinterpret_cast<S*>((char*)s.ibasis + vstride * sizeof(T));
  const long long nel = (long long)n2 * C;
  const bool f32 = sizeof(T) == 4;
  const T* dotsT = f32 ? (const T*)(s.idot + (size_t)(KIN_MAX + 2) * C) : (const T*)s.idot;
  const T* invT = f32 ? (const T*)(s.ibeta + 2 * C) : (const T*)(s.ibeta + C);
  const T* yT = f32 ? (const T*)(s.iy + (size_t)kin * C) : (const T*)s.iy;
  count_launch(3 + 4 * kin);
  // beta = ||r||, v_0 = r / beta
  col_dots<T, T>(nchunk, threads, shm, st, n2, C, 1, r, 0, T(1), r, rows_per_chunk, 0, s.ipart);
  launch_pdl(k_col_reduce, dim3(C), dim3(RED_T), 0, st, nchunk, C, 1, kin, s.ipart, s.idot, 2, 0, s.ih, s.ibeta,
             s.ibeta + C, nullptr);
  launch_pdl(k_col_update<T, S>, dim3(nb(nel / 4, 256)), dim3(256), 0, st, n2, C, 0, Vb, vstride, isc, dotsT, r, Vb,
             sc, invT);
  for (int i = 0; i < kin; ++i) {
    const S* vi = Vb + (size_t)i * vstride;
    launch_pdl(k_fd_spmm<T, S>, dim3(nb((long long)n2 * nch, 256)), dim3(256), 0, st, n2, nch,
               c->F.rowptr, c->F.col, FDv, vi, isc, w);
    // one classical Gram-Schmidt pass: dots against v_0..v_i and ||w||^2 in a
    // single sweep; the projected norm follows from the Pythagorean identity
    col_dots<T, S>(nchunk, threads, shm, st, n2, C, i + 1, Vb, vstride, isc, w, rows_per_chunk, 1, s.ipart);
    launch_pdl(k_col_reduce, dim3(C), dim3(RED_T), 0, st, nchunk, C, i + 1, kin, s.ipart, s.idot, 3, i, s.ih, s.ibeta,
                                      s.ibeta + C, s.iy);
    // v_{i+1} is needed only by a further step: the final combination uses v_0..v_{kin-1}
    if (i + 1 < kin)
      launch_pdl(k_col_update<T, S>, dim3(nb(nel / 4, 256)), dim3(256), 0, st, n2, C, i + 1, Vb, vstride, isc, dotsT,
                 w, Vb + (size_t)(i + 1) * vstride, sc, invT);
  }
  launch_pdl(k_col_final<T, S>, dim3(nb(nel / 4, 256)), dim3(256), 0, st, n2, C, kin, Vb, vstride, isc, yT, dinv, z);
}

template <typename T>
void launch_inner_gmres(const mhde_ctx* c, const Sub& s, const T* FDv, const T* dinv, const T* r, T* z, int ld,
                        int kin, cudaStream_t st, bool allow_half) {
  if constexpr (sizeof(T) == 4) {
    if (allow_half && c->opt.inner_fp16) {
      inner_gmres<float, __half>(c, s, FDv, dinv, r, z, ld, kin, st);
      return;
    }
    // the persistent form (kernels_inner_grid.cu) where the bind-time
    // autotuner found it faster
    if (c->inner_grid && launch_inner_grid(c, s, FDv, dinv, r, z, ld, kin, st)) return;
  }
  inner_gmres<T, T>(c, s, FDv, dinv, r, z, ld, kin, st);
}

template void launch_inner_gmres<double>(const mhde_ctx*, const Sub&, const double*, const double*,
                                         const double*, double*, int, int, cudaStream_t, bool);
template void launch_inner_gmres<float>(const mhde_ctx*, const Sub&, const float*, const float*, const float*,
                                        float*, int, int, cudaStream_t, bool);

}  // namespace mhde
