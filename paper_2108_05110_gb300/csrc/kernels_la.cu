// Linear-algebra kernels of the shared-matrix block solve (Section 1: one
// matrix A for all J right-hand sides, A [x_1 | ... | x_J] = [b_1 | ... | b_J],
// solved with block linear solvers).  Every multi-vector is row-major
// [rows][Jp]; a thread owns one 16-byte chunk of one row (2 doubles or 4
// floats), so the J-wide rows that a sparse row gathers are read as
// contiguous, coalesced vector loads and the matrix values / column indices of
// a row are broadcast to the threads sharing that row.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "kernels.h"

namespace mhde {

template <typename T> struct Vec;
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };

__device__ __forceinline__ double2 vzero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float4 vzero(float4) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void vfma(double2& acc, double s, const double2& x) {
  acc.x = fma(s, x.x, acc.x);
  acc.y = fma(s, x.y, acc.y);
}
__device__ __forceinline__ void vfma(float4& acc, float s, const float4& x) {
  acc.x = fmaf(s, x.x, acc.x);
  acc.y = fmaf(s, x.y, acc.y);
  acc.z = fmaf(s, x.z, acc.z);
  acc.w = fmaf(s, x.w, acc.w);
}
__device__ __forceinline__ double2 vaxpby(double a, const double2& x, double b, const double2& y) {
  return make_double2(a * x.x + b * y.x, a * x.y + b * y.y);
}
__device__ __forceinline__ float4 vaxpby(float a, const float4& x, float b, const float4& y) {
  return make_float4(a * x.x + b * y.x, a * x.y + b * y.y, a * x.z + b * y.z, a * x.w + b * y.w);
}

// four consecutive entries of a row (16-byte aligned for float, 32-byte for double)
__device__ __forceinline__ void row_ld4(const float* p, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void row_ld4(const double* p, double v[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void row_st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void row_st4(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------ saddle SpMM
// Velocity node a, chunk ch (both components):
//   Y(a, c) = sum_k F_ak X(col_k, c) + sum_i B^T_ai(c) X_p(i)
// Pressure row i:  sum_k Bx_ik X(a_k, 0) + By_ik X(a_k, 1)
// Dirichlet velocity rows and pressure row 0 are identity rows.  Each thread
// owns one 16-byte chunk of both components of a node, so F's values and
// column indices are loaded once for the two components; the nonzero loops
// are unrolled by two to keep independent gathers in flight.
template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_saddle(int n2, int np, int nch, const int* __restrict__ frp,
                                                const int* __restrict__ fcol, const T* __restrict__ Fval,
                                                const int* __restrict__ btrp, const int* __restrict__ btcol,
                                                const T* __restrict__ BTval, const int* __restrict__ brp,
                                                const int* __restrict__ bcol, const T* __restrict__ Bval,
                                                const unsigned char* __restrict__ isbnd, const T* __restrict__ X,
                                                const double* __restrict__ Bvec, T* __restrict__ Y) {
  pdl_wait();
  pdl_trigger();
  using V = typename Vec<T>::type;
  const V* Xv = reinterpret_cast<const V*>(X);
  V* Yv = reinterpret_cast<V*>(Y);
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nvel = (long long)n2 * nch;
  if (tid < nvel) {
    const int a = (int)(tid / nch), ch = (int)(tid % nch);
    const size_t o0 = ((size_t)(2 * a)) * nch + ch, o1 = o0 + nch;
    V acc0, acc1;
    if (isbnd[a]) {
      acc0 = Xv[o0];
      acc1 = Xv[o1];
    } else {
      acc0 = vzero(V());
      acc1 = vzero(V());
      int k = frp[a];
      const int e = frp[a + 1];
      for (; k + 1 < e; k += 2) {
        const int c0 = fcol[k], c1 = fcol[k + 1];
        const T f0 = Fval[k], f1 = Fval[k + 1];
        const V x00 = Xv[(size_t)(2 * c0) * nch + ch], x01 = Xv[(size_t)(2 * c0 + 1) * nch + ch];
        const V x10 = Xv[(size_t)(2 * c1) * nch + ch], x11 = Xv[(size_t)(2 * c1 + 1) * nch + ch];
        vfma(acc0, f0, x00);
        vfma(acc1, f0, x01);
        vfma(acc0, f1, x10);
        vfma(acc1, f1, x11);
      }
      if (k < e) {
        const int c0 = fcol[k];
        const T f0 = Fval[k];
        vfma(acc0, f0, Xv[(size_t)(2 * c0) * nch + ch]);
        vfma(acc1, f0, Xv[(size_t)(2 * c0 + 1) * nch + ch]);
      }
      const size_t pbase = (size_t)2 * n2 * nch;
      for (int t = btrp[a]; t < btrp[a + 1]; ++t) {
        const V xp = Xv[pbase + (size_t)btcol[t] * nch + ch];
        vfma(acc0, BTval[2 * (size_t)t], xp);
        vfma(acc1, BTval[2 * (size_t)t + 1], xp);
      }
    }
    if (MODE == 0) {
      Yv[o0] = acc0;
      Yv[o1] = acc1;
    } else {
      const V* Bb = reinterpret_cast<const V*>(Bvec);
      Yv[o0] = vaxpby(T(1), Bb[o0], T(-1), acc0);
      Yv[o1] = vaxpby(T(1), Bb[o1], T(-1), acc1);
    }
    return;
  }
  const long long p = tid - nvel;
  if (p >= (long long)np * nch) return;
  const int i = (int)(p / nch), ch = (int)(p % nch);
  const size_t out = (size_t)2 * n2 * nch + (size_t)i * nch + ch;
  V acc;
  if (i == 0) {
    acc = Xv[out];
  } else {
    acc = vzero(V());
    V acc2 = vzero(V());
    int k = brp[i];
    const int e = brp[i + 1];
    for (; k + 1 < e; k += 2) {
      const size_t x0 = ((size_t)(2 * bcol[k])) * nch + ch, x1 = ((size_t)(2 * bcol[k + 1])) * nch + ch;
      const V a0 = Xv[x0], a1 = Xv[x0 + nch], b0 = Xv[x1], b1 = Xv[x1 + nch];
      vfma(acc, Bval[2 * (size_t)k], a0);
      vfma(acc, Bval[2 * (size_t)k + 1], a1);
      vfma(acc2, Bval[2 * (size_t)k + 2], b0);
      vfma(acc2, Bval[2 * (size_t)k + 3], b1);
    }
    if (k < e) {
      const size_t x0 = ((size_t)(2 * bcol[k])) * nch + ch;
      vfma(acc, Bval[2 * (size_t)k], Xv[x0]);
      vfma(acc, Bval[2 * (size_t)k + 1], Xv[x0 + nch]);
    }
    acc = vaxpby(T(1), acc, T(1), acc2);
  }
  if (MODE == 0) {
    Yv[out] = acc;
  } else {
    const V* Bb = reinterpret_cast<const V*>(Bvec);
    Yv[out] = vaxpby(T(1), Bb[out], T(-1), acc);
  }
}

// Row-per-thread variant: one thread owns a velocity node (both components,
// all NCH 16-byte chunks of the member row) or a pressure row, so a row's
// column indices and values are loaded once and every nonzero issues 2*NCH
// independent 16-byte gathers.
template <typename T, int MODE, int NCH>
__global__ void __launch_bounds__(128) k_saddle_rows(int n2, int np, const int* __restrict__ frp,
                                                     const int* __restrict__ fcol, const T* __restrict__ Fval,
                                                     const int* __restrict__ btrp, const int* __restrict__ btcol,
                                                     const T* __restrict__ BTval, const int* __restrict__ brp,
                                                     const int* __restrict__ bcol, const T* __restrict__ Bval,
                                                     const unsigned char* __restrict__ isbnd,
                                                     const T* __restrict__ X, const double* __restrict__ Bvec,
                                                     T* __restrict__ Y) {
  using V = typename Vec<T>::type;
  const V* Xv = reinterpret_cast<const V*>(X);
  V* Yv = reinterpret_cast<V*>(Y);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < n2) {
    const int a = tid;
    const size_t o0 = (size_t)(2 * a) * NCH;
    V acc[2 * NCH];
    if (isbnd[a]) {
#pragma unroll
      for (int t = 0; t < 2 * NCH; ++t) acc[t] = Xv[o0 + t];
    } else {
#pragma unroll
      for (int t = 0; t < 2 * NCH; ++t) acc[t] = vzero(V());
      for (int k = frp[a]; k < frp[a + 1]; ++k) {
        const T f = Fval[k];
        const V* xr = Xv + (size_t)(2 * fcol[k]) * NCH;
#pragma unroll
        for (int t = 0; t < 2 * NCH; ++t) vfma(acc[t], f, xr[t]);
      }
      const size_t pbase = (size_t)2 * n2 * NCH;
      for (int k = btrp[a]; k < btrp[a + 1]; ++k) {
        const T bx = BTval[2 * (size_t)k], by = BTval[2 * (size_t)k + 1];
        const V* xp = Xv + pbase + (size_t)btcol[k] * NCH;
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
          const V x = xp[t];
          vfma(acc[t], bx, x);
          vfma(acc[NCH + t], by, x);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 2 * NCH; ++t) {
      if (MODE == 0)
        Yv[o0 + t] = acc[t];
      else
        Yv[o0 + t] = vaxpby(T(1), reinterpret_cast<const V*>(Bvec)[o0 + t], T(-1), acc[t]);
    }
    return;
  }
  const int i = tid - n2;
  if (i >= np) return;
  const size_t out = (size_t)2 * n2 * NCH + (size_t)i * NCH;
  V acc[NCH];
  if (i == 0) {
#pragma unroll
    for (int t = 0; t < NCH; ++t) acc[t] = Xv[out + t];
  } else {
#pragma unroll
    for (int t = 0; t < NCH; ++t) acc[t] = vzero(V());
    for (int k = brp[i]; k < brp[i + 1]; ++k) {
      const T bx = Bval[2 * (size_t)k], by = Bval[2 * (size_t)k + 1];
      const V* xr = Xv + (size_t)(2 * bcol[k]) * NCH;
#pragma unroll
      for (int t = 0; t < NCH; ++t) {
        vfma(acc[t], bx, xr[t]);
        vfma(acc[t], by, xr[NCH + t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < NCH; ++t) {
    if (MODE == 0)
      Yv[out + t] = acc[t];
    else
      Yv[out + t] = vaxpby(T(1), reinterpret_cast<const V*>(Bvec)[out + t], T(-1), acc[t]);
  }
}

template <typename T, int MODE, int NCH>
static void saddle_rows(const mhde_ctx* c, const T* Fval, const T* Bval, const T* BTval, const T* X,
                        const double* Bvec, T* Y, cudaStream_t st) {
  const int n = c->fe.n2 + c->fe.np;
  k_saddle_rows<T, MODE, NCH><<<nblk(n, 128), 128, 0, st>>>(c->fe.n2, c->fe.np, c->F.rowptr, c->F.col, Fval,
                                                           c->BT.rowptr, c->BT.col, BTval, c->B.rowptr, c->B.col,
                                                           Bval, c->d_isbnd, X, Bvec, Y);
}

template <typename T, int MODE>
static bool saddle_rows_dispatch(const mhde_ctx* c, const T* Fval, const T* Bval, const T* BTval, const T* X,
                                 const double* Bvec, T* Y, int nch, cudaStream_t st) {
  switch (nch) {
    case 1: saddle_rows<T, MODE, 1>(c, Fval, Bval, BTval, X, Bvec, Y, st); return true;
    case 2: saddle_rows<T, MODE, 2>(c, Fval, Bval, BTval, X, Bvec, Y, st); return true;
    case 3: saddle_rows<T, MODE, 3>(c, Fval, Bval, BTval, X, Bvec, Y, st); return true;
    case 4: saddle_rows<T, MODE, 4>(c, Fval, Bval, BTval, X, Bvec, Y, st); return true;
    case 5: saddle_rows<T, MODE, 5>(c, Fval, Bval, BTval, X, Bvec, Y, st); return true;
    case 6: saddle_rows<T, MODE, 6>(c, Fval, Bval, BTval, X, Bvec, Y, st); return true;
    case 8: saddle_rows<T, MODE, 8>(c, Fval, Bval, BTval, X, Bvec, Y, st); return true;
    case 10: saddle_rows<T, MODE, 10>(c, Fval, Bval, BTval, X, Bvec, Y, st); return true;
    default: return false;
  }
}

template <typename T>
void launch_saddle_spmm(const mhde_ctx* c, const T* Fval, const T* Bval, const T* BTval, const T* X,
                        const double* Bvec, T* Y, int mode, int ld, cudaStream_t st) {
  count_launch();
  int nch = ld / Vec<T>::W;
  if (c->spmm_rows) {
    const bool done = (mode == 0) ? saddle_rows_dispatch<T, 0>(c, Fval, Bval, BTval, X, Bvec, Y, nch, st)
                                  : saddle_rows_dispatch<T, 1>(c, Fval, Bval, BTval, X, Bvec, Y, nch, st);
    if (done) return;
  }
  long long n = ((long long)c->fe.n2 + c->fe.np) * nch;
  const int bs = c->spmm_block;
  if (mode == 0)
    launch_pdl(k_saddle<T, 0>, dim3(nblk(n, bs)), dim3(bs), 0, st, c->fe.n2, c->fe.np, nch, c->F.rowptr, c->F.col,
               Fval, c->BT.rowptr, c->BT.col, BTval, c->B.rowptr, c->B.col, Bval, c->d_isbnd, X, Bvec, Y);
  else
    launch_pdl(k_saddle<T, 1>, dim3(nblk(n, bs)), dim3(bs), 0, st, c->fe.n2, c->fe.np, nch, c->F.rowptr, c->F.col,
               Fval, c->BT.rowptr, c->BT.col, BTval, c->B.rowptr, c->B.col, Bval, c->d_isbnd, X, Bvec, Y);
}

// ------------------------------------------------------------ generic CSR
template <typename T>
__global__ void k_csr(int nrows, int nch, const int* __restrict__ rp, const int* __restrict__ col,
                      const T* __restrict__ val, const T* __restrict__ dinv, T omega,
                      const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ y, int mode) {
  pdl_wait();
  pdl_trigger();
  using V = typename Vec<T>::type;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)nrows * nch) return;
  int r = (int)(tid / nch), ch = (int)(tid % nch);
  const V* xv = reinterpret_cast<const V*>(x);
  const V* bv = reinterpret_cast<const V*>(b);
  V* yv = reinterpret_cast<V*>(y);
  size_t o = (size_t)r * nch + ch;
  if (mode == 3) {
    yv[o] = vaxpby(omega * dinv[r], bv[o], T(0), bv[o]);
    return;
  }
  V acc = vzero(V());
  for (int k = rp[r]; k < rp[r + 1]; ++k) vfma(acc, val[k], xv[(size_t)col[k] * nch + ch]);
  if (mode == 0) {
    yv[o] = acc;
  } else if (mode == 1) {
    yv[o] = vaxpby(T(1), bv[o], T(-1), acc);
  } else if (mode == 2) {
    V res = vaxpby(T(1), bv[o], T(-1), acc);
    yv[o] = vaxpby(T(1), xv[o], omega * dinv[r], res);
  } else if (mode == 4) {
    yv[o] = vaxpby(T(1), yv[o], T(1), acc);
  } else {
    yv[o] = vaxpby(T(1), bv[o], T(1), acc);
  }
}

template <typename T>
void launch_csr(int nrows, const int* rowptr, const int* col, const T* val, const T* dinv, T omega,
                const T* x, const T* b, T* y, int mode, int Jp, cudaStream_t st) {
  count_launch();
  int nch = Jp / Vec<T>::W;
  long long n = (long long)nrows * nch;
  launch_pdl(k_csr<T>, dim3(nblk(n, 256)), dim3(256), 0, st, nrows, nch, rowptr, col, val, dinv, omega, x, b, y, mode);
}

__device__ __forceinline__ void warp_sum(double2& a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, off);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, off);
  }
}
__device__ __forceinline__ void warp_sum(float4& a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, off);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, off);
    a.z += __shfl_xor_sync(0xffffffffu, a.z, off);
    a.w += __shfl_xor_sync(0xffffffffu, a.w, off);
  }
}

// y = A x for a dense n x n matrix (the coarsest AMG level's inverse): one
// warp per (row, 16-byte chunk); lanes stride over k with coalesced reads of
// the row and finish with a fixed butterfly of shuffles (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) k_dense_apply(int n, int nch, const T* __restrict__ A,
                                                     const T* __restrict__ x, T* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  using V = typename Vec<T>::type;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (long long)n * nch) return;          // whole warps exit together
  const int r = (int)(wid / nch), ch = (int)(wid % nch);
  const V* xv = reinterpret_cast<const V*>(x);
  const T* arow = A + (size_t)r * n;
  V acc = vzero(V());
#pragma unroll 4
  for (int k = lane; k < n; k += 32) vfma(acc, arow[k], xv[(size_t)k * nch + ch]);
  warp_sum(acc);
  if (lane == 0) reinterpret_cast<V*>(y)[(size_t)r * nch + ch] = acc;
}

template <typename T>
void launch_dense_apply(int n, const T* Ainv, const T* x, T* y, int Jp, cudaStream_t st) {
  count_launch();
  int nch = Jp / Vec<T>::W;
  long long threads = (long long)n * nch * 32;
  launch_pdl(k_dense_apply<T>, dim3(nblk(threads, 256)), dim3(256), 0, st, n, nch, Ainv, x, y);
}

// ------------------------------------------------------------ preconditioner pieces
template <typename T>
__global__ void k_jacobi_F(int n2, int nch, const int* __restrict__ rp, const int* __restrict__ col,
                           const T* __restrict__ F, const T* __restrict__ dinv,
                           const unsigned char* __restrict__ isbnd, T omega, const T* __restrict__ r,
                           const T* __restrict__ zin, T* __restrict__ zout) {
  using V = typename Vec<T>::type;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n2 * 2 * nch) return;
  int a = (int)(tid / (2 * nch));
  int rem = (int)(tid % (2 * nch));
  int c = rem / nch, ch = rem % nch;
  size_t o = ((size_t)(2 * a + c)) * nch + ch;
  const V* rv = reinterpret_cast<const V*>(r);
  V* zo = reinterpret_cast<V*>(zout);
  if (isbnd[a]) {
    zo[o] = rv[o];
    return;
  }
  if (zin == nullptr) {
    zo[o] = vaxpby(dinv[a], rv[o], T(0), rv[o]);
    return;
  }
  const V* zi = reinterpret_cast<const V*>(zin);
  V acc = vzero(V());
  for (int k = rp[a]; k < rp[a + 1]; ++k) vfma(acc, F[k], zi[((size_t)(2 * col[k] + c)) * nch + ch]);
  V res = vaxpby(T(1), rv[o], T(-1), acc);
  zo[o] = vaxpby(T(1), zi[o], omega * dinv[a], res);
}

template <typename T>
void launch_jacobi_F(const mhde_ctx* c, const T* Fval, const T* Fdinv, T omega, const T* r,
                     const T* zin, T* zout, int ld, cudaStream_t st) {
  count_launch();
  int nch = ld / Vec<T>::W;
  long long n = (long long)c->fe.n2 * 2 * nch;
  k_jacobi_F<T><<<nblk(n, 256), 256, 0, st>>>(c->fe.n2, nch, c->F.rowptr, c->F.col, Fval, Fdinv,
                                             c->d_isbnd, omega, r, zin, zout);
}

template <typename T>
__global__ void k_precond_p(int np, int nch, const T* __restrict__ x, const T* __restrict__ rp,
                            const T* __restrict__ mp, T inv_dt, T nu_hat, const int* __restrict__ nrp,
                            const int* __restrict__ ncol, const T* __restrict__ Np, T* __restrict__ zp) {
  pdl_wait();
  pdl_trigger();
  using V = typename Vec<T>::type;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)np * nch) return;
  int i = (int)(tid / nch), ch = (int)(tid % nch);
  const V* xv = reinterpret_cast<const V*>(x);
  const V* rv = reinterpret_cast<const V*>(rp);
  V* zv = reinterpret_cast<V*>(zp);
  if (i == 0) {
    zv[tid] = rv[tid];
    return;
  }
  V z = vaxpby(-inv_dt, xv[tid], -nu_hat / mp[i], rv[tid]);
  if (Np) {
    V acc = vzero(V());
    for (int k = nrp[i]; k < nrp[i + 1]; ++k) vfma(acc, Np[k], xv[(size_t)ncol[k] * nch + ch]);
    z = vaxpby(T(1), z, -T(1) / mp[i], acc);
  }
  zv[tid] = z;
}

template <typename T>
void launch_precond_p(int np, int Jp, const T* x, const T* rp, const T* mp, T inv_dt, T nu_hat,
                      const int* nrp, const int* ncol, const T* Np, T* zp, cudaStream_t st) {
  count_launch();
  int nch = Jp / Vec<T>::W;
  long long n = (long long)np * nch;
  launch_pdl(k_precond_p<T>, dim3(nblk(n, 256)), dim3(256), 0, st, np, nch, x, rp, mp, inv_dt, nu_hat, nrp, ncol, Np,
             zp);
}

template <typename T>
__global__ void k_bt_apply(int n2, int nch, const int* __restrict__ rp, const int* __restrict__ col,
                           const T* __restrict__ BT, const unsigned char* __restrict__ isbnd,
                           const T* __restrict__ ru, const T* __restrict__ zp, T* __restrict__ tu) {
  pdl_wait();
  pdl_trigger();
  using V = typename Vec<T>::type;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n2 * 2 * nch) return;
  int a = (int)(tid / (2 * nch));
  int rem = (int)(tid % (2 * nch));
  int c = rem / nch, ch = rem % nch;
  const V* r = reinterpret_cast<const V*>(ru);
  const V* z = reinterpret_cast<const V*>(zp);
  V* t = reinterpret_cast<V*>(tu);
  size_t o = ((size_t)(2 * a + c)) * nch + ch;
  if (isbnd[a]) {
    t[o] = r[o];
    return;
  }
  V acc = vzero(V());
  for (int k = rp[a]; k < rp[a + 1]; ++k) vfma(acc, BT[2 * (size_t)k + c], z[(size_t)col[k] * nch + ch]);
  t[o] = vaxpby(T(1), r[o], T(-1), acc);
}

template <typename T>
void launch_bt_apply(const mhde_ctx* c, const T* BTval, const T* ru, const T* zp, T* tu, int ld,
                     cudaStream_t st) {
  count_launch();
  int nch = ld / Vec<T>::W;
  long long n = (long long)c->fe.n2 * 2 * nch;
  launch_pdl(k_bt_apply<T>, dim3(nblk(n, 256)), dim3(256), 0, st,
             c->fe.n2, nch, c->BT.rowptr, c->BT.col, BTval, c->d_isbnd, ru, zp, tu);
}

// ------------------------------------------------------------ block-Jacobi smoothing
// x_out = x_in + omega Binv r over blocks of bs dofs (idx[b][i]); x_in null
// means x_in = 0.  Every thread reads x_in and writes x_out at its own row
// only, so x_out may be x_in; r must be another buffer.
template <typename T>
__global__ void k_block_jacobi(int nb, int bs, int nch, const int* __restrict__ idx, const T* __restrict__ inv,
                               T omega, const T* x_in, const T* __restrict__ r, T* x_out) {
  pdl_wait();
  pdl_trigger();
  using V = typename Vec<T>::type;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)nb * bs * nch) return;
  const int b = (int)(tid / ((long long)bs * nch));
  const int rem = (int)(tid % ((long long)bs * nch));
  const int i = rem / nch, ch = rem % nch;
  const int* id = idx + (size_t)b * bs;
  const T* Bi = inv + ((size_t)b * bs + i) * bs;
  const V* rv = reinterpret_cast<const V*>(r);
  V acc = vzero(V());
  for (int j = 0; j < bs; ++j) vfma(acc, Bi[j], rv[(size_t)id[j] * nch + ch]);
  const size_t o = (size_t)id[i] * nch + ch;
  V* xo = reinterpret_cast<V*>(x_out);
  if (x_in) {
    const V xi = reinterpret_cast<const V*>(x_in)[o];
    xo[o] = vaxpby(T(1), xi, omega, acc);
  } else {
    xo[o] = vaxpby(omega, acc, T(0), vzero(V()));
  }
}

template <typename T>
void launch_block_jacobi(int nb, int bs, const int* idx, const T* inv, T omega, const T* x_in, const T* r,
                         T* x_out, int Jp, cudaStream_t st) {
  count_launch();
  const int nch = Jp / Vec<T>::W;
  const long long n = (long long)nb * bs * nch;
  launch_pdl(k_block_jacobi<T>, dim3(nblk(n, 256)), dim3(256), 0, st, nb, bs, nch, idx, inv, omega, x_in, r, x_out);
}

// ------------------------------------------------------------ least-squares commutator
// The three products between the two pressure-Laplacian solves of
//   S^{-1} ~ L^{-1} (B D^{-1} F D^{-1} B^T) L^{-1},  L = B D^{-1} B^T,
// with D^{-1} zero on Dirichlet nodes (their velocities are fixed) and the
// pinned pressure dof 0 taken as zero on both sides.
template <typename T>
__global__ void k_lsc_bt(int n2, int nch, const int* __restrict__ rp, const int* __restrict__ col,
                         const T* __restrict__ BT, const T* __restrict__ dinv, const T* __restrict__ y,
                         T* __restrict__ t) {
  pdl_wait();
  pdl_trigger();
  using V = typename Vec<T>::type;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n2 * nch) return;
  const int a = (int)(tid / nch), ch = (int)(tid % nch);
  const V* yv = reinterpret_cast<const V*>(y);
  V* tv = reinterpret_cast<V*>(t);
  const size_t o0 = ((size_t)(2 * a)) * nch + ch, o1 = o0 + nch;
  V acc0 = vzero(V()), acc1 = vzero(V());
  const T di = dinv[a];
  if (di != T(0)) {
    for (int k = rp[a]; k < rp[a + 1]; ++k) {
      const int j = col[k];
      if (j == 0) continue;
      const V yj = yv[(size_t)j * nch + ch];
      vfma(acc0, BT[2 * (size_t)k], yj);
      vfma(acc1, BT[2 * (size_t)k + 1], yj);
    }
  }
  tv[o0] = vaxpby(di, acc0, T(0), vzero(V()));
  tv[o1] = vaxpby(di, acc1, T(0), vzero(V()));
}

template <typename T>
__global__ void k_lsc_f(int n2, int nch, const int* __restrict__ rp, const int* __restrict__ col,
                        const T* __restrict__ F, const T* __restrict__ dinv, const T* __restrict__ t,
                        T* __restrict__ s) {
  pdl_wait();
  pdl_trigger();
  using V = typename Vec<T>::type;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n2 * nch) return;
  const int a = (int)(tid / nch), ch = (int)(tid % nch);
  const V* tv = reinterpret_cast<const V*>(t);
  V* sv = reinterpret_cast<V*>(s);
  const size_t o0 = ((size_t)(2 * a)) * nch + ch, o1 = o0 + nch;
  V acc0 = vzero(V()), acc1 = vzero(V());
  const T di = dinv[a];
  if (di != T(0)) {
    for (int k = rp[a]; k < rp[a + 1]; ++k) {
      const size_t b = (size_t)(2 * col[k]) * nch + ch;
      vfma(acc0, F[k], tv[b]);
      vfma(acc1, F[k], tv[b + nch]);
    }
  }
  sv[o0] = vaxpby(di, acc0, T(0), vzero(V()));
  sv[o1] = vaxpby(di, acc1, T(0), vzero(V()));
}

template <typename T>
__global__ void k_lsc_b(int np, int nch, const int* __restrict__ rp, const int* __restrict__ col,
                        const T* __restrict__ B, const T* __restrict__ s, T* __restrict__ z) {
  pdl_wait();
  pdl_trigger();
  using V = typename Vec<T>::type;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)np * nch) return;
  const int i = (int)(tid / nch), ch = (int)(tid % nch);
  const V* sv = reinterpret_cast<const V*>(s);
  V acc = vzero(V());
  if (i != 0) {
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const size_t b = (size_t)(2 * col[k]) * nch + ch;
      vfma(acc, B[2 * (size_t)k], sv[b]);
      vfma(acc, B[2 * (size_t)k + 1], sv[b + nch]);
    }
  }
  reinterpret_cast<V*>(z)[tid] = acc;
}

template <typename T>
void launch_lsc_middle(const mhde_ctx* c, const T* Fval, const T* BTval, const T* Bval, const T* dinv,
                       const T* y, T* t, T* s, T* z, int ld, cudaStream_t st) {
  const int nch = ld / Vec<T>::W;
  const long long nv = (long long)c->fe.n2 * nch, np = (long long)c->fe.np * nch;
  count_launch();
  launch_pdl(k_lsc_bt<T>, dim3(nblk(nv, 256)), dim3(256), 0, st, c->fe.n2, nch, c->BT.rowptr, c->BT.col, BTval,
             dinv, y, t);
  count_launch();
  launch_pdl(k_lsc_f<T>, dim3(nblk(nv, 256)), dim3(256), 0, st, c->fe.n2, nch, c->F.rowptr, c->F.col, Fval, dinv,
             (const T*)t, s);
  count_launch();
  launch_pdl(k_lsc_b<T>, dim3(nblk(np, 256)), dim3(256), 0, st, c->fe.np, nch, c->B.rowptr, c->B.col, Bval,
             (const T*)s, z);
}

// ------------------------------------------------------------ block Gram
// CTA `chunk` covers a contiguous range of rows.  For every basis block i the
// CTA streams 64-row tiles of V_i and W (contiguous in memory) into shared
// memory; thread t owns a 4x4 tile of the r x r block (tile t % ntile) and
// every G-th row of the staged tile (group t / ntile).  Partial tiles are
// summed over the groups in a fixed order, so the result does not depend on
// scheduling.
constexpr int GRAM_TR = 64;

template <typename T>
__global__ void __launch_bounds__(256) k_gram(const T* __restrict__ V, size_t vstride, int kblocks,
                                              const T* __restrict__ W, int n_rows, int Jp, int r,
                                              int rows_per_chunk, double* __restrict__ part, int TR) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Vs = reinterpret_cast<T*>(smem_raw);
  T* Ws = Vs + TR * Jp;
  double* red = reinterpret_cast<double*>(Ws + TR * Jp);
  const int nt4 = (r + 3) / 4;
  const int ntile = nt4 * nt4;
  const int G = 256 / ntile;
  const int t = threadIdx.x;
  const int tile = t % ntile, grp = t / ntile;
  const int p0 = 4 * (tile / nt4), q0 = 4 * (tile % nt4);
  const int r0 = blockIdx.x * rows_per_chunk;
  const int r1 = min(n_rows, r0 + rows_per_chunk);
  const int i = blockIdx.y;                       // basis block of this CTA
  const T* Vi = V + (size_t)i * vstride;
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
  for (int tr0 = r0; tr0 < r1; tr0 += TR) {
    const int nr = min(TR, r1 - tr0);
    const int nel = nr * Jp;                      // contiguous elements of the tile
    const T* vsrc = Vi + (size_t)tr0 * Jp;
    const T* wsrc = W + (size_t)tr0 * Jp;
    for (int e = t; e < nel; e += blockDim.x) {
      Vs[e] = vsrc[e];
      Ws[e] = wsrc[e];
    }
    __syncthreads();
    if (grp < G) {
      for (int row = grp; row < nr; row += G) {
        const T* vr = Vs + row * Jp;
        const T* wr = Ws + row * Jp;
        T a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = vr[p0 + u];
          b[u] = wr[q0 + u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
      }
    }
    __syncthreads();
  }
  if (grp < G) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) red[((size_t)grp * ntile + tile) * 16 + 4 * u + v] = (double)acc[u][v];
  }
  __syncthreads();
  for (int o = t; o < ntile * 16; o += blockDim.x) {
    double sum = 0.0;
    for (int g = 0; g < G; ++g) sum += red[(size_t)g * ntile * 16 + o];
    int tl = o / 16, uv = o % 16;
    int p = 4 * (tl / nt4) + uv / 4, q = 4 * (tl % nt4) + uv % 4;
    if (p < r && q < r) part[(((size_t)blockIdx.x * kblocks) + i) * r * r + (size_t)p * r + q] = sum;
  }
}

// Pair-owned Gram: CTA (chunk, y) owns the (block i, column p) pairs
// y*PC .. y*PC+PC-1 (pair = i r + p); a thread keeps the QM-wide row
// G_i[p][0..QM) of at most PPT pairs in registers, W's rows are staged in
// shared memory 32 at a time and read as broadcasts, and every V_i value is
// loaded exactly once.  Writes the same per-chunk partials as k_gram.
constexpr int GRAM2_TR = 32;

template <typename T, int QM, int PPT>
__global__ void __launch_bounds__(256) k_gram_pairs(const T* __restrict__ V, size_t vstride, int kblocks,
                                                    const T* __restrict__ W, int n_rows, int ld, int r,
                                                    int rows_per_chunk, double* __restrict__ part) {
  __shared__ __align__(16) T Ws[GRAM2_TR][QM];
  const int r0 = blockIdx.x * rows_per_chunk;
  const int r1 = min(n_rows, r0 + rows_per_chunk);
  const int npairs = kblocks * r;
  int pi[PPT], pp[PPT];
  bool own[PPT];
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int pair = (blockIdx.y * PPT + s) * blockDim.x + threadIdx.x;
    own[s] = pair < npairs;
    pi[s] = own[s] ? pair / r : 0;
    pp[s] = own[s] ? pair % r : 0;
  }
  T acc[PPT][QM];
#pragma unroll
  for (int s = 0; s < PPT; ++s)
#pragma unroll
    for (int q = 0; q < QM; ++q) acc[s][q] = T(0);
  for (int t0 = r0; t0 < r1; t0 += GRAM2_TR) {
    const int nr = min(GRAM2_TR, r1 - t0);
    for (int e = threadIdx.x; e < GRAM2_TR * QM; e += blockDim.x) {
      const int rr = e / QM, q = e % QM;
      Ws[rr][q] = (rr < nr && q < r) ? W[(size_t)(t0 + rr) * ld + q] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
      if (!own[s]) continue;
      const T* vcol = V + (size_t)pi[s] * vstride + (size_t)t0 * ld + pp[s];
#pragma unroll 4
      for (int rr = 0; rr < nr; ++rr) {
        const T v = vcol[(size_t)rr * ld];
#pragma unroll
        for (int q = 0; q < QM; ++q) acc[s][q] += v * Ws[rr][q];
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    if (!own[s]) continue;
    double* dst = part + (((size_t)blockIdx.x * kblocks) + pi[s]) * r * r + (size_t)pp[s] * r;
#pragma unroll
    for (int q = 0; q < QM; ++q)
      if (q < r) dst[q] = (double)acc[s][q];
  }
}

// Sum of the per-chunk partials: a CTA owns 32 consecutive outputs; each of
// its 8 warps sums every 8th chunk for them (coalesced 256-byte reads), then
// the 8 partial sums are added in a fixed order (deterministic).
constexpr int GR_WARPS = 16;

__global__ void __launch_bounds__(32 * GR_WARPS) k_gram_reduce(int nparts, int total, const double* __restrict__ part,
                                                              double* __restrict__ gram) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[GR_WARPS][33];
  const int lo = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lo;
  double s = 0.0;
  if (o < total) {
#pragma unroll 8
    for (int c = g; c < nparts; c += GR_WARPS) s += part[(size_t)c * total + o];
  }
  sh[g][lo] = s;
  __syncthreads();
  if (g == 0 && o < total) {
    double v = 0.0;
#pragma unroll
    for (int h = 0; h < GR_WARPS; ++h) v += sh[h][lo];
    gram[o] = v;
  }
}

// Staged Gram (FP32): a CTA owns a range of rows and streams it through a
// GS_NST-deep ring of shared-memory stages.  One stage holds TR rows of every
// basis block and of W; each block's rows are one contiguous span in memory,
// so one thread fills a stage with one TMA bulk copy per block
// (cp.async.bulk, completion counted in bytes on the stage's mbarrier).  A
// thread owns one item (basis block i, 4-column group p4) and keeps its 4 x W
// products in registers; the W row is a shared-memory broadcast.  A block's
// tile is padded so that consecutive items read consecutive 16-byte words (no
// bank conflicts).  With few items a CTA runs S row slices, each writing its
// own partial, so every sum has a fixed order.
//
// Every wait on a stage's mbarrier is bounded: past GS_SPIN_LIMIT polls the
// thread records the failure in the caller's error word (one per subproblem,
// so concurrent subproblems never see each other's flags), waits (again bounded) for the
// CTA's copies still in flight, and the kernel returns without its partials.
constexpr int GS_T = 256;
constexpr int GS_NST = 3;
constexpr size_t GS_SMEM = 192 * 1024;
constexpr size_t GS_BAR_BYTES = 64;                   // mbarriers in front of the stages
constexpr long long GS_SPIN_LIMIT = 1ll << 24;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait for phase `parity` of the barrier; false after the limit
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  for (long long it = 0; it < GS_SPIN_LIMIT; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

template <int W, int PC, int NTH>
__global__ void __launch_bounds__(NTH, 1) k_gram_staged(const float* __restrict__ V, size_t vstride, int kblocks,
                                                      const float* __restrict__ Wm, int n_rows, int ld, int r,
                                                      int rows_per_chunk, int S, int TR, int tstride,
                                                      double* __restrict__ part, int* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  // every bulk copy needs 16-byte aligned tiles and rows; the host plan
  // guarantees it, and a launch that breaks it copies nothing
  if ((tstride & 3) || (ld & 3) || ((TR * ld) & 3)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  float* gsm = reinterpret_cast<float*>(gsm_raw + GS_BAR_BYTES);
  const unsigned bar0 = smem_u32(gsm_raw);            // GS_NST 8-byte barriers
  const int stage_floats = kblocks * tstride + TR * ld;
  const int NP = (r + PC - 1) / PC;                    // column groups of PC per block
  const int items = kblocks * NP;
  const int slice = threadIdx.x / items, item = threadIdx.x % items;
  const bool active = slice < S;
  const int i = item / NP, pg = item % NP;
  const int r0 = blockIdx.x * rows_per_chunk, r1 = min(n_rows, r0 + rows_per_chunk);
  const int ntiles = r1 > r0 ? (r1 - r0 + TR - 1) / TR : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < GS_NST; ++s) mbar_init(bar0 + 8 * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  // warp 0 fills a stage: (kblocks + 1) contiguous spans of nr * ld floats,
  // lane 0 registering the stage's bytes, then one bulk copy per lane
  const int lane = threadIdx.x & 31;
  auto issue = [&](int tile) {
    if (tile >= ntiles) return;
    const int s = tile % GS_NST;
    float* st = gsm + (size_t)s * stage_floats;
    const int t0 = r0 + tile * TR;
    const unsigned bytes = (unsigned)(min(TR, r1 - t0) * ld) * 4u;
    const unsigned bar = bar0 + 8 * s;
    // the stage's previous contents were read through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (lane == 0) mbar_expect_tx(bar, bytes * (unsigned)(kblocks + 1));
    __syncwarp();
    for (int b = lane; b <= kblocks; b += 32) {
      const float* src = (b < kblocks ? V + (size_t)b * vstride : Wm) + (size_t)t0 * ld;
      bulk_g2s(smem_u32(st + (size_t)b * tstride), src, bytes, bar);
    }
  };
  float acc[PC][W];
#pragma unroll
  for (int e = 0; e < PC; ++e)
#pragma unroll
    for (int q = 0; q < W; ++q) acc[e][q] = 0.f;
  if (threadIdx.x < 32)
    for (int s = 0; s < GS_NST - 1; ++s) issue(s);
  int ok = 1;
  int waited = 0;                                      // tiles whose copies this CTA has seen land
  for (int tile = 0; tile < ntiles; ++tile) {
    const unsigned bar = bar0 + 8 * (tile % GS_NST);
    const bool landed = mbar_wait_bounded(bar, (unsigned)((tile / GS_NST) & 1));
    if (!__syncthreads_and(landed ? 1 : 0)) {        // stage tile-1 is free once everyone is here
      ok = 0;
      break;
    }
    waited = tile + 1;
    if (threadIdx.x < 32) issue(tile + GS_NST - 1);
    if (active) {
      const float* st = gsm + (size_t)(tile % GS_NST) * stage_floats;
      const int nr = min(TR, r1 - (r0 + tile * TR));
      const float* vt = st + (size_t)i * tstride + PC * pg;
      const float* wt = st + (size_t)kblocks * tstride;
#pragma unroll 2
      for (int rr = slice; rr < nr; rr += S) {
        float v[PC];
        if constexpr (PC == 4) {
          row_ld4(vt + rr * ld, v);
        } else {
          const float2 t2 = *reinterpret_cast<const float2*>(vt + rr * ld);
          v[0] = t2.x;
          v[PC - 1] = t2.y;
        }
#pragma unroll
        for (int q4 = 0; q4 < W / 4; ++q4) {
          float w[4];
          row_ld4(wt + rr * ld + 4 * q4, w);
#pragma unroll
          for (int e = 0; e < PC; ++e)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[e][4 * q4 + u] = fmaf(v[e], w[u], acc[e][4 * q4 + u]);
        }
      }
    }
  }
  if (!ok) {
    // a stage did not land in time: record it, give every copy this CTA
    // issued a bounded chance to finish, and leave without partials
    if (threadIdx.x == 0) {
      atomicExch(err, 1);
      const int issued = min(ntiles, waited + GS_NST - 1);
      for (int tl = waited; tl < issued; ++tl)
        mbar_wait_bounded(bar0 + 8 * (tl % GS_NST), (unsigned)((tl / GS_NST) & 1));
    }
    return;
  }
  if (!active) return;
  double* dst = part + ((size_t)(blockIdx.x * S + slice) * kblocks + i) * r * r;
#pragma unroll
  for (int e = 0; e < PC; ++e) {
    const int pr = PC * pg + e;
    if (pr >= r) break;
#pragma unroll
    for (int q = 0; q < W; ++q)
      if (q < r) dst[(size_t)pr * r + q] = (double)acc[e][q];
  }
}

// Reads and clears a subproblem's bounded-wait failure word (set by a staged
// Gram or combine launch whose TMA stage did not land within its poll limit),
// on that subproblem's stream only.
int take_async_error(int* d_err, cudaStream_t st) {
  int h = 0;
  if (cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  if (h && cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) return -1;
  return h;
}

// Stage geometry of the staged Gram: rows per stage (a multiple of 8, at most
// 128) so that GS_NST stages fit in GS_SMEM, and the padded block-tile stride.
static bool gram_staged_plan(int kblocks, int ld, int r, int pc, int& TR, int& tstride, size_t& smem) {
  const int NP = (r + pc - 1) / pc;
  for (TR = 128; TR >= 8; TR -= 8) {
    // consecutive items read consecutive pc-float words across block tiles too,
    // as far as the 16-byte alignment of every tile (a TMA bulk-copy
    // destination) allows: the pad is a multiple of 4 floats
    const int pad = ((((pc * NP - TR * ld) % 32 + 32) % 32) + 3) / 4 * 4 % 32;
    tstride = TR * ld + pad;
    if (tstride % 4 != 0 || (TR * ld) % 4 != 0) return false;
    smem = GS_BAR_BYTES + (size_t)GS_NST * ((size_t)kblocks * tstride + (size_t)TR * ld) * sizeof(float);
    if (smem <= GS_SMEM) return true;
  }
  return false;
}

template <int W, int PC, int NTH>
static void gram_staged(const float* V, size_t vstride, int kblocks, const float* Wm, int n_rows, int ld, int r,
                        int nchunk, int nsm, int TR, int tstride, size_t smem, double* part, cudaStream_t st,
                        int& nparts, int* err) {
  const int items = kblocks * ((r + PC - 1) / PC);
  const int S = std::max(1, std::min(NTH / items, nchunk));
  const int nctas = std::max(1, std::min(nchunk / S, nsm));
  const int rows_per_chunk = (n_rows + nctas - 1) / nctas;
  nparts = nctas * S;
  launch_pdl(k_gram_staged<W, PC, NTH>, dim3(nctas), dim3(NTH), smem, st, V, vstride, kblocks, Wm, n_rows, ld, r,
             rows_per_chunk, S, TR, tstride, part, err);
}

static cudaError_t combine_staged_attr();

// Per-device one-time setup of the Gram kernels (shared-memory limits and the
// SM count that sizes the staged grid), done under a mutex because the two
// subproblems call in from their own host threads.
struct GramDevice {
  bool ready = false;
  int nsm = 1;
  cudaError_t err = cudaSuccess;
};
static std::mutex g_gram_mutex;
static GramDevice g_gram_dev[64];

static const GramDevice& gram_setup() {
  static const GramDevice none{false, 1, cudaErrorInvalidDevice};   // never written
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return none;
  std::lock_guard<std::mutex> lock(g_gram_mutex);
  GramDevice& d = g_gram_dev[dev];
  if (d.ready) return d;
  cudaError_t e = cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
  if (d.nsm <= 0) d.nsm = 1;
  auto set = [&](const void* f, int bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)k_gram_staged<4, 4, 256>, (int)GS_SMEM);
  set((const void*)k_gram_staged<4, 2, 512>, (int)GS_SMEM);
  set((const void*)k_gram_staged<8, 4, 256>, (int)GS_SMEM);
  set((const void*)k_gram_staged<8, 2, 512>, (int)GS_SMEM);
  set((const void*)k_gram_staged<12, 4, 256>, (int)GS_SMEM);
  set((const void*)k_gram_staged<12, 2, 512>, (int)GS_SMEM);
  set((const void*)k_gram_staged<16, 4, 256>, (int)GS_SMEM);
  set((const void*)k_gram_staged<16, 2, 512>, (int)GS_SMEM);
  set((const void*)k_gram_staged<20, 4, 256>, (int)GS_SMEM);
  set((const void*)k_gram_staged<20, 2, 512>, (int)GS_SMEM);
  set((const void*)k_gram_staged<24, 4, 256>, (int)GS_SMEM);
  set((const void*)k_gram_staged<24, 2, 512>, (int)GS_SMEM);
  set((const void*)k_gram<float>, 160 * 1024);
  if (e == cudaSuccess) e = combine_staged_attr();
  set((const void*)k_gram<double>, 160 * 1024);
  d.err = e;
  d.ready = true;
  return d;
}

// rows per staged tile: at least 64 and four per thread group, so narrow
// blocks (few tiles, many groups) keep every thread busy
static int gram_tile_rows(int r) {
  int nt4 = (r + 3) / 4;
  int G = 256 / (nt4 * nt4);
  return std::max(GRAM_TR, 4 * G);
}

template <typename T>
static size_t gram_smem(int Jp, int r) {
  int nt4 = (r + 3) / 4;
  int ntile = nt4 * nt4;
  int G = 256 / ntile;
  return 2 * (size_t)gram_tile_rows(r) * Jp * sizeof(T) + (size_t)G * ntile * 16 * sizeof(double);
}

// Partial sums go to part[nchunk][kblocks][r][r] at most (nchunk bounds the
// scratch the caller provides), then one reduction.
template <typename T>
void launch_gram(const T* V, size_t vstride, int kblocks, const T* W, int n_rows, int Jp, int r,
                 int nchunk, double* part, double* gram, cudaStream_t st, bool reduce, int* err, bool allow_tc) {
  count_launch(reduce ? 2 : 1);
  if (sizeof(T) == 4 && allow_tc && err != nullptr) {
    int np = 0;
    if (launch_gram_tc(reinterpret_cast<const float*>(V), vstride, kblocks, reinterpret_cast<const float*>(W),
                       n_rows, Jp, r, nchunk, part, st, err, np)) {
      if (reduce) launch_gram_reduce(np, kblocks * r * r, part, gram, st);
      return;
    }
  }
  const GramDevice& gd = gram_setup();               // on failure the unstaged kernels run instead
  const int w = (r + 3) / 4 * 4;
  int nparts = nchunk;
  int TR = 0, tstride = 0;
  size_t smem = 0;
  // item width: 2 columns per thread and 512 threads (16 warps per SM) unless
  // MHDE_GRAM_PC=4 asks for 4 columns and 256 threads
  static const int pc_env = [] {
    const char* e = std::getenv("MHDE_GRAM_PC");
    return (e && std::atoi(e) == 4) ? 4 : 2;
  }();
  const int pc = pc_env, nth = pc == 4 ? 256 : 512;
  // the staged kernels report a stage that never landed through `err`, so
  // they run only for callers that read it
  const bool staged = err != nullptr && gd.err == cudaSuccess && sizeof(T) == 4 && kblocks * ((r + pc - 1) / pc) <= nth && w <= 24 &&
                      gram_staged_plan(kblocks, Jp, r, pc, TR, tstride, smem);
  if (staged) {
    const float* Vf = reinterpret_cast<const float*>(V);
    const float* Wf = reinterpret_cast<const float*>(W);
#define MHDE_GS(WV)                                                                                            \
  do {                                                                                                         \
    if (pc == 4)                                                                                               \
      gram_staged<WV, 4, 256>(Vf, vstride, kblocks, Wf, n_rows, Jp, r, nchunk, gd.nsm, TR, tstride, smem, part, \
                              st, nparts, err);                                                                \
    else                                                                                                       \
      gram_staged<WV, 2, 512>(Vf, vstride, kblocks, Wf, n_rows, Jp, r, nchunk, gd.nsm, TR, tstride, smem, part, \
                              st, nparts, err);                                                                \
  } while (0)
    switch (w) {
      case 4: MHDE_GS(4); break;
      case 8: MHDE_GS(8); break;
      case 12: MHDE_GS(12); break;
      case 16: MHDE_GS(16); break;
      case 20: MHDE_GS(20); break;
      default: MHDE_GS(24); break;
    }
#undef MHDE_GS
  } else {
    const int rows_per_chunk = (n_rows + nchunk - 1) / nchunk;
    const int npairs = kblocks * r;
    if (r <= 32 && npairs >= 256 && sizeof(T) == 4) {
      constexpr int PPT = 2;
      const unsigned gy = (unsigned)((npairs + 256 * PPT - 1) / (256 * PPT));
#define MHDE_GP(QMV)                                                                                  \
  k_gram_pairs<T, QMV, PPT><<<dim3(nchunk, gy), 256, 0, st>>>(V, vstride, kblocks, W, n_rows, Jp, r, \
                                                              rows_per_chunk, part)
      if (r <= 4)
        MHDE_GP(4);
      else if (r <= 8)
        MHDE_GP(8);
      else if (r <= 16)
        MHDE_GP(16);
      else if (r <= 24)
        MHDE_GP(24);
      else
        MHDE_GP(32);
#undef MHDE_GP
    } else {
      size_t shmem = gram_smem<T>(Jp, r);
      k_gram<T><<<dim3(nchunk, kblocks), 256, shmem, st>>>(V, vstride, kblocks, W, n_rows, Jp, r, rows_per_chunk,
                                                            part, gram_tile_rows(r));
    }
  }
  if (!reduce) return;                               // partial sums only (kernel timing)
  launch_gram_reduce(nparts, kblocks * r * r, part, gram, st);
}

void launch_gram_reduce(int nparts, int total, const double* part, double* gram, cudaStream_t st) {
  launch_pdl(k_gram_reduce, dim3((total + 31) / 32), dim3(32 * GR_WARPS), 0, st, nparts, total, part, gram);
}

// ------------------------------------------------------------ one-reduce Gram-Schmidt helpers
// G holds H_0 .. H_k (H_i = V_i^T W) and W^T W as r x r blocks.  Block k + 2
// receives the projected Gram W^T W - sum_i H_i^T H_i: one warp per entry, its
// lanes striding over the (i, t) terms, then a fixed butterfly of shuffles
// (deterministic).
__global__ void __launch_bounds__(256) k_proj_gram(double* G, int k, int r) {
  pdl_wait();
  pdl_trigger();
  const int rr = r * r;
  const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= rr) return;                            // whole warps exit together
  const int p = o / r, q = o % r;
  const int nterm = (k + 1) * r;
  double acc = 0.0;
  for (int e = lane; e < nterm; e += 32) {
    const int i = e / r, t = e - i * r;
    const double* Hi = G + (size_t)i * rr + (size_t)t * r;
    acc = fma(Hi[p], Hi[q], acc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) G[(size_t)(k + 2) * rr + o] = G[(size_t)(k + 1) * rr + o] - acc;
}

void launch_proj_gram(double* G, int k, int r, cudaStream_t st) {
  count_launch();
  const long long threads = (long long)r * r * 32;
  launch_pdl(k_proj_gram, dim3(nblk(threads, 256)), dim3(256), 0, st, G, k, r);
}

// Coefficients of V_{k+1} = (W - sum_i V_i H_i) T for the block combination:
// C_i = -H_i T (i <= k) and C_{k+1} = T, in the Krylov precision.
template <typename T>
__global__ void k_make_coef(const double* __restrict__ G, const double* __restrict__ Tm, int k, int r,
                            T* __restrict__ C) {
  pdl_wait();
  pdl_trigger();
  const int rr = r * r;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= (k + 2) * rr) return;
  const int i = o / rr, pq = o % rr, p = pq / r, q = pq % r;
  double v;
  if (i <= k) {
    const double* Hi = G + (size_t)i * rr;
    double acc = 0.0;
    for (int t = 0; t < r; ++t) acc = fma(Hi[p * r + t], Tm[t * r + q], acc);
    v = -acc;
  } else {
    v = Tm[pq];
  }
  C[o] = (T)v;
}

template <typename T>
void launch_make_coef(const double* G, const double* Tm, int k, int r, T* C, cudaStream_t st) {
  count_launch();
  const int n = (k + 2) * r * r;
  launch_pdl(k_make_coef<T>, dim3(nblk(n, 256)), dim3(256), 0, st, G, Tm, k, r, C);
}

// ------------------------------------------------------------ block combine
// out[row][q] = alpha in[row][q] + sum_i sum_p V_i[row][p] C_i[p][q]  (q < r_out;
// 0 for r_out <= q < ldo).  A thread owns RPT rows: it reads each V_i row with
// 16-byte vector loads straight into registers (no staging, no barrier per
// block) and keeps the W outputs of each row in registers; the coefficient
// blocks are staged in shared memory in groups, zero-padded to W x W, and
// read as broadcasts.  The sum runs over i, then p, in a fixed order.  out
// may alias one V block or in: a row is read completely by its own thread
// before that thread writes it.
constexpr int COMB_T = 128;
constexpr size_t COMB_SMEM = 48 * 1024;


template <typename T, int W, int RPT>
__global__ void __launch_bounds__(COMB_T) k_block_combine(T* out, const T* in, T alpha, const T* V, size_t vstride,
                                                          int kblocks, int r_in, const T* __restrict__ C,
                                                          int r_out, int n_rows, int ldv, int ldo, int kgroup) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Cs = reinterpret_cast<T*>(smem_raw);                       // [kgroup][W][W]
  const int base = blockIdx.x * (COMB_T * RPT) + threadIdx.x;
  const int np4 = (r_in + 3) / 4;
  T acc[RPT][W];
#pragma unroll
  for (int s = 0; s < RPT; ++s)
#pragma unroll
    for (int q = 0; q < W; ++q) acc[s][q] = T(0);
  for (int i0 = 0; i0 < kblocks; i0 += kgroup) {
    const int nbk = min(kgroup, kblocks - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < nbk * W * W; e += COMB_T) {
      const int q = e % W, p = (e / W) % W, ib = e / (W * W);
      Cs[e] = (p < r_in && q < r_out) ? C[((size_t)(i0 + ib) * r_in + p) * r_out + q] : T(0);
    }
    __syncthreads();
    for (int ib = 0; ib < nbk; ++ib) {
      const T* Vi = V + (size_t)(i0 + ib) * vstride;
      const T* cb = Cs + (size_t)ib * W * W;
      // every load of this block's rows is issued before the first use, so
      // the thread has all of them in flight at once
      T v[RPT][W];
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const int row = base + s * COMB_T;
#pragma unroll
        for (int p4 = 0; p4 < W / 4; ++p4) {
          if (p4 < np4 && row < n_rows) {
            row_ld4(Vi + (size_t)row * ldv + 4 * p4, &v[s][4 * p4]);
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[s][4 * p4 + e] = T(0);
          }
        }
#pragma unroll
        for (int p = 0; p < W; ++p)
          if (p >= r_in) v[s][p] = T(0);                  // padding columns
      }
#pragma unroll
      for (int p = 0; p < W; ++p) {
        const T* cp = cb + p * W;
#pragma unroll
        for (int q4 = 0; q4 < W / 4; ++q4) {
          T c[4];
          row_ld4(cp + 4 * q4, c);
#pragma unroll
          for (int s = 0; s < RPT; ++s)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[s][4 * q4 + u] = fma(v[s][p], c[u], acc[s][4 * q4 + u]);
        }
      }
    }
  }
  const int ldo4 = ldo / 4;
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int row = base + s * COMB_T;
    if (row >= n_rows) continue;
    T* orow = out + (size_t)row * ldo;
    const T* irow = in ? in + (size_t)row * ldo : nullptr;
#pragma unroll
    for (int q4 = 0; q4 < W / 4; ++q4) {
      if (q4 >= ldo4) break;
      T res[4];
      if (irow) {
        row_ld4(irow + 4 * q4, res);
#pragma unroll
        for (int u = 0; u < 4; ++u) res[u] = alpha * res[u] + acc[s][4 * q4 + u];
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) res[u] = acc[s][4 * q4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (4 * q4 + u >= r_out) res[u] = T(0);
      row_st4(orow + 4 * q4, res);
    }
    const T z[4] = {T(0), T(0), T(0), T(0)};
    for (int q4 = W / 4; q4 < ldo4; ++q4) row_st4(orow + 4 * q4, z);
  }
}

// Staged combination (FP32, W <= 24): a CTA of CB_T threads owns CB_ROWS =
// 2 CB_T consecutive rows and streams that row range of every basis block through a CB_NST-deep ring of
// shared-memory stages, one TMA bulk copy per block (the rows of a block are
// one contiguous span), completion on the stage's mbarrier with the same
// bounded waits as the staged Gram.  A thread owns two rows; the coefficient
// blocks sit in shared memory (zero-padded to W x W) and are read as
// broadcasts.  out may alias a basis block or in: a CTA reads all of its
// rows before writing them.
constexpr size_t CB_COEF_MAX = 96 * 1024;

template <int W, int CB_T, int CB_NST>
__global__ void __launch_bounds__(CB_T) k_combine_staged(float* out, const float* in, float alpha, const float* V,
                                                       size_t vstride, int kblocks, int r_in,
                                                       const float* __restrict__ C, int r_out, int n_rows, int ldv,
                                                       int ldo, int* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char cb_raw[];
  if ((ldv & 3) || (ldo & 3) || (vstride & 3) || (reinterpret_cast<uintptr_t>(V) & 15)) {   // 16-byte copies
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  constexpr int CB_ROWS = 2 * CB_T;
  const unsigned bar0 = smem_u32(cb_raw);
  float* stages = reinterpret_cast<float*>(cb_raw + GS_BAR_BYTES);
  const int stage_floats = CB_ROWS * ldv;
  float* Cs = stages + (size_t)CB_NST * stage_floats;   // [kblocks][W][W]
  const int r0 = blockIdx.x * CB_ROWS;
  const int nr = min(CB_ROWS, n_rows - r0);
  const unsigned bytes = (unsigned)(nr * ldv) * 4u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < CB_NST; ++s) mbar_init(bar0 + 8 * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int b) {                            // thread 0: block b's rows into stage b % CB_NST
    if (b >= kblocks) return;
    const unsigned bar = bar0 + 8 * (b % CB_NST);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, bytes);
    bulk_g2s(smem_u32(stages + (size_t)(b % CB_NST) * stage_floats), V + (size_t)b * vstride + (size_t)r0 * ldv,
             bytes, bar);
  };
  if (threadIdx.x == 0)
    for (int b = 0; b < CB_NST - 1; ++b) issue(b);
  for (int e = threadIdx.x; e < kblocks * W * W; e += CB_T) {
    const int q = e % W, pp = (e / W) % W, ib = e / (W * W);
    Cs[e] = (pp < r_in && q < r_out) ? C[((size_t)ib * r_in + pp) * r_out + q] : 0.f;
  }
  float acc[2][W];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int q = 0; q < W; ++q) acc[s][q] = 0.f;
  const int np4 = (r_in + 3) / 4;
  int ok = 1, waited = 0;
  for (int b = 0; b < kblocks; ++b) {
    const bool landed = mbar_wait_bounded(bar0 + 8 * (b % CB_NST), (unsigned)((b / CB_NST) & 1));
    if (!__syncthreads_and(landed ? 1 : 0)) {        // also: coefficients staged, stage b-1 free
      ok = 0;
      break;
    }
    waited = b + 1;
    if (threadIdx.x == 0) issue(b + CB_NST - 1);
    const float* st = stages + (size_t)(b % CB_NST) * stage_floats;
    const float* cb = Cs + (size_t)b * W * W;
    float v[2][W];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int rr = threadIdx.x + s * CB_T;
#pragma unroll
      for (int p4 = 0; p4 < W / 4; ++p4) {
        if (p4 < np4 && rr < nr) {
          row_ld4(st + (size_t)rr * ldv + 4 * p4, &v[s][4 * p4]);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) v[s][4 * p4 + e] = 0.f;
        }
      }
#pragma unroll
      for (int pp = 0; pp < W; ++pp)
        if (pp >= r_in) v[s][pp] = 0.f;
    }
#pragma unroll
    for (int pp = 0; pp < W; ++pp) {
      const float* cp = cb + pp * W;
#pragma unroll
      for (int q4 = 0; q4 < W / 4; ++q4) {
        float c[4];
        row_ld4(cp + 4 * q4, c);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[s][4 * q4 + u] = fmaf(v[s][pp], c[u], acc[s][4 * q4 + u]);
      }
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) {
      atomicExch(err, 1);
      const int issued = min(kblocks, waited + CB_NST - 1);
      for (int b = waited; b < issued; ++b) mbar_wait_bounded(bar0 + 8 * (b % CB_NST), (unsigned)((b / CB_NST) & 1));
    }
    return;
  }
  const int ldo4 = ldo / 4;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int row = r0 + threadIdx.x + s * CB_T;
    if (row >= n_rows) continue;
    float* orow = out + (size_t)row * ldo;
    const float* irow = in ? in + (size_t)row * ldo : nullptr;
#pragma unroll
    for (int q4 = 0; q4 < W / 4; ++q4) {
      if (q4 >= ldo4) break;
      float res[4];
      if (irow) {
        row_ld4(irow + 4 * q4, res);
#pragma unroll
        for (int u = 0; u < 4; ++u) res[u] = alpha * res[u] + acc[s][4 * q4 + u];
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) res[u] = acc[s][4 * q4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (4 * q4 + u >= r_out) res[u] = 0.f;
      row_st4(orow + 4 * q4, res);
    }
    const float z[4] = {0.f, 0.f, 0.f, 0.f};
    for (int q4 = W / 4; q4 < ldo4; ++q4) row_st4(orow + 4 * q4, z);
  }
}

// CTA width x stage depth of the staged combination: 0 = 256 x 2 (default;
// two CTAs of 8 warps per SM at J = 20, 54.7 us against 62.6 us for 128 x 3 on
// the 128 x 128 cavity), 1 = 128 x 2, 2 = 128 x 3, 3 = 64 x 2 (MHDE_COMB to
// experiment).  A variant whose stages do not fit falls back to 128 x 2.
static int combine_variant() {
  static const int v = [] {
    const char* e = std::getenv("MHDE_COMB");
    const int x = e ? std::atoi(e) : 0;
    return (x >= 0 && x <= 3) ? x : 0;
  }();
  return v;
}

template <int W>
static cudaError_t combine_staged_attr_w() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GS_SMEM);
  };
  set((const void*)k_combine_staged<W, 128, 3>);
  set((const void*)k_combine_staged<W, 128, 2>);
  set((const void*)k_combine_staged<W, 256, 2>);
  set((const void*)k_combine_staged<W, 64, 2>);
  return e;
}

static cudaError_t combine_staged_attr() {
  cudaError_t e = combine_staged_attr_w<4>();
  if (e == cudaSuccess) e = combine_staged_attr_w<8>();
  if (e == cudaSuccess) e = combine_staged_attr_w<12>();
  if (e == cudaSuccess) e = combine_staged_attr_w<16>();
  if (e == cudaSuccess) e = combine_staged_attr_w<20>();
  if (e == cudaSuccess) e = combine_staged_attr_w<24>();
  return e;
}

static size_t combine_staged_smem(int kblocks, int W, int ldv, int nt, int nst) {
  return GS_BAR_BYTES + (size_t)nst * 2 * nt * ldv * sizeof(float) + (size_t)kblocks * W * W * sizeof(float);
}

template <int W, int NT, int NST>
static bool combine_staged_try(float* out, const float* in, float alpha, const float* V, size_t vstride, int kblocks,
                               int r_in, const float* C, int r_out, int n_rows, int ldv, int ldo, cudaStream_t st,
                               int* err) {
  const size_t smem = combine_staged_smem(kblocks, W, ldv, NT, NST);
  if (err == nullptr || (size_t)kblocks * W * W * sizeof(float) > CB_COEF_MAX || smem > GS_SMEM || ldv % 4 != 0 || ldo % 4 != 0 ||
      gram_setup().err != cudaSuccess)
    return false;
  launch_pdl(k_combine_staged<W, NT, NST>, dim3(nblk(n_rows, 2 * NT)), dim3(NT), smem, st, out, in, alpha, V, vstride,
             kblocks, r_in, C, r_out, n_rows, ldv, ldo, err);
  return true;
}

template <typename T, int W>
static void combine_w(T* out, const T* in, T alpha, const T* V, size_t vstride, int kblocks, int r_in,
                      const T* C, int r_out, int n_rows, int ldv, int ldo, cudaStream_t st, int* err,
                      bool allow_tc) {
  if constexpr (sizeof(T) == 4) {
    if (allow_tc && launch_combine_tc(reinterpret_cast<float*>(out), reinterpret_cast<const float*>(in), (float)alpha,
                          reinterpret_cast<const float*>(V), vstride, kblocks, r_in,
                          reinterpret_cast<const float*>(C), r_out, n_rows, ldv, ldo, st, err))
      return;
  }
  if constexpr (sizeof(T) == 4 && W <= 24) {
    float* o = reinterpret_cast<float*>(out);
    const float* i = reinterpret_cast<const float*>(in);
    const float* v = reinterpret_cast<const float*>(V);
    const float* cc = reinterpret_cast<const float*>(C);
    bool done = false;
    const float a = (float)alpha;
    switch (combine_variant()) {
      case 1: break;
      case 2: done = combine_staged_try<W, 128, 3>(o, i, a, v, vstride, kblocks, r_in, cc, r_out, n_rows, ldv, ldo, st, err);
              break;
      case 3: done = combine_staged_try<W, 64, 2>(o, i, a, v, vstride, kblocks, r_in, cc, r_out, n_rows, ldv, ldo, st, err);
              break;
      default: done = combine_staged_try<W, 256, 2>(o, i, a, v, vstride, kblocks, r_in, cc, r_out, n_rows, ldv, ldo, st, err);
    }
    if (!done) done = combine_staged_try<W, 128, 2>(o, i, a, v, vstride, kblocks, r_in, cc, r_out, n_rows, ldv, ldo, st, err);
    if (done) return;
  }
  constexpr int RPT = (sizeof(T) == 4 && W <= 24) ? 2 : 1;
  const size_t per_block = (size_t)W * W * sizeof(T);
  const int kgroup = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::max(kblocks, 1), COMB_SMEM / per_block));
  const size_t shmem = (size_t)kgroup * per_block;
  k_block_combine<T, W, RPT><<<nblk(n_rows, COMB_T * RPT), COMB_T, shmem, st>>>(
      out, in, alpha, V, vstride, kblocks, r_in, C, r_out, n_rows, ldv, ldo, kgroup);
}

cudaError_t init_la_attributes() { return gram_setup().err; }

template <typename T>
void launch_block_combine(T* out, const T* in, T alpha, const T* V, size_t vstride, int kblocks,
                          int r_in, const T* C, int r_out, int n_rows, int ldv, int Jp, cudaStream_t st,
                          int* err, bool allow_tc) {
  count_launch();
  const int w = std::max((r_in + 3) / 4, (r_out + 3) / 4) * 4;
#define MHDE_CW(WV) \
  combine_w<T, WV>(out, in, alpha, V, vstride, kblocks, r_in, C, r_out, n_rows, ldv, Jp, st, err, allow_tc)
  if (w <= 4) MHDE_CW(4);
  else if (w <= 8) MHDE_CW(8);
  else if (w <= 12) MHDE_CW(12);
  else if (w <= 16) MHDE_CW(16);
  else if (w <= 20) MHDE_CW(20);
  else if (w <= 24) MHDE_CW(24);
  else if (w <= 32) MHDE_CW(32);
  else if (w <= 48) MHDE_CW(48);
  else MHDE_CW(64);
#undef MHDE_CW
}

// out[row][q] = (T) sum_p X[row][p] C[p][q] for q < r (0 beyond), X and C in FP64:
// the first Krylov block built from the FP64 residual.
template <typename T, int QMAX>
__global__ void __launch_bounds__(128) k_combine_from_f64(T* __restrict__ out, const double* __restrict__ X,
                                                          const double* __restrict__ C, int J, int r,
                                                          int n_rows, int Jp, int ldo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Cs = reinterpret_cast<double*>(smem_raw);   // [J][QMAX]
  for (int e = threadIdx.x; e < J * QMAX; e += blockDim.x) {
    int q = e % QMAX, p = e / QMAX;
    Cs[e] = q < r ? C[(size_t)p * r + q] : 0.0;
  }
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_rows) return;
  double acc[QMAX];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) acc[q] = 0.0;
  const double* xr = X + (size_t)row * Jp;
  for (int p = 0; p < J; ++p) {
    const double v = xr[p];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) acc[q] += v * Cs[p * QMAX + q];
  }
  T* orow = out + (size_t)row * ldo;
#pragma unroll
  for (int q = 0; q < QMAX; ++q)
    if (q < ldo) orow[q] = q < r ? (T)acc[q] : T(0);
  for (int q = QMAX; q < ldo; ++q) orow[q] = T(0);
}

template <typename T>
void launch_combine_from_f64(T* out, const double* X, const double* C, int J, int r, int n_rows, int Jp,
                             int ldo, cudaStream_t st) {
  count_launch();
#define MHDE_CF(Q)                                                                                     \
  k_combine_from_f64<T, Q><<<nblk(n_rows, 128), 128, (size_t)J * Q * sizeof(double), st>>>(out, X, C, J, r, \
                                                                                           n_rows, Jp, ldo)
  if (r <= 8)
    MHDE_CF(8);
  else if (r <= 16)
    MHDE_CF(16);
  else if (r <= 24)
    MHDE_CF(24);
  else if (r <= 32)
    MHDE_CF(32);
  else
    MHDE_CF(64);
#undef MHDE_CF
}

// ------------------------------------------------------------ column norms, conversions
template <typename T>
__global__ void k_colsq(const T* __restrict__ X, int n_rows, int Jp, int rows_per_chunk,
                        double* __restrict__ out) {
  extern __shared__ double sh[];
  int G = blockDim.x / Jp;
  int j = threadIdx.x % Jp, g = threadIdx.x / Jp;
  int r0 = blockIdx.x * rows_per_chunk, r1 = min(n_rows, r0 + rows_per_chunk);
  double s = 0.0;
  if (g < G)
    for (int row = r0 + g; row < r1; row += G) {
      double x = (double)X[(size_t)row * Jp + j];
      s += x * x;
    }
  if (g < G) sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < Jp) {
    double t = 0.0;
    for (int h = 0; h < G; ++h) t += sh[h * Jp + threadIdx.x];
    out[(size_t)blockIdx.x * Jp + threadIdx.x] = t;
  }
}

template <typename T>
void launch_colsq(const T* X, int n_rows, int Jp, int nchunk, double* out, cudaStream_t st) {
  count_launch();
  int rows_per_chunk = (n_rows + nchunk - 1) / nchunk;
  int threads = (256 / Jp) * Jp;
  k_colsq<T><<<nchunk, threads, threads * sizeof(double), st>>>(X, n_rows, Jp, rows_per_chunk, out);
}

template <typename T>
__global__ void k_scale_to(const double* __restrict__ x, const double* __restrict__ scale,
                           T* __restrict__ y, size_t n, int Jp) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = (T)(x[i] * scale[i % Jp]);
}

template <typename T>
void launch_scale_to(const double* x, const double* scale, T* y, size_t n, int Jp, cudaStream_t st) {
  count_launch();
  k_scale_to<T><<<nblk((long long)n, 256), 256, 0, st>>>(x, scale, y, n, Jp);
}

template <typename T>
__global__ void k_axpy_from(const T* __restrict__ d, const double* __restrict__ scale,
                            double* __restrict__ x, size_t n, int Jp) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] += (double)d[i] * scale[i % Jp];
}

template <typename T>
void launch_axpy_from(const T* d, const double* scale, double* x, size_t n, int Jp, cudaStream_t st) {
  count_launch();
  k_axpy_from<T><<<nblk((long long)n, 256), 256, 0, st>>>(d, scale, x, n, Jp);
}

template <typename T>
__global__ void k_axpby(T* __restrict__ out, T a, const T* __restrict__ x, T b, const T* __restrict__ y,
                        size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}

template <typename T>
void launch_axpby(T* out, T a, const T* x, T b, const T* y, size_t n, cudaStream_t st) {
  count_launch();
  k_axpby<T><<<nblk((long long)n, 256), 256, 0, st>>>(out, a, x, b, y, n);
}

__global__ void k_d2f(const double* __restrict__ x, float* __restrict__ y, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

void launch_d2f(const double* x, float* y, size_t n, cudaStream_t st) {
  count_launch();
  k_d2f<<<nblk((long long)n, 256), 256, 0, st>>>(x, y, n);
}

// explicit instantiations
#define MHDE_INST(T)                                                                                 \
  template void launch_saddle_spmm<T>(const mhde_ctx*, const T*, const T*, const T*, const T*,       \
                                      const double*, T*, int, int, cudaStream_t);                    \
  template void launch_csr<T>(int, const int*, const int*, const T*, const T*, T, const T*, const T*, \
                              T*, int, int, cudaStream_t);                                           \
  template void launch_dense_apply<T>(int, const T*, const T*, T*, int, cudaStream_t);               \
  template void launch_jacobi_F<T>(const mhde_ctx*, const T*, const T*, T, const T*, const T*, T*,   \
                                   int, cudaStream_t);                                               \
  template void launch_precond_p<T>(int, int, const T*, const T*, const T*, T, T, const int*, const int*,  \
                                    const T*, T*, cudaStream_t);                                        \
  template void launch_bt_apply<T>(const mhde_ctx*, const T*, const T*, const T*, T*, int, cudaStream_t); \
  template void launch_block_jacobi<T>(int, int, const int*, const T*, T, const T*, const T*, T*, int,      \
                                      cudaStream_t);                                                   \
  template void launch_lsc_middle<T>(const mhde_ctx*, const T*, const T*, const T*, const T*, const T*, T*, \
                                     T*, T*, int, cudaStream_t);                                        \
  template void launch_gram<T>(const T*, size_t, int, const T*, int, int, int, int, double*, double*, \
                               cudaStream_t, bool, int*, bool);                                      \
  template void launch_make_coef<T>(const double*, const double*, int, int, T*, cudaStream_t);       \
  template void launch_block_combine<T>(T*, const T*, T, const T*, size_t, int, int, const T*, int,  \
                                        int, int, int, cudaStream_t, int*, bool);                    \
  template void launch_colsq<T>(const T*, int, int, int, double*, cudaStream_t);                     \
  template void launch_scale_to<T>(const double*, const double*, T*, size_t, int, cudaStream_t);     \
  template void launch_axpy_from<T>(const T*, const double*, double*, size_t, int, cudaStream_t);     \
  template void launch_axpby<T>(T*, T, const T*, T, const T*, size_t, cudaStream_t);               \
  template void launch_combine_from_f64<T>(T*, const double*, const double*, int, int, int, int,     \
                                           int, cudaStream_t);
MHDE_INST(double)
MHDE_INST(float)

}  // namespace mhde
