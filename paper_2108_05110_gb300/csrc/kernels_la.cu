// Linear-algebra kernels of the shared-matrix block solve (Section 1: one
// matrix A for all J right-hand sides, A [x_1 | ... | x_J] = [b_1 | ... | b_J],
// solved with block linear solvers).  Every multi-vector is row-major
// [rows][Jp]; a thread owns one 16-byte chunk of one row (2 doubles or 4
// floats), so the J-wide rows that a sparse row gathers are read as
// contiguous, coalesced vector loads and the matrix values / column indices of
// a row are broadcast to the threads sharing that row.
#include <algorithm>
#include <cstdint>

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
    k_saddle<T, 0><<<nblk(n, bs), bs, 0, st>>>(c->fe.n2, c->fe.np, nch, c->F.rowptr, c->F.col, Fval,
                                              c->BT.rowptr, c->BT.col, BTval, c->B.rowptr, c->B.col,
                                              Bval, c->d_isbnd, X, Bvec, Y);
  else
    k_saddle<T, 1><<<nblk(n, bs), bs, 0, st>>>(c->fe.n2, c->fe.np, nch, c->F.rowptr, c->F.col, Fval,
                                              c->BT.rowptr, c->BT.col, BTval, c->B.rowptr, c->B.col,
                                              Bval, c->d_isbnd, X, Bvec, Y);
}

// ------------------------------------------------------------ generic CSR
template <typename T>
__global__ void k_csr(int nrows, int nch, const int* __restrict__ rp, const int* __restrict__ col,
                      const T* __restrict__ val, const T* __restrict__ dinv, T omega,
                      const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ y, int mode) {
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
  } else {
    yv[o] = vaxpby(T(1), yv[o], T(1), acc);
  }
}

template <typename T>
void launch_csr(int nrows, const int* rowptr, const int* col, const T* val, const T* dinv, T omega,
                const T* x, const T* b, T* y, int mode, int Jp, cudaStream_t st) {
  count_launch();
  int nch = Jp / Vec<T>::W;
  long long n = (long long)nrows * nch;
  k_csr<T><<<nblk(n, 256), 256, 0, st>>>(nrows, nch, rowptr, col, val, dinv, omega, x, b, y, mode);
}

template <typename T>
__global__ void k_dense_apply(int n, int nch, const T* __restrict__ A, const T* __restrict__ x,
                              T* __restrict__ y) {
  using V = typename Vec<T>::type;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n * nch) return;
  int r = (int)(tid / nch), ch = (int)(tid % nch);
  const V* xv = reinterpret_cast<const V*>(x);
  V acc = vzero(V());
  for (int k = 0; k < n; ++k) vfma(acc, A[(size_t)r * n + k], xv[(size_t)k * nch + ch]);
  reinterpret_cast<V*>(y)[(size_t)r * nch + ch] = acc;
}

template <typename T>
void launch_dense_apply(int n, const T* Ainv, const T* x, T* y, int Jp, cudaStream_t st) {
  count_launch();
  int nch = Jp / Vec<T>::W;
  long long m = (long long)n * nch;
  k_dense_apply<T><<<nblk(m, 128), 128, 0, st>>>(n, nch, Ainv, x, y);
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
  k_precond_p<T><<<nblk(n, 256), 256, 0, st>>>(np, nch, x, rp, mp, inv_dt, nu_hat, nrp, ncol, Np, zp);
}

template <typename T>
__global__ void k_bt_apply(int n2, int nch, const int* __restrict__ rp, const int* __restrict__ col,
                           const T* __restrict__ BT, const unsigned char* __restrict__ isbnd,
                           const T* __restrict__ ru, const T* __restrict__ zp, T* __restrict__ tu) {
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
  k_bt_apply<T><<<nblk(n, 256), 256, 0, st>>>(c->fe.n2, nch, c->BT.rowptr, c->BT.col, BTval, c->d_isbnd,
                                             ru, zp, tu);
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

// One warp per output entry: lanes stride over the chunks, then a fixed
// butterfly of shuffles (deterministic order).
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

__global__ void k_gram_reduce(int nchunk, int total, const double* __restrict__ part,
                              double* __restrict__ gram) {
  const int o = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (o >= total) return;
  double s = 0.0;
  for (int c = lane; c < nchunk; c += 32) s += part[(size_t)c * total + o];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) gram[o] = s;
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

template <typename T>
void launch_gram(const T* V, size_t vstride, int kblocks, const T* W, int n_rows, int Jp, int r,
                 int nchunk, double* part, double* gram, cudaStream_t st) {
  count_launch(2);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_gram<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    attr_set = true;
  }
  int rows_per_chunk = (n_rows + nchunk - 1) / nchunk;
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
  int total = kblocks * r * r;
  k_gram_reduce<<<(total + 7) / 8, 256, 0, st>>>(nchunk, total, part, gram);
}

// ------------------------------------------------------------ block combine
// out[row][q] = alpha in[row][q] + sum_i sum_p V_i[row][p] C_i[p][q].
// A CTA owns 128 consecutive rows: each block's 128 x r_in tile is staged in
// shared memory with coalesced loads (odd row pitch: no bank conflicts),
// coefficient blocks are staged in groups and read as broadcasts, and a
// thread accumulates the QMAX outputs of its row in registers.  out may alias
// one of the V blocks (each row is read completely before it is written).
constexpr int COMB_T = 128;

template <typename T, int QMAX>
__global__ void __launch_bounds__(COMB_T) k_block_combine(T* out, const T* in, T alpha, const T* V, size_t vstride,
                                                          int kblocks, int r_in, const T* __restrict__ C, int r_out,
                                                          int n_rows, int ldv, int Jp, int kgroup, int pitch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Cs = reinterpret_cast<T*>(smem_raw);                       // [kgroup][r_in][QMAX]
  T* Vt = Cs + (size_t)kgroup * r_in * QMAX;                    // [COMB_T][pitch]
  const int row0 = blockIdx.x * COMB_T;
  const int row = row0 + threadIdx.x;
  T acc[QMAX];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) acc[q] = T(0);
  for (int i0 = 0; i0 < kblocks; i0 += kgroup) {
    const int nbk = min(kgroup, kblocks - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < nbk * r_in * QMAX; e += COMB_T) {
      const int q = e % QMAX, pi = e / QMAX;
      const int ib = pi / r_in, p = pi % r_in;
      Cs[e] = (q < r_out) ? C[((size_t)(i0 + ib) * r_in + p) * r_out + q] : T(0);
    }
    for (int ib = 0; ib < nbk; ++ib) {
      __syncthreads();
      const T* Vi = V + (size_t)(i0 + ib) * vstride;
      for (int e = threadIdx.x; e < COMB_T * r_in; e += COMB_T) {
        const int rr = e / r_in, p = e % r_in;
        Vt[rr * pitch + p] = (row0 + rr < n_rows) ? Vi[(size_t)(row0 + rr) * ldv + p] : T(0);
      }
      __syncthreads();
      const T* cb = Cs + (size_t)ib * r_in * QMAX;
      const T* vr = Vt + threadIdx.x * pitch;
      for (int p = 0; p < r_in; ++p) {
        const T v = vr[p];
        const T* cp = cb + p * QMAX;
#pragma unroll
        for (int q = 0; q < QMAX; ++q) acc[q] += v * cp[q];
      }
    }
  }
  if (row >= n_rows) return;
  T* orow = out + (size_t)row * Jp;
  const T* irow = in ? in + (size_t)row * Jp : nullptr;
  T res[QMAX];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) res[q] = (q < r_out) ? (irow ? alpha * irow[q] : T(0)) + acc[q] : T(0);
#pragma unroll
  for (int q = 0; q < QMAX; ++q)
    if (q < Jp) orow[q] = res[q];
  for (int q = QMAX; q < Jp; ++q) orow[q] = T(0);
}

template <typename T, int QMAX>
static void combine_q(T* out, const T* in, T alpha, const T* V, size_t vstride, int kblocks, int r_in,
                      const T* C, int r_out, int n_rows, int ldv, int Jp, cudaStream_t st) {
  const int pitch = (r_in % 2 == 0) ? r_in + 1 : r_in + 2;
  const size_t per_block = (size_t)r_in * QMAX * sizeof(T);
  int kgroup = (int)std::max<size_t>(1, (32 * 1024) / std::max<size_t>(per_block, 1));
  kgroup = std::min(kgroup, std::max(kblocks, 1));
  const size_t shmem = (size_t)kgroup * per_block + (size_t)COMB_T * pitch * sizeof(T);
  k_block_combine<T, QMAX><<<nblk(n_rows, COMB_T), COMB_T, shmem, st>>>(out, in, alpha, V, vstride, kblocks, r_in, C,
                                                                       r_out, n_rows, ldv, Jp, kgroup, pitch);
}

template <typename T>
static cudaError_t combine_attr() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  };
  set((const void*)k_block_combine<T, 4>);
  set((const void*)k_block_combine<T, 8>);
  set((const void*)k_block_combine<T, 16>);
  set((const void*)k_block_combine<T, 24>);
  set((const void*)k_block_combine<T, 32>);
  set((const void*)k_block_combine<T, 48>);
  set((const void*)k_block_combine<T, 64>);
  return e;
}

cudaError_t init_la_attributes() {
  cudaError_t e = combine_attr<float>();
  if (e != cudaSuccess) return e;
  return combine_attr<double>();
}

template <typename T>
void launch_block_combine(T* out, const T* in, T alpha, const T* V, size_t vstride, int kblocks,
                          int r_in, const T* C, int r_out, int n_rows, int ldv, int Jp, cudaStream_t st) {
  count_launch();
  if (r_out <= 4)
    combine_q<T, 4>(out, in, alpha, V, vstride, kblocks, r_in, C, r_out, n_rows, ldv, Jp, st);
  else if (r_out <= 8)
    combine_q<T, 8>(out, in, alpha, V, vstride, kblocks, r_in, C, r_out, n_rows, ldv, Jp, st);
  else if (r_out <= 16)
    combine_q<T, 16>(out, in, alpha, V, vstride, kblocks, r_in, C, r_out, n_rows, ldv, Jp, st);
  else if (r_out <= 24)
    combine_q<T, 24>(out, in, alpha, V, vstride, kblocks, r_in, C, r_out, n_rows, ldv, Jp, st);
  else if (r_out <= 32)
    combine_q<T, 32>(out, in, alpha, V, vstride, kblocks, r_in, C, r_out, n_rows, ldv, Jp, st);
  else if (r_out <= 48)
    combine_q<T, 48>(out, in, alpha, V, vstride, kblocks, r_in, C, r_out, n_rows, ldv, Jp, st);
  else
    combine_q<T, 64>(out, in, alpha, V, vstride, kblocks, r_in, C, r_out, n_rows, ldv, Jp, st);
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
  template void launch_gram<T>(const T*, size_t, int, const T*, int, int, int, int, double*, double*, \
                               cudaStream_t);                                                        \
  template void launch_block_combine<T>(T*, const T*, T, const T*, size_t, int, int, const T*, int,  \
                                        int, int, int, cudaStream_t);                                \
  template void launch_colsq<T>(const T*, int, int, int, double*, cudaStream_t);                     \
  template void launch_scale_to<T>(const double*, const double*, T*, size_t, int, cudaStream_t);     \
  template void launch_axpy_from<T>(const T*, const double*, double*, size_t, int, cudaStream_t);     \
  template void launch_axpby<T>(T*, T, const T*, T, const T*, size_t, cudaStream_t);               \
  template void launch_combine_from_f64<T>(T*, const double*, const double*, int, int, int, int,     \
                                           int, cudaStream_t);
MHDE_INST(double)
MHDE_INST(float)

}  // namespace mhde
