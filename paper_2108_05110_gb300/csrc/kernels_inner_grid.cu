// Inner GMRES(k) on F D^{-1} of the mixed path as ONE persistent kernel.
//
// Same method as the launch chain of kernels_inner.cu (per-column GMRES(k)
// with Jacobi right preconditioning and a fixed step count, the velocity
// block's approximate inverse inside the block-triangular preconditioner,
// Section 1 block solvers): per step w = F D^{-1} v_i, one classical
// Gram-Schmidt pass against v_0..v_i with the norm from the Pythagorean
// identity, v_{i+1} = (w - sum_l h_l v_l) / ||.||; then per column the
// (k+1) x k least-squares problem and z = D^{-1} sum_l y_l v_l.  What
// changes is the execution: the chain of ~4k+3 dependent launches (each a
// few microseconds of launch, ramp-up and tail on L2-resident vectors)
// becomes one cooperative launch whose CTAs own contiguous row ranges and
// meet at grid barriers:
//
//   step 0:  w' = F D^{-1} r with r.r, r.w', w'.w' partial sums | reduce |
//            v_0 = r / beta, v_1 = (w'/beta - h_00 v_0) / h_10          |
//   step i:  w = F D^{-1} v_i with v_l.w (l <= i), w.w partial sums      |
//            reduce | v_{i+1} = (w - sum_l h_l v_l) / h_{i+1,i}          |
//   end:     every CTA solves the C small least-squares problems itself
//            and writes z for its own rows (no barrier)
//
// 3k - 1 barriers for k steps instead of 4k + 3 launches.  Sums are
// deterministic: per-thread partials over a fixed row set, CTA sums over
// row groups in a fixed order, grid sums over the CTAs in a fixed order (the
// grid size is fixed per context).  w for a row chunk is produced and
// consumed by the same thread; basis rows of other CTAs are read only after
// the barrier that follows their writes, and nothing written during the
// launch is read through the non-coherent path.
//
// Co-residency of all CTAs is what the cooperative launch attribute
// guarantees; every barrier wait is still bounded: past IG_SPIN_LIMIT polls
// (or when another CTA has already given up) a CTA records the failure in
// the subproblem's error word and leaves, so a failed launch ends with an
// error status the host reads after the solve instead of hanging.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "kernels.h"

namespace mhde {

namespace {

constexpr int IG_T = 512;                       // threads per CTA
constexpr long long IG_SPIN_LIMIT = 1ll << 19;  // polls of one barrier (well under a second)
constexpr int IG_ERR = 4;                       // error-word bit of a barrier that gave up

struct IgArgs {
  int n2, C, nch, kin;
  const int* rowptr;     // F pattern (read-only)
  const int* col;
  const float* FD;       // F D^{-1} values
  const float* dinv;     // D^{-1}
  const int* row_start;  // [P + 1] first row of every CTA
  const float* r;        // input [n2][C]
  float* z;              // output [n2][C]
  float* w;              // operator output [n2][C]
  float* V;              // basis v_0..v_{k-1}, vstride apart
  size_t vstride;
  double* part;          // per-CTA partial sums [(slot C + col) P + cta]
  double* red;           // grid sums [slot C + col]
  double* H;             // Hessenberg [(l k + j) C + col], written by CTA 0
  unsigned* bar;         // [0] arrivals, [1] exits (zero between launches)
  int* err;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

__device__ __forceinline__ void fma4(float4& a, float s, const float4& x) {
  a.x = fmaf(s, x.x, a.x);
  a.y = fmaf(s, x.y, a.y);
  a.z = fmaf(s, x.z, a.z);
  a.w = fmaf(s, x.w, a.w);
}
__device__ __forceinline__ float4 ld4(const float* p, size_t i4) { return reinterpret_cast<const float4*>(p)[i4]; }
__device__ __forceinline__ void st4(float* p, size_t i4, const float4& v) { reinterpret_cast<float4*>(p)[i4] = v; }
__device__ __forceinline__ float comp(const float4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }

// The n-th barrier of a launch waits for n * P arrivals (the counter only
// grows during a launch).  Thread 0 publishes the CTA's writes (fence, then
// the arrival), polls with acquire loads, and the CTA barrier passes the
// ordering on to the other threads.  Returns false on every thread when the
// wait gave up or another CTA has.
__device__ bool grid_barrier(const IgArgs& a, unsigned target, int* sflag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(a.bar, 1u);
    long long it = 0;
    while (ld_acquire_gpu(a.bar) < target) {
      if ((++it & 63) == 0) {
        if (ld_volatile(a.err) != 0) {
          ok = 0;
          break;
        }
        if (it > IG_SPIN_LIMIT) {
          atomicOr(a.err, IG_ERR);
          ok = 0;
          break;
        }
      }
      __nanosleep(32);
    }
    __threadfence();
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

// The last CTA to leave resets the counters for the next launch on the
// stream: every other CTA has passed its last barrier by then.
__device__ void grid_exit(const IgArgs& a) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.bar + 1, 1u) == gridDim.x - 1) {
      atomicExch(a.bar, 0u);
      atomicExch(a.bar + 1, 0u);
    }
  }
}

// one row chunk of x (4 columns) times row `row` of F D^{-1}; four gathers in flight
__device__ __forceinline__ float4 spmm_chunk(const IgArgs& a, const float* x, int row, int ch) {
  float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
  int k = __ldg(a.rowptr + row);
  const int e = __ldg(a.rowptr + row + 1);
  const size_t nch = (size_t)a.nch;
  for (; k + 3 < e; k += 4) {
    const int c0 = __ldg(a.col + k), c1 = __ldg(a.col + k + 1), c2 = __ldg(a.col + k + 2), c3 = __ldg(a.col + k + 3);
    const float f0 = __ldg(a.FD + k), f1 = __ldg(a.FD + k + 1), f2 = __ldg(a.FD + k + 2), f3 = __ldg(a.FD + k + 3);
    const float4 x0 = ld4(x, c0 * nch + ch), x1 = ld4(x, c1 * nch + ch), x2 = ld4(x, c2 * nch + ch),
                 x3 = ld4(x, c3 * nch + ch);
    fma4(s0, f0, x0);
    fma4(s1, f1, x1);
    fma4(s0, f2, x2);
    fma4(s1, f3, x3);
  }
  for (; k < e; ++k) fma4(s0, __ldg(a.FD + k), ld4(x, __ldg(a.col + k) * nch + ch));
  return make_float4(s0.x + s1.x, s0.y + s1.y, s0.z + s1.z, s0.w + s1.w);
}

// Row-group partial buffers: one per output slot when they fit (the slots are
// then summed by all threads at once), else two used in turn.
template <int KB>
constexpr int ig_nbuf() {
  return KB <= 6 ? KB + 2 : 2;
}

// Shared memory of a CTA (C columns, KB = largest step count of the instantiation)
struct IgShared {
  double* sred;    // [(KB+2) C] grid sums of the current step
  double* slast;   // [(KB+1) C] newest Hessenberg column (h_l, then the norm)
  double* sbeta;   // [C]
  float* sh;       // [(KB+1) C] Gram-Schmidt coefficients of the current step
  float* sinv;     // [C] inverse norms
  float* sib;      // [C] 1 / beta
  float* sy;       // [KB C] least-squares solutions
  float* sbuf;     // [NB][G C] row-group partials (NB slots, see ig_nbuf)
  int* sflag;
};

template <int KB>
__device__ IgShared carve(unsigned char* base, int C, int G) {
  IgShared m;
  double* d = reinterpret_cast<double*>(base);
  m.sred = d;
  m.slast = m.sred + (size_t)(KB + 2) * C;
  m.sbeta = m.slast + (size_t)(KB + 1) * C;
  float* f = reinterpret_cast<float*>(m.sbeta + C);
  m.sh = f;
  m.sinv = m.sh + (size_t)(KB + 1) * C;
  m.sib = m.sinv + C;
  m.sy = m.sib + C;
  m.sbuf = m.sy + (size_t)KB * C;
  m.sflag = reinterpret_cast<int*>(m.sbuf + (size_t)ig_nbuf<KB>() * G * C);
  return m;
}

template <int KB>
size_t ig_smem_bytes(int C, int G) {
  return sizeof(double) * ((size_t)(KB + 2) * C + (size_t)(KB + 1) * C + C) +
         sizeof(float) * ((size_t)(KB + 1) * C + 2 * (size_t)C + (size_t)KB * C + (size_t)ig_nbuf<KB>() * G * C) + 16;
}

// CTA partial sums of nout slots (slot o < nout - 1: d[o], slot nout - 1:
// dn) -> part[(o C + col) P + cta]; the G row groups are added in order
// (four interleaved partial sums, combined in a fixed order)
__device__ __forceinline__ float group_sum(const float* bb, int G, int C) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int h = 0;
  for (; h + 3 < G; h += 4) {
    s0 += bb[(size_t)h * C];
    s1 += bb[(size_t)(h + 1) * C];
    s2 += bb[(size_t)(h + 2) * C];
    s3 += bb[(size_t)(h + 3) * C];
  }
  for (; h < G; ++h) s0 += bb[(size_t)h * C];
  return (s0 + s1) + (s2 + s3);
}

template <int KB>
__device__ void cta_partials(const IgArgs& a, const IgShared& m, int G, int g, int ch, bool act, int nout,
                             const float (&d)[KB + 1][4], const float (&dn)[4]) {
  const int C = a.C, P = gridDim.x;
  constexpr int NB = ig_nbuf<KB>();
  auto slot_value = [&](int o) {
    if (o == nout - 1) return make_float4(dn[0], dn[1], dn[2], dn[3]);
    const int l = o < KB + 1 ? o : 0;
    return make_float4(d[l][0], d[l][1], d[l][2], d[l][3]);
  };
  if constexpr (NB >= KB + 2) {
    if (act) {
#pragma unroll
      for (int o = 0; o < KB + 2; ++o)
        if (o < nout) reinterpret_cast<float4*>(m.sbuf + ((size_t)o * G + g) * C)[ch] = slot_value(o);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nout * C; e += blockDim.x) {
      const int o = e / C, cc = e - o * C;
      a.part[((size_t)o * C + cc) * P + blockIdx.x] = (double)group_sum(m.sbuf + (size_t)o * G * C + cc, G, C);
    }
  } else {
#pragma unroll
    for (int o = 0; o < KB + 2; ++o) {
      if (o < nout) {
        float* bb = m.sbuf + (size_t)(o & 1) * G * C;
        if (act) reinterpret_cast<float4*>(bb + (size_t)g * C)[ch] = slot_value(o);
        __syncthreads();
        for (int cc = threadIdx.x; cc < C; cc += blockDim.x)
          a.part[((size_t)o * C + cc) * P + blockIdx.x] = (double)group_sum(bb + cc, G, C);
      }
    }
  }
}

// grid sums of nout * C outputs, one warp per output, CTAs in a fixed order
__device__ void grid_reduce(const IgArgs& a, int nout) {
  const int P = gridDim.x, nw = blockDim.x >> 5, wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = nout * a.C;
  for (int o = blockIdx.x * nw + wp; o < n; o += P * nw) {
    double s = 0.0;
    const double* src = a.part + (size_t)o * P;
    for (int p = lane; p < P; p += 32) s += src[p];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) a.red[o] = s;
  }
}

template <int KB>
__global__ void __launch_bounds__(IG_T, 2) k_inner_grid(IgArgs a) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char ig_raw[];
  const int C = a.C, nch = a.nch, kin = a.kin;
  const int G = IG_T / nch;
  const int g = threadIdx.x / nch, ch = threadIdx.x - g * nch;
  const bool act = g < G;
  const IgShared m = carve<KB>(ig_raw, C, G);
  const int r0 = __ldg(a.row_start + blockIdx.x), r1 = __ldg(a.row_start + blockIdx.x + 1);
  const unsigned P = gridDim.x;
  unsigned nbar = 0;
  float d[KB + 1][4];
  float dn[4];

  // ---- step 0: w' = F D^{-1} r and the sums r.r, r.w', w'.w'
#pragma unroll
  for (int l = 0; l < KB + 1; ++l)
#pragma unroll
    for (int q = 0; q < 4; ++q) d[l][q] = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) dn[q] = 0.f;
  if (act) {
    for (int row = r0 + g; row < r1; row += G) {
      const size_t o4 = (size_t)row * nch + ch;
      const float4 wv = spmm_chunk(a, a.r, row, ch);
      st4(a.w, o4, wv);
      const float4 rv = __ldg(reinterpret_cast<const float4*>(a.r) + o4);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        d[0][q] = fmaf(comp(rv, q), comp(rv, q), d[0][q]);
        d[1][q] = fmaf(comp(rv, q), comp(wv, q), d[1][q]);
        dn[q] = fmaf(comp(wv, q), comp(wv, q), dn[q]);
      }
    }
  }
  cta_partials<KB>(a, m, G, g, ch, act, 3, d, dn);
  if (!grid_barrier(a, ++nbar * P, m.sflag)) goto out;
  grid_reduce(a, 3);
  if (!grid_barrier(a, ++nbar * P, m.sflag)) goto out;
  for (int e = threadIdx.x; e < 3 * C; e += blockDim.x) m.sred[e] = a.red[e];
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const double rr = m.sred[c], rw = m.sred[C + c], ww = m.sred[2 * C + c];
    const double beta = rr > 0.0 ? sqrt(rr) : 0.0;
    const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
    const double h00 = rw * ib * ib;
    const double n2v = ww * ib * ib - h00 * h00;
    const double nrm = n2v > 0.0 ? sqrt(n2v) : 0.0;
    m.sbeta[c] = beta;
    m.sib[c] = (float)ib;
    m.sh[c] = (float)h00;
    m.sinv[c] = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
    m.slast[c] = h00;
    m.slast[C + c] = nrm;
    if (blockIdx.x == 0) {
      a.H[(size_t)0 * C + c] = h00;
      a.H[(size_t)kin * C + c] = nrm;
    }
  }
  __syncthreads();
  if (act) {
    for (int row = r0 + g; row < r1; row += G) {
      const size_t o4 = (size_t)row * nch + ch;
      const float4 rv = __ldg(reinterpret_cast<const float4*>(a.r) + o4);
      const float4 ib = reinterpret_cast<const float4*>(m.sib)[ch];
      const float4 v0 = make_float4(rv.x * ib.x, rv.y * ib.y, rv.z * ib.z, rv.w * ib.w);
      st4(a.V, o4, v0);
      if (kin > 1) {
        const float4 wv = ld4(a.w, o4);
        const float4 h = reinterpret_cast<const float4*>(m.sh)[ch];
        const float4 iv = reinterpret_cast<const float4*>(m.sinv)[ch];
        const float4 v1 = make_float4((wv.x * ib.x - h.x * v0.x) * iv.x, (wv.y * ib.y - h.y * v0.y) * iv.y,
                                      (wv.z * ib.z - h.z * v0.z) * iv.z, (wv.w * ib.w - h.w * v0.w) * iv.w);
        st4(a.V + a.vstride, o4, v1);
      }
    }
  }

  // ---- steps 1 .. kin-1
  for (int i = 1; i < kin; ++i) {
    if (!grid_barrier(a, ++nbar * P, m.sflag)) goto out;
    const float* vi = a.V + (size_t)i * a.vstride;
#pragma unroll
    for (int l = 0; l < KB + 1; ++l)
#pragma unroll
      for (int q = 0; q < 4; ++q) d[l][q] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) dn[q] = 0.f;
    if (act) {
      // operator pass, then the dot pass over the same row chunks (w re-read
      // by the thread that wrote it), so that the gathers and the dot
      // accumulators are not live at the same time
      for (int row = r0 + g; row < r1; row += G) st4(a.w, (size_t)row * nch + ch, spmm_chunk(a, vi, row, ch));
      for (int row = r0 + g; row < r1; row += G) {
        const size_t o4 = (size_t)row * nch + ch;
        const float4 wv = ld4(a.w, o4);
#pragma unroll
        for (int l = 0; l < KB + 1; ++l) {
          if (l <= i) {
            const float4 vl = ld4(a.V + (size_t)l * a.vstride, o4);
#pragma unroll
            for (int q = 0; q < 4; ++q) d[l][q] = fmaf(comp(vl, q), comp(wv, q), d[l][q]);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) dn[q] = fmaf(comp(wv, q), comp(wv, q), dn[q]);
      }
    }
    cta_partials<KB>(a, m, G, g, ch, act, i + 2, d, dn);
    if (!grid_barrier(a, ++nbar * P, m.sflag)) goto out;
    grid_reduce(a, i + 2);
    if (!grid_barrier(a, ++nbar * P, m.sflag)) goto out;
    for (int e = threadIdx.x; e < (i + 2) * C; e += blockDim.x) m.sred[e] = a.red[e];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      double ss = 0.0;
      for (int l = 0; l <= i; ++l) {
        const double h = m.sred[(size_t)l * C + c];
        ss += h * h;
        m.sh[(size_t)l * C + c] = (float)h;
        m.slast[(size_t)l * C + c] = h;
        if (blockIdx.x == 0) a.H[((size_t)l * kin + i) * C + c] = h;
      }
      const double n2v = m.sred[(size_t)(i + 1) * C + c] - ss;
      const double nrm = n2v > 0.0 ? sqrt(n2v) : 0.0;
      m.sinv[c] = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
      m.slast[(size_t)(i + 1) * C + c] = nrm;
      if (blockIdx.x == 0) a.H[((size_t)(i + 1) * kin + i) * C + c] = nrm;
    }
    __syncthreads();
    if (i + 1 < kin && act) {
      float* vn = a.V + (size_t)(i + 1) * a.vstride;
      const float4 iv = reinterpret_cast<const float4*>(m.sinv)[ch];
      for (int row = r0 + g; row < r1; row += G) {
        const size_t o4 = (size_t)row * nch + ch;
        float4 acc = ld4(a.w, o4);
        for (int l = 0; l <= i; ++l) {
          const float4 vl = ld4(a.V + (size_t)l * a.vstride, o4);
          const float4 h = reinterpret_cast<const float4*>(m.sh + (size_t)l * C)[ch];
          acc.x = fmaf(-h.x, vl.x, acc.x);
          acc.y = fmaf(-h.y, vl.y, acc.y);
          acc.z = fmaf(-h.z, vl.z, acc.z);
          acc.w = fmaf(-h.w, vl.w, acc.w);
        }
        st4(vn, o4, make_float4(acc.x * iv.x, acc.y * iv.y, acc.z * iv.z, acc.w * iv.w));
      }
    }
  }

  // ---- per-column least squares min || beta e_1 - H y || (Givens), every
  // CTA for all columns: columns j < kin-1 of H from global memory (written
  // by CTA 0 before the barriers since), the newest one from shared memory
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double h[KB + 1][KB];
    double gv[KB + 1];
    for (int j = 0; j < kin; ++j)
      for (int l = 0; l <= kin; ++l) {
        double v = 0.0;
        if (l <= j + 1) v = (j == kin - 1) ? m.slast[(size_t)l * C + c] : a.H[((size_t)l * kin + j) * C + c];
        h[l][j] = v;
      }
    for (int l = 0; l <= kin; ++l) gv[l] = 0.0;
    gv[0] = m.sbeta[c];
    for (int i = 0; i < kin; ++i) {
      const double x = h[i][i], y = h[i + 1][i];
      const double rr = sqrt(x * x + y * y);
      const double cs = rr > 0.0 ? x / rr : 1.0, sn = rr > 0.0 ? y / rr : 0.0;
      for (int j = i; j < kin; ++j) {
        const double t1 = h[i][j], t2 = h[i + 1][j];
        h[i][j] = cs * t1 + sn * t2;
        h[i + 1][j] = -sn * t1 + cs * t2;
      }
      const double t1 = gv[i], t2 = gv[i + 1];
      gv[i] = cs * t1 + sn * t2;
      gv[i + 1] = -sn * t1 + cs * t2;
    }
    double yl[KB];
    for (int i = kin - 1; i >= 0; --i) {
      double s = gv[i];
      for (int j = i + 1; j < kin; ++j) s -= h[i][j] * yl[j];
      yl[i] = h[i][i] != 0.0 ? s / h[i][i] : 0.0;
      m.sy[(size_t)i * C + c] = (float)yl[i];
    }
  }
  __syncthreads();
  // ---- z = D^{-1} sum_l y_l v_l for the CTA's rows
  if (act) {
    for (int row = r0 + g; row < r1; row += G) {
      const size_t o4 = (size_t)row * nch + ch;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int l = 0; l < kin; ++l) {
        const float4 vl = ld4(a.V + (size_t)l * a.vstride, o4);
        const float4 y = reinterpret_cast<const float4*>(m.sy + (size_t)l * C)[ch];
        acc.x = fmaf(y.x, vl.x, acc.x);
        acc.y = fmaf(y.y, vl.y, acc.y);
        acc.z = fmaf(y.z, vl.z, acc.z);
        acc.w = fmaf(y.w, vl.w, acc.w);
      }
      const float dv = __ldg(a.dinv + row);
      st4(a.z, o4, make_float4(acc.x * dv, acc.y * dv, acc.z * dv, acc.w * dv));
    }
  }
out:
  grid_exit(a);
}

template <int KB>
const void* ig_kernel() {
  return (const void*)k_inner_grid<KB>;
}

// instantiations: the default step count (6) and the longest allowed
constexpr int IG_KB_SMALL = 6;

int bucket(int kin) { return kin <= IG_KB_SMALL ? IG_KB_SMALL : KIN_MAX; }

size_t smem_for(int kb, int C, int G) {
  return kb == IG_KB_SMALL ? ig_smem_bytes<IG_KB_SMALL>(C, G) : ig_smem_bytes<KIN_MAX>(C, G);
}

}  // namespace

cudaError_t init_inner_grid_attributes() {
  cudaError_t e = cudaFuncSetAttribute(ig_kernel<IG_KB_SMALL>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ig_kernel<KIN_MAX>(), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return e;
}

// Grid size and row ranges of the persistent inner solve for this context
// (0 CTAs: not applicable, the launch chain is used).  One CTA per SM (two
// fit, so the two subproblems' launches can be resident together;
// MHDE_IG_OCC = 2 asks for two per SM), at most one per 128 rows; rows are
// split so that every CTA gets about the same operator nonzeros plus
// per-row vector work.
int inner_grid_plan(const mhde_ctx* c, std::vector<int>& row_start) {
  row_start.clear();
  const int C = 2 * c->Jp, nch = C / 4;
  const int kin = c->opt.inner_iters;
  if (kin < 1 || nch < 1 || nch > IG_T || (C & 3)) return 0;
  const int G = IG_T / nch;
  const int kb = bucket(kin);
  const size_t smem = smem_for(kb, C, G);
  if (smem > 200 * 1024) return 0;
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb == IG_KB_SMALL ? ig_kernel<IG_KB_SMALL>() : ig_kernel<KIN_MAX>(),
                                                    IG_T, smem) != cudaSuccess || occ < 1)
    return 0;
  const int n2 = c->fe.n2;
  int per_sm = 1;
  if (const char* e = std::getenv("MHDE_IG_OCC")) per_sm = std::max(1, std::min(occ, std::atoi(e)));
  const int P = std::max(1, std::min({per_sm * nsm, IG_PMAX, n2 / 128, c->nchunk_in}));
  const std::vector<int>& rp = c->fe.F.rowptr;
  std::vector<double> cum(n2 + 1, 0.0);
  for (int r = 0; r < n2; ++r) cum[r + 1] = cum[r] + (rp[r + 1] - rp[r]) + (kin + 2);
  row_start.assign(P + 1, n2);
  row_start[0] = 0;
  int r = 0;
  for (int b = 1; b < P; ++b) {
    const double t = cum[n2] * b / P;
    while (r < n2 && cum[r] < t) ++r;
    row_start[b] = r;
  }
  return P;
}

bool launch_inner_grid(const mhde_ctx* c, const Sub& s, const float* FDv, const float* dinv, const float* r,
                       float* z, int ld, int kin, cudaStream_t st) {
  const int P = c->ig_P;
  if (P <= 0 || !c->d_ig_rows || !s.ibar || kin < 1 || ld != c->Jp) return false;
  const int n2 = c->fe.n2, C = 2 * ld, nch = C / 4, G = IG_T / nch;
  const int kb = bucket(kin);
  IgArgs a;
  a.n2 = n2;
  a.C = C;
  a.nch = nch;
  a.kin = kin;
  a.rowptr = c->F.rowptr;
  a.col = c->F.col;
  a.FD = FDv;
  a.dinv = dinv;
  a.row_start = c->d_ig_rows;
  a.r = r;
  a.z = z;
  a.vstride = (size_t)n2 * C;
  a.w = (float*)s.ibasis;
  a.V = a.w + a.vstride;
  a.part = s.ipart;
  a.red = s.idot;
  a.H = s.ih;
  a.bar = s.ibar;
  a.err = s.d_err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(IG_T);
  cfg.dynamicSmemBytes = smem_for(kb, C, G);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch(1);
  cudaError_t e = kb == IG_KB_SMALL ? cudaLaunchKernelEx(&cfg, k_inner_grid<IG_KB_SMALL>, a)
                                    : cudaLaunchKernelEx(&cfg, k_inner_grid<KIN_MAX>, a);
  return e == cudaSuccess;
}

}  // namespace mhde
