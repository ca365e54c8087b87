// The dense contractions of the block Krylov solve on the fifth-generation
// tensor cores (Section 1: one shared matrix, all J right-hand sides solved
// together with block linear solvers; the block Gram V_i^T W and the block
// combination sum_i V_i C_i are the method's only dense products).
//
// Both run tcgen05.mma kind::tf32 (M = 128, K = 8 per instruction) with the
// accumulators in tensor memory.  To keep FP32-level accuracy every operand
// x is split into hi = x with the low 13 mantissa bits cleared (exact in
// TF32) and lo = x - hi (exact in FP32), and hi*hi + hi*lo + lo*hi is
// accumulated: the dropped lo*lo term and the TF32 rounding of lo leave a
// relative error of about 2^-21 per product.  The B operand holds hi and lo
// side by side along N, so two instructions per K step do it: A_hi [B_hi |
// B_lo] into 2N accumulator columns and A_lo B_hi into the first N; the
// epilogue adds the two halves.  (Issue of one instruction costs about as
// much at N = 32 as at N = 64, so this is a third fewer than three.)  Operands reach shared memory
// by TMA bulk copies (row-major, a ring of stages); all threads then write
// the split operands in the canonical K-major no-swizzle layout (core
// matrices of 8 rows x 16 bytes, 128 contiguous bytes), double-buffered so
// that the split of one tile overlaps the MMAs of the previous one; one
// thread issues the MMAs and commits them to an mbarrier per buffer.  Every
// mbarrier wait is bounded: past the poll limit the kernel sets the
// caller's error word, gives its copies and MMAs in flight a bounded chance
// to finish, frees its tensor memory and returns.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "kernels.h"

namespace mhde {
namespace {

constexpr int TC_T = 320;                        // 10 warps: producer, MMA, 8 split warps
constexpr size_t TC_SMEM_MAX = 225 * 1024;
constexpr unsigned TC_BAR_BYTES = 1024;          // mbarriers and the TMEM address slot
constexpr long long TC_SPIN = 1ll << 24;

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool bar_wait(unsigned bar, unsigned parity) {
  for (long long it = 0; it < TC_SPIN; ++it)
    if (bar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Shared-memory matrix descriptor of a K-major operand, no swizzle: lbo is
// the byte offset between core matrices adjacent along K, sbo between core
// matrices adjacent along M (or N), i.e. between groups of 8 rows.
__device__ __forceinline__ uint64_t kdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;                        // descriptor version
  return d;                                      // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, M and N as given.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(unsigned slot, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(unsigned tmem, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns of tensor memory
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float v[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
__device__ __forceinline__ void split4(const float x[4], float4& hi, float4& lo) {
  hi = make_float4(tf32_hi(x[0]), tf32_hi(x[1]), tf32_hi(x[2]), tf32_hi(x[3]));
  lo = make_float4(x[0] - hi.x, x[1] - hi.y, x[2] - hi.z, x[3] - hi.w);
}

// ------------------------------------------------------------ block Gram
//   G_i[p][q] = sum_rows V_i[row][p] W[row][q],   i < kblocks,  p, q < r
// is a GEMM contracting over the mesh rows: A = [V_0 | ... | V_{k-1}]
// (stacked columns m = i ld + p, M = 128 per tile), B = [W_hi | W_lo]
// (2N rows: W padded to N = 16..64 columns, hi then lo), K = rows.  Per K
// step and M tile, A_hi B into 2N accumulator columns and A_lo W_hi into
// the first N.  The grid is (row ranges) x (groups of blocks whose
// accumulators fit the 512 TMEM columns).
//
// Warp-specialised pipeline, one CTA per SM, no CTA-wide barrier in the
// main loop:
//   warp 0      fills a ring of nst stages (TR rows of every block and of W)
//               with TMA bulk copies, each stage reused once the split warps
//               have released it (mbarrier `empty`);
//   warps 2..9  split a landed stage into one of nl operand buffers in the
//               canonical K-major layout (4 rows of one column per item:
//               consecutive threads take consecutive columns, so neither the
//               reads nor the writes conflict in shared-memory banks), once
//               the MMAs that last read that buffer completed (mbarrier
//               `lempty`, arrived by tcgen05.commit), then release the stage
//               and hand the buffer over (mbarrier `lfull`);
//   warp 1      allocates the tensor memory and, on one lane, issues the
//               MMAs of each buffer and commits them.
// Warps 0..7 read the accumulators out at the end.  A wait that gives up
// raises a shared abort flag that the other roles poll, so every role
// leaves its loop; the CTA then records the failure, waits (bounded) for
// the copies and MMAs it has in flight, frees its tensor memory and returns.
constexpr int GW_SPLIT = 8;                      // split warps (2 .. 9)
constexpr int GW_IMAX = 16;                      // split items per split thread and tile

__device__ __forceinline__ void bar_arrive(unsigned bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
// bounded wait that also gives up once another role has raised the abort flag
__device__ __forceinline__ bool bar_wait_ab(unsigned bar, unsigned parity, const volatile int* abort_flag) {
  for (long long it = 0; it < TC_SPIN; ++it) {
    if (bar_try(bar, parity)) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  return false;
}

template <int N>
__global__ void __launch_bounds__(TC_T, 1)
    k_gram_tc(const float* __restrict__ V, size_t vstride, int kb_total, int kgroup, const float* __restrict__ Wm,
              int n_rows, int ld, int r, int rows_per_cta, int TR, int mtiles, unsigned ncols, unsigned stage_bytes,
              int nst, int nl, unsigned off_lay, unsigned lay_bytes, double* __restrict__ part,
              int* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  const int b0 = blockIdx.y * kgroup;                  // this CTA's blocks b0 .. b0 + kblocks - 1
  const int kblocks = min(kgroup, kb_total - b0);
  V += (size_t)b0 * vstride;
  extern __shared__ __align__(1024) unsigned char tsm[];
  const unsigned base = su32(tsm);
  const unsigned bar_full = base;                      // nst (<= 8) stage landed
  const unsigned bar_empty = base + 64;                // nst stage released by the split warps
  const unsigned bar_lfull = base + 128;               // nl (<= 4) operand buffer written
  const unsigned bar_lempty = base + 160;              // nl operand buffer read by its MMAs
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(tsm + 192);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tsm + 196);
  volatile int* progress = reinterpret_cast<volatile int*>(tsm + 200);   // tiles issued, split, committed
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n_rows, r0 + rows_per_cta);
  const int ntiles = r1 > r0 ? (r1 - r0 + TR - 1) / TR : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (ntiles == 0 || kblocks <= 0) {
    for (int e = threadIdx.x; e < max(kblocks, 0) * r * r; e += TC_T)
      part[((size_t)blockIdx.x * kb_total + b0) * r * r + e] = 0.0;
    return;
  }
  const unsigned KSTRW = (unsigned)N * 32u;            // bytes per K slice of the W part: N hi rows, N lo rows
  const unsigned KSTR = (unsigned)mtiles * 2048u;      // bytes per K slice of the V part
  const unsigned vpart = (unsigned)(TR / 4) * KSTRW;   // V hi, then V lo
  const unsigned vlo = (unsigned)(TR / 4) * KSTR;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      bar_init(bar_full + 8 * s, 1);
      bar_init(bar_empty + 8 * s, GW_SPLIT);
    }
    for (int j = 0; j < nl; ++j) {
      bar_init(bar_lfull + 8 * j, GW_SPLIT);
      bar_init(bar_lempty + 8 * j, 1);
    }
    *abort_flag = 0;
    progress[0] = progress[1] = progress[2] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    proxy_fence();
  }
  if (warp == 1) tmem_alloc(su32(tmem_slot), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tmem_slot;

  if (warp == 0) {
    // ---- producer: kblocks + 1 contiguous spans of nr * ld floats per stage
    for (int tile = 0; tile < ntiles; ++tile) {
      const int s = tile % nst;
      if (tile >= nst && !bar_wait_ab(bar_empty + 8 * s, (unsigned)((tile / nst - 1) & 1), abort_flag)) {
        if (lane == 0) *abort_flag = 1;
        break;
      }
      const unsigned st = base + TC_BAR_BYTES + (unsigned)s * stage_bytes;
      const int t0 = r0 + tile * TR;
      const unsigned bytes = (unsigned)(min(TR, r1 - t0) * ld) * 4u;
      proxy_fence();                                   // the stage was last read through the generic proxy
      if (lane == 0) bar_expect_tx(bar_full + 8 * s, bytes * (unsigned)(kblocks + 1));
      __syncwarp();
      for (int b = lane; b <= kblocks; b += 32) {
        const float* g = (b < kblocks ? V + (size_t)b * vstride : Wm) + (size_t)t0 * ld;
        bulk_load(st + (unsigned)(b * TR * ld) * 4u, g, bytes, bar_full + 8 * s);
      }
      if (lane == 0) progress[0] = tile + 1;
    }
  } else if (warp == 1) {
    // ---- MMA issue
    if (lane == 0) {
      const uint32_t idesc2 = idesc_tf32(128, 2 * N), idesc1 = idesc_tf32(128, N);
      // descriptors of buffer 0; every other operand is the same descriptor
      // with its start address advanced (the 14-bit address field cannot
      // overflow inside the CTA's shared memory): leading (K) offset between
      // the two 4-row K slices of a step, stride offset between groups of 8
      // rows
      const uint64_t dA0 = kdesc(base + off_lay + vpart, KSTR, 128u);
      const uint64_t dB0 = kdesc(base + off_lay, KSTRW, 128u);
      const uint64_t dlo = (uint64_t)(vlo >> 4);
      for (int tile = 0; tile < ntiles; ++tile) {
        const int j = tile % nl;
        if (!bar_wait_ab(bar_lfull + 8 * j, (unsigned)((tile / nl) & 1), abort_flag)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint64_t dj = (uint64_t)(((unsigned)j * lay_bytes) >> 4);
        for (int k8 = 0; k8 < TR / 8; ++k8) {
          const uint64_t bk = dB0 + dj + (uint64_t)(((unsigned)(2 * k8) * KSTRW) >> 4);
          const uint64_t ak = dA0 + dj + (uint64_t)(((unsigned)(2 * k8) * KSTR) >> 4);
          const int acc = (tile > 0 || k8 > 0) ? 1 : 0;
          for (int t = 0; t < mtiles; ++t) {
            const uint64_t at = ak + (uint64_t)(t * 128);          // 2048 bytes per M tile
            const unsigned d = tmem + (unsigned)(t * 2 * N);
            mma_tf32(d, at, bk, idesc2, acc);                      // A_hi [W_hi | W_lo]
            mma_tf32(d, at + dlo, bk, idesc1, 1);                  // A_lo W_hi
          }
        }
        mma_commit(bar_lempty + 8 * j);
        progress[2] = tile + 1;
      }
    }
    __syncwarp();
  } else {
    // ---- split: this thread's items, the same for every tile: rows
    // 4 k4 .. 4 k4 + 3 of stage column col (column p of block b, W for
    // b = kblocks); -1: none
    const int sid = threadIdx.x - 64;
    const int cols = (kblocks + 1) * ld;
    const int items = cols * (TR / 4);
    int src[GW_IMAX], dst[GW_IMAX], row0[GW_IMAX], dlo[GW_IMAX];
    const int nq = (items - sid + 32 * GW_SPLIT - 1) / (32 * GW_SPLIT);   // items of this thread
#pragma unroll
    for (int q = 0; q < GW_IMAX; ++q) {
      const int it = sid + q * 32 * GW_SPLIT;
      const int k4 = it / cols, col = it - k4 * cols;
      const int b = col / ld, p = col - b * ld;
      src[q] = b * TR * ld + 4 * k4 * ld + p;
      row0[q] = 4 * k4;
      dlo[q] = b == kblocks ? 16 * N : (int)vlo;      // lo beside hi along N (W), or the V lo part
      if (it >= items || (b == kblocks && p >= N)) {   // W columns past N never enter G
        dst[q] = -1;
      } else if (b == kblocks) {
        dst[q] = (int)(k4 * KSTRW) + 16 * p;
      } else {
        dst[q] = (int)(vpart + k4 * KSTR) + 16 * (b * ld + p);
      }
    }
    for (int tile = 0; tile < ntiles; ++tile) {
      const int s = tile % nst, j = tile % nl;
      bool good = bar_wait_ab(bar_full + 8 * s, (unsigned)((tile / nst) & 1), abort_flag);
      if (good && tile >= nl) good = bar_wait_ab(bar_lempty + 8 * j, (unsigned)((tile / nl - 1) & 1), abort_flag);
      if (!good) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const float* stf = reinterpret_cast<const float*>(tsm + TC_BAR_BYTES + (size_t)s * stage_bytes);
      unsigned char* lay = tsm + off_lay + (size_t)j * lay_bytes;
      const int nr = min(TR, r1 - (r0 + tile * TR));
      // four items at a time: their sixteen loads are in flight together
#pragma unroll
      for (int q0 = 0; q0 < GW_IMAX; q0 += 4) {
        if (q0 >= nq) break;
        float x[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int jr = 0; jr < 4; ++jr)
            x[u][jr] = (dst[q0 + u] >= 0 && row0[q0 + u] + jr < nr) ? stf[src[q0 + u] + jr * ld] : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (dst[q0 + u] < 0) continue;
          float4 hi, lo;
          split4(x[u], hi, lo);
          *reinterpret_cast<float4*>(lay + dst[q0 + u]) = hi;
          *reinterpret_cast<float4*>(lay + dlo[q0 + u] + dst[q0 + u]) = lo;
        }
      }
      proxy_fence();                                   // generic writes -> visible to the tensor core
      __syncwarp();
      if (lane == 0) {
        bar_arrive(bar_lfull + 8 * j);
        bar_arrive(bar_empty + 8 * s);
        if (warp == 2) progress[1] = tile + 1;
      }
    }
  }
  __syncthreads();
  // the last buffer's commit completes after all earlier MMAs
  int good = *abort_flag == 0;
  if (good) {
    const int lt = ntiles - 1;
    good = bar_wait(bar_lempty + 8 * (lt % nl), (unsigned)((lt / nl) & 1)) ? 1 : 0;
  }
  good = __syncthreads_and(good);
  if (good && warp < 8) {
    tc_fence_after();
    const int q4 = warp & 3, grp = warp >> 2;          // TMEM lanes 32 q4 .. 32 q4 + 31
    for (int t = grp; t < mtiles; t += 2) {
      float v[N];
      const unsigned taddr = tmem + ((unsigned)(32 * q4) << 16) + (unsigned)(t * 2 * N);
#pragma unroll
      for (int c16 = 0; c16 < N / 16; ++c16) {
        float w[16];
        tmem_ld16(taddr + 16 * c16, v + 16 * c16);
        tmem_ld16(taddr + N + 16 * c16, w);
#pragma unroll
        for (int e = 0; e < 16; ++e) v[16 * c16 + e] += w[e];
      }
      const int m = 128 * t + 32 * q4 + lane;          // stacked column of the V blocks
      const int b = m / ld, p = m - b * ld;
      if (b < kblocks && p < r) {
        double* d = part + (((size_t)blockIdx.x * kb_total + b0 + b) * r + p) * r;
#pragma unroll
        for (int q = 0; q < N; ++q)
          if (q < r) d[q] = (double)v[q];
      }
    }
  } else if (!good && threadIdx.x == 0) {
    // a wait gave up: record it, let every copy and MMA in flight finish
    // (bounded), and leave without partial sums
    atomicExch(err, 1);
    const int issued = progress[0], taken = progress[1], committed = progress[2];
    for (int tl = taken; tl < issued; ++tl) bar_wait(bar_full + 8 * (tl % nst), (unsigned)((tl / nst) & 1));
    if (committed > 0) bar_wait(bar_lempty + 8 * ((committed - 1) % nl), (unsigned)(((committed - 1) / nl) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_free(tmem, ncols);
  }
}

// ------------------------------------------------------------ block combination
// out[row][q] = alpha in[row][q] + sum_i sum_p V_i[row][p] C_i[p][q]  (q < r_out,
// zero up to ldo): the new Krylov block and the solution update of the block
// GMRES.  A GEMM with M = rows, K = (block, column) and N = r_out padded to
// 16..64: A = the V row tiles, B = the coefficient blocks.  A CTA (one per
// SM) owns a row range, walked in groups of up to MT tiles of 128 rows whose
// accumulators sit in tensor memory (MT N <= 512 columns); within a group
// the stages s = (block i, row tile t) run in block order.  Same warp roles
// as the Gram:
//   warp 0      one TMA bulk copy of 128 rows per stage into a ring of nst;
//   warps 2..9  split a landed stage into one of nl A buffers (element (m, p)
//               at (p/4) 2048 + m 16 + (p%4) 4), and at a block's first tile
//               its coefficients into B buffer (block sequence number) % 2
//               (element (q, p) at (p/4) N 16 + q 16 + (p%4) 4), each buffer
//               reused once the MMAs that read it completed (mbarriers
//               aempty / bempty, arrived by tcgen05.commit);
//   warp 1      3 MMAs per K step of 8 into the tile's accumulator, a commit
//               per stage and one per block.
// At the end of a group, warps 2..5 (one per quarter of the 128 TMEM lanes)
// write out alpha in + the accumulators and release the tensor memory to
// the next group (mbarrier tfree).  The CTA has read all rows of a group in
// every block before it writes them, so out may alias in or one of the
// blocks.  Waits are bounded as in the Gram.
template <int N>
__global__ void __launch_bounds__(TC_T, 1)
    k_combine_tc(float* out, const float* in, float alpha, const float* V, size_t vstride, int kblocks, int r_in,
                 const float* __restrict__ C, int r_out, int n_rows, int ldv, int ldo, int rows_per_cta, int KC,
                 int MT, unsigned ncols, unsigned stage_bytes, int nst, int nl, unsigned off_a, unsigned a_bytes,
                 unsigned off_b, unsigned b_bytes, int* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(1024) unsigned char tsm[];
  const unsigned base = su32(tsm);
  const unsigned bar_full = base;                      // nst (<= 8)
  const unsigned bar_empty = base + 64;                // nst
  const unsigned bar_afull = base + 128;               // nl (<= 4)
  const unsigned bar_aempty = base + 160;              // nl
  const unsigned bar_bempty = base + 192;              // 2
  const unsigned bar_tfree = base + 208;               // 1
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(tsm + 216);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tsm + 220);
  volatile int* progress = reinterpret_cast<volatile int*>(tsm + 224);   // stages issued, split, committed
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n_rows, r0 + rows_per_cta);
  if (r1 <= r0) return;
  const int T = (r1 - r0 + 127) / 128;                 // row tiles of this CTA
  const int nstages = kblocks * T;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = ldv / 4;                             // 16-byte chunks of a V row
  const unsigned ahalf = a_bytes / 2;
  // stage sidx -> group g, block i, tile t of the group (mt tiles in it)
  auto decode = [&](int sidx, int& g, int& i, int& t, int& mt) {
    g = sidx / (kblocks * MT);
    const int rem = sidx - g * kblocks * MT;
    mt = min(MT, T - g * MT);
    i = rem / mt;
    t = rem - i * mt;
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      bar_init(bar_full + 8 * s, 1);
      bar_init(bar_empty + 8 * s, GW_SPLIT);
    }
    for (int j = 0; j < nl; ++j) {
      bar_init(bar_afull + 8 * j, GW_SPLIT);
      bar_init(bar_aempty + 8 * j, 1);
    }
    bar_init(bar_bempty, 1);
    bar_init(bar_bempty + 8, 1);
    bar_init(bar_tfree, 4);
    *abort_flag = 0;
    progress[0] = progress[1] = progress[2] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    proxy_fence();
  }
  // K padding chunks (columns ldv .. 4 KC - 1) of every A buffer stay zero
  for (int e = threadIdx.x; e < nl * (KC - nch) * 128; e += TC_T) {
    const int j = e / ((KC - nch) * 128), rem = e - j * (KC - nch) * 128;
    const int k4 = nch + rem / 128, m = rem % 128;
    unsigned char* a = tsm + off_a + (size_t)j * a_bytes + (size_t)k4 * 2048 + (size_t)m * 16;
    *reinterpret_cast<float4*>(a) = make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(a + ahalf) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (warp == 1) tmem_alloc(su32(tmem_slot), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tmem_slot;
  const unsigned bstride = (unsigned)N * 32u;          // between K chunks of a coefficient buffer (N hi, N lo rows)

  if (warp == 0) {
    // ---- producer
    if (lane == 0) {
      for (int sidx = 0; sidx < nstages; ++sidx) {
        const int s = sidx % nst;
        if (sidx >= nst && !bar_wait_ab(bar_empty + 8 * s, (unsigned)((sidx / nst - 1) & 1), abort_flag)) {
          *abort_flag = 1;
          break;
        }
        int g, i, t, mt;
        decode(sidx, g, i, t, mt);
        const int t0 = r0 + 128 * (g * MT + t);
        const unsigned bytes = (unsigned)(min(128, r1 - t0) * ldv) * 4u;
        proxy_fence();
        bar_expect_tx(bar_full + 8 * s, bytes);
        bulk_load(base + TC_BAR_BYTES + (unsigned)s * stage_bytes, V + (size_t)i * vstride + (size_t)t0 * ldv, bytes,
                  bar_full + 8 * s);
        progress[0] = sidx + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issue
    if (lane == 0) {
      const uint32_t idesc2 = idesc_tf32(128, 2 * N), idesc1 = idesc_tf32(128, N);
      // descriptors of A buffer 0 and B buffer 0, advanced per operand
      const uint64_t dA0 = kdesc(base + off_a, 2048u, 128u);
      const uint64_t dB0 = kdesc(base + off_b, bstride, 128u);
      const uint64_t dla = (uint64_t)(ahalf >> 4);
      for (int sidx = 0; sidx < nstages; ++sidx) {
        int g, i, t, mt;
        decode(sidx, g, i, t, mt);
        const int j = sidx % nl, bs = g * kblocks + i;
        // the tensor memory of group g - 1 has been written out
        bool good = true;
        if (g > 0 && i == 0 && t == 0) good = bar_wait_ab(bar_tfree, (unsigned)((g - 1) & 1), abort_flag);
        if (good) good = bar_wait_ab(bar_afull + 8 * j, (unsigned)((sidx / nl) & 1), abort_flag);
        if (!good) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint64_t aj = dA0 + (uint64_t)(((unsigned)j * a_bytes) >> 4);
        const uint64_t bj = dB0 + (uint64_t)(((unsigned)(bs & 1) * b_bytes) >> 4);
        const unsigned d = tmem + (unsigned)(t * 2 * N);
        for (int k8 = 0; k8 < KC / 2; ++k8) {
          const uint64_t ak = aj + (uint64_t)(k8 * 256);                    // 4096 bytes per K step
          const uint64_t bk = bj + (uint64_t)((((unsigned)k8 * 2u) * bstride) >> 4);
          mma_tf32(d, ak, bk, idesc2, (i > 0 || k8 > 0) ? 1 : 0);          // A_hi [C_hi | C_lo]
          mma_tf32(d, ak + dla, bk, idesc1, 1);                             // A_lo C_hi
        }
        mma_commit(bar_aempty + 8 * j);
        if (t == mt - 1) mma_commit(bar_bempty + 8 * (bs & 1));   // the block's coefficients are free
        progress[2] = sidx + 1;
      }
    }
    __syncwarp();
  } else {
    // ---- split (warps 2..9); warps 2..5 also write out each group
    const int sid = threadIdx.x - 64;
    int src[GW_IMAX], dst[GW_IMAX], mrow[GW_IMAX], ncol[GW_IMAX];
    const int nq = (nch * 128 - sid + 32 * GW_SPLIT - 1) / (32 * GW_SPLIT);   // items of this thread
#pragma unroll
    for (int q = 0; q < GW_IMAX; ++q) {
      const int it = sid + q * 32 * GW_SPLIT;
      const int k4 = it >> 7, m = it & 127;
      src[q] = m * ldv + 4 * k4;
      dst[q] = k4 * 2048 + m * 16;
      mrow[q] = m;
      ncol[q] = it < nch * 128 ? max(0, min(4, r_in - 4 * k4)) : -1;   // -1: no item; columns past r_in are 0
    }
    const bool writer = warp >= 2 && warp <= 5;
    for (int sidx = 0; sidx < nstages; ++sidx) {
      int g, i, t, mt;
      decode(sidx, g, i, t, mt);
      const int s = sidx % nst, j = sidx % nl, bs = g * kblocks + i;
      bool good = bar_wait_ab(bar_full + 8 * s, (unsigned)((sidx / nst) & 1), abort_flag);
      if (good && sidx >= nl) good = bar_wait_ab(bar_aempty + 8 * j, (unsigned)((sidx / nl - 1) & 1), abort_flag);
      if (good && t == 0 && bs >= 2)
        good = bar_wait_ab(bar_bempty + 8 * (bs & 1), (unsigned)((bs / 2 - 1) & 1), abort_flag);
      if (!good) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      if (t == 0) {
        const unsigned bsel = off_b + (unsigned)(bs & 1) * b_bytes;
        for (int e = sid; e < KC * N; e += 32 * GW_SPLIT) {
          const int k4 = e / N, q = e - k4 * N;
          float cv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int pp = 4 * k4 + u;
            cv[u] = (pp < r_in && q < r_out) ? C[((size_t)i * r_in + pp) * r_out + q] : 0.f;
          }
          float4 hi, lo;
          split4(cv, hi, lo);
          const size_t o = (size_t)k4 * bstride + (size_t)q * 16;
          *reinterpret_cast<float4*>(tsm + bsel + o) = hi;
          *reinterpret_cast<float4*>(tsm + bsel + 16 * N + o) = lo;
        }
      }
      const float* stf = reinterpret_cast<const float*>(tsm + TC_BAR_BYTES + (size_t)s * stage_bytes);
      unsigned char* a = tsm + off_a + (size_t)j * a_bytes;
      const int nr = min(128, r1 - (r0 + 128 * (g * MT + t)));
      // four items at a time: their loads are in flight together
#pragma unroll
      for (int q0 = 0; q0 < GW_IMAX; q0 += 4) {
        if (q0 >= nq) break;
        float4 v4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          v4[u] = (ncol[q0 + u] > 0 && mrow[q0 + u] < nr) ? *reinterpret_cast<const float4*>(stf + src[q0 + u])
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u;
          if (ncol[q] < 0) continue;
          float x[4] = {v4[u].x, v4[u].y, v4[u].z, v4[u].w};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (e >= ncol[q]) x[e] = 0.f;
          float4 hi, lo;
          split4(x, hi, lo);
          *reinterpret_cast<float4*>(a + dst[q]) = hi;
          *reinterpret_cast<float4*>(a + ahalf + dst[q]) = lo;
        }
      }
      proxy_fence();                                   // generic writes -> visible to the tensor core
      __syncwarp();
      if (lane == 0) {
        bar_arrive(bar_afull + 8 * j);
        bar_arrive(bar_empty + 8 * s);
        if (warp == 2) progress[1] = sidx + 1;
      }
      if (writer && i == kblocks - 1 && t == mt - 1) {
        // ---- the group's last stage: once its MMAs (and so all of the
        // group's) completed, write the group's rows out
        if (!bar_wait_ab(bar_aempty + 8 * j, (unsigned)((sidx / nl) & 1), abort_flag)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const int q4 = warp & 3;                       // TMEM lanes 32 q4 .. 32 q4 + 31
        for (int tt = 0; tt < mt; ++tt) {
          float v[N];
          const unsigned taddr = tmem + ((unsigned)(32 * q4) << 16) + (unsigned)(tt * 2 * N);
#pragma unroll
          for (int c16 = 0; c16 < N / 16; ++c16) {
            float w[16];
            tmem_ld16(taddr + 16 * c16, v + 16 * c16);
            tmem_ld16(taddr + N + 16 * c16, w);
#pragma unroll
            for (int e = 0; e < 16; ++e) v[16 * c16 + e] += w[e];
          }
          const int row = r0 + 128 * (g * MT + tt) + 32 * q4 + lane;
          if (row < r1) {
            float* orow = out + (size_t)row * ldo;
            const float* irow = in ? in + (size_t)row * ldo : nullptr;
#pragma unroll
            for (int q = 0; q < N; q += 4) {
              if (q < ldo) {
                float4 i4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (irow) i4 = *reinterpret_cast<const float4*>(irow + q);
                float4 o4;
                o4.x = q + 0 < r_out ? alpha * i4.x + v[q + 0] : 0.f;
                o4.y = q + 1 < r_out ? alpha * i4.y + v[q + 1] : 0.f;
                o4.z = q + 2 < r_out ? alpha * i4.z + v[q + 2] : 0.f;
                o4.w = q + 3 < r_out ? alpha * i4.w + v[q + 3] : 0.f;
                *reinterpret_cast<float4*>(orow + q) = o4;
              }
            }
            for (int q = N; q < ldo; q += 4) *reinterpret_cast<float4*>(orow + q) = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) bar_arrive(bar_tfree);
      }
    }
  }
  __syncthreads();
  if (*abort_flag != 0 && threadIdx.x == 0) {
    // a wait gave up: record it, let every copy and MMA in flight finish
    // (bounded), and leave (out is not valid)
    atomicExch(err, 1);
    const int issued = progress[0], taken = progress[1], committed = progress[2];
    for (int sl = taken; sl < issued; ++sl) bar_wait(bar_full + 8 * (sl % nst), (unsigned)((sl / nst) & 1));
    if (committed > 0) bar_wait(bar_aempty + 8 * ((committed - 1) % nl), (unsigned)(((committed - 1) / nl) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_free(tmem, ncols);
  }
}

struct TcDevice {
  bool ready = false;
  int nsm = 1;
  cudaError_t err = cudaSuccess;
};
std::mutex g_tc_mutex;
TcDevice g_tc_dev[64];

const TcDevice& tc_setup() {
  static const TcDevice none{false, 1, cudaErrorInvalidDevice};   // never written
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return none;
  std::lock_guard<std::mutex> lock(g_tc_mutex);
  TcDevice& d = g_tc_dev[dev];
  if (d.ready) return d;
  cudaError_t e = cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
  if (d.nsm <= 0) d.nsm = 1;
  int major = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e == cudaSuccess && major < 10) e = cudaErrorInvalidDeviceFunction;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_MAX);
  };
  set((const void*)k_gram_tc<16>);
  set((const void*)k_gram_tc<32>);
  set((const void*)k_gram_tc<48>);
  set((const void*)k_gram_tc<64>);
  set((const void*)k_combine_tc<16>);
  set((const void*)k_combine_tc<32>);
  set((const void*)k_combine_tc<48>);
  set((const void*)k_combine_tc<64>);
  d.err = e;
  d.ready = true;
  return d;
}

}  // namespace

// Experiment knobs (environment, read once): MHDE_TC_TR, MHDE_TC_NL and
// MHDE_TC_NST restrict the plans below to one tile height, buffer count or
// ring depth (0: free).
struct TcKnobs {
  int TR = 0, nl = 0, nst = 0;
};
const TcKnobs& tc_knobs() {
  static const TcKnobs k = [] {
    TcKnobs v;
    auto rd = [](const char* n) { const char* e = std::getenv(n); return e ? std::atoi(e) : 0; };
    v.TR = rd("MHDE_TC_TR");
    v.nl = rd("MHDE_TC_NL");
    v.nst = rd("MHDE_TC_NST");
    return v;
  }();
  return k;
}

bool gram_tc_plan(int kblocks, int ld, int r, TcGramPlan& p) {
  if (kblocks < 1 || r < 1 || r > 64 || ld < r || ld % 4 != 0 || ld > 64) return false;
  p.nch = ld / 4;
  p.N = (r + 15) / 16 * 16;
  // blocks per CTA: their accumulators (M tiles of 128 stacked columns, 2N
  // columns each) fit the 512 TMEM columns of the SM
  p.kgroup = std::min(kblocks, std::max(1, (512 / (2 * p.N)) * 128 / ld));
  while (p.kgroup > 1 && ((p.kgroup * ld + 127) / 128) * 2 * p.N > 512) --p.kgroup;
  for (; p.kgroup >= 1; --p.kgroup) {
    p.mtiles = (p.kgroup * ld + 127) / 128;
    p.ncols = 32;
    while ((int)p.ncols < p.mtiles * 2 * p.N) p.ncols *= 2;
    // one CTA per SM, nl operand buffers; the largest tile that leaves a
    // ring of at least three stages, the deepest ring (at most 6) for it
    const TcKnobs& kn = tc_knobs();
    for (int TR = 32; TR >= 8; TR -= 8)
      for (int nl = 4; nl >= 2; --nl)
        for (int nst = 6; nst >= 3; --nst) {
          if ((kn.TR && TR != kn.TR) || (kn.nst && nst != kn.nst) || nl != (kn.nl ? kn.nl : 2)) continue;
          const size_t stage = (size_t)(p.kgroup + 1) * TR * ld * 4;
          const size_t lay = 2 * (size_t)TR * 4 * (p.N + (size_t)p.mtiles * 128);   // W hi+lo, V hi, V lo
          const size_t off_lay = (TC_BAR_BYTES + nst * stage + 1023) / 1024 * 1024;
          const size_t total = off_lay + nl * lay;
          const int items = (p.kgroup + 1) * ld * (TR / 4);
          if (total <= TC_SMEM_MAX && stage < (1u << 20) && items <= GW_IMAX * GW_SPLIT * 32) {
            p.TR = TR;
            p.nst = nst;
            p.nl = nl;
            p.stage_bytes = (unsigned)stage;
            p.off_lay = (unsigned)off_lay;
            p.lay_bytes = (unsigned)lay;
            p.smem = total;
            p.ngroups = (kblocks + p.kgroup - 1) / p.kgroup;
            p.per_sm = 1;
            return true;
          }
        }
  }
  return false;
}

bool tc_gram_available() { return tc_setup().err == cudaSuccess; }

bool launch_gram_tc(const float* V, size_t vstride, int kblocks, const float* W, int n_rows, int ld, int r,
                    int max_parts, double* part, cudaStream_t st, int* err, int& nparts) {
  TcGramPlan p;
  const TcDevice& d = tc_setup();
  if (d.err != cudaSuccess || !err || !gram_tc_plan(kblocks, ld, r, p)) return false;
  if ((reinterpret_cast<uintptr_t>(V) & 15) || (reinterpret_cast<uintptr_t>(W) & 15) || (vstride & 3)) return false;
  const int nctas = std::max(1, std::min({p.per_sm * d.nsm / p.ngroups, max_parts, (n_rows + 7) / 8}));
  const int rows_per_cta = (n_rows + nctas - 1) / nctas;
  nparts = nctas;
  const dim3 grid(nctas, p.ngroups);
#define MHDE_TC(NN)                                                                                          \
  launch_pdl(k_gram_tc<NN>, grid, dim3(TC_T), p.smem, st, V, vstride, kblocks, p.kgroup, W, n_rows, ld, r, \
             rows_per_cta, p.TR, p.mtiles, p.ncols, p.stage_bytes, p.nst, p.nl, p.off_lay, p.lay_bytes, part, err)
  switch (p.N) {
    case 16: MHDE_TC(16); break;
    case 32: MHDE_TC(32); break;
    case 48: MHDE_TC(48); break;
    default: MHDE_TC(64); break;
  }
#undef MHDE_TC
  return true;
}

bool combine_tc_plan(int n_rows, int ldv, int r_in, int r_out, int nsm, TcCombinePlan& p) {
  if (r_in < 1 || r_out < 1 || r_out > 64 || ldv < r_in || ldv % 4 != 0 || ldv > 64 || n_rows < 1) return false;
  p.N = (r_out + 15) / 16 * 16;
  p.KC = (ldv + 7) / 8 * 2;                            // 16-byte K chunks, an even number (K steps of 8)
  if ((ldv / 4) * 128 > GW_IMAX * GW_SPLIT * 32) return false;
  p.stage_bytes = 128u * (unsigned)ldv * 4u;
  p.a_bytes = 2u * (unsigned)p.KC * 2048u;
  p.b_bytes = 2u * (unsigned)p.KC * (unsigned)p.N * 16u;
  // one CTA per SM over an even share of the row tiles, walked in groups of
  // MT tiles (MT 2N <= 512 tensor-memory columns)
  const int tiles = (n_rows + 127) / 128;
  const int per_cta = (tiles + std::max(nsm, 1) - 1) / std::max(nsm, 1);
  p.rows_per_cta = 128 * per_cta;
  p.nctas = (tiles + per_cta - 1) / per_cta;
  p.MT = std::max(1, std::min(256 / p.N, per_cta));
  p.ncols = 32;
  while ((int)p.ncols < p.MT * 2 * p.N) p.ncols *= 2;
  // as many A buffers (at most 4) and as deep a ring (at most 8) as fit,
  // preferring two A buffers and three stages first
  for (int pass = 0; pass < 2; ++pass)
    for (int nl = 4; nl >= 1; --nl)
      for (int nst = 8; nst >= 2; --nst) {
        if (pass == 0 && (nl < 2 || nst < 3)) continue;
        if ((tc_knobs().nl && nl != tc_knobs().nl) || (tc_knobs().nst && nst != tc_knobs().nst)) continue;
        const size_t off_a = (TC_BAR_BYTES + (size_t)nst * p.stage_bytes + 1023) / 1024 * 1024;
        const size_t off_b = off_a + (size_t)nl * p.a_bytes;
        const size_t total = off_b + 2 * (size_t)p.b_bytes;
        if (total <= TC_SMEM_MAX) {
          p.nl = nl;
          p.nst = nst;
          p.off_a = (unsigned)off_a;
          p.off_b = (unsigned)off_b;
          p.smem = total;
          return true;
        }
      }
  return false;
}

bool launch_combine_tc(float* out, const float* in, float alpha, const float* V, size_t vstride, int kblocks,
                       int r_in, const float* C, int r_out, int n_rows, int ldv, int ldo, cudaStream_t st, int* err) {
  if (!err || kblocks < 1) return false;
  const TcDevice& d = tc_setup();
  TcCombinePlan p;
  if (d.err != cudaSuccess || !combine_tc_plan(n_rows, ldv, r_in, r_out, d.nsm, p)) return false;
  if ((reinterpret_cast<uintptr_t>(V) & 15) || (reinterpret_cast<uintptr_t>(out) & 15) ||
      (reinterpret_cast<uintptr_t>(in) & 15) || (vstride & 3) || (ldo & 3) || ldo > 64 || ldo < r_out)
    return false;
#define MHDE_TCC(NN)                                                                                              \
  launch_pdl(k_combine_tc<NN>, dim3(p.nctas), dim3(TC_T), p.smem, st, out, in, alpha, V, vstride, kblocks, r_in, C, \
             r_out, n_rows, ldv, ldo, p.rows_per_cta, p.KC, p.MT, p.ncols, p.stage_bytes, p.nst, p.nl, p.off_a,    \
             p.a_bytes, p.off_b, p.b_bytes, err)
  switch (p.N) {
    case 16: MHDE_TCC(16); break;
    case 32: MHDE_TCC(32); break;
    case 48: MHDE_TCC(48); break;
    default: MHDE_TCC(64); break;
  }
#undef MHDE_TCC
  return true;
}

}  // namespace mhde
