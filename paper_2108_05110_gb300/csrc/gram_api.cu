// Context-free entry point of the batched block Gram reduction used by the
// block Krylov iterations (Section 1: the shared matrix is solved for all J
// right-hand sides with block linear solvers): G_i = V_i^T W for k blocks.
#include <algorithm>

#include "kernels.h"

namespace {
int gram_chunks(int n_rows) { return std::max(1, std::min(304, (n_rows + 255) / 256)); }
}  // namespace

extern "C" {

int mhde_block_gram_scratch_bytes(int n_rows, int r, int kblocks, size_t* bytes) {
  if (!bytes || n_rows < 1 || r < 1 || r > mhde::MAX_J || kblocks < 1 || kblocks > 65535) return MHDE_EINVAL;
  *bytes = (size_t)gram_chunks(n_rows) * kblocks * r * r * sizeof(double);
  return MHDE_OK;
}

int mhde_block_gram(const double* V, size_t v_stride, int kblocks, const double* W, int n_rows, int ld,
                    int r, double* G, void* scratch, size_t scratch_bytes, void* stream) {
  // one grid row per basis block: at most 65535 blocks (the grid's y limit)
  if (!V || !W || !G || !scratch || n_rows < 1 || kblocks < 1 || kblocks > 65535 || r < 1 || r > mhde::MAX_J ||
      ld < r || ld % 4 != 0 || ld > mhde::MAX_J)
    return MHDE_EINVAL;
  size_t need = 0;
  mhde_block_gram_scratch_bytes(n_rows, r, kblocks, &need);
  if (scratch_bytes < need) return MHDE_EWORKSPACE;
  mhde::launch_gram<double>(V, v_stride, kblocks, W, n_rows, ld, r, gram_chunks(n_rows), (double*)scratch, G,
                            (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? MHDE_OK : MHDE_ECUDA;
}

// FP32 variant (the Krylov precision of the mixed path).  Scratch: one
// 256-byte slot for the kernels' error word, then the partial sums.
int mhde_block_gram_f32_scratch_bytes(int n_rows, int r, int kblocks, size_t* bytes) {
  if (!bytes || n_rows < 1 || r < 1 || r > mhde::MAX_J || kblocks < 1 || kblocks > 65535) return MHDE_EINVAL;
  *bytes = 256 + (size_t)gram_chunks(n_rows) * kblocks * r * r * sizeof(double);
  return MHDE_OK;
}

int mhde_block_gram_f32(const float* V, size_t v_stride, int kblocks, const float* W, int n_rows, int ld, int r,
                        double* G, void* scratch, size_t scratch_bytes, int use_tensor_cores, void* stream) {
  if (!V || !W || !G || !scratch || n_rows < 1 || kblocks < 1 || kblocks > 65535 || r < 1 || r > mhde::MAX_J ||
      ld < r || ld % 4 != 0 || ld > mhde::MAX_J || (use_tensor_cores != 0 && use_tensor_cores != 1))
    return MHDE_EINVAL;
  size_t need = 0;
  mhde_block_gram_f32_scratch_bytes(n_rows, r, kblocks, &need);
  if (scratch_bytes < need) return MHDE_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = (int*)scratch;
  double* part = (double*)((char*)scratch + 256);
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return MHDE_ECUDA;
  const int nchunk = gram_chunks(n_rows);
  if (use_tensor_cores) {
    mhde::TcGramPlan plan;
    if (!mhde::gram_tc_plan(kblocks, ld, r, plan)) return MHDE_EINVAL;      // sizes outside the kernel's range
    if (!mhde::tc_gram_available()) return MHDE_ECUDA;
    int nparts = 0;
    if (!mhde::launch_gram_tc(V, v_stride, kblocks, W, n_rows, ld, r, nchunk, part, st, err, nparts))
      return MHDE_EINVAL;                                                    // misaligned pointers or stride
    mhde::launch_gram_reduce(nparts, kblocks * r * r, part, G, st);
  } else {
    mhde::launch_gram<float>(V, v_stride, kblocks, W, n_rows, ld, r, nchunk, part, G, st, true, err, false);
  }
  if (cudaGetLastError() != cudaSuccess) return MHDE_ECUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MHDE_ECUDA;
  return h ? MHDE_ECUDA : MHDE_OK;
}

// Block combination in FP32: out = alpha in + sum_i V_i C_i.  scratch: at
// least 256 bytes (the kernels' error word).
int mhde_block_combine_f32(float* out, const float* in, float alpha, const float* V, size_t v_stride, int kblocks,
                           int r_in, const float* C, int r_out, int n_rows, int ldv, int ldo, void* scratch,
                           size_t scratch_bytes, int use_tensor_cores, void* stream) {
  if (!out || !V || !C || !scratch || n_rows < 1 || kblocks < 1 || r_in < 1 || r_in > ldv || ldv % 4 != 0 ||
      ldv > mhde::MAX_J || r_out < 1 || r_out > ldo || ldo % 4 != 0 || ldo > mhde::MAX_J ||
      (use_tensor_cores != 0 && use_tensor_cores != 1))
    return MHDE_EINVAL;
  if (scratch_bytes < 256) return MHDE_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = (int*)scratch;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return MHDE_ECUDA;
  if (use_tensor_cores) {
    if (!mhde::tc_gram_available()) return MHDE_ECUDA;
    if (!mhde::launch_combine_tc(out, in, alpha, V, v_stride, kblocks, r_in, C, r_out, n_rows, ldv, ldo, st, err))
      return MHDE_EINVAL;                                                    // sizes or alignment outside its range
  } else {
    mhde::launch_block_combine<float>(out, in, alpha, V, v_stride, kblocks, r_in, C, r_out, n_rows, ldv, ldo, st,
                                      nullptr);
  }
  if (cudaGetLastError() != cudaSuccess) return MHDE_ECUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MHDE_ECUDA;
  return h ? MHDE_ECUDA : MHDE_OK;
}

}  // extern "C"
