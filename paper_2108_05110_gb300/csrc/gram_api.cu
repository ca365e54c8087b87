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

}  // extern "C"
