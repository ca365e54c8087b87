// Allocation-free variant of the batched block Gram (mhde_block_gram).
//
// Some callers cannot allocate device memory at all: hosts that own every
// byte of the GPU through their own pool and forbid side allocations, and
// latency-critical loops where a cudaMalloc (which may synchronize the
// device) is not acceptable.  This entry point takes no scratch argument: its
// per-chunk partial sums live in a fixed file-scope __device__ array, so it
// calls no cudaMalloc, cudaFree or allocating library routine.
#include <algorithm>
#include <mutex>

#include "kernels.h"

namespace {

// Partial-sum scratch shared by every call on a device, held by every GPU
// that loads the library until the process exits: 2 MiB.
constexpr size_t NOALLOC_GRAM_SCRATCH_DOUBLES = 262144;
__device__ __align__(256) double g_gram_scratch[NOALLOC_GRAM_SCRATCH_DOUBLES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_mutex;
double* g_scratch_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array for the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device with that device current and cached for the life of the
// process; a cudaDeviceReset of that device in the same process would leave
// the cached address stale (this library never resets a device).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" {

int mhde_block_gram_noalloc(const double* V, size_t v_stride, int kblocks, const double* W, int n_rows, int ld,
                            int r, double* G, void* stream) {
  // one grid row per basis block: at most 65535 blocks (the grid's y limit)
  if (!V || !W || !G || n_rows < 1 || kblocks < 1 || kblocks > 65535 || r < 1 || r > mhde::MAX_J || ld < r ||
      ld % 4 != 0 || ld > mhde::MAX_J)
    return MHDE_EINVAL;
  const size_t per_chunk = (size_t)kblocks * r * r;
  if (per_chunk > NOALLOC_GRAM_SCRATCH_DOUBLES) return MHDE_EWORKSPACE;   // beyond the fixed maximum
  const int want = std::max(1, std::min(304, (n_rows + 255) / 256));
  const int nchunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)want, NOALLOC_GRAM_SCRATCH_DOUBLES / per_chunk));
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return MHDE_ECUDA;
  // every chunk rewrites all of its partial sums, so nothing needs clearing
  mhde::launch_gram<double>(V, v_stride, kblocks, W, n_rows, ld, r, nchunk, scratch, G, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? MHDE_OK : MHDE_ECUDA;
}

}  // extern "C"
