// One-sided Jacobi SVD entry point that allocates nothing (sctm_svd_noalloc).
//
// For callers that cannot allocate device memory while they run -- code
// inside an allocator callback, or a loop held to a fixed memory budget -- and
// that have no engine handle.  The scratch of the multi-CTA Jacobi kernel lives
// in one file-scope device array per device, so calls that overlap in time
// (two streams, two host threads) race on it.  Every call copies the kernel's
// status word to the host and synchronises its stream before returning.
#include <mutex>

#include "../../include/splitctmrg.h"
#include "common.h"
#include "kernels.h"

using namespace sctm;

namespace {

// (m + n) n doubles of rotated columns and accumulated rotations, plus the
// kernel's convergence flags and column-norm words, for (m + n) n <= 2^21.
constexpr size_t kNoAllocMaxMN = size_t(1) << 21;
constexpr size_t kNoAllocScratch = kNoAllocMaxMN + 1024;

__device__ __align__(256) double g_svd_scratch[kNoAllocScratch];
__device__ int g_svd_status[64];   // word 0: sweep-limit flag (must start at zero)

struct Symbols {
  double* scratch = nullptr;
  int* status = nullptr;
};
std::mutex g_mu;
Symbols g_sym[64];   // per device ordinal

}  // namespace

int sctm_svd_noalloc(int m, int n, const double* M_dev, double* U_dev, double* S_dev, double* V_dev,
                     void* stream) {
  if (m < n || n < 1 || !M_dev || !U_dev || !S_dev || !V_dev) return SCTM_ERR_ARG;
  if ((size_t)(m + n) * (size_t)n > kNoAllocMaxMN) return SCTM_ERR_ARG;
  if (svd_work_doubles(m, n, 1) > kNoAllocScratch) return SCTM_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SCTM_ERR_CUDA;
  Symbols sym;
  {
    // the addresses of the static arrays, looked up once per device with that
    // device current
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_sym[dev].scratch) {
      void* a = nullptr;
      void* b = nullptr;
      if (cudaGetSymbolAddress(&a, g_svd_scratch) != cudaSuccess) return SCTM_ERR_CUDA;
      if (cudaGetSymbolAddress(&b, g_svd_status) != cudaSuccess) return SCTM_ERR_CUDA;
      g_sym[dev].scratch = static_cast<double*>(a);
      g_sym[dev].status = static_cast<int*>(b);
    }
    sym = g_sym[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(sym.status, 0, sizeof(int), s) != cudaSuccess) return SCTM_ERR_CUDA;
  try {
    launch_svd(m, n, 1, M_dev, U_dev, S_dev, V_dev, sym.scratch, sym.status, s);
  } catch (const std::exception&) {
    return SCTM_ERR_CUDA;
  }
  int st = 0;
  if (cudaMemcpyAsync(&st, sym.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SCTM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SCTM_ERR_CUDA;
  return st < 0 ? SCTM_ERR_SVD_NOCONV : SCTM_OK;
}
