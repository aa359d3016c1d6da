// Shared host/device definitions of the split-CTMRG engine (GPU path).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>

namespace sctm {

constexpr int kMaxDims = 8;    // dims of one index group (batch / m / n / k)
constexpr int kNumSMs = 152;   // GB300: two dies of 76 SMs; grid-size heuristics count in these

// Error carried from a CUDA call into the C-ABI status code.
struct CudaError : std::runtime_error {
  explicit CudaError(const std::string& s) : std::runtime_error(s) {}
};
struct ArgError : std::runtime_error {
  explicit ArgError(const std::string& s) : std::runtime_error(s) {}
};

#define SCTM_CUDA(expr)                                                        \
  do {                                                                         \
    cudaError_t e__ = (expr);                                                  \
    if (e__ != cudaSuccess)                                                    \
      throw ::sctm::CudaError(std::string(#expr) + ": " + cudaGetErrorString(e__)); \
  } while (0)

#define SCTM_CHECK(cond, msg)                                                  \
  do {                                                                         \
    if (!(cond)) throw ::sctm::ArgError(msg);                                  \
  } while (0)

// One index group of a strided contraction: sizes and element strides of the
// group's dims in each operand (row-major order: the last dim varies fastest).
struct Group {
  int nd = 0;
  int size[kMaxDims] = {0};
  long long sa[kMaxDims] = {0};   // stride in operand A (or 0 if absent)
  long long sb[kMaxDims] = {0};   // stride in operand B
  long long sc[kMaxDims] = {0};   // stride in the output
  __host__ __device__ long long total() const {
    long long t = 1;
    for (int i = 0; i < nd; ++i) t *= size[i];
    return t;
  }
};

// C[b, m, n] = alpha * sum_k A[b, m, k] B[b, k, n] + beta * C[b, m, n]
struct ContractDesc {
  Group bat, m, n, k;
  long long B = 1, M = 1, N = 1, K = 1;
  double alpha = 1.0, beta = 0.0;
  int a_k_inner = 1;   // 1 when A is contiguous along k (choose load mapping)
  int b_n_inner = 1;   // 1 when B is contiguous along n
};

// Offset of multi-index number `lin` of a group in operand X (stride array s).
__host__ __device__ inline long long group_offset(const Group& g, const long long* s, long long lin) {
  long long off = 0;
  if (lin >= 0 && lin <= 0xFFFFFFFFLL) {   // 32-bit divides: several times cheaper on the GPU
    unsigned l = (unsigned)lin;
    for (int i = g.nd - 1; i >= 0; --i) {
      const unsigned sz = (unsigned)g.size[i];
      const unsigned q = l / sz;
      off += (long long)(l - q * sz) * s[i];
      l = q;
    }
    return off;
  }
  for (int i = g.nd - 1; i >= 0; --i) {
    long long sz = g.size[i];
    long long q = lin / sz;
    off += (lin - q * sz) * s[i];
    lin = q;
  }
  return off;
}

}  // namespace sctm
