// Differentiable device operations of the engine.  Every op launches one of
// the kernels of this directory and, while the tape is active, records the
// closure that accumulates the adjoints of its inputs.
#pragma once
#include <array>
#include <map>
#include <string>
#include <vector>

#include "kernels.h"
#include "tensor.h"

namespace sctm {

struct Ctx {
  cudaStream_t stream = nullptr;
  Arena arena;
  Tape tape;
  double* partial = nullptr;     // reduction scratch (persistent)
  int* svd_status = nullptr;     // per-call SVD sweep counts (persistent, device)
  int svd_status_cap = 0;
  bool svd_failed = false;
  bool fp32_compute = false;     // mixed mode: contractions in FP32 arithmetic
  bool tensor_cores = true;      // mixed mode: large contractions on tcgen05 (3xTF32)
  bool bf16_slices = false;      // tensor-core contractions as BF16 digit slices (precision 4)
  int accurate = 0;              // > 0: inside an AccurateScope (see ctmrg.cu)
  // Randomized projector decompositions (U, S, V of each truncated SVD) of one
  // move: recorded by the forward pass into the arena's high stack and replayed
  // by the taped recomputation of the same move in the reverse pass, which
  // then skips the subspace iteration.  mode 0 off, 1 record, 2 replay.
  struct DecompCache {
    int mode = 0;
    std::vector<std::array<Tensor, 3>> entries;
    size_t next = 0;
  } decomp;
  // BF16-slice panels of operands that are reused while a scope runs (the rho
  // halves of the randomized projectors): `slice_keep` lists their data
  // pointers, `slice_panels` the panels packed so far (in the arena's high
  // stack), keyed by the operand's layout in the contraction.
  std::vector<const double*> slice_keep;
  std::vector<std::pair<std::vector<long long>, SlicePanel>> slice_panels;
  // Split-K autotuner (see einsum_into): per contraction shape, the split
  // counts tried, their device times, and the choice once all are timed.
  struct Tune {
    std::vector<int> cand;
    std::vector<float> ms;
    int next = 0, pending = -1, chosen = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
  };
  bool autotune = false;
  std::map<std::vector<long long>, Tune> tune;
  int svd_max_sweeps = 60;       // Jacobi sweep limit (fault-injection hook: sctm_set_limits)
  unsigned long long pipe_wait_ns = 2000000000ull;   // tensor-core main-loop wait limit (same hook)

  // new contiguous tensor of the given shape; gradient buffer (zeroed) when taping
  Tensor empty(std::initializer_list<int> shape);
  Tensor empty_shape(const int* shape, int nd);
  Tensor zeros(std::initializer_list<int> shape);
  Tensor scalar();
  void zero_grad(const Tensor& t);
  void ensure_grad(Tensor& t);
};

// C = alpha * einsum(spec, A, B) (+ beta * C when C is given and beta != 0).
// spec like "ab,aui->bui"; an index may appear in A and/or B and/or C, but an
// index of a single input must also be in C.
Tensor einsum(Ctx& c, const char* spec, const Tensor& A, const Tensor& B, double alpha = 1.0);
void einsum_into(Ctx& c, const char* spec, const Tensor& A, const Tensor& B, const Tensor& C,
                 double alpha, double beta, bool record);

// SVD of an m x n matrix, m >= n (any strides): M = U S V^T, U m x n, V n x n.
struct SVDResult {
  Tensor U, S, V;
};
SVDResult svd(Ctx& c, const Tensor& M, double eps_l);
// SVDs of equally shaped matrices in one launch, each with its own adjoint
std::vector<SVDResult> svd_many(Ctx& c, const std::vector<Tensor>& Ms, double eps_l);

// w[k] = f(S[k]) for k < kout with a cutoff relative to S[0] (see kernels.h modes)
Tensor spectrum_map(Ctx& c, const Tensor& S, int kout, double cutoff, int mode);

// Y = X scaled along `dim` by vector v (v may be a constant without gradient)
Tensor scale_dim(Ctx& c, const Tensor& X, int dim, const Tensor& v);

// Sign vector of a matrix: sign of the largest-|.| entry of each row (constant)
Tensor row_signs(Ctx& c, const Tensor& P);

// Contiguous copy of a view, or copy into an existing view (accumulating adjoints)
Tensor copy(Ctx& c, const Tensor& X);
void copy_into(Ctx& c, const Tensor& X, const Tensor& Y);

// Y = X / max|X| (contiguous X)
Tensor rescale(Ctx& c, const Tensor& X);

// scalar = sum X .* Y over two equally shaped views (copied to contiguous)
Tensor dot(Ctx& c, const Tensor& X, const Tensor& Y);

Tensor from_host(Ctx& c, std::initializer_list<int> shape, const double* host);
std::vector<double> to_host(Ctx& c, const Tensor& t);

}  // namespace sctm
