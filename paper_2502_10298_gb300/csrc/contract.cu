// Strided batched tensor contraction on CUDA cores (FP64 storage; FP64 or FP32 arithmetic).
//
// Every pairwise contraction of the split-CTMRG networks (absorption
// equations, rho networks, M = rho^B rho^T, projector application) is
// C[b,m,n] = alpha * sum_k A[b,m,k] B[b,k,n] + beta * C[b,m,n], where each of
// b, m, n, k is a group of tensor legs with arbitrary strides.  Index
// permutations are therefore never materialised: a tile loader gathers
// operand elements through per-tile offset tables kept in shared memory.
#include <algorithm>

#include "common.h"
#include "kernels.h"
#include "prof.h"

namespace sctm {

template <typename T, typename Tc, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
contract_kernel(ContractDesc d, const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ C,
                long long kchunk, double* __restrict__ W) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int TX = BN / TN;
  __shared__ long long offAm[BM], offCm[BM], offBn[BN], offCn[BN];
  __shared__ long long offAk[BK], offBk[BK];
  __shared__ Tc As[BK][BM + 1];
  __shared__ Tc Bs[BK][BN + 1];

  const int tid = threadIdx.x;
  const long long b = blockIdx.z;
  const long long ntn = (d.N + BN - 1) / BN;
  const long long tile = blockIdx.x;
  const long long m0 = (tile / ntn) * BM;
  const long long n0 = (tile % ntn) * BN;
  const long long boA = group_offset(d.bat, d.bat.sa, b);
  const long long boB = group_offset(d.bat, d.bat.sb, b);
  const long long boC = group_offset(d.bat, d.bat.sc, b);
  for (int i = tid; i < BM; i += NT) {
    long long m = m0 + i;
    if (m < d.M) {
      offAm[i] = boA + group_offset(d.m, d.m.sa, m);
      offCm[i] = boC + group_offset(d.m, d.m.sc, m);
    } else {
      offAm[i] = -1;
      offCm[i] = -1;
    }
  }
  for (int i = tid; i < BN; i += NT) {
    long long n = n0 + i;
    if (n < d.N) {
      offBn[i] = boB + group_offset(d.n, d.n.sb, n);
      offCn[i] = group_offset(d.n, d.n.sc, n);
    } else {
      offBn[i] = -1;
      offCn[i] = -1;
    }
  }
  const int ty = tid / TX, tx = tid % TX;
  Tc acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Tc(0);

  // split K (gridDim.y > 1): this CTA sums k in [kb, ke) into the FP64 buffer W
  const long long kb = (long long)blockIdx.y * kchunk;
  const long long ke = min(d.K, kb + kchunk);
  for (long long k0 = kb; k0 < ke; k0 += BK) {
    __syncthreads();
    if (tid < BK) {
      long long k = k0 + tid;
      offAk[tid] = (k < ke) ? group_offset(d.k, d.k.sa, k) : -1;
      offBk[tid] = (k < ke) ? group_offset(d.k, d.k.sb, k) : -1;
    }
    __syncthreads();
    for (int idx = tid; idx < BM * BK; idx += NT) {
      int mm, kk;
      if (d.a_k_inner) { kk = idx % BK; mm = idx / BK; }
      else { mm = idx % BM; kk = idx / BM; }
      long long om = offAm[mm], ok = offAk[kk];
      As[kk][mm] = (om >= 0 && ok >= 0) ? (Tc)A[om + ok] : Tc(0);
    }
    for (int idx = tid; idx < BN * BK; idx += NT) {
      int nn, kk;
      if (d.b_n_inner) { nn = idx % BN; kk = idx / BN; }
      else { kk = idx % BK; nn = idx / BK; }
      long long on = offBn[nn], ok = offBk[kk];
      Bs[kk][nn] = (on >= 0 && ok >= 0) ? (Tc)B[on + ok] : Tc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Tc a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + j * TX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
  }
  __syncthreads();
  const T alpha = (T)d.alpha, beta = (T)d.beta;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int mm = ty + i * (BM / TM);
    long long om = offCm[mm];
    if (om < 0) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int nn = tx + j * TX;
      long long on = offCn[nn];
      if (on < 0) continue;
      if (W) {
        atomicAdd(&W[(b * d.M + m0 + mm) * d.N + n0 + nn], (double)acc[i][j]);
        continue;
      }
      T v = alpha * (T)acc[i][j];
      if (d.beta != 0.0) v += beta * C[om + on];
      C[om + on] = v;
    }
  }
}

// C = alpha W + beta C through the output strides, W[b][m][n] (Wm x Wn per batch)
__global__ void splitk_finish_kernel(ContractDesc d, long long Wm, long long Wn, const double* __restrict__ W,
                                     double* __restrict__ C) {
  const long long total = d.B * d.M * d.N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long n = idx % d.N, m = (idx / d.N) % d.M, b = idx / (d.N * d.M);
    const long long off = group_offset(d.bat, d.bat.sc, b) + group_offset(d.m, d.m.sc, m) +
                          group_offset(d.n, d.n.sc, n);
    double v = d.alpha * W[(b * Wm + m) * Wn + n];
    if (d.beta != 0.0) v += d.beta * C[off];
    C[off] = v;
  }
}

void launch_splitk_finish(const ContractDesc& d, long long Wm, long long Wn, const double* W, double* C,
                          cudaStream_t s) {
  const long long total = d.B * d.M * d.N;
  if (total == 0) return;
  ProfScope pf(PF_MISC, s, 0.0, 8.0 * total * (d.beta != 0 ? 3 : 2), 1, "splitk_finish");
  const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, kNumSMs * 16);
  splitk_finish_kernel<<<blocks, 256, 0, s>>>(d, Wm, Wn, W, C);
  SCTM_CUDA(cudaGetLastError());
}

namespace {
constexpr int kCBM = 64, kCBN = 64, kCBK = 16;
// K splits for outputs with too few 64 x 64 tiles (Gram matrices of tall bases):
// one K block per split at the least, because an SM retires only a few FP64
// multiply-adds per clock and a small output must still occupy every SM
long long contract_splits(const ContractDesc& d) {
  const long long tiles = ((d.M + kCBM - 1) / kCBM) * ((d.N + kCBN - 1) / kCBN) * d.B;
  const long long want = (2 * kNumSMs + tiles - 1) / tiles;
  long long sp = std::min<long long>(want, d.K / kCBK);
  if (sp < 2 || d.B > 65535) return 1;
  return std::min<long long>(sp, 65535);
}
long long contract_max_splits(const ContractDesc& d) {
  const long long tiles = ((d.M + kCBM - 1) / kCBM) * ((d.N + kCBN - 1) / kCBN) * d.B;
  if (tiles >= 2 * kNumSMs || d.B > 65535) return 1;
  return std::max<long long>(1, std::min<long long>(d.K / kCBK, 65535));
}
}  // namespace

int contract_split_rule(const ContractDesc& d) { return (int)contract_splits(d); }
int contract_split_max(const ContractDesc& d) { return (int)contract_max_splits(d); }

size_t contract_scratch_doubles(const ContractDesc& d) {
  return contract_max_splits(d) > 1 ? (size_t)(d.B * d.M * d.N) + 32 : 0;
}

template <typename T>
void launch_contract(const ContractDesc& d, const T* A, const T* B, T* C, cudaStream_t s, bool fp32_compute,
                     double* scratch, int splits_req) {
  if (d.M == 0 || d.N == 0 || d.B == 0) return;
  constexpr int BM = kCBM, BN = kCBN, BK = kCBK, TM = 4, TN = 4;
  long long tiles = ((d.N + BN - 1) / BN) * ((d.M + BM - 1) / BM);
  SCTM_CHECK(tiles < (1LL << 31) && d.B <= 65535, "contraction too large for grid");
  long long splits = scratch ? contract_splits(d) : 1;
  if (scratch && splits_req > 0) splits = std::min<long long>(splits_req, contract_max_splits(d));
  const long long kchunk = splits > 1 ? (((d.K + splits - 1) / splits + BK - 1) / BK) * BK : d.K;
  const long long nsplit = (d.K + kchunk - 1) / kchunk;
  double* W = nullptr;
  if (splits > 1) {
    W = scratch;
    SCTM_CUDA(cudaMemsetAsync(W, 0, (size_t)(d.B * d.M * d.N) * sizeof(double), s));
  }
  dim3 grid((unsigned)tiles, (unsigned)(splits > 1 ? nsplit : 1), (unsigned)d.B);
  // algorithmic work: 2 B M N K flops; bytes = operands read once + result written
  {
    ProfScope ps(PF_CONTRACT, s, 2.0 * d.B * d.M * d.N * d.K,
                 (double)sizeof(T) * d.B * (d.M * d.K + d.K * d.N + d.M * d.N * (d.beta != 0 ? 2 : 1)));
    if (fp32_compute)
      contract_kernel<T, float, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(d, A, B, C, kchunk, W);
    else
      contract_kernel<T, T, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(d, A, B, C, kchunk, W);
    SCTM_CUDA(cudaGetLastError());
  }
  if (W) launch_splitk_finish(d, d.M, d.N, W, C, s);
}

template void launch_contract<double>(const ContractDesc&, const double*, const double*, double*, cudaStream_t, bool,
                                      double*, int);

// ------------------------------------------------------------ symmetric Gram
// G = Y^T Y (r x r) of a row-major m x r block Y (row stride ldy), FP64: only
// the 64 x 64 tiles on and above the diagonal are formed, each CTA summing
// one range of rows into W (zeroed) with atomics; gram_mirror_kernel then
// writes both triangles.  The product is symmetric, so this is the full Gram
// matrix for about (T + 1) / (2 T) of the multiply-adds (T tiles per side).
constexpr int kGT = 64, kGK = 16;

__global__ void __launch_bounds__(256) gram_upper_kernel(long long m, int r, const double* __restrict__ Y,
                                                         long long ldy, long long rchunk, double* __restrict__ W) {
  __shared__ double As[kGK][kGT + 1], Bs[kGK][kGT + 1];
  const int T = (r + kGT - 1) / kGT;
  // tile pair (ti <= tj) of the upper triangle, row by row
  int t = blockIdx.x, ti = 0;
  while (t >= T - ti) t -= T - ti, ++ti;
  const int tj = ti + t;
  const int i0 = ti * kGT, j0 = tj * kGT;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  double acc[4][4] = {{0.0}};
  const long long kb = (long long)blockIdx.y * rchunk, ke = min(m, kb + rchunk);
  for (long long k0 = kb; k0 < ke; k0 += kGK) {
    __syncthreads();
    for (int idx = tid; idx < kGK * kGT; idx += 256) {
      const int kk = idx / kGT, c = idx % kGT;
      const long long k = k0 + kk;
      const bool in = k < ke;
      As[kk][c] = (in && i0 + c < r) ? Y[k * ldy + i0 + c] : 0.0;
      Bs[kk][c] = (in && j0 + c < r) ? Y[k * ldy + j0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gi = i0 + ty + 16 * i, gj = j0 + tx + 16 * j;
      if (gi < r && gj < r && gi <= gj) atomicAdd(&W[(long long)gi * r + gj], acc[i][j]);
    }
}

__global__ void gram_mirror_kernel(int r, const double* __restrict__ W, double* __restrict__ G, long long ldg) {
  const long long total = (long long)r * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    G[(long long)i * ldg + j] = i <= j ? W[(long long)i * r + j] : W[(long long)j * r + i];
  }
}

void launch_gram(long long m, int r, const double* Y, long long ldy, double* G, long long ldg, double* W,
                 cudaStream_t s) {
  if (r == 0) return;
  SCTM_CUDA(cudaMemsetAsync(W, 0, (size_t)r * r * sizeof(double), s));
  const int T = (r + kGT - 1) / kGT;
  const long long tiles = (long long)T * (T + 1) / 2;
  // splits over the rows until about two CTAs per SM, at least one row block each
  long long splits = std::max<long long>(1, std::min<long long>((2 * kNumSMs + tiles - 1) / tiles,
                                                                (m + kGK - 1) / kGK));
  splits = std::min<long long>(splits, 65535);
  const long long rchunk = ((m + splits - 1) / splits + kGK - 1) / kGK * kGK;
  splits = m > 0 ? (m + rchunk - 1) / rchunk : 1;
  {
    ProfScope ps(PF_CONTRACT, s, 2.0 * m * (double)r * r, 8.0 * m * r + 8.0 * r * r, 1, "gram");
    if (m > 0) {
      gram_upper_kernel<<<dim3((unsigned)tiles, (unsigned)splits), 256, 0, s>>>(m, r, Y, ldy, rchunk, W);
      SCTM_CUDA(cudaGetLastError());
    }
  }
  ProfScope pf(PF_MISC, s, 0.0, 16.0 * r * r, 1, "gram_mirror");
  const unsigned blocks = (unsigned)std::min<long long>(((long long)r * r + 255) / 256, kNumSMs * 8);
  gram_mirror_kernel<<<blocks, 256, 0, s>>>(r, W, G, ldg);
  SCTM_CUDA(cudaGetLastError());
}

}  // namespace sctm
