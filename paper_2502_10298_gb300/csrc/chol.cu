// Batched Cholesky factorisation with deflation and triangular inversion (FP64)
// for Cholesky-QR orthonormalisation in the randomized projector path.
//
// Y (m x r) = Q R with G = Y^T Y = R^T R.  A pivot below tol_rel * max_i G_ii
// marks a column that is numerically dependent on the previous ones; its row
// of R is set to zero and the matching column of Q = Y R^+ comes out zero, so
// Q always has orthonormal or zero columns (rank-deficient sketches of
// zero-padded environments are the common case).
#include <cstdio>

#include "common.h"
#include "kernels.h"
#include "prof.h"

namespace sctm {

constexpr int kCholThreads = 1024;

// One CTA per matrix; G (row-major r x r, symmetric) is overwritten in its
// upper triangle by R (the lower triangle is left untouched).
__global__ void __launch_bounds__(kCholThreads) chol_drop_kernel(int r, double* __restrict__ G, double tol_rel) {
  double* Gb = G + (long long)blockIdx.x * r * r;
  __shared__ double piv, gmax;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < r; ++i) m = fmax(m, Gb[(long long)i * r + i]);
    gmax = m;
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (threadIdx.x == 0) {
      const double d = Gb[(long long)j * r + j];
      piv = (gmax > 0.0 && d > tol_rel * gmax) ? sqrt(d) : 0.0;
      Gb[(long long)j * r + j] = piv;
    }
    __syncthreads();
    const double p = piv;
    for (int l = j + 1 + threadIdx.x; l < r; l += blockDim.x)
      Gb[(long long)j * r + l] = p > 0.0 ? Gb[(long long)j * r + l] / p : 0.0;
    __syncthreads();
    // trailing update of the upper triangle: G[i][l] -= R[j][i] R[j][l], j < i <= l
    const int w = r - j - 1;
    if (p > 0.0) {
      for (long long e = threadIdx.x; e < (long long)w * w; e += blockDim.x) {
        const int i = j + 1 + (int)(e / w), l = j + 1 + (int)(e % w);
        if (l >= i) Gb[(long long)i * r + l] -= Gb[(long long)j * r + i] * Gb[(long long)j * r + l];
      }
    }
    __syncthreads();
  }
}

// Blocked form for r <= kPanelMaxR: the factor proceeds in panels of kPanel
// rows kept in shared memory.  A panel is factored there (pivot, deflation and
// row updates as above), written back, and the trailing upper triangle gets
// one rank-kPanel update from it, so every trailing entry is read and written
// once per panel instead of once per row.
constexpr int kPanel = 32;
constexpr int kPanelMaxR = 832;   // kPanel * r doubles of shared memory <= 208 KB
constexpr int kPanelThreads = 512;

__global__ void __launch_bounds__(kPanelThreads) chol_panel_kernel(int r, double* __restrict__ G, double tol_rel) {
  extern __shared__ double P[];   // kPanel x r: P[p * r + l] = row jb + p of the factor, column l
  __shared__ double piv_s, red[kPanelThreads / 32];
  double* Gb = G + (long long)blockIdx.x * r * r;
  const int tid = threadIdx.x, nt = blockDim.x;
  // largest diagonal entry (deflation reference)
  double m = 0.0;
  for (int i = tid; i < r; i += nt) m = fmax(m, Gb[(long long)i * r + i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  double gmax = 0.0;
  for (int w = 0; w < nt / 32; ++w) gmax = fmax(gmax, red[w]);
  for (int jb = 0; jb < r; jb += kPanel) {
    const int pw = min(kPanel, r - jb), wc = r - jb;
    for (int e = tid; e < pw * wc; e += nt) {
      const int p = e / wc, l = jb + e % wc;
      P[p * r + l] = (l >= jb + p) ? Gb[(long long)(jb + p) * r + l] : 0.0;
    }
    __syncthreads();
    for (int p = 0; p < pw; ++p) {
      const int j = jb + p;
      if (tid == 0) {
        const double d = P[p * r + j];
        piv_s = (gmax > 0.0 && d > tol_rel * gmax) ? sqrt(d) : 0.0;
        P[p * r + j] = piv_s;
      }
      __syncthreads();
      const double piv = piv_s;
      for (int l = j + 1 + tid; l < r; l += nt) P[p * r + l] = piv > 0.0 ? P[p * r + l] / piv : 0.0;
      __syncthreads();
      const int wr = r - j - 1, rows = pw - p - 1;
      if (piv > 0.0)
        for (int e = tid; e < rows * wr; e += nt) {
          const int q = p + 1 + e / wr, l = j + 1 + e % wr;
          if (l >= jb + q) P[q * r + l] -= P[p * r + jb + q] * P[p * r + l];
        }
      __syncthreads();
    }
    for (int e = tid; e < pw * wc; e += nt) {
      const int p = e / wc, l = jb + e % wc;
      if (l >= jb + p) Gb[(long long)(jb + p) * r + l] = P[p * r + l];
    }
    // trailing update: G[i][l] -= sum_p R[jb+p][i] R[jb+p][l], jb + pw <= i <= l
    const int t0 = jb + pw, w = r - t0;
    for (long long e = tid; e < (long long)w * w; e += nt) {
      const int i = t0 + (int)(e / w), l = t0 + (int)(e % w);
      if (l < i) continue;
      double acc = 0.0;
      for (int p = 0; p < pw; ++p) acc = fma(P[p * r + i], P[p * r + l], acc);
      Gb[(long long)i * r + l] -= acc;
    }
    __syncthreads();
  }
}

// T = R^+ (upper triangular; rows/columns of zero pivots are zero).  One warp
// per column; the column being built is kept in shared memory.
constexpr int kTriWarps = 8;
__global__ void __launch_bounds__(32 * kTriWarps) tri_inv_kernel(int r, const double* __restrict__ R,
                                                                 double* __restrict__ T) {
  extern __shared__ double col_sm[];   // kTriWarps x r
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cols_per_mat = (r + kTriWarps - 1) / kTriWarps;
  const int b = blockIdx.x / cols_per_mat;
  const int c = (blockIdx.x % cols_per_mat) * kTriWarps + warp;
  if (c >= r) return;
  const double* Rb = R + (long long)b * r * r;
  double* Tb = T + (long long)b * r * r;
  double* t = col_sm + warp * r;
  for (int i = lane; i < r; i += 32) t[i] = 0.0;
  __syncwarp();
  const double rcc = Rb[(long long)c * r + c];
  if (lane == 0) t[c] = rcc > 0.0 ? 1.0 / rcc : 0.0;
  __syncwarp();
  for (int i = c - 1; i >= 0; --i) {
    const double rii = Rb[(long long)i * r + i];
    double acc = 0.0;
    if (rii > 0.0)
      for (int l = i + 1 + lane; l <= c; l += 32) acc = fma(Rb[(long long)i * r + l], t[l], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) t[i] = rii > 0.0 ? -acc / rii : 0.0;
    __syncwarp();
  }
  for (int i = lane; i < r; i += 32) Tb[(long long)i * r + c] = t[i];
}

void launch_chol_qr_factor(int r, int batch, double* G, double* T, double tol_rel, cudaStream_t s) {
  if (batch == 0 || r == 0) return;
  SCTM_CHECK(r <= 2048, "Cholesky factor larger than 2048");
  char tag[64] = {0};
  if (prof_enabled()) std::snprintf(tag, sizeof(tag), "cholesky r%d batch%d", r, batch);
  ProfTag profile_label(prof_enabled() ? tag : nullptr);
  {
    ProfScope ps(PF_SVD, s, (double)batch * r * (double)r * r / 3.0, (double)batch * 16.0 * r * r);
    if (r <= kPanelMaxR) {
      const size_t psm = (size_t)kPanel * r * sizeof(double);
      // opt in once to the largest panel: the kernel's static shared memory
      // comes on top of the dynamic part, so even 48 KB of panel needs it
      static bool attr = false;
      if (!attr) {
        SCTM_CUDA(cudaFuncSetAttribute(chol_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((size_t)kPanel * kPanelMaxR * sizeof(double))));
        attr = true;
      }
      chol_panel_kernel<<<batch, kPanelThreads, psm, s>>>(r, G, tol_rel);
    } else {
      chol_drop_kernel<<<batch, kCholThreads, 0, s>>>(r, G, tol_rel);
    }
    SCTM_CUDA(cudaGetLastError());
  }
  ProfScope ps(PF_SVD, s, (double)batch * r * (double)r * r / 3.0, (double)batch * 16.0 * r * r);
  const int cols_per_mat = (r + kTriWarps - 1) / kTriWarps;
  const size_t smem = (size_t)kTriWarps * r * sizeof(double);
  if (smem >= 48 * 1024)
    SCTM_CUDA(cudaFuncSetAttribute(tri_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  tri_inv_kernel<<<batch * cols_per_mat, 32 * kTriWarps, smem, s>>>(r, G, T);
  SCTM_CUDA(cudaGetLastError());
}

}  // namespace sctm
