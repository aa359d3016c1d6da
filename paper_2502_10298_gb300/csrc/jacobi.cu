// Batched FP64 singular value decomposition by one-sided (Hestenes) Jacobi.
//
// Projectors need the full SVD M = U S V^T of square matrices (Sec. II.B);
// the reverse pass needs all singular vectors.  One-sided Jacobi rotates pairs
// of columns of W = M V until they are mutually orthogonal, then
// S = column norms and U = W S^{-1}.  It is accurate in the relative sense
// for small singular values, which matters because the projector divides by
// sqrt(s).  Column pairs follow the round-robin tournament ordering, so the
// n/2 rotations of a round are independent and run on separate warps.
//
// One CTA owns one matrix of the batch.  Small matrices (n <= kSmemN) live in
// shared memory; larger ones in a global workspace (kept in L2).
#include <mutex>
#include <algorithm>
#include <cstdio>
#include <cooperative_groups.h>

#include "common.h"
#include "kernels.h"
#include "prof.h"

namespace cg = cooperative_groups;

namespace sctm {

constexpr int kSvdThreads = 1024;

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Pair (i, j) of round r in the circle-method tournament over np (even) players.
__device__ inline void tournament_pair(int np, int r, int k, int& i, int& j) {
  if (k == 0) { i = r; j = np - 1; }
  else {
    int m = np - 1;
    i = (r + k) % m;
    j = (r - k + m) % m;
  }
}

// W: m x n column-major (column c at W + c*m), V: n x n column-major.
// Returns the number of sweeps used.
__device__ int jacobi_core(int m, int n, double* W, double* V, int max_sweeps, double tol, double tiny, int* flag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int np = n + (n & 1);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      for (int k = warp; k < np / 2; k += nwarp) {
        int i, j;
        tournament_pair(np, r, k, i, j);
        if (i >= n || j >= n) continue;
        if (i > j) { int t = i; i = j; j = t; }
        double* wi = W + (long long)i * m;
        double* wj = W + (long long)j * m;
        double a = 0, b = 0, g = 0;
        for (int e = lane; e < m; e += 32) {
          double x = wi[e], y = wj[e];
          a = fma(x, x, a); b = fma(y, y, b); g = fma(x, y, g);
        }
        a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
        if (g == 0.0 || fabs(g) <= tol * sqrt(a) * sqrt(b)) continue;
        // a column at rounding-noise level (norm^2 <= tiny) is still rotated, but
        // its pairs never count as unconverged: their relative orthogonality is
        // noise and would otherwise keep the sweep going to the limit
        const bool counts = a > tiny && b > tiny;
        double zeta = (b - a) / (2.0 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        for (int e = lane; e < m; e += 32) {
          double x = wi[e], y = wj[e];
          wi[e] = c * x - s * y;
          wj[e] = s * x + c * y;
        }
        double* vi = V + (long long)i * n;
        double* vj = V + (long long)j * n;
        for (int e = lane; e < n; e += 32) {
          double x = vi[e], y = vj[e];
          vi[e] = c * x - s * y;
          vj[e] = s * x + c * y;
        }
        if (lane == 0 && counts) *flag = 1;
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
  return sweep;
}

// M: batch of m x n row-major (m >= n); U: m x n, S: n, V: n x n (row-major),
// M = U diag(S) V^T with S descending.  work: batch * (m*n + n*n) doubles when
// the matrix does not fit in shared memory.  *status is set to -1 when a matrix
// did not converge.
__global__ void __launch_bounds__(kSvdThreads)
svd_kernel(int m, int n, const double* __restrict__ M, double* __restrict__ U, double* __restrict__ S,
           double* __restrict__ V, double* __restrict__ work, int* __restrict__ status, int max_sweeps,
           double tol, double noise_rel, int in_smem) {
  extern __shared__ double sm[];
  __shared__ int flag;
  const long long mn = (long long)m * n, nn = (long long)n * n;
  const int b = blockIdx.x;
  const double* Mb = M + b * mn;
  double *W, *Vw;
  if (in_smem) { W = sm; Vw = sm + mn; }
  else { W = work + b * (mn + nn); Vw = W + mn; }
  for (long long e = threadIdx.x; e < mn; e += blockDim.x) {
    int r = (int)(e / n), c = (int)(e % n);
    W[(long long)c * m + r] = Mb[e];
  }
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    int r = (int)(e / n), c = (int)(e % n);
    Vw[(long long)c * n + r] = (r == c) ? 1.0 : 0.0;
  }
  __shared__ double fro;
  if (threadIdx.x == 0) fro = 0.0;
  __syncthreads();
  {
    double a = 0;
    for (long long e = threadIdx.x; e < mn; e += blockDim.x) a = fma(Mb[e], Mb[e], a);
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) atomicAdd(&fro, a);
  }
  __syncthreads();
  // columns whose norm^2 is below noise_rel ||M||_F^2 do not count for convergence
  const double tiny = fro * noise_rel;
  int sw = jacobi_core(m, n, W, Vw, max_sweeps, tol, tiny, &flag);
  __syncthreads();
  double* Sb = S + (long long)b * n;
  for (int c = threadIdx.x >> 5; c < n; c += blockDim.x >> 5) {
    double a = 0;
    for (int e = threadIdx.x & 31; e < m; e += 32) a = fma(W[(long long)c * m + e], W[(long long)c * m + e], a);
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) Sb[c] = sqrt(a);   // unsorted for now
  }
  __syncthreads();
  double* Ub = U + b * mn;
  double* Vb = V + b * nn;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double sc = Sb[c];
    int rank = 0;
    for (int o = 0; o < n; ++o) {
      double so = Sb[o];
      rank += (so > sc) || (so == sc && o < c);
    }
    double inv = sc > 0 ? 1.0 / sc : 0.0;
    for (int e = 0; e < m; ++e) Ub[(long long)e * n + rank] = W[(long long)c * m + e] * inv;
    for (int e = 0; e < n; ++e) Vb[(long long)e * n + rank] = Vw[(long long)c * n + e];
  }
  __syncthreads();
  if (threadIdx.x == 0 && sw >= max_sweeps) atomicExch(status, -1);   // sticky failure flag
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double sc = Sb[c];
    int rank = 0;
    for (int o = 0; o < n; ++o) {
      double so = Sb[o];
      rank += (so > sc) || (so == sc && o < c);
    }
    W[rank] = sc;   // W is free now; stage the sorted values
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x) Sb[c] = W[c];
}

// ---------------------------------------------------------------- multi-CTA
// Large matrices: one persistent cooperative grid works on a batch of
// matrices.  In every tournament round each warp takes column pairs of any
// matrix of the batch; grid-wide barriers separate the rounds.  The number of
// sweeps is bounded (max_sweeps), so the kernel always terminates.
constexpr int kCoopThreads = 256;

__global__ void __launch_bounds__(kCoopThreads)
svd_coop_kernel(int m, int n, int batch, const double* __restrict__ M, double* __restrict__ U,
                double* __restrict__ S, double* __restrict__ V, double* __restrict__ work, int* __restrict__ flags,
                int* __restrict__ status, int max_sweeps, double tol, double noise_rel) {
  cg::grid_group grid = cg::this_grid();
  const long long mn = (long long)m * n, nn = (long long)n * n;
  const int lane = threadIdx.x & 31;
  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long gthread = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  // W (column-major) = M, V = I
  for (long long e = gthread; e < batch * mn; e += nthreads) {
    long long b = e / mn, r = (e % mn) / n, c = e % n;
    work[b * (mn + nn) + c * m + r] = M[e];
  }
  for (long long e = gthread; e < batch * nn; e += nthreads) {
    long long b = e / nn, r = (e % nn) / n, c = e % n;
    work[b * (mn + nn) + mn + c * n + r] = (r == c) ? 1.0 : 0.0;
  }
  double* tinyv = reinterpret_cast<double*>(flags + 64);
  if (gthread < batch) { flags[gthread] = 0; tinyv[gthread] = 0.0; }
  grid.sync();
  for (long long task = gwarp; task < (long long)batch * n; task += nwarps) {
    int b = (int)(task / n), c = (int)(task % n);
    const double* w = work + (long long)b * (mn + nn) + (long long)c * m;
    double a = 0;
    for (int e = lane; e < m; e += 32) a = fma(w[e], w[e], a);
    a = warp_sum(a);
    if (lane == 0) atomicAdd(&tinyv[b], a);
  }
  grid.sync();
  if (gthread < batch) tinyv[gthread] *= noise_rel;   // see svd_kernel
  grid.sync();
  const int np = n + (n & 1);
  const long long per = np / 2;
  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < np - 1; ++r) {
      for (long long task = gwarp; task < batch * per; task += nwarps) {
        int b = (int)(task / per), k = (int)(task % per);
        int i, j;
        tournament_pair(np, r, k, i, j);
        if (i >= n || j >= n) continue;
        if (i > j) { int t = i; i = j; j = t; }
        double* W = work + (long long)b * (mn + nn);
        double* Vw = W + mn;
        double* wi = W + (long long)i * m;
        double* wj = W + (long long)j * m;
        double a = 0, bb = 0, g = 0;
        for (int e = lane; e < m; e += 32) {
          double x = wi[e], y = wj[e];
          a = fma(x, x, a); bb = fma(y, y, bb); g = fma(x, y, g);
        }
        a = warp_sum(a); bb = warp_sum(bb); g = warp_sum(g);
        if (g == 0.0 || fabs(g) <= tol * sqrt(a) * sqrt(bb)) continue;
        const bool counts = a > tinyv[b] && bb > tinyv[b];   // see jacobi_core
        double zeta = (bb - a) / (2.0 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double sn = c * t;
        for (int e = lane; e < m; e += 32) {
          double x = wi[e], y = wj[e];
          wi[e] = c * x - sn * y;
          wj[e] = sn * x + c * y;
        }
        double* vi = Vw + (long long)i * n;
        double* vj = Vw + (long long)j * n;
        for (int e = lane; e < n; e += 32) {
          double x = vi[e], y = vj[e];
          vi[e] = c * x - sn * y;
          vj[e] = sn * x + c * y;
        }
        if (lane == 0 && counts) flags[b] = 1;
      }
      grid.sync();
    }
    bool any = false;
    for (int b = 0; b < batch; ++b) any |= (flags[b] != 0);
    grid.sync();
    if (gthread < batch) flags[gthread] = 0;
    grid.sync();
    if (!any) { converged = true; break; }
  }
  if (!converged && gthread == 0) atomicExch(status, -1);   // sticky failure flag
  // singular values (column norms), one warp per column
  for (long long task = gwarp; task < (long long)batch * n; task += nwarps) {
    int b = (int)(task / n), c = (int)(task % n);
    const double* w = work + (long long)b * (mn + nn) + (long long)c * m;
    double a = 0;
    for (int e = lane; e < m; e += 32) a = fma(w[e], w[e], a);
    a = warp_sum(a);
    if (lane == 0) S[(long long)b * n + c] = sqrt(a);   // unsorted
  }
  grid.sync();
  // ranks (descending, ties by index) -> write U, V columns; stash sorted S in flags-free scratch
  for (long long task = gthread; task < (long long)batch * n; task += nthreads) {
    int b = (int)(task / n), c = (int)(task % n);
    const double* Sb = S + (long long)b * n;
    double sc = Sb[c];
    int rank = 0;
    for (int o = 0; o < n; ++o) {
      double so = Sb[o];
      rank += (so > sc) || (so == sc && o < c);
    }
    const double* W = work + (long long)b * (mn + nn);
    const double* Vw = W + mn;
    double inv = sc > 0 ? 1.0 / sc : 0.0;
    double* Ub = U + (long long)b * mn;
    double* Vb = V + (long long)b * nn;
    for (int e = 0; e < m; ++e) Ub[(long long)e * n + rank] = W[(long long)c * m + e] * inv;
    for (int e = 0; e < n; ++e) Vb[(long long)e * n + rank] = Vw[(long long)c * n + e];
  }
  grid.sync();
  // sorted values: reuse the (now free) W column 0 of each matrix as staging
  for (long long task = gthread; task < (long long)batch * n; task += nthreads) {
    int b = (int)(task / n), c = (int)(task % n);
    const double* Sb = S + (long long)b * n;
    double sc = Sb[c];
    int rank = 0;
    for (int o = 0; o < n; ++o) {
      double so = Sb[o];
      rank += (so > sc) || (so == sc && o < c);
    }
    work[(long long)b * (mn + nn) + rank] = sc;
  }
  grid.sync();
  for (long long task = gthread; task < (long long)batch * n; task += nthreads) {
    int b = (int)(task / n), c = (int)(task % n);
    S[(long long)b * n + c] = work[(long long)b * (mn + nn) + c];
  }
}

constexpr int kMaxDevices = 64;

static bool fits_smem(int m, int n) { return (long long)(m + n) * n * 8 <= 40 * 1024; }

void launch_svd(int m, int n, int batch, const double* M, double* U, double* S, double* V, double* work,
                int* status, cudaStream_t s, double noise_rel, double tol_rel, int max_sweeps) {
  if (batch == 0 || n == 0) return;
  SCTM_CHECK(m >= n, "svd expects rows >= columns");
  char tag[96] = {0};
  if (prof_enabled())
    std::snprintf(tag, sizeof(tag), "jacobi m%d n%d batch%d%s", m, n, batch, fits_smem(m, n) ? " smem" : " coop");
  ProfTag profile_label(prof_enabled() ? tag : nullptr);
  SCTM_CHECK(max_sweeps >= 1, "svd: max_sweeps must be >= 1");
  const double tol = tol_rel > 0.0 ? tol_rel : 2.3e-16 * 4.0 * sqrt((double)m);
  const int in_smem = fits_smem(m, n);
  size_t smem = in_smem ? (size_t)(m + n) * n * sizeof(double) : 0;
  if (!in_smem) {
    // cooperative multi-CTA path; grid limited to the co-resident CTAs of the
    // current device (looked up once per device ordinal, under a lock)
    static std::mutex mu;
    static int max_ctas_of[kMaxDevices] = {0};
    int dev = 0, max_ctas = 0;
    SCTM_CUDA(cudaGetDevice(&dev));
    SCTM_CHECK(dev >= 0 && dev < kMaxDevices, "device ordinal out of range");
    {
      std::lock_guard<std::mutex> lock(mu);
      if (!max_ctas_of[dev]) {
        int sms = 0, per_sm = 0;
        SCTM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        SCTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, svd_coop_kernel, kCoopThreads, 0));
        max_ctas_of[dev] = sms * (per_sm > 0 ? per_sm : 1);
      }
      max_ctas = max_ctas_of[dev];
    }
    long long tasks = (long long)batch * ((n + 1) / 2);
    long long want = (tasks * 32 + kCoopThreads - 1) / kCoopThreads;
    int grid = (int)std::min<long long>(std::max<long long>(want, 1), max_ctas);
    SCTM_CHECK(batch <= 64, "svd batch larger than 64");
    int* flags = reinterpret_cast<int*>(work + (size_t)batch * (m + n) * n);
    ProfScope ps(PF_SVD, s, (double)batch * 8.0 * 0.5 * n * (n - 1) * (12.0 * m + 6.0 * n),
                 (double)batch * 8.0 * (2.0 * m * n + 2.0 * n * n + n));
    void* args[] = {(void*)&m, (void*)&n, (void*)&batch, (void*)&M, (void*)&U, (void*)&S, (void*)&V,
                    (void*)&work, (void*)&flags, (void*)&status, (void*)&max_sweeps, (void*)&tol, (void*)&noise_rel};
    SCTM_CUDA(cudaLaunchCooperativeKernel((void*)svd_coop_kernel, dim3(grid), dim3(kCoopThreads), args, 0, s));
    return;
  }
  // flops: one-sided Jacobi ~ 8 sweeps x n(n-1)/2 pairs x (6m + 6m + 6n) (estimate)
  ProfScope ps(PF_SVD, s, (double)batch * 8.0 * 0.5 * n * (n - 1) * (12.0 * m + 6.0 * n),
               (double)batch * 8.0 * (2.0 * m * n + 2.0 * n * n + n));
  svd_kernel<<<batch, kSvdThreads, smem, s>>>(m, n, M, U, S, V, work, status, max_sweeps, tol, noise_rel, in_smem);
  SCTM_CUDA(cudaGetLastError());
}

size_t svd_work_doubles(int m, int n, int batch) {
  return fits_smem(m, n) ? 0 : (size_t)batch * (m + n) * n + 64 + 64 + 2 * (size_t)batch;  // + flags, norms
}

}  // namespace sctm
