// Small memory-bound kernels of the engine: strided copies, row/column
// scaling, spectrum maps, sign fixing, max-abs rescaling and dot products.
#include <algorithm>

#include "common.h"
#include "kernels.h"
#include "prof.h"

namespace sctm {

constexpr int kThreads = 256;

template <typename T>
__global__ void copy_kernel(Group g, long long total, T alpha, const T* __restrict__ in, T beta,
                            T* __restrict__ out) {
  for (long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x; lin < total;
       lin += (long long)gridDim.x * blockDim.x) {
    long long oi = group_offset(g, g.sa, lin);
    long long oo = group_offset(g, g.sc, lin);
    T v = alpha * in[oi];
    if (beta != T(0)) v += beta * out[oo];
    out[oo] = v;
  }
}

static unsigned grid_for(long long total) {
  long long g = (total + kThreads - 1) / kThreads;
  if (g > kNumSMs * 32) g = kNumSMs * 32;
  if (g < 1) g = 1;
  return (unsigned)g;
}

template <typename T>
void launch_copy(const Group& g, T alpha, const T* in, T beta, T* out, cudaStream_t s) {
  long long total = g.total();
  if (total == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 8.0 * total * (beta != T(0) ? 3 : 2), 1, "copy");
  copy_kernel<T><<<grid_for(total), kThreads, 0, s>>>(g, total, alpha, in, beta, out);
  SCTM_CUDA(cudaGetLastError());
}
template void launch_copy<double>(const Group&, double, const double*, double, double*, cudaStream_t);
template void launch_copy<float>(const Group&, float, const float*, float, float*, cudaStream_t);

__global__ void scale_rc_kernel(int batch, int rows, int cols, double* X, const double* v, int vstride,
                                bool row) {
  long long per = (long long)rows * cols, total = per * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long b = e / per, r = (e % per) / cols, c = e % cols;
    X[e] *= v[b * vstride + (row ? r : c)];
  }
}

void launch_scale_rc(int batch, int rows, int cols, double* X, const double* v, int vstride, bool row,
                     cudaStream_t s) {
  long long total = (long long)batch * rows * cols;
  if (total == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "scale_rc");
  scale_rc_kernel<<<grid_for(total), kThreads, 0, s>>>(batch, rows, cols, X, v, vstride, row);
  SCTM_CUDA(cudaGetLastError());
}

__global__ void spectrum_map_kernel(int batch, int n, int kout, const double* S, double* w, double cutoff,
                                    int mode) {
  int total = batch * kout;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int b = e / kout, k = e % kout;
    double s0 = S[(long long)b * n];
    double sk = (k < n) ? S[(long long)b * n + k] : 0.0;
    bool keep = (k < n) && (sk > cutoff * s0) && (s0 > 0);
    double r = 0.0;
    if (keep) r = (mode == 0) ? 1.0 / sqrt(sk) : (mode == 1 ? sqrt(sk) : 1.0);
    w[e] = r;
  }
}

void launch_spectrum_map(int batch, int n, int kout, const double* S, double* w, double cutoff, int mode,
                         cudaStream_t s) {
  if (batch * kout == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "spectrum_map");
  spectrum_map_kernel<<<grid_for(batch * kout), kThreads, 0, s>>>(batch, n, kout, S, w, cutoff, mode);
  SCTM_CUDA(cudaGetLastError());
}

// one warp per row
__global__ void sign_find_kernel(int rows, int cols, const double* P, long long rs, long long cs, double* sgn) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= rows) return;
  const double* row = P + (long long)warp * rs;
  double best = -1.0, val = 0.0;
  int bi = 0x7fffffff;
  for (int e = lane; e < cols; e += 32) {
    double x = row[e * cs], ax = fabs(x);
    if (ax > best || (ax == best && e < bi)) { best = ax; val = x; bi = e; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    double ov = __shfl_xor_sync(0xffffffffu, val, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; val = ov; bi = oi; }
  }
  if (lane == 0) sgn[warp] = (val < 0) ? -1.0 : 1.0;
}

void launch_sign_find(int rows, int cols, const double* P, long long rs, long long cs, double* sgn,
                      cudaStream_t s) {
  if (rows == 0) return;
  long long threads = (long long)rows * 32;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "sign_find");
  sign_find_kernel<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, s>>>(rows, cols, P, rs, cs, sgn);
  SCTM_CUDA(cudaGetLastError());
}

__global__ void svd_adj_inner_kernel(int n, const double* S, const double* J, const double* K,
                                     const double* Sbar, double* inner, double eps) {
  double smax = S[0];
  double e4 = eps * smax * smax * smax * smax;
  long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    double v;
    if (i == j) v = Sbar ? Sbar[i] : 0.0;
    else {
      double si = S[i], sj = S[j];
      double d = sj * sj - si * si;
      double F = d / (d * d + e4 + 1e-300);
      double jj = J[(long long)i * n + j] - J[(long long)j * n + i];
      double kk = K[(long long)i * n + j] - K[(long long)j * n + i];
      v = F * jj * sj + si * F * kk;
    }
    inner[e] = v;
  }
}

void launch_svd_adj_inner(int n, const double* S, const double* J, const double* K, const double* Sbar,
                          double* inner, double eps, cudaStream_t s) {
  long long total = (long long)n * n;
  if (total == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "svd_adj_inner");
  svd_adj_inner_kernel<<<grid_for(total), kThreads, 0, s>>>(n, S, J, K, Sbar, inner, eps);
  SCTM_CUDA(cudaGetLastError());
}

__global__ void spectrum_adj_kernel(int n, int kout, const double* S, const double* wbar, double* Sbar,
                                    double cutoff, int mode) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kout || k >= n) return;
  double s0 = S[0], sk = S[k];
  bool keep = (sk > cutoff * s0) && (s0 > 0);
  if (!keep || mode == 2) return;
  double d = (mode == 0) ? -0.5 / (sk * sqrt(sk)) : 0.5 / sqrt(sk);
  Sbar[k] += wbar[k] * d;
}

void launch_spectrum_adj(int n, int kout, const double* S, const double* wbar, double* Sbar, double cutoff,
                         int mode, cudaStream_t s) {
  if (kout == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "spectrum_adj");
  spectrum_adj_kernel<<<(kout + 255) / 256, 256, 0, s>>>(n, kout, S, wbar, Sbar, cutoff, mode);
  SCTM_CUDA(cudaGetLastError());
}

__global__ void rescale_adj_kernel(long long n, const double* ybar, const double* y, const double* m,
                                   const long long* k, const double* xk_sign, const double* dot, double* xbar) {
  double mm = *m;
  if (mm <= 0) return;
  double inv = 1.0 / mm;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double v = ybar[e] * inv;
    if (e == *k) v -= (xk_sign ? *xk_sign : y[e]) * (*dot) * inv;
    xbar[e] += v;
  }
}

void launch_rescale_adj(long long n, const double* ybar, const double* y, const double* m, const long long* k,
                        const double* xk_sign, const double* dot, double* xbar, cudaStream_t s) {
  if (n == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "rescale_adj");
  rescale_adj_kernel<<<grid_for(n), kThreads, 0, s>>>(n, ybar, y, m, k, xk_sign, dot, xbar);
  SCTM_CUDA(cudaGetLastError());
}

// ---- max-abs rescale: two-level reduction (value, index) then scaling
struct MaxIdx { double v; long long i; };

__device__ inline MaxIdx better(MaxIdx a, MaxIdx b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}

constexpr int kRedBlocks = 64;

__global__ void maxabs_partial_kernel(long long n, const double* X, long long stride, double* partial) {
  int b = blockIdx.y;
  const double* x = X + b * stride;
  MaxIdx m{-1.0, 0x7fffffffffffffffLL};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    m = better(m, MaxIdx{fabs(x[e]), e});
  __shared__ double sv[kThreads];
  __shared__ long long si[kThreads];
  sv[threadIdx.x] = m.v; si[threadIdx.x] = m.i;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      MaxIdx r = better(MaxIdx{sv[threadIdx.x], si[threadIdx.x]}, MaxIdx{sv[threadIdx.x + o], si[threadIdx.x + o]});
      sv[threadIdx.x] = r.v; si[threadIdx.x] = r.i;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[(b * kRedBlocks + blockIdx.x) * 2] = sv[0];
    partial[(b * kRedBlocks + blockIdx.x) * 2 + 1] = (double)si[0];
  }
}

__global__ void maxabs_final_scale_kernel(long long n, double* X, long long stride, const double* partial,
                                          double* scale, long long* argmax) {
  int b = blockIdx.x;
  __shared__ double m;
  __shared__ long long mi;
  (void)mi;
  if (threadIdx.x == 0) {
    MaxIdx r{-1.0, 0x7fffffffffffffffLL};
    for (int i = 0; i < kRedBlocks; ++i)
      r = better(r, MaxIdx{partial[(b * kRedBlocks + i) * 2], (long long)partial[(b * kRedBlocks + i) * 2 + 1]});
    m = r.v; mi = r.i;
    scale[b] = r.v;
    if (argmax) argmax[b] = r.i;
  }
  __syncthreads();
  if (m <= 0) return;
  double inv = 1.0 / m;
  double* x = X + b * stride;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) x[e] *= inv;
}

void launch_rescale(int batch, long long n, double* X, long long stride, double* scale, long long* argmax,
                    double* partial, cudaStream_t s) {
  if (batch == 0 || n == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 2, "rescale");
  maxabs_partial_kernel<<<dim3(kRedBlocks, batch), kThreads, 0, s>>>(n, X, stride, partial);
  SCTM_CUDA(cudaGetLastError());
  maxabs_final_scale_kernel<<<batch, 1024, 0, s>>>(n, X, stride, partial, scale, argmax);
  SCTM_CUDA(cudaGetLastError());
}

__global__ void dot_partial_kernel(long long n, const double* x, const double* y, long long stride, double* partial) {
  int b = blockIdx.y;
  double acc = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    acc = fma(x[b * stride + e], y[b * stride + e], acc);
  __shared__ double sv[kThreads];
  sv[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sv[threadIdx.x] += sv[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[b * kRedBlocks + blockIdx.x] = sv[0];
}

__global__ void dot_final_kernel(int batch, const double* partial, double* out) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double acc = 0;
  for (int i = 0; i < kRedBlocks; ++i) acc += partial[b * kRedBlocks + i];
  out[b] = acc;
}

void launch_dot(int batch, long long n, const double* x, const double* y, long long stride, double* out,
                double* partial, cudaStream_t s) {
  if (batch == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 2, "dot");
  dot_partial_kernel<<<dim3(kRedBlocks, batch), kThreads, 0, s>>>(n, x, y, stride, partial);
  SCTM_CUDA(cudaGetLastError());
  dot_final_kernel<<<(batch + 127) / 128, 128, 0, s>>>(batch, partial, out);
  SCTM_CUDA(cudaGetLastError());
}

__global__ void fill_kernel(long long n, double v, double* x) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    x[e] = v;
}
__global__ void axpy_kernel(long long n, double a, const double* x, double* y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = fma(a, x[e], y[e]);
}
void launch_fill(long long n, double v, double* x, cudaStream_t s) {
  if (n == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "fill");
  fill_kernel<<<grid_for(n), kThreads, 0, s>>>(n, v, x);
  SCTM_CUDA(cudaGetLastError());
}
void launch_axpy(long long n, double a, const double* x, double* y, cudaStream_t s) {
  if (n == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "axpy");
  axpy_kernel<<<grid_for(n), kThreads, 0, s>>>(n, a, x, y);
  SCTM_CUDA(cudaGetLastError());
}

// SplitMix64 finaliser as a counter-based generator; two uniforms -> one normal
__device__ inline unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void gaussian_kernel(long long n, unsigned long long seed, double* X) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    unsigned long long a = mix64(seed ^ (2 * (unsigned long long)e)), b = mix64(seed ^ (2 * (unsigned long long)e + 1));
    double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740994.0);   // (0, 1]
    double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    X[e] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

void launch_gaussian(long long rows, long long cols, unsigned long long seed, double* X, cudaStream_t s) {
  long long n = rows * cols;
  if (n == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "gaussian");
  gaussian_kernel<<<grid_for(n), kThreads, 0, s>>>(n, seed, X);
  SCTM_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- scaling
__global__ void axpy_dev_kernel(long long n, const double* __restrict__ a, const double* __restrict__ x,
                                double* __restrict__ y) {
  const double av = a[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(av, x[i], y[i]);
}

void launch_axpy_dev(long long n, const double* a, const double* x, double* y, cudaStream_t s) {
  if (n == 0) return;
  ProfScope ps_(PF_MISC, s, 2.0 * n, 24.0 * n, 1, "axpy_dev");
  axpy_dev_kernel<<<grid_for(n), kThreads, 0, s>>>(n, a, x, y);
  SCTM_CUDA(cudaGetLastError());
}

// out[g] = in[g] * v[index of dim `dim`] + beta * out[g] over the group g (strides .sa = in, .sc = out)
__global__ void scale_dim_kernel(Group g, long long total, int dim, const double* __restrict__ in,
                                 const double* __restrict__ v, double beta, double* __restrict__ out) {
  long long inner = 1;
  for (int i = g.nd - 1; i > dim; --i) inner *= g.size[i];
  const long long sz = g.size[dim];
  for (long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x; lin < total;
       lin += (long long)gridDim.x * blockDim.x) {
    const long long oi = group_offset(g, g.sa, lin), oo = group_offset(g, g.sc, lin);
    double r = in[oi] * v[(lin / inner) % sz];
    if (beta != 0.0) r += beta * out[oo];
    out[oo] = r;
  }
}

void launch_scale_dim(const Group& g, int dim, const double* in, const double* v, double beta, double* out,
                      cudaStream_t s) {
  const long long total = g.total();
  if (total == 0) return;
  ProfScope ps_(PF_MISC, s, (double)total, 24.0 * total, 1, "scale_dim");
  scale_dim_kernel<<<grid_for(total), kThreads, 0, s>>>(g, total, dim, in, v, beta, out);
  SCTM_CUDA(cudaGetLastError());
}

// vbar[j] += sum over the other indices of a[g] * b[g] with j the index of dim
// `dim` (strides .sa = a, .sb = b); grid.y splits the work, one atomic per block
__global__ void scale_dim_reduce_kernel(Group g, int dim, const double* __restrict__ a, const double* __restrict__ b,
                                        double* __restrict__ vbar) {
  long long inner = 1;
  for (int i = g.nd - 1; i > dim; --i) inner *= g.size[i];
  const long long sz = g.size[dim];
  const long long per_j = g.total() / sz;   // (outer x inner) entries per index j
  const long long j = blockIdx.x;
  double acc = 0.0;
  for (long long t = blockIdx.y * (long long)blockDim.x + threadIdx.x; t < per_j;
       t += (long long)gridDim.y * blockDim.x) {
    const long long o = t / inner, i = t % inner;
    const long long lin = (o * sz + j) * inner + i;
    acc = fma(a[group_offset(g, g.sa, lin)], b[group_offset(g, g.sb, lin)], acc);
  }
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    atomicAdd(&vbar[j], t);
  }
}

void launch_scale_dim_reduce(const Group& g, int dim, const double* a, const double* b, double* vbar,
                             cudaStream_t s) {
  const long long total = g.total();
  if (total == 0) return;
  ProfScope ps_(PF_MISC, s, 2.0 * total, 16.0 * total, 1, "scale_dim_reduce");
  const long long sz = g.size[dim];
  const long long per_j = total / sz;
  const unsigned ys = (unsigned)std::max<long long>(1, std::min<long long>((per_j + kThreads - 1) / kThreads,
                                                                           (kNumSMs * 8 + sz - 1) / sz));
  scale_dim_reduce_kernel<<<dim3((unsigned)sz, ys), kThreads, 0, s>>>(g, dim, a, b, vbar);
  SCTM_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- column CG
// Conjugate-gradient steps for r independent shifted systems (s_j^2 - B) y_j =
// b_j stored as the columns of rows x r row-major blocks (one scalar per column).
// A column is frozen (its step set to zero from then on) as soon as the
// Rayleigh quotient pq / pp of its search direction drops below 0.1 s_j^2:
// the operator is then not safely positive definite along it and further
// steps would amplify rounding instead of converging.

// out[j] = sum_a X[a, j] Y[a, j] (FP64), X, Y rows x r row-major
__global__ void coldot_kernel(long long rows, int r, const double* __restrict__ X, const double* __restrict__ Y,
                              double* __restrict__ out) {
  __shared__ double part[8][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j = blockIdx.x * 32 + tx;
  double acc = 0.0;
  if (j < r)
    for (long long a = ty; a < rows; a += 8) acc = fma(X[a * r + j], Y[a * r + j], acc);
  part[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && j < r) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += part[i][tx];
    out[j] = t;
  }
}

void launch_coldot(long long rows, int r, const double* X, const double* Y, double* out, cudaStream_t s) {
  if (r == 0) return;
  ProfScope ps_(PF_MISC, s, 2.0 * rows * r, 16.0 * rows * r, 1, "coldot");
  coldot_kernel<<<(r + 31) / 32, dim3(32, 8), 0, s>>>(rows, r, X, Y, out);
  SCTM_CUDA(cudaGetLastError());
}

__global__ void cg_update_kernel(long long rows, int r, const double* __restrict__ P, const double* __restrict__ Q,
                                 double* __restrict__ Y, double* __restrict__ R, const double* __restrict__ rr,
                                 const double* __restrict__ pq, const double* __restrict__ pp,
                                 const double* __restrict__ s2, int* __restrict__ frozen) {
  const long long total = rows * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % r);
    const bool ok = !frozen[j] && rr[j] > 0.0 && pq[j] > 0.1 * s2[j] * pp[j];
    if (!ok) {
      if (e < r) frozen[j] = 1;   // one writer per column (the row-0 thread)
      continue;
    }
    const double a = rr[j] / pq[j];
    Y[e] = fma(a, P[e], Y[e]);
    R[e] = fma(-a, Q[e], R[e]);
  }
}

__global__ void cg_direction_kernel(long long rows, int r, double* __restrict__ P, const double* __restrict__ R,
                                    const double* __restrict__ rr_new, const double* __restrict__ rr,
                                    const int* __restrict__ frozen) {
  const long long total = rows * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % r);
    if (frozen[j]) continue;
    const double b = rr[j] > 0.0 ? rr_new[j] / rr[j] : 0.0;
    P[e] = fma(b, P[e], R[e]);
  }
}

void launch_cg_update(long long rows, int r, const double* P, const double* Q, double* Y, double* R,
                      const double* rr, const double* pq, const double* pp, const double* s2, int* frozen,
                      cudaStream_t s) {
  if (rows * r == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "cg_update");
  cg_update_kernel<<<grid_for(rows * r), kThreads, 0, s>>>(rows, r, P, Q, Y, R, rr, pq, pp, s2, frozen);
  SCTM_CUDA(cudaGetLastError());
}

void launch_cg_direction(long long rows, int r, double* P, const double* R, const double* rr_new, const double* rr,
                         const int* frozen, cudaStream_t s) {
  if (rows * r == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 0.0, 1, "cg_direction");
  cg_direction_kernel<<<grid_for(rows * r), kThreads, 0, s>>>(rows, r, P, R, rr_new, rr, frozen);
  SCTM_CUDA(cudaGetLastError());
}

// out[0] = max |a - b|, out[1] = max |a| over n entries (out zeroed by the
// caller).  The bit patterns of non-negative doubles order like the values, so
// an integer atomicMax on them is a max of the doubles.
__global__ void maxabs_pair_kernel(long long n, const double* __restrict__ a, const double* __restrict__ b,
                                   unsigned long long* out) {
  double md = 0.0, ma = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    md = fmax(md, fabs(a[e] - b[e]));
    ma = fmax(ma, fabs(a[e]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
    ma = fmax(ma, __shfl_xor_sync(0xffffffffu, ma, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(md));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(ma));
  }
}

void launch_maxabs_pair(long long n, const double* a, const double* b, double* out, cudaStream_t s) {
  SCTM_CUDA(cudaMemsetAsync(out, 0, 2 * sizeof(double), s));
  if (n == 0) return;
  ProfScope ps_(PF_MISC, s, 0.0, 16.0 * n, 1, "maxabs_pair");
  maxabs_pair_kernel<<<grid_for(n), kThreads, 0, s>>>(n, a, b, reinterpret_cast<unsigned long long*>(out));
  SCTM_CUDA(cudaGetLastError());
}

}  // namespace sctm
