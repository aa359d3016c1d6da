// Launch wrappers of the engine's CUDA kernels.
#pragma once
#include "common.h"

namespace sctm {

// fp32_compute: operands rounded to FP32 on load, FP32 accumulation (mixed mode)
// scratch: contract_scratch_doubles(d) doubles (may be null: no K split).  Outputs
// with few 64 x 64 tiles and a long K are then split over K into an FP64
// buffer and finished by launch_splitk_finish.
template <typename T>
// splits_req > 0 asks for that many K splits (clamped to contract_split_max);
// 0 takes the rule (contract_split_rule)
void launch_contract(const ContractDesc& d, const T* A, const T* B, T* C, cudaStream_t s, bool fp32_compute,
                     double* scratch = nullptr, int splits_req = 0);
size_t contract_scratch_doubles(const ContractDesc& d);
// G (r x r, row stride ldg) = Y^T Y of a row-major m x r block Y (row stride ldy), FP64;
// W: r * r doubles of scratch
void launch_gram(long long m, int r, const double* Y, long long ldy, double* G, long long ldg, double* W,
                 cudaStream_t s);
int contract_split_rule(const ContractDesc& d);
int contract_split_max(const ContractDesc& d);
// C = alpha W + beta C through the output strides of d; W[b][m][n] with Wm x Wn per batch
void launch_splitk_finish(const ContractDesc& d, long long Wm, long long Wn, const double* W, double* C,
                          cudaStream_t s);

// Tensor-core form of the same contraction (mixed mode): operands split into
// TF32 hi/lo pairs, 3xTF32 tcgen05 MMAs with FP32 accumulation, FP64 output.
// scratch: tc_scratch_floats(d) floats, 128-byte aligned; status: device word
// set to -2 if a pipeline wait timed out.
bool tc_eligible(const ContractDesc& d);
// the shape conditions of tc_eligible alone (tiles representable, M, N >= 64,
// K >= 128), without its minimum amount of work
bool tc_shape_ok(const ContractDesc& d);
size_t tc_scratch_floats(const ContractDesc& d);
// wait_ns: main-loop mbarrier wait limit (global time); the drain waits after a
// timeout keep the full default limit of two seconds
void launch_contract_tc(const ContractDesc& d, const double* A, const double* B, double* C, cudaStream_t s,
                        float* scratch, int* status, unsigned long long wait_ns = 2000000000ull, int splits_req = 0);
int tc_split_rule(const ContractDesc& d);
int tc_split_max(const ContractDesc& d);

// Tensor-core form with FP64-grade accuracy (precision 4): operands scaled per
// row / column by powers of two and split into four BF16 digit slices, ten
// tcgen05 kind::f16 products per 16 of K with exact FP32 accumulation of the
// two leading levels, FP64 output (tc_slices.cu).  Same eligibility as the
// 3xTF32 form.  scratch: slice_scratch_bytes(d) bytes; status as above.
size_t slice_scratch_bytes(const ContractDesc& d);
// One operand packed for the slice kernel: the four BF16 slice panels
// [slice][batch][rows padded to 128][K padded to 32] and the per-row exponents.
struct SlicePanel {
  uint16_t* panel = nullptr;
  int* expo = nullptr;
};
// bytes (256-aligned start included) of operand A (b_operand false) or B of d, packed
size_t slice_panel_bytes(const ContractDesc& d, bool b_operand);
SlicePanel slice_pack(const ContractDesc& d, bool b_operand, const double* X, void* dst, cudaStream_t s);
// preA / preB: operands packed beforehand (by slice_pack on a contraction with
// the same operand layout); null = pack them here into the scratch
void launch_contract_slices(const ContractDesc& d, const double* A, const double* B, double* C, cudaStream_t s,
                            void* scratch, int* status, unsigned long long wait_ns = 2000000000ull,
                            const SlicePanel* preA = nullptr, const SlicePanel* preB = nullptr, int splits_req = 0);
int slice_split_rule(const ContractDesc& d);
int slice_split_max(const ContractDesc& d);

// deterministic N(0,1) test matrix (counter-based hash + Box-Muller), rows x cols
void launch_gaussian(long long rows, long long cols, unsigned long long seed, double* X, cudaStream_t s);

// Batched SVD of m x n row-major matrices (m >= n): M = U diag(S) V^T with
// U m x n, V n x n, S descending.
// noise_rel > 0: a column pair in which either column has norm^2 below
// noise_rel ||M||_F^2 still rotates but never keeps the sweep loop going (for
// decompositions whose noise-level directions are discarded afterwards).
// tol_rel > 0 replaces the default orthogonality threshold |w_i.w_j| <= tol |w_i||w_j|
// (4 eps sqrt(m)) for decompositions that need less.
// max_sweeps bounds the Jacobi sweeps (a run that reaches it sets status word 0 to -1).
void launch_svd(int m, int n, int batch, const double* M, double* U, double* S, double* V,
                double* work, int* status, cudaStream_t s, double noise_rel = 0.0, double tol_rel = 0.0,
                int max_sweeps = 60);
size_t svd_work_doubles(int m, int n, int batch);

// out[g] = alpha * in[g] + beta * out[g] over one index group g (strides sa = in, sc = out).
template <typename T>
void launch_copy(const Group& g, T alpha, const T* in, T beta, T* out, cudaStream_t s);

// X[b, i, j] *= (row ? v[b, i] : v[b, j]); X row-major (rows x cols), batch stride rows*cols.
void launch_scale_rc(int batch, int rows, int cols, double* X, const double* v, int vstride, bool row,
                     cudaStream_t s);

// w[b, k] = f(S[b, k]) for k < kout, with cutoff relative to S[b, 0]:
// mode 0: S^{-1/2} (0 below cutoff);  mode 1: S^{1/2} (0 below cutoff);
// mode 2: 1 if kept else 0.
void launch_spectrum_map(int batch, int n, int kout, const double* S, double* w, double cutoff,
                         int mode, cudaStream_t s);

// sgn[r] = sign of the largest-|.| entry of row r of a (rows x cols) matrix with
// element (r, e) at P[r*rs + e*cs] (ties: first index).
void launch_sign_find(int rows, int cols, const double* P, long long rs, long long cs, double* sgn,
                      cudaStream_t s);

// Reverse pass of the square SVD M = U S V^T (Lorentzian-broadened):
// inner[i,j] = F_ij (J_ij - J_ji) s_j + d_ij Sbar_i + s_i F_ij (K_ij - K_ji),
// F_ij = d / (d^2 + eps * s_max^4), d = s_j^2 - s_i^2.
void launch_svd_adj_inner(int n, const double* S, const double* J, const double* K, const double* Sbar,
                          double* inner, double eps, cudaStream_t s);

// Sbar[k] += wbar[k] * f'(S[k]) for kept k (same modes and cutoff as launch_spectrum_map)
void launch_spectrum_adj(int n, int kout, const double* S, const double* wbar, double* Sbar, double cutoff,
                         int mode, cudaStream_t s);

// Reverse pass of y = x / m, m = |x[k]| = max |x|:  xbar += ybar/m - e_k sign(x_k) (ybar.y)/m
void launch_rescale_adj(long long n, const double* ybar, const double* y, const double* m,
                        const long long* k, const double* xk_sign, const double* dot, double* xbar,
                        cudaStream_t s);

// Divide each tensor of a batch by its max |entry|; records the scale (and the
// flat index of the maximum) for the reverse pass.
void launch_rescale(int batch, long long n, double* X, long long stride, double* scale,
                    long long* argmax, double* partial, cudaStream_t s);

// out[b] = sum_i x[b, i] * y[b, i]  (deterministic tree reduction)
void launch_dot(int batch, long long n, const double* x, const double* y, long long stride,
                double* out, double* partial, cudaStream_t s);

void launch_fill(long long n, double v, double* x, cudaStream_t s);

// y += a[0] * x with the scalar a on the device
void launch_axpy_dev(long long n, const double* a, const double* x, double* y, cudaStream_t s);
// out[g] = in[g] * v[j] + beta * out[g], j = index of dimension `dim` of g (.sa = in, .sc = out strides)
void launch_scale_dim(const Group& g, int dim, const double* in, const double* v, double beta, double* out,
                      cudaStream_t s);
// vbar[j] += sum over g with index j in dimension `dim` of a[g] b[g] (.sa = a, .sb = b strides)
void launch_scale_dim_reduce(const Group& g, int dim, const double* a, const double* b, double* vbar,
                             cudaStream_t s);

// Column-wise conjugate gradient on rows x r blocks (row-major), one shifted
// system (s_j^2 - B) y_j = b_j per column: update Y += a P, R -= a Q with
// a_j = rr_j / pq_j; a column freezes (a = 0 from then on, direction kept) once
// pq_j <= 0.1 s2_j pp_j or rr_j <= 0.  Direction P = R + (rr_new_j / rr_j) P.
void launch_cg_update(long long rows, int r, const double* P, const double* Q, double* Y, double* R,
                      const double* rr, const double* pq, const double* pp, const double* s2, int* frozen,
                      cudaStream_t s);
void launch_cg_direction(long long rows, int r, double* P, const double* R, const double* rr_new, const double* rr,
                         const int* frozen, cudaStream_t s);
// out[j] = sum_a X[a, j] Y[a, j] for rows x r row-major X, Y (FP64)
void launch_coldot(long long rows, int r, const double* X, const double* Y, double* out, cudaStream_t s);

// Batched Cholesky QR factor: G (batch of r x r Gram matrices, overwritten) ->
// T = R^+ with G = R^T R; pivots below tol_rel * max diag deflated (zero row of
// R, zero column of T).
void launch_chol_qr_factor(int r, int batch, double* G, double* T, double tol_rel, cudaStream_t s);
void launch_axpy(long long n, double a, const double* x, double* y, cudaStream_t s);
// out[0] = max |a - b|, out[1] = max |a| (device, two doubles)
void launch_maxabs_pair(long long n, const double* a, const double* b, double* out, cudaStream_t s);

}  // namespace sctm
