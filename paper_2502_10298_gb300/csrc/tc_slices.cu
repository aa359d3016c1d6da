// Tensor-core contraction with BF16 digit slices (precision 4; sm_103a,
// tcgen05 + TMA).
//
// C[b,m,n] = alpha * sum_k A[b,m,k] B[b,k,n] + beta * C[b,m,n] with FP64
// operands in any strided layout (the ContractDesc of the CUDA-core kernel).
//
// The splitting follows the error-free transformation of matrix products of
// Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59, 2012): every row of A
// (column of B) is scaled by a power of two 2^e, e the smallest with
// max |row| < 2^e, so that x = v / 2^e lies in (-1, 1); x is written as
//     x = 2^-7 (d1 + 2^-8 d2 + 2^-16 d3 + 2^-24 d4) + O(2^-32),
// with integer digits |d_i| <= 128 obtained by repeated rounding to nearest.
// The four slices S_i = d_i 2^(-8(i-1)) are exact BF16 numbers.  A product of
// two slices of levels a, b is an integer multiple of 2^(-8(a+b-2)) of
// magnitude <= 2^14 2^(-8(a+b-2)), and the tensor core's FP32 accumulator
// adds such terms without rounding as long as the exact sum fits 24 bits:
//   level 0 (S1 S1):           512 terms of K, <= 2^23           exact
//   level 1 (S1 S2 + S2 S1):   2 x 512 terms, <= 2^16 in 2^-8    exact
//   levels 2-3 (seven pairs):  accumulated in FP32 with rounding; their
//                              weight 2^-16 leaves < 1e-10 of the result
// The dropped pairs (levels 4..6) and the digit remainder are O(2^-32) of
// 2^(eA+eB) per product term.  Every 512 of K the three accumulators are read
// out of tensor memory and added into double-float (two FP32) register sums
// with an error-free two-sum, so no precision is lost across windows either.
//
// Three kernels: (1) the exponent of every operand row (max over K, by
// atomicMax of the binary exponent); (2) pack: gather through the strides,
// scale, split into the four slices, write a K-major BF16 panel
// [slice][batch][rows][Kp]; (3) gemm: one 128 x 128 output tile per CTA, a
// 3-stage ring of 32-wide K slabs (4 A + 4 B slices, 64 KB) filled by TMA with
// 64-byte swizzle, ten tcgen05.mma kind::f16 per 16 of K, eight drain warps.
//
// Every mbarrier wait is bounded; on timeout the kernel records -2 in the
// status word, waits (bounded) for what it issued, frees tensor memory and
// returns.  The main-loop limit is a launch argument so that a test can make
// the waits run out; the drain waits always keep the full limit.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>

#include "common.h"
#include "kernels.h"
#include "prof.h"
#include "tcgen05_util.cuh"

namespace sctm {

using namespace tcx;

namespace {

constexpr int SL_NS = 4;                        // digit slices per operand
constexpr int SL_BM = 128, SL_BN = 128;         // output tile
constexpr int SL_BK = 32;                       // K slab: 32 BF16 = 64 bytes = one 64-byte swizzle row
constexpr int SL_STAGES = 3;
constexpr int SL_SLICE = SL_BM * SL_BK * 2;     // bytes of one slice of one slab (8 KB; BM == BN)
constexpr int SL_STAGE = 2 * SL_NS * SL_SLICE;  // 64 KB
constexpr int SL_SMEM = SL_STAGES * SL_STAGE + 1024;
constexpr int SL_WINDOW = 16;                   // slabs (512 of K) per exact accumulation window
constexpr int SL_DRAIN_WARPS = 8;
constexpr int SL_THREADS = 64 + 32 * SL_DRAIN_WARPS;
constexpr int SL_TMEM_COLS = 512;               // 3 x 128 accumulator columns, allocated as a power of two
constexpr int kNoExp = (int)0x80808080;         // exponent of an all-zero row (memset pattern)
static_assert(SL_BM == SL_BN, "slices of A and B share one size");
static_assert(SL_NS == 4, "the pack kernel writes four slices");
static_assert(2 * SL_WINDOW * SL_BK * 64 <= (1 << 16), "level-1 window sums must stay exact in FP32");

// shared-memory matrix descriptor: K-major, 64-byte swizzle, rows of 64
// bytes, 8-row atoms 512 bytes apart
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)1 << 16;                    // leading-dimension offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;           // stride-dimension offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                    // descriptor version of tcgen05
  d |= (uint64_t)4 << 61;                    // 64-byte swizzle
  return d;
}

// instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = 128
constexpr uint32_t kIdescBF16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(SL_BN >> 3) << 17) |
                                ((uint32_t)(SL_BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdescBF16), "r"(accumulate)
      : "memory");
}

// 2^n for -1022 <= n <= 1023, built from the exponent bits (exact)
__device__ __forceinline__ double pow2_normal(int n) {
  n = n < -1022 ? -1022 : (n > 1023 ? 1023 : n);
  return __longlong_as_double((long long)(n + 1023) << 52);
}
// v 2^n for |n| <= 2044 in two exact steps (no library call in the hot loops)
__device__ __forceinline__ double times_pow2(double v, int n) {
  const int n1 = n / 2;
  return v * pow2_normal(n1) * pow2_normal(n - n1);
}
// the same, by an integer add to the exponent field when v and the result
// are normal numbers (no FP64 instruction); otherwise times_pow2
__device__ __forceinline__ double scale_pow2(double v, int n) {
  const long long bits = __double_as_longlong(v);
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF || E + n <= 0 || E + n >= 0x7FF) return times_pow2(v, n);
  return __longlong_as_double(bits + ((long long)n << 52));
}

// One operand seen as rows x k through its strides (batch b on grid y).
struct SlicePack {
  Group bat, rows, k;          // strides of the operand in .sa
  long long nb, R, K, Rp, Kp;
  int k_inner;                 // 1 when the operand is contiguous along k
};

// Binary exponent e with |v| < 2^e (the exponent field minus 1022; subnormals
// take -1022), or kNoExp for v = 0: integer work on the bits only, since every
// FP64 instruction is expensive on this GPU.
__device__ __forceinline__ int exponent_bound(double v) {
  const long long bits = __double_as_longlong(v);
  if ((bits & 0x7FFFFFFFFFFFFFFFLL) == 0) return kNoExp;
  const int E = (int)((bits >> 52) & 0x7FF);
  return E == 0 ? -1022 : E - 1022;
}

// Pack kernels: 256 threads per CTA, a tile of 32 rows x TK values of k
// gathered through the operand's strides into shared memory (both the strided
// read and the shared-memory write coalesced), then read back by row in chunks
// of 8 consecutive k, so that every slice is written with 16-byte stores.
constexpr int SP_ROWS = 32;
constexpr int SP_THREADS = 256;

template <int TK>
__device__ __forceinline__ void gather_tile(const SlicePack& p, const double* __restrict__ X, long long r0,
                                            long long k0, long long b, double (*tile)[TK + 1], long long* offR,
                                            long long* offK) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < SP_ROWS) {
    const long long r = r0 + tid;
    offR[tid] = r < p.R ? group_offset(p.rows, p.rows.sa, r) : -1;
  } else if (tid < SP_ROWS + TK) {
    const long long k = k0 + tid - SP_ROWS;
    offK[tid - SP_ROWS] = k < p.K ? group_offset(p.k, p.k.sa, k) : -1;
  }
  const long long ob = group_offset(p.bat, p.bat.sa, b);
  __syncthreads();
  if (p.k_inner) {   // a warp reads along k within one row
#pragma unroll
    for (int i = warp; i < SP_ROWS; i += SP_THREADS / 32) {
      const long long orr = offR[i];
#pragma unroll
      for (int j = lane; j < TK; j += 32) {
        const long long ok = offK[j];
        tile[i][j] = (orr >= 0 && ok >= 0) ? X[ob + orr + ok] : 0.0;
      }
    }
  } else {           // a warp reads along the rows for one k
    const long long orr = offR[lane];
#pragma unroll 4
    for (int j = warp; j < TK; j += SP_THREADS / 32) {
      const long long ok = offK[j];
      tile[lane][j] = (orr >= 0 && ok >= 0) ? X[ob + orr + ok] : 0.0;
    }
  }
  __syncthreads();
}

// Largest exponent_bound over 8 consecutive values of one tile row.
template <int TK>
__device__ __forceinline__ int chunk_exponent(const double (*tile)[TK + 1], int row, int kc) {
  int e = kNoExp;
#pragma unroll
  for (int j = 0; j < 8; ++j) e = max(e, exponent_bound(tile[row][kc + j]));
  return e;
}

// Four balanced base-256 digits of v / 2^e (see slice_pack_kernel), each as
// the raw bits of its BF16 slice value d_i 2^(-8(i-1)).
__device__ __forceinline__ void slice_digits(double v, int e, uint16_t* d) {
  const long long bits = __double_as_longlong(v);
  long long Xv = 0;
  if (e != kNoExp && (bits & 0x7FFFFFFFFFFFFFFFLL) != 0) {
    const int E = (int)((bits >> 52) & 0x7FF);
    const long long mant = (bits & ((1LL << 52) - 1)) | (E != 0 ? (1LL << 52) : 0);
    const int lsb = (E == 0 ? 1 : E) - 1075;        // v = mant 2^lsb
    const int sh = e - 38 - lsb;                     // X = round(mant / 2^sh), sh >= 14
    const long long mag = sh >= 64 ? 0 : (((mant >> (sh - 1)) + 1) >> 1);
    Xv = bits < 0 ? -mag : mag;
  }
  const long long d1 = (Xv + (1LL << 30)) >> 31;
  long long r = Xv - (d1 << 31);
  const long long d2 = (r + (1LL << 22)) >> 23;
  r -= d2 << 23;
  const long long d3 = (r + (1LL << 14)) >> 15;
  r -= d3 << 15;
  const long long d4 = (r + (1LL << 6)) >> 7;
  d[0] = __bfloat16_as_ushort(__float2bfloat16_rn((float)d1));
  d[1] = __bfloat16_as_ushort(__float2bfloat16_rn((float)d2 * 0x1p-8f));
  d[2] = __bfloat16_as_ushort(__float2bfloat16_rn((float)d3 * 0x1p-16f));
  d[3] = __bfloat16_as_ushort(__float2bfloat16_rn((float)d4 * 0x1p-24f));
}

// The four slices of 8 consecutive values of one row, stored as one 16-byte
// word per slice at panel[slice][b][r][k .. k+7].
template <int TK>
__device__ __forceinline__ void pack_chunk(const SlicePack& p, const double (*tile)[TK + 1], int row, int kc, int e,
                                           long long o, uint16_t* __restrict__ out) {
  const long long plane = p.nb * p.Rp * p.Kp;
  uint32_t w[4][4];
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    uint16_t a[4], c[4];
    slice_digits(tile[row][kc + j], e, a);
    slice_digits(tile[row][kc + j + 1], e, c);
#pragma unroll
    for (int s = 0; s < SL_NS; ++s) w[s][j / 2] = (uint32_t)a[s] | ((uint32_t)c[s] << 16);
  }
#pragma unroll
  for (int s = 0; s < SL_NS; ++s)
    *reinterpret_cast<uint4*>(out + s * plane + o) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// expo[b][r] = max over k of exponent_bound(X[b, r, k]): the smallest e with
// |X[b, r, k]| < 2^e for every k; kNoExp (the initial value) for a zero row.
// Tiles of 32 rows x 64 k; a row's 8 chunks sit on 8 neighbouring lanes.
__global__ void __launch_bounds__(SP_THREADS) slice_exponent_kernel(SlicePack p, const double* __restrict__ X,
                                                                   int* __restrict__ expo) {
  constexpr int TK = 64;
  __shared__ long long offR[SP_ROWS], offK[TK];
  __shared__ double tile[SP_ROWS][TK + 1];
  const long long nkt = (p.Kp + TK - 1) / TK, t = blockIdx.x;
  const long long k0 = (t % nkt) * TK, r0 = (t / nkt) * SP_ROWS, b = blockIdx.y;
  gather_tile<TK>(p, X, r0, k0, b, tile, offR, offK);
  const int row = threadIdx.x >> 3, kc = (threadIdx.x & 7) * 8;
  int e = chunk_exponent<TK>(tile, row, kc);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 7) == 0 && e != kNoExp && r0 + row < p.R) atomicMax(&expo[b * p.Rp + r0 + row], e);
}

// Four BF16 slices per value: panel[slice][b][r][k] (as raw 16-bit words).
// With x = v / 2^e, X = round(x 2^38) is formed by shifting the mantissa (the
// shift is at least 14 because |v| < 2^e), and the balanced base-256 digits
// d1 = round(X / 2^31), d2 = round(r1 / 2^23), d3, d4 (each |d| <= 128) come
// from arithmetic shifts of the remainders: x = 2^-7 (d1 + 2^-8 d2 + 2^-16 d3
// + 2^-24 d4) + r with |r| <= 2^-32.  Integer arithmetic only.
__global__ void __launch_bounds__(SP_THREADS) slice_pack_kernel(SlicePack p, const double* __restrict__ X,
                                                               const int* __restrict__ expo,
                                                               uint16_t* __restrict__ out) {
  constexpr int TK = 64;
  __shared__ long long offR[SP_ROWS], offK[TK];
  __shared__ double tile[SP_ROWS][TK + 1];
  const long long nkt = (p.Kp + TK - 1) / TK, t = blockIdx.x;
  const long long k0 = (t % nkt) * TK, r0 = (t / nkt) * SP_ROWS, b = blockIdx.y;
  gather_tile<TK>(p, X, r0, k0, b, tile, offR, offK);
  const int row = threadIdx.x >> 3, kc = (threadIdx.x & 7) * 8;
  if (k0 + kc >= p.Kp) return;                      // past the padded row (Kp is a multiple of 32)
  const int e = expo[b * p.Rp + r0 + row];
  pack_chunk<TK>(p, tile, row, kc, e, (b * p.Rp + r0 + row) * p.Kp + k0 + kc, out);
}

// Operands with Kp <= 128: one tile holds whole rows, so the exponents and the
// slices come from one read of the operand.  A row's 16 chunks sit on the 16
// lanes of a half warp; each thread takes rows r and r + 16.
__global__ void __launch_bounds__(SP_THREADS) slice_pack_rows_kernel(SlicePack p, const double* __restrict__ X,
                                                                    int* __restrict__ expo,
                                                                    uint16_t* __restrict__ out) {
  constexpr int TK = 128;
  __shared__ long long offR[SP_ROWS], offK[TK];
  __shared__ double tile[SP_ROWS][TK + 1];
  const long long r0 = (long long)blockIdx.x * SP_ROWS, b = blockIdx.y;
  gather_tile<TK>(p, X, r0, 0, b, tile, offR, offK);
  const int kc = (threadIdx.x & 15) * 8;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int row = (threadIdx.x >> 4) + 16 * half;
    int e = kc < p.Kp ? chunk_exponent<TK>(tile, row, kc) : kNoExp;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 15) == 0) expo[b * p.Rp + r0 + row] = e;
    if (kc < p.Kp) pack_chunk<TK>(p, tile, row, kc, e, (b * p.Rp + r0 + row) * p.Kp + kc, out);
  }
}

struct SlEpi {
  Group bat, m, n;             // output strides in .sc
  long long M, N, Mp, Np;
  double alpha, beta;
  int num_m, num_n;            // tiles
};

__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

// Warp roles: warp 0 lane 0 issues TMA, warp 1 owns tensor memory and its
// lane 0 issues the MMAs, warps 2..9 drain the accumulators.  Tensor memory
// columns [0,128) level 0, [128,256) level 1, [256,384) levels 2 and 3.
__global__ void __launch_bounds__(SL_THREADS, 1)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, SlEpi e,
                      const int* __restrict__ expA, const int* __restrict__ expB, int nk_total, int slabs_per_split,
                      double* __restrict__ C, double* __restrict__ W, int* status, unsigned long long wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[SL_STAGES], empty[SL_STAGES], acc_full, acc_empty, done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int issued_parity[SL_STAGES];
  __shared__ long long offCm[SL_BM], offCn[SL_BN];
  __shared__ int eRow[SL_BM], eCol[SL_BN];

  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.y;
  // grouped raster: 8 row tiles share their B panels in L2
  const int t = blockIdx.x, GM = 8;
  const int group = t / (GM * e.num_n), first_m = group * GM;
  const int gsz = min(e.num_m - first_m, GM);
  const int m_tile = first_m + (t % (GM * e.num_n)) % gsz;
  const int n_tile = (t % (GM * e.num_n)) / gsz;
  const long long m0 = (long long)m_tile * SL_BM, n0 = (long long)n_tile * SL_BN;
  const int s0 = blockIdx.z * slabs_per_split;
  const int nk = min(nk_total - s0, slabs_per_split);

  if (tid == 0) {
    for (int s = 0; s < SL_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      issued_parity[s] = -1;
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, SL_DRAIN_WARPS);
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(SL_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const long long boC = group_offset(e.bat, e.bat.sc, b);
  for (int i = tid; i < SL_BM; i += blockDim.x) {
    long long m = m0 + i;
    offCm[i] = m < e.M ? boC + group_offset(e.m, e.m.sc, m) : -1;
    eRow[i] = expA[(long long)b * e.Mp + m0 + i];
  }
  for (int i = tid; i < SL_BN; i += blockDim.x) {
    long long n = n0 + i;
    offCn[i] = n < e.N ? group_offset(e.n, e.n.sc, n) : -1;
    eCol[i] = expB[(long long)b * e.Np + n0 + i];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* ab = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      // producer: TMA slabs (four A slices, four B slices) into the ring
      for (int s = 0; s < nk && !*ab; ++s) {
        const int st = s % SL_STAGES;
        if (s >= SL_STAGES && !mbar_wait(&empty[st], ((s / SL_STAGES) - 1) & 1, ab, wait_ns)) break;
        uint8_t* sp = base + st * SL_STAGE;
        mbar_expect_tx(&full[st], SL_STAGE);
        issued_parity[st] = (s / SL_STAGES) & 1;
        const int kc = (s0 + s) * SL_BK;
#pragma unroll
        for (int i = 0; i < SL_NS; ++i) {
          tma_load_4d(sp + i * SL_SLICE, &mapA, &full[st], kc, (int)m0, b, i);
          tma_load_4d(sp + (SL_NS + i) * SL_SLICE, &mapB, &full[st], kc, (int)n0, b, i);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: window w = s / SL_WINDOW accumulates afresh
      for (int s = 0; s < nk; ++s) {
        const int st = s % SL_STAGES, w = s / SL_WINDOW;
        const bool first = (s % SL_WINDOW) == 0;
        const bool last = (s % SL_WINDOW) == SL_WINDOW - 1 || s == nk - 1;
        if (!mbar_wait(&full[st], (s / SL_STAGES) & 1, ab, wait_ns)) break;
        if (first && w >= 1 && !mbar_wait(&acc_empty, (w - 1) & 1, ab, wait_ns)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d0 = tmem, d1 = tmem + 128, d2 = tmem + 256;
        const uint32_t sa = smem_addr(base + st * SL_STAGE);
        uint64_t a[SL_NS], bb[SL_NS];
#pragma unroll
        for (int i = 0; i < SL_NS; ++i) {
          a[i] = desc_sw64(sa + i * SL_SLICE);
          bb[i] = desc_sw64(sa + (SL_NS + i) * SL_SLICE);
        }
#pragma unroll
        for (int kk = 0; kk < SL_BK / 16; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 16 * 2) >> 4;   // 16 BF16 values = 32 bytes along K
          const uint32_t acc0 = (first && kk == 0) ? 0u : 1u;
          mma_bf16(d0, a[0] + adv, bb[0] + adv, acc0);                    // level 0
          mma_bf16(d1, a[0] + adv, bb[1] + adv, acc0);                    // level 1
          mma_bf16(d1, a[1] + adv, bb[0] + adv, 1u);
          mma_bf16(d2, a[0] + adv, bb[2] + adv, acc0);                    // level 2
          mma_bf16(d2, a[1] + adv, bb[1] + adv, 1u);
          mma_bf16(d2, a[2] + adv, bb[0] + adv, 1u);
          mma_bf16(d2, a[0] + adv, bb[3] + adv, 1u);                      // level 3
          mma_bf16(d2, a[1] + adv, bb[2] + adv, 1u);
          mma_bf16(d2, a[2] + adv, bb[1] + adv, 1u);
          mma_bf16(d2, a[3] + adv, bb[0] + adv, 1u);
        }
        mma_commit(&empty[st]);              // the slab's shared memory is free once these complete
        if (last) mma_commit(&acc_full);     // the window's sums are ready
      }
      mma_commit(&done_bar);                 // tracks every MMA issued; waited before TMEM is freed
      mbar_wait_bounded(&done_bar, 0);
    }
    __syncwarp();
  } else {
    // drain warps: rows 32 (warp % 4) + lane, columns 64 g .. 64 g + 63
    const int q = warp & 3, g = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    // running double-float sums: hi in registers, lo in tensor-memory columns
    // 384..511, which no MMA writes (64 more registers per thread would spill)
    float hi[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) hi[j] = 0.f;
    bool ok = true;
    const int nwin = (nk + SL_WINDOW - 1) / SL_WINDOW;
    const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * 64);
    for (int w = 0; w < nwin; ++w) {
      if (!mbar_wait(&acc_full, w & 1, ab, wait_ns)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        uint32_t v0[8], v1[8], v2[8], vl[8];
        SCTM_TMEM_LD8(tb + h * 8, v0);
        SCTM_TMEM_LD8(tb + 128 + h * 8, v1);
        SCTM_TMEM_LD8(tb + 256 + h * 8, v2);
        if (w > 0) SCTM_TMEM_LD8(tb + 384 + h * 8, vl);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float lo = w > 0 ? __uint_as_float(vl[j]) : 0.f;
          two_sum_into(hi[h * 8 + j], lo, __uint_as_float(v0[j]));
          two_sum_into(hi[h * 8 + j], lo, __uint_as_float(v1[j]));
          lo += __uint_as_float(v2[j]);
          vl[j] = __float_as_uint(lo);
        }
        SCTM_TMEM_ST8(tb + 384 + h * 8, vl);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty);
    }
    // stage the scaled tile in the (now idle) ring: every MMA has completed and
    // every TMA copy has landed before the last window's sums were ready
    double* tile = reinterpret_cast<double*>(base);   // [SL_BM][SL_BN + 1]
    if (ok && !*ab) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int er = eRow[row];
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        uint32_t vl[8];
        SCTM_TMEM_LD8(tb + 384 + h * 8, vl);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = g * 64 + h * 8 + j, ec = eCol[c];
          const double v = (double)hi[h * 8 + j] + (double)__uint_as_float(vl[j]);
          tile[row * (SL_BN + 1) + c] = (er == kNoExp || ec == kNoExp) ? 0.0 : scale_pow2(v, er + ec - 14);
        }
      }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * SL_DRAIN_WARPS) : "memory");
    if (!*ab) {
      const int dt = tid - 64;
      for (int idx = dt; idx < SL_BM * SL_BN; idx += 32 * SL_DRAIN_WARPS) {
        const int r = idx / SL_BN, cn = idx % SL_BN;
        const long long oc = offCm[r], on = offCn[cn];
        if (oc < 0 || on < 0) continue;
        if (W) {
          // partial sum of this K range; splitk_finish_kernel applies alpha, beta
          atomicAdd(&W[((long long)b * e.Mp + m0 + r) * e.Np + n0 + cn], tile[r * (SL_BN + 1) + cn]);
          continue;
        }
        double v = tile[r * (SL_BN + 1) + cn];
        if (e.alpha != 1.0) v *= e.alpha;
        if (e.beta != 0.0) v += e.beta * C[oc + on];
        C[oc + on] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*ab) {
    // drain: wait (bounded, full limit) for the TMA copies and MMAs this CTA issued
    if (tid == 0) {
      atomicExch(status, -2);
      for (int st = 0; st < SL_STAGES; ++st)
        if (issued_parity[st] >= 0) mbar_wait_bounded(&full[st], (uint32_t)issued_parity[st]);
      mbar_wait_bounded(&done_bar, 0);
    }
    __syncthreads();
  }
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SL_TMEM_COLS) : "memory");
  }
}

// tensor map over a slice panel [SL_NS][nb][rows][Kp] BF16, box 32 x 128
CUtensorMap slice_map(uint16_t* base, long long nb, long long rows, long long Kp) {
  CUtensorMap m;
  cuuint64_t dims[4] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)nb, (cuuint64_t)SL_NS};
  cuuint64_t strides[3] = {(cuuint64_t)Kp * 2, (cuuint64_t)(rows * Kp * 2), (cuuint64_t)(nb * rows * Kp * 2)};
  cuuint32_t box[4] = {SL_BK, (cuuint32_t)SL_BM, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  SCTM_CHECK(r == CUDA_SUCCESS, "cuTensorMapEncodeTiled failed (slice panel)");
  return m;
}

}  // namespace

// K splits: only when the output has too few tiles to fill the GPU; at least
// one window (512 of K) per split
int slice_split_rule(const ContractDesc& d) {
  const long long tiles = (round_up(d.M, SL_BM) / SL_BM) * (round_up(d.N, SL_BN) / SL_BN) * d.B;
  const long long nk = round_up(d.K, SL_BK) / SL_BK;
  const long long want = (2 * kNumSMs + tiles - 1) / tiles;
  long long sp = std::min<long long>(want, nk / SL_WINDOW);
  if (sp < 2) return 1;
  const long long per = (nk + sp - 1) / sp;
  return (int)((nk + per - 1) / per);
}

// largest split count worth trying: outputs with too few tiles to fill the
// GPU, at least 4 slabs (128 of K) per split
int slice_split_max(const ContractDesc& d) {
  const long long tiles = (round_up(d.M, SL_BM) / SL_BM) * (round_up(d.N, SL_BN) / SL_BN) * d.B;
  if (tiles >= 2 * kNumSMs) return 1;
  return (int)std::max<long long>(1, std::min<long long>(65535, round_up(d.K, SL_BK) / SL_BK / 4));
}

namespace {

struct SliceLayout {
  long long Kp, Mp, Np;
  size_t panelA, panelB, W, total;   // byte offsets; each packed operand holds its panel and exponents
};

size_t slice_panel_bytes_of(long long nb, long long Rp, long long Kp) {
  return (size_t)round_up((long long)SL_NS * nb * Rp * Kp * 2, 256) + (size_t)nb * Rp * 4 + 256;
}

SliceLayout slice_layout(const ContractDesc& d) {
  SliceLayout L;
  L.Kp = round_up(d.K, SL_BK), L.Mp = round_up(d.M, SL_BM), L.Np = round_up(d.N, SL_BN);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = (size_t)round_up((long long)(o + bytes), 256);
    return at;
  };
  L.panelA = take(slice_panel_bytes_of(d.B, L.Mp, L.Kp));
  L.panelB = take(slice_panel_bytes_of(d.B, L.Np, L.Kp));
  L.W = slice_split_max(d) > 1 ? take((size_t)d.B * L.Mp * L.Np * 8) : 0;
  L.total = o;
  return L;
}

}  // namespace

size_t slice_scratch_bytes(const ContractDesc& d) { return slice_layout(d).total + 256; }

namespace {
SlicePack operand_pack(const ContractDesc& d, bool b_operand) {
  const long long Kp = round_up(d.K, SL_BK);
  SlicePack p;
  if (!b_operand) {
    p.bat = d.bat, p.rows = d.m, p.k = d.k;
    p.nb = d.B, p.R = d.M, p.K = d.K, p.Rp = round_up(d.M, SL_BM), p.Kp = Kp, p.k_inner = d.a_k_inner;
  } else {
    p.bat = d.bat, p.rows = d.n, p.k = d.k;
    for (int i = 0; i < kMaxDims; ++i) {
      p.bat.sa[i] = d.bat.sb[i];
      p.rows.sa[i] = d.n.sb[i];
      p.k.sa[i] = d.k.sb[i];
    }
    p.nb = d.B, p.R = d.N, p.K = d.K, p.Rp = round_up(d.N, SL_BN), p.Kp = Kp, p.k_inner = d.b_n_inner ? 0 : 1;
  }
  return p;
}
}  // namespace

size_t slice_panel_bytes(const ContractDesc& d, bool b_operand) {
  const SlicePack p = operand_pack(d, b_operand);
  return slice_panel_bytes_of(p.nb, p.Rp, p.Kp);
}

SlicePanel slice_pack(const ContractDesc& d, bool b_operand, const double* X, void* dst, cudaStream_t s) {
  const SlicePack p = operand_pack(d, b_operand);
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dst) + 255) & ~uintptr_t(255));
  SlicePanel out;
  out.panel = reinterpret_cast<uint16_t*>(base);
  out.expo = reinterpret_cast<int*>(base + round_up((long long)SL_NS * p.nb * p.Rp * p.Kp * 2, 256));
  SCTM_CUDA(cudaMemsetAsync(out.expo, 0x80, (size_t)p.nb * p.Rp * 4, s));
  if (p.Kp <= 128) {
    // whole rows in one tile: exponents and slices from one read
    ProfScope ps(PF_MISC, s, 0.0, 8.0 * p.nb * p.R * p.K + 2.0 * SL_NS * p.nb * p.Kp * p.Rp, 1, "slice_pack_rows");
    slice_pack_rows_kernel<<<dim3((unsigned)(p.Rp / SP_ROWS), (unsigned)p.nb), SP_THREADS, 0, s>>>(p, X, out.expo,
                                                                                                   out.panel);
    SCTM_CUDA(cudaGetLastError());
    return out;
  }
  // exponents (one gather), then the slices (another); the panel is written once
  const dim3 g((unsigned)(((p.Kp + 63) / 64) * (p.Rp / SP_ROWS)), (unsigned)p.nb);
  {
    ProfScope ps(PF_MISC, s, 0.0, 8.0 * p.nb * p.R * p.K, 1, "slice_exponent");
    slice_exponent_kernel<<<g, SP_THREADS, 0, s>>>(p, X, out.expo);
    SCTM_CUDA(cudaGetLastError());
  }
  {
    ProfScope ps(PF_MISC, s, 0.0, 8.0 * p.nb * p.R * p.K + 2.0 * SL_NS * p.nb * p.Kp * p.Rp, 1, "slice_pack");
    slice_pack_kernel<<<g, SP_THREADS, 0, s>>>(p, X, out.expo, out.panel);
    SCTM_CUDA(cudaGetLastError());
  }
  return out;
}

void launch_contract_slices(const ContractDesc& d, const double* A, const double* B, double* C, cudaStream_t s,
                            void* scratch, int* status, unsigned long long wait_ns, const SlicePanel* preA,
                            const SlicePanel* preB, int splits_req) {
  if (d.M == 0 || d.N == 0 || d.B == 0) return;
  SCTM_CHECK(tc_shape_ok(d), "contraction shape not representable on the tensor cores");
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(scratch) + 255) & ~uintptr_t(255));
  const SliceLayout L = slice_layout(d);
  const SlicePanel pa = preA ? *preA : slice_pack(d, false, A, base + L.panelA, s);
  const SlicePanel pb = preB ? *preB : slice_pack(d, true, B, base + L.panelB, s);
  CUtensorMap mA = slice_map(pa.panel, d.B, L.Mp, L.Kp);
  CUtensorMap mB = slice_map(pb.panel, d.B, L.Np, L.Kp);
  SlEpi e;
  e.bat = d.bat, e.m = d.m, e.n = d.n;
  e.M = d.M, e.N = d.N, e.Mp = L.Mp, e.Np = L.Np, e.alpha = d.alpha, e.beta = d.beta;
  e.num_m = (int)(L.Mp / SL_BM), e.num_n = (int)(L.Np / SL_BN);
  static bool attr = false;
  if (!attr) {
    SCTM_CUDA(cudaFuncSetAttribute(slice_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SL_SMEM));
    attr = true;
  }
  const int nk = (int)(L.Kp / SL_BK);
  int splits = slice_split_rule(d);
  if (splits_req > 0) splits = std::min(splits_req, slice_split_max(d));
  const int per = (nk + splits - 1) / splits;
  splits = (nk + per - 1) / per;
  double* W = nullptr;
  if (splits > 1) {
    W = reinterpret_cast<double*>(base + L.W);
    SCTM_CUDA(cudaMemsetAsync(W, 0, (size_t)d.B * L.Mp * L.Np * sizeof(double), s));
  }
  dim3 grid((unsigned)((long long)e.num_m * e.num_n), (unsigned)d.B, (unsigned)splits);
  // algorithmic work 2 B M N K (the tensor pipe executes ten BF16 products per
  // multiply-add); bytes: the slice panels read once, the FP64 result written
  {
    ProfScope ps(PF_TENSOR, s, 2.0 * d.B * d.M * d.N * d.K,
                 2.0 * SL_NS * d.B * L.Kp * (L.Mp + L.Np) + 8.0 * d.B * d.M * d.N * (d.beta != 0 ? 2 : 1));
    slice_gemm_kernel<<<grid, SL_THREADS, SL_SMEM, s>>>(mA, mB, e, pa.expo, pb.expo, nk, per, C, W, status,
                                                         wait_ns);
    SCTM_CUDA(cudaGetLastError());
  }
  if (W) launch_splitk_finish(d, L.Mp, L.Np, W, C, s);
}

}  // namespace sctm
