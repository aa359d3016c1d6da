// Tensor-core contraction for the mixed-precision mode (sm_103a, tcgen05 + TMA).
//
// C[b,m,n] = alpha * sum_k A[b,m,k] B[b,k,n] + beta * C[b,m,n] with FP64
// operands in any strided layout (the same ContractDesc as the CUDA-core
// kernel).  Two kernels:
//
//  1. pack: gathers one operand through its group strides (a 32x32 tile
//     staged in shared memory, so both the strided read and the write are
//     coalesced) and splits every value v into two TF32 numbers
//     hi = rna_tf32(v), lo = rna_tf32(v - hi), stored as FP32 words in a
//     K-major panel [part][batch][rows][Kp] (rows padded to the tile, K to 32).
//  2. gemm: one 128 x 128 output tile per CTA.  A producer thread streams
//     32-wide K slabs of A_hi, A_lo, B_hi, B_lo with TMA (128-byte swizzle) into
//     a 3-stage shared-memory ring; one thread issues tcgen05.mma kind::tf32
//     for A_hi B_hi + A_hi B_lo + A_lo B_hi (the 3xTF32 split: the dropped
//     A_lo B_lo term is 2^-22 relative) into FP32 accumulators in tensor
//     memory, two K slabs at a time; eight warps read every chunk's partial sums
//     with tcgen05.ld, add them into FP32 register sums, and finally write
//     alpha * sum (+ beta * C) in FP64 through the output strides.
//
// Every wait on an mbarrier is bounded (about two seconds of global time);
// on timeout the kernel records the failure in a status word, drains what it
// issued and returns, so the host sees an error instead of a hung context.
#include <cuda.h>

#include <algorithm>

#include "common.h"
#include "kernels.h"
#include "prof.h"
#include "tcgen05_util.cuh"

namespace sctm {

using namespace tcx;

namespace {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32;   // BK = 128 bytes of FP32 = one swizzle atom
constexpr int TC_STAGES = 3;
constexpr int TC_TILE_A = TC_BM * TC_BK * 4;          // bytes of one A slab (16 KB)
constexpr int TC_TILE_B = TC_BN * TC_BK * 4;          // bytes of one B slab (16 KB)
constexpr int TC_STAGE = 2 * TC_TILE_A + 2 * TC_TILE_B;
constexpr int TC_SMEM = TC_STAGES * TC_STAGE + 1024;  // + alignment slack (swizzle atoms need 1024 B)
// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row atoms 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)1 << 16;                    // leading-dimension offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride-dimension offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                    // descriptor version of tcgen05
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = TC_BN
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                            ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
// Panel of one operand: rows x k gathered from strided FP64, split into TF32 hi/lo.
struct PackDesc {
  Group bat, rows, k;          // strides of the operand in .sa
  long long nb, R, K, Rp, Kp;
  int k_inner;                 // 1 when the operand is contiguous along k
};

__global__ void __launch_bounds__(256) pack_tf32x2_kernel(PackDesc p, const double* __restrict__ X,
                                                          float* __restrict__ out) {
  __shared__ long long offR[32], offK[32];
  __shared__ double tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  // one flat grid dimension of 32 x 32 tiles (k fastest), the batch on y:
  // row counts beyond 65535 tiles do not fit the y dimension
  const long long nkt = p.Kp / 32, t = blockIdx.x;
  const long long k0 = (t % nkt) * 32, r0 = (t / nkt) * 32, b = blockIdx.y;
  if (tid < 32) {
    long long r = r0 + tid;
    offR[tid] = r < p.R ? group_offset(p.rows, p.rows.sa, r) : -1;
  } else if (tid < 64) {
    long long k = k0 + tid - 32;
    offK[tid - 32] = k < p.K ? group_offset(p.k, p.k.sa, k) : -1;
  }
  const long long ob = group_offset(p.bat, p.bat.sa, b);
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    // k_inner: lanes walk k (contiguous); otherwise lanes walk rows
    int rr = p.k_inner ? i : tx, kk = p.k_inner ? tx : i;
    long long orr = offR[rr], ok = offK[kk];
    tile[rr][kk] = (orr >= 0 && ok >= 0) ? X[ob + orr + ok] : 0.0;
  }
  __syncthreads();
  const long long plane = p.nb * p.Rp * p.Kp;
  for (int i = ty; i < 32; i += 8) {
    double v = tile[i][tx];
    uint32_t hi, lo;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"((float)v));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"((float)(v - (double)__uint_as_float(hi))));
    long long o = (b * p.Rp + r0 + i) * p.Kp + k0 + tx;
    out[o] = __uint_as_float(hi);
    out[plane + o] = __uint_as_float(lo);
  }
}

struct TcEpi {
  Group bat, m, n;             // output strides in .sc
  long long M, N;
  double alpha, beta;
  int num_m, num_n;            // tiles
};

// Warp roles: warp 0 lane 0 issues TMA, warp 1 owns tensor memory and its
// lane 0 issues the MMAs, warps 2..9 drain the accumulators.  Tensor memory
// (512 columns): two buffers x {main = A_hi B_hi, corr = A_hi B_lo + A_lo B_hi}
// x 128 columns.  Every chunk of TC_CHUNK K slabs is accumulated afresh in one
// buffer; the drain warps add it into FP32 register sums (round to nearest)
// while the next chunk fills the other buffer.  The tensor core adds into its
// FP32 accumulator with truncation toward zero, so short per-chunk accumulation
// (8 additions into `main`, the corrections being 2^-11 smaller) bounds that
// bias to a few 2^-24 of the chunk's partial sum instead of letting it grow with
// K; the round-to-nearest sums over chunks add an unbiased 2^-24 per chunk.
constexpr int TC_DRAIN_WARPS = 8;
constexpr int TC_CHUNK = 2;   // K slabs accumulated in tensor memory between drains
constexpr int TC_THREADS_V2 = 64 + 32 * TC_DRAIN_WARPS;
constexpr int TC_TMEM_COLS = 512;

__global__ void __launch_bounds__(TC_THREADS_V2, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcEpi e,
                   int nk_total, int slabs_per_split, double* __restrict__ C, double* __restrict__ W,
                   long long Wm, long long Wn, int* status, unsigned long long wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], acc_full[2], acc_empty[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int issued_parity[TC_STAGES];
  __shared__ long long offCm[TC_BM], offCn[TC_BN];

  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.y;
  // grouped raster: 8 row tiles share their B panels in L2
  const int t = blockIdx.x, GM = 8;
  const int group = t / (GM * e.num_n), first_m = group * GM;
  const int gsz = min(e.num_m - first_m, GM);
  const int m_tile = first_m + (t % (GM * e.num_n)) % gsz;
  const int n_tile = (t % (GM * e.num_n)) / gsz;
  const long long m0 = (long long)m_tile * TC_BM, n0 = (long long)n_tile * TC_BN;
  // split K: this CTA accumulates slabs [s0, s0 + nk) into the FP64 buffer W
  const int s0 = blockIdx.z * slabs_per_split;
  const int nk = min(nk_total - s0, slabs_per_split);

  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      issued_parity[s] = -1;
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], TC_DRAIN_WARPS);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const long long boC = group_offset(e.bat, e.bat.sc, b);
  for (int i = tid; i < TC_BM; i += blockDim.x) {
    long long m = m0 + i;
    offCm[i] = m < e.M ? boC + group_offset(e.m, e.m.sc, m) : -1;
  }
  for (int i = tid; i < TC_BN; i += blockDim.x) {
    long long n = n0 + i;
    offCn[i] = n < e.N ? group_offset(e.n, e.n.sc, n) : -1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* ab = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      // producer: TMA slabs into the ring
      for (int s = 0; s < nk && !*ab; ++s) {
        const int st = s % TC_STAGES;
        if (s >= TC_STAGES && !mbar_wait(&empty[st], ((s / TC_STAGES) - 1) & 1, ab, wait_ns)) break;
        uint8_t* sp = base + st * TC_STAGE;
        mbar_expect_tx(&full[st], TC_STAGE);
        issued_parity[st] = (s / TC_STAGES) & 1;
        const int kc = (s0 + s) * TC_BK;
        tma_load_4d(sp, &mapA, &full[st], kc, (int)m0, b, 0);
        tma_load_4d(sp + TC_TILE_A, &mapA, &full[st], kc, (int)m0, b, 1);
        tma_load_4d(sp + 2 * TC_TILE_A, &mapB, &full[st], kc, (int)n0, b, 0);
        tma_load_4d(sp + 2 * TC_TILE_A + TC_TILE_B, &mapB, &full[st], kc, (int)n0, b, 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: chunk ch = s / TC_CHUNK accumulates afresh in buffer ch & 1
      for (int s = 0; s < nk; ++s) {
        const int st = s % TC_STAGES, ch = s / TC_CHUNK, buf = ch & 1;
        const bool first = (s % TC_CHUNK) == 0;
        const bool last = (s % TC_CHUNK) == TC_CHUNK - 1 || s == nk - 1;
        if (!mbar_wait(&full[st], (s / TC_STAGES) & 1, ab, wait_ns)) break;
        if (first && ch >= 2 && !mbar_wait(&acc_empty[buf], ((ch >> 1) - 1) & 1, ab, wait_ns)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dmain = tmem + (uint32_t)(buf * 256), dcorr = dmain + 128;
        const uint32_t sa = smem_addr(base + st * TC_STAGE);
        const uint64_t ahi = smem_desc(sa), alo = smem_desc(sa + TC_TILE_A);
        const uint64_t bhi = smem_desc(sa + 2 * TC_TILE_A), blo = smem_desc(sa + 2 * TC_TILE_A + TC_TILE_B);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 8; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 8 * 4) >> 4;   // 8 TF32 values = 32 bytes along K
          const uint32_t acc0 = (first && kk == 0) ? 0u : 1u;
          mma_tf32(dmain, ahi + adv, bhi + adv, acc0);
          mma_tf32(dcorr, ahi + adv, blo + adv, acc0);
          mma_tf32(dcorr, alo + adv, bhi + adv, 1u);
        }
        mma_commit(&empty[st]);                  // slab's shared memory free once these MMAs complete
        if (last) mma_commit(&acc_full[buf]);    // chunk's partial sums ready
      }
      // tracks every MMA issued (normal end or abort); waited before tensor memory is freed
      mma_commit(&done_bar);
      const unsigned long long t0 = global_ns();
      while (!mbar_test(&done_bar, 0) && global_ns() - t0 < kWaitNs) {
      }
    }
    __syncwarp();
  } else {
    // drain warps: rows 32 (warp % 4) + lane, columns 64 g .. 64 g + 63
    const int q = warp & 3, g = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    float acc[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc[j] = 0.f;
    bool ok = true;
    const int nch = (nk + TC_CHUNK - 1) / TC_CHUNK;
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch & 1;
      if (!mbar_wait(&acc_full[buf], (ch >> 1) & 1, ab, wait_ns)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 256 + g * 64);
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        uint32_t vm[8], vc[8];
        SCTM_TMEM_LD8(tbase + h * 8, vm);
        SCTM_TMEM_LD8(tbase + 128 + h * 8, vc);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[h * 8 + j] += __uint_as_float(vm[j]) + __uint_as_float(vc[j]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    // stage the tile in the (now idle) ring buffer: every MMA has completed
    // and every TMA copy has landed before the last slab's sums were ready
    double* tile = reinterpret_cast<double*>(base);   // [TC_BM][TC_BN + 1]
    if (ok && !*ab) {
#pragma unroll
      for (int j = 0; j < 64; ++j) tile[row * (TC_BN + 1) + g * 64 + j] = (double)acc[j];
    }
    // named barrier over the drain warps only
    asm volatile("bar.sync 1, %0;" ::"n"(32 * TC_DRAIN_WARPS) : "memory");
    if (!*ab) {
      // coalesced write-out: consecutive threads take consecutive columns
      const int dt = tid - 64;
      for (int idx = dt; idx < TC_BM * TC_BN; idx += 32 * TC_DRAIN_WARPS) {
        const int r = idx / TC_BN, cn = idx % TC_BN;
        const long long oc = offCm[r], on = offCn[cn];
        if (oc < 0 || on < 0) continue;
        if (W) {
          // partial sum of this K range; splitk_finish_kernel applies alpha, beta
          atomicAdd(&W[((long long)b * Wm + m0 + r) * Wn + n0 + cn], tile[r * (TC_BN + 1) + cn]);
          continue;
        }
        double v = e.alpha * tile[r * (TC_BN + 1) + cn];
        if (e.beta != 0.0) v += e.beta * C[oc + on];
        C[oc + on] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*ab) {
    // drain: wait (bounded) for the TMA copies and MMAs this CTA issued
    if (tid == 0) {
      atomicExch(status, -2);
      for (int st = 0; st < TC_STAGES; ++st) {
        if (issued_parity[st] < 0) continue;
        const unsigned long long t0 = global_ns();
        while (!mbar_test(&full[st], (uint32_t)issued_parity[st]) && global_ns() - t0 < kWaitNs) {
        }
      }
      const unsigned long long t0 = global_ns();
      while (!mbar_test(&done_bar, 0) && global_ns() - t0 < kWaitNs) {
      }
    }
    __syncthreads();
  }
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// tensor map over a packed panel [2][nb][rows][Kp] FP32, box 32 x 128
CUtensorMap panel_map(float* base, long long nb, long long rows, long long Kp, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[4] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)nb, 2};
  cuuint64_t strides[3] = {(cuuint64_t)Kp * 4, (cuuint64_t)(rows * Kp * 4), (cuuint64_t)(nb * rows * Kp * 4)};
  cuuint32_t box[4] = {TC_BK, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  SCTM_CHECK(r == CUDA_SUCCESS, "cuTensorMapEncodeTiled failed");
  return m;
}

}  // namespace

bool tc_shape_ok(const ContractDesc& d) {
  // representable by the tensor maps and the grid; below 128 of K (four slabs)
  // the per-tile set-up and epilogue outweigh the MMAs
  const long long kt = round_up(d.K, TC_BK) / 32;   // 32 x 32 pack tiles along k
  return d.M >= 64 && d.N >= 64 && d.K >= 128 && d.B <= 65535 &&
         round_up(d.M, TC_BM) / TC_BM * (round_up(d.N, TC_BN) / TC_BN) < (1LL << 31) &&
         kt * (round_up(std::max(d.M, d.N), TC_BM) / 32) < (1LL << 31);
}

bool tc_eligible(const ContractDesc& d) {
  // worth a tile of 128 x 128: below 1e8 flops the CUDA-core kernel is faster
  return tc_shape_ok(d) && 2.0 * d.B * d.M * d.N * d.K >= 1e8;
}

// K splits: only when the output has too few tiles to fill the GPU; at least
// 4 slabs (128 of K) per split
int tc_split_rule(const ContractDesc& d) {
  const long long tiles = (round_up(d.M, TC_BM) / TC_BM) * (round_up(d.N, TC_BN) / TC_BN) * d.B;
  const long long nk = round_up(d.K, TC_BK) / TC_BK;
  const long long want = (2 * kNumSMs + tiles - 1) / tiles;
  long long sp = std::min<long long>(want, nk / 4);
  if (sp < 2) return 1;
  const long long per = (nk + sp - 1) / sp;
  return (int)((nk + per - 1) / per);
}

// largest split count worth trying: outputs with too few tiles to fill the
// GPU, at least 4 slabs (128 of K) per split
int tc_split_max(const ContractDesc& d) {
  const long long tiles = (round_up(d.M, TC_BM) / TC_BM) * (round_up(d.N, TC_BN) / TC_BN) * d.B;
  if (tiles >= 2 * kNumSMs) return 1;
  return (int)std::max<long long>(1, std::min<long long>(65535, round_up(d.K, TC_BK) / TC_BK / 4));
}

size_t tc_scratch_floats(const ContractDesc& d) {
  const long long Kp = round_up(d.K, TC_BK), Mp = round_up(d.M, TC_BM), Np = round_up(d.N, TC_BN);
  size_t f = (size_t)2 * d.B * Kp * (Mp + Np) + 64;
  if (tc_split_max(d) > 1) f += (size_t)2 * d.B * Mp * Np + 64;   // FP64 partial sums
  return f;
}

void launch_contract_tc(const ContractDesc& d, const double* A, const double* B, double* C, cudaStream_t s,
                        float* scratch, int* status, unsigned long long wait_ns, int splits_req) {
  if (d.M == 0 || d.N == 0 || d.B == 0) return;
  const long long Kp = round_up(d.K, TC_BK), Mp = round_up(d.M, TC_BM), Np = round_up(d.N, TC_BN);
  float* pa = scratch;
  float* pb = scratch + 2 * d.B * Mp * Kp;
  SCTM_CHECK((reinterpret_cast<uintptr_t>(pa) & 127) == 0 && (reinterpret_cast<uintptr_t>(pb) & 127) == 0,
             "tensor-core scratch misaligned");
  // operand A: rows = m, strides .sa ; operand B: rows = n, strides .sb
  PackDesc pA;
  pA.bat = d.bat, pA.rows = d.m, pA.k = d.k;
  pA.nb = d.B, pA.R = d.M, pA.K = d.K, pA.Rp = Mp, pA.Kp = Kp, pA.k_inner = d.a_k_inner;
  PackDesc pB;
  pB.bat = d.bat, pB.rows = d.n, pB.k = d.k;
  for (int i = 0; i < kMaxDims; ++i) {
    pB.bat.sa[i] = d.bat.sb[i];
    pB.rows.sa[i] = d.n.sb[i];
    pB.k.sa[i] = d.k.sb[i];
  }
  pB.nb = d.B, pB.R = d.N, pB.K = d.K, pB.Rp = Np, pB.Kp = Kp, pB.k_inner = d.b_n_inner ? 0 : 1;
  // packing is a gather: reads the FP64 operand once, writes its hi and lo panels
  {
    ProfScope ps(PF_MISC, s, 0.0, 8.0 * d.B * d.M * d.K + 8.0 * d.B * Kp * Mp, 1, "tf32_pack");
    pack_tf32x2_kernel<<<dim3((unsigned)((Kp / 32) * (Mp / 32)), (unsigned)d.B), dim3(32, 8), 0, s>>>(pA, A, pa);
    SCTM_CUDA(cudaGetLastError());
  }
  {
    ProfScope ps(PF_MISC, s, 0.0, 8.0 * d.B * d.N * d.K + 8.0 * d.B * Kp * Np, 1, "tf32_pack");
    pack_tf32x2_kernel<<<dim3((unsigned)((Kp / 32) * (Np / 32)), (unsigned)d.B), dim3(32, 8), 0, s>>>(pB, B, pb);
    SCTM_CUDA(cudaGetLastError());
  }
  CUtensorMap mA = panel_map(pa, d.B, Mp, Kp, TC_BM);
  CUtensorMap mB = panel_map(pb, d.B, Np, Kp, TC_BN);
  TcEpi e;
  e.bat = d.bat, e.m = d.m, e.n = d.n;
  e.M = d.M, e.N = d.N, e.alpha = d.alpha, e.beta = d.beta;
  e.num_m = (int)(Mp / TC_BM), e.num_n = (int)(Np / TC_BN);
  static bool attr = false;
  if (!attr) {
    SCTM_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    attr = true;
  }
  const int nk = (int)(Kp / TC_BK);
  int splits = tc_split_rule(d);
  if (splits_req > 0) splits = std::min(splits_req, tc_split_max(d));
  const int per = (nk + splits - 1) / splits;
  splits = (nk + per - 1) / per;
  double* W = nullptr;
  if (splits > 1) {
    W = reinterpret_cast<double*>(pb + 2 * d.B * Np * Kp + 32);   // 128-byte aligned (offsets are multiples of 32 floats)
    W = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(W) + 255) & ~uintptr_t(255));
    SCTM_CUDA(cudaMemsetAsync(W, 0, (size_t)d.B * Mp * Np * sizeof(double), s));
  }
  dim3 grid((unsigned)((long long)e.num_m * e.num_n), (unsigned)d.B, (unsigned)splits);
  // algorithmic work 2 B M N K (the tensor pipe executes three TF32 products
  // per multiply-add); bytes: the hi/lo panels read once, the FP64 result written
  {
    ProfScope ps(PF_TENSOR, s, 2.0 * d.B * d.M * d.N * d.K,
                 8.0 * d.B * Kp * (Mp + Np) + 8.0 * d.B * d.M * d.N * (d.beta != 0 ? 2 : 1));
    tc_gemm_kernel<<<grid, TC_THREADS_V2, TC_SMEM, s>>>(mA, mB, e, nk, per, C, W, Mp, Np, status, wait_ns);
    SCTM_CUDA(cudaGetLastError());
  }
  if (W) launch_splitk_finish(d, Mp, Np, W, C, s);
}

}  // namespace sctm
