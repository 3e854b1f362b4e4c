// Tensor-core GEMMs for the mixed-precision path (sm_103a, tcgen05 + TMA).
//
// C (FP64 out) = alpha * sum_s A_{a(s)} B_{b(s)}^T over "segments" s, where
// A_i (M x K) and B_j (N x K) are BF16 slices of FP64 operands, both stored
// K-major (row-major with K contiguous, leading dimension ld).
//
// Slicing is fixed-point per row: with 2^e_r > max_k |X_rk|, the slices of
// x are the balanced base-256 digits (in [-128, 128]) of the integer
// round(x 2^(7 + 8(S-1) - e_r)), digit a scaled by 2^(e_r - 7 - 8a), so
// X ~ X0 + X1 + ... keeps 8 bits per slice relative to the row maximum.  A
// product of slices a and b of rows r and s is then an integer of magnitude
// <= 2^14 times the single scale 2^(e_r + e_s - 14 - 8(a + b)); a sum of up
// to 512 such products (one accumulation chunk) stays below 2^23 and is
// exact in the FP32 tensor-core accumulator.  The product keeps the slice
// pairs with a + b < slices (1, 3, 6 or 10 terms for 1-4 slices).
//
// One CTA computes a 128 x 128 tile with 18 warps:
//   warp 0 / lane 0 : TMA producer (128B-swizzled boxes of 128 rows x 64 K)
//   warp 1          : allocates / frees TMEM; lane 0 issues tcgen05.mma
//                     (M = 128, N = 128, K = 16 slices)
//   warps 2-17      : epilogue; warp w reads TMEM lane quarter w % 4 and
//                     the 32-column group (w - 2) / 4
// K is consumed in chunks of kChunk k-tiles that never straddle two
// segments.  Each chunk accumulates (exactly, see above) in FP32 in one of
// two TMEM buffers (2 x 128 columns); the epilogue warps fold every finished
// chunk into double-float registers (FP32 hi + lo, TwoSum).  The final tile
// is written in FP64.
// A ring of kStages shared-memory stages is guarded by mbarriers (full: TMA
// transaction bytes; empty: tcgen05.commit); the TMEM buffers by acc_full
// (tcgen05.commit) and acc_empty (one arrival per epilogue warp).  Every wait is
// bounded; on expiry the kernel raises an error flag, waits (bounded) for its
// own TMA copies, frees its TMEM and returns.
// With sym != 0 (M == N, result known symmetric) only tiles with
// row-tile <= col-tile run and values are mirrored, so C is bitwise symmetric.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tc_gemm.h"

namespace kx {

constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 5;
constexpr int kChunk = 8;                    // k-tiles (512 K) per exact FP32 accumulation chunk
constexpr int kEpiWarps = 16;                // 4 lane quarters x 4 column groups of 32
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kTileBytesA = kBM * kBK * 2;   // 16 KB
constexpr int kTileBytesB = kBN * kBK * 2;   // 16 KB
constexpr int kSmemBytes = kStages * (kTileBytesA + kTileBytesB) + 1024 + 256;
constexpr long long kWaitLimit = 1LL << 22;

struct SegTable {
  int nseg;
  int a[10];
  int b[10];
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false on timeout or when another thread flagged an error
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, long long limit = kWaitLimit) {
  for (long long it = 0; it < limit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 1023) == 1023 && *(volatile int*)err) return false;
  }
  atomicOr(err, 1);
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row atoms of 1024 B
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // layout: 128B swizzle
  return d;
}
// instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = 128
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4)                      // D format FP32
         | (1u << 7)                    // A format BF16
         | (1u << 10)                   // B format BF16
         | ((uint32_t)(kBN >> 3) << 17) // N / 8
         | ((uint32_t)(kBM >> 4) << 24);// M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 consecutive TMEM columns of this warp's lane quarter (half the registers
// of the 32-column load, which keeps the epilogue's accumulators in registers)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 8 consecutive TMEM columns (the grouped kernel's epilogue folds two
// accumulators per chunk and keeps its double-float registers without spills)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcMaps {
  CUtensorMap a[kTcMaxSlices];
  CUtensorMap b[kTcMaxSlices];
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// error-free FP32 addition folded into a (hi, lo) pair
__device__ __forceinline__ void twosum_acc(float& hi, float& lo, float b) {
  float s = hi + b;
  float bb = s - hi;
  float err = (hi - (s - bb)) + (b - bb);
  hi = s;
  lo += err;
}

__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ TcMaps maps, SegTable seg, int M, int N, int K, double alpha,
                   double* __restrict__ C, int ldc, int sym, int beta, int* err, const int* gate, int kt_split,
                   long long c_zstride) {
  if (gate && *gate == 0) return;      // whole CTA, before any barrier or TMEM use
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (sym && bi > bj) return;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + kStages * kTileBytesA;
  uint64_t* full = (uint64_t*)(sB + kStages * kTileBytesB);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = bi * kBM, n0 = bj * kBN;
  // split-K (kt_split > 0): CTA z takes k-tiles [z kt_split, (z + 1) kt_split) and
  // writes its partial product to C + z c_zstride
  const int ktiles_all = (K + kBK - 1) / kBK;
  const int kt0 = (kt_split > 0) ? (int)blockIdx.z * kt_split : 0;
  int ktiles = (kt_split > 0) ? min(kt_split, ktiles_all - kt0) : ktiles_all;
  if (ktiles < 0) ktiles = 0;
  C += (long long)blockIdx.z * c_zstride;
  const int total = seg.nseg * ktiles;
  const int cps = (ktiles + kChunk - 1) / kChunk;   // chunks per segment
  const int nchunks = seg.nseg * cps;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * kBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer
      int issued = 0;
      bool ok = true;
      for (int it = 0; it < total && ok; ++it) {
        int s = it % kStages;
        uint32_t ph = (uint32_t)(it / kStages) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, err)) { ok = false; break; }
        int sg = it / ktiles, kt = it % ktiles;
        mbar_expect_tx(&full[s], kTileBytesA + kTileBytesB);
        tma_load_2d(sA + s * kTileBytesA, &maps.a[seg.a[sg]], &full[s], (kt0 + kt) * kBK, m0);
        tma_load_2d(sB + s * kTileBytesB, &maps.b[seg.b[sg]], &full[s], (kt0 + kt) * kBK, n0);
        issued = it + 1;
      }
      if (!ok) {
        // let our own copies land before the CTA can exit
        for (int it = (issued > kStages ? issued - kStages : 0); it < issued; ++it) {
          int s = it % kStages;
          uint32_t ph = (uint32_t)(it / kStages) & 1u;
          for (long long w = 0; w < kWaitLimit && !mbar_try(&full[s], ph); ++w) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: chunk c accumulates into TMEM buffer c & 1
      const uint32_t idesc = make_idesc();
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1;
        if (!mbar_wait(&acc_empty[b], ((uint32_t)(c >> 1) & 1u) ^ 1u, err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t dst = tmem + (uint32_t)(b * kBN);
        const int sg = c / cps, cc = c % cps;
        const int it0 = sg * ktiles + cc * kChunk;
        const int seg_end = (sg + 1) * ktiles;
        const int it1 = (it0 + kChunk < seg_end) ? it0 + kChunk : seg_end;
        for (int it = it0; it < it1; ++it) {
          int s = it % kStages;
          uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!mbar_wait(&full[s], ph, err)) { ok = false; break; }
          tc_fence_after();
          uint32_t a_addr = smem_u32(sA + s * kTileBytesA);
          uint32_t b_addr = smem_u32(sB + s * kTileBytesB);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            uint64_t da = smem_desc(a_addr + k * 32);
            uint64_t db = smem_desc(b_addr + k * 32);
            umma_bf16(dst, da, db, idesc, (it > it0 || k > 0) ? 1u : 0u);
          }
          umma_commit(&empty[s]);
        }
        if (ok) umma_commit(&acc_full[b]);
      }
    }
  } else {
    // epilogue warps: fold each chunk into double-float accumulators
    const int quarter = warp & 3;              // TMEM lanes 32 * quarter ...
    const int cg = (warp - 2) >> 2;            // columns 32 * cg ...
    float hi[32], lo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) { hi[j] = 0.0f; lo[j] = 0.0f; }
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1;
      bool got = mbar_wait(&acc_full[b], (uint32_t)(c >> 1) & 1u, err);
      got = __all_sync(0xffffffffu, got);
      if (!got) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kBN + cg * 32 + h * 16), r);
#pragma unroll
        for (int j = 0; j < 16; ++j) twosum_acc(hi[h * 16 + j], lo[h * 16 + j], __uint_as_float(r[j]));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
    if (ok && total > 0) {
      const int row = m0 + quarter * 32 + lane;
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          int col = n0 + cg * 32 + j;
          if (col >= N) break;
          if (sym && row > col) continue;
          double v = alpha * ((double)hi[j] + (double)lo[j]);
          if (beta) v += C[(size_t)row * ldc + col];
          C[(size_t)row * ldc + col] = v;
          if (sym && row != col) C[(size_t)col * ldc + row] = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kBN) : "memory");
  }
}

// the same for 64-byte swizzled K-major tiles (8-row atoms of 512 B)
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;                 // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)4 << 61;                          // layout: 64B swizzle
  return d;
}

// Slice-grouped products of S-slice operands (S = 3: the DMPT products of
// eq. 36; S = 4: the density product of eq. 19 and the back-transformation).
// Same tile, warps and bounded waits as tc_gemm_kernel, but one pipeline stage
// holds all S slices of A and of B for one BK-deep k-tile, and the S(S+1)/2
// kept slice products of that k-tile are issued from it: every byte brought
// into shared memory feeds S(S+1)/(2S) times the tensor work of the
// per-segment kernel.  Two accumulators per TMEM buffer:
//   acc0 : A0 B0, summed exactly over a 512-K chunk (as in tc_gemm_kernel);
//   acc1 : every product A_a B_b with 1 <= a + b < S (weights 2^-8 ... of
//          acc0's), smallest weights first, summed in FP32 over the chunk.
// Both are folded into the double-float registers after every chunk.  The
// FP32 rounding of acc1 is ~2^-(24 + 7) of sum |a||b| per addition, so the
// result is the S-slice product to within ~2^-26 (S = 3) or ~2^-28 (S = 4)
// of sum_k |a_ik||b_jk|, below or at the truncation of the slices, rather
// than bitwise the sum of its slice products.
// Layouts: BK = 64 with 128-byte swizzled boxes (2 stages of 96 KB for S = 3),
// BK = 32 with 64-byte swizzled boxes (3 stages of 64 KB for S = 4); the
// tensor maps passed in must use the matching box and swizzle.
// Split-K (kt_split > 0): CTA z takes k-tiles [z kt_split, (z + 1) kt_split)
// and writes its partial product to C + z c_zstride.  beta != 0 adds to C.
// The output tile goes through shared memory (the stages are idle by then).
// TMEM: 4 x 128 columns (acc0 and acc1, double-buffered).
template <int S, int BK>
struct GroupedCfg {
  static constexpr int kTile = kBM * BK * 2;                 // one slice tile of A or B
  static constexpr int kStageBytes = 2 * S * kTile;
  static constexpr int kStages = (192 * 1024) / kStageBytes;
  static constexpr int kChunkTiles = 512 / BK;               // k-tiles per exact chunk
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 256;
  static_assert(kBM == kBN, "A and B tiles share one size");
  static_assert(kBM * (kBN + 1) * (int)sizeof(double) <= kStages * kStageBytes, "output tile fits the stages");
  static_assert(kStages >= 2, "at least two stages");
};

template <int BK>
__device__ __forceinline__ uint64_t grouped_desc(uint32_t addr) {
  if constexpr (BK == 64)
    return smem_desc(addr);
  else
    return smem_desc_sw64(addr);
}

template <int S, int BK>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_grouped_kernel(const __grid_constant__ TcMaps maps, int M, int N, int K, double alpha,
                           double* __restrict__ C, int ldc, int sym, int beta, int* err, const int* gate,
                           int kt_split, long long c_zstride) {
  using Cfg = GroupedCfg<S, BK>;
  constexpr int T = Cfg::kTile, kStages = Cfg::kStages, kStageBytes = Cfg::kStageBytes;
  if (gate && *gate == 0) return;      // whole CTA, before any barrier or TMEM use
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (sym && bi > bj) return;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(base + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = bi * kBM, n0 = bj * kBN;
  const int ktiles_all = (K + BK - 1) / BK;
  const int kt0 = (kt_split > 0) ? (int)blockIdx.z * kt_split : 0;
  int ktiles = (kt_split > 0) ? min(kt_split, ktiles_all - kt0) : ktiles_all;
  if (ktiles < 0) ktiles = 0;
  C += (long long)blockIdx.z * c_zstride;
  const int nchunks = (ktiles + Cfg::kChunkTiles - 1) / Cfg::kChunkTiles;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(4 * kBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer: the S slices of A and of B of k-tile `it` into one stage
      int issued = 0;
      bool ok = true;
      for (int it = 0; it < ktiles && ok; ++it) {
        const int st = it % kStages;
        const uint32_t ph = (uint32_t)(it / kStages) & 1u;
        if (!mbar_wait(&empty[st], ph ^ 1u, err)) { ok = false; break; }
        uint8_t* sbase = base + st * kStageBytes;
        mbar_expect_tx(&full[st], kStageBytes);
#pragma unroll
        for (int a = 0; a < S; ++a) {
          tma_load_2d(sbase + a * T, &maps.a[a], &full[st], (kt0 + it) * BK, m0);
          tma_load_2d(sbase + (S + a) * T, &maps.b[a], &full[st], (kt0 + it) * BK, n0);
        }
        issued = it + 1;
      }
      if (!ok) {
        for (int it = (issued > kStages ? issued - kStages : 0); it < issued; ++it) {
          const int st = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          for (long long w = 0; w < kWaitLimit && !mbar_try(&full[st], ph); ++w) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc();
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1;
        if (!mbar_wait(&acc_empty[b], ((uint32_t)(c >> 1) & 1u) ^ 1u, err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d0 = tmem + (uint32_t)(b * kBN);
        const uint32_t d1 = tmem + (uint32_t)((2 + b) * kBN);
        const int it0 = c * Cfg::kChunkTiles;
        const int it1 = (it0 + Cfg::kChunkTiles < ktiles) ? it0 + Cfg::kChunkTiles : ktiles;
        for (int it = it0; it < it1; ++it) {
          const int st = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!mbar_wait(&full[st], ph, err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(base + st * kStageBytes);
          const uint32_t sb = sa + S * T;
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint32_t acc = (it > it0 || k > 0) ? 1u : 0u;
            // weight 1: A0 B0
            umma_bf16(d0, grouped_desc<BK>(sa + k * 32), grouped_desc<BK>(sb + k * 32), idesc, acc);
            // weights 2^-8(S-1) ... 2^-8, smallest first; the first one starts acc1 in a new chunk
#pragma unroll
            for (int dsum = S - 1; dsum >= 1; --dsum)
#pragma unroll
              for (int a = dsum; a >= 0; --a) {
                const uint32_t acc1 = (dsum == S - 1 && a == dsum) ? acc : 1u;
                umma_bf16(d1, grouped_desc<BK>(sa + a * T + k * 32), grouped_desc<BK>(sb + (dsum - a) * T + k * 32),
                          idesc, acc1);
              }
          }
          umma_commit(&empty[st]);
        }
        if (ok) umma_commit(&acc_full[b]);
      }
    }
  } else {
    // epilogue warps: fold both accumulators of each chunk into double-float registers
    const int quarter = warp & 3;
    const int cg = (warp - 2) >> 2;
    float hi[32], lo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) { hi[j] = 0.0f; lo[j] = 0.0f; }
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1;
      bool got = mbar_wait(&acc_full[b], (uint32_t)(c >> 1) & 1u, err);
      got = __all_sync(0xffffffffu, got);
      if (!got) { ok = false; break; }
      tc_fence_after();
      const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        uint32_t r[8];
        tmem_ld8(tmem + lane_base + (uint32_t)(b * kBN + cg * 32 + h * 8), r);
#pragma unroll
        for (int j = 0; j < 8; ++j) twosum_acc(hi[h * 8 + j], lo[h * 8 + j], __uint_as_float(r[j]));
        tmem_ld8(tmem + lane_base + (uint32_t)((2 + b) * kBN + cg * 32 + h * 8), r);
#pragma unroll
        for (int j = 0; j < 8; ++j) twosum_acc(hi[h * 8 + j], lo[h * 8 + j], __uint_as_float(r[j]));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
    // the tile through shared memory: the thread's 32 values at constant
    // offsets, then row-contiguous stores of the tile and, for a symmetric
    // result, of its transpose.  Every epilogue warp reaches the named
    // barrier; the global stores run only when no wait of any CTA expired.
    constexpr int kLdT = kBN + 1;                      // padded row: conflict-free transposed reads
    double* tile = (double*)base;
    if (ok) {
      const int rl = quarter * 32 + lane;
#pragma unroll
      for (int j = 0; j < 32; ++j) tile[rl * kLdT + cg * 32 + j] = alpha * ((double)hi[j] + (double)lo[j]);
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
    if (ktiles > 0 && *(volatile int*)err == 0) {
      const int t = threadIdx.x - 64;
      for (int idx = t; idx < kBM * kBN; idx += kEpiWarps * 32) {
        const int rr = idx / kBN, cc = idx - rr * kBN;
        const int row = m0 + rr, col = n0 + cc;
        if (row < M && col < N && !(sym && row > col)) {
          const size_t at = (size_t)row * ldc + col;
          C[at] = beta ? C[at] + tile[rr * kLdT + cc] : tile[rr * kLdT + cc];
        }
      }
      if (sym) {
        // C[col][row] for row < col: rows of the output are columns of the tile
        for (int idx = t; idx < kBM * kBN; idx += kEpiWarps * 32) {
          const int cr = idx / kBM, rc = idx - cr * kBM;   // output row n0 + cr, column m0 + rc
          const int row = m0 + rc, col = n0 + cr;
          if (row < M && col < N && row < col) {
            const size_t at = (size_t)col * ldc + row;
            C[at] = beta ? C[at] + tile[rc * kLdT + cr] : tile[rc * kLdT + cr];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * kBN) : "memory");
  }
}

// per-row scale exponent: e_r with max_k |X_rk| < 2^e_r (rows of X^T if transpose).
// |x| is compared as an integer (the bit patterns of non-negative doubles
// order like their values), keeping the FP64 pipe free.
__device__ __forceinline__ int exponent_of_max(unsigned long long bits) {
  // frexp exponent of a finite double given by its |x| bit pattern (0 -> 0)
  if (bits == 0) return 0;
  int be = (int)(bits >> 52);
  if (be == 0) {                       // subnormal
    int lz = __clzll((long long)(bits & 0xFFFFFFFFFFFFFULL)) - 12;
    return -1021 - lz;
  }
  return be - 1022;
}

__global__ void row_exponent_kernel(int n, const double* __restrict__ X, int transpose, int* __restrict__ ex,
                                    const int* gate) {
  if (gate && *gate == 0) return;
  int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (r >= n) return;
  unsigned long long m = 0;
  for (int k = lane; k < n; k += 32) {
    double v = transpose ? X[(size_t)k * n + r] : X[(size_t)r * n + k];
    unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
    m = (b > m) ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = (t > m) ? t : m;
  }
  if (lane == 0) ex[r] = exponent_of_max(m);
}

// Balanced base-256 digits of X = round(x 2^(7 + 8(S-1) - e)): slice a is digit
// a (most significant first) times 2^(e - 7 - 8a).  Digits lie in [-128, 128],
// so each slice value is exact in BF16.  X is formed from the bit pattern of x
// (x = +-M 2^(E - 1075), so |X| = M 2^-s0 rounded half up, s0 = 1075 - E - top
// + e) by 32-bit integer operations: when the row maximum is a normal number
// (e >= -1021) and top = 7 + 8(S-1) <= 31, s0 >= 22, so only the top 32 bits
// q = M >> 21 of the significand can reach X or its rounding bit, and
// |X| = (q >> s) + bit (s - 1) of q with s = s0 - 21 >= 1 (the same rounding
// as (M + 2^(s0-1)) >> s0: the dropped 21 bits cannot carry past a multiple of
// 2^s0).  Rows with a subnormal maximum and non-finite x take the 64-bit form.
// The element needs no FP64 instruction.
__device__ __forceinline__ void slice_digits(double x, int e, int slices, __nv_bfloat16* v) {
  const int top = 7 + 8 * (slices - 1);
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  const int E = (int)((bh >> 20) & 0x7FF);
  const unsigned q = (((bh & 0xFFFFFu) | (E != 0 ? 0x100000u : 0u)) << 11) | (bl >> 21);
  const int s0 = 1075 - (E != 0 ? E : 1) - top + e;
  long long X;
  if (s0 >= 22) {
    const int s = s0 - 21;
    unsigned mag = 0;
    if (s < 32)
      mag = (q >> s) + ((q >> (s - 1)) & 1u);
    else if (s == 32)
      mag = q >> 31;
    X = (long long)mag;
  } else {
    // a row whose maximum is subnormal (e <= -1022), or a non-finite x: 64-bit path
    unsigned long long M = b & 0xFFFFFFFFFFFFFULL;
    if (E != 0) M |= 1ULL << 52;
    const int sh = -s0;
    X = 0;
    if (sh >= 0)
      X = (long long)(M << (sh < 11 ? sh : 11));
    else if (sh > -64)
      X = (long long)((M + (1ULL << (-sh - 1))) >> (-sh));
  }
  if (bh >> 31) X = -X;
  // digits from the least significant (slice slices-1) up; unrolled over the
  // maximum slice count so that the digits stay in registers
  int dig[kTcMaxSlices];
#pragma unroll
  for (int a = kTcMaxSlices - 1; a > 0; --a) {
    if (a < slices) {
      int r = (int)(X & 0xFF);
      if (r >= 128) r -= 256;
      dig[a] = r;
      X = (X - r) >> 8;
    } else {
      dig[a] = 0;
    }
  }
  dig[0] = (int)X;
#pragma unroll
  for (int a = 0; a < kTcMaxSlices; ++a) {
    if (a < slices) {
      const int k = e - 7 - 8 * a;                         // slice scale 2^k
      const float p2 = (k >= -126 && k <= 127) ? __int_as_float((k + 127) << 23) : 0.0f;
      v[a] = __float2bfloat16_rn((float)dig[a] * p2);
    }
  }
}

__device__ __forceinline__ void slice_value(double x, int e, int slices, __nv_bfloat16* out, size_t stride,
                                            size_t t) {
  __nv_bfloat16 v[kTcMaxSlices];
  slice_digits(x, e, slices, v);
#pragma unroll
  for (int a = 0; a < kTcMaxSlices; ++a)
    if (a < slices) out[a * stride + t] = v[a];
}

// FP64 -> fixed-point BF16 slices relative to the row exponent; ld-padded rows
__global__ void split_bf16_kernel(int n, const double* __restrict__ X, int ld, int slices, int transpose,
                                  const int* __restrict__ ex, __nv_bfloat16* const* __restrict__ P,
                                  const int* gate) {
  if (gate && *gate == 0) return;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)n * ld;
  if (t >= tot) return;
  int i = (int)(t / ld), j = (int)(t % ld);
  double x = 0.0;
  if (j < n) x = transpose ? X[(size_t)j * n + i] : X[(size_t)i * n + j];
  __nv_bfloat16 v[kTcMaxSlices];
  slice_digits(x, ex[i], slices, v);
#pragma unroll
  for (int a = 0; a < kTcMaxSlices; ++a)
    if (a < slices) P[a][t] = v[a];
}

// same slicing as split_bf16_kernel, slices at base + a * stride (no pointer table)
__global__ void split_bf16_strided_kernel(int n, const double* __restrict__ X, int ld, int slices, int transpose,
                                          const int* __restrict__ ex, __nv_bfloat16* __restrict__ base,
                                          size_t stride) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)n * ld;
  if (t >= tot) return;
  int i = (int)(t / ld), j = (int)(t % ld);
  double x = 0.0;
  if (j < n) x = transpose ? X[(size_t)j * n + i] : X[(size_t)i * n + j];
  slice_value(x, ex[i], slices, base, stride, t);
}

// per-row exponent of op(X), op(X) = X (rows x cols, ldx) or X^T (X stored cols x rows)
__global__ void row_exponent_general_kernel(int rows, int cols, const double* __restrict__ X, int ldx,
                                            int transpose, int* __restrict__ ex) {
  int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (r >= rows) return;
  unsigned long long m = 0;
  for (int k = lane; k < cols; k += 32) {
    double v = transpose ? X[(size_t)k * ldx + r] : X[(size_t)r * ldx + k];
    unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
    m = (b > m) ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = (t > m) ? t : m;
  }
  if (lane == 0) ex[r] = exponent_of_max(m);
}

__global__ void split_general_kernel(int rows, int cols, const double* __restrict__ X, int ldx, int transpose,
                                     int slices, const int* __restrict__ ex, __nv_bfloat16* __restrict__ base,
                                     int ld, size_t stride) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)rows * ld;
  if (t >= tot) return;
  int i = (int)(t / ld), j = (int)(t % ld);
  double x = 0.0;
  if (j < cols) x = transpose ? X[(size_t)j * ldx + i] : X[(size_t)i * ldx + j];
  slice_value(x, ex[i], slices, base, stride, t);
}

// Row-wise slicing in one pass per row (a warp per row: the row maximum by
// shuffles, then the slices); columns cols..ld-1 are written as zeros.  Used
// by the back-transformation, whose operands change shape block by block.
// Batched forms: blockIdx.y is a block of reflectors b (kblk of them, rows
// k = b kblk .. of the reflector store, columns c0 = b kblk + 1 .. n-1).
struct RowSplit {
  int rows, cols;          // rows of op(X), K extent
  const double* X;         // row r at X + r * ldx
  long long ldx;
  __nv_bfloat16* base;     // slice a, row r, column k at base + a * stride + r * ld + k
  int ld;
  size_t stride;
};

__device__ __forceinline__ void split_row_warp(const RowSplit& q, int r, int slices, int lane) {
  const double* x = q.X + (long long)r * q.ldx;
  unsigned long long m = 0;
  for (int k = lane; k < q.cols; k += 32) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x[k]) & 0x7FFFFFFFFFFFFFFFULL;
    m = (b > m) ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = (t > m) ? t : m;
  }
  const int e = exponent_of_max(m);
  // eight consecutive columns per lane and step: all eight loads are issued
  // before the slicing and its stores (the stores may alias nothing the loads
  // read, but the compiler cannot know that), and each slice gets two aligned
  // 8-byte stores (ld is a multiple of 8)
  __nv_bfloat16* out = q.base + (size_t)r * q.ld;
  for (int k0 = 8 * lane; k0 < q.ld; k0 += 256) {
    double xv[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) xv[c] = (k0 + c < q.cols) ? x[k0 + c] : 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      __nv_bfloat16 v[4][kTcMaxSlices];
#pragma unroll
      for (int c = 0; c < 4; ++c) slice_digits(xv[4 * h + c], e, slices, v[c]);
#pragma unroll
      for (int a = 0; a < kTcMaxSlices; ++a) {
        if (a < slices) {
          __nv_bfloat162 lo2, hi2;
          lo2.x = v[0][a]; lo2.y = v[1][a];
          hi2.x = v[2][a]; hi2.y = v[3][a];
          uint2 w;
          w.x = *(const uint32_t*)&lo2;
          w.y = *(const uint32_t*)&hi2;
          *(uint2*)(out + a * q.stride + k0 + 4 * h) = w;
        }
      }
    }
  }
}

// One pass per row of a square n x n operand, one block of kSqThreads per row:
// the row maximum (block reduction), then the slices of four consecutive
// columns per thread, stored as 8-byte groups per slice (ld is a multiple of
// 64, so every group is aligned); columns n..ld-1 are zeros.  The second sweep
// re-reads the row from L1/L2, so X leaves HBM once.
constexpr int kSqThreads = 128;
__global__ void __launch_bounds__(kSqThreads) split_rows_sq_kernel(int n, const double* __restrict__ X, int ld,
                                                                 int slices, int* __restrict__ ex,
                                                                 __nv_bfloat16* __restrict__ base, size_t stride,
                                                                 const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ unsigned long long s_max[kSqThreads / 32];
  const int r = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double* x = X + (size_t)r * n;
  unsigned long long m = 0;
  for (int k = tid; k < n; k += kSqThreads) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x[k]) & 0x7FFFFFFFFFFFFFFFULL;
    m = (b > m) ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = (t > m) ? t : m;
  }
  if (lane == 0) s_max[wid] = m;
  __syncthreads();
#pragma unroll
  for (int w = 0; w < kSqThreads / 32; ++w) m = (s_max[w] > m) ? s_max[w] : m;
  const int e = exponent_of_max(m);
  if (tid == 0) ex[r] = e;
  for (int k0 = 4 * tid; k0 < ld; k0 += 4 * kSqThreads) {
    __nv_bfloat16 v[4][kTcMaxSlices];
#pragma unroll
    for (int c = 0; c < 4; ++c) slice_digits((k0 + c < n) ? x[k0 + c] : 0.0, e, slices, v[c]);
#pragma unroll
    for (int a = 0; a < kTcMaxSlices; ++a) {
      if (a < slices) {
        __nv_bfloat162 lo2, hi2;
        lo2.x = v[0][a]; lo2.y = v[1][a];
        hi2.x = v[2][a]; hi2.y = v[3][a];
        uint2 w;
        w.x = *(const uint32_t*)&lo2;
        w.y = *(const uint32_t*)&hi2;
        *(uint2*)(base + a * stride + (size_t)r * ld + k0) = w;
      }
    }
  }
}

__global__ void split_rows_kernel(RowSplit q, int slices) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= q.rows) return;
  split_row_warp(q, r, slices, threadIdx.x & 31);
}

// mode 0: V_b (kb_b x m_b) from the reflector store;  mode 1: Y_b^T (m_b x kb_b)
// from YT + b n kblk (row length kblk)
__global__ void split_blocks_kernel(int mode, int n, int nref, int kblk, const double* __restrict__ src,
                                    __nv_bfloat16* base, size_t blk_stride, size_t slice_stride, int slices) {
  const int b = blockIdx.y;
  const int k0 = b * kblk;
  const int kb = min(kblk, nref - k0);
  const int m = n - (k0 + 1);
  RowSplit q;
  q.base = base + (size_t)b * blk_stride;
  q.stride = slice_stride;
  if (mode == 0) {
    q.rows = kb; q.cols = m; q.X = src + (size_t)k0 * n + (k0 + 1); q.ldx = n; q.ld = (m + 63) / 64 * 64;
  } else {
    q.rows = m; q.cols = kb; q.X = src + (size_t)b * n * kblk; q.ldx = kblk; q.ld = kblk;
  }
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= q.rows) return;
  split_row_warp(q, r, slices, threadIdx.x & 31);
}

// U = sum_z P_z (in order), then its slices (rows x cols, ld ldp; parts at P + z rows ldp)
__global__ void reduce_split_rows_kernel(int rows, int cols, const double* __restrict__ P, int parts, int ldp,
                                         int slices, __nv_bfloat16* base, int ld, size_t stride) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  constexpr int kMaxPer = 4;                 // cols <= 128
  double v[kMaxPer];
  unsigned long long m = 0;
#pragma unroll
  for (int c = 0; c < kMaxPer; ++c) {
    const int k = lane + 32 * c;
    double a = 0.0;
    if (k < cols)
      for (int z = 0; z < parts; ++z) a += P[((size_t)z * rows + r) * ldp + k];
    v[c] = a;
    unsigned long long bits = (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFULL;
    m = (bits > m) ? bits : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = (t > m) ? t : m;
  }
  const int e = exponent_of_max(m);
#pragma unroll
  for (int c = 0; c < kMaxPer; ++c) {
    const int k = lane + 32 * c;
    if (k < ld) slice_value(v[c], e, slices, base, stride, (size_t)r * ld + k);
  }
}

// Test of the bounded wait itself: one thread waits on an mbarrier that no one
// arrives at (no copy, no tensor-core work in flight), with `limit` tries.
__global__ void mbar_expiry_kernel(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_fence_init();
  mbar_wait(&bar, 0, err, limit);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

struct TcBuffers {
  int n, ld;
  __nv_bfloat16* piece[kTcPieceSlots][kTcMaxSlices];
  __nv_bfloat16** dpieces;            // device copy of the slice pointers, per slot
  CUtensorMap map[kTcPieceSlots][kTcMaxSlices];
  CUtensorMap map64[kTcPieceSlots][kTcMaxSlices];   // 32-wide boxes, 64-byte swizzle (grouped 4-slice kernel)
  int* ex;                            // per-row exponents, one array per slot
  int* err;
  bool maps_ok;
};

static int ld_for(int n) { return ((n + 63) / 64) * 64; }

size_t tc_work_bytes(int n) {
  size_t ld = (size_t)ld_for(n);
  size_t one = ((size_t)n * ld * 2 + 1023) & ~(size_t)1023;
  size_t exb = (((size_t)kTcPieceSlots * n * sizeof(int)) + 1023) & ~(size_t)1023;
  return 2048 + exb + 1024 + (size_t)kTcPieceSlots * kTcMaxSlices * one + 256;
}

// rows x cols BF16 operand (row length ld), boxes of `bk` columns x kBM rows:
// bk = 64 with the 128-byte swizzle, bk = 32 with the 64-byte swizzle
static bool make_map_rc_box(CUtensorMap* m, void* ptr, int rows, int cols, int ld, int bk) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)kBM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static bool make_map_rc(CUtensorMap* m, void* ptr, int rows, int cols, int ld) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static bool make_map(CUtensorMap* m, void* ptr, int n, int ld) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

void tc_work_bind(TcWork& w, void* base, int n) {
  // host-side bookkeeping lives in a heap object; the device arena holds the pieces
  TcBuffers* tb = new TcBuffers();
  tb->n = n;
  tb->ld = ld_for(n);
  size_t one = ((size_t)n * tb->ld * 2 + 1023) & ~(size_t)1023;
  uint8_t* p = (uint8_t*)(((uintptr_t)base + 1023) & ~(uintptr_t)1023);
  tb->err = (int*)p;
  tb->dpieces = (__nv_bfloat16**)(p + 64);
  p += 2048;
  tb->ex = (int*)p;
  p += (((size_t)kTcPieceSlots * n * sizeof(int)) + 1023) & ~(size_t)1023;
  tb->maps_ok = true;
  for (int s = 0; s < kTcPieceSlots; ++s)
    for (int k = 0; k < kTcMaxSlices; ++k) {
      tb->piece[s][k] = (__nv_bfloat16*)p;
      p += one;
      tb->maps_ok = tb->maps_ok && make_map(&tb->map[s][k], tb->piece[s][k], n, tb->ld);
      tb->maps_ok = tb->maps_ok && make_map_rc_box(&tb->map64[s][k], tb->piece[s][k], n, n, tb->ld, 32);
    }
  w.base = tb;
  w.bytes = tc_work_bytes(n);
  cudaMemset(tb->err, 0, sizeof(int));
  cudaMemcpy(tb->dpieces, tb->piece, sizeof(tb->piece), cudaMemcpyHostToDevice);
}

void tc_work_release(TcWork& w) {
  delete (TcBuffers*)w.base;
  w.base = nullptr;
}

bool tc_available() { return encode_fn() != nullptr; }

bool tc_ready(const TcWork& w) { return w.base && ((TcBuffers*)w.base)->maps_ok; }

int* tc_error_flag(const TcWork& w) { return w.base ? ((TcBuffers*)w.base)->err : nullptr; }

// the opt-in shared-memory size is a per-device attribute of the kernel
static void set_smem_attribute() {
  static PerDeviceOnce flag;
  once_per_device(flag, [] {
    return cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) ==
           cudaSuccess;
  });
}

void tc_split(cudaStream_t s, const TcWork& w, int slot, const double* X, int slices, int transpose,
              const int* gate) {
  TcBuffers* tb = (TcBuffers*)w.base;
  int n = tb->n;
  int* ex = tb->ex + (size_t)slot * n;
  if (!transpose) {
    split_rows_sq_kernel<<<n, kSqThreads, 0, s>>>(n, X, tb->ld, slices, ex, tb->piece[slot][0],
                                                  (size_t)(tb->piece[0][1] - tb->piece[0][0]), gate);
    count_launch();
    return;
  }
  row_exponent_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(n, X, transpose, ex, gate);
  count_launch();
  size_t tot = (size_t)n * tb->ld;
  split_bf16_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, X, tb->ld, slices, transpose, ex,
                                                                   tb->dpieces + (size_t)slot * kTcMaxSlices, gate);
  count_launch();
}

void tc_gemm(cudaStream_t s, const TcWork& w, int slotA, int slotB, int terms, double alpha, double* C, int sym,
             const int* gate) {
  TcBuffers* tb = (TcBuffers*)w.base;
  set_smem_attribute();
  TcMaps maps;
  for (int k = 0; k < kTcMaxSlices; ++k) {
    maps.a[k] = tb->map[slotA][k];
    maps.b[k] = tb->map[slotB][k];
  }
  // slice pairs (a, b) with a + b < slices, smallest terms first
  int slices = (terms == 10) ? 4 : (terms == 6) ? 3 : (terms == 3) ? 2 : 1;
  SegTable seg;
  seg.nseg = 0;
  for (int d = slices - 1; d >= 0; --d)
    for (int a = 0; a <= d; ++a) {
      seg.a[seg.nseg] = a;
      seg.b[seg.nseg] = d - a;
      ++seg.nseg;
    }
  int n = tb->n;
  dim3 grid((n + kBN - 1) / kBN, (n + kBM - 1) / kBM);
  tc_gemm_kernel<<<grid, kThreads, kSmemBytes, s>>>(maps, seg, n, n, n, alpha, C, n, sym, 0, tb->err, gate, 0, 0);
  count_launch();
}

template <int S, int BK>
static void grouped_attribute() {
  static PerDeviceOnce flag;
  once_per_device(flag, [] {
    return cudaFuncSetAttribute(tc_gemm_grouped_kernel<S, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                GroupedCfg<S, BK>::kSmem) == cudaSuccess;
  });
}

template <int S, int BK>
static void grouped_launch(cudaStream_t s, const TcMaps& maps, int M, int N, int K, double alpha, double* C, int ldc,
                           int sym, int beta, int* err, const int* gate, int kt_split, int z, long long zstride) {
  grouped_attribute<S, BK>();
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, z);
  tc_gemm_grouped_kernel<S, BK><<<grid, kThreads, GroupedCfg<S, BK>::kSmem, s>>>(
      maps, M, N, K, alpha, C, ldc, sym, beta, err, gate, kt_split, zstride);
  count_launch();
}

void tc_gemm_grouped(cudaStream_t s, const TcWork& w, int slotA, int slotB, double alpha, double* C, int sym,
                     const int* gate) {
  TcBuffers* tb = (TcBuffers*)w.base;
  TcMaps maps;
  for (int k = 0; k < kTcMaxSlices; ++k) {
    maps.a[k] = tb->map[slotA][k];
    maps.b[k] = tb->map[slotB][k];
  }
  const int n = tb->n;
  grouped_launch<3, 64>(s, maps, n, n, n, alpha, C, n, sym, 0, tb->err, gate, 0, 1, 0);
}

void tc_gemm_grouped4(cudaStream_t s, const TcWork& w, int slotA, int slotB, double alpha, double* C, int sym,
                      const int* gate) {
  TcBuffers* tb = (TcBuffers*)w.base;
  TcMaps maps;
  for (int k = 0; k < kTcMaxSlices; ++k) {
    maps.a[k] = tb->map64[slotA][k];
    maps.b[k] = tb->map64[slotB][k];
  }
  const int n = tb->n;
  grouped_launch<4, 32>(s, maps, n, n, n, alpha, C, n, sym, 0, tb->err, gate, 0, 1, 0);
}

static bool grouped_rc_maps(TcMaps* maps, int M, int N, int K, const __nv_bfloat16* Abase, int lda, size_t astride,
                            const __nv_bfloat16* Bbase, int ldb, size_t bstride) {
  for (int a = 0; a < kTcMaxSlices; ++a) {
    if (!make_map_rc_box(&maps->a[a], (void*)(Abase + a * astride), M, K, lda, 32)) return false;
    if (!make_map_rc_box(&maps->b[a], (void*)(Bbase + a * bstride), N, K, ldb, 32)) return false;
  }
  return true;
}

int tc_gemm_grouped_rc(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Abase, int lda, size_t astride,
                       const __nv_bfloat16* Bbase, int ldb, size_t bstride, double alpha, double* C, int ldc,
                       int beta, int* err) {
  TcMaps maps;
  if (!grouped_rc_maps(&maps, M, N, K, Abase, lda, astride, Bbase, ldb, bstride)) return -1;
  grouped_launch<4, 32>(s, maps, M, N, K, alpha, C, ldc, 0, beta, err, nullptr, 0, 1, 0);
  return 0;
}

int tc_gemm_grouped_rc_splitk(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Abase, int lda,
                              size_t astride, const __nv_bfloat16* Bbase, int ldb, size_t bstride, double alpha,
                              double* P, int ldp, int splits, int* err) {
  TcMaps maps;
  if (!grouped_rc_maps(&maps, M, N, K, Abase, lda, astride, Bbase, ldb, bstride)) return -1;
  constexpr int kCh = GroupedCfg<4, 32>::kChunkTiles;
  const int ktiles = (K + 31) / 32;
  int per = (ktiles + splits - 1) / splits;
  per = ((per + kCh - 1) / kCh) * kCh;                   // whole exact-sum chunks
  const int z = (ktiles + per - 1) / per;
  grouped_launch<4, 32>(s, maps, M, N, K, alpha, P, ldp, 0, 0, err, nullptr, per, z, (long long)M * ldp);
  return z;
}

int tc_ld(int n) { return ld_for(n); }

__nv_bfloat16* tc_slot_base(const TcWork& w, int slot) { return ((TcBuffers*)w.base)->piece[slot][0]; }
size_t tc_slot_stride(const TcWork& w) {
  TcBuffers* tb = (TcBuffers*)w.base;
  return (size_t)(tb->piece[0][1] - tb->piece[0][0]);
}
int* tc_slot_exponents(const TcWork& w, int slot) {
  TcBuffers* tb = (TcBuffers*)w.base;
  return tb->ex + (size_t)slot * tb->n;
}

// Slices of op(X) (rows x cols, K = cols) into `base` with row length ld and
// slice stride `stride` elements; ex receives the row exponents.
void tc_split_rc(cudaStream_t s, int rows, int cols, const double* X, int ldx, int transpose, int slices, int* ex,
                 __nv_bfloat16* base, int ld, size_t stride) {
  row_exponent_general_kernel<<<(rows * 32 + 255) / 256, 256, 0, s>>>(rows, cols, X, ldx, transpose, ex);
  count_launch();
  size_t tot = (size_t)rows * ld;
  split_general_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(rows, cols, X, ldx, transpose, slices, ex,
                                                                       base, ld, stride);
  count_launch();
}

// C (M x N, ldc) = alpha * sum slice products A_a B_b^T (+ C if beta), A: M x K slices, B: N x K slices
int tc_gemm_rc(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Abase, int lda, size_t astride,
               const __nv_bfloat16* Bbase, int ldb, size_t bstride, int terms, double alpha, double* C, int ldc,
               int beta, int* err) {
  set_smem_attribute();
  int slices = (terms == 10) ? 4 : (terms == 6) ? 3 : (terms == 3) ? 2 : 1;
  TcMaps maps;
  for (int a = 0; a < kTcMaxSlices; ++a) {
    int sa = (a < slices) ? a : 0;
    if (!make_map_rc(&maps.a[a], (void*)(Abase + sa * astride), M, K, lda)) return -1;
    if (!make_map_rc(&maps.b[a], (void*)(Bbase + sa * bstride), N, K, ldb)) return -1;
  }
  SegTable seg;
  seg.nseg = 0;
  for (int d = slices - 1; d >= 0; --d)
    for (int a = 0; a <= d; ++a) {
      seg.a[seg.nseg] = a;
      seg.b[seg.nseg] = d - a;
      ++seg.nseg;
    }
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
  tc_gemm_kernel<<<grid, kThreads, kSmemBytes, s>>>(maps, seg, M, N, K, alpha, C, ldc, 0, beta, err, nullptr,
                                                     0, 0);
  count_launch();
  return 0;
}

// Split-K variant of tc_gemm_rc: the K range is cut into `splits` parts (each a
// whole number of exact-sum chunks), part z writes alpha * (its partial sum) to
// P + z * M * ldp (M x N, ld ldp); the caller adds the parts in order.
int tc_gemm_rc_splitk(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Abase, int lda, size_t astride,
                      const __nv_bfloat16* Bbase, int ldb, size_t bstride, int terms, double alpha, double* P,
                      int ldp, int splits, int* err) {
  set_smem_attribute();
  int slices = (terms == 10) ? 4 : (terms == 6) ? 3 : (terms == 3) ? 2 : 1;
  TcMaps maps;
  for (int a = 0; a < kTcMaxSlices; ++a) {
    int sa = (a < slices) ? a : 0;
    if (!make_map_rc(&maps.a[a], (void*)(Abase + sa * astride), M, K, lda)) return -1;
    if (!make_map_rc(&maps.b[a], (void*)(Bbase + sa * bstride), N, K, ldb)) return -1;
  }
  SegTable seg;
  seg.nseg = 0;
  for (int d = slices - 1; d >= 0; --d)
    for (int a = 0; a <= d; ++a) {
      seg.a[seg.nseg] = a;
      seg.b[seg.nseg] = d - a;
      ++seg.nseg;
    }
  const int ktiles = (K + kBK - 1) / kBK;
  int per = (ktiles + splits - 1) / splits;
  per = ((per + kChunk - 1) / kChunk) * kChunk;          // whole exact-sum chunks
  const int z = (ktiles + per - 1) / per;
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, z);
  tc_gemm_kernel<<<grid, kThreads, kSmemBytes, s>>>(maps, seg, M, N, K, alpha, P, ldp, 0, 0, err, nullptr, per,
                                                     (long long)M * ldp);
  count_launch();
  return z;
}

void tc_split_rows(cudaStream_t s, int rows, int cols, const double* X, long long ldx, int slices,
                   __nv_bfloat16* base, int ld, size_t stride) {
  if (rows <= 0) return;
  RowSplit q{rows, cols, X, ldx, base, ld, stride};
  split_rows_kernel<<<(rows + 7) / 8, 256, 0, s>>>(q, slices);
  count_launch();
}

void tc_split_blocks(cudaStream_t s, int mode, int n, int nref, int kblk, const double* src, __nv_bfloat16* base,
                     size_t blk_stride, size_t slice_stride, int slices) {
  const int nblk = (nref + kblk - 1) / kblk;
  if (nblk <= 0) return;
  const int maxrows = (mode == 0) ? kblk : n;
  split_blocks_kernel<<<dim3((maxrows + 7) / 8, nblk), 256, 0, s>>>(mode, n, nref, kblk, src, base, blk_stride,
                                                                    slice_stride, slices);
  count_launch();
}

void tc_reduce_split_rows(cudaStream_t s, int rows, int cols, const double* P, int parts, int ldp, int slices,
                          __nv_bfloat16* base, int ld, size_t stride) {
  if (rows <= 0) return;
  reduce_split_rows_kernel<<<(rows + 7) / 8, 256, 0, s>>>(rows, cols, P, parts, ldp, slices, base, ld, stride);
  count_launch();
}

void tc_mbar_expiry(cudaStream_t s, int* err, long long limit) {
  mbar_expiry_kernel<<<1, 32, 0, s>>>(err, limit);
  count_launch();
}

bool tc_encode_map(CUtensorMap* m, void* ptr, int n, int ld) { return make_map(m, ptr, n, ld); }

void tc_split_strided(cudaStream_t s, int n, int ld, const double* X, int slices, int transpose, int* ex,
                      __nv_bfloat16* base, size_t stride) {
  row_exponent_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(n, X, transpose, ex, nullptr);
  count_launch();
  size_t tot = (size_t)n * ld;
  split_bf16_strided_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, X, ld, slices, transpose, ex, base,
                                                                           stride);
  count_launch();
}

void tc_gemm_on_maps(cudaStream_t s, int n, const CUtensorMap* mapsA, const CUtensorMap* mapsB, int terms,
                     double alpha, double* C, int sym, int* err) {
  set_smem_attribute();
  TcMaps maps;
  for (int k = 0; k < kTcMaxSlices; ++k) {
    maps.a[k] = mapsA[k];
    maps.b[k] = mapsB[k];
  }
  int slices = (terms == 10) ? 4 : (terms == 6) ? 3 : (terms == 3) ? 2 : 1;
  SegTable seg;
  seg.nseg = 0;
  for (int d = slices - 1; d >= 0; --d)
    for (int a = 0; a <= d; ++a) {
      seg.a[seg.nseg] = a;
      seg.b[seg.nseg] = d - a;
      ++seg.nseg;
    }
  dim3 grid((n + kBN - 1) / kBN, (n + kBM - 1) / kBM);
  tc_gemm_kernel<<<grid, kThreads, kSmemBytes, s>>>(maps, seg, n, n, n, alpha, C, n, sym, 0, err, nullptr, 0, 0);
  count_launch();
}

}  // namespace kx
