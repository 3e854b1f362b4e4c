// FP64 symmetric eigensolver for F = Q diag(eps) Q^T (eq. 19 needs the
// eigenpairs; eq. 36 needs them again for the DMPT response).
//
//  1. Householder tridiagonalisation in ONE persistent kernel: the rank-2
//     update of column k is applied lazily, fused with the symmetric
//     matrix-vector product of column k + 1, so every column costs one read
//     and one write of the trailing matrix and one grid-wide barrier.  All
//     blocks compute the reflector redundantly (same data, same reduction
//     order, bitwise identical), so no broadcast is needed.  The barrier is a
//     counter/generation pair with a bounded spin: on expiry the kernel sets
//     kStatusTimeout and returns.
//     The mixed-precision path runs the same algorithm in double-float
//     arithmetic (df.cuh): the trailing matrix is held as FP32 (hi, lo)
//     pairs and the O(n^2)-per-column update and matrix-vector product run on
//     the FP32 pipe, 64 times GB300's FP64 rate, at about 48 significant bits;
//     the reflector scalars (beta, tau) stay FP64.
//  2. Eigenvalues of the tridiagonal matrix by bisection on Sturm counts,
//     one thread per eigenvalue (ascending order by construction): a coarse
//     FP32 phase, an FP64 bracket check, then FP64 bisection.
//  3. Eigenvectors by inverse iteration (two steps) with a partially pivoted
//     tridiagonal LU, one thread per cluster of close eigenvalues; members of
//     a cluster are re-orthogonalised (modified Gram-Schmidt) in order.
//  4. Back-transformation Q = H_0 ... H_{n-3} Z with blocks of reflectors in
//     compact WY form (I - V T V^T): FP64 GEMMs (64 per block) on the FP64
//     path; on the mixed path (128 per block) the two large products
//     V^T Z and V (T W) run on the tensor cores with 4 fixed-point BF16
//     slices, while the T factor and T W stay in FP64.
#include <mutex>

#include "common.cuh"
#include "df.cuh"
#include "kernels.h"
#include "tc_gemm.h"

namespace kx {

constexpr int kTriThreads = 512;
constexpr int kBtBlock = 64;          // reflectors per back-transform block (FP64 path)
constexpr int kBtBlockTc = 128;       // reflectors per back-transform block (tensor-core path)
constexpr double kEps = 2.220446049250313e-16;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of the persistent tridiagonalisation.  The wait is bounded
// in wall time (kBarrierNs) and by an iteration cap; a block that gives up, or
// that finds another block's timeout flag set, records kStatusTimeout and the
// kernel returns.  Correct operation needs every block resident at once
// (cooperative launch; callers that run several such grids concurrently keep
// their total within what the device holds at one time, eig_tridiag_weight).
constexpr unsigned long long kBarrierNs = 2000000000ull;   // 2 s
// the wall-time limit the barriers use (per device; tests set it through
// eig_set_barrier_limit; 0 makes every wait expire at once, even one that
// would be satisfied, so a test can force the expiry path of a real step)
__device__ unsigned long long g_barrier_ns = kBarrierNs;

__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    unsigned g = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    if (g_barrier_ns == 0) {
      atomicOr(status, (int)kStatusTimeout);
    } else if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      long long it = 0;
      while (*vgen == g) {
        ++it;
        if ((it & 63) == 0 &&
            (global_ns() - t0 > g_barrier_ns || it > (1LL << 27) ||
             ((*(volatile int*)status) & kStatusTimeout))) {
          atomicOr(status, (int)kStatusTimeout);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    s_ok = ((*(volatile int*)status) & kStatusTimeout) ? 0 : 1;
  }
  __syncthreads();
  return s_ok != 0;
}

// Split-phase grid barrier on a monotonically increasing arrival counter
// (reset to 0 before the launch): the e-th barrier of a block is passed once
// the counter reaches e * nblocks.  grid_arrive makes the block's earlier
// writes visible (CTA barrier, then a release reduction by thread 0), so
// independent work can run before grid_wait (an acquire load, bounded in wall
// time like grid_barrier; on expiry kStatusTimeout is set and false returned).
__device__ __forceinline__ void grid_arrive(unsigned* cnt) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(cnt) : "memory");
}
__device__ bool grid_wait(const unsigned* cnt, unsigned target, int* status) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    const unsigned long long t0 = global_ns();
    long long it = 0;
    if (g_barrier_ns == 0) atomicOr(status, (int)kStatusTimeout);
    for (; g_barrier_ns != 0;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
      if ((int)(v - target) >= 0) break;
      ++it;
      if ((it & 63) == 0 && (global_ns() - t0 > g_barrier_ns || it > (1LL << 27) ||
                             ((*(volatile int*)status) & kStatusTimeout))) {
        atomicOr(status, (int)kStatusTimeout);
        break;
      }
      __nanosleep(16);
    }
    s_ok = ((*(volatile int*)status) & kStatusTimeout) ? 0 : 1;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kTriThreads) tridiag_kernel(int n, double* __restrict__ A,
                                                              double* __restrict__ Vst,
                                                              double* __restrict__ d,
                                                              double* __restrict__ e,
                                                              double* __restrict__ tau,
                                                              double* __restrict__ pbuf,
                                                              unsigned* bar, int* status) {
  extern __shared__ double sm[];
  double* vp = sm;           // previous reflector (valid for indices >= k)
  double* wp = sm + n;       // previous w
  double* vc = sm + 2 * n;   // current reflector
  double* red = sm + 3 * n;  // 32 doubles of reduction scratch
  __shared__ double s_par[4];  // beta, tau, scale, d_k
  const int tid = threadIdx.x, lane = tid & 31;
  const int wpb = blockDim.x >> 5;
  // row r of the trailing matrix goes to block r % G, warp (r / G) % wpb: every
  // block keeps an equal share of rows as the trailing matrix shrinks
  const int gw = blockIdx.x + gridDim.x * (tid >> 5);
  const int totw = gridDim.x * wpb;
  bool prev = false;

  for (int k = 0; k < n - 2; ++k) {
    // 1. row k of the lazily updated matrix
    double loc = 0.0;
    for (int j = k + 2 + tid; j < n; j += blockDim.x) {
      double x = A[(size_t)k * n + j];
      if (prev) x -= vp[k] * wp[j] + wp[k] * vp[j];
      vc[j] = x;
      loc += x * x;
    }
    double sigma = block_sum(loc, red);
    if (tid == 0) {
      double xk = A[(size_t)k * n + k];
      double x1 = A[(size_t)k * n + k + 1];
      if (prev) {
        xk -= 2.0 * vp[k] * wp[k];
        x1 -= vp[k] * wp[k + 1] + wp[k] * vp[k + 1];
      }
      double beta, t, scale;
      if (sigma == 0.0) {
        beta = x1; t = 0.0; scale = 0.0;
      } else {
        double nrm = ::sqrt(x1 * x1 + sigma);
        beta = (x1 >= 0.0) ? -nrm : nrm;
        t = (beta - x1) / beta;
        scale = 1.0 / (x1 - beta);
      }
      s_par[0] = beta; s_par[1] = t; s_par[2] = scale; s_par[3] = xk;
    }
    __syncthreads();
    const double t = s_par[1], scale = s_par[2];
    for (int j = k + 2 + tid; j < n; j += blockDim.x) vc[j] *= scale;
    if (tid == 0) vc[k + 1] = 1.0;
    __syncthreads();
    if (blockIdx.x == 0) {
      if (tid == 0) { d[k] = s_par[3]; e[k] = s_par[0]; tau[k] = t; }
      for (int j = tid; j < n; j += blockDim.x) Vst[(size_t)k * n + j] = (j > k) ? vc[j] : 0.0;
    }
    // 2. fused: apply the previous rank-2 update to rows/cols >= k+1 and
    //    form p = tau A v for the current reflector
    double* pb = pbuf + (size_t)(k & 1) * n;
    for (int i = k + 1 + gw; i < n; i += totw) {
      double* row = A + (size_t)i * n;
      double acc = 0.0, acc2 = 0.0, acc3 = 0.0, acc4 = 0.0;   // four chains hide the FP64 latency
      if (prev) {
        const double vi = vp[i], wi = wp[i];
        int j = k + 1 + lane;
        for (; j + 96 < n; j += 128) {
          double a = fma(-vi, wp[j], fma(-wi, vp[j], row[j]));
          double b = fma(-vi, wp[j + 32], fma(-wi, vp[j + 32], row[j + 32]));
          double c = fma(-vi, wp[j + 64], fma(-wi, vp[j + 64], row[j + 64]));
          double e = fma(-vi, wp[j + 96], fma(-wi, vp[j + 96], row[j + 96]));
          row[j] = a;
          row[j + 32] = b;
          row[j + 64] = c;
          row[j + 96] = e;
          acc = fma(a, vc[j], acc);
          acc2 = fma(b, vc[j + 32], acc2);
          acc3 = fma(c, vc[j + 64], acc3);
          acc4 = fma(e, vc[j + 96], acc4);
        }
        for (; j < n; j += 32) {
          double a = fma(-vi, wp[j], fma(-wi, vp[j], row[j]));
          row[j] = a;
          acc = fma(a, vc[j], acc);
        }
      } else {
        int j = k + 1 + lane;
        for (; j + 32 < n; j += 64) {
          acc = fma(row[j], vc[j], acc);
          acc2 = fma(row[j + 32], vc[j + 32], acc2);
        }
        for (; j < n; j += 32) acc = fma(row[j], vc[j], acc);
      }
      acc = warp_sum((acc + acc2) + (acc3 + acc4));
      if (lane == 0) pb[i] = t * acc;
    }
    if (!grid_barrier(bar, gridDim.x, status)) return;
    // 3. w = p - (tau/2)(p.v) v
    loc = 0.0;
    for (int j = k + 1 + tid; j < n; j += blockDim.x) loc += pb[j] * vc[j];
    double pv = block_sum(loc, red);
    for (int j = k + 1 + tid; j < n; j += blockDim.x) {
      wp[j] = pb[j] - 0.5 * t * pv * vc[j];
      vp[j] = vc[j];
    }
    prev = true;
    __syncthreads();
  }
  if (blockIdx.x == 0 && tid == 0) {
    if (n == 1) {
      d[0] = A[0];
    } else {
      int a = n - 2, b = n - 1;
      double a00 = A[(size_t)a * n + a], a10 = A[(size_t)b * n + a], a11 = A[(size_t)b * n + b];
      if (prev) {
        a00 -= 2.0 * vp[a] * wp[a];
        a10 -= vp[b] * wp[a] + wp[b] * vp[a];
        a11 -= 2.0 * vp[b] * wp[b];
      }
      d[a] = a00; d[b] = a11; e[a] = a10;
    }
  }
}

// ---- double-float tridiagonalisation (mixed path) -------------------------
// block-wide double-float sum in a fixed order; every thread gets the total.
// `scratch` holds >= 32 dfl of shared memory.
__device__ __forceinline__ dfl df_block_sum(dfl v, dfl* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = df_warp_sum(df_norm(v));
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  dfl t = (threadIdx.x < nw) ? scratch[threadIdx.x] : dfl{0.0f, 0.0f};
  if (wid == 0) t = df_warp_sum(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  dfl r = scratch[0];
  __syncthreads();
  return r;
}

__global__ void to_df_kernel(size_t len, const double* __restrict__ x, dfl* __restrict__ y) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) y[i] = df_from_double_bits(x[i]);
}

// Same reduction as tridiag_kernel (lazy rank-2 update fused with the
// matrix-vector product, one grid barrier per column), with the per-column
// critical path shortened for a kernel that is latency- rather than FP64-bound:
//  * after the barrier every block reads p_{k-1} and row k in one pass, forms
//    w_{k-1} = p - (tau/2)(p.v)v and the updated row k (x = row k of A_k);
//  * the matrix-vector product uses the unscaled x (x_{k+1} = x_1) and
//    keeps a_{i,k+1}, so it need not wait for beta, tau and the scale, which
//    thread 0 forms meanwhile:
//    p_i = tau scale (sum_j a_ij x_j - beta a_{i,k+1}) since v = scale (x - beta e_{k+1});
//  * a block's rows (i = k+1+b+rG) are cut into segments of 512 columns (256
//    and 128 once the trailing matrix is narrower than 500 and 200 columns)
//    and the (row, segment) items dealt over the warps, so the warps stay
//    balanced while the trailing matrix shrinks; warp 0, which forms the
//    reflector scalars first, takes the last item of each round, so it never
//    holds more items than another warp; each lane issues the loads of its
//    item before the arithmetic;
//  * block reductions take one CTA barrier each.
// Shared memory: PW[j] = (v_{k-1}, w_{k-1}) as one 16-byte pair (during the
// first passes it holds row k and p_{k-1}), VC[j] = x_k, then v_k, plus
// reduction scratch and the (row, segment) partial sums.
constexpr int kTriThreadsDf = 512;    // threads per block of the double-float kernel
constexpr int kDfRed = 32;
constexpr int kDfSeg = 512;           // columns per (row, segment) work item: 16 per lane
constexpr int kDfNarrow1 = 500;       // trailing width at and below which items are 256 columns
constexpr int kDfNarrow2 = 200;       // ... and 128 columns
static_assert(kTriThreadsDf / 32 <= kDfRed, "one reduction slot per warp");
// rows per block at the first column, for a grid of G blocks
static int tridiag_df_rmax(int n, int G) { return (n - 1 + G - 1) / G; }
static size_t tridiag_smem_df(int n, int G) {
  // at most 2 segments per row while the narrow items are in use
  const size_t rmax = (size_t)tridiag_df_rmax(n, G),
               smax = std::max<size_t>((size_t)(n - 1 + kDfSeg - 1) / kDfSeg, 2);
  return (3 * (size_t)n + 2 * kDfRed + rmax + rmax * smax) * sizeof(dfl);
}

// Loads of data other blocks wrote since the last grid barrier (and of rows
// this block does not own in every column) go past L1 to L2.
__device__ __forceinline__ dfl ldcg_df(const dfl* p) {
  const float2 v = __ldcg((const float2*)p);
  return dfl{v.x, v.y};
}
// read-only data of this launch (written by an earlier one): cached loads
__device__ __forceinline__ dfl ldg_df(const dfl* p) {
  const float2 v = __ldg((const float2*)p);
  return dfl{v.x, v.y};
}

// every thread gets the sum of the kTriThreadsDf / 32 warp partials (written to
// scratch[warp] by lane 0 before a CTA barrier), added as a pairwise tree
__device__ __forceinline__ dfl df_sum_partials(const dfl* scratch) {
  constexpr int NW = kTriThreadsDf / 32;
  dfl t[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) t[w] = scratch[w];
#pragma unroll
  for (int st = 1; st < NW; st <<= 1)
#pragma unroll
    for (int w = 0; w + st < NW; w += 2 * st) t[w] = df_add(t[w], t[w + st]);
  return t[0];
}

__device__ __forceinline__ dfl lo2(float4 a) { return dfl{a.x, a.y}; }
__device__ __forceinline__ dfl hi2(float4 a) { return dfl{a.z, a.w}; }
__device__ __forceinline__ float4 pack4(dfl a, dfl b) { return make_float4(a.hi, a.lo, b.hi, b.lo); }

// The fused items of column k for one block: the pending rank-2 update
// (v_{k-1}, w_{k-1}) of rows/cols >= k+1, stored back, and sum_j a_ij x_j of
// each (row, SEG-column segment) item into part[r * S + sg] (a_{i,k+1} of the
// block's rows into ak1s).  Warp w starts at item w - 1, warp 0 at NW - 1.
template <int SEG>
__device__ __forceinline__ void df_items(dfl* __restrict__ A, int n, int k, int G, int R, int wid, int lane,
                                         bool prev, const float4* PW, const dfl* VC, dfl* part, dfl* ak1s) {
  constexpr int PER = SEG / 32, NW = kTriThreadsDf / 32;
  const int S = (n - (k + 1) + SEG - 1) / SEG;
  const int Q = R * S;
  for (int q = (wid == 0) ? NW - 1 : wid - 1; q < Q; q += NW) {
    const int r = q / S, sg = q - r * S;
    const int i = k + 1 + (int)blockIdx.x + r * G;
    float2* row = (float2*)(A + (size_t)i * n);
    const int jb = k + 1 + sg * SEG + lane;
    const bool full = (k + 1 + (sg + 1) * SEG) <= n;
    dfl a0 = {0.0f, 0.0f}, a1 = {0.0f, 0.0f}, first = {0.0f, 0.0f};
    if (full) {
      float2 xr[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) xr[u] = __ldcg(row + jb + 32 * u);
      if (prev) {
        const float4 pwi = PW[i];
        const dfl vi = lo2(pwi), wi = hi2(pwi);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int j = jb + 32 * u;
          const float4 pw = PW[j];
          const dfl x = df_rank2(dfl{xr[u].x, xr[u].y}, vi, hi2(pw), wi, lo2(pw));
          row[j] = make_float2(x.hi, x.lo);
          if (u == 0) first = x;
          if (u & 1) df_acc_mul(a1, x, VC[j]); else df_acc_mul(a0, x, VC[j]);
        }
      } else {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int j = jb + 32 * u;
          const dfl x = dfl{xr[u].x, xr[u].y};
          if (u == 0) first = x;
          if (u & 1) df_acc_mul(a1, x, VC[j]); else df_acc_mul(a0, x, VC[j]);
        }
      }
    } else {
      float2 xr[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int j = jb + 32 * u;
        xr[u] = (j < n) ? __ldcg(row + j) : make_float2(0.0f, 0.0f);
      }
      const float4 pwi = prev ? PW[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const dfl vi = lo2(pwi), wi = hi2(pwi);
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int j = jb + 32 * u;
        if (j < n) {
          dfl x = dfl{xr[u].x, xr[u].y};
          if (prev) {
            const float4 pw = PW[j];
            x = df_rank2(x, vi, hi2(pw), wi, lo2(pw));
            row[j] = make_float2(x.hi, x.lo);
          }
          if (u == 0) first = x;
          if (u & 1) df_acc_mul(a1, x, VC[j]); else df_acc_mul(a0, x, VC[j]);
        }
      }
    }
    const dfl acc = df_warp_sum(df_add(df_norm(a0), df_norm(a1)));
    if (lane == 0) {
      part[r * S + sg] = acc;
      if (sg == 0) ak1s[r] = first;        // lane 0, u = 0 is column k+1
    }
  }
}

__global__ void __launch_bounds__(kTriThreadsDf) tridiag_df_kernel(int n, dfl* __restrict__ A,
                                                                 double* __restrict__ Vst,
                                                                 double* __restrict__ d,
                                                                 double* __restrict__ e,
                                                                 double* __restrict__ tau,
                                                                 dfl* __restrict__ pbuf,
                                                                 unsigned* bar, int* status, int rmax) {
  extern __shared__ float4 sm4[];
  float4* PW = sm4;                          // n pairs
  dfl* VC = (dfl*)(sm4 + n);                 // n
  dfl* redA = VC + n;                        // partials of p.v
  dfl* redB = redA + kDfRed;                 // partials of sigma
  dfl* ak1s = redB + kDfRed;                 // a_{i,k+1} of the block's rows (rmax)
  dfl* part = ak1s + rmax;                   // (row, segment) partial sums (rmax x smax)
  __shared__ dfl s_df[4];                    // beta, tau * scale, tau, scale
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int T = kTriThreadsDf, NW = kTriThreadsDf / 32;
  const int G = gridDim.x;
  dfl tau_prev = {0.0f, 0.0f};               // tau_{k-1}
  if (n == 1) {
    if (blockIdx.x == 0 && tid == 0) d[0] = df_to_double(A[0]);
    return;
  }
  for (int k = 0;; ++k) {
    const bool prev = k > 0;
    const bool last = (k == n - 2);
    const dfl* pbp = pbuf + (size_t)((k + 1) & 1) * n;   // p_{k-1}
    // pass 1: row k and p_{k-1} in one sweep of loads (kept in PW); partial p.v
    dfl loc = {0.0f, 0.0f};
#pragma unroll 4
    for (int j = k + tid; j < n; j += T) {
      const dfl a = ldcg_df(A + (size_t)k * n + j);
      dfl p = {0.0f, 0.0f};
      if (prev) {
        p = ldcg_df(pbp + j);
        df_acc_mul(loc, p, VC[j]);           // VC = v_{k-1}
      }
      PW[j] = pack4(a, p);
    }
    dfl wk = {0.0f, 0.0f}, vk = {0.0f, 0.0f}, coef = {0.0f, 0.0f};
    if (prev) {
      loc = df_warp_sum(df_norm(loc));
      if (lane == 0) redA[wid] = loc;
      __syncthreads();
      const dfl pv = df_sum_partials(redA);
      coef = df_mul(df_mul(dfl{0.5f, 0.0f}, tau_prev), pv);
      vk = VC[k];
      wk = df_sub(hi2(PW[k]), df_mul(coef, vk));   // PW[k] is not overwritten below
    }
    // pass 2: w_{k-1} and the updated row k; sigma = sum_{j >= k+2} x_j^2
    dfl sig = {0.0f, 0.0f};
    dfl dk = {0.0f, 0.0f};
    for (int j = k + tid; j < n; j += T) {
      const float4 ap = PW[j];
      dfl x = lo2(ap);
      if (prev) {
        const dfl vj = VC[j];
        const dfl wj = (j == k) ? wk : df_sub(hi2(ap), df_mul(coef, vj));
        x = df_rank2(x, vk, wj, wk, vj);
        if (j > k) PW[j] = pack4(vj, wj);
      }
      if (j == k) {
        dk = x;
      } else {
        VC[j] = x;
        if (j >= k + 2) df_acc_mul(sig, x, x);
      }
    }
    if (last) {
      __syncthreads();
      if (blockIdx.x == 0 && tid == 0) {
        const int b = n - 1;
        dfl abb = ldcg_df(A + (size_t)b * n + b);
        if (prev) abb = df_rank2(abb, lo2(PW[b]), hi2(PW[b]), hi2(PW[b]), lo2(PW[b]));
        d[n - 2] = df_to_double(dk);
        e[n - 2] = df_to_double(VC[b]);
        d[b] = df_to_double(abb);
      }
      return;
    }
    sig = df_warp_sum(df_norm(sig));
    if (lane == 0) redB[wid] = sig;
    __syncthreads();
    // thread 0: reflector scalars (double-float: GB300's FP64 divide and square
    // root are long dependent chains) while the other warps start the product
    if (tid == 0) {
      const dfl sigma = df_sum_partials(redB);
      const dfl x1 = VC[k + 1];
      dfl beta, t, scale;
      if (sigma.hi == 0.0f) {
        beta = x1; t = dfl{0.0f, 0.0f}; scale = dfl{0.0f, 0.0f};
      } else {
        const dfl nrm = df_sqrt(df_add(df_mul(x1, x1), sigma));
        beta = (x1.hi >= 0.0f) ? df_neg(nrm) : nrm;
        t = df_mul(df_sub(beta, x1), df_recip(beta));
        scale = df_recip(df_sub(x1, beta));
      }
      s_df[0] = beta;
      s_df[1] = df_mul(t, scale);
      s_df[2] = t;
      s_df[3] = scale;
      if (blockIdx.x == 0) { d[k] = df_to_double(dk); e[k] = df_to_double(beta); tau[k] = df_to_double(t); }
    }
    // fused: pending rank-2 update (v_{k-1}, w_{k-1}) of rows/cols >= k+1 and
    // sum_j a_ij x_j over (row, segment) items
    const int R = (n - (k + 1) - (int)blockIdx.x + G - 1) / G;
    const int m1 = n - (k + 1);
    const int segw = (m1 > kDfNarrow1) ? kDfSeg : ((m1 > kDfNarrow2) ? 256 : 128);
    const int S = (m1 + segw - 1) / segw;
    if (segw == kDfSeg) df_items<kDfSeg>(A, n, k, G, R, wid, lane, prev, PW, VC, part, ak1s);
    else if (segw == 256) df_items<256>(A, n, k, G, R, wid, lane, prev, PW, VC, part, ak1s);
    else df_items<128>(A, n, k, G, R, wid, lane, prev, PW, VC, part, ak1s);
    __syncthreads();
    const dfl beta_df = s_df[0], ts_df = s_df[1], scale_df = s_df[3];
    tau_prev = s_df[2];
    // p_i = tau scale (sum_j a_ij x_j - beta a_{i,k+1}), segments summed as a
    // fixed tree (one warp per row while a row has at most 32 segments)
    dfl* pb = pbuf + (size_t)(k & 1) * n;
    if (S <= 32) {
      int lpr = 1;                                  // lanes per row: power of two >= S
      while (lpr < S) lpr <<= 1;
      const int rpw = 32 / lpr;                     // rows per warp
      const int sub = lane / lpr, sl = lane - sub * lpr;
      for (int r0 = wid * rpw; r0 < R; r0 += NW * rpw) {
        const int r = r0 + sub;
        dfl v = (r < R && sl < S) ? part[r * S + sl] : dfl{0.0f, 0.0f};
        for (int o = lpr >> 1; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
        if (r < R && sl == 0) pb[k + 1 + (int)blockIdx.x + r * G] = df_mul(ts_df, df_sub(v, df_mul(beta_df, ak1s[r])));
      }
    } else {
      for (int r = tid; r < R; r += T) {
        dfl* pr = part + r * S;
        for (int st = 1; st < S; st <<= 1)
          for (int sg = 0; sg + st < S; sg += 2 * st) pr[sg] = df_add(pr[sg], pr[sg + st]);
        pb[k + 1 + (int)blockIdx.x + r * G] = df_mul(ts_df, df_sub(pr[0], df_mul(beta_df, ak1s[r])));
      }
    }
    grid_arrive(bar);
    // while the other blocks finish: v_k = scale x (v_{k+1} = 1) and the
    // reflector store row k, spread over blocks
    for (int j = k + 1 + tid; j < n; j += T) {
      const dfl v = (j == k + 1) ? dfl{1.0f, 0.0f} : df_mul(VC[j], scale_df);
      VC[j] = v;
      if (j % G == (int)blockIdx.x) Vst[(size_t)k * n + j] = df_to_double_fast(v);
    }
    if (!grid_wait(bar, (unsigned)(k + 1) * (unsigned)G, status)) return;
  }
}

// Gershgorin interval, squared off-diagonals, pivmin; one block
__global__ void gersh_kernel(int n, const double* __restrict__ d, const double* __restrict__ e,
                             double* __restrict__ e2, double* __restrict__ scal, float* __restrict__ df,
                             float* __restrict__ e2f, dfl* __restrict__ d_dfl, dfl* __restrict__ e2_dfl,
                             dfl* __restrict__ e_dfl) {
  double lo = 1e300, hi = -1e300, em = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double r = 0.0;
    df[i] = (float)d[i];                 // FP32 copies for the coarse phase (no per-step conversions)
    e2f[i] = 0.0f;
    d_dfl[i] = df_from_double(d[i]);     // double-float copies for the multisection and the
    e2_dfl[i] = dfl{0.0f, 0.0f};         // inverse iteration (mixed path)
    e_dfl[i] = (i < n - 1) ? df_from_double(e[i]) : dfl{0.0f, 0.0f};
    if (i > 0) r += fabs(e[i - 1]);
    if (i < n - 1) {
      r += fabs(e[i]);
      e2[i] = e[i] * e[i];
      e2f[i] = (float)e2[i];
      e2_dfl[i] = df_from_double(e2[i]);
      em = fmax(em, e[i] * e[i]);
    }
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
  }
  // min/max reductions through negation-free warp shuffles
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    em = fmax(em, __shfl_xor_sync(0xffffffffu, em, o));
  }
  __shared__ double slo[32], shi[32], sem[32];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { slo[w] = lo; shi[w] = hi; sem[w] = em; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 1; i < nw; ++i) { lo = fmin(lo, slo[i]); hi = fmax(hi, shi[i]); em = fmax(em, sem[i]); }
    double tn = fmax(fabs(lo), fabs(hi));
    double pivmin = 1e-290 * fmax(1.0, em);
    lo -= 4.0 * kEps * tn + 2.0 * pivmin;
    hi += 4.0 * kEps * tn + 2.0 * pivmin;
    scal[0] = lo; scal[1] = hi; scal[2] = tn; scal[3] = pivmin;
  }
}

// Number of eigenvalues of T below x: sign changes of the leading principal
// minors p_j = (d_j - x) p_{j-1} - e_{j-1}^2 p_{j-2} (Sturm sequence), kept in
// range by exact power-of-two rescaling, so each step is two FMAs and no
// division.  An exact zero minor counts as negative (the pivmin convention).
__device__ __forceinline__ int sturm_count(int n, const double* __restrict__ d,
                                           const double* __restrict__ e2, double x, double) {
  // FP64 work per step is one multiply and one FMA; signs, zero tests and the
  // rescaling test read the bit pattern with integer instructions.
  double pm = 1.0;                    // p_{j-1}
  double p = d[0] - x;                // p_0
  long long b = __double_as_longlong(p);
  int sp = (b < 0 || (b & 0x7FFFFFFFFFFFFFFFLL) == 0) ? 1 : 0;   // 1: negative (zero counts as negative)
  int c = sp;
  for (int j = 1; j < n; ++j) {
    double pn = fma(d[j] - x, p, -e2[j - 1] * pm);
    pm = p;
    p = pn;
    b = __double_as_longlong(pn);
    int zero = (b & 0x7FFFFFFFFFFFFFFFLL) == 0;
    int sn = zero ? (sp ^ 1) : (int)((unsigned long long)b >> 63);
    c += sn ^ sp;
    sp = sn;
    int ex = (int)((b >> 52) & 0x7FF);             // biased exponent of p_j
    if (ex > 1023 + 400) {
      p *= 0x1p-400; pm *= 0x1p-400;
    } else if (ex < 1023 - 400 && (int)((__double_as_longlong(pm) >> 52) & 0x7FF) < 1023 - 400) {
      p *= 0x1p400; pm *= 0x1p400;
    }
  }
  return c;
}

// FP32 Sturm count (ratio form with a pivot floor) for the coarse phase
__device__ __forceinline__ int sturm_count_f32(int n, const float* __restrict__ d,
                                               const float* __restrict__ e2, float x, float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) <= pivmin) q = -pivmin;
  int c = (q < 0.0f);
  for (int j = 1; j < n; ++j) {
    q = (d[j] - x) - e2[j - 1] / q;
    if (fabsf(q) <= pivmin) q = -pivmin;
    c += (q < 0.0f);
  }
  return c;
}

// Eigenvalue i of T: a coarse FP32 bisection down to ~2^-22 of the
// Gershgorin width, a bracket check in FP64 (widened until
// count(lo) <= i < count(hi)), then FP64 bisection to full accuracy.
__global__ void bisect_kernel(int n, const double* __restrict__ d, const double* __restrict__ e2,
                              const double* __restrict__ scal, const float* __restrict__ df,
                              const float* __restrict__ e2f, double rel_tol, double* __restrict__ ev) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double glo = scal[0], ghi = scal[1], pivmin = scal[3];
  const double width = ghi - glo;
  // coarse phase (FP32)
  float lo32 = (float)glo, hi32 = (float)ghi;
  const float piv32 = fmaxf((float)(1e-30 * fmax(1.0, width)), 1e-30f);
  for (int it = 0; it < 22; ++it) {
    float mid = 0.5f * (lo32 + hi32);
    if (sturm_count_f32(n, df, e2f, mid, piv32) > i) hi32 = mid; else lo32 = mid;
  }
  // bracket check in FP64, widening geometrically if the FP32 counts erred
  double w = fmax((double)hi32 - (double)lo32, 1e-12 * width);
  double lo = (double)lo32 - w, hi = (double)hi32 + w;
  for (int k = 0; k < 60; ++k) {
    bool ok_lo = (lo <= glo) || sturm_count(n, d, e2, lo, pivmin) <= i;
    bool ok_hi = (hi >= ghi) || sturm_count(n, d, e2, hi, pivmin) > i;
    if (ok_lo && ok_hi) break;
    w *= 4.0;
    if (!ok_lo) lo = fmax(glo, lo - w);
    if (!ok_hi) hi = fmin(ghi, hi + w);
  }
  // rel_tol (1e-12) of the spectral range is far below what the occupations and
  // the DMPT weights resolve, and inverse iteration converges from such a shift
  // in two steps.  A looser shift costs orthogonality: after two steps the
  // component along a neighbour at distance g is ~(shift error / g)^2, which at
  // 1e-9 of the range left Q^T Q - I at 5e-7 for n = 3360.
  const double tol = fmax(2.0 * kEps * fmax(fabs(lo), fabs(hi)), rel_tol * fmax(1.0, scal[2])) + pivmin;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (hi - lo <= tol) break;
    if (sturm_count(n, d, e2, mid, pivmin) > i) hi = mid; else lo = mid;
  }
  ev[i] = 0.5 * (lo + hi);
}

// Mixed path: eigenvalue i by multisection in double-float arithmetic.  A
// group of kMsLanes lanes evaluates the Sturm count at kMsLanes interior
// points of the current interval, which shrinks (kMsLanes + 1)-fold per round;
// every group starts from the Gershgorin interval, so all groups take the same
// number of rounds.  The count is the product form of sturm_count on the FP32
// pipe (about 48-bit arithmetic), kept in range by exact power-of-two scaling.
constexpr int kMsLanes = 8;

__device__ __forceinline__ int sturm_count_df(int n, const dfl* __restrict__ d, const dfl* __restrict__ e2,
                                              dfl x) {
  dfl pm = {1.0f, 0.0f};
  dfl p = df_sub(ldg_df(d), x);
  int sp = (p.hi < 0.0f || p.hi == 0.0f) ? 1 : 0;        // zero counts as negative
  int c = sp;
#pragma unroll 4
  for (int j = 1; j < n; ++j) {
    const dfl dj = ldg_df(d + j), ej = ldg_df(e2 + j - 1);
    const dfl pn = df_sub(df_mul(df_sub(dj, x), p), df_mul(ej, pm));
    const int sn = (pn.hi == 0.0f) ? (sp ^ 1) : (int)(__float_as_uint(pn.hi) >> 31);
    c += sn ^ sp;
    sp = sn;
    // keep |p| within [2^-32, 2^32] (both p and pm scale by the same power of two)
    const int ex = (int)((__float_as_uint(pn.hi) >> 23) & 0xFF);
    const float sc = (ex > 127 + 32) ? 0x1p-64f : ((ex < 127 - 32) ? 0x1p+64f : 1.0f);
    pm = dfl{KX_FMUL(p.hi, sc), KX_FMUL(p.lo, sc)};
    p = dfl{KX_FMUL(pn.hi, sc), KX_FMUL(pn.lo, sc)};
  }
  return c;
}

__global__ void bisect_df_kernel(int n, const dfl* __restrict__ d, const dfl* __restrict__ e2,
                                 const double* __restrict__ scal, double rel_tol, double* __restrict__ ev) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / kMsLanes;                 // eigenvalue of this group
  const int m = t % kMsLanes;                 // point m + 1 of the group
  const int gbase = (threadIdx.x & 31) & ~(kMsLanes - 1);
  const bool live = i < n;                    // whole groups are live or not (n * kMsLanes threads)
  const double glo = scal[0], ghi = scal[1], pivmin = scal[3];
  double lo = glo, hi = ghi;
  const double tol = fmax(2.0 * kEps * fmax(fabs(glo), fabs(ghi)), rel_tol * fmax(1.0, scal[2])) + pivmin;
  int rounds = 0;
  for (double w = ghi - glo; w > tol && rounds < 64; w /= (double)(kMsLanes + 1)) ++rounds;
  for (int r = 0; r < rounds; ++r) {
    const double h = (hi - lo) / (double)(kMsLanes + 1);
    const double x = lo + (double)(m + 1) * h;
    const bool above = live && sturm_count_df(n, d, e2, df_from_double(x)) > i;
    const unsigned bal = __ballot_sync(0xffffffffu, above);
    const unsigned g = (bal >> gbase) & ((1u << kMsLanes) - 1u);
    // counts grow with x: the first point with count > i is the new upper end
    const int f = g ? (__ffs(g) - 1) : kMsLanes;      // 0-based point index, kMsLanes: none
    const double nlo = (f == 0) ? lo : lo + (double)f * h;
    const double nhi = (f == kMsLanes) ? hi : lo + (double)(f + 1) * h;
    lo = nlo;
    hi = nhi;
  }
  if (live && m == 0) ev[i] = 0.5 * (lo + hi);
}

__global__ void cluster_kernel(int n, const double* __restrict__ ev, const double* __restrict__ scal,
                               int* __restrict__ clus) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ctol = 1e-7 * fmax(1.0, scal[2]);
  // a NaN gap starts a new cluster: non-finite input must not merge the whole
  // spectrum into one cluster (one thread would then orthogonalise n vectors)
  clus[i] = (i == 0 || !(ev[i] - ev[i - 1] <= ctol)) ? 1 : 0;
}

__device__ __forceinline__ unsigned start_hash(int row, int col) {
  unsigned h = (unsigned)row * 0x9E3779B1u ^ ((unsigned)col * 0x85EBCA77u + 0x165667B1u);
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return h;
}
__device__ __forceinline__ double start_value(int row, int col) {
  return ((double)(start_hash(row, col) & 0xFFFFF) / 524288.0) - 1.0 + 1e-3;
}
// the same pseudo-random start entry in FP32 arithmetic (a start vector only
// needs a component along the eigenvector, not FP64 values)
__device__ __forceinline__ float start_value_f(int row, int col) {
  return __fadd_rn(__fmul_rn((float)(start_hash(row, col) & 0xFFFFF), 0x1p-19f), -0.999f);
}

// inverse iteration; one thread per cluster leader; lu: 5 x n x n workspace.
// The recurrences carry their running values in registers, and the loads of
// each sweep are issued kIvB rows at a time ahead of the dependent arithmetic
// (one thread walks n rows of a column: a load-use chain per row would put
// the memory latency on the critical path n times); the arithmetic and its
// order are those of the textbook pivoted tridiagonal LU and its
// forward/backward substitutions.
constexpr int kIvB = 8;

__global__ void invit_kernel(int n, const double* __restrict__ d, const double* __restrict__ e,
                             const double* __restrict__ ev, const double* __restrict__ scal,
                             const int* __restrict__ clus, double* __restrict__ lu,
                             double* __restrict__ Z) {
  int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= n || !clus[L]) return;
  int end = L + 1;
  while (end < n && !clus[end]) ++end;
  const double tn = fmax(scal[2], 1e-300);
  const double tiny = kEps * tn;
  const size_t nn = (size_t)n * n;
  double* __restrict__ dl = lu + 0 * nn;
  double* __restrict__ rdd = lu + 1 * nn;   // reciprocal pivots
  double* __restrict__ du = lu + 2 * nn;
  double* __restrict__ du2 = lu + 3 * nn;
  double* __restrict__ pv = lu + 4 * nn;
#define LU(a, r) a[(size_t)(r) * n + L]
#define ZC(r, c) Z[(size_t)(r) * n + (c)]
  double prevlam = 0.0;
  for (int j = L; j < end; ++j) {
    double lam = ev[j];
    if (j > L && lam - prevlam < 10.0 * tiny) lam = prevlam + 10.0 * tiny;
    prevlam = lam;
    if (n == 1) { ZC(0, j) = 1.0; continue; }
    // LU of T - lam I with partial pivoting; a, u: pivot-row diagonal and superdiagonal
    double a = d[0] - lam, u = e[0];
    for (int r = 0; r < n - 1; ++r) {
      const double b = e[r];
      const double dn = d[r + 1] - lam;
      const double un = (r < n - 2) ? e[r + 1] : 0.0;
      if (fabs(a) >= fabs(b)) {
        LU(pv, r) = 0.0;
        if (fabs(a) < tiny) a = (a >= 0.0) ? tiny : -tiny;
        const double ra = 1.0 / a;          // one division per row (the FP64 divide is slow)
        const double f = b * ra;
        LU(dl, r) = f;
        LU(rdd, r) = ra;
        LU(du, r) = u;
        LU(du2, r) = 0.0;
        a = dn - f * u;
        u = un;
      } else {
        LU(pv, r) = 1.0;
        const double rb = 1.0 / b;
        const double f = a * rb;
        LU(rdd, r) = rb;
        LU(dl, r) = f;
        LU(du, r) = dn;
        const double na = u - f * dn;
        if (r < n - 2) {
          LU(du2, r) = un;
          u = -f * un;
        } else {
          LU(du2, r) = 0.0;
        }
        a = na;
      }
    }
    if (fabs(a) < tiny) a = (a >= 0.0) ? tiny : -tiny;
    LU(rdd, n - 1) = 1.0 / a;
    for (int r = 0; r < n; ++r) ZC(r, j) = start_value(r, j);
    for (int it = 0; it < 2; ++it) {
      // forward (L with pivots); cur = current row r of the right-hand side
      double cur = ZC(0, j);
      for (int r0 = 0; r0 < n - 1; r0 += kIvB) {
        double nx[kIvB], fv[kIvB], pf[kIvB];
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 + q;
          if (r < n - 1) { nx[q] = ZC(r + 1, j); fv[q] = LU(dl, r); pf[q] = LU(pv, r); }
        }
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 + q;
          if (r < n - 1) {
            if (pf[q] == 0.0) {
              ZC(r, j) = cur;
              cur = nx[q] - fv[q] * cur;
            } else {
              ZC(r, j) = nx[q];
              cur = cur - fv[q] * nx[q];
            }
          }
        }
      }
      // backward (U, three diagonals, reciprocal pivots); z1 = x[r+1], z2 = x[r+2]
      double z2 = cur * LU(rdd, n - 1);
      ZC(n - 1, j) = z2;
      double z1 = z2;
      if (n > 1) {
        z1 = (ZC(n - 2, j) - LU(du, n - 2) * z2) * LU(rdd, n - 2);
        ZC(n - 2, j) = z1;
      }
      for (int r0 = n - 3; r0 >= 0; r0 -= kIvB) {
        double zv[kIvB], uv[kIvB], u2[kIvB], rv[kIvB];
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 - q;
          if (r >= 0) { zv[q] = ZC(r, j); uv[q] = LU(du, r); u2[q] = LU(du2, r); rv[q] = LU(rdd, r); }
        }
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 - q;
          if (r >= 0) {
            const double x = (zv[q] - uv[q] * z1 - u2[q] * z2) * rv[q];
            ZC(r, j) = x;
            z2 = z1;
            z1 = x;
          }
        }
      }
      // scale, re-orthogonalise within the cluster, normalise
      double mx = 0.0;
#pragma unroll 8
      for (int r = 0; r < n; ++r) mx = fmax(mx, fabs(ZC(r, j)));
      double s = (mx > 0.0) ? 1.0 / mx : 1.0;
#pragma unroll 8
      for (int r = 0; r < n; ++r) ZC(r, j) *= s;
      for (int c = L; c < j; ++c) {
        double dot = 0.0;
#pragma unroll 8
        for (int r = 0; r < n; ++r) dot += ZC(r, c) * ZC(r, j);
#pragma unroll 8
        for (int r = 0; r < n; ++r) ZC(r, j) -= dot * ZC(r, c);
      }
      double nrm = 0.0;
#pragma unroll 8
      for (int r = 0; r < n; ++r) nrm += ZC(r, j) * ZC(r, j);
      nrm = ::sqrt(nrm);
      s = (nrm > 0.0) ? 1.0 / nrm : 0.0;
#pragma unroll 8
      for (int r = 0; r < n; ++r) ZC(r, j) *= s;
    }
  }
#undef LU
#undef ZC
}

// Mixed path: the same inverse iteration in double-float arithmetic.  The LU
// factors and the iterates are held as (hi, lo) pairs in the same workspace
// (the iterates in Q, converted to FP64 at the end); one reciprocal per row
// from the FP32 estimate and one Newton step; the pivot floor and the shift
// separation use the double-float unit 2^-46 |T| instead of the FP64 epsilon.
__device__ __forceinline__ float df_abs_hi(dfl a) { return fabsf(a.hi); }

// Each cluster leader runs its recurrences alone, so the kernel is bound by
// their latency: kIvLanes active lanes per 32-thread block spread the n
// chains over n / kIvLanes warps (about 5 per SM at n = 3360 instead of
// one), so each SM interleaves several independent chains; four lanes keep
// every access a whole 32-byte sector and limit divergence at the pivots.
constexpr int kIvLanes = 4;
__global__ void __launch_bounds__(32) invit_df_kernel(int n, const dfl* __restrict__ d, const double* __restrict__ e,
                                                    const dfl* __restrict__ edf,
                                                    const double* __restrict__ ev, const double* __restrict__ scal,
                                                    const int* __restrict__ clus, dfl* __restrict__ lu,
                                                    double* __restrict__ Zout) {
  if (threadIdx.x >= kIvLanes) return;
  int L = blockIdx.x * kIvLanes + threadIdx.x;
  if (L >= n || !clus[L]) return;
  int end = L + 1;
  while (end < n && !clus[end]) ++end;
  const double tn = fmax(scal[2], 1e-300);
  const double tiny_d = 0x1p-46 * tn;
  const dfl tiny = df_from_double(tiny_d);
  const size_t nn = (size_t)n * n;
  dfl* __restrict__ dl = lu + 0 * nn;
  dfl* __restrict__ rdd = lu + 1 * nn;   // reciprocal pivots
  dfl* __restrict__ du = lu + 2 * nn;
  dfl* __restrict__ du2 = lu + 3 * nn;
  int* __restrict__ pv = (int*)(lu + 4 * nn);
  dfl* __restrict__ Z = (dfl*)Zout;      // iterates in place of the FP64 output
#define LU(a, r) a[(size_t)(r) * n + L]
#define ZC(r, c) Z[(size_t)(r) * n + (c)]
  if (end == L + 1 && n > 1) {
    // An eigenvalue alone in its cluster (the common case): the same two
    // inverse-iteration steps with the passes fused.  Step 1 solves from the
    // start vector without storing it, its backward sweep tracks max|x|;
    // step 2 reads x scaled by 1/max (inverse iteration is linear, the scale
    // only keeps the values in range), its backward sweep accumulates ||x||^2;
    // one last pass writes x / ||x|| in FP64.  Six sweeps of n instead of 15.
    // no FP64 instruction per row: GB300 issues one FP64 warp instruction per
    // ~76 cycles per scheduler, which would put the FP64 pipe on the chain
    const dfl lam = df_from_double(ev[L]);
    dfl a = df_sub(ldg_df(d), lam), u = ldg_df(edf);
    for (int r = 0; r < n - 1; ++r) {
      const dfl b = ldg_df(edf + r);
      const dfl dn = df_sub(ldg_df(d + r + 1), lam);
      const dfl un = (r < n - 2) ? ldg_df(edf + r + 1) : dfl{0.0f, 0.0f};
      if (df_abs_hi(a) >= df_abs_hi(b)) {
        LU(pv, r) = 0;
        if (df_abs_hi(a) < tiny.hi) a = (a.hi >= 0.0f) ? tiny : df_neg(tiny);
        const dfl ra = df_recip(a);
        const dfl f = df_mul(b, ra);
        LU(dl, r) = f;
        LU(rdd, r) = ra;
        LU(du, r) = u;
        LU(du2, r) = dfl{0.0f, 0.0f};
        a = df_sub(dn, df_mul(f, u));
        u = un;
      } else {
        LU(pv, r) = 1;
        const dfl rb = df_recip(b);
        const dfl f = df_mul(a, rb);
        LU(rdd, r) = rb;
        LU(dl, r) = f;
        LU(du, r) = dn;
        const dfl na = df_sub(u, df_mul(f, dn));
        if (r < n - 2) {
          LU(du2, r) = un;
          u = df_neg(df_mul(f, un));
        } else {
          LU(du2, r) = dfl{0.0f, 0.0f};
        }
        a = na;
      }
    }
    if (df_abs_hi(a) < tiny.hi) a = (a.hi >= 0.0f) ? tiny : df_neg(tiny);
    LU(rdd, n - 1) = df_recip(a);
    dfl scl = {1.0f, 0.0f};
    dfl nrm = {0.0f, 0.0f};
    for (int it = 0; it < 2; ++it) {
      // forward (L with pivots); step 1 takes the start vector, step 2 the scaled x
      dfl cur = (it == 0) ? dfl{start_value_f(0, L), 0.0f} : df_mul(ZC(0, L), scl);
      for (int r0 = 0; r0 < n - 1; r0 += kIvB) {
        dfl nx[kIvB], fv[kIvB];
        int pf[kIvB];
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 + q;
          if (r < n - 1) {
            nx[q] = (it == 0) ? dfl{start_value_f(r + 1, L), 0.0f} : df_mul(ZC(r + 1, L), scl);
            fv[q] = LU(dl, r);
            pf[q] = LU(pv, r);
          }
        }
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 + q;
          if (r < n - 1) {
            if (pf[q] == 0) {
              ZC(r, L) = cur;
              cur = df_sub(nx[q], df_mul(fv[q], cur));
            } else {
              ZC(r, L) = nx[q];
              cur = df_sub(cur, df_mul(fv[q], nx[q]));
            }
          }
        }
      }
      // backward (U, three diagonals, reciprocal pivots), with max|x| or ||x||^2
      float mx = 0.0f;
      dfl z2 = df_mul(cur, LU(rdd, n - 1));
      ZC(n - 1, L) = z2;
      mx = fmaxf(mx, df_abs_hi(z2));
      if (it == 1) df_acc_mul(nrm, z2, z2);
      dfl z1 = z2;
      if (n > 1) {
        z1 = df_mul(df_sub(ZC(n - 2, L), df_mul(LU(du, n - 2), z2)), LU(rdd, n - 2));
        ZC(n - 2, L) = z1;
        mx = fmaxf(mx, df_abs_hi(z1));
        if (it == 1) df_acc_mul(nrm, z1, z1);
      }
      for (int r0 = n - 3; r0 >= 0; r0 -= kIvB) {
        dfl zv[kIvB], uv[kIvB], u2[kIvB], rv[kIvB];
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 - q;
          if (r >= 0) { zv[q] = ZC(r, L); uv[q] = LU(du, r); u2[q] = LU(du2, r); rv[q] = LU(rdd, r); }
        }
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 - q;
          if (r >= 0) {
            const dfl x = df_mul(df_sub(df_sub(zv[q], df_mul(uv[q], z1)), df_mul(u2[q], z2)), rv[q]);
            ZC(r, L) = x;
            mx = fmaxf(mx, df_abs_hi(x));
            if (it == 1) df_acc_mul(nrm, x, x);
            z2 = z1;
            z1 = x;
          }
        }
      }
      if (it == 0) scl = (mx > 0.0f) ? df_recip(dfl{mx, 0.0f}) : dfl{1.0f, 0.0f};
    }
    const double nd = ::sqrt(df_to_double(df_norm(nrm)));
    const dfl sc = (nd > 0.0) ? df_from_double(1.0 / nd) : dfl{0.0f, 0.0f};
#pragma unroll 8
    for (int r = 0; r < n; ++r) {
      const dfl z = df_mul(ZC(r, L), sc);
      Zout[(size_t)r * n + L] = df_to_double_fast(z);
    }
    return;
  }
  double prevlam = 0.0;
  for (int j = L; j < end; ++j) {
    double lamd = ev[j];
    if (j > L && lamd - prevlam < 10.0 * tiny_d) lamd = prevlam + 10.0 * tiny_d;
    prevlam = lamd;
    if (n == 1) { ZC(0, j) = dfl{1.0f, 0.0f}; continue; }
    const dfl lam = df_from_double(lamd);
    // LU of T - lam I with partial pivoting; a, u: pivot-row diagonal and superdiagonal
    dfl a = df_sub(ldg_df(d), lam), u = df_from_double(e[0]);
    for (int r = 0; r < n - 1; ++r) {
      const dfl b = df_from_double(e[r]);
      const dfl dn = df_sub(ldg_df(d + r + 1), lam);
      const dfl un = (r < n - 2) ? df_from_double(e[r + 1]) : dfl{0.0f, 0.0f};
      if (df_abs_hi(a) >= df_abs_hi(b)) {
        LU(pv, r) = 0;
        if (df_abs_hi(a) < tiny.hi) a = (a.hi >= 0.0f) ? tiny : df_neg(tiny);
        const dfl ra = df_recip(a);
        const dfl f = df_mul(b, ra);
        LU(dl, r) = f;
        LU(rdd, r) = ra;
        LU(du, r) = u;
        LU(du2, r) = dfl{0.0f, 0.0f};
        a = df_sub(dn, df_mul(f, u));
        u = un;
      } else {
        LU(pv, r) = 1;
        const dfl rb = df_recip(b);
        const dfl f = df_mul(a, rb);
        LU(rdd, r) = rb;
        LU(dl, r) = f;
        LU(du, r) = dn;
        const dfl na = df_sub(u, df_mul(f, dn));
        if (r < n - 2) {
          LU(du2, r) = un;
          u = df_neg(df_mul(f, un));
        } else {
          LU(du2, r) = dfl{0.0f, 0.0f};
        }
        a = na;
      }
    }
    if (df_abs_hi(a) < tiny.hi) a = (a.hi >= 0.0f) ? tiny : df_neg(tiny);
    LU(rdd, n - 1) = df_recip(a);
    for (int r = 0; r < n; ++r) ZC(r, j) = df_from_double(start_value(r, j));
    for (int it = 0; it < 2; ++it) {
      // forward (L with pivots)
      dfl cur = ZC(0, j);
      for (int r0 = 0; r0 < n - 1; r0 += kIvB) {
        dfl nx[kIvB], fv[kIvB];
        int pf[kIvB];
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 + q;
          if (r < n - 1) { nx[q] = ZC(r + 1, j); fv[q] = LU(dl, r); pf[q] = LU(pv, r); }
        }
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 + q;
          if (r < n - 1) {
            if (pf[q] == 0) {
              ZC(r, j) = cur;
              cur = df_sub(nx[q], df_mul(fv[q], cur));
            } else {
              ZC(r, j) = nx[q];
              cur = df_sub(cur, df_mul(fv[q], nx[q]));
            }
          }
        }
      }
      // backward (U, three diagonals, reciprocal pivots)
      dfl z2 = df_mul(cur, LU(rdd, n - 1));
      ZC(n - 1, j) = z2;
      dfl z1 = z2;
      if (n > 1) {
        z1 = df_mul(df_sub(ZC(n - 2, j), df_mul(LU(du, n - 2), z2)), LU(rdd, n - 2));
        ZC(n - 2, j) = z1;
      }
      for (int r0 = n - 3; r0 >= 0; r0 -= kIvB) {
        dfl zv[kIvB], uv[kIvB], u2[kIvB], rv[kIvB];
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 - q;
          if (r >= 0) { zv[q] = ZC(r, j); uv[q] = LU(du, r); u2[q] = LU(du2, r); rv[q] = LU(rdd, r); }
        }
#pragma unroll
        for (int q = 0; q < kIvB; ++q) {
          const int r = r0 - q;
          if (r >= 0) {
            const dfl x = df_mul(df_sub(df_sub(zv[q], df_mul(uv[q], z1)), df_mul(u2[q], z2)), rv[q]);
            ZC(r, j) = x;
            z2 = z1;
            z1 = x;
          }
        }
      }
      // scale, re-orthogonalise within the cluster, normalise
      float mx = 0.0f;
#pragma unroll 8
      for (int r = 0; r < n; ++r) mx = fmaxf(mx, df_abs_hi(ZC(r, j)));
      dfl sc = (mx > 0.0f) ? df_recip(dfl{mx, 0.0f}) : dfl{1.0f, 0.0f};
#pragma unroll 8
      for (int r = 0; r < n; ++r) ZC(r, j) = df_mul(ZC(r, j), sc);
      for (int c = L; c < j; ++c) {
        dfl dot = {0.0f, 0.0f};
#pragma unroll 8
        for (int r = 0; r < n; ++r) df_acc_mul(dot, ZC(r, c), ZC(r, j));
        dot = df_norm(dot);
#pragma unroll 8
        for (int r = 0; r < n; ++r) ZC(r, j) = df_sub(ZC(r, j), df_mul(dot, ZC(r, c)));
      }
      dfl nrm = {0.0f, 0.0f};
#pragma unroll 8
      for (int r = 0; r < n; ++r) df_acc_mul(nrm, ZC(r, j), ZC(r, j));
      const double nd = ::sqrt(df_to_double(df_norm(nrm)));
      sc = (nd > 0.0) ? df_from_double(1.0 / nd) : dfl{0.0f, 0.0f};
#pragma unroll 8
      for (int r = 0; r < n; ++r) ZC(r, j) = df_mul(ZC(r, j), sc);
    }
  }
  // FP64 output (same slots, same thread)
  for (int j = L; j < end; ++j)
    for (int r = 0; r < n; ++r) {
      const dfl z = ZC(r, j);
      Zout[(size_t)r * n + j] = df_to_double_fast(z);
    }
#undef LU
#undef ZC
}

// T factor of a block of kb reflectors (forward, columnwise): one block,
// T held in shared memory, each entry a dot product split over 4 partial sums
__device__ void tfactor_body(int kb, const double* __restrict__ tau, const double* __restrict__ G, int ldg,
                             double* __restrict__ T, int ldt) {
  extern __shared__ double ts[];          // kb x kb
  __shared__ double gcol[kBtBlockTc];
  const int i = threadIdx.x;
  for (int e = i; e < kb * kb; e += blockDim.x) ts[e] = 0.0;
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (i < j) gcol[i] = G[i * ldg + j];
    __syncthreads();
    if (i < j) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int l = i;
      for (; l + 3 < j; l += 4) {
        a0 = fma(ts[i * kb + l], gcol[l], a0);
        a1 = fma(ts[i * kb + l + 1], gcol[l + 1], a1);
        a2 = fma(ts[i * kb + l + 2], gcol[l + 2], a2);
        a3 = fma(ts[i * kb + l + 3], gcol[l + 3], a3);
      }
      for (; l < j; ++l) a0 = fma(ts[i * kb + l], gcol[l], a0);
      ts[i * kb + j] = -tau[j] * ((a0 + a1) + (a2 + a3));
    }
    if (i == j) ts[j * kb + j] = tau[j];
    __syncthreads();
  }
  for (int e = i; e < kb * kb; e += blockDim.x) T[(e / kb) * ldt + e % kb] = ts[e];
}

__global__ void tfactor_kernel(int kb, const double* __restrict__ tau, const double* __restrict__ G,
                               int ldg, double* __restrict__ T, int ldt) {
  tfactor_body(kb, tau, G, ldg, T, ldt);
}

// T factors of every block of kblk reflectors at once (block b: reflectors
// b*kblk .. ; they depend on the reflectors only, not on the vectors updated)
__global__ void tfactor_all_kernel(int nref, int kblk, const double* __restrict__ tau,
                                   const double* __restrict__ Gall, double* __restrict__ Tall) {
  const int b = blockIdx.x;
  const int k0 = b * kblk;
  const int kb = (k0 + kblk < nref) ? kblk : nref - k0;
  const size_t off = (size_t)b * kblk * kblk;
  tfactor_body(kb, tau + k0, Gall + off, kblk, Tall + off, kblk);
}

// number of blocks of kBtBlockTc reflectors (n - 2 reflectors)
static int tc_blocks(int n) { return n > 2 ? (n - 2 + kBtBlockTc - 1) / kBtBlockTc : 1; }

struct BtScratch;
static size_t bt_scratch_layout(int n, void* base, BtScratch* out);
// the inverse-iteration workspace (5 n^2) also serves as back-transformation scratch
static size_t lu_doubles(int n) {
  const size_t a = 5 * (size_t)n * n;
  const size_t b = (bt_scratch_layout(n, nullptr, nullptr) + 7) / 8;
  return a > b ? a : b;
}

// One layout for sizing and binding.  Every buffer starts on a 256-byte
// boundary: the back-transformation cuts BF16 slices into the lu region and
// hands them to TMA, whose tensor maps need 16-byte aligned bases (with odd n
// an unpadded layout would leave the region 8 bytes off).
static size_t eig_layout(int n, void* base, EigWork* w) {
  const size_t nn = (size_t)n * n;
  size_t off = 0;
  auto take = [&](size_t doubles) {
    double* q = base ? (double*)base + off : nullptr;
    off += (doubles + 31) & ~(size_t)31;
    return q;
  };
  double* A = take(nn);
  double* Vst = take(nn);
  double* d = take(n);
  double* e = take(n);
  double* e2 = take(n);
  double* tau = take(n);
  double* pbuf = take(4 * (size_t)n);
  double* lu = take(lu_doubles(n));
  double* Tm = take((size_t)tc_blocks(n) * kBtBlockTc * kBtBlockTc);   // T and Gram of every reflector block
  double* Gm = take((size_t)tc_blocks(n) * kBtBlockTc * kBtBlockTc);
  double* Wt = take((size_t)kBtBlockTc * n);
  double* Wt2 = take((size_t)kBtBlockTc * n);
  double* scal = take(16);
  double* bar = take(8);
  double* clus = take(((size_t)n * sizeof(int) + 7) / 8);
  if (w) {
    w->A = A; w->Vst = Vst; w->d = d; w->e = e; w->e2 = e2; w->tau = tau; w->pbuf = pbuf; w->lu = lu;
    w->Tm = Tm; w->Gm = Gm; w->Wt = Wt; w->Wt2 = Wt2; w->scal = scal;
    w->bar = (unsigned*)bar;
    w->clus = (int*)clus;
  }
  return off * sizeof(double) + 256;
}

size_t eig_work_bytes(int n) { return eig_layout(n, nullptr, nullptr); }

// base must be 256-byte aligned (arena allocations are)
void eig_work_bind(EigWork& w, void* base, int n) { eig_layout(n, base, &w); }

// About 64K (FP64 kernel) or 32K (double-float kernel, whose columns cost
// less arithmetic and more latency) elements of the initial matrix per block,
// at most one block per SM; small systems keep small grids, so that many of
// them fit on the device at once (molecule batches, serving).
static int tridiag_blocks(int n, int sm_count, bool df) {
  const int sh = df ? 15 : 16;
  long long work = ((long long)n * n + (1LL << sh) - 1) >> sh;
  int blocks = (int)work;
  if (blocks < 1) blocks = 1;
  if (blocks > sm_count) blocks = sm_count;           // one block per SM (two were slower)
  return blocks;
}

static size_t tridiag_smem(int n) { return (3 * (size_t)n + 32) * sizeof(double); }

// raise the kernel's opt-in dynamic shared memory monotonically, per device
// (the attribute belongs to the device that is current; thread-safe)
static bool tridiag_smem_attribute(size_t smem, bool df) {
  if (smem <= 48 * 1024) return true;
  static std::mutex mu;
  static size_t smem_set[2][kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  std::lock_guard<std::mutex> lk(mu);
  if (smem > smem_set[df][dev]) {
    const void* fn = df ? (const void*)tridiag_df_kernel : (const void*)tridiag_kernel;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    smem_set[df][dev] = smem;
  }
  return true;
}

// (the larger share of the FP64 and the double-float kernel)
int eig_set_barrier_limit(unsigned long long ns) {
  return cudaMemcpyToSymbol(g_barrier_ns, &ns, sizeof(ns)) == cudaSuccess ? 0 : -1;
}

int eig_tridiag_weight(int n, int sm_count) {
  if (n <= 0) return 0;
  int weight = 0;
  for (int df = 0; df < 2; ++df) {
    int p = 0;
    const long long b = tridiag_blocks(n, sm_count, df != 0);
    const size_t smem = df ? tridiag_smem_df(n, (int)b) : tridiag_smem(n);
    const void* fn = df ? (const void*)tridiag_df_kernel : (const void*)tridiag_kernel;
    if (!tridiag_smem_attribute(smem, df != 0) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, fn, df ? kTriThreadsDf : kTriThreads, smem) !=
            cudaSuccess ||
        p < 1) {
      cudaGetLastError();
      p = 1;
    }
    const int wgt = (int)((1000LL * b + p - 1) / p);
    weight = (wgt > weight) ? wgt : weight;
  }
  return weight;
}

int eig_tridiagonalize(cudaStream_t s, int n, const double* F, EigWork& w, int* status, int sm_count, bool df) {
  if (n <= 0) return 0;
  const size_t nn2 = (size_t)n * n;
  if (df) {
    // the workspace holds n x n (hi, lo) pairs: the same bytes as n x n doubles
    to_df_kernel<<<(unsigned)((nn2 + 255) / 256), 256, 0, s>>>(nn2, F, (dfl*)w.A);
    count_launch();
  } else {
    cudaMemcpyAsync(w.A, F, nn2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s);
  cudaMemsetAsync(w.e, 0, (size_t)n * sizeof(double), s);
  // 1. tridiagonalisation
  int blocks = tridiag_blocks(n, sm_count, df);
  size_t smem = df ? tridiag_smem_df(n, blocks) : tridiag_smem(n);
  if (!tridiag_smem_attribute(smem, df)) return -1;
  if (df) cudaMemsetAsync(w.Vst, 0, nn2 * sizeof(double), s);   // entries left of the reflectors
  int nn = n;
  double *A = w.A, *V = w.Vst, *d = w.d, *e = w.e, *t = w.tau, *pb = w.pbuf;
  unsigned* bar = w.bar;
  int* st = status;
  int rmax = tridiag_df_rmax(n, blocks);
  void* args_fp64[] = {&nn, &A, &V, &d, &e, &t, &pb, &bar, &st};
  void* args_df[] = {&nn, &A, &V, &d, &e, &t, &pb, &bar, &st, &rmax};
  void** args = df ? args_df : args_fp64;
  const void* fn = df ? (const void*)tridiag_df_kernel : (const void*)tridiag_kernel;
  if (cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(df ? kTriThreadsDf : kTriThreads), args, smem, s) !=
      cudaSuccess)
    return -2;
  count_launch();
  return 0;
}

void eig_bisect(cudaStream_t s, int n, double* eps, EigWork& w, double rel_tol, bool df_path) {
  if (n <= 0) return;
  // 2. eigenvalues
  // pbuf (4n doubles, free after the tridiagonalisation) holds the FP32 and double-float copies
  float* df = (float*)w.pbuf;
  float* e2f = df + n;
  dfl* d_dfl = (dfl*)(w.pbuf + n);
  dfl* e2_dfl = d_dfl + n;
  dfl* e_dfl = e2_dfl + n;
  gersh_kernel<<<1, 1024, 0, s>>>(n, w.d, w.e, w.e2, w.scal, df, e2f, d_dfl, e2_dfl, e_dfl);
  count_launch();
  if (df_path) {
    const long long thr = (long long)n * kMsLanes;
    // one warp (4 eigenvalues) per block, so the n / 4 blocks spread over all SMs
    bisect_df_kernel<<<(unsigned)((thr + 31) / 32), 32, 0, s>>>(n, d_dfl, e2_dfl, w.scal, rel_tol, eps);
  } else {
    bisect_kernel<<<(n + 31) / 32, 32, 0, s>>>(n, w.d, w.e2, w.scal, df, e2f, rel_tol, eps);   // spread over all SMs
  }
  count_launch();
}

void eig_vectors(cudaStream_t s, int n, const double* eps, double* Q, EigWork& w, bool df_path) {
  if (n <= 0) return;
  // 3. eigenvectors of the tridiagonal matrix
  cluster_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, eps, w.scal, w.clus);
  count_launch();
  if (df_path) {
    const dfl* d_dfl = (const dfl*)(w.pbuf + n);     // written by eig_bisect
    const dfl* e_dfl = d_dfl + 2 * (size_t)n;
    invit_df_kernel<<<(n + kIvLanes - 1) / kIvLanes, 32, 0, s>>>(n, d_dfl, w.e, e_dfl, eps, w.scal, w.clus,
                                                                (dfl*)w.lu, Q);
  } else {
    invit_kernel<<<(n + 31) / 32, 32, 0, s>>>(n, w.d, w.e, eps, w.scal, w.clus, w.lu, Q);
  }
  count_launch();
}

// tensor-core back-transformation (mixed path), carried out on Z^T so that
// every large operand is K-major: Z^T <- Z^T (I - V T V^T)^T block by block,
//   U   = Z^T_sub V_b^T     (n x kb)      tensor cores, 4 slices, split over K
//   Z^T_sub -= U Y_b        (n x m_b)     tensor cores, 4 slices
// with Y_b = T_b^T V_b formed for all blocks before the loop (it does not
// depend on Z).  The Gram matrices V_b V_b^T (for the T factors) and Y_b are
// double-float products on the FP32 pipe, one launch each for all blocks; the
// slices of V_b and Y_b^T are cut once, in two launches.
__global__ void transpose_sq_kernel(int n, const double* __restrict__ A, double* __restrict__ At) {
  __shared__ double tile[32][33];
  int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && j < n) ? A[(size_t)i * n + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int j = j0 + r, i = i0 + threadIdx.x;
    if (i < n && j < n) At[(size_t)j * n + i] = tile[threadIdx.x][r];
  }
}

static void transpose_sq(cudaStream_t s, int n, const double* A, double* At) {
  int t = (n + 31) / 32;
  transpose_sq_kernel<<<dim3(t, t), dim3(32, 8), 0, s>>>(n, A, At);
  count_launch();
}

// G_b = V_b V_b^T (upper 32 x 32 tiles) for every block b of kBtBlockTc
// reflectors; V_b = rows k0.. of the reflector store, columns c0 = k0 + 1 ..
__global__ void __launch_bounds__(256) gram_df_kernel(int n, int nref, const double* __restrict__ Vst,
                                                      double* __restrict__ Gall) {
  constexpr int KB = kBtBlockTc, TL = 32, CH = 64;
  const int b = blockIdx.y;
  const int k0 = b * KB, kb = min(KB, nref - k0), c0 = k0 + 1, m = n - c0;
  const int ti = blockIdx.x / (KB / TL), tj = blockIdx.x % (KB / TL);
  if (ti > tj || ti * TL >= kb || tj * TL >= kb) return;
  __shared__ dfl sa[TL][CH + 1], sb[TL][CH + 1];
  const int t = threadIdx.x, ii = t >> 3, jj = (t & 7) * 4;
  dfl acc[4] = {};
  for (int l0 = 0; l0 < m; l0 += CH) {
    for (int e = t; e < TL * CH; e += blockDim.x) {
      const int r = e / CH, c = e % CH;
      const int l = l0 + c;
      const int ra = ti * TL + r, rb = tj * TL + r;
      sa[r][c] = (ra < kb && l < m) ? df_from_double(Vst[(size_t)(k0 + ra) * n + c0 + l]) : dfl{0.0f, 0.0f};
      sb[r][c] = (rb < kb && l < m) ? df_from_double(Vst[(size_t)(k0 + rb) * n + c0 + l]) : dfl{0.0f, 0.0f};
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < CH; ++c) {
      const dfl a = sa[ii][c];
#pragma unroll
      for (int q = 0; q < 4; ++q) df_acc_mul(acc[q], a, sb[jj + q][c]);
    }
    __syncthreads();
  }
  const int i = ti * TL + ii;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = tj * TL + jj + q;
    if (i < kb && j < kb) Gall[(size_t)b * KB * KB + (size_t)i * KB + j] = df_to_double_fast(df_norm(acc[q]));
  }
}

// Y_b^T = V_b^T T_b (m_b x kb, row length KB) for every block b; T_b upper
// triangular (kb x kb, ld KB); 64 rows of Y_b^T per CTA, T_b and the V_b
// columns in shared memory as double-float
constexpr int kYRows = 64;
constexpr size_t kYSmem = (size_t)(kBtBlockTc * kBtBlockTc + kBtBlockTc * kYRows) * sizeof(dfl);
__global__ void __launch_bounds__(256) y_df_kernel(int n, int nref, const double* __restrict__ Vst,
                                                   const double* __restrict__ Tall, double* __restrict__ YT) {
  constexpr int KB = kBtBlockTc;
  extern __shared__ dfl ysm[];
  dfl* sT = ysm;                   // KB x KB
  dfl* sV = ysm + KB * KB;         // KB (reflector) x kYRows (column)
  const int b = blockIdx.y;
  const int k0 = b * KB, kb = min(KB, nref - k0), c0 = k0 + 1, m = n - c0;
  const int l0 = blockIdx.x * kYRows;
  if (l0 >= m) return;
  const double* Tb = Tall + (size_t)b * KB * KB;
  for (int e = threadIdx.x; e < KB * KB; e += blockDim.x) {
    const int i = e / KB, j = e % KB;
    sT[e] = (i < kb && j < kb && i <= j) ? df_from_double(Tb[(size_t)i * KB + j]) : dfl{0.0f, 0.0f};
  }
  for (int e = threadIdx.x; e < KB * kYRows; e += blockDim.x) {
    const int i = e / kYRows, c = e % kYRows;
    const int l = l0 + c;
    sV[e] = (i < kb && l < m) ? df_from_double(Vst[(size_t)(k0 + i) * n + c0 + l]) : dfl{0.0f, 0.0f};
  }
  __syncthreads();
  // thread t: row c = t / 4 of the tile, columns j = (t % 4) * 32 .. + 31
  const int c = threadIdx.x >> 2, jb = (threadIdx.x & 3) * 32;
  dfl acc[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) acc[q] = dfl{0.0f, 0.0f};
  for (int i = 0; i < kb; ++i) {
    const dfl v = sV[i * kYRows + c];
#pragma unroll
    for (int q = 0; q < 32; ++q) df_acc_mul(acc[q], v, sT[i * KB + jb + q]);
  }
  const int l = l0 + c;
  if (l < m) {
    double* out = YT + (size_t)b * n * KB + (size_t)l * KB;
#pragma unroll
    for (int q = 0; q < 32; ++q) out[jb + q] = (jb + q < kb) ? df_to_double_fast(df_norm(acc[q])) : 0.0;
  }
}

// back-transformation scratch (in the inverse-iteration workspace, free by then)
static int bt_blocks(int n) { return n > 2 ? (n - 2 + kBtBlockTc - 1) / kBtBlockTc : 0; }
constexpr int kBtSplitK = 6;
struct BtScratch {
  __nv_bfloat16* vs;   size_t vs_blk, vs_slice;   // V_b slices
  double* yt;                                     // Y_b^T, FP64
  __nv_bfloat16* ys;   size_t ys_blk, ys_slice;   // Y_b^T slices
  double* part;                                   // split-K partial products of U
};
static size_t bt_scratch_layout(int n, void* base, BtScratch* out) {
  const size_t nblk = (size_t)bt_blocks(n), KB = kBtBlockTc;
  const size_t ldn = (size_t)tc_ld(n > 1 ? n : 1);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
  const size_t vs_slice = KB * ldn, vs_blk = (size_t)kTcMaxSlices * vs_slice;
  const size_t o_vs = take(nblk * vs_blk * 2);
  const size_t o_yt = take(nblk * (size_t)n * KB * 8);
  const size_t ys_slice = (size_t)n * KB, ys_blk = (size_t)kTcMaxSlices * ys_slice;
  const size_t o_ys = take(nblk * ys_blk * 2);
  const size_t o_part = take((size_t)(kBtSplitK + 1) * n * KB * 8);
  if (out) {
    char* c = (char*)base;
    out->vs = (__nv_bfloat16*)(c + o_vs); out->vs_blk = vs_blk; out->vs_slice = vs_slice;
    out->yt = (double*)(c + o_yt);
    out->ys = (__nv_bfloat16*)(c + o_ys); out->ys_blk = ys_blk; out->ys_slice = ys_slice;
    out->part = (double*)(c + o_part);
  }
  return off;
}

static int eig_backtransform_tc(cudaStream_t s, int n, double* Q, EigWork& w, const TcWork& tw) {
  static PerDeviceOnce attr;
  once_per_device(attr, [] {
    return cudaFuncSetAttribute(tfactor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kBtBlockTc * kBtBlockTc * (int)sizeof(double)) == cudaSuccess &&
           cudaFuncSetAttribute(tfactor_all_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kBtBlockTc * kBtBlockTc * (int)sizeof(double)) == cudaSuccess &&
           cudaFuncSetAttribute(y_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kYSmem) ==
               cudaSuccess;
  });
  const int nref = n - 2;
  const int nblk = bt_blocks(n);
  const size_t stride = tc_slot_stride(tw);
  int* err = tc_error_flag(tw);
  BtScratch sc;
  bt_scratch_layout(n, w.lu, &sc);
  double* Zt = w.A;                      // tridiagonalisation workspace is free now
  transpose_sq(s, n, Q, Zt);
  // Gram matrices and T factors of all blocks, then Y_b^T = V_b^T T_b, then slices
  gram_df_kernel<<<dim3((kBtBlockTc / 32) * (kBtBlockTc / 32), nblk), 256, 0, s>>>(n, nref, w.Vst, w.Gm);
  count_launch();
  tfactor_all_kernel<<<nblk, kBtBlockTc, kBtBlockTc * kBtBlockTc * sizeof(double), s>>>(nref, kBtBlockTc, w.tau,
                                                                                      w.Gm, w.Tm);
  count_launch();
  y_df_kernel<<<dim3((n + kYRows - 1) / kYRows, nblk), 256, kYSmem, s>>>(n, nref, w.Vst, w.Tm, sc.yt);
  count_launch();
  tc_split_blocks(s, 0, n, nref, kBtBlockTc, w.Vst, sc.vs, sc.vs_blk, sc.vs_slice, 4);
  tc_split_blocks(s, 1, n, nref, kBtBlockTc, sc.yt, sc.ys, sc.ys_blk, sc.ys_slice, 4);
  __nv_bfloat16* sZ = tc_slot_base(tw, kSlotT0);
  __nv_bfloat16* sU = tc_slot_base(tw, kSlotT1);
  for (int b = nblk - 1; b >= 0; --b) {
    const int k0 = b * kBtBlockTc, kb = (k0 + kBtBlockTc < nref) ? kBtBlockTc : nref - k0;
    const int c0 = k0 + 1, m = n - c0;
    const int ldm = tc_ld(m);
    double* Zs = Zt + c0;                                // n x m, ld n
    tc_split_rows(s, n, m, Zs, n, 4, sZ, ldm, stride);
    const int parts = tc_gemm_grouped_rc_splitk(s, n, kb, m, sZ, ldm, stride, sc.vs + (size_t)b * sc.vs_blk, ldm,
                                                sc.vs_slice, 1.0, sc.part, kBtBlockTc, kBtSplitK, err);   // U parts
    if (parts <= 0) return -1;
    const int ldk = tc_ld(kb);                           // U slices fit the slot: kb <= n
    tc_reduce_split_rows(s, n, kb, sc.part, parts, kBtBlockTc, 4, sU, ldk, stride);
    if (tc_gemm_grouped_rc(s, n, m, kb, sU, ldk, stride, sc.ys + (size_t)b * sc.ys_blk, kBtBlockTc, sc.ys_slice,
                           -1.0, Zs, n, 1, err) != 0)                                        // Zs -= U Y_b
      return -1;
  }
  transpose_sq(s, n, Zt, Q);
  return 0;
}

int eig_backtransform(cudaStream_t s, int n, double* Q, EigWork& w, const TcWork* tw) {
  if (tw && n > 2) return eig_backtransform_tc(s, n, Q, w, *tw);
  // 4. back-transformation, last block of reflectors first
  int nref = n - 2;
  if (nref > 0) {
    int nblk = (nref + kBtBlock - 1) / kBtBlock;
    for (int b = nblk - 1; b >= 0; --b) {
      int k0 = b * kBtBlock, k1 = (k0 + kBtBlock < nref) ? k0 + kBtBlock : nref;
      int kb = k1 - k0, c0 = k0 + 1, m = n - c0;
      const double* Vb = w.Vst + (size_t)k0 * n + c0;
      dgemm(s, 0, 1, kb, kb, m, 1.0, Vb, n, Vb, n, 0.0, w.Gm, kBtBlock);
      tfactor_kernel<<<1, kBtBlock, kb * kb * sizeof(double), s>>>(kb, w.tau + k0, w.Gm, kBtBlock, w.Tm, kBtBlock);
      count_launch();
      dgemm(s, 0, 0, kb, n, m, 1.0, Vb, n, Q + (size_t)c0 * n, n, 0.0, w.Wt, n);
      dgemm(s, 0, 0, kb, n, kb, 1.0, w.Tm, kBtBlock, w.Wt, n, 0.0, w.Wt2, n);
      dgemm(s, 1, 0, m, n, kb, -1.0, Vb, n, w.Wt2, n, 1.0, Q + (size_t)c0 * n, n);
    }
  }
  return 0;
}

int symmetric_eig(cudaStream_t s, int n, const double* F, double* eps, double* Q, EigWork& w,
                  int* status, int sm_count) {
  int rc = eig_tridiagonalize(s, n, F, w, status, sm_count, false);
  if (rc) return rc;
  eig_bisect(s, n, eps, w, 1e-12, false);
  eig_vectors(s, n, eps, Q, w, false);
  eig_backtransform(s, n, Q, w, nullptr);
  return 0;
}

}  // namespace kx
