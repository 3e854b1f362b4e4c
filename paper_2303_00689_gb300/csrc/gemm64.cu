// FP64 GEMM on the CUDA cores (the FP64 reference path and the eigensolver's
// back-transformation).  Row-major C = alpha op(A) op(B) + beta C, 64 x 64
// output tiles, 16-deep K slices staged in shared memory, 4 x 4 outputs per
// thread.  With sym != 0 the result is known to be symmetric (M == N): only
// tiles on or above the diagonal run, and each value is stored at (i, j) and
// (j, i), so the output is bitwise symmetric (D0 = Q f Q^T, Q^T F1 Q and
// Q Y Q^T of eqs. 19 and 36 are symmetric by definition).
#include "common.cuh"
#include "kernels.h"

namespace kx {

constexpr int GBM = 64, GBN = 64, GBK = 16;

__global__ void __launch_bounds__(256) dgemm_kernel(int ta, int tb, int M, int N, int K, double alpha,
                                                    const double* __restrict__ A, int lda,
                                                    const double* __restrict__ B, int ldb, double beta,
                                                    double* __restrict__ C, int ldc, int sym, const int* gate) {
  if (gate && *gate == 0) return;
  int bi = blockIdx.y, bj = blockIdx.x;
  if (sym && bi > bj) return;
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int m0 = bi * GBM, n0 = bj * GBN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < K; k0 += GBK) {
    // A tile: (i, k) for i < 64, k < 16
    for (int e = threadIdx.x; e < GBM * GBK; e += 256) {
      int i, k;
      if (!ta) { k = e % GBK; i = e / GBK; } else { i = e % GBM; k = e / GBM; }
      int gi = m0 + i, gk = k0 + k;
      double v = 0.0;
      if (gi < M && gk < K) v = ta ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
      As[k][i] = v;
    }
    // B tile: (k, j) for k < 16, j < 64
    for (int e = threadIdx.x; e < GBN * GBK; e += 256) {
      int j, k;
      if (!tb) { j = e % GBN; k = e / GBN; } else { k = e % GBK; j = e / GBK; }
      int gj = n0 + j, gk = k0 + k;
      double v = 0.0;
      if (gj < N && gk < K) v = tb ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
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
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
      if (gi >= M || gj >= N) continue;
      if (sym && gi > gj) continue;
      double v = alpha * acc[i][j];
      if (beta != 0.0) v += beta * C[(size_t)gi * ldc + gj];
      C[(size_t)gi * ldc + gj] = v;
      if (sym && gi != gj) C[(size_t)gj * ldc + gi] = v;
    }
}

void dgemm(cudaStream_t s, int ta, int tb, int M, int N, int K, double alpha, const double* A, int lda,
           const double* B, int ldb, double beta, double* C, int ldc, int sym, const int* gate) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  dgemm_kernel<<<grid, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym, gate);
  count_launch();
}

}  // namespace kx
