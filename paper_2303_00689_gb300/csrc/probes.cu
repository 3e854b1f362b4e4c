// Measurement and failure-path hooks of the C ABI (see include/sim.h):
//  * sim_measure_peak: FP64 / FP32 FMA throughput of the device, the
//    denominators of the arithmetic-bound roofline fractions (the eigensolver
//    runs FP64-equivalent arithmetic in double-float on the FP32 pipe), and the
//    L2 read + write rate of the tridiagonalisation's launch shape;
//  * sim_debug_barrier_limit: the wall-time limit of the eigensolver's grid
//    barriers, so a test can make a real step's barrier wait expire;
//  * sim_debug_wait_expiry: one bounded mbarrier wait that nothing satisfies.
#include <cstdio>
#include <string>

#include "../../include/sim.h"
#include "common.cuh"
#include "kernels.h"
#include "tc_gemm.h"

namespace kx {

constexpr int kPeakChains = 8;   // independent FMA chains per thread

template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(int iters, T a, T b, T* sink) {
  T x[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = fma(x[c], a, b);
  T s = 0;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += x[c];
  if (s == (T)-12345.0) *sink = s;   // keeps the chains live; never true for these inputs
}

// L2 read + write rate with the double-float tridiagonalisation's launch shape
// (one block of 512 threads per SM): every element of an L2-resident buffer is
// read and written back once per pass, four loads in flight per thread.
constexpr int kL2Threads = 512, kL2Passes = 20;
constexpr size_t kL2Bytes = (size_t)3360 * 3360 * 8;   // the n = 3360 double-float matrix: 90 MB

__global__ void __launch_bounds__(kL2Threads) l2_rw_kernel(float2* __restrict__ p, size_t len, int passes) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int it = 0; it < passes; ++it)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += 4 * stride) {
      float2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = (i + u * stride < len) ? __ldcg(p + i + u * stride) : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i + u * stride < len) p[i + u * stride] = make_float2(v[u].x * 1.0000001f, v[u].y);
    }
}

}  // namespace kx

using namespace kx;

extern "C" {

static int measure_l2(int device, double* tbs);

int sim_measure_peak(int device, int kind, double* tflops) {
  if (!tflops || kind < 0 || kind > 2) return SIM_EINVAL;
  if (kind == 2) return measure_l2(device, tflops);
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return SIM_EINVAL;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* sink = nullptr;
  int rc = SIM_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMalloc(&sink, 16) != cudaSuccess)
    rc = SIM_EINTERNAL;
  const dim3 grid(sms * 8), block(256);
  const int iters = (kind == 0) ? 4096 : 262144;
  float ms = 0.0f;
  if (rc == SIM_OK) {
    for (int rep = 0; rep < 2 && rc == SIM_OK; ++rep) {   // first launch warms up
      cudaEventRecord(e0, s);
      if (kind == 0)
        fma_rate_kernel<double><<<grid, block, 0, s>>>(iters, 0.999999, 1e-7, (double*)sink);
      else
        fma_rate_kernel<float><<<grid, block, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)sink);
      count_launch();
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = SIM_EINTERNAL;
      cudaEventElapsedTime(&ms, e0, e1);
    }
  }
  if (rc == SIM_OK) {
    const double fl = 2.0 * grid.x * block.x * (double)kPeakChains * iters;
    *tflops = fl / (ms * 1e-3) / 1e12;
  }
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

// kind 2 of sim_measure_peak: TB/s of L2 read + write bytes (the buffer is
// zeroed, so the values stay 0; the first launch brings it into L2)
static int measure_l2(int device, double* tbs) {
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return SIM_EINVAL;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* buf = nullptr;
  int rc = SIM_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMalloc(&buf, kL2Bytes) != cudaSuccess || cudaMemsetAsync(buf, 0, kL2Bytes, s) != cudaSuccess)
    rc = SIM_EINTERNAL;
  const size_t len = kL2Bytes / sizeof(float2);
  float ms = 0.0f;
  for (int rep = 0; rep < 2 && rc == SIM_OK; ++rep) {   // first launch warms up
    cudaEventRecord(e0, s);
    l2_rw_kernel<<<sms, kL2Threads, 0, s>>>((float2*)buf, len, kL2Passes);
    count_launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = SIM_EINTERNAL;
    cudaEventElapsedTime(&ms, e0, e1);
  }
  if (rc == SIM_OK) *tbs = 2.0 * (double)kL2Bytes * kL2Passes / (ms * 1e-3) / 1e12;
  if (buf) cudaFree(buf);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

int sim_debug_barrier_limit(int device, unsigned long long ns) {
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return SIM_EINVAL;
  const int rc = (eig_set_barrier_limit(ns) == 0) ? SIM_OK : SIM_EINTERNAL;
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

int sim_debug_wait_expiry(int device, long long tries) {
  if (tries < 1) return SIM_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return SIM_EINVAL;
  int* err = nullptr;
  int flag = 0, rc = SIM_OK;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess || cudaMemset(err, 0, sizeof(int)) != cudaSuccess) {
    rc = SIM_EINTERNAL;
  } else {
    tc_mbar_expiry(0, err, tries);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = SIM_EINTERNAL;
    else
      rc = flag ? SIM_ETIMEOUT : SIM_OK;
  }
  if (err) cudaFree(err);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

}  // extern "C"
