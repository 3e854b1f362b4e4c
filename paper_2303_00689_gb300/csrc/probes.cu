// Measurement and failure-path hooks of the C ABI (see include/sim.h):
//  * sim_measure_peak: FP64 / FP32 FMA throughput of the device, the
//    denominators of the arithmetic-bound roofline fractions (the eigensolver
//    runs FP64-equivalent arithmetic in double-float on the FP32 pipe);
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

}  // namespace kx

using namespace kx;

extern "C" {

int sim_measure_peak(int device, int kind, double* tflops) {
  if (!tflops || (kind != 0 && kind != 1)) return SIM_EINVAL;
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
