// Allocation-free variant of the tensor-core slice GEMM (sim_tc_gemm_noalloc).
//
// Some callers cannot allocate device memory: a serving process that has
// carved all of the GPU's memory into fixed per-request slots under a hard
// budget, or a latency-critical loop in which cudaMalloc / cudaFree would
// synchronise the whole device.  This entry point takes device inputs and
// outputs from the caller and keeps its own scratch (the BF16 slices of both
// operands, their per-row exponents and an error flag) in one file-scope
// device array of fixed size, so it performs no allocation at all.
//
// Limits and sharing: n <= kNoAllocMaxN.  Every call on a device uses the
// same scratch array, which keeps the previous call's contents; the error
// flag is cleared at the start of each call and the slices are rewritten
// in full.  Calls whose work overlaps on the GPU (other streams, other
// threads) race on the scratch and must be serialised by the caller.  The
// first call on a device resolves the array's device address with
// cudaGetSymbolAddress (with that device current); it should come before
// any stream capture on that device.  Each call encodes its tensor maps on
// the host and finishes with a synchronisation of the given stream.
#include <mutex>

#include "../../include/sim.h"
#include "common.cuh"
#include "tc_gemm.h"

namespace kx {

constexpr int kNoAllocMaxN = 256;
constexpr int kNoAllocLd = 256;                                         // tc_ld(kNoAllocMaxN)
constexpr size_t kSliceElems = (size_t)kNoAllocMaxN * kNoAllocLd;       // one slice
constexpr size_t kSliceBytes = kSliceElems * 2;                         // 128 KB
constexpr size_t kOperandBytes = (size_t)kTcMaxSlices * kSliceBytes;    // 512 KB
constexpr size_t kExpBytes = (size_t)kNoAllocMaxN * sizeof(int);
constexpr size_t kNoAllocBytes = 2 * kOperandBytes + 2 * kExpBytes + 256;   // ~1.0 MB

// the only scratch this entry point uses; resident on every device that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch
};
static NoAllocDevice g_noalloc_dev[64];
static std::mutex g_noalloc_mutex;

// one-time per-device set-up, with the device current
static int noalloc_setup(int dev, const char** why) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (d.ready) return SIM_OK;
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return SIM_EINTERNAL;
  }
  d.base = (unsigned char*)ptr;
  d.ready = true;
  return SIM_OK;
}

}  // namespace kx

using namespace kx;

extern "C" int sim_tc_gemm_noalloc(int n, const double* A, const double* B, int terms, int sym, double* C,
                                   void* stream) {
  if (n < 1 || n > kNoAllocMaxN) return SIM_EINVAL;
  if (!A || !B || !C || (terms != 1 && terms != 3 && terms != 6 && terms != 10)) return SIM_EINVAL;
  if (!tc_available()) return SIM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SIM_EINTERNAL;
  const char* why = nullptr;
  int rc = noalloc_setup(dev, &why);
  if (rc != SIM_OK) return rc;
  NoAllocDevice& d = g_noalloc_dev[dev];
  cudaStream_t s = (cudaStream_t)stream;
  const int ld = tc_ld(n);
  const int slices = (terms == 10) ? 4 : (terms == 6) ? 3 : (terms == 3) ? 2 : 1;
  __nv_bfloat16* sa = (__nv_bfloat16*)(d.base);
  __nv_bfloat16* sb = (__nv_bfloat16*)(d.base + kOperandBytes);
  int* exA = (int*)(d.base + 2 * kOperandBytes);
  int* exB = (int*)(d.base + 2 * kOperandBytes + kExpBytes);
  int* err = (int*)(d.base + 2 * kOperandBytes + 2 * kExpBytes);
  // tensor maps for this n (host-side encoding only; no device memory involved)
  CUtensorMap mA[kTcMaxSlices], mB[kTcMaxSlices];
  size_t stride = (size_t)n * ld;                        // slices packed for this n
  for (int a = 0; a < kTcMaxSlices; ++a) {
    if (!tc_encode_map(&mA[a], sa + a * stride, n, ld) || !tc_encode_map(&mB[a], sb + a * stride, n, ld))
      return SIM_EINTERNAL;
  }
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return SIM_EINTERNAL;
  tc_split_strided(s, n, ld, A, slices, 0, exA, sa, stride);
  tc_split_strided(s, n, ld, B, slices, 0, exB, sb, stride);
  tc_gemm_on_maps(s, n, mA, mB, terms, 1.0, C, sym ? 1 : 0, err);
  int flag = 0;
  if (cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SIM_EINTERNAL;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SIM_EINTERNAL;
  if (cudaGetLastError() != cudaSuccess) return SIM_EINTERNAL;
  return flag ? SIM_ETIMEOUT : SIM_OK;
}
