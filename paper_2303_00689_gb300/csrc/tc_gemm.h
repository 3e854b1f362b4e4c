// Tensor-core (tcgen05) GEMMs for the mixed-precision path (internal header).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace kx {

// slots of BF16 slice matrices (each holds up to kTcMaxSlices slices of one n x n operand)
constexpr int kTcPieceSlots = 6;
constexpr int kTcMaxSlices = 4;
enum TcSlot { kSlotQs = 0, kSlotQ = 1, kSlotQt = 2, kSlotT0 = 3, kSlotT1 = 4, kSlotSpare = 5 };

struct TcWork {
  void* base = nullptr;   // host-side bookkeeping (tensor maps, piece pointers)
  size_t bytes = 0;
};
size_t tc_work_bytes(int n);
void tc_work_bind(TcWork& w, void* device_base, int n);
void tc_work_release(TcWork& w);
bool tc_available();                  // driver entry point for tensor maps present
bool tc_ready(const TcWork& w);       // tensor maps encoded for this handle
int* tc_error_flag(const TcWork& w);  // device word set when a bounded wait expired
// X (n x n FP64) -> `slices` fixed-point BF16 slices in slot (transpose != 0 slices X^T)
void tc_split(cudaStream_t s, const TcWork& w, int slot, const double* X, int slices, int transpose);
// C = alpha * sum over `terms` (1, 3, 6 or 10 for 1-4 slices) slice products A_a B_b^T
void tc_gemm(cudaStream_t s, const TcWork& w, int slotA, int slotB, int terms, double alpha, double* C,
             int sym);

// Building blocks on caller-provided buffers (used by the allocation-free entry point)
int tc_ld(int n);                                                   // padded slice row length
bool tc_encode_map(CUtensorMap* m, void* ptr, int n, int ld);       // BF16 slice tensor map
void tc_split_strided(cudaStream_t s, int n, int ld, const double* X, int slices, int transpose, int* ex,
                      __nv_bfloat16* base, size_t stride);
void tc_gemm_on_maps(cudaStream_t s, int n, const CUtensorMap* mapsA, const CUtensorMap* mapsB, int terms,
                     double alpha, double* C, int sym, int* err);

}  // namespace kx
