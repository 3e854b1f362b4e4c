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
// gate (nullable device int): the kernels return at once when *gate == 0
void tc_split(cudaStream_t s, const TcWork& w, int slot, const double* X, int slices, int transpose,
              const int* gate = nullptr);
// C = alpha * sum over `terms` (1, 3, 6 or 10 for 1-4 slices) slice products A_a B_b^T
void tc_gemm(cudaStream_t s, const TcWork& w, int slotA, int slotB, int terms, double alpha, double* C,
             int sym, const int* gate = nullptr);

// The DMPT's 3-slice product (terms 6) with all slices of a k-tile staged together:
// the weight-1 slice product summed exactly per 512-K chunk, the lower-weight ones
// in FP32; within 2^-26 of sum |a||b| of the exact 6-term slice product
void tc_gemm_grouped(cudaStream_t s, const TcWork& w, int slotA, int slotB, double alpha, double* C, int sym,
                     const int* gate = nullptr);
// the 4-slice product (terms 10) the same way (density product): within ~2^-28 of
// sum |a||b| of the exact 10-term slice product
void tc_gemm_grouped4(cudaStream_t s, const TcWork& w, int slotA, int slotB, double alpha, double* C, int sym,
                      const int* gate = nullptr);
// general shapes with 4 slices (back-transformation); the same operands and
// partial-product layout as tc_gemm_rc / tc_gemm_rc_splitk; < 0 on a tensor-map error
int tc_gemm_grouped_rc(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Abase, int lda, size_t astride,
                       const __nv_bfloat16* Bbase, int ldb, size_t bstride, double alpha, double* C, int ldc,
                       int beta, int* err);
int tc_gemm_grouped_rc_splitk(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Abase, int lda,
                              size_t astride, const __nv_bfloat16* Bbase, int ldb, size_t bstride, double alpha,
                              double* P, int ldp, int splits, int* err);

// Building blocks on caller-provided buffers (used by the allocation-free entry point)
int tc_ld(int n);                                                   // padded slice row length
bool tc_encode_map(CUtensorMap* m, void* ptr, int n, int ld);       // BF16 slice tensor map
void tc_split_strided(cudaStream_t s, int n, int ld, const double* X, int slices, int transpose, int* ex,
                      __nv_bfloat16* base, size_t stride);
void tc_gemm_on_maps(cudaStream_t s, int n, const CUtensorMap* mapsA, const CUtensorMap* mapsB, int terms,
                     double alpha, double* C, int sym, int* err);

// General shapes (back-transformation): slices of op(X) (rows x cols, K = cols, row
// length ld, slice stride `stride` elements) and C (M x N, ldc) (+)= alpha sum A_a B_b^T
void tc_split_rc(cudaStream_t s, int rows, int cols, const double* X, int ldx, int transpose, int slices, int* ex,
                 __nv_bfloat16* base, int ld, size_t stride);
int tc_gemm_rc(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Abase, int lda, size_t astride,
               const __nv_bfloat16* Bbase, int ldb, size_t bstride, int terms, double alpha, double* C, int ldc,
               int beta, int* err);
// split-K: returns the number of parts z actually used (partials at P + z M ldp), < 0 on error
int tc_gemm_rc_splitk(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Abase, int lda, size_t astride,
                      const __nv_bfloat16* Bbase, int ldb, size_t bstride, int terms, double alpha, double* P,
                      int ldp, int splits, int* err);
// one-pass row slicing (row maximum and slices per warp), columns cols..ld-1 zero
void tc_split_rows(cudaStream_t s, int rows, int cols, const double* X, long long ldx, int slices,
                   __nv_bfloat16* base, int ld, size_t stride);
// all reflector blocks at once: mode 0 slices V_b (kb x m_b, rows of the reflector
// store from column b kblk + 1, row length tc_ld(m_b)), mode 1 slices Y_b^T (m_b x kb,
// src + b n kblk, row length kblk); block b at base + b blk_stride, slices slice_stride apart
void tc_split_blocks(cudaStream_t s, int mode, int n, int nref, int kblk, const double* src, __nv_bfloat16* base,
                     size_t blk_stride, size_t slice_stride, int slices);
// sum of `parts` partial products (rows x cols <= 128, at P + z rows ldp) and its slices
void tc_reduce_split_rows(cudaStream_t s, int rows, int cols, const double* P, int parts, int ldp, int slices,
                          __nv_bfloat16* base, int ld, size_t stride);
// test of the pipeline's bounded mbarrier wait: sets *err when `limit` tries expire
void tc_mbar_expiry(cudaStream_t s, int* err, long long limit);
// raw access to a slot's slice buffers (for the back-transformation)
__nv_bfloat16* tc_slot_base(const TcWork& w, int slot);
size_t tc_slot_stride(const TcWork& w);
int* tc_slot_exponents(const TcWork& w, int slot);

}  // namespace kx
