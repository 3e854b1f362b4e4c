// Tensor-core (tcgen05) GEMMs for the mixed-precision path (internal header).
#pragma once
#include <cuda_runtime.h>

namespace kx {

struct TcWork {
  void* base = nullptr;
  size_t bytes = 0;
};
size_t tc_work_bytes(int n);
void tc_work_bind(TcWork& w, void* base, int n);
bool tc_available();
// D = Qs Qs^T (symmetric), operands split into `pieces` BF16 parts
void tc_syrk_split(cudaStream_t s, int n, const double* Qs, double* D, TcWork& w, int pieces);
// transpose_first: C = Q^T M Q ; else C = Q M Q^T (M symmetric); C symmetric
void tc_similarity(cudaStream_t s, int n, const double* Q, const double* M, double* C, TcWork& w,
                   int transpose_first);

}  // namespace kx
