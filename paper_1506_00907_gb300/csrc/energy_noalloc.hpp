// Energy reduction that allocates no device memory (see energy_noalloc.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ridg {

// Largest number of element slots the fixed scratch array supports.
int64_t energy_noalloc_max_slots();

// Writes sum_k J_k/2 (p^T M p/(rho c^2) + rho v^T M v) of the slot-layout fields q to out (device),
// asynchronously on st.  Allocates nothing; returns cudaErrorInvalidValue above the size limit.
cudaError_t energy_noalloc(int N, bool fp64, const void* q, int64_t n_slots, const double* J, const void* mat,
                           const int* meta, const double* M, double* out, cudaStream_t st);

}  // namespace ridg
