// Power-of-two scale of injected receiver data (see data_scale.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ridg {

// work: device memory of kDataScaleWorkBytes.  Writes, asynchronously on st, the scale s = 2^k that
// brings max |x[0..n)| into [1, 2) to ((double*)work)[1] and 1/s to ((double*)work)[2] (both 1 for an
// all-zero or non-finite x).
constexpr size_t kDataScaleWorkBytes = 3 * sizeof(double);
cudaError_t data_scale(const double* x, int64_t n, void* work, cudaStream_t st);
// The scale and its inverse from the maximum bits already in work[0] (for a maximum combined over
// the parts of a partitioned mesh).
cudaError_t data_scale_finish(void* work, cudaStream_t st);

}  // namespace ridg
