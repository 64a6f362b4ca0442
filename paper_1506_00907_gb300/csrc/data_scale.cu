// Power-of-two scale of the receiver data injected by the backward receiver run.
//
// The receiver wavefield is linear in the data it re-injects, and multiplying by a power of two is
// exact in floating point, so running it on data scaled by s = 2^k gives exactly s times the fields
// of the unscaled run -- except where the unscaled run leaves the exponent range of the working
// precision.  The image increments multiply the source and receiver fields (Eqs. imageP, imageQ);
// in FP32 such products underflow once the two fields' magnitudes multiply below ~1e-38, which
// happens for shots of small amplitude.  Scaling the data so that max |data| lies in [1, 2) keeps the
// receiver fields near the magnitude of the data's Green's function, and the accumulated FP64 image
// is divided by s (again exactly) when it is read out.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "data_scale.hpp"

namespace ridg {

namespace {

constexpr int kThreads = 256;

// max |x| over n values as the bit pattern of a non-negative double (whose unsigned order is the
// numeric order; NaN patterns sort above infinity)
__global__ void max_abs_bits_kernel(const double* __restrict__ x, int64_t n, unsigned long long* __restrict__ out) {
  __shared__ unsigned long long red[kThreads];
  unsigned long long m = 0ull;
  for (int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x; i < n; i += int64_t(gridDim.x) * kThreads) {
    const unsigned long long b = __double_as_longlong(x[i]) & 0x7fffffffffffffffull;
    m = b > m ? b : m;
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w && red[threadIdx.x + w] > red[threadIdx.x]) red[threadIdx.x] = red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, red[0]);
}

// scale[0] = 2^(1 - e) with max = m 2^e, m in [0.5, 1) (so max * scale lies in [1, 2)); scale[1] = its
// inverse; both 1 when the maximum is zero or not finite
__global__ void scale_from_max_kernel(const unsigned long long* __restrict__ max_bits, double* __restrict__ scale) {
  const double mx = __longlong_as_double(static_cast<long long>(*max_bits));
  double s = 1.0;
  if (mx > 0.0 && isfinite(mx)) {
    int e = 0;
    frexp(mx, &e);
    s = ldexp(1.0, 1 - e);
  }
  scale[0] = s;
  scale[1] = 1.0 / s;
}

}  // namespace

cudaError_t data_scale(const double* x, int64_t n, void* work, cudaStream_t st) {
  unsigned long long* bits = static_cast<unsigned long long*>(work);
  double* scale = reinterpret_cast<double*>(bits + 1);
  cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    const int64_t want = (n + kThreads - 1) / kThreads;
    const unsigned blocks = unsigned(want < 1216 ? want : 1216);
    max_abs_bits_kernel<<<blocks, kThreads, 0, st>>>(x, n, bits);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  scale_from_max_kernel<<<1, 1, 0, st>>>(bits, scale);
  return cudaGetLastError();
}

cudaError_t data_scale_finish(void* work, cudaStream_t st) {
  unsigned long long* bits = static_cast<unsigned long long*>(work);
  scale_from_max_kernel<<<1, 1, 0, st>>>(bits, reinterpret_cast<double*>(bits + 1));
  return cudaGetLastError();
}

}  // namespace ridg
