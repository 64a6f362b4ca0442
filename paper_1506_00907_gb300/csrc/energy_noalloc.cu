// Discrete energy without any device allocation, for callers that cannot call cudaMalloc.
//
// Some callers of this library cannot allocate device memory at the moment they want the energy
// check: a host application that hands the library a fixed device-memory budget up front and owns
// every allocation itself, a time-critical stepping loop in which cudaMalloc/cudaFree must not run
// because they can block the host and synchronise the device, or a caller on a thread that must
// never enter the CUDA allocator.  This variant of the energy reduction keeps its per-block partial
// sums in a file-scope device array instead of a per-call allocation and writes the result to
// device memory the caller owns.
//
// The scratch array holds kMaxBlocks partial sums (32 KiB); every device that loads the library
// keeps it until the process exits.  Solvers with more than kMaxBlocks * 256 element slots are
// rejected.  The first call on a device looks up the array's device address with that device
// current (the host-side name of a __device__ array is only a stand-in); make that first call
// before any stream capture.  Every call on a device shares the array, and the array keeps the
// last call's contents: pass 1 overwrites every entry that pass 2 reads, so nothing needs
// clearing, but calls that overlap on the GPU (different streams, or different solvers on one
// device without ordering) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "energy_noalloc.hpp"
#include "aux_kernels.cuh"

namespace ridg {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 4096;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_partials[kMaxBlocks];

// device address of g_energy_partials per device, looked up once with that device current
double* g_partials_ptr[kMaxDevices] = {};
std::mutex g_partials_mutex;

template <int N, typename real>
__global__ void energy_partials_kernel(const real* __restrict__ q, int64_t n_slots, const double* __restrict__ Jdet,
                                       const real* __restrict__ mat, const int* __restrict__ meta,
                                       const double* __restrict__ M, double* __restrict__ partials) {
  __shared__ double red[kThreads];
  const int64_t s = int64_t(blockIdx.x) * kThreads + threadIdx.x;
  double e = 0.0;
  if (s < n_slots && (meta[s] & kMetaValid)) e = slot_energy<N, real>(q, s, Jdet, mat, M);
  red[threadIdx.x] = e;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void energy_sum_kernel(const double* __restrict__ partials, int n, double* __restrict__ out) {
  __shared__ double red[kThreads];
  double e = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) e += partials[i];
  red[threadIdx.x] = e;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Set-up, once per device and with that device current: the host-side name of a __device__ array
// is only a stand-in, so its device address must be looked up before a kernel can be given it.
cudaError_t partials_of_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_partials_mutex);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_partials);
    if (e != cudaSuccess) return e;
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  return cudaSuccess;
}

template <int N, typename real>
cudaError_t launch(const void* q, int64_t n_slots, const double* J, const void* mat, const int* meta, const double* M,
                   double* out, cudaStream_t st) {
  double* partials = nullptr;
  cudaError_t e = partials_of_current_device(&partials);
  if (e != cudaSuccess) return e;
  const int blocks = int((n_slots + kThreads - 1) / kThreads);
  energy_partials_kernel<N, real><<<blocks, kThreads, 0, st>>>(static_cast<const real*>(q), n_slots, J,
                                                                 static_cast<const real*>(mat), meta, M, partials);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  energy_sum_kernel<<<1, kThreads, 0, st>>>(partials, blocks, out);
  return cudaGetLastError();
}

}  // namespace

int64_t energy_noalloc_max_slots() { return int64_t(kMaxBlocks) * kThreads; }

cudaError_t energy_noalloc(int N, bool fp64, const void* q, int64_t n_slots, const double* J, const void* mat,
                           const int* meta, const double* M, double* out, cudaStream_t st) {
  if (n_slots > energy_noalloc_max_slots()) return cudaErrorInvalidValue;
  switch (N) {
    case 1: return fp64 ? launch<1, double>(q, n_slots, J, mat, meta, M, out, st) : launch<1, float>(q, n_slots, J, mat, meta, M, out, st);
    case 2: return fp64 ? launch<2, double>(q, n_slots, J, mat, meta, M, out, st) : launch<2, float>(q, n_slots, J, mat, meta, M, out, st);
    case 3: return fp64 ? launch<3, double>(q, n_slots, J, mat, meta, M, out, st) : launch<3, float>(q, n_slots, J, mat, meta, M, out, st);
    case 4: return fp64 ? launch<4, double>(q, n_slots, J, mat, meta, M, out, st) : launch<4, float>(q, n_slots, J, mat, meta, M, out, st);
    case 5: return fp64 ? launch<5, double>(q, n_slots, J, mat, meta, M, out, st) : launch<5, float>(q, n_slots, J, mat, meta, M, out, st);
    default: return fp64 ? launch<6, double>(q, n_slots, J, mat, meta, M, out, st) : launch<6, float>(q, n_slots, J, mat, meta, M, out, st);
  }
}

}  // namespace ridg
