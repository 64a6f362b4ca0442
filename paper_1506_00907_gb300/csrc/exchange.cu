// Interface-trace transfer between the parts of a partitioned mesh (Sec. 4.2).
//
// A part pushes the traces of its elements across every face into the neighbour's face inbox; for a
// neighbour of another part that inbox belongs to the part's ghost copy of the neighbour.  After a
// fine step the pushed rows (all three time slots of each interface face whose pushing element was
// advanced at that step) are gathered into one contiguous buffer, copied to the owning part, and
// scattered into the inbox rows of its own element.  Rows of time slots not written at the step
// carry what the last transfer already delivered, so copying them is harmless.
#include "exchange.hpp"

namespace ridg {

namespace {

template <typename real>
__global__ void pack_rows_kernel(const real* __restrict__ trace, int64_t n_slots, int row_len,
                                 const int64_t* __restrict__ rows, int64_t n, real* __restrict__ out) {
  const int64_t total = n * 3 * row_len;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t item = i / row_len, j = i - item * row_len;
    const int64_t e = item / 3, t = item - e * 3;
    out[i] = trace[(t * n_slots * 4 + rows[e]) * row_len + j];
  }
}

template <typename real>
__global__ void unpack_rows_kernel(real* __restrict__ trace, int64_t n_slots, int row_len,
                                   const int64_t* __restrict__ rows, int64_t n, const real* __restrict__ in) {
  const int64_t total = n * 3 * row_len;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t item = i / row_len, j = i - item * row_len;
    const int64_t e = item / 3, t = item - e * 3;
    trace[(t * n_slots * 4 + rows[e]) * row_len + j] = in[i];
  }
}

unsigned grid_for(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return unsigned(b < 1216 ? (b > 0 ? b : 1) : 1216);
}

}  // namespace

template <typename real>
cudaError_t pack_face_rows(const real* trace, int64_t n_slots, int row_len, const int64_t* rows, int64_t n, real* out,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  pack_rows_kernel<real><<<grid_for(n * 3 * row_len), 256, 0, st>>>(trace, n_slots, row_len, rows, n, out);
  return cudaGetLastError();
}

template <typename real>
cudaError_t unpack_face_rows(real* trace, int64_t n_slots, int row_len, const int64_t* rows, int64_t n, const real* in,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  unpack_rows_kernel<real><<<grid_for(n * 3 * row_len), 256, 0, st>>>(trace, n_slots, row_len, rows, n, in);
  return cudaGetLastError();
}

template cudaError_t pack_face_rows<float>(const float*, int64_t, int, const int64_t*, int64_t, float*, cudaStream_t);
template cudaError_t pack_face_rows<double>(const double*, int64_t, int, const int64_t*, int64_t, double*,
                                            cudaStream_t);
template cudaError_t unpack_face_rows<float>(float*, int64_t, int, const int64_t*, int64_t, const float*, cudaStream_t);
template cudaError_t unpack_face_rows<double>(double*, int64_t, int, const int64_t*, int64_t, const double*,
                                              cudaStream_t);

}  // namespace ridg
