// Interface-trace transfer between the parts of a partitioned mesh (Sec. 4.2; see exchange.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ridg {

// Face rows of a trace array [3 time slots][n_slots][4 faces][row_len] (row_len = 2 NFPP values:
// the (p, n.v) of one face's nodes).  pack: out[(i * 3 + t) * row_len + j] = trace[t][rows[i]][j]
// for the n rows listed (rows[i] = slot * 4 + face); unpack: the inverse, into another part's array.
template <typename real>
cudaError_t pack_face_rows(const real* trace, int64_t n_slots, int row_len, const int64_t* rows, int64_t n, real* out,
                           cudaStream_t st);
template <typename real>
cudaError_t unpack_face_rows(real* trace, int64_t n_slots, int row_len, const int64_t* rows, int64_t n, const real* in,
                             cudaStream_t st);

}  // namespace ridg
