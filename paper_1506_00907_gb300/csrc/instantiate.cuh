// Explicit instantiation of the kernels of one order (RIDG_ORDER), included by kernels_n<N>.cu.
#include "aux_kernels.cuh"
#include "dispatch.hpp"
#include "step_kernel_tc.cuh"

#include <type_traits>

namespace ridg {

template <int N, typename real, int W>
static cudaError_t launch_step_w(const StepArgs<real>& a, cudaStream_t st) {
  int64_t blocks = (a.slot_hi - a.slot_lo) / (32 / W);
  if (blocks <= 0) return cudaSuccess;
  if constexpr (std::is_same<real, float>::value) {
    // FP32: element products on tensor cores (TF32 three-term split)
    constexpr size_t smem = SmemTc<N, W>::bytes;
    static bool configured = false;
    if (!configured) {
      cudaError_t e = cudaFuncSetAttribute(dg_step_kernel_tc<N, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(smem));
      if (e != cudaSuccess) return e;
      configured = true;
    }
    dg_step_kernel_tc<N, W><<<dim3(unsigned(blocks)), TcOrder<N>::NT, smem, st>>>(a);
  } else {
    constexpr size_t smem = step_smem_bytes<N, real, W>();
    static bool configured = false;
    if (!configured) {
      cudaError_t e = cudaFuncSetAttribute(dg_step_kernel<N, real, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(smem));
      if (e != cudaSuccess) return e;
      configured = true;
    }
    dg_step_kernel<N, real, W><<<dim3(unsigned(blocks)), Order<N>::NT, smem, st>>>(a);
  }
  return cudaGetLastError();
}

template <int N, typename real>
cudaError_t Launch<N, real>::step(const StepArgs<real>& a, int W, cudaStream_t st) {
  return W == 1 ? launch_step_w<N, real, 1>(a, st) : launch_step_w<N, real, 2>(a, st);
}

template <int N, typename real>
cudaError_t Launch<N, real>::init_traces(const real* q, real* trace, int slot, int64_t n_slots, const double* geo,
                                         const int* meta, const int* fmask, const int* nbr, const uint8_t* finfo,
                                         const int* perm, cudaStream_t st) {
  int64_t n = n_slots * 4 * Order<N>::Nfp;
  init_traces_kernel<N, real><<<unsigned((n + 255) / 256), 256, 0, st>>>(q, trace, slot, n_slots, geo, meta, fmask,
                                                                           nbr, finfo, perm);
  return cudaGetLastError();
}

template <int N, typename real>
cudaError_t Launch<N, real>::sample(const real* q, const int64_t* rec_slot, const real* rec_row, int nrec,
                                    double* out, int64_t n_time, int64_t col, cudaStream_t st) {
  if (nrec <= 0) return cudaSuccess;
  sample_receivers_kernel<N, real><<<unsigned((nrec + 127) / 128), 128, 0, st>>>(q, rec_slot, rec_row, nrec, out,
                                                                                   n_time, col);
  return cudaGetLastError();
}

template <int N, typename real>
cudaError_t Launch<N, real>::energy(const real* q, int64_t n_slots, const double* J, const real* mat, const int* meta,
                                    const double* M, double* out, cudaStream_t st) {
  energy_kernel<N, real><<<unsigned((n_slots + 255) / 256), 256, 0, st>>>(q, n_slots, J, mat, meta, M, out);
  return cudaGetLastError();
}

template <int N, typename real>
cudaError_t Launch<N, real>::image_out(const double* img, const int64_t* slot_of, const int* pos_of, int64_t K,
                                       double* out, cudaStream_t st) {
  int64_t n = K * Order<N>::Np;
  image_to_elements_kernel<N><<<unsigned((n + 255) / 256), 256, 0, st>>>(img, slot_of, pos_of, K, out);
  return cudaGetLastError();
}

template struct Launch<RIDG_ORDER, float>;
template struct Launch<RIDG_ORDER, double>;

}  // namespace ridg
