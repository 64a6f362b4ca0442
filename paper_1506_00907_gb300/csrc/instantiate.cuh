// Explicit instantiation of the kernels of one order (RIDG_ORDER), included by kernels_n<N>.cu.
#include "ridg.h"

#include "adjoint_kernels.cuh"
#include "adjoint_mr_kernels.cuh"
#include "aux_kernels.cuh"
#include "dispatch.hpp"
#include "step_kernel_tc.cuh"

#include <type_traits>

namespace ridg {

// FP32 on tensor cores with the split format KIND; BATCH: n_shots shots of one solver in one launch
template <int N, int W, int KIND, bool BATCH>
static cudaError_t launch_step_tc(const StepArgs<float>& a, const BatchArgs<float>* batch, int n_shots, int64_t blocks,
                                  cudaStream_t st) {
  constexpr size_t smem = SmemTc<N, W, KIND>::bytes;
  static PerDeviceSetup setup;
  const cudaError_t configured = setup.run([] {
    return cudaFuncSetAttribute(dg_step_kernel_tc<N, W, KIND, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(smem));
  });
  if (configured != cudaSuccess) return configured;
  if constexpr (BATCH) {
    dg_step_kernel_tc<N, W, KIND, true><<<dim3(unsigned(blocks * n_shots)), TcOrder<N>::NT, smem, st>>>(a, *batch);
  } else {
    (void)batch;
    (void)n_shots;
    dg_step_kernel_tc<N, W, KIND, false><<<dim3(unsigned(blocks)), TcOrder<N>::NT, smem, st>>>(a, NoBatch{0});
  }
  return cudaGetLastError();
}

template <int N, int W, int KIND>
static cudaError_t launch_step_tc_any(const StepArgs<float>& a, const BatchArgs<float>* batch, int n_shots,
                                      int64_t blocks, cudaStream_t st) {
  if (batch) return launch_step_tc<N, W, KIND, true>(a, batch, n_shots, blocks, st);
  return launch_step_tc<N, W, KIND, false>(a, nullptr, 1, blocks, st);
}

template <int N, typename real, int W>
static cudaError_t launch_step_w(const StepArgs<real>& a, const BatchArgs<real>* batch, int n_shots, cudaStream_t st) {
  int64_t blocks = (a.slot_hi - a.slot_lo) / (32 / W);
  if (blocks <= 0) return cudaSuccess;
  if (batch && (n_shots < 1 || n_shots > kMaxBatch || batch->shot_blocks != blocks)) return cudaErrorInvalidValue;
  if constexpr (std::is_same<real, float>::value) {
    if (a.contraction == RIDG_CONTRACT_TENSOR) return launch_step_tc_any<N, W, kSplitTf32>(a, batch, n_shots, blocks, st);
    if (a.contraction == RIDG_CONTRACT_TENSOR_BF16)
      return launch_step_tc_any<N, W, kSplitBf16>(a, batch, n_shots, blocks, st);
    if (a.contraction == RIDG_CONTRACT_TENSOR_FP16)
      return launch_step_tc_any<N, W, kSplitFp16>(a, batch, n_shots, blocks, st);
  }
  // FP64, or FP32 on CUDA cores: one shot per launch (the engine launches a batch shot by shot)
  if (batch) return cudaErrorInvalidValue;
  constexpr size_t smem = step_smem_bytes<N, real, W>();
  static PerDeviceSetup setup;
  const cudaError_t configured = setup.run([] {
    return cudaFuncSetAttribute(dg_step_kernel<N, real, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  });
  if (configured != cudaSuccess) return configured;
  dg_step_kernel<N, real, W><<<dim3(unsigned(blocks)), Order<N>::NT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int N, typename real>
cudaError_t Launch<N, real>::step(const StepArgs<real>& a, int W, cudaStream_t st, const BatchArgs<real>* batch,
                                  int n_shots) {
  return W == 1 ? launch_step_w<N, real, 1>(a, batch, n_shots, st) : launch_step_w<N, real, 2>(a, batch, n_shots, st);
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
                                       const double* inv_scale, double* out, cudaStream_t st) {
  int64_t n = K * Order<N>::Np;
  image_to_elements_kernel<N><<<unsigned((n + 255) / 256), 256, 0, st>>>(img, slot_of, pos_of, K, inv_scale, out);
  return cudaGetLastError();
}

template <int N, typename real>
cudaError_t Launch<N, real>::state_io(bool to_slots, const double* q_abi_in, double* q_abi_out, real* q,
                                      const int64_t* slot_of, const int* pos_of, int64_t K, cudaStream_t st) {
  int64_t n = K * 4 * Order<N>::Np;
  if (n <= 0) return cudaSuccess;
  if (to_slots)
    state_from_abi_kernel<N, real><<<unsigned((n + 255) / 256), 256, 0, st>>>(q_abi_in, slot_of, pos_of, K, q);
  else
    state_to_abi_kernel<N, real><<<unsigned((n + 255) / 256), 256, 0, st>>>(q, slot_of, pos_of, K, q_abi_out);
  return cudaGetLastError();
}

template <int N, typename real>
cudaError_t Launch<N, real>::adj_rhs(real* lam, real* own, real* inbox, real* out, int64_t n_slots, const double* geo,
                                     const real* mat, const int* meta, const real* Dt4, const real* Lt, int NPa,
                                     const int* fmask, const int* nbr, const uint8_t* finfo, const int* perm,
                                     const real* s1, const real* s2, double h, cudaStream_t st) {
  const int64_t blocks = n_slots / 32;
  if (blocks <= 0) return cudaSuccess;
  constexpr size_t sm_t = adj_traces_smem<N, real>(), sm_r = adj_rhs_smem<N, real>();
  static_assert(sm_t <= 227 * 1024 && sm_r <= 227 * 1024, "adjoint kernels exceed the shared memory of a block");
  static PerDeviceSetup setup;
  const cudaError_t configured = setup.run([] {
    cudaError_t e =
        cudaFuncSetAttribute(adj_traces_kernel<N, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_t));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(adj_rhs_kernel<N, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_r));
    return e;
  });
  if (configured != cudaSuccess) return configured;
  adj_traces_kernel<N, real><<<unsigned(blocks), 256, sm_t, st>>>(lam, own, inbox, n_slots, geo, mat, meta, Lt, NPa,
                                                                   nbr, finfo, perm);
  adj_rhs_kernel<N, real><<<unsigned(blocks), 256, sm_r, st>>>(lam, own, inbox, out, n_slots, geo, mat, meta, Dt4,
                                                                fmask, finfo, s1, s2, real(h));
  return cudaGetLastError();
}

template <int N, typename real>
cudaError_t Launch<N, real>::adj_inject(real* lam, const int* grp, const int* rec_sorted, int n_groups,
                                        const int64_t* rec_slot, const real* rec_row, const double* res,
                                        int64_t n_time, int64_t col, double coef, cudaStream_t st) {
  if (n_groups <= 0) return cudaSuccess;
  adj_inject_kernel<N, real><<<unsigned(n_groups), 64, 0, st>>>(lam, grp, rec_sorted, rec_slot, rec_row, res, n_time,
                                                                 col, coef);
  return cudaGetLastError();
}

template <int N, typename real>
cudaError_t Launch<N, real>::adjml_step(const AdjMrArgs<real>& a, cudaStream_t st) {
  const int64_t blocks = (a.n_slots - a.slot_lo) / 32;
  if (blocks <= 0) return cudaSuccess;
  constexpr size_t sm_t = adjml_traces_smem<N, real>(), sm_r = adjml_rhs_smem<N, real>();
  constexpr size_t sm_p = adjml_pull_smem<N, real>();
  static_assert(sm_t <= 227 * 1024 && sm_r <= 227 * 1024 && sm_p <= 200 * 1024,
                "multi-rate adjoint kernels exceed the shared memory");
  static PerDeviceSetup setup;
  const cudaError_t configured = setup.run([] {
    cudaError_t e =
        cudaFuncSetAttribute(adjml_traces_kernel<N, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_t));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(adjml_rhs_kernel<N, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_r));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(adjml_pull_kernel<N, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_p));
    return e;
  });
  if (configured != cudaSuccess) return configured;
  adjml_pull_kernel<N, real><<<unsigned(blocks), 256, sm_p, st>>>(a);
  adjml_traces_kernel<N, real><<<unsigned(blocks), 256, sm_t, st>>>(a);
  adjml_rhs_kernel<N, real><<<unsigned(blocks), 256, sm_r, st>>>(a);
  return cudaGetLastError();
}

template <int N, typename real>
cudaError_t Launch<N, real>::adj_grad(const real* lam, const real* q1, const real* q0, int64_t n_slots,
                                      int64_t src_slot, const real* w_src, double F, double* acc, cudaStream_t st) {
  const int64_t blocks = n_slots / 32;
  if (blocks <= 0) return cudaSuccess;
  adj_grad_kernel<N, real><<<unsigned(blocks), 256, 0, st>>>(lam, q1, q0, n_slots, src_slot, w_src, F, acc);
  return cudaGetLastError();
}

template struct Launch<RIDG_ORDER, float>;
template struct Launch<RIDG_ORDER, double>;

}  // namespace ridg
