// Per-order launch entry points, instantiated in kernels_n<N>.cu.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "step_kernel.cuh"

namespace ridg {

// Kernel attributes (the dynamic shared-memory limit) belong to each device's context: they are set
// once per device, with that device current, the first time a kernel is launched there.  Launches
// come from several host threads (shot-server slots), so the set-up is serialised and its outcome
// kept per device.
struct PerDeviceSetup {
  static constexpr int kMaxDevices = 64;
  std::atomic<bool> done[kMaxDevices] = {};
  cudaError_t result[kMaxDevices] = {};
  std::mutex m;

  template <typename F>
  cudaError_t run(F&& configure) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (done[dev].load(std::memory_order_acquire)) return result[dev];
    std::lock_guard<std::mutex> lock(m);
    if (!done[dev].load(std::memory_order_relaxed)) {
      result[dev] = configure();
      done[dev].store(true, std::memory_order_release);
    }
    return result[dev];
  }
};

// Arguments of one reverse fine step of the multi-rate adjoint (adjoint_mr_kernels.cuh): the
// adjoint state, the active slots and each level's ring and trace-slot indices at that step.
template <typename real>
struct AdjMrArgs {
  real* mu;        // [fields]
  real* mu_ring;   // [3][fields]
  real* mu_in;     // [3][n_slots][8 NFPP]
  real* own;       // [n_slots][8 NFPP] scratch: the element's own-trace weights of this step
  int64_t slot_lo, n_slots;
  int64_t level_begin[kMaxLevels + 1];
  int n_levels;
  int ring_new[kMaxLevels], ring_old1[kMaxLevels], ring_old2[kMaxLevels];
  real h[kMaxLevels];
  int slot_read;
  int slot_full[kMaxLevels], slot_half[kMaxLevels];
  const double* geo;
  const real* mat;
  const int* meta;
  const real* Dt4;
  const real* Lt;
  int NPa;
  const int* fmask;
  const int* inv_fmask;  // [Np][3]: f * 32 + jf of each face node that is node m, in (f, jf) order, or -1
  const int* nbr;
  const uint8_t* finfo;
  const int* perm;
  // gradient: the forward right-hand side of this step (saved, source included), the source slot,
  // its projected Dirac and amplitude at this step, and the per-slot sums
  const real* rsaved;
  int64_t src_slot;
  const real* w_src;
  real F;
  double* acc;
};

template <int N, typename real>
struct Launch {
  // batch != null: a merged launch of n_shots shots (FP32 tensor-core contractions only), the grid
  // n_shots x batch->shot_blocks blocks
  static cudaError_t step(const StepArgs<real>& a, int W, cudaStream_t st, const BatchArgs<real>* batch = nullptr,
                          int n_shots = 1);
  static cudaError_t init_traces(const real* q, real* trace, int slot, int64_t n_slots, const double* geo,
                                 const int* meta, const int* fmask, const int* nbr, const uint8_t* finfo,
                                 const int* perm, cudaStream_t st);
  static cudaError_t sample(const real* q, const int64_t* rec_slot, const real* rec_row, int nrec, double* out,
                            int64_t n_time, int64_t col, cudaStream_t st);
  static cudaError_t energy(const real* q, int64_t n_slots, const double* J, const real* mat, const int* meta,
                            const double* M, double* out, cudaStream_t st);
  static cudaError_t state_io(bool to_slots, const double* q_abi_in, double* q_abi_out, real* q,
                              const int64_t* slot_of, const int* pos_of, int64_t K, cudaStream_t st);
  static cudaError_t image_out(const double* img, const int64_t* slot_of, const int* pos_of, int64_t K,
                               const double* inv_scale, double* out, cudaStream_t st);
  // discrete adjoint (adjoint_kernels.cuh)
  // out = A^T lam; own, inbox: scratch adjoint traces [n_slots][4][2][NFPP] each; Dt4: [Np][Np][4]
  // (D_0, D_1, D_2, 0)[n][m] at (m, n).  With s1 != null the adjoint Adams-Bashforth update
  // lam += h (a1 out + a2 s1 + a3 s2) is applied in place as well.
  static cudaError_t adj_rhs(real* lam, real* own, real* inbox, real* out, int64_t n_slots, const double* geo,
                             const real* mat, const int* meta, const real* Dt4, const real* Lt, int NPa, const int* fmask,
                             const int* nbr, const uint8_t* finfo, const int* perm, const real* s1, const real* s2,
                             double h, cudaStream_t st);
  static cudaError_t adj_inject(real* lam, const int* grp, const int* rec_sorted, int n_groups, const int64_t* rec_slot,
                                const real* rec_row, const double* res, int64_t n_time, int64_t col, double coef,
                                cudaStream_t st);
  // one reverse fine step of the multi-rate adjoint over the active slots [a.slot_lo, a.n_slots)
  static cudaError_t adjml_step(const AdjMrArgs<real>& a, cudaStream_t st);
  // acc[slot] += sum over the pressure nodes of lam_p (q1_p - q0_p - F w), per element slot
  static cudaError_t adj_grad(const real* lam, const real* q1, const real* q0, int64_t n_slots, int64_t src_slot,
                              const real* w_src, double F, double* acc, cudaStream_t st);
};

}  // namespace ridg
