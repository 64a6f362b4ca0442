// Small kernels around the fused step: trace initialisation, receiver sampling, energy,
// and layout conversions of the images.
#pragma once
#include "step_kernel.cuh"

namespace ridg {

// Traces (p, n.v) of the fields q pushed into the neighbours' face inboxes of trace slot `slot`
// (see WaveArgs::trace): node j of face f of slot s lands at index perm[j] of face f2 of the
// neighbour s2, with n.v taken with the neighbour's normal.
template <int N, typename real>
__global__ void init_traces_kernel(const real* __restrict__ q, real* __restrict__ trace, int slot, int64_t n_slots,
                                   const double* __restrict__ geo, const int* __restrict__ meta,
                                   const int* __restrict__ fmask, const int* __restrict__ nbr,
                                   const uint8_t* __restrict__ finfo, const int* __restrict__ perm) {
  using O = Order<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NFPP = O::NFPP;
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_slots * 4 * Nfp) return;
  int64_t s = i / (4 * Nfp);
  int r = int(i - s * 4 * Nfp);
  int f = r / Nfp, j = r - f * Nfp;
  if (!(meta[s] & kMetaValid)) return;
  const uint8_t info = finfo[s * 4 + f];
  if (finfo_bc(info) != 0) return;
  int n = fmask[f * 32 + j];
  int64_t blk = s >> 5;
  int lane = int(s & 31);
  auto at = [&](int fld) { return q[((blk * 4 + fld) * Np + n) * 32 + lane]; };
  const double* g = geo + s * kGeo;
  real p = at(0);
  real vn = real(g[9 + 3 * f]) * at(1) + real(g[10 + 3 * f]) * at(2) + real(g[11 + 3 * f]) * at(3);
  const int64_t s2 = nbr[s * 4 + f];
  const int j2 = perm[finfo_perm(info) * 32 + j];
  real* t = trace + (int64_t(slot) * n_slots + s2) * (8 * NFPP) + finfo_face(info) * 2 * NFPP;
  t[j2] = p;
  t[NFPP + j2] = -vn;
}

// Receiver pressures: out[r * n_time + col] = sum_m row_r[m] p(slot_r, m).
template <int N, typename real>
__global__ void sample_receivers_kernel(const real* __restrict__ q, const int64_t* __restrict__ rec_slot,
                                        const real* __restrict__ rec_row, int nrec, double* __restrict__ out,
                                        int64_t n_time, int64_t col) {
  using O = Order<N>;
  constexpr int Np = O::Np;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrec) return;
  int64_t s = rec_slot[r];
  if (s < 0) return;  // a receiver another part of a partitioned mesh samples
  int64_t blk = s >> 5;
  int lane = int(s & 31);
  double acc = 0.0;
  for (int m = 0; m < Np; ++m) acc += double(rec_row[int64_t(r) * Np + m]) * double(q[((blk * 4) * Np + m) * 32 + lane]);
  out[int64_t(r) * n_time + col] = acc;
}

// Discrete energy of the element in slot s (a valid slot): J/2 (p^T M p / (rho c^2) + rho v^T M v),
// with FP64 products and sums.  Shared by energy_kernel and the allocation-free variant.
template <int N, typename real>
__device__ __forceinline__ double slot_energy(const real* __restrict__ q, int64_t s, const double* __restrict__ Jdet,
                                              const real* __restrict__ mat, const double* __restrict__ M) {
  constexpr int Np = Order<N>::Np;
  const int64_t blk = s >> 5;
  const int lane = int(s & 31);
  const double rc2 = double(mat[s * kMat + 0]), irho = double(mat[s * kMat + 1]);
  double e = 0.0;
  for (int fld = 0; fld < 4; ++fld) {
    double acc = 0.0;
    for (int a = 0; a < Np; ++a) {
      const double xa = double(q[((blk * 4 + fld) * Np + a) * 32 + lane]);
      double row = 0.0;
      for (int b = 0; b < Np; ++b) row += M[a * Np + b] * double(q[((blk * 4 + fld) * Np + b) * 32 + lane]);
      acc += xa * row;
    }
    e += (fld == 0 ? acc / rc2 : acc / irho);
  }
  return 0.5 * Jdet[s] * e;
}

// Discrete energy sum_k J_k/2 (p^T M p / (rho c^2) + rho v^T M v), FP64 accumulation.
template <int N, typename real>
__global__ void energy_kernel(const real* __restrict__ q, int64_t n_slots, const double* __restrict__ Jdet,
                              const real* __restrict__ mat, const int* __restrict__ meta, const double* __restrict__ M,
                              double* __restrict__ out) {
  __shared__ double red[256];
  int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (s < n_slots && (meta[s] & kMetaValid)) e = slot_energy<N, real>(q, s, Jdet, mat, M);
  red[threadIdx.x] = e;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// Image from the slot layout [n_slots/32][Np][32] to element order [K][Np], times *inv_scale (a power
// of two; null = 1).
template <int N>
__global__ void image_to_elements_kernel(const double* __restrict__ img, const int64_t* __restrict__ slot_of,
                                         const int* __restrict__ pos_of, int64_t K, const double* __restrict__ inv_scale,
                                         double* __restrict__ out) {
  using O = Order<N>;
  constexpr int Np = O::Np;
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= K * Np) return;
  int64_t k = i / Np;
  int n = int(i - k * Np);  // reference numbering; pos_of[n] is the node's place in the slot layout
  int64_t s = slot_of[k];
  if (s < 0) {  // an element another part of a partitioned mesh images
    out[i] = 0.0;
    return;
  }
  const double v = img[((s >> 5) * Np + pos_of[n]) * 32 + (s & 31)];
  out[i] = inv_scale ? v * *inv_scale : v;
}

// Fields between the C-ABI layout [K][4][Np] (double, reference node numbering) and the slot
// layout [n_slots/32][4][Np][32] (working precision, device node numbering pos_of).
template <int N, typename real>
__global__ void state_from_abi_kernel(const double* __restrict__ q_abi, const int64_t* __restrict__ slot_of,
                                      const int* __restrict__ pos_of, int64_t K, real* __restrict__ q) {
  constexpr int Np = Order<N>::Np;
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= K * 4 * Np) return;
  int64_t k = i / (4 * Np);
  int r = int(i - k * 4 * Np), fld = r / Np, n = r - fld * Np;
  int64_t s = slot_of[k];
  if (s < 0) return;
  q[(((s >> 5) * 4 + fld) * Np + pos_of[n]) * 32 + (s & 31)] = real(q_abi[i]);
}
template <int N, typename real>
__global__ void state_to_abi_kernel(const real* __restrict__ q, const int64_t* __restrict__ slot_of,
                                    const int* __restrict__ pos_of, int64_t K, double* __restrict__ q_abi) {
  constexpr int Np = Order<N>::Np;
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= K * 4 * Np) return;
  int64_t k = i / (4 * Np);
  int r = int(i - k * 4 * Np), fld = r / Np, n = r - fld * Np;
  int64_t s = slot_of[k];
  q_abi[i] = s < 0 ? 0.0 : double(q[(((s >> 5) * 4 + fld) * Np + pos_of[n]) * 32 + (s & 31)]);
}

}  // namespace ridg
