// Discrete adjoint of the single-rate scheme: the transposed right-hand-side operator A^T, the
// adjoint Adams-Bashforth recursion and the velocity gradient (CUDA cores, any precision).
//
// Forward operator (Sec. 3.1, Eqs. dgLocalSchemeP/U with the penalty fluxes of Eqs. weakFormP/V):
//   r_p   = -rho c^2 sum_j D_j (sum_i g_ij v_i) + sum_f L_f [alpha_f (jv - tau_p jp)]
//   r_v_i = -(1/rho) sum_j g_ij D_j p          + sum_f n_fi L_f [beta_f (jp - tau_v jv)]
// with alpha_f = -Fs_f rho c^2 / 2, beta_f = -Fs_f / (2 rho), jp = p+ - p-, jv = vn+ - vn-.
// Its transpose applied to lambda, element by element:
//   volume:  (A^T l)_v_i = -rho c^2 sum_j g_ij D_j^T l_p,  (A^T l)_p = -(1/rho) sum_ij g_ij D_j^T l_v_i
//   faces:   adjoint traces at = alpha_f L_f^T l_p, bt = beta_f L_f^T (n_f . l_v) (adj_traces_kernel);
//            the flux depends on jp with weight (-tau_p at + bt) and on jv with weight (at - tau_v bt),
//            so the interior traces (p-, vn-) of the element receive minus these weights and, through
//            jp, jv of the neighbour's flux, the neighbour's weights (its vn+ is minus this element's
//            n.v); boundary ghosts fold p+ and vn+ into p- and vn- (free: jp = -2p-, jv = 0;
//            transparent: jp = -p-, jv = -vn-; rigid: jp = 0, jv = -2vn-).
// Layouts are the solver's: fields [K/32][4][Np][32] in the device node numbering, adjoint traces
// [slot][4 faces][2][NFPP].
#pragma once
#include <cuda_runtime.h>

#include "step_kernel.cuh"

namespace ridg {

template <int N, typename real>
__global__ void adj_traces_kernel(const real* __restrict__ lam, real* __restrict__ adjt, int64_t n_slots,
                                  const double* __restrict__ geo, const real* __restrict__ mat,
                                  const int* __restrict__ meta, const real* __restrict__ Lt, int NPa) {
  using O = Order<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NFPP = O::NFPP;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_slots * 4 * Nfp) return;
  const int64_t s = i / (4 * Nfp);
  const int r = int(i - s * 4 * Nfp);
  const int f = r / Nfp, j = r - f * Nfp;
  real* out = adjt + s * (8 * NFPP) + f * 2 * NFPP;
  if (!(meta[s] & kMetaValid)) {
    out[j] = real(0);
    out[NFPP + j] = real(0);
    return;
  }
  const int64_t blk = s >> 5;
  const int lane = int(s & 31);
  const double* g = geo + s * kGeo;
  const real* m = mat + s * kMat;
  const double nx = g[9 + 3 * f], ny = g[10 + 3 * f], nz = g[11 + 3 * f], fs = g[21 + f];
  const real* row = Lt + int64_t(f * Nfp + j) * NPa;
  auto at = [&](int fld, int n) { return lam[((blk * 4 + fld) * Np + n) * 32 + lane]; };
  real ap = 0, av = 0;
  for (int n = 0; n < Np; ++n) {
    const real l = row[n];
    ap += l * at(0, n);
    av += l * (real(nx) * at(1, n) + real(ny) * at(2, n) + real(nz) * at(3, n));
  }
  out[j] = real(-0.5 * fs) * m[0] * ap;
  out[NFPP + j] = real(-0.5 * fs) * m[1] * av;
}

template <int N, typename real>
__global__ void adj_rhs_kernel(const real* __restrict__ lam, const real* __restrict__ adjt, real* __restrict__ out,
                               int64_t n_slots, const double* __restrict__ geo, const real* __restrict__ mat,
                               const int* __restrict__ meta, const real* __restrict__ Dt, int NPa,
                               const int* __restrict__ fmask, const int* __restrict__ nbr,
                               const uint8_t* __restrict__ finfo, const int* __restrict__ perm) {
  using O = Order<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NFPP = O::NFPP;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_slots * Np) return;
  const int64_t s = i / Np;
  const int mnode = int(i - s * Np);
  const int64_t blk = s >> 5;
  const int lane = int(s & 31);
  auto idx = [&](int fld) { return ((blk * 4 + fld) * Np + mnode) * 32 + lane; };
  if (!(meta[s] & kMetaValid)) {
    for (int fld = 0; fld < 4; ++fld) out[idx(fld)] = real(0);
    return;
  }
  auto at = [&](int fld, int n) { return lam[((blk * 4 + fld) * Np + n) * 32 + lane]; };
  const double* g = geo + s * kGeo;
  const real* m = mat + s * kMat;
  // D_j^T applied to lambda_p and to each lambda_v_i at node mnode
  real dp[3] = {0, 0, 0}, dv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int j = 0; j < 3; ++j) {
    const real* row = Dt + int64_t(j * Np + mnode) * NPa;
    for (int n = 0; n < Np; ++n) {
      const real d = row[n];
      dp[j] += d * at(0, n);
      for (int c = 0; c < 3; ++c) dv[c][j] += d * at(1 + c, n);
    }
  }
  real op = 0, ov[3] = {0, 0, 0};
  for (int c = 0; c < 3; ++c)
    for (int j = 0; j < 3; ++j) {
      const real gij = real(g[3 * c + j]);
      op -= m[1] * gij * dv[c][j];
      ov[c] -= m[0] * gij * dp[j];
    }
  // faces that hold this node
  for (int f = 0; f < 4; ++f) {
    for (int jf = 0; jf < Nfp; ++jf) {
      if (fmask[f * 32 + jf] != mnode) continue;
      const real* t = adjt + s * (8 * NFPP) + f * 2 * NFPP;
      const real a = t[jf], b = t[NFPP + jf];
      const real taup = m[3 + f], tauv = m[7 + f];
      const uint8_t info = finfo[s * 4 + f];
      const int bc = finfo_bc(info);
      real sp = 0, sv = 0;
      if (bc == 0) {
        sp = taup * a - b;
        sv = tauv * b - a;
        const int64_t s2 = nbr[s * 4 + f];
        const int j2 = perm[finfo_perm(info) * 32 + jf];
        const real* t2 = adjt + s2 * (8 * NFPP) + finfo_face(info) * 2 * NFPP;
        const real a2 = t2[j2], b2 = t2[NFPP + j2];
        sp += b2 - taup * a2;
        sv += tauv * b2 - a2;
      } else if (bc == 1) {  // free surface
        sp = real(2) * (taup * a - b);
      } else if (bc == 2) {  // transparent
        sp = taup * a - b;
        sv = tauv * b - a;
      } else {  // rigid wall
        sv = real(2) * (tauv * b - a);
      }
      op += sp;
      for (int c = 0; c < 3; ++c) ov[c] += real(g[9 + 3 * f + c]) * sv;
    }
  }
  out[idx(0)] = op;
  for (int c = 0; c < 3; ++c) out[idx(1 + c)] = ov[c];
}

// lambda += h (a1 s0 + a2 s1 + a3 s2), elementwise over the whole field array
template <typename real>
__global__ void adj_update_kernel(real* __restrict__ lam, const real* __restrict__ s0, const real* __restrict__ s1,
                                  const real* __restrict__ s2, double h, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  lam[i] += real(h) * (real(AB::a1) * s0[i] + real(AB::a2) * s1[i] + real(AB::a3) * s2[i]);
}

// lambda_p -= coef res_r(col) l(x_r) for every receiver (receivers taken in order: deterministic)
template <int N, typename real>
__global__ void adj_inject_kernel(real* __restrict__ lam, const int64_t* __restrict__ rec_slot,
                                  const real* __restrict__ rec_row, int nrec, const double* __restrict__ res,
                                  int64_t n_time, int64_t col, double coef) {
  using O = Order<N>;
  constexpr int Np = O::Np;
  for (int n = threadIdx.x; n < Np; n += blockDim.x)
    for (int r = 0; r < nrec; ++r) {
      const int64_t s = rec_slot[r];
      const int64_t at = ((s >> 5) * 4 * Np + n) * 32 + (s & 31);
      lam[at] -= real(coef * res[int64_t(r) * n_time + col]) * rec_row[int64_t(r) * Np + n];
    }
}

// acc[s] += sum_m lambda_p[m] (q1_p[m] - q0_p[m] - F w[m]) (w on the source slot only)
template <int N, typename real>
__global__ void adj_grad_kernel(const real* __restrict__ lam, const real* __restrict__ q1, const real* __restrict__ q0,
                                int64_t n_slots, const int* __restrict__ meta, int64_t src_slot,
                                const real* __restrict__ w_src, double F, double* __restrict__ acc) {
  using O = Order<N>;
  constexpr int Np = O::Np;
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n_slots || !(meta[s] & kMetaValid)) return;
  const int64_t base = (s >> 5) * 4 * Np * 32 + (s & 31);
  double sum = 0.0;
  for (int m = 0; m < Np; ++m) {
    const int64_t at = base + int64_t(m) * 32;
    double dq = double(q1[at]) - double(q0[at]);
    if (s == src_slot) dq -= F * double(w_src[m]);
    sum += double(lam[at]) * dq;
  }
  acc[s] += sum;
}

}  // namespace ridg
