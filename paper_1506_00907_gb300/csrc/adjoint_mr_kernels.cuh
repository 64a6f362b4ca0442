// Discrete adjoint of the multi-rate scheme as the library runs it (reverse accumulation).
//
// Forward fine step tau (Algorithm 1 in the library's fused form), for every element k of an
// active level l (stride d, step h = d dt):
//   r = A_k(q_k, x_k)              x_k: the element's inbox slot tau mod 3 (its neighbours' traces)
//   ring: r_new <- r (the two older right-hand sides r1, r2 stay)
//   q_k <- q_k + h (a1 r + a2 r1 + a3 r2)                       (Eq. updateAB, at the step's start)
//   traces of q_k pushed into the neighbours' inbox slot (tau + d) mod 3, and, for elements with a
//   finer neighbour, traces of q_k + h (b1 r + b2 r1 + b3 r2) into slot (tau + d/2) mod 3
//   (Eq. updateABcoarse).
// Its reverse, per fine step from the last to the first, with mu = dJ/d(state):
//   pull:    the adjoint of each pushed trace is taken (and cleared) from the neighbour's inbox
//            adjoint; mu_q' = mu_q + T^T g_full, mu_h = T^T g_half; mu_q <- mu_q' + mu_h and the
//            ring adjoints gain h (a_s mu_q' + b_s mu_h) (adjml_pull_kernel);
//   rhs:     mu_r = the ring adjoint of r_new (then cleared); the volume transposes and the
//            element's own face traces go to mu_q, and the weights of the neighbour's traces to the
//            element's inbox adjoint at slot tau mod 3 (adjml_traces_kernel, adjml_rhs_kernel);
//   gradient: dJ/dc_k += (2/c_k) mu_r,p . (A q)_p, with A q the saved right-hand side less the
//            source term (in adjml_rhs_kernel).
// Every entry has one writer per pass: an element writes its own rows and clears only the inbox
// entries it filled in the forward run.  Layouts are the solver's (fields [K/32][4][Np][32], ring
// [3][fields], inboxes [3 slots][n_slots][4 faces][2][NFPP]); the face terms are those of the
// single-rate kernels (adjoint_kernels.cuh).
#pragma once
#include <cuda_runtime.h>

#include "adjoint_kernels.cuh"
#include "dispatch.hpp"

namespace ridg {


// per-column coefficients staged in shared memory, [k][32] (lanes of consecutive columns read
// consecutive words): traces: normals (12), alpha_f, beta_f, tau_p, tau_v (4 each); rhs: rx (9),
// normals (12), rho c^2, 1/rho
constexpr int kAdjMlTc = 28;
constexpr int kAdjMlRc = 23;

template <typename real>
__device__ __forceinline__ int adjml_level(const AdjMrArgs<real>& A, int64_t slot0) {
  int lev = 0;
  for (int l = 0; l < A.n_levels; ++l)
    if (slot0 >= A.level_begin[l]) lev = l;
  return lev;
}

// faces holding each node: sInv[m * 3 + i] = f * 32 + jf (or -1), from the table built on the host
template <int N>
__device__ __forceinline__ void adjml_inverse_fmask(const int* __restrict__ inv_fmask, int* sInv) {
  for (int i = threadIdx.x; i < Order<N>::Np * 3; i += blockDim.x) sInv[i] = inv_fmask[i];
}

// Reverse of the trace pushes and of the update.  First the adjoints of the traces this block's
// elements pushed are taken (and cleared) from the neighbours' inbox adjoints into shared memory, a
// fixed set of (column, face, face node) entries per thread with the neighbour and face-node tables
// staged, so that a thread's loads are all in flight together; the per-column normals and flags are
// staged once.  Then a thread per (node, column) sums, per
// node, the entries of the faces that hold it (in face order) and updates mu and the ring adjoints.
template <int N, typename real>
constexpr size_t adjml_pull_smem() {
  return size_t(2) * 4 * 2 * Order<N>::Nfp * 33 * sizeof(real);
}

// blocks per SM the pull kernel's registers are held to: three at low orders in FP32 (its loads are in
// flight together, so more resident warps hide more latency), the compiler's choice otherwise
template <int N, typename real>
constexpr int adjml_pull_min_blocks() {
  return (sizeof(real) == 4 && N <= 4) ? 3 : 1;
}

template <int N, typename real>
__global__ void __launch_bounds__(256, adjml_pull_min_blocks<N, real>()) adjml_pull_kernel(AdjMrArgs<real> A) {
  using O = Order<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NFPP = O::NFPP;
  __shared__ int sInv[Np * 3];
  __shared__ real sN[12][32];  // outward normals per column
  __shared__ int sMeta[32];
  __shared__ uint8_t sInfo[32 * 4];
  __shared__ int sNbr[32 * 4];
  __shared__ int sPerm[6 * 32];
  // full (set 0) and half-step (set 1) trace adjoints per face, (p, v), face node and column; columns
  // innermost with a stride of 33 per face node, so that neither lanes over columns nor lanes over
  // face nodes meet in a bank
  extern __shared__ __align__(16) unsigned char smem_pull[];
  real* sG = reinterpret_cast<real*>(smem_pull);
  auto G = [&](int set, int c, int f, int comp, int jf) -> real& {
    return sG[(((set * 4 + f) * 2 + comp) * Nfp + jf) * 33 + c];
  };
  const int64_t slot0 = A.slot_lo + int64_t(blockIdx.x) * 32;
  const int64_t blk = slot0 >> 5;
  const int lev = adjml_level(A, slot0);
  const real h = A.h[lev];
  const int64_t qsize = (A.n_slots >> 5) * 4 * Np * 32;
  const int64_t tsz = A.n_slots * (8 * NFPP);
  real* rn = A.mu_ring + A.ring_new[lev] * qsize;
  real* r1 = A.mu_ring + A.ring_old1[lev] * qsize;
  real* r2 = A.mu_ring + A.ring_old2[lev] * qsize;
  real* xfull = A.mu_in + A.slot_full[lev] * tsz;
  real* xhalf = A.mu_in + A.slot_half[lev] * tsz;
  adjml_inverse_fmask<N>(A.inv_fmask, sInv);
  for (int i = threadIdx.x; i < 32; i += blockDim.x) sMeta[i] = A.meta[slot0 + i];
  for (int i = threadIdx.x; i < 32 * 4; i += blockDim.x) {
    sInfo[i] = A.finfo[slot0 * 4 + i];
    sNbr[i] = A.nbr[slot0 * 4 + i];
  }
  for (int i = threadIdx.x; i < 6 * 32; i += blockDim.x) sPerm[i] = A.perm[i];
  for (int i = threadIdx.x; i < 12 * 32; i += blockDim.x) {
    const int k = i >> 5, c = i & 31;
    sN[k][c] = real(A.geo[(slot0 + c) * kGeo + 9 + k]);
  }
  __syncthreads();
  {
    // thread per (column, face, face node) entry, a fixed number per thread: every entry's neighbour
    // row and permuted index come from shared memory, so all of a thread's loads are issued before any
    // of its clearing stores
    constexpr int NE = 32 * 4 * Nfp;
    constexpr int PER = (NE + 255) / 256;  // launched with 256 threads
    real gp[PER], gv[PER], hp[PER], hv[PER];
    int64_t at[PER];
    bool take[PER], half[PER];
    // entry e = (c * 4 + f) * Nfp + jf: lanes run over a face's nodes, whose row is contiguous
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int ee = e < NE ? e : 0;
      const int c = ee / (4 * Nfp), fj = ee - c * (4 * Nfp), f = fj / Nfp, jf = fj - f * Nfp;
      const int meta = sMeta[c];
      const uint8_t info = sInfo[c * 4 + f];
      take[u] = e < NE && (meta & kMetaValid) && finfo_bc(info) == 0;  // boundary faces push nothing
      half[u] = take[u] && (meta & kMetaHalf);
      at[u] = take[u] ? int64_t(sNbr[c * 4 + f]) * (8 * NFPP) + finfo_face(info) * 2 * NFPP +
                            sPerm[finfo_perm(info) * 32 + jf]
                      : 0;
      gp[u] = take[u] ? xfull[at[u]] : real(0);
      gv[u] = take[u] ? xfull[at[u] + NFPP] : real(0);
      hp[u] = half[u] ? xhalf[at[u]] : real(0);
      hv[u] = half[u] ? xhalf[at[u] + NFPP] : real(0);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + 256 * u;
      if (e >= NE) continue;
      const int c = e / (4 * Nfp), fj = e - c * (4 * Nfp), f = fj / Nfp, jf = fj - f * Nfp;
      G(0, c, f, 0, jf) = gp[u];
      G(0, c, f, 1, jf) = gv[u];
      G(1, c, f, 0, jf) = hp[u];
      G(1, c, f, 1, jf) = hv[u];
      if (take[u]) {
        xfull[at[u]] = real(0);
        xfull[at[u] + NFPP] = real(0);
      }
      if (half[u]) {
        xhalf[at[u]] = real(0);
        xhalf[at[u] + NFPP] = real(0);
      }
    }
  }
  __syncthreads();
  for (int item = threadIdx.x; item < Np * 32; item += blockDim.x) {
    const int m = item >> 5, c = item & 31;
    const int meta = sMeta[c];
    if (!(meta & kMetaValid)) continue;
    const bool half = (meta & kMetaHalf) != 0;
    const int64_t s = slot0 + c;
    real gq[4] = {0, 0, 0, 0}, hq[4] = {0, 0, 0, 0};
    for (int k = 0; k < 3; ++k) {
      const int e = sInv[m * 3 + k];
      if (e < 0) break;
      const int f = e >> 5, jf = e & 31;
      if (finfo_bc(sInfo[c * 4 + f]) != 0) continue;  // boundary faces push nothing
      // the pushed pair is (p, -n.v) in this element's normal: its adjoint goes to p and to v
      const real gp = G(0, c, f, 0, jf), gv = G(0, c, f, 1, jf);
      gq[0] += gp;
#pragma unroll
      for (int i = 0; i < 3; ++i) gq[1 + i] -= sN[3 * f + i][c] * gv;
      if (half) {
        const real hp = G(1, c, f, 0, jf), hv = G(1, c, f, 1, jf);
        hq[0] += hp;
#pragma unroll
        for (int i = 0; i < 3; ++i) hq[1 + i] -= sN[3 * f + i][c] * hv;
      }
    }
    // every value is read before any is written (the arrays may alias as far as the compiler knows),
    // so the sixteen loads are in flight together
    real vm[4], vn[4], v1[4], v2[4];
#pragma unroll
    for (int fld = 0; fld < 4; ++fld) {
      const int64_t at = ((blk * 4 + fld) * Np + m) * 32 + c;
      vm[fld] = A.mu[at];
      vn[fld] = rn[at];
      v1[fld] = r1[at];
      v2[fld] = r2[at];
    }
#pragma unroll
    for (int fld = 0; fld < 4; ++fld) {
      const int64_t at = ((blk * 4 + fld) * Np + m) * 32 + c;
      const real mq = vm[fld] + gq[fld], mh = hq[fld];
      A.mu[at] = mq + mh;
      rn[at] = vn[fld] + h * (real(AB::a1) * mq + real(AB::b1) * mh);
      r1[at] = v1[fld] + h * (real(AB::a2) * mq + real(AB::b2) * mh);
      r2[at] = v2[fld] + h * (real(AB::a3) * mq + real(AB::b3) * mh);
    }
  }
}

// Adjoint traces of mu_r (the ring adjoint of this step's right-hand side): per face node the
// weights of the jumps, w_p = -tau_p at + bt and w_v = at - tau_v bt with at = alpha_f L_f^T mu_r,p
// and bt = beta_f L_f^T (n_f . mu_r,v).  The neighbour's traces receive (w_p, w_v) in the element's
// inbox adjoint; the element's own traces receive minus them, with the boundary ghosts folded in,
// in the scratch rows (a half-warp per face and four columns, LIFT^T staged where it fits).
template <int N, typename real>
__global__ void adjml_traces_kernel(AdjMrArgs<real> A) {
  using O = Order<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NFPP = O::NFPP;
  constexpr bool STAGE_LT = adj_traces_stage_lt<N, real>();
  extern __shared__ __align__(16) unsigned char smem_adjml[];
  real* sL = reinterpret_cast<real*>(smem_adjml);  // [4][Np][32]
  real* sV = sL + 4 * Np * 32;                     // [4 faces][Np][32]: n_f . mu_r,v
  real* sC = sV + 4 * Np * 32;                     // [kAdjMlTc][32]: normals, alpha_f, beta_f, tau_p, tau_v
  real* sLt = sC + kAdjMlTc * 32;                  // [Np][4 Nfp] (if staged): LIFT^T, lanes read consecutive entries
  int* sI = reinterpret_cast<int*>(sLt + (STAGE_LT ? Np * 4 * Nfp : 0));  // [4][32] boundary kinds, [32] valid
  const int64_t slot0 = A.slot_lo + int64_t(blockIdx.x) * 32;
  const int64_t blk = slot0 >> 5;
  const int lev = adjml_level(A, slot0);
  const int64_t qsize = (A.n_slots >> 5) * 4 * Np * 32;
  load_lambda_tile<N, real>(A.mu_ring + A.ring_new[lev] * qsize, sL, blk);
  if constexpr (STAGE_LT)
    for (int i = threadIdx.x; i < 4 * Nfp * Np; i += blockDim.x) {
      const int fj = i / Np, n = i - fj * Np;
      cp_async_small<sizeof(real)>(sLt + n * (4 * Nfp) + fj, A.Lt + int64_t(fj) * A.NPa + n);
    }
  cp_async_commit();
  for (int i = threadIdx.x; i < kAdjMlTc * 32; i += blockDim.x) {
    const int k = i >> 5, c = i & 31;
    const int64_t s = slot0 + c;
    const double* g = A.geo + s * kGeo;
    const real* mt = A.mat + s * kMat;
    sC[i] = k < 12 ? real(g[9 + k]) : k < 20 ? real(-0.5 * g[21 + (k & 3)]) * mt[k < 16 ? 0 : 1] : mt[k - 17];
  }
  for (int i = threadIdx.x; i < 5 * 32; i += blockDim.x)
    sI[i] = i < 128 ? finfo_bc(A.finfo[(slot0 + (i & 31)) * 4 + (i >> 5)])
                    : int((A.meta[slot0 + (i & 31)] & kMetaValid) != 0);
  cp_async_wait_all();
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * Np * 32; i += blockDim.x) {
    const int f = i / (Np * 32), r = i - f * (Np * 32), n = r >> 5, c = r & 31;
    const real* nf = sC + 3 * f * 32 + c;
    sV[i] = nf[0] * sL[(1 * Np + n) * 32 + c] + nf[32] * sL[(2 * Np + n) * 32 + c] + nf[64] * sL[(3 * Np + n) * 32 + c];
  }
  __syncthreads();
  // half-warp per (face, group of four columns), lanes over the face's nodes: each LIFT^T entry serves
  // four columns, whose mu_r values come in one vector load per node.  Per face node the weights of the
  // jumps, w_p = -tau_p at + bt and w_v = at - tau_v bt (at = alpha_f L_f^T mu_r,p, bt = beta_f L_f^T
  // (n_f . mu_r,v)); the neighbour's traces receive them in the element's inbox adjoint, the element's
  // own traces minus them, with the boundary ghosts folded in, in its scratch rows.
  real* xin = A.mu_in + int64_t(A.slot_read) * A.n_slots * (8 * NFPP);
  constexpr int NJ = (Nfp + 15) / 16;
  const int hw = threadIdx.x >> 4, lane16 = threadIdx.x & 15, nhw = blockDim.x >> 4;
  for (int item = hw; item < 4 * 8; item += nhw) {
    const int f = item >> 3, c0 = (item & 7) * 4;
    const real* vf = sV + f * Np * 32;
#pragma unroll
    for (int t = 0; t < NJ; ++t) {
      const int j = lane16 + 16 * t;
      if (j >= Nfp) {
        if (j < NFPP)  // pad words of the own rows: their 32-byte sectors are written whole
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            real* ow = A.own + (slot0 + c0 + u) * (8 * NFPP) + f * 2 * NFPP;
            ow[j] = real(0);
            ow[NFPP + j] = real(0);
          }
        continue;
      }
      real ap[4] = {0, 0, 0, 0}, av[4] = {0, 0, 0, 0};
#pragma unroll 4
      for (int n = 0; n < Np; ++n) {
        const real l = STAGE_LT ? sLt[n * (4 * Nfp) + f * Nfp + j] : A.Lt[int64_t(f * Nfp + j) * A.NPa + n];
        real lp[4], lv[4];
        load4(sL + n * 32 + c0, lp);
        load4(vf + n * 32 + c0, lv);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ap[u] += l * lp[u];
          av[u] += l * lv[u];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u;
        const int64_t s = slot0 + c;
        real* ow = A.own + s * (8 * NFPP) + f * 2 * NFPP;
        if (!sI[128 + c]) {
          ow[j] = real(0);
          ow[NFPP + j] = real(0);
          continue;
        }
        const real* cc = sC + c;  // coefficient k of this column at cc[32 k]
        const real a = cc[32 * (12 + f)] * ap[u], b = cc[32 * (16 + f)] * av[u];
        const real taup = cc[32 * (20 + f)], tauv = cc[32 * (24 + f)];
        const real wp = -taup * a + b, wv = a - tauv * b;
        const int bc = sI[f * 32 + c];
        real op = 0, ov = 0;
        if (bc == 0) {
          op = -wp;
          ov = -wv;
          real* x = xin + s * (8 * NFPP) + f * 2 * NFPP;
          x[j] += wp;
          x[NFPP + j] += wv;
        } else if (bc == 1) {  // free surface: jp = -2 p-, jv = 0
          op = real(-2) * wp;
        } else if (bc == 2) {  // transparent: jp = -p-, jv = -vn-
          op = -wp;
          ov = -wv;
        } else {  // rigid wall: jp = 0, jv = -2 vn-
          ov = real(-2) * wv;
        }
        ow[j] = op;
        ow[NFPP + j] = ov;
      }
    }
  }
}

// mu_q += (volume transposes) mu_r + the own-trace weights at the face nodes; the ring adjoint of
// this step's right-hand side is cleared (thread per (node, column); with 256 threads a thread
// keeps one column).  acc[slot] += sum_m mu_r,p (r_p - F w)_m, the source-free right-hand side,
// summed in a fixed order (eight warp partial sums, added in FP64).
// the interleaved derivative rows (D_0, D_1, D_2, 0)[n][m] are staged in shared memory where they
// take at most 24 KB (FP32 up to N = 4, FP64 up to N = 3): every thread of a warp reads the same
// entry, a broadcast from shared memory instead of an L1 lookup per entry
template <int N, typename real>
constexpr bool adjml_rhs_stage_d() {
  return size_t(Order<N>::Np) * Order<N>::Np * 4 * sizeof(real) <= 24 * 1024;
}

template <int N, typename real>
__global__ void __launch_bounds__(256) adjml_rhs_kernel(AdjMrArgs<real> A) {
  using O = Order<N>;
  constexpr int Np = O::Np, NFPP = O::NFPP;
  constexpr bool STAGE_D = adjml_rhs_stage_d<N, real>();
  constexpr int DS = STAGE_D ? Np * Np * 4 : 0;
  extern __shared__ __align__(16) unsigned char smem_adjml[];
  real* sD = reinterpret_cast<real*>(smem_adjml);  // [Np][Np][4] (if staged)
  real* sL = sD + DS;                              // [4][Np][32]
  real* sC = sL + 4 * Np * 32;                     // [kAdjMlRc][32]: rx, normals, rho c^2, 1/rho
  int* sInv = reinterpret_cast<int*>(sC + kAdjMlRc * 32);  // [Np][3]
  int* sValid = sInv + Np * 3;                             // [32]
  const int64_t slot0 = A.slot_lo + int64_t(blockIdx.x) * 32;
  const int64_t blk = slot0 >> 5;
  const int lev = adjml_level(A, slot0);
  const int64_t qsize = (A.n_slots >> 5) * 4 * Np * 32;
  real* rnew = A.mu_ring + A.ring_new[lev] * qsize + blk * 4 * Np * 32;
  load_lambda_tile<N, real>(A.mu_ring + A.ring_new[lev] * qsize, sL, blk);
  if constexpr (STAGE_D) {
    constexpr int CH = DS * int(sizeof(real)) / 16;
    const char* src = reinterpret_cast<const char*>(A.Dt4);
    char* dst = reinterpret_cast<char*>(sD);
    for (int i = threadIdx.x; i < CH; i += blockDim.x) cp_async_bytes16(dst + 16 * i, src + 16 * i);
  }
  cp_async_commit();
  for (int i = threadIdx.x; i < kAdjMlRc * 32; i += blockDim.x) {
    const int k = i >> 5, c = i & 31;
    const int64_t s = slot0 + c;
    sC[i] = k < 21 ? real(A.geo[s * kGeo + k]) : A.mat[s * kMat + (k - 21)];
  }
  for (int i = threadIdx.x; i < 32; i += blockDim.x) sValid[i] = (A.meta[slot0 + i] & kMetaValid) != 0;
  adjml_inverse_fmask<N>(A.inv_fmask, sInv);
  cp_async_wait_all();
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * Np * 32; i += blockDim.x) rnew[i] = real(0);
  __shared__ double part[8][32];
  real gsum = 0;
  for (int item = threadIdx.x; item < Np * 32; item += blockDim.x) {
    const int m = item >> 5, c = item & 31;
    const int64_t s = slot0 + c;
    if (!sValid[c]) continue;
    {
      real r = A.rsaved[((blk * 4 + 0) * Np + m) * 32 + c];
      if (s == A.src_slot) r -= A.F * A.w_src[m];
      gsum += sL[(0 * Np + m) * 32 + c] * r;
    }
    const real* cc = sC + c;  // coefficient k of this column at cc[32 k]
    real dp[3] = {0, 0, 0}, dv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int n = 0; n < Np; ++n) {
      real d[3];
      if constexpr (STAGE_D)
        load_d3(sD + (m * Np + n) * 4, d);
      else
        load_d3(A.Dt4 + (int64_t(m) * Np + n) * 4, d);
      const real lp = sL[(0 * Np + n) * 32 + c];
      const real lv[3] = {sL[(1 * Np + n) * 32 + c], sL[(2 * Np + n) * 32 + c], sL[(3 * Np + n) * 32 + c]};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        dp[j] += d[j] * lp;
#pragma unroll
        for (int i = 0; i < 3; ++i) dv[i][j] += d[j] * lv[i];
      }
    }
    real op = 0, ov[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const real gij = cc[32 * (3 * i + j)];
        op -= cc[32 * 22] * gij * dv[i][j];
        ov[i] -= cc[32 * 21] * gij * dp[j];
      }
    for (int k = 0; k < 3; ++k) {
      const int e = sInv[m * 3 + k];
      if (e < 0) break;
      const int f = e >> 5, jf = e & 31;
      const real* ow = A.own + s * (8 * NFPP) + f * 2 * NFPP;
      op += ow[jf];
#pragma unroll
      for (int i = 0; i < 3; ++i) ov[i] += cc[32 * (9 + 3 * f + i)] * ow[NFPP + jf];
    }
    A.mu[((blk * 4 + 0) * Np + m) * 32 + c] += op;
#pragma unroll
    for (int i = 0; i < 3; ++i) A.mu[((blk * 4 + 1 + i) * Np + m) * 32 + c] += ov[i];
  }
  part[threadIdx.x >> 5][threadIdx.x & 31] = double(gsum);
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = part[0][threadIdx.x];
#pragma unroll
    for (int k = 1; k < 8; ++k) t += part[k][threadIdx.x];
    A.acc[slot0 + threadIdx.x] += t;
  }
}

template <int N, typename real>
constexpr size_t adjml_traces_smem() {
  return (size_t(8) * Order<N>::Np * 32 + size_t(kAdjMlTc) * 32 +
          (adj_traces_stage_lt<N, real>() ? size_t(4) * Order<N>::Nfp * Order<N>::Np : 0)) *
             sizeof(real) +
         size_t(5) * 32 * sizeof(int);
}
template <int N, typename real>
constexpr size_t adjml_rhs_smem() {
  return (size_t(4) * Order<N>::Np * 32 + size_t(kAdjMlRc) * 32 +
          (adjml_rhs_stage_d<N, real>() ? size_t(Order<N>::Np) * Order<N>::Np * 4 : 0)) *
             sizeof(real) +
         (size_t(Order<N>::Np) * 3 + 32) * sizeof(int);
}

}  // namespace ridg
