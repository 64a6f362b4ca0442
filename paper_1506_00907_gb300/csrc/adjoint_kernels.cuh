// Discrete adjoint of the single-rate scheme: the transposed right-hand-side operator A^T, the
// adjoint Adams-Bashforth recursion and the velocity gradient (CUDA cores, any precision).
//
// Forward operator (Sec. 3.1, Eqs. dgLocalSchemeP/U with the penalty fluxes of Eqs. weakFormP/V):
//   r_p   = -rho c^2 sum_j D_j (sum_i g_ij v_i) + sum_f L_f [alpha_f (jv - tau_p jp)]
//   r_v_i = -(1/rho) sum_j g_ij D_j p          + sum_f n_fi L_f [beta_f (jp - tau_v jv)]
// with alpha_f = -Fs_f rho c^2 / 2, beta_f = -Fs_f / (2 rho), jp = p+ - p-, jv = vn+ - vn-.
// Its transpose applied to lambda, element by element:
//   volume:  (A^T l)_v_i = -rho c^2 sum_j g_ij D_j^T l_p,  (A^T l)_p = -(1/rho) sum_ij g_ij D_j^T l_v_i
//   faces:   adjoint traces at = alpha_f L_f^T l_p, bt = beta_f L_f^T (n_f . l_v) (adj_traces_kernel,
//            which also pushes them into the neighbour's inbox);
//            the flux depends on jp with weight (-tau_p at + bt) and on jv with weight (at - tau_v bt),
//            so the interior traces (p-, vn-) of the element receive minus these weights and, through
//            jp, jv of the neighbour's flux, the neighbour's weights (its vn+ is minus this element's
//            n.v); boundary ghosts fold p+ and vn+ into p- and vn- (free: jp = -2p-, jv = 0;
//            transparent: jp = -p-, jv = -vn-; rigid: jp = 0, jv = -2vn-).
// Layouts are the solver's: fields [K/32][4][Np][32] in the device node numbering, adjoint traces
// and inboxes [slot][4 faces][2][NFPP]; the derivative matrices interleaved, Dt4 [Np][Np][4] with
// (D_0, D_1, D_2, 0)[n][m] at (m, n), so that one vector load brings the three entries a node needs.
#pragma once
#include <cuda_runtime.h>

#include "step_kernel.cuh"

namespace ridg {

// One block per 32 element slots (one column block of the field layout).  The block's lambda tile
// is staged in shared memory, [4][Np][32]: thread (row, column c) reads row entries of consecutive
// columns (no bank conflicts), and the operator rows it multiplies by are the same for the whole
// warp (broadcast loads).  The tiles are fetched with asynchronous copies (global to shared
// without a register round trip, all in flight at once); the caller commits and waits for them.
template <int N, typename real>
__device__ __forceinline__ void load_lambda_tile(const real* __restrict__ lam, real* sL, int64_t blk) {
  using O = Order<N>;
  constexpr int CH = 4 * O::Np * 32 * int(sizeof(real)) / 16;  // 16-byte chunks of the contiguous tile
  const char* src = reinterpret_cast<const char*>(lam + blk * 4 * O::Np * 32);
  char* dst = reinterpret_cast<char*>(sL);
  for (int i = threadIdx.x; i < CH; i += blockDim.x) cp_async_bytes16(dst + 16 * i, src + 16 * i);
}

// per-column coefficients staged in shared memory, [k][32]: lanes of consecutive columns read
// consecutive words.  Traces: normals (12) and the face factors alpha_f, beta_f (8).  A^T: rx (9),
// normals (12), rho c^2, 1/rho, tau_p[4], tau_v[4]; the boundary kinds follow as ints [4][32].
constexpr int kAdjTc = 20;
constexpr int kAdjRc = 31;

// shared memory of the two kernels (the LIFT^T columns are staged where they still fit)
template <int N, typename real>
constexpr bool adj_traces_stage_lt() {
  return (size_t(8) * Order<N>::Np * 32 + size_t(kAdjTc) * 32 + size_t(4) * Order<N>::Nfp * Order<N>::Np) *
             sizeof(real) <=
         227 * 1024;
}
template <int N, typename real>
constexpr size_t adj_traces_smem() {
  return (size_t(8) * Order<N>::Np * 32 + size_t(kAdjTc) * 32 +
          (adj_traces_stage_lt<N, real>() ? size_t(4) * Order<N>::Nfp * Order<N>::Np : 0)) *
         sizeof(real);
}
template <int N, typename real>
constexpr size_t adj_rhs_smem() {
  return (size_t(4) * Order<N>::Np * 32 + size_t(2) * 32 * (8 * Order<N>::NFPP + 1) + size_t(kAdjRc) * 32) *
             sizeof(real) +
         (size_t(Order<N>::Np) * 3 + size_t(4) * 32) * sizeof(int);
}

// four consecutive entries (16-byte aligned for float, two 16-byte loads for double)
__device__ __forceinline__ void load4(const float* p, float v[4]) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x;
  v[1] = x.y;
  v[2] = x.z;
  v[3] = x.w;
}
__device__ __forceinline__ void load4(const double* p, double v[4]) {
  const double2 x = *reinterpret_cast<const double2*>(p), y = *reinterpret_cast<const double2*>(p + 2);
  v[0] = x.x;
  v[1] = x.y;
  v[2] = y.x;
  v[3] = y.y;
}

// Adjoint traces of every face of the block's elements (at = alpha_f L_f^T l_p, bt = beta_f L_f^T
// (n_f . l_v)), written to the element's own rows and, for interior faces, pushed into the
// neighbour's inbox at the neighbour's face-node index of each node (the correspondence codes of
// the two sides are mutually inverse).
template <int N, typename real>
__global__ void adj_traces_kernel(const real* __restrict__ lam, real* __restrict__ own, real* __restrict__ inbox,
                                  int64_t n_slots, const double* __restrict__ geo, const real* __restrict__ mat,
                                  const int* __restrict__ meta, const real* __restrict__ Lt, int NPa,
                                  const int* __restrict__ nbr, const uint8_t* __restrict__ finfo,
                                  const int* __restrict__ perm) {
  using O = Order<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NFPP = O::NFPP;
  constexpr bool STAGE_LT = adj_traces_stage_lt<N, real>();
  extern __shared__ __align__(16) unsigned char smem_adj[];
  real* sL = reinterpret_cast<real*>(smem_adj);  // [4][Np][32]
  real* sV = sL + 4 * Np * 32;                   // [4 faces][Np][32]: n_f . lambda_v
  real* sC = sV + 4 * Np * 32;                   // [kAdjTc][32]: normals, alpha_f, beta_f
  real* sLt = sC + kAdjTc * 32;                  // [Np][4 Nfp]: LIFT^T columns, lanes read consecutive entries
  const int64_t blk = blockIdx.x;
  load_lambda_tile<N, real>(lam, sL, blk);
  if constexpr (STAGE_LT)
    for (int i = threadIdx.x; i < 4 * Nfp * Np; i += blockDim.x) {
      const int fj = i / Np, n = i - fj * Np;
      cp_async_small<sizeof(real)>(sLt + n * (4 * Nfp) + fj, Lt + int64_t(fj) * NPa + n);
    }
  cp_async_commit();
  for (int i = threadIdx.x; i < kAdjTc * 32; i += blockDim.x) {
    const int k = i >> 5, c = i & 31;
    const int64_t s = blk * 32 + c;
    const double* g = geo + s * kGeo;
    sC[i] = k < 12 ? real(g[9 + k]) : real(-0.5 * g[21 + (k & 3)]) * mat[s * kMat + (k < 16 ? 0 : 1)];
  }
  cp_async_wait_all();
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * Np * 32; i += blockDim.x) {
    const int f = i / (Np * 32), r = i - f * (Np * 32), n = r >> 5, c = r & 31;
    const real* nf = sC + 3 * f * 32 + c;
    sV[i] = nf[0] * sL[(1 * Np + n) * 32 + c] + nf[32] * sL[(2 * Np + n) * 32 + c] + nf[64] * sL[(3 * Np + n) * 32 + c];
  }
  __syncthreads();
  // half-warp per (face, group of four columns) item, lanes over the face's nodes: each LIFT^T entry
  // a lane reads serves four columns, whose lambda values come in one vector load per node; the
  // element's own rows and the neighbour's inbox row are written as one 64-byte segment each
  constexpr int NJ = (Nfp + 15) / 16;
  const int hw = threadIdx.x >> 4, lane16 = threadIdx.x & 15, nhw = blockDim.x >> 4;
  for (int item = hw; item < 4 * 8; item += nhw) {
    const int f = item >> 3, c0 = (item & 7) * 4;
    const real* vf = sV + f * Np * 32;
#pragma unroll
    for (int t = 0; t < NJ; ++t) {
      const int j = lane16 + 16 * t;
      if (j >= Nfp) continue;
      real ap[4] = {0, 0, 0, 0}, av[4] = {0, 0, 0, 0};
#pragma unroll 4
      for (int n = 0; n < Np; ++n) {
        const real l = STAGE_LT ? sLt[n * (4 * Nfp) + f * Nfp + j] : Lt[int64_t(f * Nfp + j) * NPa + n];
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
        const int64_t s = blk * 32 + c;
        real* out = own + s * (8 * NFPP) + f * 2 * NFPP;
        if (!(meta[s] & kMetaValid)) {
          out[j] = real(0);
          out[NFPP + j] = real(0);
          continue;
        }
        const real a = sC[(12 + f) * 32 + c] * ap[u], b = sC[(16 + f) * 32 + c] * av[u];
        out[j] = a;
        out[NFPP + j] = b;
        const uint8_t info = finfo[s * 4 + f];
        if (finfo_bc(info) == 0) {
          const int64_t s2 = nbr[s * 4 + f];
          const int j2 = perm[finfo_perm(info) * 32 + j];
          real* x = inbox + s2 * (8 * NFPP) + finfo_face(info) * 2 * NFPP;
          x[j2] = a;
          x[NFPP + j2] = b;
        }
      }
    }
  }
}

// the three derivative entries at Dt4 + 4 (m Np + n)
__device__ __forceinline__ void load_d3(const float* p, float d[3]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  d[0] = v.x;
  d[1] = v.y;
  d[2] = v.z;
}
__device__ __forceinline__ void load_d3(const double* p, double d[3]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  d[0] = v.x;
  d[1] = v.y;
  d[2] = p[2];
}

// A^T lambda for the block's elements: the transposed volume terms (D_j^T rows, broadcast over the
// warp) and, at each face node, the weights of the jumps from the element's own adjoint traces and
// from the neighbour's (its inbox), with the boundary ghosts folded in.  With s1 != null the block
// then applies the adjoint Adams-Bashforth update to its own lambda tile, in place (no other block
// reads it): lam += h (a1 A^T lam + a2 s1 + a3 s2).
template <int N, typename real>
__global__ void __launch_bounds__(256, N <= 4 ? 4 : 2) adj_rhs_kernel(real* lam, const real* __restrict__ own, const real* __restrict__ inbox,
                               real* __restrict__ out, int64_t n_slots, const double* __restrict__ geo,
                               const real* __restrict__ mat, const int* __restrict__ meta,
                               const real* __restrict__ Dt4, const int* __restrict__ fmask,
                               const uint8_t* __restrict__ finfo, const real* __restrict__ s1,
                               const real* __restrict__ s2, real h) {
  using O = Order<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NFPP = O::NFPP;
  constexpr int OS = 8 * NFPP + 1;  // trace rows of one slot, padded: column-wise reads hit distinct banks
  extern __shared__ __align__(16) unsigned char smem_adj[];
  real* sL = reinterpret_cast<real*>(smem_adj);  // [4][Np][32]
  real* sOwn = sL + 4 * Np * 32;                 // [32][OS]
  real* sIn = sOwn + 32 * OS;                    // [32][OS]
  real* sC = sIn + 32 * OS;                      // [kAdjRc][32]: rx, normals, rho c^2, 1/rho, tau_p, tau_v
  int* sInv = reinterpret_cast<int*>(sC + kAdjRc * 32);  // [Np][3]: f * 32 + jf of the faces holding node m
  int* sBc = sInv + Np * 3;                              // [4][32]: boundary kind of each face
  const int64_t blk = blockIdx.x;
  load_lambda_tile<N, real>(lam, sL, blk);
  for (int i = threadIdx.x; i < 32 * 8 * NFPP; i += blockDim.x) {
    const int c = i / (8 * NFPP), r = i - c * (8 * NFPP);
    cp_async_small<sizeof(real)>(sOwn + c * OS + r, own + (blk * 32) * (8 * NFPP) + i);
    cp_async_small<sizeof(real)>(sIn + c * OS + r, inbox + (blk * 32) * (8 * NFPP) + i);
  }
  cp_async_commit();
  for (int i = threadIdx.x; i < kAdjRc * 32; i += blockDim.x) {
    const int k = i >> 5, c = i & 31;
    const int64_t s = blk * 32 + c;
    // geo[0..20] are rx and the normals; mat[0], mat[1] and mat[3..10] follow at 21..30
    sC[i] = k < 21 ? real(geo[s * kGeo + k]) : mat[s * kMat + (k < 23 ? k - 21 : k - 20)];
  }
  for (int i = threadIdx.x; i < 4 * 32; i += blockDim.x) sBc[i] = finfo_bc(finfo[(blk * 32 + (i & 31)) * 4 + (i >> 5)]);
  for (int m = threadIdx.x; m < Np; m += blockDim.x) {
    int cnt = 0;
    for (int f = 0; f < 4; ++f)
      for (int jf = 0; jf < Nfp; ++jf)
        if (fmask[f * 32 + jf] == m && cnt < 3) sInv[m * 3 + cnt++] = f * 32 + jf;
    for (; cnt < 3; ++cnt) sInv[m * 3 + cnt] = -1;
  }
  cp_async_wait_all();
  __syncthreads();
  // thread per (row pair, column): the rows r and r + H of one column share every lambda value they
  // read (FP32; FP64 takes one row per thread, for its registers)
  constexpr int RT = sizeof(real) == 4 ? 2 : 1;
  constexpr int H = (Np + RT - 1) / RT;
  for (int item = threadIdx.x; item < H * 32; item += blockDim.x) {
    const int r = item >> 5, c = item & 31;  // warp: one row (pair) of 32 columns
    const int64_t s = blk * 32 + c;
    const bool valid = (meta[s] & kMetaValid) != 0;
    auto idx = [&](int fld, int mnode) { return ((blk * 4 + fld) * Np + mnode) * 32 + c; };
    // out = r and, with s1, lam += h (a1 r + a2 s1 + a3 s2) for the four fields of each row; the
    // older terms are loaded first, so that their latency hides behind the contraction
    real older[RT][4];
#pragma unroll
    for (int t = 0; t < RT; ++t) {
      const int mnode = r + t * H < Np ? r + t * H : Np - 1;
#pragma unroll
      for (int fld = 0; fld < 4; ++fld)
        older[t][fld] = s1 ? real(AB::a2) * s1[idx(fld, mnode)] + real(AB::a3) * s2[idx(fld, mnode)] : real(0);
    }
    real dp[RT][3], dv[RT][3][3];
#pragma unroll
    for (int t = 0; t < RT; ++t)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        dp[t][j] = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) dv[t][i][j] = 0;
      }
    if (valid) {
      const real* dm[RT];
#pragma unroll
      for (int t = 0; t < RT; ++t) dm[t] = Dt4 + int64_t(r + t * H < Np ? r + t * H : Np - 1) * Np * 4;
#pragma unroll 4
      for (int n = 0; n < Np; ++n) {
        const real lp = sL[(0 * Np + n) * 32 + c];
        const real lv[3] = {sL[(1 * Np + n) * 32 + c], sL[(2 * Np + n) * 32 + c], sL[(3 * Np + n) * 32 + c]};
#pragma unroll
        for (int t = 0; t < RT; ++t) {
          real d[3];
          load_d3(dm[t] + 4 * n, d);
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            dp[t][j] += d[j] * lp;
#pragma unroll
            for (int i = 0; i < 3; ++i) dv[t][i][j] += d[j] * lv[i];
          }
        }
      }
    }
    const real* cc = sC + c;  // coefficient k of this column at cc[32 k]
#pragma unroll
    for (int t = 0; t < RT; ++t) {
      const int mnode = r + t * H;
      if (mnode >= Np) break;
      auto store = [&](int fld, real v) {
        const int64_t at = idx(fld, mnode);
        out[at] = v;
        if (s1) lam[at] = sL[(fld * Np + mnode) * 32 + c] + h * (real(AB::a1) * v + older[t][fld]);
      };
      if (!valid) {
        for (int fld = 0; fld < 4; ++fld) store(fld, real(0));
        continue;
      }
      real op = 0, ov[3] = {0, 0, 0};
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const real gij = cc[32 * (3 * i + j)];
          op -= cc[32 * 22] * gij * dv[t][i][j];
          ov[i] -= cc[32 * 21] * gij * dp[t][j];
        }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int e = sInv[mnode * 3 + k];
        if (e < 0) break;
        const int f = e >> 5, jf = e & 31;
        const real a = sOwn[c * OS + f * 2 * NFPP + jf], b = sOwn[c * OS + f * 2 * NFPP + NFPP + jf];
        const real taup = cc[32 * (23 + f)], tauv = cc[32 * (27 + f)];
        const int bc = sBc[f * 32 + c];
        real sp = 0, sv = 0;
        if (bc == 0) {
          const real a2 = sIn[c * OS + f * 2 * NFPP + jf], b2 = sIn[c * OS + f * 2 * NFPP + NFPP + jf];
          sp = taup * a - b + b2 - taup * a2;
          sv = tauv * b - a + tauv * b2 - a2;
        } else if (bc == 1) {  // free surface
          sp = real(2) * (taup * a - b);
        } else if (bc == 2) {  // transparent
          sp = taup * a - b;
          sv = tauv * b - a;
        } else {  // rigid wall
          sv = real(2) * (tauv * b - a);
        }
        op += sp;
#pragma unroll
        for (int i = 0; i < 3; ++i) ov[i] += cc[32 * (9 + 3 * f + i)] * sv;
      }
      store(0, op);
#pragma unroll
      for (int i = 0; i < 3; ++i) store(1 + i, ov[i]);
    }
  }
}

// lambda_p -= coef res_r(col) l(x_r): block g handles the receivers rec_sorted[grp[g] .. grp[g+1])
// (all in one element slot), taken in order, threads over the nodes: deterministic
template <int N, typename real>
__global__ void adj_inject_kernel(real* __restrict__ lam, const int* __restrict__ grp, const int* __restrict__ rec_sorted,
                                  const int64_t* __restrict__ rec_slot, const real* __restrict__ rec_row,
                                  const double* __restrict__ res, int64_t n_time, int64_t col, double coef) {
  using O = Order<N>;
  constexpr int Np = O::Np;
  const int g0 = grp[blockIdx.x], g1 = grp[blockIdx.x + 1];
  const int64_t s = rec_slot[rec_sorted[g0]];
  for (int n = threadIdx.x; n < Np; n += blockDim.x) {
    const int64_t at = ((s >> 5) * 4 * Np + n) * 32 + (s & 31);
    real v = lam[at];
    for (int i = g0; i < g1; ++i) {
      const int r = rec_sorted[i];
      v -= real(coef * res[int64_t(r) * n_time + col]) * rec_row[int64_t(r) * Np + n];
    }
    lam[at] = v;
  }
}

// acc[slot] += sum_m lambda_p (q1_p - q0_p - F w)_m over the pressure nodes m of the slot (w on the
// source slot only).  One block per 32 slots: warp w takes the rows w, w + 8, ..., lane = slot, in
// the working precision (FP64 arithmetic is slow on this part), and the eight partial sums are
// added in FP64 in a fixed order (deterministic).
template <int N, typename real>
__global__ void adj_grad_kernel(const real* __restrict__ lam, const real* __restrict__ q1, const real* __restrict__ q0,
                                int64_t n_slots, int64_t src_slot, const real* __restrict__ w_src, double F,
                                double* __restrict__ acc) {
  using O = Order<N>;
  constexpr int Np = O::Np;
  __shared__ double part[8][32];
  const int64_t blk = blockIdx.x;
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool src = blk * 32 + lane == src_slot;
  real sum = 0;
#pragma unroll 4
  for (int m = wp; m < Np; m += 8) {
    const int64_t at = (blk * 4 * Np + m) * 32 + lane;  // pressure row of the field layout
    real dq = q1[at] - q0[at];
    if (src) dq -= real(F) * w_src[m];
    sum += lam[at] * dq;
  }
  part[wp][lane] = double(sum);
  __syncthreads();
  if (wp == 0) {
    double t = part[0][lane];
#pragma unroll
    for (int k = 1; k < 8; ++k) t += part[k][lane];
    acc[blk * 32 + lane] += t;
  }
}

}  // namespace ridg
