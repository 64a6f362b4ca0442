// Fused multi-rate DG step kernel for sm_103a.
//
// One launch processes every element whose unknowns sit at the current fine time t_start
// (Algorithm 1: the active elements form a suffix of the level-ordered slots) and, per element:
//   * the volume term (Eqs. dgLocalSchemeP/U, volume part): r_p = sum_j D_j (-rho c^2 sum_i rx_ij v_i),
//     r_vi = -(1/rho) sum_j rx_ij (D_j p);
//   * the surface term with the penalty fluxes of Eqs. weakFormP/V (factor 1/2, tau from the mean
//     impedance, negated backward in time) and the boundary conditions of Sec. 2 through ghost
//     states; r -= sum_f (J_f/J) L_f P_f, with the velocity lift taken per face and combined
//     with the normals afterwards (L_f (n_f s_f) = n_f (L_f s_f));
//   * the point injections of Eq. sourceTerm (source wavelet or re-injected receiver traces);
//   * the Adams-Bashforth update of its level (Eq. updateAB) -- done right away, since it only
//     needs the history -- and its traces at t_start + Delta t_l, written to a trace slot chosen
//     by time modulo 3 so that neighbours still read the traces at t_start;
//   * the half-step traces at t_start + Delta t_l / 2 (Eq. updateABcoarse) when it has finer
//     neighbours;
//   * forward runs: the traces of its domain-boundary faces into the boundary-trace arena;
//     backward source runs: those recorded traces as the exterior state of its boundary faces;
//   * backward runs with two wavefields (source S, receivers R): the AB3-exact increments of the
//     classical and characteristic images (Eq. updateABcorr), accumulated in FP64.
//
// A CTA owns 32 "columns": 32 elements of one wavefield (W = 1) or 16 elements x 2 wavefields
// (W = 2).  All per-element matrix products are done as small GEMMs out of shared memory: each
// thread owns a register tile of 2 nodes x 4 columns and accumulates, per node and column, the
// pressure right-hand side, the three reference derivatives of p and the four per-face velocity
// lifts (64 FP32 accumulators).  The reference matrices are read through the read-only data path
// (they stay resident in L1); field columns are read as 16-byte vectors.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ridg {

constexpr int kMaxLevels = 8;

// finfo byte per (element, face): bits 0-1 neighbour face, bits 2-4 correspondence code,
// bits 5-6 boundary code (0 = interior)
__host__ __device__ inline int finfo_face(uint8_t x) { return x & 3; }
__host__ __device__ inline int finfo_perm(uint8_t x) { return (x >> 2) & 7; }
__host__ __device__ inline int finfo_bc(uint8_t x) { return (x >> 5) & 3; }

// meta flags per slot
constexpr int kMetaValid = 1;
constexpr int kMetaHalf = 2;

// kernel modes
constexpr int kModeRecord = 1;   // forward: record boundary-face traces
constexpr int kModeReplay = 2;   // wavefield 0 takes recorded traces as exterior state on boundary faces
constexpr int kModeImageP = 4;   // accumulate the classical image (W == 2)
constexpr int kModeImageQ = 16;  // accumulate the characteristic image (W == 2)
constexpr int kModeImage = kModeImageP | kModeImageQ;
constexpr int kModeRhsOnly = 8;  // only write the right-hand side to rhs_out

// per-element geometry (double): rx[9], normal[12], fscale[4]
constexpr int kGeo = 25;
// per-element material (working precision): rho c^2, 1/rho, rho c, tau_p[4], tau_v[4]
constexpr int kMat = 11;
// per-element coefficients of the FP32 tensor-core kernel, in 16-byte groups: -rho c^2 rx[9] and
// rho c at kGtU; -rx/rho[9] at kGtV; per face (normal, 0) at kGtN + 4 f and the penalty
// coefficients (A, B, C, D) at kGtP + 4 f
constexpr int kGtU = 0, kGtZ = 9, kGtV = 12, kGtN = 24, kGtP = 40;
constexpr int kGtab = 56;

template <typename real>
struct WaveArgs {
  real* q;           // [n_slots/32][4][Np][32]
  real* ring;        // 3 x q-sized
  real* trace;       // face inboxes, 3 time slots x [n_slots][4][2][NFPP]: (p, n.v) of the neighbour
                     // across face f of slot s, in s's face-node order and with s's outward normal
  const int2* inj_range;  // [n_slots] (first, count) or null
  const real* inj_w;      // [n_inj][Np]
  const int* inj_row;     // [n_inj] data row
  int amp_mode;           // 0 none, 1 constant amplitude, 2 interpolated data rows
  real amp;               // amp_mode 1
  const double* data;     // amp_mode 2: [rows][n_time]
  const double* data_scale;  // amp_mode 2: the rows are injected times *data_scale (a power of two), or null
  int n_time;
};

template <typename real>
struct StepArgs {
  WaveArgs<real> wave[2];
  // interpolation of data rows at this time: samples interp_n0 .. interp_n0+3 with weights
  int interp_n0;
  double interp_w[4];
  int64_t slot_lo, slot_hi;  // active slots [slot_lo, slot_hi), multiples of 32
  int64_t level_begin[kMaxLevels + 1];
  int n_levels;
  int ring_new[kMaxLevels], ring_old1[kMaxLevels], ring_old2[kMaxLevels];
  real h[kMaxLevels];  // signed local step of each level
  int trace_read;
  int trace_write[kMaxLevels], trace_half[kMaxLevels];
  real tau_sign;
  int mode;
  int64_t n_slots;
  // boundary-trace arena: records of face index b (global boundary-face numbering) at this step
  // live at arena + (arena_offset + b) * 2 * NFPP
  real* arena_write;
  const real* arena_read;
  int64_t arena_offset;
  // images [n_slots/32][Np][32] (double)
  double* image_p;
  double* image_q;
  real e_up[3];
  // static tables
  const double* geo;     // [n_slots][kGeo]
  const real* mat;       // [n_slots][kMat]
  const int* nbr;        // [n_slots][4] neighbour slot or -1
  const uint8_t* finfo;  // [n_slots][4]
  const int* bface;      // [n_slots] index of the first boundary face of the slot
  const int* meta;       // [n_slots]
  const real* Dt;        // [3][Np][NPa]  Dt[j][m][n] = D_j[n][m]
  const real* Lt;        // [4*Nfp][NPa]  Lt[fm][n] = LIFT[n][fm]
  const int* fmask;      // [4][32]
  const int* perm;       // [6][32]
  real* rhs_out;         // kModeRhsOnly: q-sized
  const uint32_t* afrag; // tensor-core variant: operator fragments (TF32 hi/lo), see step_kernel_tc.cuh
  const float* gtab;     // tensor-core variant: per-element coefficients [n_slots][kGtab] (this tau sign)
  int contraction;       // FP32 element products: RIDG_CONTRACT_TENSOR / _CUDA_CORES / _TENSOR_BF16
};

// Merged launch of several shots of one solver (same mesh, tables and fine-step schedule, run in
// lockstep; the serving form): blocks [b * shot_blocks, (b + 1) * shot_blocks) step shot b, whose
// wavefields, boundary-record arena and images are shot[b]; everything else is the step's StepArgs.
constexpr int kMaxBatch = 4;
template <typename real>
struct ShotArgs {
  WaveArgs<real> wave[2];
  real* arena_write;
  const real* arena_read;
  double* image_p;
  double* image_q;
};
template <typename real>
struct BatchArgs {
  int shot_blocks;  // blocks of one shot in this launch
  ShotArgs<real> shot[kMaxBatch];
};
// the merged-launch argument of a kernel built for one shot: nothing
struct NoBatch {
  int unused;
};

template <int N>
struct Order {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NPP = (Np + 1) / 2;
  static constexpr int NPa = 2 * NPP;
  static constexpr int NT = ((8 * NPP + 31) / 32) * 32;
  static constexpr int NFPP = Nfp <= 16 ? 16 : 32;
};

template <typename real>
struct ColStride {
  static constexpr int value = 36;
};
template <>
struct ColStride<double> {
  static constexpr int value = 34;
};

// AB3 (Eq. updateAB), half-step (Eq. updateABcoarse) and image (Eq. updateABcorr) coefficients
struct AB {
  static constexpr double a1 = 23.0 / 12.0, a2 = -16.0 / 12.0, a3 = 5.0 / 12.0;
  static constexpr double b1 = 17.0 / 24.0, b2 = -7.0 / 24.0, b3 = 2.0 / 24.0;
  static constexpr double c1 = 19.0 / 24.0, c2 = -5.0 / 12.0, c3 = 1.0 / 8.0;
};

template <typename real>
__device__ __forceinline__ real fmaf_t(real a, real b, real c) {
  return fma(a, b, c);
}

template <typename real>
__device__ __forceinline__ void ld4(const real* p, real v[4]) {
  if constexpr (sizeof(real) == 4) {
    float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  } else {
    double2 x = *reinterpret_cast<const double2*>(p);
    double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = y.x;
    v[3] = y.y;
  }
}

template <typename real>
__device__ __forceinline__ void ld2g(const real* p, real v[2]) {
  if constexpr (sizeof(real) == 4) {
    float2 x = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = x.x;
    v[1] = x.y;
  } else {
    double2 x = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = x.x;
    v[1] = x.y;
  }
}

// Load/store the 4 columns (c0..c0+3) of one (field,node) row from/to the global q-layout of the
// two wavefields.  W == 1: 4 consecutive slots of one array.  W == 2: columns alternate S, R.
template <typename real, int W>
__device__ __forceinline__ void gload_cols(real* const base[2], int64_t off, real v[4]) {
  if constexpr (W == 1) {
    ld4<real>(base[0] + off, v);
  } else {
    // off points at the first of 2 consecutive elements
    real a0 = base[0][off], a1 = base[0][off + 1];
    real b0 = base[1][off], b1 = base[1][off + 1];
    v[0] = a0;
    v[1] = b0;
    v[2] = a1;
    v[3] = b1;
  }
}

template <typename real, int W>
__device__ __forceinline__ void gstore_cols(real* const base[2], int64_t off, const real v[4], const bool ok[4]) {
  if constexpr (W == 1) {
    if (ok[0] && ok[1] && ok[2] && ok[3]) {
      if constexpr (sizeof(real) == 4) {
        *reinterpret_cast<float4*>(base[0] + off) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
        *reinterpret_cast<double2*>(base[0] + off) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2*>(base[0] + off + 2) = make_double2(v[2], v[3]);
      }
    } else {
      for (int k = 0; k < 4; ++k)
        if (ok[k]) base[0][off + k] = v[k];
    }
  } else {
    if (ok[0]) base[0][off] = v[0];
    if (ok[1]) base[1][off] = v[1];
    if (ok[2]) base[0][off + 1] = v[2];
    if (ok[3]) base[1][off + 1] = v[3];
  }
}

// ---------------------------------------------------------------- asynchronous copies
__device__ __forceinline__ void cp_async_bytes16(void* smem, const void* gmem) {
  unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
template <int B>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
  unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(B));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename real>
__device__ __forceinline__ void st4(real* p, const real v[4]) {
  if constexpr (sizeof(real) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
}

// Shared-memory plan of dg_step_kernel<N, real, W> (offsets in reals).
template <int N, typename real, int W>
struct Smem {
  using O = Order<N>;
  static constexpr int Np = O::Np, Nfp = O::Nfp;
  // padded column rows (face-node gathers); unpadded for FP64 at N = 6, whose tile would not fit
  // in a block's shared memory with the padding
  static constexpr int CS = (sizeof(real) == 8 && N >= 6) ? 32 : ColStride<real>::value;
  static constexpr int RS = 32;                      // ring rows: read by their owner thread only
  static constexpr int XS = 33;                      // exterior-trace staging rows
  static constexpr int NG = 49;                      // per-element coefficients (odd: conflict-free)
  static constexpr int EPB = 32 / W;
  static constexpr int Q = 4 * Np * CS;
  static constexpr int R = 4 * Np * RS;
  static constexpr int ST = 4 * Nfp * CS;
  static constexpr int UX = (3 * Np * CS > 8 * Nfp * XS) ? 3 * Np * CS : 8 * Nfp * XS;
  static constexpr int G = EPB * NG;
  static constexpr int INTS = 4 * EPB + 4 * EPB + EPB + EPB + 128 + 192;
  static constexpr size_t bytes_with(bool ring) {
    return (size_t(Q) + (ring ? 2 * size_t(R) : 0) + 2 * size_t(ST) + UX + G) * sizeof(real) + INTS * sizeof(int);
  }
  // the history is staged in shared memory when it leaves room for at least one block
  static constexpr bool ring_in_smem = bytes_with(true) <= 200 * 1024;
  static constexpr size_t bytes = bytes_with(ring_in_smem);
  static_assert(4 * Np * CS <= 2 * ST + UX, "half-step staging must fit in the penalty/U region");
};

template <int N, typename real, int W>
__global__ void __launch_bounds__(Order<N>::NT) dg_step_kernel(const StepArgs<real> A) {
  using O = Order<N>;
  using SM = Smem<N, real, W>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NPa = O::NPa, NT = O::NT, NFPP = O::NFPP;
  constexpr int CS = SM::CS, RS = SM::RS, XS = SM::XS, NG = SM::NG, EPB = SM::EPB;
  constexpr bool RING = SM::ring_in_smem;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sQ = reinterpret_cast<real*>(smem_raw);  // [4][Np][CS]  q at t_start, then q at t_new
  real* sR1 = sQ + SM::Q;                         // [4][Np][RS]  history r^{m-1}   (if RING)
  real* sR2 = sR1 + (RING ? SM::R : 0);           // [4][Np][RS]  history r^{m-2}   (if RING)
  real* sS = sR2 + (RING ? SM::R : 0);            // [4*Nfp][CS]  velocity penalty scalars
  real* sT = sS + SM::ST;                         // [4*Nfp][CS]  pressure penalties
  real* sU = sT + SM::ST;                         // [3][Np][CS]  U_j (aliases sX)
  real* sX = sU;                                  // [4*Nfp][2][XS] exterior traces
  real* sG = sU + SM::UX;                         // [EPB][NG]
  int* sI = reinterpret_cast<int*>(sG + SM::G);
  int* sNbr = sI;                // [EPB][4]
  int* sInfo = sNbr + 4 * EPB;   // [EPB][4]
  int* sBf = sInfo + 4 * EPB;    // [EPB]
  int* sMeta = sBf + EPB;        // [EPB]
  int* sFm = sMeta + EPB;        // [4][32]
  int* sPerm = sFm + 128;        // [6][32]
  real* sH = sS;                 // [4][Np][CS] half-step fields, after the products

  const int tid = threadIdx.x;
  const int64_t slot0 = A.slot_lo + int64_t(blockIdx.x) * EPB;
  if (slot0 >= A.slot_hi) return;
  const int64_t blk = slot0 >> 5;     // 32-slot block of the field layout
  const int lane0 = int(slot0 & 31);  // first element's lane in that block (0 or 16)
  int lev = 0;
  for (int l = 0; l < A.n_levels; ++l)
    if (slot0 >= A.level_begin[l]) lev = l;
  const real h = A.h[lev];
  const bool rhs_only = (A.mode & kModeRhsOnly) != 0;
  const int64_t qsize = (A.n_slots >> 5) * 4 * Np * 32;
  const int rn = A.ring_new[lev], r1i = A.ring_old1[lev], r2i = A.ring_old2[lev];

  // ---------------------------------------------------------------- phase 1: async field loads
  // q at t_start and (unless only the right-hand side is wanted) the two older right-hand sides
  {
    const int64_t fbase = (blk * 4) * Np * 32;
    if constexpr (W == 1) {
      constexpr int CH = 16 / sizeof(real);  // reals per 16-byte chunk
      constexpr int NCH = 32 / CH;           // chunks per row
      const real* src0 = A.wave[0].q + fbase;
      const real* src1 = A.wave[0].ring + r1i * qsize + fbase;
      const real* src2 = A.wave[0].ring + r2i * qsize + fbase;
      const int narr = (RING && !rhs_only) ? 3 : 1;
      for (int i = tid; i < narr * 4 * Np * NCH; i += NT) {
        int arr = i / (4 * Np * NCH);
        int rem = i - arr * 4 * Np * NCH;
        int row = rem / NCH, ch = rem - row * NCH;
        real* dst = arr == 0 ? sQ + row * CS : (arr == 1 ? sR1 : sR2) + row * RS;
        const real* src = arr == 0 ? src0 : (arr == 1 ? src1 : src2);
        cp_async_bytes16(dst + ch * CH, src + row * 32 + ch * CH);
      }
    } else {
      const int narr = (RING && !rhs_only) ? 3 : 1;
      for (int i = tid; i < narr * 4 * Np * 32; i += NT) {
        int arr = i / (4 * Np * 32);
        int rem = i - arr * 4 * Np * 32;
        int row = rem >> 5, c = rem & 31;
        int e = c >> 1, w = c & 1;
        const real* base = arr == 0 ? A.wave[w].q : A.wave[w].ring + (arr == 1 ? r1i : r2i) * qsize;
        real* dst = arr == 0 ? sQ + row * CS + c : (arr == 1 ? sR1 : sR2) + row * RS + c;
        cp_async_small<sizeof(real)>(dst, base + fbase + row * 32 + lane0 + e);
      }
    }
    cp_async_commit();
  }

  // ---------------------------------------------------------------- phase 0: tables
  for (int i = tid; i < 128; i += NT) sFm[i] = A.fmask[i];
  for (int i = tid; i < 192; i += NT) sPerm[i] = A.perm[i];
  for (int i = tid; i < EPB * 4; i += NT) {
    int e = i >> 2, f = i & 3;
    int64_t s = slot0 + e;
    sNbr[i] = A.nbr[s * 4 + f];
    sInfo[i] = A.finfo[s * 4 + f];
  }
  for (int e = tid; e < EPB; e += NT) {
    int64_t s = slot0 + e;
    sBf[e] = A.bface[s];
    sMeta[e] = A.meta[s];
    const double* g = A.geo + s * kGeo;
    const real* m = A.mat + s * kMat;
    real* G = sG + e * NG;
    real rc2 = m[0], irho = m[1];
    // G[0..8]: -rho c^2 rx_ij (volume p equation), G[9..17]: -rx_ij / rho (volume v equation)
    for (int ij = 0; ij < 9; ++ij) {
      real rxij = real(g[ij]);
      G[ij] = -rc2 * rxij;
      G[9 + ij] = -irho * rxij;
    }
    // G[18..29]: outward normals
    for (int k = 0; k < 12; ++k) G[18 + k] = real(g[9 + k]);
    // G[30..45]: penalty coefficients per face: t = A_f [nv] + B_f [p], s = C_f [p] + D_f [nv]
    for (int f = 0; f < 4; ++f) {
      real fs = real(g[21 + f]);
      real taup = A.tau_sign * m[3 + f], tauv = A.tau_sign * m[7 + f];
      G[30 + 4 * f + 0] = -real(0.5) * fs * rc2;
      G[30 + 4 * f + 1] = real(0.5) * fs * rc2 * taup;
      G[30 + 4 * f + 2] = real(0.5) * fs * irho;
      G[30 + 4 * f + 3] = -real(0.5) * fs * irho * tauv;
    }
    G[46] = m[2];  // rho c
  }
  __syncthreads();

  // ---------------------------------------------------------------- phase 2a: exterior traces
  // half-warp per (column, face), lanes over face nodes: coalesced reads of this element's own
  // face inbox, which the neighbour filled in our face-node order and with our normal; four items'
  // loads are issued before any store.  Boundary faces of the backward source run read the
  // recorded forward traces instead.
  {
    constexpr int NH = NT / 16;
    const int hw = tid >> 4, j = tid & 15;
    for (int base = hw; base < 32 * 4; base += 4 * NH) {
      real xp[4][2], xv[4][2];
      bool have[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        have[u] = false;
        int item = base + u * NH;
        if (item >= 128) continue;
        int c = item >> 2, f = item & 3;
        int e = c / W, w = c % W;
        if (!(sMeta[e] & kMetaValid)) continue;
        int info = sInfo[e * 4 + f];
        int bc = finfo_bc(uint8_t(info));
        if (bc == 0) {
          const real* tb =
              A.wave[w].trace + (int64_t(A.trace_read) * A.n_slots + slot0 + e) * (8 * NFPP) + f * 2 * NFPP;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            int jj = j + 16 * t;
            if (jj < Nfp) {
              xp[u][t] = tb[jj];
              xv[u][t] = tb[NFPP + jj];
            }
          }
          have[u] = true;
        } else if (w == 0 && (A.mode & kModeReplay)) {
          // backward source run: the recorded forward traces are the exterior state
          int b = sBf[e];
          for (int ff = 0; ff < f; ++ff) b += (finfo_bc(uint8_t(sInfo[e * 4 + ff])) != 0);
          const real* rec = A.arena_read + (A.arena_offset + b) * (2 * NFPP);
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            int jj = j + 16 * t;
            if (jj < Nfp) {
              xp[u][t] = rec[jj];
              xv[u][t] = rec[NFPP + jj];
            }
          }
          have[u] = true;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (!have[u]) continue;
        int item = base + u * NH;
        int c = item >> 2, f = item & 3;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          int jj = j + 16 * t;
          if (jj < Nfp) {
            sX[((f * Nfp + jj) * 2 + 0) * XS + c] = xp[u][t];
            sX[((f * Nfp + jj) * 2 + 1) * XS + c] = xv[u][t];
          }
        }
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // ---------------------------------------------------------------- phase 2b: penalties
  for (int i = tid; i < 4 * Nfp * 32; i += NT) {
    int c = i & 31, fj = i >> 5;
    int f = fj / Nfp, jj = fj - f * Nfp;
    int e = c / W, w = c % W;
    const real* G = sG + e * NG;
    int n = sFm[f * 32 + jj];
    real p = sQ[(0 * Np + n) * CS + c];
    real vn = G[18 + 3 * f] * sQ[(1 * Np + n) * CS + c] + G[19 + 3 * f] * sQ[(2 * Np + n) * CS + c] +
              G[20 + 3 * f] * sQ[(3 * Np + n) * CS + c];
    int info = sInfo[e * 4 + f];
    int bc = finfo_bc(uint8_t(info));
    const bool valid = (sMeta[e] & kMetaValid) != 0;
    if (bc != 0 && valid && w == 0 && (A.mode & kModeRecord)) {
      // forward run: record the traces of this boundary face at t_start
      int b = sBf[e];
      for (int ff = 0; ff < f; ++ff) b += (finfo_bc(uint8_t(sInfo[e * 4 + ff])) != 0);
      real* rec = A.arena_write + (A.arena_offset + b) * (2 * NFPP);
      rec[jj] = p;
      rec[NFPP + jj] = vn;
    }
    real jp, jv;
    bool replay = (A.mode & kModeReplay) && w == 0 && bc != 0;
    if (bc == 0 || replay) {
      jp = sX[((f * Nfp + jj) * 2 + 0) * XS + c] - p;
      jv = sX[((f * Nfp + jj) * 2 + 1) * XS + c] - vn;
    } else if (bc == 1) {  // free surface: p+ = -p-, n.v+ = n.v-
      jp = -2 * p;
      jv = 0;
    } else if (bc == 2) {  // transparent: p+ = 0, v+ = 0
      jp = -p;
      jv = -vn;
    } else {  // rigid: p+ = p-, n.v+ = -n.v-
      jp = 0;
      jv = -2 * vn;
    }
    const real* pc = G + 30 + 4 * f;
    real t = pc[0] * jv + pc[1] * jp;
    real sv = pc[2] * jp + pc[3] * jv;
    if (!valid) {
      t = 0;
      sv = 0;
    }
    sT[fj * CS + c] = t;
    sS[fj * CS + c] = sv;
  }
  __syncthreads();

  // ---------------------------------------------------------------- phase 2c: U_j = G_p v
  for (int i = tid; i < Np * 32; i += NT) {
    int c = i & 31, m = i >> 5;
    int e = c / W;
    const real* G = sG + e * NG;
    real vx = sQ[(1 * Np + m) * CS + c], vy = sQ[(2 * Np + m) * CS + c], vz = sQ[(3 * Np + m) * CS + c];
    for (int j = 0; j < 3; ++j) sU[(j * Np + m) * CS + c] = G[0 + j] * vx + G[3 + j] * vy + G[6 + j] * vz;
  }
  __syncthreads();

  // ---------------------------------------------------------------- phase 3: element products
  const int np = tid >> 3;  // node pair
  const int cq = tid & 7;   // column quad
  const bool gemm = np < O::NPP;
  const int c0 = cq * 4;
  real rp[2][4], dp[3][2][4], ls[4][2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      rp[i][k] = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) dp[j][i][k] = 0;
#pragma unroll
      for (int f = 0; f < 4; ++f) ls[f][i][k] = 0;
    }
  if (gemm) {
    const real* Dt = A.Dt + 2 * np;
#pragma unroll 5
    for (int m = 0; m < Np; ++m) {
      real bp[4], bu[3][4], a[3][2];
      ld4<real>(sQ + m * CS + c0, bp);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        ld4<real>(sU + (j * Np + m) * CS + c0, bu[j]);
        ld2g<real>(Dt + (j * Np + m) * NPa, a[j]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            dp[j][i][k] = fmaf_t(a[j][i], bp[k], dp[j][i][k]);
            rp[i][k] = fmaf_t(a[j][i], bu[j][k], rp[i][k]);
          }
        }
    }
    const real* Lt = A.Lt + 2 * np;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
#pragma unroll 5
      for (int jj = 0; jj < Nfp; ++jj) {
        const int fm = f * Nfp + jj;
        real bt[4], bs[4], a[2];
        ld4<real>(sT + fm * CS + c0, bt);
        ld4<real>(sS + fm * CS + c0, bs);
        ld2g<real>(Lt + fm * NPa, a);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            rp[i][k] = fmaf_t(a[i], bt[k], rp[i][k]);
            ls[f][i][k] = fmaf_t(a[i], bs[k], ls[f][i][k]);
          }
      }
    }
  }
  __syncthreads();  // all reads of sS/sT/sU are done: sH may now reuse them

  // ---------------------------------------------------------------- phase 4: update
  if (gemm) {
    real* qb[2] = {A.wave[0].q, W == 2 ? A.wave[1].q : nullptr};
    real* rnew[2] = {A.wave[0].ring + rn * qsize, W == 2 ? A.wave[1].ring + rn * qsize : nullptr};
    real* rold1[2] = {A.wave[0].ring + r1i * qsize, W == 2 ? A.wave[1].ring + r1i * qsize : nullptr};
    real* rold2[2] = {A.wave[0].ring + r2i * qsize, W == 2 ? A.wave[1].ring + r2i * qsize : nullptr};
    real* rout[2] = {A.rhs_out, nullptr};
    bool ok[4];
    int eidx[4];
    const real* Gk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      eidx[k] = (c0 + k) / W;
      ok[k] = (sMeta[eidx[k]] & kMetaValid) != 0;
      Gk[k] = sG + eidx[k] * NG;
    }
    const int64_t col_off = (W == 1) ? (lane0 + c0) : (lane0 + c0 / 2);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int n = 2 * np + i;
      if (n >= Np) continue;
      real r[4][4];  // [field][column]
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const real* G = Gk[k];
        r[0][k] = rp[i][k];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          real v = G[9 + 3 * d + 0] * dp[0][i][k] + G[9 + 3 * d + 1] * dp[1][i][k] + G[9 + 3 * d + 2] * dp[2][i][k];
#pragma unroll
          for (int f = 0; f < 4; ++f) v -= G[18 + 3 * f + d] * ls[f][i][k];
          r[1 + d][k] = v;
        }
      }
      // point injections (source wavelet or receiver traces)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int w = (c0 + k) % W;
        const WaveArgs<real>& wa = A.wave[w];
        if (wa.amp_mode == 0 || !ok[k]) continue;
        int2 ir = wa.inj_range[slot0 + eidx[k]];
        for (int q = ir.x; q < ir.x + ir.y; ++q) {
          real amp;
          if (wa.amp_mode == 1) {
            amp = wa.amp;
          } else {
            double acc = 0.0;
            int row = wa.inj_row[q];
            for (int t = 0; t < 4; ++t) {
              int nt = A.interp_n0 + t;
              if (nt >= 0 && nt < wa.n_time) acc += A.interp_w[t] * wa.data[int64_t(row) * wa.n_time + nt];
            }
            if (wa.data_scale) acc *= *wa.data_scale;
            amp = real(acc);
          }
          r[0][k] += amp * wa.inj_w[int64_t(q) * Np + n];
        }
      }
      if (rhs_only) {
#pragma unroll
        for (int fld = 0; fld < 4; ++fld) {
          const int64_t off = ((blk * 4 + fld) * Np + n) * 32 + col_off;
          gstore_cols<real, W>(rout, off, r[fld], ok);
        }
        continue;
      }
      real q0[4][4], r1[4][4], r2[4][4];
#pragma unroll
      for (int fld = 0; fld < 4; ++fld) {
        ld4<real>(sQ + (fld * Np + n) * CS + c0, q0[fld]);
        if constexpr (RING) {
          ld4<real>(sR1 + (fld * Np + n) * RS + c0, r1[fld]);
          ld4<real>(sR2 + (fld * Np + n) * RS + c0, r2[fld]);
        } else {
          const int64_t off = ((blk * 4 + fld) * Np + n) * 32 + col_off;
          gload_cols<real, W>(rold1, off, r1[fld]);
          gload_cols<real, W>(rold2, off, r2[fld]);
        }
      }
      // images from the fields and histories at t_start, before the update
      if ((A.mode & kModeImage) && W == 2) {
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
          const int kS = 2 * pr, kR = 2 * pr + 1;
          if (!ok[kS]) continue;
          const real Z = Gk[kS][46];
          const real* eu = A.e_up;
          real xS = q0[0][kS], xR = q0[0][kR];
          real vS = eu[0] * q0[1][kS] + eu[1] * q0[2][kS] + eu[2] * q0[3][kS];
          real vR = eu[0] * q0[1][kR] + eu[1] * q0[2][kR] + eu[2] * q0[3][kR];
          real rS[3] = {r[0][kS], r1[0][kS], r2[0][kS]};
          real rR[3] = {r[0][kR], r1[0][kR], r2[0][kR]};
          real rvS[3] = {eu[0] * r[1][kS] + eu[1] * r[2][kS] + eu[2] * r[3][kS],
                         eu[0] * r1[1][kS] + eu[1] * r1[2][kS] + eu[2] * r1[3][kS],
                         eu[0] * r2[1][kS] + eu[1] * r2[2][kS] + eu[2] * r2[3][kS]};
          real rvR[3] = {eu[0] * r[1][kR] + eu[1] * r[2][kR] + eu[2] * r[3][kR],
                         eu[0] * r1[1][kR] + eu[1] * r1[2][kR] + eu[2] * r1[3][kR],
                         eu[0] * r2[1][kR] + eu[1] * r2[2][kR] + eu[2] * r2[3][kR]};
          const real c[3] = {real(AB::c1), real(AB::c2), real(AB::c3)};
          const real C[3][3] = {{real(4703.0 / 5040.0), real(-457.0 / 840.0), real(52.0 / 315.0)},
                                {real(-457.0 / 840.0), real(103.0 / 315.0), real(-251.0 / 2520.0)},
                                {real(52.0 / 315.0), real(-251.0 / 2520.0), real(17.0 / 560.0)}};
          real incP, incQ;
          {
            real t2 = 0, t3 = 0;
#pragma unroll
            for (int s = 0; s < 3; ++s) {
              t2 += c[s] * (xS * rR[s] + rS[s] * xR);
#pragma unroll
              for (int u = 0; u < 3; ++u) t3 += C[s][u] * rS[s] * rR[u];
            }
            incP = h * (xS * xR + h * (t2 + h * t3));
          }
          {
            // characteristic image: q^-_S = p - Z e.v, q^+_R = p + Z e.v
            real qS = xS - Z * vS, qR = xR + Z * vR;
            real sS3[3], sR3[3];
#pragma unroll
            for (int s = 0; s < 3; ++s) {
              sS3[s] = rS[s] - Z * rvS[s];
              sR3[s] = rR[s] + Z * rvR[s];
            }
            real t2 = 0, t3 = 0;
#pragma unroll
            for (int s = 0; s < 3; ++s) {
              t2 += c[s] * (qS * sR3[s] + sS3[s] * qR);
#pragma unroll
              for (int u = 0; u < 3; ++u) t3 += C[s][u] * sS3[s] * sR3[u];
            }
            incQ = h * (qS * qR + h * (t2 + h * t3));
          }
          const int64_t io = (blk * Np + n) * 32 + lane0 + eidx[kS];
          if (A.mode & kModeImageP) A.image_p[io] -= double(incP);
          if (A.mode & kModeImageQ) A.image_q[io] -= double(incQ);
        }
      }
#pragma unroll
      for (int fld = 0; fld < 4; ++fld) {
        real qn[4], qh[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          real upd = real(AB::a1) * r[fld][k] + real(AB::a2) * r1[fld][k] + real(AB::a3) * r2[fld][k];
          qn[k] = q0[fld][k] + h * upd;
          real hb = real(AB::b1) * r[fld][k] + real(AB::b2) * r1[fld][k] + real(AB::b3) * r2[fld][k];
          qh[k] = q0[fld][k] + h * hb;
        }
        const int64_t off = ((blk * 4 + fld) * Np + n) * 32 + col_off;
        gstore_cols<real, W>(qb, off, qn, ok);
        gstore_cols<real, W>(rnew, off, r[fld], ok);
        st4<real>(sQ + (fld * Np + n) * CS + c0, qn);
        st4<real>(sH + (fld * Np + n) * CS + c0, qh);
      }
    }
  }
  if (rhs_only) return;
  __syncthreads();

  // ---------------------------------------------------------------- phase 5: traces
  // pushed into the neighbour's inbox: face f2 of slot s2, at the neighbour's face-node index
  // perm[j] of our node j (the correspondences of the two sides are mutually inverse), with n.v
  // taken with the neighbour's normal.  Boundary faces have no reader.
  {
    const int hw = tid >> 4, j = tid & 15;
    const int ws = A.trace_write[lev], hs = A.trace_half[lev];
    for (int item = hw; item < 32 * 4; item += NT / 16) {
      int c = item >> 2, f = item & 3;
      int e = c / W, w = c % W;
      int meta = sMeta[e];
      if (!(meta & kMetaValid)) continue;
      const int info = sInfo[e * 4 + f];
      if (finfo_bc(uint8_t(info)) != 0) continue;
      const real* G = sG + e * NG;
      const int64_t s2 = sNbr[e * 4 + f];
      const int f2 = finfo_face(uint8_t(info));
      const int* pm = sPerm + finfo_perm(uint8_t(info)) * 32;
      real* tw = A.wave[w].trace + (int64_t(ws) * A.n_slots + s2) * (8 * NFPP) + f2 * 2 * NFPP;
      real* th = A.wave[w].trace + (int64_t(hs) * A.n_slots + s2) * (8 * NFPP) + f2 * 2 * NFPP;
      for (int jj = j; jj < Nfp; jj += 16) {
        int n = sFm[f * 32 + jj];
        int j2 = pm[jj];
        real p = sQ[(0 * Np + n) * CS + c];
        real vn = G[18 + 3 * f] * sQ[(1 * Np + n) * CS + c] + G[19 + 3 * f] * sQ[(2 * Np + n) * CS + c] +
                  G[20 + 3 * f] * sQ[(3 * Np + n) * CS + c];
        tw[j2] = p;
        tw[NFPP + j2] = -vn;
        if (meta & kMetaHalf) {
          real ph = sH[(0 * Np + n) * CS + c];
          real vh = G[18 + 3 * f] * sH[(1 * Np + n) * CS + c] + G[19 + 3 * f] * sH[(2 * Np + n) * CS + c] +
                    G[20 + 3 * f] * sH[(3 * Np + n) * CS + c];
          th[j2] = ph;
          th[NFPP + j2] = -vh;
        }
      }
    }
  }
}

// shared-memory bytes of dg_step_kernel<N, real, W>
template <int N, typename real, int W>
constexpr size_t step_smem_bytes() {
  return Smem<N, real, W>::bytes;
}

}  // namespace ridg
