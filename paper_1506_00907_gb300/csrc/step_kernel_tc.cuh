// Fused multi-rate DG step kernel, FP32, with the element-local contractions on tensor cores.
//
// Same algorithm and data flow as dg_step_kernel (step_kernel.cuh); this variant computes the
// per-element products D_j p, D_j U_j and L_f (penalties) -- the dense Dr/Ds/Dt and LIFT
// contractions of Eqs. dgLocalSchemeP/U, shared by every element -- as warp-level tensor-core
// products (mma.sync m16n8k8, TF32 inputs, FP32 accumulation).  FP32 accuracy is kept with the
// three-term split x = x_hi + x_lo (x_hi, x_lo TF32): A B ~ A_lo B_hi + A_hi B_lo + A_hi B_hi.
// The operator fragments (hi and lo) are prepared on the host in fragment order.
//
// Work split: a CTA owns 32 columns (32 elements, or 16 elements x 2 wavefields with the source
// wavefield in columns 0-15 and the receiver wavefield in 16-31).  Warp (mt, pair) computes, for
// the 16 nodes of node tile mt and the two 8-column blocks pair and pair+2, the pressure
// right-hand side, the three reference derivatives of p and the four per-face velocity lifts,
// and then runs the update/image epilogue for its nodes and columns straight from registers.
#pragma once
#include "step_kernel.cuh"

namespace ridg {

template <int N>
struct TcOrder {
  using O = Order<N>;
  static constexpr int Np = O::Np, Nfp = O::Nfp;
  static constexpr int MT = (Np + 15) / 16;  // 16-node tiles
  static constexpr int KSD = (Np + 7) / 8;   // k-steps over the nodes
  static constexpr int KSF = (Nfp + 7) / 8;  // k-steps over the nodes of one face
  static constexpr int NWARP = 2 * MT;
  static constexpr int NT = 32 * NWARP;
  // operator fragments: [3][MT][KSD][32 lanes][8] then [4][MT][KSF][32][8]; 8 = 4 hi + 4 lo
  static constexpr int FRAG_D = 3 * MT * KSD * 32 * 8;
  static constexpr int FRAG_L = 4 * MT * KSF * 32 * 8;
  static constexpr int FRAG = FRAG_D + FRAG_L;
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// acc += A * B with A = (a_hi, a_lo), B = (b_hi, b_lo): small terms first
__device__ __forceinline__ void mma3(float c[4], const uint32_t ah[4], const uint32_t al[4], const uint32_t bh[2],
                                     const uint32_t bl[2]) {
  mma_tf32(c, al, bh);
  mma_tf32(c, ah, bl);
  mma_tf32(c, ah, bh);
}

// B fragment (8 x 8, column major) of rows kb*8 + t, kb*8 + t + 4 (valid below kvalid) and column
// col of a shared-memory matrix with row stride CS, split into TF32 hi/lo.
template <int CS>
__device__ __forceinline__ void load_b(const float* X, int row0, int kvalid_rel, int t, int col, uint32_t bh[2],
                                       uint32_t bl[2]) {
  float x0 = (t < kvalid_rel) ? X[(row0 + t) * CS + col] : 0.f;
  float x1 = (t + 4 < kvalid_rel) ? X[(row0 + t + 4) * CS + col] : 0.f;
  bh[0] = to_tf32(x0);
  bh[1] = to_tf32(x1);
  bl[0] = to_tf32(x0 - __uint_as_float(bh[0]));
  bl[1] = to_tf32(x1 - __uint_as_float(bh[1]));
}

__device__ __forceinline__ void load_a(const uint32_t* frag, int lane, uint32_t ah[4], uint32_t al[4]) {
  const uint4* p = reinterpret_cast<const uint4*>(frag + lane * 8);
  uint4 h = __ldg(p), l = __ldg(p + 1);
  ah[0] = h.x;
  ah[1] = h.y;
  ah[2] = h.z;
  ah[3] = h.w;
  al[0] = l.x;
  al[1] = l.y;
  al[2] = l.z;
  al[3] = l.w;
}

template <int N, int W>
struct SmemTc {
  using O = Order<N>;
  static constexpr int Np = O::Np, Nfp = O::Nfp;
  static constexpr int CS = 36;  // column rows (16-byte aligned, few conflicts in fragment loads)
  static constexpr int XS = 33;
  static constexpr int NG = 49;
  static constexpr int EPB = 32 / W;
  static constexpr int Q = 4 * Np * CS;
  static constexpr int ST = 4 * Nfp * CS;
  static constexpr int UX = (3 * Np * CS > 8 * Nfp * XS) ? 3 * Np * CS : 8 * Nfp * XS;
  static constexpr int G = EPB * NG;
  static constexpr int INTS = 4 * EPB + 4 * EPB + EPB + EPB + 128 + 192;
  static constexpr size_t bytes_with(bool ring) {
    return (size_t(Q) * (ring ? 3 : 1) + 2 * size_t(ST) + UX + G) * sizeof(float) + INTS * sizeof(int);
  }
  static constexpr bool ring_in_smem = bytes_with(true) <= 200 * 1024;
  static constexpr size_t bytes = bytes_with(ring_in_smem);
  static_assert(4 * Np * CS <= 2 * ST + UX, "half-step staging must fit in the penalty/U region");
};

template <int N, int W>
__global__ void __launch_bounds__(TcOrder<N>::NT) dg_step_kernel_tc(const StepArgs<float> A) {
  using O = Order<N>;
  using T = TcOrder<N>;
  using SM = SmemTc<N, W>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NT = T::NT, NFPP = O::NFPP;
  constexpr int CS = SM::CS, XS = SM::XS, NG = SM::NG, EPB = SM::EPB;
  constexpr bool RING = SM::ring_in_smem;
  constexpr int MT = T::MT, KSD = T::KSD, KSF = T::KSF;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sQ = reinterpret_cast<float*>(smem_raw);  // [4][Np][CS]
  float* sR1 = sQ + SM::Q;                         // [4][Np][CS] (if RING)
  float* sR2 = sR1 + (RING ? SM::Q : 0);           // [4][Np][CS] (if RING)
  float* sS = sR2 + (RING ? SM::Q : 0);            // [4*Nfp][CS]
  float* sT = sS + SM::ST;                         // [4*Nfp][CS]
  float* sU = sT + SM::ST;                         // [3][Np][CS] (aliases sX)
  float* sX = sU;                                  // [4*Nfp][2][XS]
  float* sG = sU + SM::UX;                         // [EPB][NG]
  int* sI = reinterpret_cast<int*>(sG + SM::G);
  int* sNbr = sI;
  int* sInfo = sNbr + 4 * EPB;
  int* sBf = sInfo + 4 * EPB;
  int* sMeta = sBf + EPB;
  int* sFm = sMeta + EPB;
  int* sPerm = sFm + 128;
  float* sH = sS;  // [4][Np][CS] half-step fields, after the products

  const int tid = threadIdx.x;
  const int64_t slot0 = A.slot_lo + int64_t(blockIdx.x) * EPB;
  if (slot0 >= A.slot_hi) return;
  const int64_t blk = slot0 >> 5;
  const int lane0 = int(slot0 & 31);
  int lev = 0;
  for (int l = 0; l < A.n_levels; ++l)
    if (slot0 >= A.level_begin[l]) lev = l;
  const float h = A.h[lev];
  const bool rhs_only = (A.mode & kModeRhsOnly) != 0;
  const int64_t qsize = (A.n_slots >> 5) * 4 * Np * 32;
  const int rn = A.ring_new[lev], r1i = A.ring_old1[lev], r2i = A.ring_old2[lev];

  // column c -> (element, wavefield)
  auto col_e = [](int c) { return W == 1 ? c : (c & 15); };
  auto col_w = [](int c) { return W == 1 ? 0 : (c >> 4); };

  // ---------------------------------------------------------------- phase 1: async field loads
  {
    const int64_t fbase = (blk * 4) * Np * 32 + lane0;
    constexpr int CPR = EPB / 4;             // 16-byte chunks per row and wavefield
    constexpr int PER = 4 * Np * W * CPR;    // chunks per array
    const int narr = (RING && !rhs_only) ? 3 : 1;
    for (int i = tid; i < narr * PER; i += NT) {
      int arr = i / PER;
      int rem = i - arr * PER;
      int row = rem / (W * CPR);
      int r2 = rem - row * (W * CPR);
      int w = r2 / CPR, ch = r2 - w * CPR;
      const float* base = arr == 0 ? A.wave[w].q : A.wave[w].ring + (arr == 1 ? r1i : r2i) * qsize;
      float* dst = (arr == 0 ? sQ : (arr == 1 ? sR1 : sR2)) + row * CS + w * 16 + ch * 4;
      cp_async_bytes16(dst, base + fbase + row * 32 + ch * 4);
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
    const float* m = A.mat + s * kMat;
    float* G = sG + e * NG;
    float rc2 = m[0], irho = m[1];
    for (int ij = 0; ij < 9; ++ij) {
      float rxij = float(g[ij]);
      G[ij] = -rc2 * rxij;
      G[9 + ij] = -irho * rxij;
    }
    for (int k = 0; k < 12; ++k) G[18 + k] = float(g[9 + k]);
    for (int f = 0; f < 4; ++f) {
      float fs = float(g[21 + f]);
      float taup = A.tau_sign * m[3 + f], tauv = A.tau_sign * m[7 + f];
      G[30 + 4 * f + 0] = -0.5f * fs * rc2;
      G[30 + 4 * f + 1] = 0.5f * fs * rc2 * taup;
      G[30 + 4 * f + 2] = 0.5f * fs * irho;
      G[30 + 4 * f + 3] = -0.5f * fs * irho * tauv;
    }
    G[46] = m[2];
  }
  __syncthreads();

  // ---------------------------------------------------------------- phase 2a: exterior traces
  {
    constexpr int NH = NT / 16;
    const int hw = tid >> 4, j = tid & 15;
    for (int base = hw; base < 32 * 4; base += 4 * NH) {
      float xp[4][2], xv[4][2];
      bool have[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        have[u] = false;
        int item = base + u * NH;
        if (item >= 128) continue;
        int c = item >> 2, f = item & 3;
        int e = col_e(c), w = col_w(c);
        if (!(sMeta[e] & kMetaValid)) continue;
        int info = sInfo[e * 4 + f];
        int bc = finfo_bc(uint8_t(info));
        if (bc == 0) {
          int64_t s2 = sNbr[e * 4 + f];
          int f2 = finfo_face(uint8_t(info));
          const float* tb = A.wave[w].trace + (int64_t(A.trace_read) * A.n_slots + s2) * (8 * NFPP) + f2 * 2 * NFPP;
          const int* pm = sPerm + finfo_perm(uint8_t(info)) * 32;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            int jj = j + 16 * t;
            if (jj < Nfp) {
              int j2 = pm[jj];
              xp[u][t] = tb[j2];
              xv[u][t] = -tb[NFPP + j2];
            }
          }
          have[u] = true;
        } else if (w == 0 && (A.mode & kModeReplay)) {
          int b = sBf[e];
          for (int ff = 0; ff < f; ++ff) b += (finfo_bc(uint8_t(sInfo[e * 4 + ff])) != 0);
          const float* rec = A.arena_read + (A.arena_offset + b) * (2 * NFPP);
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
    int e = col_e(c), w = col_w(c);
    const float* G = sG + e * NG;
    int n = sFm[f * 32 + jj];
    float p = sQ[(0 * Np + n) * CS + c];
    float vn = G[18 + 3 * f] * sQ[(1 * Np + n) * CS + c] + G[19 + 3 * f] * sQ[(2 * Np + n) * CS + c] +
               G[20 + 3 * f] * sQ[(3 * Np + n) * CS + c];
    int info = sInfo[e * 4 + f];
    int bc = finfo_bc(uint8_t(info));
    const bool valid = (sMeta[e] & kMetaValid) != 0;
    if (bc != 0 && valid && w == 0 && (A.mode & kModeRecord)) {
      int b = sBf[e];
      for (int ff = 0; ff < f; ++ff) b += (finfo_bc(uint8_t(sInfo[e * 4 + ff])) != 0);
      float* rec = A.arena_write + (A.arena_offset + b) * (2 * NFPP);
      rec[jj] = p;
      rec[NFPP + jj] = vn;
    }
    float jp, jv;
    bool replay = (A.mode & kModeReplay) && w == 0 && bc != 0;
    if (bc == 0 || replay) {
      jp = sX[((f * Nfp + jj) * 2 + 0) * XS + c] - p;
      jv = sX[((f * Nfp + jj) * 2 + 1) * XS + c] - vn;
    } else if (bc == 1) {
      jp = -2.f * p;
      jv = 0.f;
    } else if (bc == 2) {
      jp = -p;
      jv = -vn;
    } else {
      jp = 0.f;
      jv = -2.f * vn;
    }
    const float* pc = G + 30 + 4 * f;
    float t = pc[0] * jv + pc[1] * jp;
    float sv = pc[2] * jp + pc[3] * jv;
    if (!valid) {
      t = 0.f;
      sv = 0.f;
    }
    sT[fj * CS + c] = t;
    sS[fj * CS + c] = sv;
  }
  __syncthreads();

  // ---------------------------------------------------------------- phase 2c: U_j = G_p v
  for (int i = tid; i < Np * 32; i += NT) {
    int c = i & 31, m = i >> 5;
    const float* G = sG + col_e(c) * NG;
    float vx = sQ[(1 * Np + m) * CS + c], vy = sQ[(2 * Np + m) * CS + c], vz = sQ[(3 * Np + m) * CS + c];
#pragma unroll
    for (int jd = 0; jd < 3; ++jd) sU[(jd * Np + m) * CS + c] = G[0 + jd] * vx + G[3 + jd] * vy + G[6 + jd] * vz;
  }
  __syncthreads();

  // ---------------------------------------------------------------- phase 3: tensor-core products
  const int lane = tid & 31, wid = tid >> 5;
  const int mt = wid >> 1, pair = wid & 1;
  const int g = lane >> 2, t4 = lane & 3;
  const int colb[2] = {pair * 8 + g, (pair + 2) * 8 + g};  // B-fragment columns of the two blocks
  float rp[2][4], dp[3][2][4], ls[4][2][4];
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      rp[b][q] = 0.f;
#pragma unroll
      for (int jd = 0; jd < 3; ++jd) dp[jd][b][q] = 0.f;
#pragma unroll
      for (int f = 0; f < 4; ++f) ls[f][b][q] = 0.f;
    }
  {
    const uint32_t* fragD = A.afrag;
    const uint32_t* fragL = A.afrag + T::FRAG_D;
#pragma unroll
    for (int jd = 0; jd < 3; ++jd) {
      const float* Ub = sU + jd * Np * CS;
#pragma unroll
      for (int kb = 0; kb < KSD; ++kb) {
        uint32_t ah[4], al[4];
        load_a(fragD + ((jd * MT + mt) * KSD + kb) * 256, lane, ah, al);
        const int kv = Np - kb * 8;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          uint32_t bh[2], bl[2];
          load_b<CS>(sQ, kb * 8, kv, t4, colb[b], bh, bl);
          mma3(dp[jd][b], ah, al, bh, bl);
          load_b<CS>(Ub, kb * 8, kv, t4, colb[b], bh, bl);
          mma3(rp[b], ah, al, bh, bl);
        }
      }
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
#pragma unroll
      for (int kb = 0; kb < KSF; ++kb) {
        uint32_t ah[4], al[4];
        load_a(fragL + ((f * MT + mt) * KSF + kb) * 256, lane, ah, al);
        const int kv = Nfp - kb * 8;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          uint32_t bh[2], bl[2];
          load_b<CS>(sT, f * Nfp + kb * 8, kv, t4, colb[b], bh, bl);
          mma3(rp[b], ah, al, bh, bl);
          load_b<CS>(sS, f * Nfp + kb * 8, kv, t4, colb[b], bh, bl);
          mma3(ls[f][b], ah, al, bh, bl);
        }
      }
    }
  }
  __syncthreads();  // every warp is done reading sQ/sS/sT/sU

  // ---------------------------------------------------------------- phase 4: update
  {
    // accumulator entry q of block b: node mt*16 + g + 8*(q>>1), column (pair + 2b)*8 + 2 t4 + (q&1)
    float* rout = A.rhs_out;
#pragma unroll
    for (int hn = 0; hn < 2; ++hn) {
      const int n = mt * 16 + g + 8 * hn;
      if (n >= Np) continue;
      // r[b][k][fld] for the two columns k of block b
      float r[2][2][4];
      int cols[2][2], es[2][2];
      bool ok[2][2];
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int q = 2 * hn + k;
          const int c = (pair + 2 * b) * 8 + 2 * t4 + k;
          cols[b][k] = c;
          const int e = col_e(c);
          es[b][k] = e;
          ok[b][k] = (sMeta[e] & kMetaValid) != 0;
          const float* G = sG + e * NG;
          r[b][k][0] = rp[b][q];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            float v = G[9 + 3 * d + 0] * dp[0][b][q] + G[9 + 3 * d + 1] * dp[1][b][q] + G[9 + 3 * d + 2] * dp[2][b][q];
#pragma unroll
            for (int f = 0; f < 4; ++f) v -= G[18 + 3 * f + d] * ls[f][b][q];
            r[b][k][1 + d] = v;
          }
          // point injections
          const int w = col_w(c);
          const WaveArgs<float>& wa = A.wave[w];
          if (wa.amp_mode != 0 && ok[b][k]) {
            int2 ir = wa.inj_range[slot0 + e];
            for (int qq = ir.x; qq < ir.x + ir.y; ++qq) {
              float amp;
              if (wa.amp_mode == 1) {
                amp = wa.amp;
              } else {
                double acc = 0.0;
                int row = wa.inj_row[qq];
                for (int tt = 0; tt < 4; ++tt) {
                  int nt = A.interp_n0 + tt;
                  if (nt >= 0 && nt < wa.n_time) acc += A.interp_w[tt] * wa.data[int64_t(row) * wa.n_time + nt];
                }
                amp = float(acc);
              }
              r[b][k][0] += amp * wa.inj_w[int64_t(qq) * Np + n];
            }
          }
        }
      if (rhs_only) {
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int k = 0; k < 2; ++k)
            if (ok[b][k])
#pragma unroll
              for (int fld = 0; fld < 4; ++fld)
                rout[((blk * 4 + fld) * Np + n) * 32 + lane0 + es[b][k]] = r[b][k][fld];
        continue;
      }
      float q0[2][2][4], r1[2][2][4], r2[2][2][4];
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int c = cols[b][k];
#pragma unroll
          for (int fld = 0; fld < 4; ++fld) {
            q0[b][k][fld] = sQ[(fld * Np + n) * CS + c];
            if constexpr (RING) {
              r1[b][k][fld] = sR1[(fld * Np + n) * CS + c];
              r2[b][k][fld] = sR2[(fld * Np + n) * CS + c];
            } else {
              const int64_t off = ((blk * 4 + fld) * Np + n) * 32 + lane0 + es[b][k];
              const int w = col_w(c);
              r1[b][k][fld] = A.wave[w].ring[r1i * qsize + off];
              r2[b][k][fld] = A.wave[w].ring[r2i * qsize + off];
            }
          }
        }
      // images (two wavefields): block 0 holds the source wavefield, block 1 the receivers'
      if (W == 2 && (A.mode & kModeImage)) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (!ok[0][k]) continue;
          const float* G = sG + es[0][k] * NG;
          const float Z = G[46];
          const float* eu = A.e_up;
          const float* qS_ = q0[0][k];
          const float* qR_ = q0[1][k];
          float xS = qS_[0], xR = qR_[0];
          float vS = eu[0] * qS_[1] + eu[1] * qS_[2] + eu[2] * qS_[3];
          float vR = eu[0] * qR_[1] + eu[1] * qR_[2] + eu[2] * qR_[3];
          const float* hS[3] = {r[0][k], r1[0][k], r2[0][k]};
          const float* hR[3] = {r[1][k], r1[1][k], r2[1][k]};
          float rS[3], rR[3], rvS[3], rvR[3];
#pragma unroll
          for (int s = 0; s < 3; ++s) {
            rS[s] = hS[s][0];
            rR[s] = hR[s][0];
            rvS[s] = eu[0] * hS[s][1] + eu[1] * hS[s][2] + eu[2] * hS[s][3];
            rvR[s] = eu[0] * hR[s][1] + eu[1] * hR[s][2] + eu[2] * hR[s][3];
          }
          const float cc[3] = {float(AB::c1), float(AB::c2), float(AB::c3)};
          const float C[3][3] = {{float(4703.0 / 5040.0), float(-457.0 / 840.0), float(52.0 / 315.0)},
                                 {float(-457.0 / 840.0), float(103.0 / 315.0), float(-251.0 / 2520.0)},
                                 {float(52.0 / 315.0), float(-251.0 / 2520.0), float(17.0 / 560.0)}};
          float incP, incQ;
          {
            float t2 = 0.f, t3 = 0.f;
#pragma unroll
            for (int s = 0; s < 3; ++s) {
              t2 += cc[s] * (xS * rR[s] + rS[s] * xR);
#pragma unroll
              for (int u = 0; u < 3; ++u) t3 += C[s][u] * rS[s] * rR[u];
            }
            incP = h * (xS * xR + h * (t2 + h * t3));
          }
          {
            float qS = xS - Z * vS, qR = xR + Z * vR;
            float sS3[3], sR3[3];
#pragma unroll
            for (int s = 0; s < 3; ++s) {
              sS3[s] = rS[s] - Z * rvS[s];
              sR3[s] = rR[s] + Z * rvR[s];
            }
            float t2 = 0.f, t3 = 0.f;
#pragma unroll
            for (int s = 0; s < 3; ++s) {
              t2 += cc[s] * (qS * sR3[s] + sS3[s] * qR);
#pragma unroll
              for (int u = 0; u < 3; ++u) t3 += C[s][u] * sS3[s] * sR3[u];
            }
            incQ = h * (qS * qR + h * (t2 + h * t3));
          }
          const int64_t io = (blk * Np + n) * 32 + lane0 + es[0][k];
          A.image_p[io] -= double(incP);
          A.image_q[io] -= double(incQ);
        }
      }
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int c = cols[b][k];
          const int w = col_w(c);
#pragma unroll
          for (int fld = 0; fld < 4; ++fld) {
            const float rr = r[b][k][fld];
            const float upd = float(AB::a1) * rr + float(AB::a2) * r1[b][k][fld] + float(AB::a3) * r2[b][k][fld];
            const float hb = float(AB::b1) * rr + float(AB::b2) * r1[b][k][fld] + float(AB::b3) * r2[b][k][fld];
            const float qn = q0[b][k][fld] + h * upd;
            sQ[(fld * Np + n) * CS + c] = qn;
            sH[(fld * Np + n) * CS + c] = q0[b][k][fld] + h * hb;
            if (ok[b][k]) {
              const int64_t off = ((blk * 4 + fld) * Np + n) * 32 + lane0 + es[b][k];
              A.wave[w].q[off] = qn;
              A.wave[w].ring[rn * qsize + off] = rr;
            }
          }
        }
    }
  }
  if (rhs_only) return;
  __syncthreads();

  // ---------------------------------------------------------------- phase 5: traces
  {
    const int hw = tid >> 4, j = tid & 15;
    const int ws = A.trace_write[lev], hs = A.trace_half[lev];
    for (int item = hw; item < 32 * 4; item += NT / 16) {
      int c = item >> 2, f = item & 3;
      int e = col_e(c), w = col_w(c);
      int meta = sMeta[e];
      if (!(meta & kMetaValid)) continue;
      const float* G = sG + e * NG;
      int64_t s = slot0 + e;
      float* tw = A.wave[w].trace + (int64_t(ws) * A.n_slots + s) * (8 * NFPP) + f * 2 * NFPP;
      float* th = A.wave[w].trace + (int64_t(hs) * A.n_slots + s) * (8 * NFPP) + f * 2 * NFPP;
      for (int jj = j; jj < Nfp; jj += 16) {
        int n = sFm[f * 32 + jj];
        float p = sQ[(0 * Np + n) * CS + c];
        float vn = G[18 + 3 * f] * sQ[(1 * Np + n) * CS + c] + G[19 + 3 * f] * sQ[(2 * Np + n) * CS + c] +
                   G[20 + 3 * f] * sQ[(3 * Np + n) * CS + c];
        tw[jj] = p;
        tw[NFPP + jj] = vn;
        if (meta & kMetaHalf) {
          float ph = sH[(0 * Np + n) * CS + c];
          float vh = G[18 + 3 * f] * sH[(1 * Np + n) * CS + c] + G[19 + 3 * f] * sH[(2 * Np + n) * CS + c] +
                     G[20 + 3 * f] * sH[(3 * Np + n) * CS + c];
          th[jj] = ph;
          th[NFPP + jj] = vh;
        }
      }
    }
  }
}

}  // namespace ridg
