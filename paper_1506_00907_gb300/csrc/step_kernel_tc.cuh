// Fused multi-rate DG step kernel, FP32, with the element-local contractions on tensor cores.
//
// Same algorithm and data flow as dg_step_kernel (step_kernel.cuh); this variant computes the
// per-element products D_j p, D_j U_j and L_f (penalties) -- the dense Dr/Ds/Dt and LIFT
// contractions of Eqs. dgLocalSchemeP/U, shared by every element -- as warp-level tensor-core
// products (mma.sync m16n8k8, TF32 inputs, FP32 accumulation), with the three-term split
// x = x_hi + x_lo (x_hi, x_lo TF32): A B ~ A_lo B_hi + A_hi B_lo + A_hi B_hi (errors of a whole
// shot against FP64 near 1e-6, a few times those of plain FP32 FMAs).
// The operator fragments (hi and lo) are prepared on the host in fragment order.
//
// Work split: a CTA owns 32 columns (32 elements, or 16 elements x 2 wavefields with the source
// wavefield in columns 0-15 and the receiver wavefield in 16-31).  Everything it reads is issued
// at once as asynchronous copies: the fields, the per-element coefficients (precomputed, with the
// penalty sign of the run) and the face inboxes, into which each neighbour pushed its traces in
// this element's face-node order.  Warp (mt, pair) computes, for the 16 nodes of node tile mt and
// the two 8-column blocks pair and pair+2, the pressure right-hand side, the three reference
// derivatives of p and the four per-face velocity lifts, and leaves the right-hand sides in shared
// memory; the update then runs with a thread per (node, element), so that every global store is
// 32 (or 2 x 16) consecutive columns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "step_kernel.cuh"

namespace ridg {
// Split formats of the tensor-core products: TF32 hi + lo with m16n8k8 (k-steps of 8 nodes), or
// BF16 hi + lo with m16n8k16 (k-steps of 16 nodes, half the instructions, 16 significand bits), or
// FP16 hi + lo with m16n8k16 (22 significand bits; FP16's range holds the fields only after a
// per-column power-of-two scale, applied to each operand tile before the split and removed from the
// FP32 accumulators).
constexpr int kSplitTf32 = 0, kSplitBf16 = 1, kSplitFp16 = 2;

template <int N, int KIND = kSplitTf32>
struct TcOrder {
  using O = Order<N>;
  static constexpr int Np = O::Np, Nfp = O::Nfp;
  static constexpr int MT = (Np + 15) / 16;  // 16-node tiles
  static constexpr int KS = KIND == kSplitTf32 ? 8 : 16;  // nodes per k-step
  static constexpr int KSD = (Np + KS - 1) / KS;   // k-steps over the nodes
  static constexpr int KSF = (Nfp + KS - 1) / KS;  // k-steps over the nodes of one face
  static constexpr int NWARP = 2 * MT;
  static constexpr int NT = 32 * NWARP;
  // operator fragments, one contiguous stream per node tile: [MT][NSTEP][32 lanes][8], 8 = 4 hi +
  // 4 lo; steps jd * KSD + kb (D_jd, k-step kb) then 3 KSD + f * KSF + kb (LIFT block f)
  static constexpr int NSTEP = 3 * KSD + 4 * KSF;
  static constexpr int FRAG = MT * NSTEP * 32 * 8;
  static constexpr int LAST_ROWS = Np - 16 * (MT - 1);  // rows of the last node tile
  // resident blocks per SM the kernel is built for (registers and shared memory are sized to it)
  static constexpr int MINB = N <= 4 ? 3 : (N == 5 ? 2 : 1);
};

struct FragA {
  uint32_t h[4], l[4];
};

__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// TF32 split by truncation: hi keeps the top 10 mantissa bits of x, lo = x - hi is exact in FP32
// and is itself truncated to TF32 (the discarded part is below 2^-20 |x|).  Rounding both parts to
// nearest instead (an integer add before the mask) lowered the error of a whole shot against FP64
// by 1.2-2x and cost 3 % of kernel time; the truncated split is kept.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(x) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi)) & 0xffffe000u;
}

// B fragment (8 x 8, column major) of rows kb*8 + t, kb*8 + t + 4 (valid below kvalid) and column
// col of a shared-memory matrix with row stride CS, split into TF32 hi/lo.
template <int CS>
__device__ __forceinline__ void load_b(const float* X, int row0, int kvalid_rel, int t, int col, uint32_t bh[2],
                                       uint32_t bl[2]) {
  float x0 = (t < kvalid_rel) ? X[(row0 + t) * CS + col] : 0.f;
  float x1 = (t + 4 < kvalid_rel) ? X[(row0 + t + 4) * CS + col] : 0.f;
  split_tf32(x0, bh[0], bl[0]);
  split_tf32(x1, bh[1], bl[1]);
}

// m16n8k16 BF16 product with FP32 accumulation (A 16 x 16 row major, B 16 x 8 column major).
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Two values as BF16 hi + lo pairs (round to nearest even): hi = bf16(x), lo = bf16(x - hi); the
// value with the lower k index goes to the low half of each register.
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - __low2float(h), x1 - __high2float(h));
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// m16n8k16 FP16 product with FP32 accumulation (A 16 x 16 row major, B 16 x 8 column major).
__device__ __forceinline__ void mma_f16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Two values as FP16 hi + lo pairs (round to nearest even): hi = fp16(x), lo = fp16(x - hi).
__device__ __forceinline__ void split_f16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const __half2 l = __floats2half2_rn(x0 - __low2float(h), x1 - __high2float(h));
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// B fragment of a 16-bit k-step (16 x 8, column major).  The k index is permuted inside the step so
// that lane (g, t) reads rows t, t + 4, t + 8, t + 12 (the conflict-free rows of the TF32 loads):
// fragment positions 2t, 2t+1, 2t+8, 2t+9 hold rows t, t+4, t+8, t+12; the host orders the operator
// columns of each step the same way, so the product is unchanged.  FP16 values are scaled by sc (the
// power of two of their column and operand) before the split.
template <int CS, int KIND>
__device__ __forceinline__ void load_b16(const float* X, int row0, int kvalid_rel, int t, int col, uint32_t bh[2],
                                         uint32_t bl[2], float sc) {
  float x[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = (t + 4 * i < kvalid_rel) ? X[(row0 + t + 4 * i) * CS + col] : 0.f;
  if constexpr (KIND == kSplitFp16) {
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] *= sc;
    split_f16x2(x[0], x[1], bh[0], bl[0]);
    split_f16x2(x[2], x[3], bh[1], bl[1]);
  } else {
    split_bf16x2(x[0], x[1], bh[0], bl[0]);
    split_bf16x2(x[2], x[3], bh[1], bl[1]);
  }
}

// The power of two that brings a column's largest magnitude m into [2^13, 2^14) (1 for m = 0), and its
// inverse; both exact.
__device__ __forceinline__ float2 fp16_column_scale(float m) {
  if (!(m > 0.f) || !isfinite(m)) return make_float2(1.f, 1.f);
  const int e = int((__float_as_uint(m) >> 23) & 0xff) - 127;  // m in [2^e, 2^(e+1)) (normal m)
  int k = 13 - e;
  k = k > 126 ? 126 : (k < -126 ? -126 : k);
  return make_float2(__uint_as_float(uint32_t(127 + k) << 23), __uint_as_float(uint32_t(127 - k) << 23));
}

__device__ __forceinline__ void load_a(const uint32_t* frag, int lane, FragA& a) {
  const uint4* p = reinterpret_cast<const uint4*>(frag + lane * 8);
  uint4 h = __ldg(p), l = __ldg(p + 1);
  a.h[0] = h.x;
  a.h[1] = h.y;
  a.h[2] = h.z;
  a.h[3] = h.w;
  a.l[0] = l.x;
  a.l[1] = l.y;
  a.l[2] = l.z;
  a.l[3] = l.w;
}

template <int N, int W, int KIND = kSplitTf32>
struct SmemTc {
  using O = Order<N>;
  static constexpr int Np = O::Np, Nfp = O::Nfp;
  static constexpr int CS = 36;  // column rows (16-byte aligned, few conflicts in fragment loads)
  static constexpr int EPB = 32 / W;
  static constexpr int Q = 4 * Np * CS;
  static constexpr int ST = 4 * Nfp * CS;
  static constexpr int NFPP = O::NFPP;
  static constexpr int XR = 32 * 8 * NFPP;  // face inboxes of the 32 columns
  static constexpr int UX = (3 * Np * CS > XR) ? 3 * Np * CS : XR;
  static constexpr int GS = kGtab + 4;  // coefficient rows: 16-byte aligned, 16-byte loads over lanes conflict-free
  static constexpr int G = EPB * GS + 4;  // coefficients [EPB][GS], rows 16.. shifted by 4 words (see grow)
  static constexpr int IMG = (W == 2) ? 2 * 2 * Np * EPB : 0;  // two FP64 image tiles, in floats
  static constexpr int INTS = 4 * EPB + EPB + EPB + EPB + 128 + 192 + 4 * EPB;  // nbr, finfo bytes, bface, meta, ...
  static constexpr int SC = KIND == kSplitFp16 ? 6 * 32 : 0;  // FP16: column scales (p, r, s) and inverses
  static constexpr size_t bytes_with(bool ring) {
    return (size_t(Q) * (ring ? 3 : 1) + 2 * size_t(ST) + UX + G + IMG + SC) * sizeof(float) + INTS * sizeof(int);
  }
  // the history is staged in shared memory only where that still leaves room for MINB blocks
  static constexpr bool ring_in_smem = TcOrder<N>::MINB * (bytes_with(true) + 1024) <= 228 * 1024;
  static constexpr size_t bytes = bytes_with(ring_in_smem);
  static_assert(4 * Np * CS <= 2 * ST + UX, "right-hand-side staging must fit in the penalty/U region");
};

// BATCH: a merged launch of several shots (BatchArgs); otherwise one shot (B unused)
template <int N, int W, int KIND, bool BATCH = false>
__global__ void __launch_bounds__(TcOrder<N>::NT, TcOrder<N>::MINB)
    dg_step_kernel_tc(const StepArgs<float> A, const std::conditional_t<BATCH, BatchArgs<float>, NoBatch> B) {
  using O = Order<N>;
  using T = TcOrder<N, KIND>;
  constexpr int KS = T::KS;
  // one k-step of the split product: B pieces from shared memory, and the MMA of the split format
  auto load_bk = [](const float* X, int row0, int kv, int t, int col, uint32_t bh[2], uint32_t bl[2], float sc) {
    if constexpr (KIND == kSplitTf32)
      load_b<SmemTc<N, W, KIND>::CS>(X, row0, kv, t, col, bh, bl);
    else
      load_b16<SmemTc<N, W, KIND>::CS, KIND>(X, row0, kv, t, col, bh, bl, sc);
  };
  auto mma = [](float c[4], const uint32_t a[4], const uint32_t b[2]) {
    if constexpr (KIND == kSplitBf16)
      mma_bf16(c, a, b);
    else if constexpr (KIND == kSplitFp16)
      mma_f16(c, a, b);
    else
      mma_tf32(c, a, b);
  };
  using SM = SmemTc<N, W, KIND>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NT = T::NT, NFPP = O::NFPP;
  constexpr int CS = SM::CS, EPB = SM::EPB, GS = SM::GS;
  constexpr bool RING = SM::ring_in_smem;
  constexpr int MT = T::MT, KSD = T::KSD, KSF = T::KSF, NSTEP = T::NSTEP;
  // the k-steps are unrolled (the fragment registers then rotate by renaming)
  constexpr int KUNROLL = 16;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sQ = reinterpret_cast<float*>(smem_raw);  // [4][Np][CS]
  float* sR1 = sQ + SM::Q;                         // [4][Np][CS] (if RING)
  float* sR2 = sR1 + (RING ? SM::Q : 0);           // [4][Np][CS] (if RING)
  float* sS = sR2 + (RING ? SM::Q : 0);            // [4*Nfp][CS]
  float* sT = sS + SM::ST;                         // [4*Nfp][CS]
  float* sU = sT + SM::ST;                         // [3][Np][CS]
  float* sX = sU;                                  // [32 columns][4][2][NFPP] face inboxes (before U)
  float* sG = sU + SM::UX;                         // [EPB][GS] (+4)
  double* sImg = reinterpret_cast<double*>(sG + SM::G);  // W == 2: [2][Np][EPB] image tiles
  int* sI = reinterpret_cast<int*>(sG + SM::G + SM::IMG);
  int* sNbr = sI;                                           // [EPB][4]
  uint8_t* sInfo = reinterpret_cast<uint8_t*>(sNbr + 4 * EPB);  // [EPB][4] face info bytes
  int* sBf = sNbr + 4 * EPB + EPB;                          // [EPB]
  int* sMeta = sBf + EPB;                                   // [EPB]
  int* sFm = sMeta + EPB;                                   // [4][32]
  int* sPerm = sFm + 128;                                   // [6][32]
  int2* sInj = reinterpret_cast<int2*>(sPerm + 192);        // [2][EPB] injection ranges per wavefield
  float* sSc = reinterpret_cast<float*>(sInj + 2 * EPB);   // FP16: [3][32] column scales, [3][32] inverses
  float* sRhs = sS;  // [4][Np][CS] right-hand sides after the products, then the half-step fields

  const int tid = threadIdx.x;
  // merged launch: this block's shot, whose per-shot arguments are staged in shared memory
  __shared__ std::conditional_t<BATCH, ShotArgs<float>, int> sShot;
  int64_t bidx = blockIdx.x;
  if constexpr (BATCH) {
    const int shot = int(blockIdx.x / unsigned(B.shot_blocks));
    bidx -= int64_t(shot) * B.shot_blocks;
    if (tid == 0) {
#pragma unroll
      for (int b = 0; b < kMaxBatch; ++b)
        if (b == shot) sShot = B.shot[b];
    }
    __syncthreads();
  }
  auto WV = [&](int w) -> const WaveArgs<float>& {
    if constexpr (BATCH)
      return sShot.wave[w];
    else
      return A.wave[w];
  };
  // per-shot pointers, read where they are used (kernel parameters stay in the constant bank)
  auto arena_write = [&]() -> float* {
    if constexpr (BATCH)
      return sShot.arena_write;
    else
      return A.arena_write;
  };
  auto arena_read = [&]() -> const float* {
    if constexpr (BATCH)
      return sShot.arena_read;
    else
      return A.arena_read;
  };
  auto image_p = [&]() -> double* {
    if constexpr (BATCH)
      return sShot.image_p;
    else
      return A.image_p;
  };
  auto image_q = [&]() -> double* {
    if constexpr (BATCH)
      return sShot.image_q;
    else
      return A.image_q;
  };
  const int64_t slot0 = A.slot_lo + bidx * EPB;
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
  // coefficient row of element e; elements e and e + 16 (read together by the folds) sit 4 banks apart
  auto grow = [](int e) { return e * GS + ((e >> 4) << 2); };
  auto gcoef = [&](int k, int e) { return sG[grow(e) + k]; };
  auto gcoef4 = [&](int k, int e) { return *reinterpret_cast<const float4*>(sG + grow(e) + k); };

  // ---------------------------------------------------------------- phase 1: asynchronous loads
  // group 0, nothing depends on anything: the tables, the coefficients, the fields at t_start and
  // the face inboxes (the neighbours' traces at t_start, already in this element's face-node order).
  // Then, once the tables are in: group 1, the recorded traces of boundary faces (backward source
  // run only), and group 2, the two older right-hand sides and the image tiles, which only the
  // update needs.  All copies are 16 bytes.
  const int64_t fbase = (blk * 4) * Np * 32 + lane0;
  constexpr int CPR = EPB / 4;  // 16-byte chunks per row and wavefield
  {
    auto copy_bytes = [&](void* dst, const void* src, int bytes) {
      for (int i = tid; i < bytes / 16; i += NT)
        cp_async_bytes16(static_cast<char*>(dst) + 16 * i, static_cast<const char*>(src) + 16 * i);
    };
    copy_bytes(sNbr, A.nbr + slot0 * 4, EPB * 4 * 4);
    copy_bytes(sInfo, A.finfo + slot0 * 4, EPB * 4);
    copy_bytes(sBf, A.bface + slot0, EPB * 4);
    copy_bytes(sMeta, A.meta + slot0, EPB * 4);
    copy_bytes(sFm, A.fmask, 128 * 4);
    copy_bytes(sPerm, A.perm, 192 * 4);
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      if (w < W && WV(w).amp_mode != 0) {
        copy_bytes(sInj + w * EPB, WV(w).inj_range + slot0, EPB * 8);
      } else {
        for (int i = tid; i < EPB; i += NT) sInj[w * EPB + i] = make_int2(0, 0);
      }
    }
    constexpr int CPE = kGtab / 4;  // 16-byte chunks per element
    for (int i = tid; i < EPB * CPE; i += NT) {
      const int e = i / CPE, ch = i - e * CPE;
      cp_async_bytes16(sG + grow(e) + ch * 4, A.gtab + (slot0 + e) * kGtab + ch * 4);
    }
    constexpr int PER = 4 * Np * 8;  // 16-byte chunks of one field array (8 per 32-column row)
    for (int i = tid; i < PER; i += NT) {
      const int row = i >> 3, sub = i & 7;  // sub = w * CPR + ch
      const int w = sub / CPR, ch = sub - w * CPR;
      cp_async_bytes16(sQ + row * CS + sub * 4, WV(w).q + fbase + row * 32 + ch * 4);
    }
    constexpr int CHW = EPB * 8 * NFPP / 4;  // 16-byte chunks of one wavefield's inboxes
    for (int i = tid; i < W * CHW; i += NT) {
      const int w = i / CHW, ch = i - w * CHW;
      cp_async_bytes16(sX + w * (EPB * 8 * NFPP) + ch * 4,
                       WV(w).trace + (int64_t(A.trace_read) * A.n_slots + slot0) * (8 * NFPP) + ch * 4);
    }
    cp_async_commit();
    // the history slices this block reads from global memory in the update: into L2 now
    if (!RING && !rhs_only && tid < 2 * W) {
      const int w = tid >> 1, ring = (tid & 1) ? r2i : r1i;
      const float* src = WV(w).ring + ring * qsize + blk * 4 * Np * 32;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"(4 * Np * 32 * 4) : "memory");
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  // recorded forward traces as the exterior state of boundary faces (backward source run), into the
  // inbox places of those faces; only blocks that have boundary faces take part
  bool replay_block = false;
  if (A.mode & kModeReplay) {
    int nlast = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) nlast += finfo_bc(sInfo[(EPB - 1) * 4 + f]) != 0;
    replay_block = sBf[EPB - 1] + nlast > sBf[0];
    if (replay_block) {
      constexpr int CHI = 2 * NFPP / 4;  // 16-byte chunks per face record
      for (int i = tid; i < EPB * 4 * CHI; i += NT) {
        const int item = i / CHI, ch = i - item * CHI;
        const int e = item >> 2, f = item & 3;
        if (!(sMeta[e] & kMetaValid) || finfo_bc(sInfo[e * 4 + f]) == 0) continue;
        int b = sBf[e];
        for (int ff = 0; ff < f; ++ff) b += (finfo_bc(sInfo[e * 4 + ff]) != 0);
        cp_async_bytes16(sX + e * (8 * NFPP) + f * 2 * NFPP + ch * 4,
                         arena_read() + (A.arena_offset + b) * (2 * NFPP) + ch * 4);
      }
    }
  }
  cp_async_commit();
  // the history (and the image tiles), needed only by the update
  if (RING && !rhs_only) {
    constexpr int PER = 4 * Np * 8;
    for (int arr = 1; arr < 3; ++arr) {
      const int ring = arr == 1 ? r1i : r2i;
      float* dbase = arr == 1 ? sR1 : sR2;
      for (int i = tid; i < PER; i += NT) {
        const int row = i >> 3, sub = i & 7;
        const int w = sub / CPR, ch = sub - w * CPR;
        cp_async_bytes16(dbase + row * CS + sub * 4, WV(w).ring + ring * qsize + fbase + row * 32 + ch * 4);
      }
    }
  }
  if (W == 2 && (A.mode & kModeImage)) {
    constexpr int CPN = EPB * 8 / 16;  // 16-byte chunks per node row of one image
    for (int i = tid; i < 2 * Np * CPN; i += NT) {
      const int im = i / (Np * CPN), rem = i - im * Np * CPN;
      if (!(A.mode & (im == 0 ? kModeImageP : kModeImageQ))) continue;
      const int n = rem / CPN, ch = rem - n * CPN;
      const double* src = (im == 0 ? image_p() : image_q()) + (blk * Np + n) * 32 + lane0 + ch * 2;
      cp_async_bytes16(sImg + (im * Np + n) * EPB + ch * 2, src);
    }
  }
  cp_async_commit();
  if (replay_block) {
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
  }

  // ---------------------------------------------------------------- phase 2: face penalties
  // half-warp per (face, column) item, lanes over face nodes; the two half-warps of a warp take
  // neighbouring columns of the same face.  Interior faces take the neighbour's traces at t_start
  // from the inbox; boundary faces use the ghost state of their condition, or, in the backward
  // source run, the recorded forward traces; forward runs record the traces of boundary faces.
  // All items are evaluated before any is stored.
  {
    constexpr int NH = NT / 16;               // half-warps
    constexpr int NU = (128 + NH - 1) / NH;   // items per half-warp
    constexpr int NJ = (Nfp + 15) / 16;       // face nodes per lane
    static_assert(NH % 2 == 0, "half-warp pairs must share a face");
    const int hw = tid >> 4, j = tid & 15;
    const int par = hw & 1;  // the odd half-warp reads n.v before p: no bank conflicts between the halves
    float tv[NU][NJ], sv[NU][NJ], pv[NU][NJ], vv[NU][NJ];
    bool recu[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int item = hw + u * NH;
      recu[u] = false;
      if (item >= 128) continue;
      const int c = item & 31, f = item >> 5;
      const int e = col_e(c), w = col_w(c);
      const bool valid = (sMeta[e] & kMetaValid) != 0;
      const int bc = finfo_bc(sInfo[e * 4 + f]);
      const float4 nf = gcoef4(kGtN + 4 * f, e), pf = gcoef4(kGtP + 4 * f, e);
      const float n0 = nf.x, n1 = nf.y, n2 = nf.z;
      const float pa = pf.x, pb = pf.y, pcc = pf.z, pd = pf.w;
      recu[u] = bc != 0 && valid && w == 0 && (A.mode & kModeRecord);
      const bool ext = bc == 0 || (w == 0 && (A.mode & kModeReplay));
      const float* xb = sX + c * (8 * NFPP) + f * 2 * NFPP;
#pragma unroll
      for (int t = 0; t < NJ; ++t) {
        const int jj = j + 16 * t;
        if (jj >= Nfp) continue;
        const int n = sFm[f * 32 + jj];
        const float p = sQ[(0 * Np + n) * CS + c];
        const float vn = n0 * sQ[(1 * Np + n) * CS + c] + n1 * sQ[(2 * Np + n) * CS + c] + n2 * sQ[(3 * Np + n) * CS + c];
        pv[u][t] = p;
        vv[u][t] = vn;
        float jp, jv;
        if (ext) {
          // exterior state in our node order and with our normal: the neighbour's traces, or the
          // recorded traces of this very face
          const float x1 = xb[par * NFPP + jj], x2 = xb[(1 - par) * NFPP + jj];
          jp = (par ? x2 : x1) - p;
          jv = (par ? x1 : x2) - vn;
        } else if (bc == 1) {  // free surface: p+ = -p-, n.v+ = n.v-
          jp = -2.f * p;
          jv = 0.f;
        } else if (bc == 2) {  // transparent: p+ = 0, v+ = 0
          jp = -p;
          jv = -vn;
        } else {  // rigid: p+ = p-, n.v+ = -n.v-
          jp = 0.f;
          jv = -2.f * vn;
        }
        tv[u][t] = valid ? pa * jv + pb * jp : 0.f;
        sv[u][t] = valid ? pcc * jp + pd * jv : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int item = hw + u * NH;
      if (item >= 128) continue;
      const int c = item & 31, f = item >> 5;
      float* rec = nullptr;
      if (recu[u]) {
        const int e = col_e(c);
        int b = sBf[e];
        for (int ff = 0; ff < f; ++ff) b += (finfo_bc(sInfo[e * 4 + ff]) != 0);
        rec = arena_write() + (A.arena_offset + b) * (2 * NFPP);
      }
#pragma unroll
      for (int t = 0; t < NJ; ++t) {
        const int jj = j + 16 * t;
        if (jj >= Nfp) continue;
        const int fj = f * Nfp + jj;
        sT[fj * CS + c] = tv[u][t];
        sS[fj * CS + c] = sv[u][t];
        if (rec) {
          rec[jj] = pv[u][t];
          rec[NFPP + jj] = vv[u][t];
        }
      }
    }
  }
  __syncthreads();

// ---------------------------------------------------------------- phase 2c: U_j = G_p v
  for (int i = tid; i < Np * 32; i += NT) {
    int c = i & 31, m = i >> 5;
    const int e = col_e(c);
    float vx = sQ[(1 * Np + m) * CS + c], vy = sQ[(2 * Np + m) * CS + c], vz = sQ[(3 * Np + m) * CS + c];
    const float4 g0 = gcoef4(kGtU, e), g1 = gcoef4(kGtU + 4, e);
    const float g8 = gcoef(kGtU + 8, e);
    // U_jd = sum_i (-rho c^2 rx_{i,jd}) v_i
    sU[(0 * Np + m) * CS + c] = g0.x * vx + g0.w * vy + g1.z * vz;
    sU[(1 * Np + m) * CS + c] = g0.y * vx + g1.x * vy + g1.w * vz;
    sU[(2 * Np + m) * CS + c] = g0.z * vx + g1.y * vy + g8 * vz;
  }
  __syncthreads();
  // FP16 split: per-column power-of-two scales of the product operands, from their largest magnitudes:
  // p (the derivatives D_j p, one accumulator each), U_j with the penalty traces t (both accumulate
  // into r_p), and s (each L_f s_f its own accumulator).  sSc[0..2][c] scales, sSc[3..5][c] inverses.
  if constexpr (KIND == kSplitFp16) {
    for (int task = tid; task < 6 * 32; task += NT) {
      const int c = task & 31, part = task >> 5;
      const float* X = part == 0 ? sQ : (part <= 3 ? sU + (part - 1) * Np * CS : (part == 4 ? sT : sS));
      const int rows = part <= 3 ? Np : 4 * Nfp;
      float m = 0.f;
      for (int r = 0; r < rows; ++r) m = fmaxf(m, fabsf(X[r * CS + c]));
      sSc[task] = m;
    }
    __syncthreads();
    if (tid < 32) {
      float mx[6];
#pragma unroll
      for (int part = 0; part < 6; ++part) mx[part] = sSc[part * 32 + tid];
      const float2 sp = fp16_column_scale(mx[0]);
      const float2 sr = fp16_column_scale(fmaxf(fmaxf(mx[1], mx[2]), fmaxf(mx[3], mx[4])));
      const float2 ss = fp16_column_scale(mx[5]);
      sSc[0 * 32 + tid] = sp.x;
      sSc[1 * 32 + tid] = sr.x;
      sSc[2 * 32 + tid] = ss.x;
      sSc[3 * 32 + tid] = sp.y;
      sSc[4 * 32 + tid] = sr.y;
      sSc[5 * 32 + tid] = ss.y;
    }
    __syncthreads();
  }

// ---------------------------------------------------------------- phase 3: tensor-core products
  const int lane = tid & 31, wid = tid >> 5;
  const int mt = wid >> 1, pair = wid & 1;
  const int g = lane >> 2, t4 = lane & 3;
  // Column block beta (0..3) holds the data columns 4 beta + {0..3} and 16 + 4 beta + {0..3}; fragment
  // column n of block beta is data column bcol(beta, n).  With rows of 36 floats this makes every
  // B-fragment load (lanes: row t4 or t4 + 4, column bcol(g)) hit 32 distinct banks.  Warp pair
  // takes blocks pair and pair + 2.
  auto bcol = [](int beta, int n) { return 4 * beta + (n & 3) + 16 * (n >> 2); };
  const int colb[2] = {bcol(pair, g), bcol(pair + 2, g)};  // B-fragment columns of the two blocks
  // FP16: the operand scales of the B-fragment columns (p, r, s), 1 for the other split formats
  float scp[2] = {1.f, 1.f}, scr[2] = {1.f, 1.f}, scs[2] = {1.f, 1.f};
  if constexpr (KIND == kSplitFp16) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      scp[b] = sSc[0 * 32 + colb[b]];
      scr[b] = sSc[1 * 32 + colb[b]];
      scs[b] = sSc[2 * 32 + colb[b]];
    }
  }
  // FP16: the inverse scale of accumulator column (b, k) of operand family fam (0 p, 1 r, 2 s)
  auto inv_sc = [&](int fam, int b, int k) {
    if constexpr (KIND == kSplitFp16)
      return sSc[(3 + fam) * 32 + bcol(pair + 2 * b, 2 * t4 + k)];
    else
      return 1.f;
  };
  // accumulator entry q = 2 hn + k of block b: node mt*16 + g + 8 hn, column bcol(pair + 2b, 2 t4 + k).
  // r_p = sum_j D_j U_j + sum_f L_f t_f (Eq. dgLocalSchemeP) accumulates in rp; each D_j p and each
  // L_f s_f is folded into r_v = -(1/rho) grad p - sum_f n_f (L_f s_f) (Eq. dgLocalSchemeU) as soon
  // as it is complete.
  float rp[2][4], rv[3][2][4];
  int ecol[2][2];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
#pragma unroll
    for (int k = 0; k < 2; ++k) ecol[b][k] = col_e(bcol(pair + 2 * b, 2 * t4 + k));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      rp[b][q] = 0.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) rv[d][b][q] = 0.f;
    }
  }
  {
    // operator fragments stream from L2 three steps ahead of their use; unrolled steps rotate the
    // fragment registers by renaming (a register copy would wait for the load to land)
    const uint32_t* fr = A.afrag + mt * (NSTEP * 256);
    // lanes whose fragment rows all lie beyond the last node (possible in the last tile) skip the
    // load: their fragment is zero
    const bool lane_rows = mt < MT - 1 || (lane >> 2) < T::LAST_ROWS;
    auto fetch = [&](const uint32_t* f, FragA& a) {
      if (lane_rows) {
        load_a(f, lane, a);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) a.h[q] = a.l[q] = 0u;
      }
    };
    FragA F0, F1, F2;
    fetch(fr, F0);
    fetch(fr + (NSTEP > 1 ? 256 : 0), F1);
    fetch(fr + (NSTEP > 2 ? 512 : 0), F2);
    auto next = [&](int s) {
      FragA F3 = F2;
      if (s + 3 < NSTEP) fetch(fr + (s + 3) * 256, F3);
      return F3;
    };
#pragma unroll
    for (int jd = 0; jd < 3; ++jd) {
      const float* Ub = sU + jd * Np * CS;
      float acc[2][4];
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[b][q] = 0.f;
#pragma unroll(KUNROLL)
      for (int kb = 0; kb < KSD; ++kb) {
        const FragA F3 = next(jd * KSD + kb);
        const int kv = Np - kb * KS;
        uint32_t ph[2][2], pl[2][2], uh[2][2], ul[2][2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          load_bk(sQ, kb * KS, kv, t4, colb[b], ph[b], pl[b], scp[b]);
          load_bk(Ub, kb * KS, kv, t4, colb[b], uh[b], ul[b], scr[b]);
        }
        // the three split terms of four independent accumulators, interleaved
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          mma(acc[b], F0.l, ph[b]);
          mma(rp[b], F0.l, uh[b]);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          mma(acc[b], F0.h, pl[b]);
          mma(rp[b], F0.h, ul[b]);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          mma(acc[b], F0.h, ph[b]);
          mma(rp[b], F0.h, uh[b]);
        }
        F0 = F1;
        F1 = F2;
        F2 = F3;
      }
      // r_v += (-rx_{d,jd} / rho) D_jd p
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const float iv = inv_sc(0, b, k);
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float gvk = gcoef(kGtV + 3 * d + jd, ecol[b][k]) * iv;
            rv[d][b][k] += gvk * acc[b][k];
            rv[d][b][2 + k] += gvk * acc[b][2 + k];
          }
        }
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      float acc[2][4];
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[b][q] = 0.f;
#pragma unroll(KUNROLL)
      for (int kb = 0; kb < KSF; ++kb) {
        const FragA F3 = next(3 * KSD + f * KSF + kb);
        const int kv = Nfp - kb * KS;
        uint32_t th[2][2], tl[2][2], sh[2][2], sl[2][2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          load_bk(sT, f * Nfp + kb * KS, kv, t4, colb[b], th[b], tl[b], scr[b]);
          load_bk(sS, f * Nfp + kb * KS, kv, t4, colb[b], sh[b], sl[b], scs[b]);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          mma(rp[b], F0.l, th[b]);
          mma(acc[b], F0.l, sh[b]);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          mma(rp[b], F0.h, tl[b]);
          mma(acc[b], F0.h, sl[b]);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          mma(rp[b], F0.h, th[b]);
          mma(acc[b], F0.h, sh[b]);
        }
        F0 = F1;
        F1 = F2;
        F2 = F3;
      }
      // r_v -= n_f (L_f s_f)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const float4 nf = gcoef4(kGtN + 4 * f, ecol[b][k]);
          const float iv = inv_sc(2, b, k);
          const float nfd[3] = {nf.x * iv, nf.y * iv, nf.z * iv};
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            rv[d][b][k] -= nfd[d] * acc[b][k];
            rv[d][b][2 + k] -= nfd[d] * acc[b][2 + k];
          }
        }
    }
  }
  __syncthreads();  // the products have read sS, sT and sU: they now hold the right-hand sides

  // ---------------------------------------------------------------- phase 4a: right-hand sides
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = mt * 16 + g + 8 * (q >> 1);
      if (n >= Np) continue;
      const int cb = bcol(pair + 2 * b, 2 * t4 + (q & 1));
      sRhs[(0 * Np + n) * CS + cb] = rp[b][q] * inv_sc(1, b, q & 1);
#pragma unroll
      for (int d = 0; d < 3; ++d) sRhs[((1 + d) * Np + n) * CS + cb] = rv[d][b][q];
    }
  cp_async_wait_all();  // the history slots and image tiles
  __syncthreads();

  // ---------------------------------------------------------------- phase 4b: update
  // thread per (node, element), all its wavefields: point injections, the images from the fields
  // and histories at t_start (Eq. updateABcorr), the new fields (Eq. updateAB) and the half-step
  // fields (Eq. updateABcoarse).  One wavefield: a warp per node row.  Two: the half-warps take
  // rows n and n + 4 (36-float rows: disjoint banks).  Shared-memory accesses are conflict-free and
  // global stores are 32 (or 2 x 16) consecutive columns.
  constexpr int NE = W == 1 ? Np * 32 : 4 * ((Np + 7) / 8) * 32;  // entry slots
#pragma unroll 2
  for (int i = tid; i < NE; i += NT) {
    int n, e;
    if (W == 1) {
      n = i >> 5;
      e = i & 31;
    } else {
      const int j = i >> 5;
      n = 8 * (j >> 2) + (j & 3) + 4 * ((i >> 4) & 1);
      e = i & 15;
      if (n >= Np) continue;
    }
    const bool ok = (sMeta[e] & kMetaValid) != 0;
    const int64_t gofs = ((blk * 4) * Np + n) * 32 + lane0 + e;
    float r[W][4], q0[W][4], r1[W][4], r2[W][4];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const int c = w * 16 + e;
#pragma unroll
      for (int fld = 0; fld < 4; ++fld) {
        const int sidx = (fld * Np + n) * CS + c;
        r[w][fld] = sRhs[sidx];
        q0[w][fld] = sQ[sidx];
      }
      // point injections (source wavelet or receiver traces)
      const WaveArgs<float>& wa = WV(w);
      const int2 ir = sInj[w * EPB + e];
      if (ir.y > 0 && ok) {
        for (int qq = ir.x; qq < ir.x + ir.y; ++qq) {
          float amp;
          if (wa.amp_mode == 1) {
            amp = wa.amp;
          } else {
            double acc = 0.0;
            const int row = wa.inj_row[qq];
            for (int tt = 0; tt < 4; ++tt) {
              const int nt = A.interp_n0 + tt;
              if (nt >= 0 && nt < wa.n_time) acc += A.interp_w[tt] * wa.data[int64_t(row) * wa.n_time + nt];
            }
            if (wa.data_scale) acc *= *wa.data_scale;
            amp = float(acc);
          }
          r[w][0] += amp * wa.inj_w[int64_t(qq) * Np + n];
        }
      }
    }
    if (rhs_only) {
      if (ok)
#pragma unroll
        for (int fld = 0; fld < 4; ++fld) A.rhs_out[gofs + fld * Np * 32] = r[0][fld];
      continue;
    }
#pragma unroll
    for (int w = 0; w < W; ++w)
#pragma unroll
      for (int fld = 0; fld < 4; ++fld) {
        if constexpr (RING) {
          const int sidx = (fld * Np + n) * CS + w * 16 + e;
          r1[w][fld] = sR1[sidx];
          r2[w][fld] = sR2[sidx];
        } else {
          r1[w][fld] = WV(w).ring[r1i * qsize + gofs + fld * Np * 32];
          r2[w][fld] = WV(w).ring[r2i * qsize + gofs + fld * Np * 32];
        }
      }
    // images from the fields and histories at t_start, before the update
    if (W == 2 && (A.mode & kModeImage) && ok) {
      const int wR = W - 1;  // receiver wavefield (1 when W == 2)
      const float Z = gcoef(kGtZ, e);
      const float* eu = A.e_up;
      auto up = [&](const float* x) { return eu[0] * x[1] + eu[1] * x[2] + eu[2] * x[3]; };
      const float xS = q0[0][0], xR = q0[wR][0];
      const float vS = up(q0[0]), vR = up(q0[wR]);
      const float rS[3] = {r[0][0], r1[0][0], r2[0][0]};
      const float rR[3] = {r[wR][0], r1[wR][0], r2[wR][0]};
      const float sS3[3] = {rS[0] - Z * up(r[0]), rS[1] - Z * up(r1[0]), rS[2] - Z * up(r2[0])};
      const float sR3[3] = {rR[0] + Z * up(r[wR]), rR[1] + Z * up(r1[wR]), rR[2] + Z * up(r2[wR])};
      const float cc[3] = {float(AB::c1), float(AB::c2), float(AB::c3)};
      const float C[3][3] = {{float(4703.0 / 5040.0), float(-457.0 / 840.0), float(52.0 / 315.0)},
                             {float(-457.0 / 840.0), float(103.0 / 315.0), float(-251.0 / 2520.0)},
                             {float(52.0 / 315.0), float(-251.0 / 2520.0), float(17.0 / 560.0)}};
      const float qS = xS - Z * vS, qR = xR + Z * vR;
      float t2p = 0.f, t3p = 0.f, t2q = 0.f, t3q = 0.f;
#pragma unroll
      for (int s3 = 0; s3 < 3; ++s3) {
        t2p += cc[s3] * (xS * rR[s3] + rS[s3] * xR);
        t2q += cc[s3] * (qS * sR3[s3] + sS3[s3] * qR);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          t3p += C[s3][u] * rS[s3] * rR[u];
          t3q += C[s3][u] * sS3[s3] * sR3[u];
        }
      }
      const float incP = h * (xS * xR + h * (t2p + h * t3p));
      const float incQ = h * (qS * qR + h * (t2q + h * t3q));
      const int64_t io = (blk * Np + n) * 32 + lane0 + e;
      if (A.mode & kModeImageP) image_p()[io] = sImg[(0 * Np + n) * EPB + e] - double(incP);
      if (A.mode & kModeImageQ) image_q()[io] = sImg[(1 * Np + n) * EPB + e] - double(incQ);
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
      float* qg = WV(w).q + gofs;
      float* rg = WV(w).ring + rn * qsize + gofs;
#pragma unroll
      for (int fld = 0; fld < 4; ++fld) {
        const float rr = r[w][fld];
        const float upd = float(AB::a1) * rr + float(AB::a2) * r1[w][fld] + float(AB::a3) * r2[w][fld];
        const float hb = float(AB::b1) * rr + float(AB::b2) * r1[w][fld] + float(AB::b3) * r2[w][fld];
        const float qn = q0[w][fld] + h * upd;
        const int sidx = (fld * Np + n) * CS + w * 16 + e;
        sQ[sidx] = qn;
        sRhs[sidx] = q0[w][fld] + h * hb;  // half-step fields, in place
        if (ok) {
          qg[fld * Np * 32] = qn;
          rg[fld * Np * 32] = rr;
        }
      }
    }
  }
  if (rhs_only) return;
  __syncthreads();

// ---------------------------------------------------------------- phase 5: traces
  // pushed into the neighbour's inbox: face f2 of slot s2, at the neighbour's face-node index
  // perm[j] of our node j (the correspondences of the two sides are mutually inverse), with n.v
  // taken with the neighbour's normal; half-step traces too where a finer neighbour needs them.
  // Boundary faces have no reader.
  {
    const float* sH = sRhs;
    const int hw = tid >> 4, j = tid & 15;
    const int ws = A.trace_write[lev], hs = A.trace_half[lev];
#pragma unroll 4
    for (int item = hw; item < 32 * 4; item += NT / 16) {
      const int c = item & 31, f = item >> 5;
      const int e = col_e(c), w = col_w(c);
      const int meta = sMeta[e];
      const int info = sInfo[e * 4 + f];
      if (!(meta & kMetaValid) || finfo_bc(uint8_t(info)) != 0) continue;
      const float4 nf = gcoef4(kGtN + 4 * f, e);
      const float n0 = nf.x, n1 = nf.y, n2 = nf.z;
      const int64_t s2 = sNbr[e * 4 + f];
      const int* pm = sPerm + finfo_perm(uint8_t(info)) * 32;
      const int64_t fo = s2 * (8 * NFPP) + finfo_face(uint8_t(info)) * 2 * NFPP;
      float* tw = WV(w).trace + int64_t(ws) * A.n_slots * (8 * NFPP) + fo;
      float* th = WV(w).trace + int64_t(hs) * A.n_slots * (8 * NFPP) + fo;
      for (int jj = j; jj < Nfp; jj += 16) {
        const int n = sFm[f * 32 + jj];
        const int j2 = pm[jj];
        const float p = sQ[(0 * Np + n) * CS + c];
        const float vn = n0 * sQ[(1 * Np + n) * CS + c] + n1 * sQ[(2 * Np + n) * CS + c] + n2 * sQ[(3 * Np + n) * CS + c];
        tw[j2] = p;
        tw[NFPP + j2] = -vn;
        if (meta & kMetaHalf) {
          const float ph = sH[(0 * Np + n) * CS + c];
          const float vh =
              n0 * sH[(1 * Np + n) * CS + c] + n1 * sH[(2 * Np + n) * CS + c] + n2 * sH[(3 * Np + n) * CS + c];
          th[j2] = ph;
          th[NFPP + j2] = -vh;
        }
      }
    }
  }
}

}  // namespace ridg
