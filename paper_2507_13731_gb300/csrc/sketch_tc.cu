// tcgen05 tensor-core sketch products  Y = A X  (op N)  and  Z = A^H Y  (op H).
//
// The Hamilton product of eq. (1) (Section 2), summed over the inner index, is one real GEMM of
// the plane-stacked A against a sign-structured expansion of the thin sketch:
//     Y_d = sum_c  s(c, d) * A_c * X_{c xor d}          (op N)
//     Z_d = sum_c  s'(c, d) * A_c^T * Y_{c xor d}       (op H, A^H = A1^T - A2^T i - A3^T j - A4^T k)
// with s(c, d) = -1 exactly for (c, d) in {(1,0),(2,0),(3,0),(1,2),(2,3),(3,1)} and
// s'(c, d) = -s(c, d) for c != 0.  The expansion is never materialised: each (c, d) pair is one
// tcgen05.mma of A's plane-c tile against X's plane (c xor d) tile, with the instruction
// descriptor's negate-B bit carrying the sign, accumulating into output plane d's TMEM columns.
//
// Per CTA: a 128-row tile of the output (M = m for op N, M = n for op H) and a block of nb <= 128
// output columns of all four planes (4 nb <= 512 TMEM columns), over a contiguous range of the
// reduction (stream-K when the tiles do not fill whole waves: every SM takes an equal share of
// the tiles' reduction stages; with several column blocks, one CTA per block in each group, so the
// blocks read every A stage together and A comes from DRAM about once).  A's tiles come through
// TMA into a 2-8 stage shared-memory ring.  Op N stages A K-major (TMA swizzled tiles).  Op H reads A along
// its rows: for BF16 the MMA consumes the MN-major tile directly; for the 4-byte modes the tile is
// loaded unswizzled and the worker warps transpose it into the K-major swizzled layout (splitting
// it into hi / lo on the way for 3xTF32).
// Warp roles: 0 = TMA producer, 1 = MMA issuer (owns TMEM), 2-3 = workers (hi/lo split,
// rounding and/or transpose of A), 4-7 = epilogue (TMEM -> registers -> global, or a stream-K
// partial + the last piece's reduction).
//
// Precision modes: BF16 (kind::f16, A stored BF16, X rounded to BF16), TF32 (kind::tf32, one
// product on FP32 data, which the tensor cores truncate to TF32), rounded TF32 (one product, A and
// X rounded to the nearest TF32 value first: by the staging kernel for X, by the worker warps in
// shared memory for A), TF32X3 (kind::tf32: A = A_hi + A_lo and X = X_hi + X_lo with A_hi = A
// with its 13 low mantissa bits cleared, three products A_hi X_hi + A_lo X_hi + A_hi X_lo).
// Accumulation is FP32 in TMEM throughout; the FP32-accurate modes (TF32X3, rounded TF32) add it
// in chunks summed with round-to-nearest.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "qlr_internal.h"
#include "tc_common.cuh"

namespace {

using namespace qlr_tc;

constexpr int TC_THREADS = 256;
constexpr int TBM = 128;          // output rows per CTA (MMA M)
constexpr int MAX_STAGES = 8;    // pipeline stages (as many as fit in shared memory, at most 8)
constexpr int PMAX_STAGES = MAX_STAGES;

enum Kind { K_BF16 = 0, K_TF32 = 1, K_TF32X3 = 2 };
enum AMode { A_K = 0, A_MN = 1, A_T = 2 };   // K-major TMA, MN-major descriptors, transposed by workers

struct TcParams {
  CUtensorMap tmA[4];
  CUtensorMap tmX[4];
  CUtensorMap tmXlo[4];
  float* y[4];
  int64_t ldy;
  float* part;              // stream-K partial tiles (two slots per CTA)
  unsigned* counters;       // one arrival counter per output tile
  int64_t M;                // output rows
  int l;                    // valid output columns
  int nb;                   // output columns per CTA block
  int ncb;                  // column blocks
  int kiters;               // K stages in total
  int mtiles;               // row tiles (the stream-K kernel's tile count is mtiles * ncb)
  int c_first;              // 1 for a pure quaternion A (plane 0 absent)
  uint32_t neg_mask;        // bit c*4+d set: negate the (c, d) product
  uint32_t idesc_base;
  uint32_t tmem_cols;
  int stages;
  int* err;
  int flush;                // K stages per accumulation chunk (0: the whole piece in one chunk)
  int nbuf;                 // TMEM chunk accumulators (2: the MMA fills one while the other drains)
  int ttotal;               // 1: the chunks' running sum is kept in TMEM columns [4 nb, 8 nb)
  int apl;                  // A planes per stage: 3 for a pure quaternion A (plane 0 absent), else 4
  int fd;                   // 1: fused output planes (one MMA per input plane, N = 4 nb; see issue_stage)
  int rn;                   // 1 (TF32): A rounded to nearest TF32 in shared memory before the MMAs read it
  int cgroup;               // stream-K in column-block groups (gridDim.x a multiple of ncb)
};

// The scalar part of TcParams, copied into registers once: with the parameters in global memory
// (grouped launches), every asm statement with a memory clobber and every store of the output
// would otherwise force the fields to be reloaded.
struct TcScalars {
  float *y0, *y1, *y2, *y3;                // output planes (selected without an indexed array)
  int64_t ldy;
  float* part;
  unsigned* counters;
  int64_t M;
  int l, nb, ncb, kiters, c_first, stages;
  uint32_t neg_mask, idesc_base, tmem_cols;
  int* err;
  int flush, nbuf, ttotal, apl, fd, rn;
  __device__ __forceinline__ float* y(int d) const { return d == 0 ? y0 : d == 1 ? y1 : d == 2 ? y2 : y3; }
};
__device__ __forceinline__ TcScalars tc_scalars(const TcParams& p) {
  TcScalars v;
  v.y0 = p.y[0]; v.y1 = p.y[1]; v.y2 = p.y[2]; v.y3 = p.y[3];
  v.ldy = p.ldy; v.part = p.part; v.counters = p.counters; v.M = p.M; v.l = p.l; v.nb = p.nb; v.ncb = p.ncb;
  v.kiters = p.kiters; v.c_first = p.c_first; v.stages = p.stages;
  v.neg_mask = p.neg_mask; v.idesc_base = p.idesc_base; v.tmem_cols = p.tmem_cols; v.err = p.err;
  v.flush = p.flush; v.nbuf = p.nbuf < 1 ? 1 : p.nbuf; v.ttotal = p.ttotal; v.apl = p.apl == 3 ? 3 : 4; v.fd = p.fd;
  v.rn = p.rn;
  return v;
}

// Round an FP32 value to the nearest TF32 value (10 explicit mantissa bits, ties away from zero).
// The tensor cores read a 4-byte operand's top 19 bits and drop the rest, which rounds every
// element toward zero: on data of one sign that shrinks a product by ~2^-12 relative on average.
__device__ __forceinline__ uint32_t tf32_rna(uint32_t bits) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(__uint_as_float(bits)));
  return r;
}
__device__ __forceinline__ uint4 tf32_rna4(uint4 v) {
  return make_uint4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
}

// ---------------------------------------------------------------------------------------
template <int KIND>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
  if (KIND == K_BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  }
}
// Stage geometry.  WIDE (K-major A, column blocks of at most 64): 128-byte rows per stage (128 B
// swizzle), so every TMA row fetch of A moves 128 contiguous bytes; otherwise 64-byte rows.
template <int KIND, bool WIDE = false> struct Cfg;
template <> struct Cfg<K_BF16, false> {     // 2-byte operands, 64 B swizzle, 32 K-elements per stage
  static constexpr int ESZ = 2, SW = 64, BK = 32, MMA_K = 16, MODE = 4;
};
template <> struct Cfg<K_BF16, true> {      // 2-byte operands, 128 B swizzle, 64 K-elements per stage
  static constexpr int ESZ = 2, SW = 128, BK = 64, MMA_K = 16, MODE = 2;
};
template <> struct Cfg<K_TF32, false> {     // 4-byte operands, 64 B swizzle, 16 K-elements per stage
  static constexpr int ESZ = 4, SW = 64, BK = 16, MMA_K = 8, MODE = 4;
};
template <> struct Cfg<K_TF32, true> {      // 4-byte operands, 128 B swizzle, 32 K-elements per stage
  static constexpr int ESZ = 4, SW = 128, BK = 32, MMA_K = 8, MODE = 2;
};
template <> struct Cfg<K_TF32X3, false> {   // 4-byte operands, 32 B swizzle, 8 K-elements per stage
  static constexpr int ESZ = 4, SW = 32, BK = 8, MMA_K = 8, MODE = 6;
};
template <> struct Cfg<K_TF32X3, true> : Cfg<K_TF32X3, false> {};

// ---------------------------------------------------------------------------------------
// MMA issue.  The shared-memory descriptors of stage 0's operand tiles are built once; stage s
// and K step ks only move the start address, whose field holds (address >> 4) in the low 14 bits
// of the descriptor, so they are plain 64-bit additions.  A stage is then issued as a fully
// unrolled run of tcgen05.mma with no per-MMA address arithmetic: with 64-column blocks an MMA
// takes ~32 tensor-pipe cycles, so the issuing thread must spend only a few instructions on each.
struct StageDescs {
  uint64_t a[4], alo[4], x[4], xlo[4];
  uint64_t sstep;                 // one stage, in descriptor address units (16 bytes)
};

template <int KIND, int AMODE, bool WIDE = false>
__device__ __forceinline__ StageDescs make_stage_descs(uint32_t sbase, int stage_bytes, int hi_off, int a_bytes,
                                                       int a_set, int x_bytes, int apl, int nxp) {
  using C = Cfg<KIND, WIDE>;
  StageDescs D;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    // plane c of the hi (and lo) set at slot c - (4 - apl): hi_off is the set's offset minus
    // (4 - apl) planes; the slots of absent planes are never used
    const uint32_t ah = sbase + (uint32_t)(hi_off + c * a_bytes), al = ah + (uint32_t)(apl * a_bytes);
    if (AMODE == A_MN) {   // MN-major: LBO = stride between MN atoms, SBO = stride between 8-row K groups
      D.a[c] = make_desc(ah, C::BK * C::SW, 8 * C::SW, C::MODE);
      D.alo[c] = make_desc(al, C::BK * C::SW, 8 * C::SW, C::MODE);
    } else {
      D.a[c] = make_desc(ah, 16, 8 * C::SW, C::MODE);
      D.alo[c] = make_desc(al, 16, 8 * C::SW, C::MODE);
    }
    // X tile c of the hi (and lo) set: nxp tiles of x_bytes each
    const uint32_t xh = sbase + (uint32_t)(a_set + c * x_bytes), xl = xh + (uint32_t)(nxp * x_bytes);
    D.x[c] = make_desc(xh, 16, 8 * C::SW, C::MODE);
    D.xlo[c] = make_desc(xl, 16, 8 * C::SW, C::MODE);
  }
  D.sstep = (uint64_t)(stage_bytes >> 4);
  return D;
}

// All MMAs of stage s into the accumulator at TMEM column abase (output plane d at abase + d nb).
// Plain form: per K step and input plane c, one MMA per output plane d of A_c against X_{c xor d}
// (three for 3xTF32: hi hi, lo hi, hi lo), the sign of the Hamilton product in the negate-B bit.
// Fused form (fd): per K step and input plane c, one MMA of N = 4 nb of A_c against the staged
// operand X~_c whose rows d nb + j hold sign(c, d) X_{c xor d}(:, j) -- all four output planes in
// one instruction.  A tcgen05 MMA of M = 128 takes about the same time for every N up to ~100
// (measured on GB300: ~53 cycles for N = 32..96, then ~N / 2), so the fused form issues a quarter
// of the MMAs at four times the width.  `fresh`: the first stage of an accumulation chunk (its
// first MMA overwrites the accumulator).
template <int KIND, int AMODE, bool WIDE = false>
__device__ __forceinline__ void issue_stage(const StageDescs& D, int s, uint32_t abase, int nb, int c_first,
                                            uint32_t idesc_base, uint32_t neg_mask, bool fresh, int fd, int c0) {
  using C = Cfg<KIND, WIDE>;
  constexpr bool X3 = (KIND == K_TF32X3);
  constexpr int KSTEPS = C::BK / C::MMA_K;
  constexpr uint64_t KA = (AMODE == A_MN) ? (uint64_t)((C::MMA_K * C::SW) >> 4) : (uint64_t)((C::MMA_K * C::ESZ) >> 4);
  constexpr uint64_t KB = (uint64_t)((C::MMA_K * C::ESZ) >> 4);
  const uint64_t so = (uint64_t)s * D.sstep;
  if (fd) {
#pragma unroll
    for (int ks = 0; ks < KSTEPS; ++ks) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < c_first) continue;
        const uint64_t ad = D.a[c] + so + ks * KA;
        const uint64_t bd = D.x[c - c0] + so + ks * KB;
        const uint32_t acc = (!fresh || ks > 0 || c > c_first) ? 1u : 0u;
        umma<KIND>(abase, ad, bd, idesc_base, acc);
        if (X3) {
          umma<KIND>(abase, D.alo[c] + so + ks * KA, bd, idesc_base, 1u);
          umma<KIND>(abase, ad, D.xlo[c - c0] + so + ks * KB, idesc_base, 1u);
        }
      }
    }
    return;
  }
#pragma unroll
  for (int ks = 0; ks < KSTEPS; ++ks) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c < c_first) continue;
      const uint64_t ad = D.a[c] + so + ks * KA;
      const uint64_t adlo = D.alo[c] + so + ks * KA;
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const int q = c ^ d;
        const uint64_t bd = D.x[q] + so + ks * KB;
        const uint32_t idesc = idesc_base | (((neg_mask >> (c * 4 + d)) & 1u) << 14);
        const uint32_t dt = abase + (uint32_t)(d * nb);
        const uint32_t acc = (!fresh || ks > 0 || c > c_first) ? 1u : 0u;
        umma<KIND>(dt, ad, bd, idesc, acc);
        if (X3) {
          umma<KIND>(dt, adlo, bd, idesc, 1u);
          umma<KIND>(dt, ad, D.xlo[q] + so + ks * KB, idesc, 1u);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// A contiguous piece of one output tile's reduction: stages [it0, it1).  A tile reduced in
// nseg > 1 pieces (stream-K) has them from CTAs c0 .. c0 + nseg - 1 of its group; piece o writes
// its partial to slot 2 ((c0 + o) cs + coff) + (o == 0 ? b0 : 0) (b0 = 1 when the tile starts
// inside CTA c0's range, as that CTA's second piece), and the last piece to arrive adds the
// partials in slot order.  A group is every CTA (cs = 1, coff = 0), or, with column-block groups,
// the CTAs coff, coff + cs, coff + 2 cs, ... of one column block (cs = the number of blocks).
struct Seg {
  int it0, it1, slot, nseg, c0, b0;
  int more;   // another piece follows in this CTA: keep the right to allocate TMEM
  int cs = 1, coff = 0;
};

// One output tile (column block cb, row tile mt) over the reduction piece sg.
template <int KIND, int AMODE, bool WIDE = false>
__device__ __forceinline__ void sketch_tile(const TcParams& p, const int cb, const int mt, const Seg sg) {
  using C = Cfg<KIND, WIDE>;
  const TcScalars pv = tc_scalars(p);
  constexpr bool X3 = (KIND == K_TF32X3);
  constexpr bool MN = (AMODE == A_MN);
  constexpr bool TR = (AMODE == A_T);
  // worker warps touch every A stage: the 3xTF32 split, the transpose, or (RN) the rounding
  const bool RN = (KIND == K_TF32) && pv.rn != 0;
  const bool WORKERS = X3 || TR || RN;
  constexpr int A_BYTES = TBM * C::SW;                 // one plane of the A tile (== raw tile bytes)
  constexpr int KSTEPS = C::BK / C::MMA_K;
  constexpr int ATOM_MN = C::SW / C::ESZ;              // MN-major: elements per atom row
  constexpr int NATOM = TBM / ATOM_MN;
  constexpr int CH = C::SW / 16;                       // 16-byte chunks per K-major row
  const int STAGES = pv.stages;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nb = pv.nb;
  const bool FD = pv.fd != 0;
  const int X_BYTES = (FD ? 4 * nb : nb) * C::SW;       // one X tile: nb rows, or 4 nb fused rows
  // A sets [raw][hi][lo] of APL planes each: plane c at slot c - (4 - APL) (APL = 3 for a pure
  // quaternion A, whose plane 0 is absent)
  const int APL = pv.apl, C0 = 4 - APL;
  const int A_SET = APL * A_BYTES * (X3 ? 2 : 1);   // [hi][lo]; a transposed A lands raw in [hi]
  const int NXP = FD ? APL : 4;                          // X tiles per set (per input plane when fused)
  const int stage_bytes = A_SET + NXP * X_BYTES * (X3 ? 2 : 1);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + MAX_STAGES;
  uint64_t* ready = bars + 2 * MAX_STAGES;
  uint64_t* tmem_full = bars + 3 * MAX_STAGES;        // [2] a chunk accumulator is complete
  uint64_t* tmem_empty = bars + 3 * MAX_STAGES + 2;   // [2] a chunk accumulator has been drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * MAX_STAGES + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* last_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);
  // Accumulation chunks: the tensor cores' FP32 accumulation does not round to nearest, and on
  // data of one sign its error grows with the number of MMAs added into one accumulator (~1 ulp
  // each).  With pv.flush > 0 the piece is reduced in chunks of pv.flush stages, each started from
  // zero in TMEM, and the epilogue adds the chunks in FP32 with round-to-nearest: into a running
  // sum kept in TMEM (pv.ttotal; the MMAs wait while a chunk is read out), or into the output in
  // global memory (the MMAs fill the other of two chunk buffers meanwhile).
  const int F = pv.flush > 0 ? pv.flush : (1 << 30);
  const int NBUF = pv.nbuf;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t m0 = (int64_t)mt * TBM;
  const int j0 = cb * nb;
  const int it0 = sg.it0;
  const int it1 = sg.it1;
  const int nit = it1 - it0;

  const int HI_OFF = 0;
  auto raw_plane = [&](int s, int c) { return smem + s * stage_bytes + (c - C0) * A_BYTES; };   // = a_plane
  auto a_plane = [&](int s, int c) { return smem + s * stage_bytes + HI_OFF + (c - C0) * A_BYTES; };
  auto alo_plane = [&](int s, int c) { return smem + s * stage_bytes + HI_OFF + (APL + c - C0) * A_BYTES; };
  auto x_plane = [&](int s, int q) { return smem + s * stage_bytes + A_SET + q * X_BYTES; };
  auto xlo_plane = [&](int s, int q) { return smem + s * stage_bytes + A_SET + (NXP + q) * X_BYTES; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < MAX_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&ready[s], 64);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tmem_full[b], 1);
      mbar_init(&tmem_empty[b], 128);
    }
    *abort_flag = 0;
    *last_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(pv.tmem_cols)
                 : "memory");
    if (!sg.more) asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      const uint32_t tx = (uint32_t)((4 - pv.c_first) * A_BYTES + (FD ? 4 - pv.c_first : 4) * X_BYTES * (X3 ? 2 : 1));
      // One column block: every A stage is read once, while the staged thin operand is read by
      // every row tile, so A is loaded evict-first and the operand evict-last (it then stays in
      // L2 while A streams through).  Several blocks share A stages through L2 (column-block
      // groups), so their loads keep the default priority.
      const bool hint = (pv.ncb == 1);
      const uint64_t pol_a = l2_evict_first_policy(), pol_x = l2_evict_last_policy();
      int issued = 0;
      for (int i = 0; i < nit; ++i) {
        const int s = i % STAGES;
        const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, pv.err)) break;
        mbar_expect_tx(&full[s], tx);
        const int k0 = (it0 + i) * C::BK;
        for (int c = pv.c_first; c < 4; ++c) {
          if (MN) {
#pragma unroll
            for (int a = 0; a < NATOM; ++a)
              tma_load_2d(smem_u32(a_plane(s, c) + a * C::BK * C::SW), &p.tmA[c], (int)m0 + a * ATOM_MN, k0, &full[s]);
          } else if (TR) {   // [BK][128] unswizzled
            if (hint) tma_load_2d_hint(smem_u32(raw_plane(s, c)), &p.tmA[c], (int)m0, k0, &full[s], pol_a);
            else tma_load_2d(smem_u32(raw_plane(s, c)), &p.tmA[c], (int)m0, k0, &full[s]);
          } else {
            if (hint) tma_load_2d_hint(smem_u32(a_plane(s, c)), &p.tmA[c], k0, (int)m0, &full[s], pol_a);
            else tma_load_2d(smem_u32(a_plane(s, c)), &p.tmA[c], k0, (int)m0, &full[s]);
          }
        }
        if (FD) {   // X~_c, rows [cb 4 nb, (cb + 1) 4 nb)
          for (int c = pv.c_first; c < 4; ++c) {
            if (hint) tma_load_2d_hint(smem_u32(x_plane(s, c - C0)), &p.tmX[c], k0, 4 * j0, &full[s], pol_x);
            else tma_load_2d(smem_u32(x_plane(s, c - C0)), &p.tmX[c], k0, 4 * j0, &full[s]);
            if (X3) tma_load_2d(smem_u32(xlo_plane(s, c - C0)), &p.tmXlo[c], k0, 4 * j0, &full[s]);
          }
        } else {
          for (int q = 0; q < 4; ++q) {
            tma_load_2d(smem_u32(x_plane(s, q)), &p.tmX[q], k0, j0, &full[s]);
            if (X3) tma_load_2d(smem_u32(xlo_plane(s, q)), &p.tmXlo[q], k0, j0, &full[s]);
          }
        }
        ++issued;
      }
      // drain: every issued stage must have landed before the CTA may exit
      for (int i = max(0, issued - STAGES); i < issued; ++i) {
        const int s = i % STAGES;
        const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
        const uint64_t t0 = now_ns();
        while (!mbar_try_wait(&full[s], ph) && now_ns() - t0 < WAIT_NS) __nanosleep(64);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      int chunk = 0;
      const StageDescs D = make_stage_descs<KIND, AMODE, WIDE>(smem_u32(smem), stage_bytes, HI_OFF - C0 * A_BYTES,
                                                               A_BYTES, A_SET, X_BYTES, APL, NXP);
      for (int i = 0; i < nit && ok; ++i) {
        const int ic = i % F;                      // stage within the accumulation chunk
        if (i > 0 && ic == 0) {                    // chunk boundary: hand the finished chunk over
          umma_commit(&tmem_full[chunk % NBUF]);
          ++chunk;
          if (chunk >= NBUF) {                     // its buffer must have been drained first
            ok = mbar_wait(&tmem_empty[chunk % NBUF], (uint32_t)((chunk / NBUF) - 1) & 1u, abort_flag, pv.err);
            if (!ok) break;
            tc_fence_after();
          }
        }
        const uint32_t abase = tmem + (uint32_t)((chunk % NBUF) * 4 * nb);
        const int s = i % STAGES;
        const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
        ok = mbar_wait(WORKERS ? &ready[s] : &full[s], ph, abort_flag, pv.err);
        if (!ok) break;
        tc_fence_after();
        issue_stage<KIND, AMODE, WIDE>(D, s, abase, nb, pv.c_first, pv.idesc_base, pv.neg_mask, ic == 0, pv.fd, C0);
        umma_commit(&empty[s]);   // frees the stage once these MMAs have read it
      }
      umma_commit(&tmem_full[chunk % NBUF]);   // last chunk complete (also fires after an abort)
    }
  } else if (warp < 4) {
    // ---------------- workers: hi/lo split (3xTF32) and/or transpose of A ----------------
    if (WORKERS) {
      const int st = threadIdx.x - 64;   // 0..63
      for (int i = 0; i < nit; ++i) {
        const int s = i % STAGES;
        const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
        if (!mbar_wait(&full[s], ph, abort_flag, pv.err)) break;
        for (int c = pv.c_first; c < 4; ++c) {
          uint4* hi = reinterpret_cast<uint4*>(a_plane(s, c));
          uint4* lo = reinterpret_cast<uint4*>(alo_plane(s, c));
          if (TR) {
            // raw[k][r] (k < BK, r < 128) -> row r of the K-major tile, 16-byte chunk cch holding
            // k = 4 cch .. 4 cch + 3, stored at chunk position cch ^ swizzle(r).  In place: the
            // workers read the whole raw plane into registers, meet at a named barrier, then write.
            const uint32_t* raw = reinterpret_cast<const uint32_t*>(raw_plane(s, c));
            constexpr int NPER = TBM * CH / 64;
            uint4 vv[NPER];
#pragma unroll
            for (int q = 0; q < NPER; ++q) {
              const int e = st + 64 * q, r = e % TBM, cch = e / TBM;
              vv[q].x = raw[(4 * cch + 0) * TBM + r];
              vv[q].y = raw[(4 * cch + 1) * TBM + r];
              vv[q].z = raw[(4 * cch + 2) * TBM + r];
              vv[q].w = raw[(4 * cch + 3) * TBM + r];
            }
            asm volatile("bar.sync 2, 64;" ::: "memory");
#pragma unroll
            for (int q = 0; q < NPER; ++q) {
              const int e = st + 64 * q, r = e % TBM, cch = e / TBM;
              const int sw = (CH == 2) ? ((r >> 2) & 1) : (CH == 4) ? ((r >> 1) & 3) : (r & 7);
              const uint4 v = vv[q];
              const int o = r * CH + (cch ^ sw);
              if (X3) {
                uint4 h, rr;
                h.x = v.x & 0xFFFFE000u; h.y = v.y & 0xFFFFE000u; h.z = v.z & 0xFFFFE000u; h.w = v.w & 0xFFFFE000u;
                rr.x = __float_as_uint(__uint_as_float(v.x) - __uint_as_float(h.x));
                rr.y = __float_as_uint(__uint_as_float(v.y) - __uint_as_float(h.y));
                rr.z = __float_as_uint(__uint_as_float(v.z) - __uint_as_float(h.z));
                rr.w = __float_as_uint(__uint_as_float(v.w) - __uint_as_float(h.w));
                hi[o] = h;
                lo[o] = rr;
              } else {
                hi[o] = RN ? tf32_rna4(v) : v;
              }
            }
          } else if (!X3) {   // RN: round the K-major tile in place
            for (int e = st; e < A_BYTES / 16; e += 64) hi[e] = tf32_rna4(hi[e]);
          } else {
            for (int e = st; e < A_BYTES / 16; e += 64) {
              uint4 v = hi[e], h, r;
              h.x = v.x & 0xFFFFE000u; h.y = v.y & 0xFFFFE000u; h.z = v.z & 0xFFFFE000u; h.w = v.w & 0xFFFFE000u;
              r.x = __float_as_uint(__uint_as_float(v.x) - __uint_as_float(h.x));
              r.y = __float_as_uint(__uint_as_float(v.y) - __uint_as_float(h.y));
              r.z = __float_as_uint(__uint_as_float(v.z) - __uint_as_float(h.z));
              r.w = __float_as_uint(__uint_as_float(v.w) - __uint_as_float(h.w));
              hi[e] = h;
              lo[e] = r;
            }
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&ready[s]);
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int row = q * 32 + lane;
    const int64_t grow = m0 + row;
    const int tile = mt * pv.ncb + cb;
    const size_t tile_elems = (size_t)4 * TBM * nb;
    const int nchunks = (nit > 0) ? (nit + F - 1) / F : 1;
    bool ok = true;
    for (int ch = 0; ch < nchunks && ok; ++ch) {
      const int b = ch % NBUF;
      ok = mbar_wait(&tmem_full[b], (uint32_t)(ch / NBUF) & 1u, abort_flag, pv.err) && !*abort_flag;
      tc_fence_after();
      if (!ok || nit == 0) break;
      const bool first = (ch == 0);
      const bool last = (ch == nchunks - 1);
      const uint32_t abase = tmem + (uint32_t)(b * 4 * nb);
      const uint32_t tbase = tmem + (uint32_t)(4 * nb);   // running sum (pv.ttotal)
      const bool to_total = pv.ttotal && !last;             // this chunk only updates the TMEM sum
      const bool add_total = pv.ttotal && !first;           // the TMEM sum enters this chunk's values
      for (int d = 0; d < 4; ++d) {
        // the output plane d of this tile: Y itself (a whole tile) or this piece's partial slot
        float* dst;
        int64_t stride;
        bool valid_row;
        if (sg.nseg == 1) {
          dst = pv.y(d) + grow;
          stride = pv.ldy;
          valid_row = grow < pv.M;
        } else {
          dst = pv.part + (size_t)sg.slot * tile_elems + (size_t)d * TBM * nb + row;
          stride = TBM;
          valid_row = true;
        }
        for (int cc = 0; cc < nb; cc += 32) {
          // two TMEM loads in flight per wait (nb is a multiple of 16)
          uint32_t r0[16], r1[16], s0[16], s1[16];
          const uint32_t lane_off = ((uint32_t)(q * 32) << 16) + (uint32_t)(d * nb + cc);
          tmem_ld16_issue(abase + lane_off, r0);
          if (cc + 16 < nb) tmem_ld16_issue(abase + lane_off + 16, r1);
          if (add_total) {
            tmem_ld16_issue(tbase + lane_off, s0);
            if (cc + 16 < nb) tmem_ld16_issue(tbase + lane_off + 16, s1);
          }
          tmem_wait_ld();
          if (add_total) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              r0[jj] = __float_as_uint(__uint_as_float(s0[jj]) + __uint_as_float(r0[jj]));
              r1[jj] = __float_as_uint(__uint_as_float(s1[jj]) + __uint_as_float(r1[jj]));
            }
          }
          if (to_total) {
            tmem_st16(tbase + lane_off, r0);
            if (cc + 16 < nb) tmem_st16(tbase + lane_off + 16, r1);
            continue;
          }
          if (!valid_row) continue;
          const bool accumulate = !first && !pv.ttotal;     // global running sum
          float old[32];
          if (accumulate) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const bool in = (cc + jj < nb) && (sg.nseg > 1 || j0 + cc + jj < pv.l);
              old[jj] = in ? dst[(int64_t)(cc + jj) * stride + (sg.nseg == 1 ? (int64_t)j0 * stride : 0)] : 0.f;
            }
          }
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const bool in = (cc + jj < nb) && (sg.nseg > 1 || j0 + cc + jj < pv.l);
            const float v = __uint_as_float(jj < 16 ? r0[jj] : r1[jj - 16]);
            if (in) dst[(int64_t)(cc + jj) * stride + (sg.nseg == 1 ? (int64_t)j0 * stride : 0)] = accumulate ? old[jj] + v : v;
          }
        }
      }
      if (to_total) tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&tmem_empty[b]);   // this chunk's accumulator may be overwritten
    }
    if (sg.nseg > 1) {
      __threadfence();
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (threadIdx.x == 128) {
        const unsigned old = atomicAdd(&pv.counters[tile], 1u);
        *last_flag = (old == (unsigned)(sg.nseg - 1)) ? 1 : 0;
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (*last_flag) {
        __threadfence();
        if (grow < pv.M) {
          for (int d = 0; d < 4; ++d)
            for (int jc0 = 0; jc0 < nb; jc0 += 16) {
              float acc[16];
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) acc[jj] = 0.f;
              for (int o = 0; o < sg.nseg; ++o) {
                const int slot = 2 * ((sg.c0 + o) * sg.cs + sg.coff) + (o == 0 ? sg.b0 : 0);
                const float* P = pv.part + (size_t)slot * tile_elems + (size_t)d * TBM * nb + (size_t)jc0 * TBM + row;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) acc[jj] += __ldcg(P + (size_t)jj * TBM);   // 16 loads in flight
              }
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const int j = j0 + jc0 + jj;
                if (jc0 + jj < nb && j < pv.l) pv.y(d)[grow + (int64_t)j * pv.ldy] = acc[jj];
              }
            }
        }
        if (threadIdx.x == 128) pv.counters[tile] = 0u;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(pv.tmem_cols) : "memory");
  }
}

// One CTA per output tile, the whole reduction.
template <int KIND, int AMODE, bool WIDE>
__global__ void __launch_bounds__(TC_THREADS, 1) sketch_tc_kernel(const __grid_constant__ TcParams p) {
  sketch_tile<KIND, AMODE, WIDE>(p, blockIdx.x, blockIdx.y, Seg{0, p.kiters, 0, 1, 0, 0, 0});
}

// Stream-K: the reduction stages of all tiles, taken in tile order, are cut into gridDim.x equal
// ranges, one per CTA.  A range may start inside one tile (its tail piece), run through whole
// tiles, and end inside another (its head piece); each piece is reduced as in sketch_tile, a
// whole tile writes its output directly, and the pieces of a split tile are added by the last one
// to finish.  A CTA writes at most two partial tiles: slot 2c for its tail piece, slot 2c + 1 for a
// head piece that is not its first piece.
// Column-block groups (p.cgroup, gridDim.x a multiple of ncb): CTA c works on column block
// c mod ncb only, and the CTAs of each block split that block's row tiles' stages the same way,
// so CTAs c, c + 1, ..., c + ncb - 1 read the same A stages at about the same time: A comes from
// DRAM once and from L2 for the other blocks (with one list over all blocks, the CTAs reading a
// given A stage for different blocks are a tile's length apart in time and A is re-read from
// DRAM once per block).
template <int KIND, int AMODE, bool WIDE>
__global__ void __launch_bounds__(TC_THREADS, 1) sketch_tc_streamk_kernel(const __grid_constant__ TcParams p) {
  const int NG = (p.cgroup && p.ncb > 1) ? p.ncb : 1;             // CTAs per group step
  const int cbg = (int)(blockIdx.x % NG);                         // this CTA's block (groups)
  const int64_t K = p.kiters, W = (int64_t)p.mtiles * (p.ncb / NG) * K, G = gridDim.x / NG, c = blockIdx.x / NG;
  auto start = [&](int64_t cc) { return cc * W / G; };
  // the CTA whose range holds stage x: the largest cc with start(cc) <= x
  auto owner = [&](int64_t x) { return ((x + 1) * G + W - 1) / W - 1; };
  int64_t pos = start(c);
  const int64_t end = start(c + 1);
  bool first = true;
  while (pos < end) {
    const int64_t t = pos / K;
    const int it0 = (int)(pos - t * K);
    const int it1 = (int)min(K, (int64_t)it0 + (end - pos));
    const int64_t c0 = owner(t * K), c1 = owner((t + 1) * K - 1);
    const int b0 = (start(c0) < t * K) ? 1 : 0;
    const int more = (pos + (it1 - it0) < end) ? 1 : 0;
    const Seg sg{it0, it1, (int)(2 * (c * NG + cbg) + (c == c0 ? b0 : 0)), (int)(c1 - c0 + 1), (int)c0, b0, more,
                 NG, cbg};
    if (!first) __syncthreads();
    if (NG > 1) sketch_tile<KIND, AMODE, WIDE>(p, cbg, (int)t, sg);
    else sketch_tile<KIND, AMODE, WIDE>(p, (int)(t % p.ncb), (int)(t / p.ncb), sg);
    first = false;
    pos += it1 - it0;
  }
}

// Grouped launch over many problems: CTA b computes the tile items[b] = (problem, row tile,
// column block) with that problem's parameters (tensor maps in global memory, 64-byte aligned).
template <int KIND, int AMODE>
__global__ void __launch_bounds__(TC_THREADS, 1) sketch_tc_grouped_kernel(const TcParams* __restrict__ probs,
                                                                          const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const TcParams& p = probs[it.x];
  if (threadIdx.x == 0) {   // the TMA-issuing thread: tensor maps written before the launch
    for (int c = p.c_first; c < 4; ++c)
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&p.tmA[c]) : "memory");
    for (int q = 0; q < 4; ++q) {
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&p.tmX[q]) : "memory");
      if (KIND == K_TF32X3)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&p.tmXlo[q]) : "memory");
    }
  }
  sketch_tile<KIND, AMODE>(p, it.z, it.y, Seg{0, p.kiters, 0, 1, 0, 0, 0});
}

// Persistent grouped form: gridDim.x CTAs (one per SM) walk the item list, CTA b taking items
// b, b + gridDim.x, ...  The TMA ring, the worker and MMA stage counters run on across items, and
// the accumulators alternate between the two ends of the CTA's 512 TMEM columns: item t (4 nb_t
// columns) sits at column 0 when t is even and ends at column 512 when t is odd, so the epilogue
// drains item t while the MMA warp already accumulates item t + 1 (and the producer streams A for
// the next ones) unless the two items' columns overlap (nb_t + nb_t+1 > 128); only then does the
// MMA warp wait for item t's epilogue.  Shared-memory stages are laid out for the widest column
// block (nb_max); every problem's tiles use its own nb <= nb_max.
template <int KIND, int AMODE, bool WIDE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    sketch_tc_persistent_kernel(const TcParams* __restrict__ probs, const int4* __restrict__ items, int nitems,
                                int nb_max, int stages, int apl, int fd, uint32_t tmem_cols, int* err) {
  using C = Cfg<KIND, WIDE>;
  constexpr bool X3 = (KIND == K_TF32X3);
  constexpr bool MN = (AMODE == A_MN);
  constexpr bool TR = (AMODE == A_T);
  constexpr bool WORKERS = X3 || TR;
  constexpr int A_BYTES = TBM * C::SW;
  constexpr int KSTEPS = C::BK / C::MMA_K;
  constexpr int ATOM_MN = C::SW / C::ESZ;
  constexpr int NATOM = TBM / ATOM_MN;
  constexpr int CH = C::SW / 16;
  const int STAGES = stages;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int X_BYTES = (fd ? 4 * nb_max : nb_max) * C::SW;   // one X tile (4 nb_max fused rows when fd)
  // apl A planes per set: 3 when every problem is pure quaternion (plane 0 absent), else 4; plane
  // c is stored at slot c - (4 - apl)
  const int c0 = 4 - apl;
  const int A_SET = apl * A_BYTES * (X3 ? 2 : 1);   // [hi][lo]; a transposed A lands raw in [hi]
  const int NXP = fd ? apl : 4;
  const int stage_bytes = A_SET + NXP * X_BYTES * (X3 ? 2 : 1);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + PMAX_STAGES;
  uint64_t* ready = bars + 2 * PMAX_STAGES;
  uint64_t* acc_full = bars + 3 * PMAX_STAGES;        // [2]
  uint64_t* acc_empty = bars + 3 * PMAX_STAGES + 2;   // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * PMAX_STAGES + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int my_items = (nitems - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int HI_OFF = 0;
  auto raw_plane = [&](int s, int c) { return smem + s * stage_bytes + (c - c0) * A_BYTES; };   // = a_plane
  auto a_plane = [&](int s, int c) { return smem + s * stage_bytes + HI_OFF + (c - c0) * A_BYTES; };
  auto alo_plane = [&](int s, int c) { return smem + s * stage_bytes + HI_OFF + (apl + c - c0) * A_BYTES; };
  auto x_plane = [&](int s, int q) { return smem + s * stage_bytes + A_SET + q * X_BYTES; };
  auto xlo_plane = [&](int s, int q) { return smem + s * stage_bytes + A_SET + (NXP + q) * X_BYTES; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < PMAX_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&ready[s], 64);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 128);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int t = 0; t < my_items && ok; ++t) {
        const int4 it = items[blockIdx.x + t * gridDim.x];
        const TcParams& p = probs[it.x];
        const TcScalars pv = tc_scalars(p);
        for (int c = pv.c_first; c < 4; ++c)
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&p.tmA[c]) : "memory");
        for (int q = 0; q < 4; ++q) {
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&p.tmX[q]) : "memory");
          if (X3) asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&p.tmXlo[q]) : "memory");
        }
        const int64_t m0 = (int64_t)it.y * TBM;
        const int j0 = it.z * pv.nb;
        const uint32_t tx = (uint32_t)((4 - pv.c_first) * A_BYTES +
                                       (fd ? (4 - pv.c_first) * 4 * pv.nb : 4 * pv.nb) * C::SW * (X3 ? 2 : 1));
        for (int i = 0; i < pv.kiters; ++i, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, err)) { ok = false; break; }
          mbar_expect_tx(&full[s], tx);
          const int k0 = i * C::BK;
          for (int c = pv.c_first; c < 4; ++c) {
            if (MN) {
#pragma unroll
              for (int a = 0; a < NATOM; ++a)
                tma_load_2d(smem_u32(a_plane(s, c) + a * C::BK * C::SW), &p.tmA[c], (int)m0 + a * ATOM_MN, k0, &full[s]);
            } else if (TR) {
              tma_load_2d(smem_u32(raw_plane(s, c)), &p.tmA[c], (int)m0, k0, &full[s]);
            } else {
              tma_load_2d(smem_u32(a_plane(s, c)), &p.tmA[c], k0, (int)m0, &full[s]);
            }
          }
          if (fd) {   // X~_c, rows [cb 4 nb, (cb + 1) 4 nb)
            for (int c = pv.c_first; c < 4; ++c) {
              tma_load_2d(smem_u32(x_plane(s, c - c0)), &p.tmX[c], k0, 4 * j0, &full[s]);
              if (X3) tma_load_2d(smem_u32(xlo_plane(s, c - c0)), &p.tmXlo[c], k0, 4 * j0, &full[s]);
            }
          } else {
            for (int q = 0; q < 4; ++q) {
              tma_load_2d(smem_u32(x_plane(s, q)), &p.tmX[q], k0, j0, &full[s]);
              if (X3) tma_load_2d(smem_u32(xlo_plane(s, q)), &p.tmXlo[q], k0, j0, &full[s]);
            }
          }
        }
      }
      // drain: every issued stage must have landed before the CTA may exit
      for (int i = max(0, g - STAGES); i < g; ++i) {
        const int s = i % STAGES;
        const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
        const uint64_t t0 = now_ns();
        while (!mbar_try_wait(&full[s], ph) && now_ns() - t0 < WAIT_NS) __nanosleep(64);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      const StageDescs D = make_stage_descs<KIND, AMODE, WIDE>(smem_u32(smem), stage_bytes, HI_OFF - c0 * A_BYTES,
                                                               A_BYTES, A_SET, X_BYTES, apl, NXP);
      int prev_nb = 0;
      for (int t = 0; t < my_items && ok; ++t) {
        const int4 it = items[blockIdx.x + t * gridDim.x];
        const TcParams& p = probs[it.x];
        const TcScalars pv = tc_scalars(p);
        const int a = t & 1;
        if (t >= 2) {   // item t - 2 (same end of TMEM) drained
          ok = mbar_wait(&acc_empty[a], (uint32_t)((t >> 1) - 1) & 1u, abort_flag, err);
          if (!ok) break;
        }
        if (t >= 1 && 4 * (pv.nb + prev_nb) > (int)tmem_cols) {   // overlaps item t - 1: wait for its drain
          ok = mbar_wait(&acc_empty[a ^ 1], (uint32_t)((t - 1) >> 1) & 1u, abort_flag, err);
          if (!ok) break;
        }
        if (t >= 1) tc_fence_after();
        prev_nb = pv.nb;
        const uint32_t acc_base = tmem + (a ? tmem_cols - (uint32_t)(4 * pv.nb) : 0u);
        for (int i = 0; i < pv.kiters; ++i, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          ok = mbar_wait(WORKERS ? &ready[s] : &full[s], ph, abort_flag, err);
          if (!ok) break;
          tc_fence_after();
          issue_stage<KIND, AMODE, WIDE>(D, s, acc_base, pv.nb, pv.c_first, pv.idesc_base, pv.neg_mask, i == 0, fd, c0);
          umma_commit(&empty[s]);
        }
        umma_commit(&acc_full[a]);   // accumulator of item t complete (also after an abort)
      }
    }
  } else if (warp < 4) {
    // ---------------- workers: hi/lo split (3xTF32) and/or transpose of A ----------------
    if (WORKERS) {
      const int st = threadIdx.x - 64;
      int g = 0;
      bool ok = true;
      for (int t = 0; t < my_items && ok; ++t) {
        const int4 it = items[blockIdx.x + t * gridDim.x];
        const TcParams& p = probs[it.x];
        const TcScalars pv = tc_scalars(p);
        for (int i = 0; i < pv.kiters; ++i, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          if (!mbar_wait(&full[s], ph, abort_flag, err)) { ok = false; break; }
          for (int c = pv.c_first; c < 4; ++c) {
            uint4* hi = reinterpret_cast<uint4*>(a_plane(s, c));
            uint4* lo = reinterpret_cast<uint4*>(alo_plane(s, c));
            if (TR) {   // in place, as in sketch_tile
              const uint32_t* raw = reinterpret_cast<const uint32_t*>(raw_plane(s, c));
              constexpr int NPER = TBM * CH / 64;
              uint4 vv[NPER];
#pragma unroll
              for (int q = 0; q < NPER; ++q) {
                const int e = st + 64 * q, r = e % TBM, cch = e / TBM;
                vv[q].x = raw[(4 * cch + 0) * TBM + r];
                vv[q].y = raw[(4 * cch + 1) * TBM + r];
                vv[q].z = raw[(4 * cch + 2) * TBM + r];
                vv[q].w = raw[(4 * cch + 3) * TBM + r];
              }
              asm volatile("bar.sync 2, 64;" ::: "memory");
#pragma unroll
              for (int q = 0; q < NPER; ++q) {
                const int e = st + 64 * q, r = e % TBM, cch = e / TBM;
                const int sw = (CH == 2) ? ((r >> 2) & 1) : (CH == 4) ? ((r >> 1) & 3) : (r & 7);
                const uint4 v = vv[q];
                const int o = r * CH + (cch ^ sw);
                if (X3) {
                  uint4 h, rr;
                  h.x = v.x & 0xFFFFE000u; h.y = v.y & 0xFFFFE000u; h.z = v.z & 0xFFFFE000u; h.w = v.w & 0xFFFFE000u;
                  rr.x = __float_as_uint(__uint_as_float(v.x) - __uint_as_float(h.x));
                  rr.y = __float_as_uint(__uint_as_float(v.y) - __uint_as_float(h.y));
                  rr.z = __float_as_uint(__uint_as_float(v.z) - __uint_as_float(h.z));
                  rr.w = __float_as_uint(__uint_as_float(v.w) - __uint_as_float(h.w));
                  hi[o] = h;
                  lo[o] = rr;
                } else {
                  hi[o] = v;
                }
              }
            } else {
              for (int e = st; e < A_BYTES / 16; e += 64) {
                uint4 v = hi[e], h, r;
                h.x = v.x & 0xFFFFE000u; h.y = v.y & 0xFFFFE000u; h.z = v.z & 0xFFFFE000u; h.w = v.w & 0xFFFFE000u;
                r.x = __float_as_uint(__uint_as_float(v.x) - __uint_as_float(h.x));
                r.y = __float_as_uint(__uint_as_float(v.y) - __uint_as_float(h.y));
                r.z = __float_as_uint(__uint_as_float(v.z) - __uint_as_float(h.z));
                r.w = __float_as_uint(__uint_as_float(v.w) - __uint_as_float(h.w));
                hi[e] = h;
                lo[e] = r;
              }
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(&ready[s]);
        }
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int q = warp & 3;
    const int row = q * 32 + lane;
    for (int t = 0; t < my_items; ++t) {
      const int4 it = items[blockIdx.x + t * gridDim.x];
      const TcParams& p = probs[it.x];
      const TcScalars pv = tc_scalars(p);
      const int a = t & 1;
      const bool ok = mbar_wait(&acc_full[a], (uint32_t)(t >> 1) & 1u, abort_flag, err) && !*abort_flag;
      tc_fence_after();
      if (!ok) break;
      const int64_t grow = (int64_t)it.y * TBM + row;
      const int j0 = it.z * pv.nb;
      const uint32_t acc_base = tmem + (a ? tmem_cols - (uint32_t)(4 * pv.nb) : 0u);
      for (int d = 0; d < 4; ++d) {
        for (int cc = 0; cc < pv.nb; cc += 32) {
          uint32_t r0[16], r1[16];
          const uint32_t ta = acc_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(d * pv.nb + cc);
          tmem_ld16_issue(ta, r0);
          if (cc + 16 < pv.nb) tmem_ld16_issue(ta + 16, r1);
          tmem_wait_ld();
          if (grow < pv.M) {
            float* yd = pv.y(d) + grow;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int j = j0 + cc + jj;
              if (j < pv.l && cc + jj < pv.nb) yd[(int64_t)j * pv.ldy] = __uint_as_float(jj < 16 ? r0[jj] : r1[jj - 16]);
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&acc_empty[a]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

// Operand staging: the thin operand X (FP32, column-major) into the layout the sketch's TMA reads,
// as rows (one per operand column) of K elements at pitch ldo, converted to the MMA type (BF16,
// TF32, or the 3xTF32 hi / lo pair).  Plain layout: row q cols + j = X_q(:, j).  Fused layout
// (fd): per input plane c >= c0 and column block cb, 4 nb rows, row (c - c0) ncb 4 nb + cb 4 nb
// + d nb + j = sign(c, d) X_{c xor d}(:, cb nb + j) (zero past the last column), so one MMA of
// N = 4 nb forms every output plane (issue_stage).
struct StageArg {
  const float* x[4];
  int64_t ldx, rows, cols, ldo;   // rows: K (the reduction), cols: l
  void* out;
  void* out_lo;
  int fd, nb, ncb, c0;
  uint32_t neg;                   // bit c*4+d: sign(c, d) = -1
  int nrows;                      // staged rows: 4 cols, or (4 - c0) ncb 4 nb
  int rn;                         // TF32: round to nearest TF32 (else the FP32 bits, truncated by the MMA)
};

template <int MODE>
__device__ __forceinline__ void stage_row(const StageArg& a, int r, int64_t k0, int64_t k1, int t, int nt) {
  int q, j;
  float sg = 1.f;
  bool valid = true;
  if (!a.fd) {
    q = r / (int)a.cols;
    j = r % (int)a.cols;
  } else {
    const int per = a.ncb * 4 * a.nb;
    const int c = a.c0 + r / per, rr = r % per;
    const int d = (rr % (4 * a.nb)) / a.nb;
    j = (rr / (4 * a.nb)) * a.nb + rr % a.nb;
    q = c ^ d;
    sg = ((a.neg >> (c * 4 + d)) & 1u) ? -1.f : 1.f;
    valid = j < a.cols;
  }
  const float* src = a.x[q] + (int64_t)(valid ? j : 0) * a.ldx;
  const size_t o0 = (size_t)r * a.ldo;
  for (int64_t i = k0 + t; i < k1; i += nt) {
    const float v = valid ? sg * src[i] : 0.f;
    if (MODE == K_BF16) {
      static_cast<__nv_bfloat16*>(a.out)[o0 + i] = __float2bfloat16_rn(v);
    } else if (MODE == K_TF32) {
      static_cast<float*>(a.out)[o0 + i] = a.rn ? __uint_as_float(tf32_rna(__float_as_uint(v))) : v;
    } else {
      const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
      static_cast<float*>(a.out)[o0 + i] = h;
      static_cast<float*>(a.out_lo)[o0 + i] = v - h;
    }
  }
}

// Grouped: problem blockIdx.y; a warp per staged row, the rows over the grid's x blocks.
template <int MODE>
__global__ void __launch_bounds__(256) stage_x_grouped_kernel(const StageArg* __restrict__ args) {
  const StageArg a = args[blockIdx.y];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int r = blockIdx.x * 8 + warp; r < a.nrows; r += gridDim.x * 8) stage_row<MODE>(a, r, 0, a.rows, lane, 32);
}

// One problem: grid (reduction chunks of STAGE_ROWS, staged rows).
constexpr int STAGE_ROWS = 2048;
template <int MODE>
__global__ void __launch_bounds__(256) stage_x_kernel(const StageArg a) {
  const int64_t k0 = (int64_t)blockIdx.x * STAGE_ROWS;
  stage_row<MODE>(a, (int)blockIdx.y, k0, min(a.rows, k0 + STAGE_ROWS), threadIdx.x, blockDim.x);
}

// Staged X bytes of one problem (hi set; the 3xTF32 lo set is as large again).
size_t staged_x_bytes(bool fd, int apl, int64_t ldo, int l, int nb, int ncb, size_t esz) {
  return fd ? (size_t)apl * ncb * 4 * nb * ldo * esz : (size_t)4 * l * ldo * esz;
}

uint32_t neg_table(int op) {
  // op N: negative for (c,d) in {(1,0),(2,0),(3,0),(1,2),(2,3),(3,1)}; op H flips every c != 0
  uint32_t neg = 0;
  const int negN[6][2] = {{1, 0}, {2, 0}, {3, 0}, {1, 2}, {2, 3}, {3, 1}};
  for (auto& e : negN) neg |= 1u << (e[0] * 4 + e[1]);
  if (op == QLR_OP_H) neg ^= 0xFFF0u;
  return neg;
}

int kind_of(int compute) {
  return compute == QLR_COMPUTE_BF16 ? K_BF16
         : (compute == QLR_COMPUTE_TF32 || compute == QLR_COMPUTE_TF32_RN) ? K_TF32 : K_TF32X3;
}

struct Plan {
  int kind, amode, sw, bk, esz, nb, ncb, mtiles, kiters, stages, apl;
  bool fd;                       // fused output planes (N = 4 nb per MMA; column blocks <= 64)
  int grid_sk;                   // stream-K CTAs (0: one CTA per output tile)
  int flush, nbuf, ttotal;       // accumulation chunks (stages per chunk, TMEM buffers, TMEM sum)
  bool wide;                     // 128-byte stage rows (Cfg<KIND, true>)
  bool rn;                       // TF32 with operands rounded to nearest and chunked sums
  bool cgroup;                   // stream-K CTAs in column-block groups (grid_sk a multiple of ncb)
  uint32_t tmem_cols;
  size_t smem;
};

// 3xTF32 (the FP32-accurate mode) adds at most this many stages into one TMEM accumulator before
// the epilogue takes the chunk over (a stage adds 3 MMAs per input plane into each output plane):
// the accumulation's rounding error on one-signed data then stays near 32 x 12 MMA additions
// instead of growing with the reduction length (~0.5 ulp per addition was measured on GB300).
// Column blocks are at most 128 wide in this mode.  Up to 64 columns the chunks' running sum
// stays in TMEM beside the chunk accumulator; wider blocks add each finished chunk into the output
// while the MMAs wait (a few percent of a chunk's time), which still beats two narrower blocks:
// measured on GB300 at 4096 x 4096 x 110, one 112-wide block takes 0.38 ms where two 56-wide
// ones took 0.48 ms (each A tile read once, and half as many MMAs of twice the width).
constexpr int X3_FLUSH_STAGES = 32;
constexpr int X3_MAX_NB = 128;
// Rounded TF32 (QLR_COMPUTE_TF32_RN): one product per K step and input plane, so a chunk of this
// many K elements adds about as many MMAs into an accumulator as a 3xTF32 chunk of 32 stages.
constexpr int RN_FLUSH_K = 512;

Plan make_plan(int compute, int op, int64_t M, int64_t K, int l, int num_sms, bool allow_wide = true, int apl = 4,
               bool allow_fd = true) {
  Plan pl{};
  pl.apl = apl;
  pl.kind = kind_of(compute);
  pl.rn = (compute == QLR_COMPUTE_TF32_RN);
  pl.amode = (op == QLR_OP_N) ? A_K : (pl.kind == K_BF16 ? A_MN : A_T);
  pl.esz = pl.kind == K_BF16 ? 2 : 4;
  const int lp = (l + 15) / 16 * 16;
  const int max_nb = (pl.kind == K_TF32X3) ? X3_MAX_NB : 128;
  pl.ncb = (lp + max_nb - 1) / max_nb;
  pl.nb = ((lp + pl.ncb - 1) / pl.ncb + 15) / 16 * 16;
  // fused output planes when one MMA of N = 4 nb fits (nb <= 64): a quarter of the MMAs, but a
  // fused X set (4 - c0) times larger; kept only while the ring still holds 3 stages (with two, the
  // transposed-A form lost more to exposed loads than it gained: 1.16 against 0.87 ms at
  // 20000 x 10000 x 60, TF32 op H)
  const bool x3 = pl.kind == K_TF32X3;
  const bool chunked = x3 || pl.rn;   // accumulation in chunks (FP32-accurate modes)
  const size_t budget = (size_t)227 * 1024 - 1024 - 256;
  const int sw0 = x3 ? 32 : 64;
  const size_t aset = (size_t)apl * TBM * sw0 * (x3 ? 2 : 1);
  pl.fd = allow_fd && pl.nb <= 64 && budget / (aset + (size_t)apl * 4 * pl.nb * sw0 * (x3 ? 2 : 1)) >= 3;
  if (allow_fd && !pl.fd && chunked && pl.ncb >= 2) {
    // 3xTF32 (or rounded TF32) over several column blocks anyway: fused planes in blocks of <= 64
    // (one more read of A, but a quarter of the MMAs and the chunk sums kept in TMEM): 5.27
    // against 6.02 ms at 20000 x 10000 x 180, 3xTF32 op N
    const int ncb = (lp + 63) / 64, nb = ((lp + ncb - 1) / ncb + 15) / 16 * 16;
    if (budget / (aset + (size_t)apl * 4 * nb * sw0 * (x3 ? 2 : 1)) >= 3) {
      pl.ncb = ncb;
      pl.nb = nb;
      pl.fd = true;
    }
  }
  pl.wide = allow_wide && (pl.amode == A_K) && (pl.kind != K_TF32X3) && (pl.nb <= 64);
  if (pl.wide && pl.fd)   // 128-byte rows double the stage: only with 2+ stages
    pl.wide = budget / (2 * (aset + (size_t)apl * 4 * pl.nb * sw0)) >= 2;
  pl.sw = pl.kind == K_TF32X3 ? 32 : (pl.wide ? 128 : 64);
  pl.bk = pl.sw / pl.esz;
  pl.mtiles = (int)((M + TBM - 1) / TBM);
  pl.kiters = (int)((K + pl.bk - 1) / pl.bk);
  // Stream-K over every SM (each CTA at least 8 stages) when the tiles do not fill whole waves:
  // fewer tiles than SMs, or a last wave that would leave SMs idle (e.g. 157 row tiles on 152
  // SMs would take two full tile times).  A CTA's range then holds at most two partial pieces
  // (the tail of one tile and the head of another) around any number of whole tiles.
  const int64_t tiles = (int64_t)pl.mtiles * pl.ncb;
  const int64_t g = std::min<int64_t>(num_sms, tiles * pl.kiters / 8);
  if (g > tiles) pl.grid_sk = (int)g;
  else if (tiles > num_sms && tiles % num_sms != 0 && g == num_sms) pl.grid_sk = num_sms;
  else pl.grid_sk = 0;
  // several column blocks: the stream-K CTAs in groups of one CTA per block (a whole number of
  // groups), so the blocks' CTAs read each A stage together
  if (pl.grid_sk > 0 && pl.ncb > 1 && pl.grid_sk >= 2 * pl.ncb) {
    pl.grid_sk -= pl.grid_sk % pl.ncb;
    pl.cgroup = true;
  }
  pl.flush = (pl.kind == K_TF32X3) ? X3_FLUSH_STAGES : pl.rn ? RN_FLUSH_K / pl.bk : 0;
  // chunk sums in TMEM next to the chunk accumulator when both fit (column blocks <= 64), else in
  // the output with two chunk buffers
  pl.ttotal = (pl.flush > 0 && 8 * pl.nb <= 512) ? 1 : 0;
  pl.nbuf = (pl.flush > 0 && !pl.ttotal && 8 * pl.nb <= 512) ? 2 : 1;
  const int cols = (pl.ttotal ? 2 : pl.nbuf) * 4 * pl.nb;
  pl.tmem_cols = cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
  const size_t stage = (size_t)apl * TBM * pl.sw * (x3 ? 2 : 1) +
                       (size_t)(pl.fd ? apl : 1) * 4 * pl.nb * pl.sw * (x3 ? 2 : 1);
  pl.stages = (int)std::min<size_t>(MAX_STAGES, budget / stage);
  pl.smem = pl.stages * stage + 1024 + 256;
  return pl;
}

template <int KIND, int AMODE, bool WIDE = false>
int launch_kernel(qlr_ctx* ctx, const Plan& pl, const TcParams& prm, int kid) {
  if constexpr (AMODE == A_K && KIND != K_TF32X3 && !WIDE) {
    if (pl.wide) return launch_kernel<KIND, AMODE, true>(ctx, pl, prm, kid);
  }
  auto kern = sketch_tc_kernel<KIND, AMODE, WIDE>;
  QLR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
  KTimer kt(ctx, kid);
  if (pl.grid_sk > 0) {
    auto sk = sketch_tc_streamk_kernel<KIND, AMODE, WIDE>;
    QLR_CUDA_TRY(cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
    sk<<<pl.grid_sk, TC_THREADS, pl.smem, ctx->stream>>>(prm);
  } else {
    kern<<<dim3((unsigned)pl.ncb, (unsigned)pl.mtiles, 1u), TC_THREADS, pl.smem, ctx->stream>>>(prm);
  }
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

namespace qlr_tc {

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

// 2-D tiled map over a (inner x outer) array with row pitch `pitch_bytes`; box (bi x bo).
bool encode_2d(CUtensorMap* tm, const void* base, CUtensorMapDataType dt, uint64_t inner, uint64_t outer,
               uint64_t pitch_bytes, uint32_t bi, uint32_t bo, CUtensorMapSwizzle sw) {
  auto fn = get_encode();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {pitch_bytes};
  cuuint32_t box[2] = {bi, bo};
  cuuint32_t es[2] = {1, 1};
  return fn(tm, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace qlr_tc

namespace qlr {

bool sketch_tc_supported(int op, const qlr_qmat& A, const qlr_qmat& X, int compute) {
  (void)op; (void)X;
  if (compute != QLR_COMPUTE_BF16 && compute != QLR_COMPUTE_TF32 && compute != QLR_COMPUTE_TF32X3 &&
      compute != QLR_COMPUTE_TF32_RN)
    return false;
  const int want = compute == QLR_COMPUTE_BF16 ? QLR_BF16 : QLR_F32;
  if (A.dtype != want || A.layout != QLR_ROW_MAJOR) return false;
  const size_t esz = qlr_dtype_size(A.dtype);
  if ((A.ld * esz) % 16 != 0) return false;
  for (int c = 0; c < 4; ++c)
    if (A.plane[c] && !aligned16(A.plane[c])) return false;
  if (!get_encode()) return false;
  return A.rows < (1LL << 31) && A.cols < (1LL << 31);
}

// ---------------------------------------------------------------------------------------
// Grouped form.
namespace {
struct GDims {
  int64_t M, K;
  int l, nb, ncb, mtiles, kiters;
  int64_t ldo;
};
GDims gdims(int op, const qlr_qmat& A, const qlr_qmat& X, const Plan& base, int ncap) {
  GDims g{};
  g.M = (op == QLR_OP_N) ? A.rows : A.cols;
  g.K = (op == QLR_OP_N) ? A.cols : A.rows;
  g.l = (int)X.cols;
  const int lp = (g.l + 15) / 16 * 16;
  g.ncb = (lp + ncap - 1) / ncap;
  g.nb = ((lp + g.ncb - 1) / g.ncb + 15) / 16 * 16;
  g.mtiles = (int)((g.M + TBM - 1) / TBM);
  g.kiters = (int)((g.K + base.bk - 1) / base.bk);
  g.ldo = (g.K + 7) / 8 * 8;
  return g;
}
size_t align256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

size_t sketch_tc_grouped_bytes(int op, int count, const qlr_qmat* A, const qlr_qmat* X, int compute) {
  const Plan base = make_plan(compute, op, 1, 1, 16, 1, false);
  const size_t xesz = (base.kind == K_BF16) ? 2 : 4;
  size_t b = align256((size_t)count * sizeof(TcParams)) + align256((size_t)count * sizeof(StageArg));
  size_t items = 0;
  for (int i = 0; i < count; ++i) {
    const GDims g = gdims(op, A[i], X[i], base, 64);   // the narrowest column blocks: the most items
    const GDims g2 = gdims(op, A[i], X[i], base, 128);
    items += (size_t)g.mtiles * g.ncb;
    const size_t xb = std::max({staged_x_bytes(false, 4, g.ldo, g.l, g.nb, g.ncb, xesz),
                                staged_x_bytes(true, 4, g.ldo, g.l, g.nb, g.ncb, xesz),
                                staged_x_bytes(true, 4, g2.ldo, g2.l, g2.nb, g2.ncb, xesz)});
    b += align256(xb) * (base.kind == K_TF32X3 ? 2 : 1);
  }
  return b + align256(items * sizeof(int4)) + 4096;
}

int sketch_tc_grouped_plan(qlr_ctx* ctx, int op, int count, const qlr_qmat* A, const qlr_qmat* X, const qlr_qmat* Y,
                           int compute, int variant, char* dev, size_t bytes, GroupedSketch& gs) {
  const int order = variant & 1;
  const bool persistent = (variant >> 1) & 1;
  if (count <= 0) return QLR_EINVAL;
  Plan base = make_plan(compute, op, 1, 1, 16, 1, false);
  // tile shape: 128-byte stage rows (twice the K elements per stage) for the persistent form of
  // a K-major A, and column blocks of at most 128 or 64
  if (persistent && ((variant >> 2) & 1) && base.amode == A_K && base.kind != K_TF32X3) {
    base.sw = 128;
    base.bk = base.sw / base.esz;
  }
  const int ncap = ((variant >> 3) & 1) ? 64 : 128;
  const size_t xesz = (base.kind == K_BF16) ? 2 : 4;
  const bool x3 = base.kind == K_TF32X3;
  std::vector<GDims> dims(count);
  int max_nb = 16;
  for (int i = 0; i < count; ++i) {
    if (!sketch_tc_supported(op, A[i], X[i], compute)) return QLR_EUNSUPPORTED;
    dims[i] = gdims(op, A[i], X[i], base, ncap);
    const GDims& g = dims[i];
    if (g.M <= 0 || g.K <= 0 || g.l <= 0) return QLR_ESHAPE;
    if (X[i].dtype != QLR_F32 || X[i].layout != QLR_COL_MAJOR || X[i].rows != g.K) return QLR_EINVAL;
    if (Y[i].dtype != QLR_F32 || Y[i].layout != QLR_COL_MAJOR || Y[i].rows != g.M || Y[i].cols != g.l) return QLR_ESHAPE;
    max_nb = std::max(max_nb, g.nb);
  }
  // only the A planes some problem has (3 when all are pure quaternion)
  bool all_pure = true;
  for (int i = 0; i < count; ++i) all_pure = all_pure && (A[i].plane[0] == nullptr);
  const int apl = all_pure ? 3 : 4;
  const size_t budget = (size_t)227 * 1024 - 1024 - 256;
  const size_t aset = (size_t)apl * TBM * base.sw * (x3 ? 2 : 1);
  auto xset = [&](bool f) { return (size_t)(f ? apl : 1) * 4 * max_nb * base.sw * (x3 ? 2 : 1); };
  // fused output planes for every problem when N = 4 nb <= 256 and the ring keeps 3 stages; with
  // 128-byte rows that leave fewer than 2 stages, 64-byte rows instead
  bool fd = max_nb <= 64 && budget / (aset + xset(true)) >= 3;
  if (base.sw == 128 && budget / (aset + xset(fd)) < 2) {
    return sketch_tc_grouped_plan(ctx, op, count, A, X, Y, compute, variant & ~4, dev, bytes, gs);
  }
  const size_t stage = aset + xset(fd);
  const int stages = (int)std::min<size_t>(MAX_STAGES, budget / stage);
  if (stages < 2) return QLR_EUNSUPPORTED;
  const size_t pstage = stage;
  const int pstages = stages;
  const int cols = 4 * max_nb;
  const uint32_t tmem_cols = cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;

  // device layout: params | stage args | items | staged X buffers
  char* cur = dev;
  auto take = [&](size_t n) { char* r = cur; cur += align256(n); return r; };
  TcParams* d_probs = reinterpret_cast<TcParams*>(take((size_t)count * sizeof(TcParams)));
  StageArg* d_stage = reinterpret_cast<StageArg*>(take((size_t)count * sizeof(StageArg)));
  size_t nitems = 0;
  for (const auto& g : dims) nitems += (size_t)g.mtiles * g.ncb;
  int4* d_items = reinterpret_cast<int4*>(take(nitems * sizeof(int4)));

  std::vector<TcParams> hp(count);
  std::vector<StageArg> hs(count);
  std::vector<int4> hi;
  hi.reserve(nitems);
  const CUtensorMapDataType dt = (base.kind == K_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const CUtensorMapSwizzle sw = (base.sw == 32) ? CU_TENSOR_MAP_SWIZZLE_32B
                                : (base.sw == 64) ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  const uint32_t neg = neg_table(op);
  const uint32_t fmt = (base.kind == K_BF16) ? 1u : 2u;
  int max_stage_blocks = 1;
  for (int i = 0; i < count; ++i) {
    const GDims& g = dims[i];
    const qlr_qmat& a = A[i];
    TcParams& prm = hp[i];
    memset(&prm, 0, sizeof(prm));
    const size_t xb = staged_x_bytes(fd, apl, g.ldo, g.l, g.nb, g.ncb, xesz);
    char* xs = take(xb);
    char* xlo = x3 ? take(xb) : nullptr;
    if ((size_t)(cur - dev) > bytes) return QLR_ENOMEM;
    prm.c_first = (a.plane[0] == nullptr) ? 1 : 0;
    prm.apl = apl;
    prm.fd = fd ? 1 : 0;
    for (int c = prm.c_first; c < 4; ++c) {
      bool ok;
      if (op == QLR_OP_N)
        ok = encode_2d(&prm.tmA[c], a.plane[c], dt, (uint64_t)a.cols, (uint64_t)a.rows, (uint64_t)a.ld * base.esz,
                       (uint32_t)base.bk, TBM, sw);
      else if (base.amode == A_MN)
        ok = encode_2d(&prm.tmA[c], a.plane[c], dt, (uint64_t)a.cols, (uint64_t)a.rows, (uint64_t)a.ld * base.esz,
                       (uint32_t)(base.sw / base.esz), (uint32_t)base.bk, sw);
      else
        ok = encode_2d(&prm.tmA[c], a.plane[c], dt, (uint64_t)a.cols, (uint64_t)a.rows, (uint64_t)a.ld * base.esz, TBM,
                       (uint32_t)base.bk, CU_TENSOR_MAP_SWIZZLE_NONE);
      if (!ok) return QLR_ECUDA;
    }
    if (fd) {   // X~_c of input plane c >= c0: ncb 4 nb rows, boxes of 4 nb rows
      const int64_t fr = (int64_t)g.ncb * 4 * g.nb;
      for (int c = 4 - apl; c < 4; ++c) {
        const size_t off = (size_t)(c - (4 - apl)) * fr * g.ldo;
        if (!encode_2d(&prm.tmX[c], xs + off * xesz, dt, (uint64_t)g.K, (uint64_t)fr, (uint64_t)g.ldo * xesz,
                       (uint32_t)base.bk, (uint32_t)(4 * g.nb), sw))
          return QLR_ECUDA;
        if (xlo && !encode_2d(&prm.tmXlo[c], xlo + off * 4, dt, (uint64_t)g.K, (uint64_t)fr, (uint64_t)g.ldo * 4,
                              (uint32_t)base.bk, (uint32_t)(4 * g.nb), sw))
          return QLR_ECUDA;
      }
    } else {
      for (int q = 0; q < 4; ++q) {
        if (!encode_2d(&prm.tmX[q], xs + (size_t)q * g.ldo * g.l * xesz, dt, (uint64_t)g.K, (uint64_t)g.l,
                       (uint64_t)g.ldo * xesz, (uint32_t)base.bk, (uint32_t)g.nb, sw))
          return QLR_ECUDA;
        if (xlo && !encode_2d(&prm.tmXlo[q], xlo + (size_t)q * g.ldo * g.l * 4, dt, (uint64_t)g.K, (uint64_t)g.l,
                              (uint64_t)g.ldo * 4, (uint32_t)base.bk, (uint32_t)g.nb, sw))
          return QLR_ECUDA;
      }
    }
    for (int c = 0; c < 4; ++c) prm.y[c] = static_cast<float*>(Y[i].plane[c]);
    prm.ldy = Y[i].ld;
    prm.M = g.M;
    prm.l = g.l;
    prm.nb = g.nb;
    prm.ncb = g.ncb;
    prm.kiters = g.kiters;
    prm.mtiles = g.mtiles;
    prm.neg_mask = neg;
    prm.idesc_base = (1u << 4) | (fmt << 7) | (fmt << 10) | ((base.amode == A_MN ? 1u : 0u) << 15) |
                     ((uint32_t)((fd ? 4 * g.nb : g.nb) >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);
    prm.tmem_cols = tmem_cols;
    prm.stages = stages;
    prm.err = ctx->d_err;
    StageArg& sa = hs[i];
    for (int c = 0; c < 4; ++c) sa.x[c] = static_cast<const float*>(X[i].plane[c]);
    sa.ldx = X[i].ld;
    sa.rows = g.K;
    sa.cols = g.l;
    sa.ldo = g.ldo;
    sa.out = xs;
    sa.out_lo = xlo;
    sa.fd = fd ? 1 : 0;
    sa.nb = g.nb;
    sa.ncb = g.ncb;
    sa.c0 = 4 - apl;
    sa.neg = neg;
    sa.nrows = fd ? apl * g.ncb * 4 * g.nb : 4 * g.l;
    max_stage_blocks = std::max<int>(max_stage_blocks, std::min<int>((sa.nrows + 7) / 8, 64));   // 8 rows per CTA
    for (int mt = 0; mt < g.mtiles; ++mt)
      for (int cb = 0; cb < g.ncb; ++cb) hi.push_back(make_int4(i, mt, cb, 0));
  }
  if (order == 1)
    std::stable_sort(hi.begin(), hi.end(), [&](const int4& a, const int4& b) { return dims[a.x].K > dims[b.x].K; });
  // ordered on the context stream before any launch that reads them (a plain cudaMemcpy from
  // pageable memory may still be in flight when it returns and is not ordered with that stream)
  QLR_CUDA_TRY(cudaMemcpyAsync(d_probs, hp.data(), hp.size() * sizeof(TcParams), cudaMemcpyHostToDevice, ctx->stream));
  QLR_CUDA_TRY(cudaMemcpyAsync(d_stage, hs.data(), hs.size() * sizeof(StageArg), cudaMemcpyHostToDevice, ctx->stream));
  QLR_CUDA_TRY(cudaMemcpyAsync(d_items, hi.data(), hi.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
  QLR_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  gs.kind = base.kind;
  gs.amode = base.amode;
  gs.count = count;
  gs.nitems = (int)hi.size();
  gs.persistent = persistent ? 1 : 0;
  gs.wide = base.sw == 128 ? 1 : 0;
  gs.stage_k = base.bk;
  gs.nb_max = max_nb;
  gs.stages = gs.persistent ? pstages : stages;
  gs.apl = apl;
  gs.fd = fd ? 1 : 0;
  {   // two accumulators of the widest block when they fit in fewer columns, else all 512
    const int pc = 2 * 4 * max_nb;
    gs.tmem_cols = pc <= 32 ? 32 : pc <= 64 ? 64 : pc <= 128 ? 128 : pc <= 256 ? 256 : 512;
  }
  gs.grid = std::min(gs.nitems, ctx->num_sms > 0 ? ctx->num_sms : 148);
  gs.stage_grid_x = max_stage_blocks;
  gs.smem = gs.persistent ? pstages * pstage + 1024 + 256 : stages * stage + 1024 + 256;
  gs.d_probs = d_probs;
  gs.d_items = d_items;
  gs.d_stage = d_stage;
  return QLR_OK;
}

namespace {
template <int KIND, int AMODE>
int launch_grouped(qlr_ctx* ctx, const GroupedSketch& gs) {
  if (gs.persistent) {
    auto pk = sketch_tc_persistent_kernel<KIND, AMODE, false>;
    if constexpr (AMODE == A_K && KIND != K_TF32X3)
      if (gs.wide) pk = sketch_tc_persistent_kernel<KIND, AMODE, true>;
    QLR_CUDA_TRY(cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gs.smem));
    KTimer kt(ctx, QLR_KID_SKETCH_TC);
    pk<<<(unsigned)gs.grid, TC_THREADS, gs.smem, ctx->stream>>>(static_cast<const TcParams*>(gs.d_probs), gs.d_items,
                                                               gs.nitems, gs.nb_max, gs.stages, gs.apl, gs.fd, gs.tmem_cols,
                                                               ctx->d_err);
    qlr_count_launch();
    QLR_CUDA_TRY(cudaGetLastError());
    return QLR_OK;
  }
  auto kern = sketch_tc_grouped_kernel<KIND, AMODE>;
  QLR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gs.smem));
  KTimer kt(ctx, QLR_KID_SKETCH_TC);
  kern<<<(unsigned)gs.nitems, TC_THREADS, gs.smem, ctx->stream>>>(static_cast<const TcParams*>(gs.d_probs), gs.d_items);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}
}  // namespace

int sketch_tc_grouped_run(qlr_ctx* ctx, const GroupedSketch& gs) {
  if (gs.nitems == 0) return QLR_OK;
  {
    KTimer kt(ctx, QLR_KID_MISC);
    const dim3 grid((unsigned)gs.stage_grid_x, (unsigned)gs.count);
    const StageArg* sa = static_cast<const StageArg*>(gs.d_stage);
    if (gs.kind == K_BF16) stage_x_grouped_kernel<K_BF16><<<grid, 256, 0, ctx->stream>>>(sa);
    else if (gs.kind == K_TF32) stage_x_grouped_kernel<K_TF32><<<grid, 256, 0, ctx->stream>>>(sa);
    else stage_x_grouped_kernel<K_TF32X3><<<grid, 256, 0, ctx->stream>>>(sa);
    qlr_count_launch();
    QLR_CUDA_TRY(cudaGetLastError());
  }
  const bool n = (gs.amode == A_K);
  if (gs.kind == K_BF16) return n ? launch_grouped<K_BF16, A_K>(ctx, gs) : launch_grouped<K_BF16, A_MN>(ctx, gs);
  if (gs.kind == K_TF32) return n ? launch_grouped<K_TF32, A_K>(ctx, gs) : launch_grouped<K_TF32, A_T>(ctx, gs);
  return n ? launch_grouped<K_TF32X3, A_K>(ctx, gs) : launch_grouped<K_TF32X3, A_T>(ctx, gs);
}

size_t sketch_tc_ws(int64_t rows_in, int64_t l, int num_sms) {
  const int64_t ldo = (rows_in + 7) / 8 * 8;
  // staged X (hi and lo sets, 4-byte elements): 4 planes of l rows, or per input plane the fused
  // rows (4 nb per column block, at most 4 (l + 64) in all)
  const int64_t rows = std::max<int64_t>(l, 4 * (l + 64));
  return (size_t)2 * 4 * ldo * rows * 4 + (size_t)2 * (num_sms + 8) * 4 * TBM * 128 * 4 + 65536 + 4096;
}

size_t sketch_tc_need(int op, int64_t M, int64_t K, int l, int compute, int num_sms) {
  const Plan pl = make_plan(compute, op, M, K, l, num_sms);   // a full quaternion A: the largest staging
  const int64_t ldo = (K + 7) / 8 * 8;
  const size_t xesz = (pl.kind == K_BF16) ? 2 : 4;
  const size_t xb = staged_x_bytes(pl.fd, 4, ldo, l, pl.nb, pl.ncb, xesz);
  size_t b = align256(xb);
  if (pl.kind == K_TF32X3) b += align256(xb);
  if (pl.grid_sk > 0) b += align256((size_t)2 * pl.grid_sk * 4 * TBM * pl.nb * sizeof(float));
  return b + align256((size_t)pl.mtiles * pl.ncb * sizeof(unsigned));
}

int sketch_tc(qlr_ctx* ctx, int op, const qlr_qmat& A, const qlr_qmat& X, qlr_qmat& Y, int compute, WsArena& ws) {
  if (!sketch_tc_supported(op, A, X, compute)) return QLR_EUNSUPPORTED;
  if (op != QLR_OP_N && op != QLR_OP_H) return QLR_EINVAL;
  const int64_t M = (op == QLR_OP_N) ? A.rows : A.cols;
  const int64_t K = (op == QLR_OP_N) ? A.cols : A.rows;
  const int l = (int)X.cols;
  if (M == 0 || l == 0) return QLR_OK;
  if (K == 0) return zero_qmat(ctx, Y);
  if (X.dtype != QLR_F32 && !(compute == QLR_COMPUTE_BF16 && X.dtype == QLR_BF16)) return QLR_EINVAL;
  const Plan pl = make_plan(compute, op, M, K, l, ctx->num_sms > 0 ? ctx->num_sms : 148, true,
                            A.plane[0] == nullptr ? 3 : 4, X.dtype == QLR_F32);
  if (pl.stages < 2) return QLR_EUNSUPPORTED;
  size_t mark = ws.off;
  // stage the thin operand with a 16-byte aligned column pitch
  const int64_t ldo = (K + 7) / 8 * 8;
  const size_t xesz = (pl.kind == K_BF16) ? 2 : 4;
  const size_t xb = staged_x_bytes(pl.fd, pl.apl, ldo, l, pl.nb, pl.ncb, xesz);
  void* xs = ws.take<char>(xb);
  void* xlo = (pl.kind == K_TF32X3) ? ws.take<char>(xb) : nullptr;
  const size_t tile_elems = (size_t)4 * TBM * pl.nb;
  float* part = pl.grid_sk > 0 ? ws.take<float>((size_t)2 * pl.grid_sk * tile_elems) : nullptr;
  unsigned* counters = ws.take<unsigned>((size_t)pl.mtiles * pl.ncb);
  if (!ws.ok) return QLR_ENOMEM;
  if (X.dtype == QLR_BF16) {
    qlr_qmat dst = X;
    dst.ld = ldo;
    for (int c = 0; c < 4; ++c) dst.plane[c] = static_cast<char*>(xs) + (size_t)c * ldo * l * 2;
    QLR_TRY(convert_qmat(ctx, X, dst));
  } else {
    StageArg sa{};
    for (int c = 0; c < 4; ++c) sa.x[c] = static_cast<const float*>(X.plane[c]);
    sa.ldx = X.ld;
    sa.rows = K;
    sa.cols = l;
    sa.ldo = ldo;
    sa.out = xs;
    sa.out_lo = xlo;
    sa.fd = pl.fd ? 1 : 0;
    sa.nb = pl.nb;
    sa.ncb = pl.ncb;
    sa.c0 = 4 - pl.apl;
    sa.neg = neg_table(op);
    sa.nrows = pl.fd ? pl.apl * pl.ncb * 4 * pl.nb : 4 * l;
    sa.rn = pl.rn ? 1 : 0;
    if (sa.nrows > 65535) return QLR_EUNSUPPORTED;
    const dim3 grid((unsigned)((K + STAGE_ROWS - 1) / STAGE_ROWS), (unsigned)sa.nrows);
    KTimer kt(ctx, QLR_KID_MISC);
    if (pl.kind == K_BF16) stage_x_kernel<K_BF16><<<grid, 256, 0, ctx->stream>>>(sa);
    else if (pl.kind == K_TF32) stage_x_kernel<K_TF32><<<grid, 256, 0, ctx->stream>>>(sa);
    else stage_x_kernel<K_TF32X3><<<grid, 256, 0, ctx->stream>>>(sa);
    qlr_count_launch();
    QLR_CUDA_TRY(cudaGetLastError());
  }
  QLR_CUDA_TRY(cudaMemsetAsync(counters, 0, (size_t)pl.mtiles * pl.ncb * sizeof(unsigned), ctx->stream));

  TcParams prm;
  memset(&prm, 0, sizeof(prm));
  const CUtensorMapDataType dt = (pl.kind == K_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const CUtensorMapSwizzle sw = (pl.sw == 32) ? CU_TENSOR_MAP_SWIZZLE_32B
                                : (pl.sw == 64) ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  const int esz = pl.esz;
  prm.c_first = (A.plane[0] == nullptr) ? 1 : 0;
  prm.apl = pl.apl;
  for (int c = prm.c_first; c < 4; ++c) {
    bool ok;
    if (op == QLR_OP_N)   // K-major: inner = n (reduction), outer = m (output rows); box {BK, 128}
      ok = encode_2d(&prm.tmA[c], A.plane[c], dt, (uint64_t)A.cols, (uint64_t)A.rows, (uint64_t)A.ld * esz,
                     (uint32_t)pl.bk, TBM, sw);
    else if (pl.amode == A_MN)   // MN-major: inner = n (output rows), outer = m (reduction); box {SW/esz, BK}
      ok = encode_2d(&prm.tmA[c], A.plane[c], dt, (uint64_t)A.cols, (uint64_t)A.rows, (uint64_t)A.ld * esz,
                     (uint32_t)(pl.sw / esz), (uint32_t)pl.bk, sw);
    else                         // raw tile for the worker transpose: box {128, BK}, unswizzled
      ok = encode_2d(&prm.tmA[c], A.plane[c], dt, (uint64_t)A.cols, (uint64_t)A.rows, (uint64_t)A.ld * esz, TBM,
                     (uint32_t)pl.bk, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (!ok) { ws.off = mark; return QLR_ECUDA; }
  }
  if (pl.fd) {   // X~_c of input plane c >= c_first: ncb 4 nb rows, boxes of 4 nb rows
    const int64_t fr = (int64_t)pl.ncb * 4 * pl.nb;
    for (int c = 4 - pl.apl; c < 4; ++c) {
      const size_t off = (size_t)(c - (4 - pl.apl)) * fr * ldo;
      if (!encode_2d(&prm.tmX[c], static_cast<const char*>(xs) + off * xesz, dt, (uint64_t)K, (uint64_t)fr,
                     (uint64_t)ldo * xesz, (uint32_t)pl.bk, (uint32_t)(4 * pl.nb), sw)) { ws.off = mark; return QLR_ECUDA; }
      if (xlo && !encode_2d(&prm.tmXlo[c], static_cast<const char*>(xlo) + off * 4, dt, (uint64_t)K, (uint64_t)fr,
                            (uint64_t)ldo * 4, (uint32_t)pl.bk, (uint32_t)(4 * pl.nb), sw)) { ws.off = mark; return QLR_ECUDA; }
    }
  }
  for (int q = 0; q < 4 && !pl.fd; ++q) {
    const char* base = static_cast<const char*>(xs) + (size_t)q * ldo * l * xesz;
    if (!encode_2d(&prm.tmX[q], base, dt, (uint64_t)K, (uint64_t)l, (uint64_t)ldo * xesz, (uint32_t)pl.bk,
                   (uint32_t)pl.nb, sw)) { ws.off = mark; return QLR_ECUDA; }
    if (xlo) {
      const char* lb = static_cast<const char*>(xlo) + (size_t)q * ldo * l * 4;
      if (!encode_2d(&prm.tmXlo[q], lb, dt, (uint64_t)K, (uint64_t)l, (uint64_t)ldo * 4, (uint32_t)pl.bk,
                     (uint32_t)pl.nb, sw)) { ws.off = mark; return QLR_ECUDA; }
    }
  }
  for (int c = 0; c < 4; ++c) prm.y[c] = static_cast<float*>(Y.plane[c]);
  prm.ldy = Y.ld;
  prm.part = part;
  prm.counters = counters;
  prm.M = M;
  prm.l = l;
  prm.nb = pl.nb;
  prm.ncb = pl.ncb;
  prm.kiters = pl.kiters;
  prm.mtiles = pl.mtiles;
  prm.neg_mask = neg_table(op);
  prm.fd = pl.fd ? 1 : 0;
  const uint32_t fmt = (pl.kind == K_BF16) ? 1u : 2u;
  prm.idesc_base = (1u << 4) | (fmt << 7) | (fmt << 10) | ((pl.amode == A_MN ? 1u : 0u) << 15) |
                   ((uint32_t)((pl.fd ? 4 * pl.nb : pl.nb) >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);
  prm.tmem_cols = pl.tmem_cols;
  prm.stages = pl.stages;
  prm.err = ctx->d_err;
  prm.flush = pl.flush;
  prm.nbuf = pl.nbuf;
  prm.ttotal = pl.ttotal;
  prm.rn = pl.rn ? 1 : 0;
  prm.cgroup = pl.cgroup ? 1 : 0;
  int rc;
  const bool h = (op != QLR_OP_N);
  const int kid = (pl.kind == K_TF32X3) ? QLR_KID_SKETCH_X3 : pl.rn ? QLR_KID_SKETCH_RN : QLR_KID_SKETCH_TC;
  if (pl.kind == K_BF16) rc = h ? launch_kernel<K_BF16, A_MN>(ctx, pl, prm, kid) : launch_kernel<K_BF16, A_K>(ctx, pl, prm, kid);
  else if (pl.kind == K_TF32) rc = h ? launch_kernel<K_TF32, A_T>(ctx, pl, prm, kid) : launch_kernel<K_TF32, A_K>(ctx, pl, prm, kid);
  else rc = h ? launch_kernel<K_TF32X3, A_T>(ctx, pl, prm, kid) : launch_kernel<K_TF32X3, A_K>(ctx, pl, prm, kid);
  ws.off = mark;
  return rc;
}

}  // namespace qlr
