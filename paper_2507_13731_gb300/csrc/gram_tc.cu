// FP64-class Gram matrix G = Y^H Y of an FP32 thin quaternion sketch on the tcgen05 tensor cores
// (the Gram product of CholeskyQR, Def. 1 eq. QQR and every QR of Algorithms 1-4).
//
// G's components are sums of the real Gram W = Yh^T Yh of the plane-stacked Yh = [Y0 Y1 Y2 Y3]
// (m x 4l).  W is formed exactly enough for FP64-class use by an error-free splitting:
//  - every column c of Yh gets the exponent e_c with max_r |Yh(r, c)| < 2^e_c, and each entry is
//    written as y = 2^(e_c - 6) (q_1 + q_2 2^-6 + ... + q_8 2^-42) + rest with integers
//    |q_i| <= 63 (48 bits below the column maximum; an entry of at least 2^-24 of the column
//    maximum is represented exactly, a smaller one to 2^-48 of the maximum);
//  - the q_i are exact in BF16, their products exact in FP32, and the tensor core's FP32 sums of
//    such integer products stay exact while they stay below 2^24: the slice pairs (i, j) of equal
//    weight s = i + j - 2 share one TMEM accumulator, at most 8 pairs x 512 rows x 63^2 < 2^24,
//    so every CTA reduces a chunk of at most 512 rows;
//  - pairs with i + j > 9 (weight below 2^-48) are left out: 36 BF16 products per entry and row;
//  - the 8 exact integer sums of a chunk are scaled by 2^-6s (exact) and added in double-FP32,
//    the chunks are added in double-FP32, and the result is scaled by 2^(e_a + e_b - 12).
// The error of W(a, b) is about 2^-45 of max|y_a| max|y_b| m: FP64-class, as the Gram of the
// double-FP32 SIMT path (orth.cu), at tensor-core throughput.
//
// Kernels: gram_slice_kernel (one CTA per column: exponent, then the 8 slices, BF16, column-major
// per slice with rows padded to a multiple of 8), gram_tc_kernel (one CTA per (128 x 64 tile of
// W's upper part, 512-row chunk): TMA of the 8 slices of both operands into a 4-stage ring of
// 16-row stages, 12 MMAs of 128 x (64..256) x 16 per stage into 8 x 64 TMEM columns, epilogue to
// double-FP32 partial tiles), gram_tc_combine_kernel (chunk sums, scaling, the quaternion
// components of G).
#include <algorithm>
#include <cstring>

#include "qlr_internal.h"
#include "tc_common.cuh"

namespace {

using namespace qlr_tc;

constexpr int GS = 8;            // slices per entry, 6 bits each
constexpr int GBITS = 6;
constexpr int GPAIR_MAX = 9;     // slice pairs (i, j), 1-based, with i + j <= 9
constexpr int NGRP = GPAIR_MAX - 1;   // weights s = i + j - 2 = 0 .. 7
constexpr int GA = 128;          // W rows per tile (MMA M)
constexpr int GB = 64;           // W columns per tile (MMA N)
constexpr int GK = 16;           // rows of Y per pipeline stage (32-byte swizzled BF16 rows, one MMA K)
constexpr int GCHUNK = 512;      // rows of Y per CTA (exactness of the TMEM sums)
constexpr int GSTAGES = 4;
constexpr int GTHREADS = 256;
constexpr int GSW = GK * 2;           // bytes per K-major row = swizzle span
constexpr int GMODE = 6;              // descriptor swizzle mode: 32 bytes
constexpr int A_TILE = GA * GK * 2;   // bytes of one slice's A tile
constexpr int B_TILE = GB * GK * 2;
constexpr int STAGE_BYTES = GS * (A_TILE + B_TILE);
constexpr size_t GSMEM = (size_t)GSTAGES * STAGE_BYTES + 1024 + 256;

struct GramTcParams {
  CUtensorMap tmA;      // slices as (mp rows inner) x (GS L4p columns outer), box {GK, GA}
  CUtensorMap tmB;      // the same array, box {GK, GB}
  float2* part;         // [chunk] L4 x L4 column-major: W(a, b) at b L4 + a, double-FP32 (h, l)
  int L4, nA, nB;       // W order, a-blocks of GA, b-blocks of GB
  int L4p;              // columns per slice (L4 rounded up to GB; an A tile may run into the
                        // next slice: those W rows a >= L4 are never stored)
  int kiters;           // GK-row stages over all m rows
  int* err;
};

// A problem of a batch plan: the MMA parameters (tensor maps first, 64-byte aligned) and what the
// slicing and the combine need.
struct GramTcProb {
  GramTcParams tc;
  const float* y[4];
  int64_t m, ld, mp;
  int l, nchunks;
  __nv_bfloat16* S;
  int* ex;
  float* G;             // double-FP32 upper triangle, 8 floats per entry at G + 8 (j l + i)
};

// Columns of Yh (L4p columns, the padding zero) by CTAs of 8 warps, WPC warps per column (8 for
// one tall problem, 1 for the many short ones of a batch): the column exponent, then the 8
// slices; each lane takes row pairs, stored as BF16 pairs.
template <int WPC>
__device__ __forceinline__ void gram_slice_cols(const float* __restrict__ y0, const float* __restrict__ y1,
                                                const float* __restrict__ y2, const float* __restrict__ y3, int64_t m,
                                                int l, int64_t ld, int L4p, int64_t mp, __nv_bfloat16* __restrict__ S,
                                                int* __restrict__ ex, const int g) {
  __shared__ float red[8];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int c = g * (8 / WPC) + warp / WPC, sub = warp % WPC;
  const bool valid = c < L4p;
  const float* y = nullptr;
  if (valid && c < 4 * l) {
    const int pl = c / l, j = c % l;
    y = (pl == 0 ? y0 : pl == 1 ? y1 : pl == 2 ? y2 : y3) + (int64_t)j * ld;
  }
  float mx = 0.f;
  if (y)
    for (int64_t r = sub * 32 + lane; r < m; r += 32 * WPC) mx = fmaxf(mx, fabsf(y[r]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (WPC > 1) {
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    const int w0 = warp - sub;
    for (int w = 0; w < WPC; ++w) mx = fmaxf(mx, red[w0 + w]);
  }
  if (!valid) return;
  int e = 0;
  if (mx > 0.f) frexpf(mx, &e);   // max < 2^e
  if (sub == 0 && lane == 0) ex[c] = e;
  for (int64_t r = 2 * (sub * 32 + lane); r < mp; r += 64 * WPC) {   // mp is even
    float v0 = (y && r < m) ? ldexpf(y[r], GBITS - e) : 0.f;       // |v| < 64, exact
    float v1 = (y && r + 1 < m) ? ldexpf(y[r + 1], GBITS - e) : 0.f;
#pragma unroll
    for (int i = 0; i < GS; ++i) {
      const float q0 = truncf(v0), q1 = truncf(v1);                // |q| <= 63
      *reinterpret_cast<__nv_bfloat162*>(S + ((size_t)i * L4p + c) * mp + r) = __floats2bfloat162_rn(q0, q1);
      v0 = (v0 - q0) * 64.f;                                        // exact
      v1 = (v1 - q1) * 64.f;
    }
  }
}

__global__ void __launch_bounds__(256) gram_slice_kernel(const float* __restrict__ y0, const float* __restrict__ y1,
                                                         const float* __restrict__ y2, const float* __restrict__ y3,
                                                         int64_t m, int l, int64_t ld, int L4p, int64_t mp,
                                                         __nv_bfloat16* __restrict__ S, int* __restrict__ ex) {
  gram_slice_cols<8>(y0, y1, y2, y3, m, l, ld, L4p, mp, S, ex, blockIdx.x);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

// (s, e) += x exactly into a two-float sum (Knuth's two-sum, the rounding error kept in e).
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x) {
  const float t = __fadd_rn(s, x);
  const float v = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, v)), __fsub_rn(x, v));
  s = t;
  e = __fadd_rn(e, err);
}

// One tile of W for one chunk of rows: tile index tl enumerates (ab, bb) with bb >= 2 ab (the
// upper part of W).
__device__ __forceinline__ void gram_tc_tile(const GramTcParams& p, int tl, const int chunk) {
  int ab = 0;
  while (ab < p.nA && tl >= max(0, p.nB - 2 * ab)) { tl -= max(0, p.nB - 2 * ab); ++ab; }
  const int bb = 2 * ab + tl;
  const int a0 = ab * GA, b0 = bb * GB;
  const int it0 = chunk * (GCHUNK / GK);
  const int it1 = min(p.kiters, it0 + GCHUNK / GK);
  const int nit = it1 - it0;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + GSTAGES * STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + GSTAGES;
  uint64_t* tmem_full = bars + 2 * GSTAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * GSTAGES + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto a_tile = [&](int s, int i) { return smem + s * STAGE_BYTES + i * A_TILE; };
  auto b_tile = [&](int s, int j) { return smem + s * STAGE_BYTES + GS * A_TILE + j * B_TILE; };

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < GSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tmem_full, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(NGRP * GB)
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
      int issued = 0;
      for (int i = 0; i < nit; ++i) {
        const int s = i % GSTAGES;
        const uint32_t ph = (uint32_t)(i / GSTAGES) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, p.err)) break;
        mbar_expect_tx(&full[s], (uint32_t)STAGE_BYTES);
        const int k0 = (it0 + i) * GK;
        for (int q = 0; q < GS; ++q) {
          tma_load_2d(smem_u32(a_tile(s, q)), &p.tmA, k0, q * p.L4p + a0, &full[s]);
          tma_load_2d(smem_u32(b_tile(s, q)), &p.tmB, k0, q * p.L4p + b0, &full[s]);
        }
        ++issued;
      }
      // drain: every issued stage must have landed before the CTA may exit
      for (int i = max(0, issued - GSTAGES); i < issued; ++i) {
        const int s = i % GSTAGES;
        const uint32_t ph = (uint32_t)(i / GSTAGES) & 1u;
        const uint64_t t0 = now_ns();
        while (!mbar_try_wait(&full[s], ph) && now_ns() - t0 < WAIT_NS) __nanosleep(64);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      // BF16 A and B, FP32 D, both K-major, M = GA; N = t GB for t consecutive B slices: the B
      // slice tiles are adjacent in shared memory, and one MMA of A_i against slices j .. j+t-1
      // writes pair (i, j + u) to TMEM columns (i + j + u) GB, the accumulator of its weight group
      const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GA >> 4) << 24);
      bool ok = true;
      for (int i = 0; i < nit && ok; ++i) {
        const int s = i % GSTAGES;
        const uint32_t ph = (uint32_t)(i / GSTAGES) & 1u;
        ok = mbar_wait(&full[s], ph, abort_flag, p.err);
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int ks = 0; ks < GK / 16; ++ks) {
#pragma unroll
          for (int qi = 0; qi < GS; ++qi) {
            const uint64_t ad = make_desc(smem_u32(a_tile(s, qi)) + (uint32_t)(ks * 32), 16, 8 * GSW, GMODE);
#pragma unroll
            for (int qj = 0; qj <= GPAIR_MAX - 2 - qi; qj += 4) {
              const int t = min(4, GPAIR_MAX - 1 - qi - qj);   // slices qj .. qj + t - 1
              const uint64_t bd = make_desc(smem_u32(b_tile(s, qj)) + (uint32_t)(ks * 32), 16, 8 * GSW, GMODE);
              const uint32_t idesc = idesc0 | ((uint32_t)((t * GB) >> 3) << 17);
              // first products of the weight groups in this chunk: qi == 0, first stage and k-step
              const uint32_t acc = (i > 0 || ks > 0 || qi > 0) ? 1u : 0u;
              umma_bf16(tmem + (uint32_t)((qi + qj) * GB), ad, bd, idesc, acc);
            }
          }
        }
        umma_commit(&empty[s]);   // frees the stage once these MMAs have read it
      }
      umma_commit(tmem_full);     // accumulators complete (also fires after an abort)
    }
  } else if (warp >= 4) {
    // ---------------- epilogue: 8 exact integer sums -> double-FP32 ----------------
    const int q = warp & 3;
    const int a = a0 + q * 32 + lane;
    const bool ok = mbar_wait(tmem_full, 0, abort_flag, p.err) && !*abort_flag;
    tc_fence_after();
    if (ok && nit > 0) {
      float h[GB], e[GB];
#pragma unroll
      for (int jj = 0; jj < GB; ++jj) h[jj] = e[jj] = 0.f;
#pragma unroll
      for (int g = NGRP - 1; g >= 0; --g) {
        const float w = __int_as_float((127 - GBITS * g) << 23);   // 2^-6g
#pragma unroll
        for (int cc = 0; cc < GB; cc += 32) {
          uint32_t r0[16], r1[16];
          const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * GB + cc);
          tmem_ld16_issue(ta, r0);
          tmem_ld16_issue(ta + 16, r1);
          tmem_wait_ld();
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            two_sum_acc(h[cc + jj], e[cc + jj], __uint_as_float(r0[jj]) * w);
            two_sum_acc(h[cc + 16 + jj], e[cc + 16 + jj], __uint_as_float(r1[jj]) * w);
          }
        }
      }
      if (a < p.L4) {
        float2* P = p.part + (size_t)chunk * p.L4 * p.L4;
#pragma unroll
        for (int jj = 0; jj < GB; ++jj) {
          const int b = b0 + jj;
          if (b < p.L4) P[(size_t)b * p.L4 + a] = make_float2(h[jj], e[jj]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NGRP * GB) : "memory");
  }
}

__global__ void __launch_bounds__(GTHREADS, 1) gram_tc_kernel(const __grid_constant__ GramTcParams p) {
  gram_tc_tile(p, blockIdx.x, blockIdx.y);
}

// Batch plans: item (problem, tile, chunk) with that problem's parameters in global memory
// (tensor maps 64-byte aligned, written before the launch).
__global__ void __launch_bounds__(GTHREADS, 1) gram_tc_grouped_kernel(const GramTcProb* __restrict__ probs,
                                                                      const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const GramTcParams& p = probs[it.x].tc;
  if (threadIdx.x == 0) {   // the TMA-issuing thread
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&p.tmA) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&p.tmB) : "memory");
  }
  gram_tc_tile(p, it.y, it.z);
}

// W(I, J) for I <= J: the chunk partials added in double-FP32, scaled by 2^(e_I + e_J - 12).
__device__ __forceinline__ double w_tc(const float2* __restrict__ part, int nchunks, const int* __restrict__ ex, int L4,
                                       int I, int J) {
  if (I > J) { const int t = I; I = J; J = t; }
  const size_t o = (size_t)J * L4 + I, step = (size_t)L4 * L4;
  float s = 0.f, e = 0.f;
  for (int c = 0; c < nchunks; ++c) {
    const float2 v = part[c * step + o];
    two_sum_acc(s, e, v.x);
    e = __fadd_rn(e, v.y);
  }
  return ldexp((double)s + (double)e, ex[I] + ex[J] - 2 * GBITS);
}

// W(I, J), I <= J, as a scaled double-FP32 pair (s, e).
__device__ __forceinline__ float2 w_tc_d32(const float2* __restrict__ part, int nchunks, const int* __restrict__ ex,
                                           int L4, int I, int J) {
  if (I > J) { const int t = I; I = J; J = t; }
  const size_t o = (size_t)J * L4 + I, step = (size_t)L4 * L4;
  float s = 0.f, e = 0.f;
  for (int c = 0; c < nchunks; ++c) {
    const float2 v = part[c * step + o];
    two_sum_acc(s, e, v.x);
    e = __fadd_rn(e, v.y);
  }
  const int k = ex[I] + ex[J] - 2 * GBITS;
  return make_float2(ldexpf(s, k), ldexpf(e, k));
}

// Batch plans: item (problem, block of 128 entries); G's upper triangle in double-FP32.
__global__ void __launch_bounds__(128) gram_tc_combine_grouped_kernel(const GramTcProb* __restrict__ probs,
                                                                      const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const GramTcProb& a = probs[it.x];
  const int l = a.l, L4 = 4 * l;
  const int idx = it.y * 128 + (int)threadIdx.x;
  if (idx >= l * l) return;
  const int i = idx % l, j = idx / l;
  if (i > j) return;
  // component signs of conj(y_i) y_j from the 16 plane products W(c l + i, d l + j)
  const float sg[4][4][4] = {{{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}},
                             {{0, -1, 0, 0}, {1, 0, 0, 0}, {0, 0, 0, -1}, {0, 0, 1, 0}},
                             {{0, 0, -1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, -1, 0, 0}},
                             {{0, 0, 0, -1}, {0, 0, -1, 0}, {0, 1, 0, 0}, {1, 0, 0, 0}}};
  float gs[4] = {0.f, 0.f, 0.f, 0.f}, ge[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const float2 w = w_tc_d32(a.tc.part, a.nchunks, a.ex, L4, c * l + i, d * l + j);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (sg[c][d][q] != 0.f) {
          two_sum_acc(gs[q], ge[q], sg[c][d][q] * w.x);
          ge[q] = __fadd_rn(ge[q], sg[c][d][q] * w.y);
        }
    }
  float h[4], lo[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    h[q] = __fadd_rn(gs[q], ge[q]);
    lo[q] = __fsub_rn(ge[q], __fsub_rn(h[q], gs[q]));
    if (i == j && q > 0) h[q] = lo[q] = 0.f;
  }
  float4* o = reinterpret_cast<float4*>(a.G + 8 * ((size_t)j * l + i));
  o[0] = make_float4(h[0], h[1], h[2], h[3]);
  o[1] = make_float4(lo[0], lo[1], lo[2], lo[3]);
}

__global__ void __launch_bounds__(256) gram_slice_grouped_kernel(const GramTcProb* __restrict__ probs,
                                                                 const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const GramTcProb& a = probs[it.x];
  gram_slice_cols<1>(a.y[0], a.y[1], a.y[2], a.y[3], a.m, a.l, a.ld, a.tc.L4p, a.mp, a.S, a.ex, it.y);
}

// The quaternion Gram from W, FP64 planes: 16 threads per entry (i <= j), thread (c, d) forms
// W(c l + i, d l + j); component q = c xor d of conj(y_i) y_j takes it with the sign of the
// Hamilton table (negative for (c, d) in {(1,0),(2,0),(3,0),(1,2),(2,3),(3,1)}), and the four
// threads of each component add their terms by two shuffles.
__global__ void __launch_bounds__(128) gram_tc_combine_kernel(const float2* __restrict__ part, int nchunks,
                                                              const int* __restrict__ ex, int l, double* __restrict__ G) {
  const int e = blockIdx.x * 8 + (int)(threadIdx.x >> 4);
  const int lane16 = threadIdx.x & 15, c = lane16 >> 2, d = lane16 & 3;
  const int ntri = l * (l + 1) / 2;
  // entry e of the column-by-column listing of the upper triangle: j the largest with j (j + 1) / 2 <= e
  int j = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (j > 0 && j * (j + 1) / 2 > e) --j;
  while ((j + 1) * (j + 2) / 2 <= e) ++j;
  const int i = e - j * (j + 1) / 2;
  double v = 0.0;
  if (e < ntri) {
    v = w_tc(part, nchunks, ex, 4 * l, c * l + i, d * l + j);
    if ((0x3950u >> (c * 4 + d)) & 1u) v = -v;
  }
  v += __shfl_xor_sync(0xffffffffu, v, 5);
  v += __shfl_xor_sync(0xffffffffu, v, 10);
  if (e < ntri && c == 0) {   // thread (0, q) holds component q
    const int q = d;
    const size_t ll = (size_t)l * l;
    const double gq = (i == j && q > 0) ? 0.0 : v;
    G[q * ll + (size_t)j * l + i] = gq;
    if (i != j) G[q * ll + (size_t)i * l + j] = (q == 0) ? gq : -gq;
  }
}

struct GramTcDims {
  int L4, L4p, nA, nB, ntiles, nchunks, kiters;
  int64_t mp;
};
GramTcDims gram_tc_dims(int64_t m, int l) {
  GramTcDims d{};
  d.L4 = 4 * l;
  d.L4p = (d.L4 + GB - 1) / GB * GB;
  d.nA = (d.L4 + GA - 1) / GA;
  d.nB = (d.L4 + GB - 1) / GB;
  d.ntiles = 0;
  for (int ab = 0; ab < d.nA; ++ab) d.ntiles += std::max(0, d.nB - 2 * ab);
  d.mp = std::max<int64_t>(GK, (m + 7) / 8 * 8);   // at least one TMA box of rows
  d.kiters = (int)((m + GK - 1) / GK);
  d.nchunks = (int)((m + GCHUNK - 1) / GCHUNK);
  return d;
}

struct GramTcBufs {
  __nv_bfloat16* S;
  int* ex;
  float2* part;
};
size_t rup256(size_t b) { return (b + 255) / 256 * 256; }
GramTcBufs gram_tc_carve(char* base, const GramTcDims& d) {
  GramTcBufs b;
  b.S = reinterpret_cast<__nv_bfloat16*>(base);
  base += rup256((size_t)GS * d.L4p * d.mp * 2);
  b.ex = reinterpret_cast<int*>(base);
  base += rup256((size_t)d.L4p * 4);
  b.part = reinterpret_cast<float2*>(base);
  return b;
}

// Tensor maps and dimensions of one problem (host side).
bool gram_tc_params(GramTcParams& prm, const GramTcDims& d, const GramTcBufs& bufs, int* err) {
  memset(&prm, 0, sizeof(prm));
  const uint64_t cols = (uint64_t)GS * d.L4p;
  if (!encode_2d(&prm.tmA, bufs.S, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (uint64_t)d.mp, cols, (uint64_t)d.mp * 2, GK, GA,
                 CU_TENSOR_MAP_SWIZZLE_32B) ||
      !encode_2d(&prm.tmB, bufs.S, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (uint64_t)d.mp, cols, (uint64_t)d.mp * 2, GK, GB,
                 CU_TENSOR_MAP_SWIZZLE_32B))
    return false;
  prm.part = bufs.part;
  prm.L4 = d.L4;
  prm.nA = d.nA;
  prm.nB = d.nB;
  prm.L4p = d.L4p;
  prm.kiters = d.kiters;
  prm.err = err;
  return true;
}

}  // namespace

namespace qlr {

size_t gram_tc_ws(int64_t m, int l) {
  const GramTcDims d = gram_tc_dims(m, l);
  return rup256((size_t)GS * d.L4p * d.mp * 2) + rup256((size_t)d.L4p * 4) + rup256((size_t)d.nchunks * d.L4 * d.L4 * 8);
}

bool gram_tc_supported(const qlr_qmat& Y) {
  if (Y.dtype != QLR_F32 || Y.layout != QLR_COL_MAJOR || Y.rows <= 0 || Y.cols <= 0) return false;
  for (int c = 0; c < 4; ++c)
    if (Y.plane[c] == nullptr) return false;
  const GramTcDims d = gram_tc_dims(Y.rows, (int)Y.cols);
  return Y.cols <= 1024 && (int64_t)GS * d.L4p < (1 << 30) && d.nchunks < 65536 && get_encode() != nullptr;
}

int gram_tc(qlr_ctx* ctx, const qlr_qmat& Y, double* G, WsArena& ws) {
  const int64_t m = Y.rows;
  const int l = (int)Y.cols;
  const GramTcDims d = gram_tc_dims(m, l);
  const size_t mark = ws.off;
  char* base = ws.take<char>(gram_tc_ws(m, l));
  if (!ws.ok) { ws.off = mark; ws.ok = true; return QLR_ENOMEM; }
  const GramTcBufs bufs = gram_tc_carve(base, d);
  __nv_bfloat16* S = bufs.S;
  int* ex = bufs.ex;
  float2* part = bufs.part;
  GramTcParams prm;
  if (!gram_tc_params(prm, d, bufs, ctx->d_err)) {
    ws.off = mark;
    return QLR_ECUDA;
  }
  KTimer kt(ctx, QLR_KID_GRAM);
  gram_slice_kernel<<<d.L4p, 256, 0, ctx->stream>>>(
      static_cast<const float*>(Y.plane[0]), static_cast<const float*>(Y.plane[1]), static_cast<const float*>(Y.plane[2]),
      static_cast<const float*>(Y.plane[3]), m, l, Y.ld, d.L4p, d.mp, S, ex);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  QLR_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GSMEM));
  gram_tc_kernel<<<dim3((unsigned)d.ntiles, (unsigned)d.nchunks), GTHREADS, GSMEM, ctx->stream>>>(prm);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  const int64_t ntri = (int64_t)l * (l + 1) / 2;
  gram_tc_combine_kernel<<<(unsigned)((ntri + 7) / 8), 128, 0, ctx->stream>>>(part, d.nchunks, ex, l, G);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  ws.off = mark;   // the buffers are dead once the combine is enqueued (stream order)
  return QLR_OK;
}

size_t gram_tc_record_bytes() { return sizeof(GramTcProb); }

int gram_tc_record(void* dst, const qlr_qmat& Y, char* scratch, float* G, int* err) {
  const int l = (int)Y.cols;
  const GramTcDims d = gram_tc_dims(Y.rows, l);
  const GramTcBufs bufs = gram_tc_carve(scratch, d);
  GramTcProb r;
  memset(&r, 0, sizeof(r));
  if (!gram_tc_params(r.tc, d, bufs, err)) return QLR_ECUDA;
  for (int c = 0; c < 4; ++c) r.y[c] = static_cast<const float*>(Y.plane[c]);
  r.m = Y.rows;
  r.ld = Y.ld;
  r.mp = d.mp;
  r.l = l;
  r.nchunks = d.nchunks;
  r.S = bufs.S;
  r.ex = bufs.ex;
  r.G = G;
  memcpy(dst, &r, sizeof(r));
  return QLR_OK;
}

void gram_tc_grouped_items(int64_t m, int l, int prob, std::vector<int4>& slice, std::vector<int4>& mma,
                           std::vector<int4>& comb) {
  const GramTcDims d = gram_tc_dims(m, l);
  for (int g = 0; g < (d.L4p + 7) / 8; ++g) slice.push_back(make_int4(prob, g, 0, 0));
  for (int ch = 0; ch < d.nchunks; ++ch)
    for (int t = 0; t < d.ntiles; ++t) mma.push_back(make_int4(prob, t, ch, 0));
  for (int b = 0; b < (l * l + 127) / 128; ++b) comb.push_back(make_int4(prob, b, 0, 0));
}

int gram_tc_grouped(qlr_ctx* ctx, const void* d_probs, const int4* slice, int n_slice, const int4* mma, int n_mma,
                    const int4* comb, int n_comb) {
  if (n_slice <= 0) return QLR_OK;
  const GramTcProb* probs = static_cast<const GramTcProb*>(d_probs);
  KTimer kt(ctx, QLR_KID_GRAM);
  gram_slice_grouped_kernel<<<n_slice, 256, 0, ctx->stream>>>(probs, slice);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  QLR_CUDA_TRY(cudaFuncSetAttribute(gram_tc_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GSMEM));
  gram_tc_grouped_kernel<<<n_mma, GTHREADS, GSMEM, ctx->stream>>>(probs, mma);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  gram_tc_combine_grouped_kernel<<<n_comb, 128, 0, ctx->stream>>>(probs, comb);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

}  // namespace qlr
