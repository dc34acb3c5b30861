// FP32 Gram G = Q^H Q of a nearly orthonormal thin quaternion basis (the Gram product of Def. 1
// eq. QQR in the last step of CholeskyQR2 / shifted CholeskyQR3), for batch plans.
//
// In the last step of CholeskyQR2 the input Q1 = Y R1^{-1} already has condition number close to
// one: its Gram is I + E with |E| far below one, so an FP32 Gram perturbs the factor R2 by
// rounding-level amounts only, the same order as the FP32 storage of Q1 itself (mixed-precision
// CholeskyQR: the higher precision is needed only where the Gram of an ill-conditioned matrix is
// formed).  The FP64-class tensor-core Gram (gram_tc.cu) stays on every step whose input may be
// ill-conditioned.
//
// One CTA of 64 threads per (problem, 16 x 16 tile (I, J) of G with J >= I): thread (i, g) sums
// conj(Q(k, I16 + i)) Q(k, J16 + g + 4u), u = 0..3, over all rows k (four entries per thread:
// five shared-memory loads per 64 FMAs), the rows staged 32 at a time in shared memory as
// interleaved quaternions, with two accumulators per entry over even and odd rows, added at the
// end.  The result goes to the double-FP32 layout the grouped Cholesky reads (8 floats per entry
// at G + 8 (j l + i), upper triangle; the low parts zero).
#include "qlr_internal.h"

namespace qlr {

namespace {

constexpr int GF_T = 16;      // tile edge (entries)
constexpr int GF_KC = 32;     // rows per shared-memory chunk

// acc += conj(a) * b (Hamilton product of the conjugate, Section 2), as 16 FMAs
__device__ __forceinline__ void qcfma(float4& acc, const float4& a, const float4& b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x); acc.x = fmaf(a.z, b.z, acc.x); acc.x = fmaf(a.w, b.w, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y); acc.y = fmaf(-a.z, b.w, acc.y); acc.y = fmaf(a.w, b.z, acc.y);
  acc.z = fmaf(a.x, b.z, acc.z); acc.z = fmaf(a.y, b.w, acc.z); acc.z = fmaf(-a.z, b.x, acc.z); acc.z = fmaf(-a.w, b.y, acc.z);
  acc.w = fmaf(a.x, b.w, acc.w); acc.w = fmaf(-a.y, b.z, acc.w); acc.w = fmaf(a.z, b.y, acc.w); acc.w = fmaf(-a.w, b.x, acc.w);
}

constexpr int GF_THREADS = 64;

__global__ void __launch_bounds__(GF_THREADS) gram_f32_grouped_kernel(const GramF32Args* __restrict__ args,
                                                                      const int4* __restrict__ items) {
  __shared__ float4 Ya[GF_KC][GF_T + 1], Yb[GF_KC][GF_T + 1];   // padded rows: conflict-free staging
  const int4 it = items[blockIdx.x];
  const GramF32Args& a = args[it.x];
  const int l = a.l;
  const int64_t m = a.m, ld = a.ld;
  const int i0 = it.y * GF_T, j0 = it.z * GF_T;
  const int t = threadIdx.x, ti = t / 4, tg = t % 4;
  const float* y0 = a.y[0];
  const float* y1 = a.y[1];
  const float* y2 = a.y[2];
  const float* y3 = a.y[3];
  float4 s0[4], s1[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) s0[u] = s1[u] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t k0 = 0; k0 < m; k0 += GF_KC) {
    __syncthreads();
    // stage rows k0 .. k0 + 31 of the two column blocks (consecutive threads: consecutive rows)
    for (int e = t; e < 2 * GF_KC * GF_T; e += GF_THREADS) {
      const int blk = e / (GF_KC * GF_T), rem = e % (GF_KC * GF_T);
      const int c = rem / GF_KC, r = rem % GF_KC;
      const int col = (blk == 0 ? i0 : j0) + c;
      const int64_t k = k0 + r;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (col < l && k < m) {
        const int64_t o = (int64_t)col * ld + k;
        v = make_float4(y0[o], y1[o], y2[o], y3[o]);
      }
      if (blk == 0) Ya[r][c] = v; else Yb[r][c] = v;
    }
    __syncthreads();
#pragma unroll 2
    for (int r = 0; r < GF_KC; r += 2) {
      const float4 a0 = Ya[r][ti], a1 = Ya[r + 1][ti];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        qcfma(s0[u], a0, Yb[r][tg + 4 * u]);
        qcfma(s1[u], a1, Yb[r + 1][tg + 4 * u]);
      }
    }
  }
  const int i = i0 + ti;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = j0 + tg + 4 * u;
    if (i < l && j < l && i <= j) {
      float4* g = reinterpret_cast<float4*>(a.G + 8 * ((size_t)j * l + i));
      g[0] = make_float4(s0[u].x + s1[u].x, s0[u].y + s1[u].y, s0[u].z + s1[u].z, s0[u].w + s1[u].w);
      g[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

}  // namespace

void gram_f32_items(int l, int prob, std::vector<int4>& items) {
  const int nt = (l + GF_T - 1) / GF_T;
  for (int I = 0; I < nt; ++I)
    for (int J = I; J < nt; ++J) items.push_back(make_int4(prob, I, J, 0));
}

int gram_f32_grouped(qlr_ctx* ctx, const GramF32Args* d_args, const int4* d_items, int nitems) {
  if (nitems <= 0) return QLR_OK;
  KTimer kt(ctx, QLR_KID_GRAM);
  gram_f32_grouped_kernel<<<nitems, GF_THREADS, 0, ctx->stream>>>(d_args, d_items);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

}  // namespace qlr
