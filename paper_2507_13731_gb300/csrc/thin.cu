// Thin x small products C = T S: T (rows x l) a tall quaternion basis stored column-major, S a
// small l x k factor (R^{-1} of a CholeskyQR step, or the core QSVD's singular vectors for the
// lifts U = Q1 U_hat, V = Q2 V_hat).  FP32 operands run on thin_small_kernel; FP64 operands on
// the generic SIMT GEMM.  The tensor-core sketch kernel was measured on this shape (4096 x 110 x
// 110) and gained nothing: with K = l its CTAs run a dozen pipeline stages each and the 3xTF32
// split costs three MMAs.
#include <algorithm>

#include "qlr_internal.h"

namespace qlr {

namespace {
__global__ void small_to_f32_kernel(const double* __restrict__ S, float* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)S[e];
}

// FP32 thin x small product, one row of C per thread: a CTA takes TS_ROWS rows and COLS columns
// of C, stages S's rows for those columns in shared memory (TS_KC rows at a time, each entry a
// quaternion broadcast to every thread), and streams T's rows k into COLS quaternion
// accumulators, a few rows k at a time (the coalesced loads of the next 4 (16 columns: 2) rows
// are in flight while the quaternion multiply-adds of the current ones run; each multiply-add is
// 16 FMAs into the accumulator).  With an upper-triangular S (R^{-1}) rows k >= j0 + COLS of the chunk are zero
// and skipped.  Batches use 16 columns per CTA (many problems fill the GPU); a single product
// uses 8, for twice the CTAs.
constexpr int TS_ROWS = 128, TS_COLS = 16, TS_COLS1 = 8, TS_KC = 64;

// acc += a * b (Hamilton product, Section 2 eq. 1), as 16 FMAs
__device__ __forceinline__ void qfma(Quat<float>& acc, const Quat<float>& a, const float4& b) {
  acc.w = fmaf(a.w, b.x, acc.w); acc.w = fmaf(-a.x, b.y, acc.w); acc.w = fmaf(-a.y, b.z, acc.w); acc.w = fmaf(-a.z, b.w, acc.w);
  acc.x = fmaf(a.w, b.y, acc.x); acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.w, acc.x); acc.x = fmaf(-a.z, b.z, acc.x);
  acc.y = fmaf(a.w, b.z, acc.y); acc.y = fmaf(-a.x, b.w, acc.y); acc.y = fmaf(a.y, b.x, acc.y); acc.y = fmaf(a.z, b.y, acc.y);
  acc.z = fmaf(a.w, b.w, acc.z); acc.z = fmaf(a.x, b.z, acc.z); acc.z = fmaf(-a.y, b.y, acc.z); acc.z = fmaf(a.z, b.x, acc.z);
}

template <int COLS>
__device__ __forceinline__ void thin_small_tile(const GemmArgs& g, int64_t rb, int cc) {
  __shared__ float4 Bs[TS_KC][COLS + 1];   // padded rows: conflict-free staging
  const int t = threadIdx.x;
  const int j0 = cc * COLS;
  const int N = (int)g.N, K = (int)g.K;
  const int ncol = min(COLS, N - j0);
  const int kend = g.b_upper ? min(K, j0 + COLS) : K;
  const int64_t i = rb * TS_ROWS + t;
  const bool row_ok = i < g.M;
  const int64_t lda = g.sa_k, ldb = g.ldb;
  const float* __restrict__ a0 = static_cast<const float*>(g.a[0]) + i;
  const float* __restrict__ a1 = static_cast<const float*>(g.a[1]) + i;
  const float* __restrict__ a2 = static_cast<const float*>(g.a[2]) + i;
  const float* __restrict__ a3 = static_cast<const float*>(g.a[3]) + i;
  const float* b0 = static_cast<const float*>(g.b[0]);
  const float* b1 = static_cast<const float*>(g.b[1]);
  const float* b2 = static_cast<const float*>(g.b[2]);
  const float* b3 = static_cast<const float*>(g.b[3]);
  Quat<float> acc[COLS];
#pragma unroll
  for (int jj = 0; jj < COLS; ++jj) acc[jj] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < kend; k0 += TS_KC) {
    const int kn = min(TS_KC, kend - k0);
    __syncthreads();
    for (int e = t; e < kn * COLS; e += TS_ROWS) {
      const int kk = e % kn, jj = e / kn;   // consecutive threads: consecutive rows of one column
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (jj < ncol) {
        const int64_t o = (int64_t)(k0 + kk) + (int64_t)(j0 + jj) * ldb;
        v = make_float4(b0[o], b1[o], b2[o], b3[o]);
      }
      Bs[kk][jj] = v;
    }
    __syncthreads();
    if (row_ok) {
      // software pipeline: the loads of the next U rows are issued before the multiply-adds of
      // the current ones
      constexpr int U = (COLS > 8) ? 2 : 4;   // rows k per batch of loads (register budget)
      const int kfull = kn / U * U;
      Quat<float> cur[U], nxt[U];
      auto load = [&](Quat<float>* a, int kb) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t o = (int64_t)(k0 + kb + u) * lda;
          a[u] = {a0[o], a1[o], a2[o], a3[o]};
        }
      };
      if (kfull > 0) load(cur, 0);
      for (int kk = 0; kk < kfull; kk += U) {
        if (kk + U < kfull) load(nxt, kk + U);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int jj = 0; jj < COLS; ++jj) qfma(acc[jj], cur[u], Bs[kk + u][jj]);
#pragma unroll
        for (int u = 0; u < U; ++u) cur[u] = nxt[u];
      }
      for (int kk = kfull; kk < kn; ++kk) {
        const int64_t o = (int64_t)(k0 + kk) * lda;
        const Quat<float> a = {a0[o], a1[o], a2[o], a3[o]};
#pragma unroll
        for (int jj = 0; jj < COLS; ++jj) qfma(acc[jj], a, Bs[kk][jj]);
      }
    }
  }
  if (!row_ok) return;
  float* c0 = static_cast<float*>(g.c[0]) + i;
  float* c1 = static_cast<float*>(g.c[1]) + i;
  float* c2 = static_cast<float*>(g.c[2]) + i;
  float* c3 = static_cast<float*>(g.c[3]) + i;
#pragma unroll
  for (int jj = 0; jj < COLS; ++jj)
    if (jj < ncol) {
      const int64_t o = (int64_t)(j0 + jj) * g.ldc;
      c0[o] = acc[jj].w; c1[o] = acc[jj].x; c2[o] = acc[jj].y; c3[o] = acc[jj].z;
    }
}

__global__ void __launch_bounds__(TS_ROWS) thin_small_kernel(GemmArgs g) {
  thin_small_tile<TS_COLS1>(g, blockIdx.x, blockIdx.y);
}

// Many independent products in one launch (batch plans): item (problem, row block, column chunk).
__global__ void __launch_bounds__(TS_ROWS, 4) thin_small_grouped_kernel(const GemmArgs* __restrict__ args,
                                                                    const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  thin_small_tile<TS_COLS>(args[it.x], it.y, it.z);
}
}  // namespace

void thin_small_items(int64_t M, int64_t N, int prob, std::vector<int4>& items) {
  for (int64_t c = 0; c < (N + TS_COLS - 1) / TS_COLS; ++c)
    for (int64_t r = 0; r < (M + TS_ROWS - 1) / TS_ROWS; ++r) items.push_back(make_int4(prob, (int)r, (int)c, 0));
}

int thin_small_grouped(qlr_ctx* ctx, const GemmArgs* d_args, const int4* d_items, int nitems) {
  if (nitems <= 0) return QLR_OK;
  KTimer kt(ctx, QLR_KID_APPLY);
  thin_small_grouped_kernel<<<nitems, TS_ROWS, 0, ctx->stream>>>(d_args, d_items);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

int thin_times_small(qlr_ctx* ctx, const qlr_qmat& T, const double* S, int l, int k, qlr_qmat& C, WsArena& ws,
                     bool S_upper) {
  // FP32 products: the small factor goes to FP32 once (every CTA of the GEMM would otherwise
  // convert its FP64 tile of S again, on the slow FP64 pipe)
  const bool f32 = (T.dtype != QLR_F64 && C.dtype != QLR_F64);
  const size_t mark = ws.off;
  float* s32 = f32 ? ws.take<float>((size_t)4 * l * k) : nullptr;
  if (s32) {
    const int64_t n = (int64_t)4 * l * k;
    KTimer kt(ctx, QLR_KID_MISC);
    small_to_f32_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, ctx->stream>>>(S, s32, n);
    qlr_count_launch();
    QLR_CUDA_TRY(cudaGetLastError());
  } else {
    ws.ok = true;
  }
  GemmArgs g{};
  for (int c = 0; c < 4; ++c) {
    g.a[c] = T.plane[c];
    g.b[c] = s32 ? static_cast<const void*>(s32 + (size_t)c * l * k) : static_cast<const void*>(S + (size_t)c * l * k);
    g.c[c] = C.plane[c];
  }
  g.sa_i = 1; g.sa_k = T.ld; g.a_dtype = T.dtype; g.conj_a = false; g.i_contig = true;
  g.ldb = l; g.b_dtype = s32 ? QLR_F32 : QLR_F64;
  g.ldc = C.ld; g.c_dtype = C.dtype;
  g.M = T.rows; g.N = k; g.K = l;
  g.alpha = 1.0; g.beta = 0.0;
  g.acc64 = (T.dtype == QLR_F64 || C.dtype == QLR_F64);
  g.b_upper = S_upper;
  int rc = QLR_OK;
  if (f32 && T.dtype == QLR_F32 && C.dtype == QLR_F32 && T.plane[0] != nullptr && T.rows > 0 && k > 0) {
    KTimer kt(ctx, g.kid);
    const dim3 grid((unsigned)((T.rows + TS_ROWS - 1) / TS_ROWS), (unsigned)((k + TS_COLS1 - 1) / TS_COLS1));
    thin_small_kernel<<<grid, TS_ROWS, 0, ctx->stream>>>(g);
    qlr_count_launch();
    rc = (cudaGetLastError() == cudaSuccess) ? QLR_OK : QLR_ECUDA;
  } else {
    rc = gemm_simt(ctx, g);
  }
  ws.off = mark;
  return rc;
}

}  // namespace qlr
