// Thin x small products C = T S: T (rows x l) a tall quaternion basis stored column-major, S a
// small FP64 l x k factor (R^{-1} of a CholeskyQR step, or the core QSVD's singular vectors for
// the lifts U = Q1 U_hat, V = Q2 V_hat), on the SIMT kernel (FP32, FP64 for FP64 operands).  The
// tensor-core sketch kernel was measured on this shape (4096 x 110 x 110) and gained nothing:
// with K = l its CTAs run a dozen pipeline stages each and the 3xTF32 split costs three MMAs.
#include <algorithm>

#include "qlr_internal.h"

namespace qlr {

namespace {
__global__ void small_to_f32_kernel(const double* __restrict__ S, float* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)S[e];
}
}  // namespace

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
  const int rc = gemm_simt(ctx, g);
  ws.off = mark;
  return rc;
}

}  // namespace qlr
