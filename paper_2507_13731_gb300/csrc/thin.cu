// Thin x small products C = T S: T (rows x l) a tall quaternion basis stored column-major, S a
// small FP64 l x k factor (R^{-1} of a CholeskyQR step, or the core QSVD's singular vectors for
// the lifts U = Q1 U_hat, V = Q2 V_hat), on the SIMT kernel (FP32, FP64 for FP64 operands).  The
// tensor-core sketch kernel was measured on this shape (4096 x 110 x 110) and gained nothing:
// with K = l its CTAs run a dozen pipeline stages each and the 3xTF32 split costs three MMAs.
#include "qlr_internal.h"

namespace qlr {

int thin_times_small(qlr_ctx* ctx, const qlr_qmat& T, const double* S, int l, int k, qlr_qmat& C, WsArena& ws) {
  (void)ws;
  GemmArgs g{};
  for (int c = 0; c < 4; ++c) {
    g.a[c] = T.plane[c];
    g.b[c] = S + (size_t)c * l * k;
    g.c[c] = C.plane[c];
  }
  g.sa_i = 1; g.sa_k = T.ld; g.a_dtype = T.dtype; g.conj_a = false; g.i_contig = true;
  g.ldb = l; g.b_dtype = QLR_F64;
  g.ldc = C.ld; g.c_dtype = C.dtype;
  g.M = T.rows; g.N = k; g.K = l;
  g.alpha = 1.0; g.beta = 0.0;
  g.acc64 = (T.dtype == QLR_F64 || C.dtype == QLR_F64);
  return gemm_simt(ctx, g);
}

}  // namespace qlr
