// Quaternion matrix completion (Section 7): the masked update of eq. Step2,
//   C = mask .* M + (1 - mask) .* X,   X = U diag(S) V^H (the rank-k approximation of eq. Step1),
// as one kernel: every CTA forms its tile of X in registers from U diag(S) and V staged in shared
// memory, then stores M's value at observed entries and X's elsewhere -- X is never written out.
// k = 0 gives the starting point P_Omega(M).
#include <algorithm>

#include "qlr_internal.h"

namespace qlr {

namespace {

// A quaternion with the alignment of its four components, so shared-memory reads are one
// vector load (16 bytes in FP32).
template <class T>
struct alignas(4 * sizeof(T)) QV {
  Quat<T> q;
};

// Tile TM x TN of C per CTA of 256 threads: thread (ty, tx) owns column j0 + tx and rows
// i0 + ty + 4 s, s < 8, so each row of the tile is written by 64 consecutive threads (coalesced
// row-major stores).  U diag(S) and V come through shared memory KC rank columns at a time.
constexpr int CM_TM = 32, CM_TN = 64, CM_THREADS = 256;
constexpr int CM_ROWSTEP = CM_THREADS / CM_TN;    // 4
constexpr int CM_RPT = CM_TM / CM_ROWSTEP;        // 8 rows per thread

template <class T>
__global__ void __launch_bounds__(CM_THREADS) complete_update_kernel(CompleteArgs a) {
  constexpr int KC = (sizeof(T) == 4) ? 16 : 8;
  __shared__ QV<T> Us[KC][CM_TM];
  __shared__ QV<T> Vs[KC][CM_TN];
  const int t = threadIdx.x, tx = t % CM_TN, ty = t / CM_TN;
  const int64_t i0 = (int64_t)blockIdx.y * CM_TM, j0 = (int64_t)blockIdx.x * CM_TN;
  const T* u[4];
  const T* v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    u[c] = static_cast<const T*>(a.U[c]);
    v[c] = static_cast<const T*>(a.V[c]);
  }
  Quat<T> acc[CM_RPT];
#pragma unroll
  for (int s = 0; s < CM_RPT; ++s) acc[s] = {0, 0, 0, 0};
  for (int r0 = 0; r0 < a.k; r0 += KC) {
    for (int e = t; e < KC * CM_TM; e += CM_THREADS) {   // U(i, r) s_r, column-major U
      const int ii = e % CM_TM, rr = e / CM_TM;
      const int64_t i = i0 + ii;
      const int r = r0 + rr;
      Quat<T> q = {0, 0, 0, 0};
      if (i < a.m && r < a.k) {
        const size_t o = (size_t)r * a.ldu + i;
        const T s = (T)a.S[r];
        q = {u[0][o] * s, u[1][o] * s, u[2][o] * s, u[3][o] * s};
      }
      Us[rr][ii].q = q;
    }
    for (int e = t; e < KC * CM_TN; e += CM_THREADS) {   // V(j, r), column-major V
      const int jj = e % CM_TN, rr = e / CM_TN;
      const int64_t j = j0 + jj;
      const int r = r0 + rr;
      Quat<T> q = {0, 0, 0, 0};
      if (j < a.n && r < a.k) {
        const size_t o = (size_t)r * a.ldv + j;
        q = {v[0][o], v[1][o], v[2][o], v[3][o]};
      }
      Vs[rr][jj].q = q;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < KC; ++rr) {
      const Quat<T> vq = Vs[rr][tx].q;
#pragma unroll
      for (int s = 0; s < CM_RPT; ++s) {
        const Quat<T> p = qmulc(Us[rr][ty + s * CM_ROWSTEP].q, vq);   // (U_ir s_r) conj(V_jr)
        acc[s].w += p.w; acc[s].x += p.x; acc[s].y += p.y; acc[s].z += p.z;
      }
    }
    __syncthreads();
  }
  const int64_t j = j0 + tx;
  if (j >= a.n) return;
  const T* m[4];
  T* cp[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    m[c] = static_cast<const T*>(a.M[c]);
    cp[c] = static_cast<T*>(a.C[c]);
  }
#pragma unroll
  for (int s = 0; s < CM_RPT; ++s) {
    const int64_t i = i0 + ty + s * CM_ROWSTEP;
    if (i >= a.m) break;
    const size_t oc = (size_t)i * a.ldc + j;
    if (a.mask[(size_t)i * a.ldk + j] != 0) {             // observed: M's entry
      const size_t om = (size_t)i * a.ldm + j;
      cp[0][oc] = m[0] ? m[0][om] : (T)0;
      cp[1][oc] = m[1][om];
      cp[2][oc] = m[2][om];
      cp[3][oc] = m[3][om];
    } else {                                              // unobserved: the low-rank value
      cp[0][oc] = acc[s].w;
      cp[1][oc] = acc[s].x;
      cp[2][oc] = acc[s].y;
      cp[3][oc] = acc[s].z;
    }
  }
}

}  // namespace

int complete_update(qlr_ctx* ctx, const CompleteArgs& a, int dtype) {
  if (a.m == 0 || a.n == 0) return QLR_OK;
  const int64_t gy = (a.m + CM_TM - 1) / CM_TM, gx = (a.n + CM_TN - 1) / CM_TN;
  if (gy > 65535 || gx > 0x7fffffff) return QLR_EUNSUPPORTED;
  KTimer kt(ctx, QLR_KID_COMPLETE);
  const dim3 grid((unsigned)gx, (unsigned)gy);
  if (dtype == QLR_F64) complete_update_kernel<double><<<grid, CM_THREADS, 0, ctx->stream>>>(a);
  else complete_update_kernel<float><<<grid, CM_THREADS, 0, ctx->stream>>>(a);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

}  // namespace qlr
