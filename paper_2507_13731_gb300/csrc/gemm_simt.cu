// SIMT (CUDA-core) quaternion GEMM:  C = alpha * op(A) * B + beta * C.
//
// Used for (i) the plain FP32 / FP64 sketch passes Y = A X and Z = A^H Y (the comparator path
// and the FP64 mode), and (ii) thin-times-small products Q = Y R^{-1}, U = Q1 U_hat, V = Q2 V_hat.
// Each output entry is a sum of Hamilton products (Section 2, eq. 1); op(A) = A or conj(A)
// elementwise, with A's (i, k) addressing given by two strides so that A, A^T-views and
// column-major thin matrices all use the same kernel.
#include "qlr_internal.h"

namespace {

constexpr int BM = 64, BN = 32, BK = 16, NT = 256;

template <class TAcc>
__device__ __forceinline__ TAcc load_elem(const void* p, int64_t idx, int dt) {
  if (dt == QLR_F64) return (TAcc)static_cast<const double*>(p)[idx];
  if (dt == QLR_F32) return (TAcc)static_cast<const float*>(p)[idx];
  return (TAcc)__bfloat162float(static_cast<const __nv_bfloat16*>(p)[idx]);
}

// One BM x BN output tile (row tile bx, column tile by) of C.
template <class TAcc, bool I_CONTIG, bool CONJ>
__device__ __forceinline__ void gemm_simt_tile(const qlr::GemmArgs& g, int64_t bx, int64_t by) {
  // one element of padding for 4-byte types (bank conflicts); none for doubles (48 KB static limit)
  constexpr int PAD = sizeof(TAcc) == 4 ? 1 : 0;
  __shared__ TAcc As[4][BK][BM + PAD];
  __shared__ TAcc Bs[4][BK][BN + PAD];
  const int t = threadIdx.x;
  const int tx = t % 16, ty = t / 16;
  const int64_t i0 = bx * BM, j0 = by * BN;

  Quat<TAcc> acc[4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 2; ++s) acc[r][s] = {0, 0, 0, 0};

  TAcc ra[4][4], rb[4][2];
  auto load_tile = [&](int64_t k0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int ii, kk;
        if (I_CONTIG) { ii = t % BM; kk = t / BM + 4 * r; }
        else { kk = t % BK; ii = t / BK + 16 * r; }
        int64_t gi = i0 + ii, gk = k0 + kk;
        TAcc v = 0;
        if (g.a[c] != nullptr && gi < g.M && gk < g.K) v = load_elem<TAcc>(g.a[c], gi * g.sa_i + gk * g.sa_k, g.a_dtype);
        ra[c][r] = v;
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        int kk = t % BK, jj = t / BK + 16 * r;
        int64_t gk = k0 + kk, gj = j0 + jj;
        TAcc v = 0;
        if (gk < g.K && gj < g.N) v = load_elem<TAcc>(g.b[c], gk + gj * g.ldb, g.b_dtype);
        rb[c][r] = v;
      }
    }
  };
  auto store_tile = [&]() {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int ii, kk;
        if (I_CONTIG) { ii = t % BM; kk = t / BM + 4 * r; }
        else { kk = t % BK; ii = t / BK + 16 * r; }
        As[c][kk][ii] = ra[c][r];
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        int kk = t % BK, jj = t / BK + 16 * r;
        Bs[c][kk][jj] = rb[c][r];
      }
    }
  };

  // rows of an upper-triangular B below the column tile's last column are zero
  const int64_t kend = g.b_upper ? min(g.K, j0 + BN) : g.K;
  load_tile(0);
  for (int64_t k0 = 0; k0 < kend; k0 += BK) {
    store_tile();
    __syncthreads();
    if (k0 + BK < kend) load_tile(k0 + BK);   // prefetch next tile into registers
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      Quat<TAcc> a[4], b[2];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int ii = tx + 16 * r;
        a[r] = {As[0][kk][ii], As[1][kk][ii], As[2][kk][ii], As[3][kk][ii]};
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        int jj = 2 * ty + s;
        b[s] = {Bs[0][kk][jj], Bs[1][kk][jj], Bs[2][kk][jj], Bs[3][kk][jj]};
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          Quat<TAcc> p = CONJ ? qcmul(a[r], b[s]) : qmul(a[r], b[s]);
          acc[r][s].w += p.w; acc[r][s].x += p.x; acc[r][s].y += p.y; acc[r][s].z += p.z;
        }
    }
    __syncthreads();
  }

  const TAcc alpha = (TAcc)g.alpha, beta = (TAcc)g.beta;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      int64_t gi = i0 + tx + 16 * r, gj = j0 + 2 * ty + s;
      if (gi >= g.M || gj >= g.N) continue;
      TAcc v[4] = {acc[r][s].w, acc[r][s].x, acc[r][s].y, acc[r][s].z};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        int64_t o = gi + gj * g.ldc;
        TAcc out = alpha * v[c];
        if (g.c_dtype == QLR_F64) {
          double* C = static_cast<double*>(g.c[c]);
          C[o] = (g.beta != 0.0) ? (double)out + g.beta * C[o] : (double)out;
        } else {
          float* C = static_cast<float*>(g.c[c]);
          C[o] = (g.beta != 0.0) ? (float)out + (float)beta * C[o] : (float)out;
        }
      }
    }
}

template <class TAcc, bool I_CONTIG, bool CONJ>
__global__ void __launch_bounds__(NT) gemm_simt_kernel(qlr::GemmArgs g) {
  gemm_simt_tile<TAcc, I_CONTIG, CONJ>(g, blockIdx.x, blockIdx.y);
}

template <class TAcc>
void launch(const qlr::GemmArgs& g, cudaStream_t s) {
  dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + BN - 1) / BN));
  if (g.i_contig) {
    if (g.conj_a) gemm_simt_kernel<TAcc, true, true><<<grid, NT, 0, s>>>(g);
    else gemm_simt_kernel<TAcc, true, false><<<grid, NT, 0, s>>>(g);
  } else {
    if (g.conj_a) gemm_simt_kernel<TAcc, false, true><<<grid, NT, 0, s>>>(g);
    else gemm_simt_kernel<TAcc, false, false><<<grid, NT, 0, s>>>(g);
  }
  qlr_count_launch();
}

}  // namespace

namespace qlr {
int gemm_simt(qlr_ctx* ctx, const GemmArgs& g) {
  if (g.M == 0 || g.N == 0) return QLR_OK;
  if (g.N > 65535LL * BN || g.M > (int64_t)INT32_MAX * BM) return QLR_EUNSUPPORTED;
  KTimer kt(ctx, g.kid);
  if (g.acc64) launch<double>(g, ctx->stream);
  else launch<float>(g, ctx->stream);
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}
}  // namespace qlr
