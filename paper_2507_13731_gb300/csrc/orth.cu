// Orthonormalisation of thin quaternion sketches: the "QR" step after every pass of
// Algorithms 1-4 (Def. 1, eq. QQR).  CholeskyQR2: G = Y^H Y (FP64), R1 = chol(G) (FP64),
// Q' = Y R1^{-1}, then once more on Q'; R = R2 R1.  Shifted CholeskyQR3 (Fukaya, Kannan,
// Nakatsukasa, Zhang and Yamamoto, SISC 2020) adds s I to the first Gram matrix so the
// Cholesky factorisation exists for ill-conditioned input (Algorithm 4's stacked basis).
#include "qlr_internal.h"

namespace {

// ---------------------------------------------------------------------------------------
// Gram partial sums: part[chunk] = sum over the chunk's rows r of conj(y_ri) y_rj, for tiles
// (ti <= tj) of the upper triangle.  32 x 32 quaternion tiles, 256 threads, 2 x 2 per thread.
constexpr int GT = 32, GR = 16;

template <class TY>
__global__ void __launch_bounds__(256) gram_partial_kernel(const TY* __restrict__ y0, const TY* __restrict__ y1,
                                                           const TY* __restrict__ y2, const TY* __restrict__ y3,
                                                           int64_t m, int l, int64_t ld, int64_t rows_per_chunk,
                                                           const int2* __restrict__ tiles, double* __restrict__ part) {
  __shared__ double Yi[4][GR][GT + 1];
  __shared__ double Yj[4][GR][GT + 1];
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int2 tile = tiles[blockIdx.x];
  const int i0 = tile.x * GT, j0 = tile.y * GT;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r_end = min(m, r_begin + rows_per_chunk);
  const TY* yp[4] = {y0, y1, y2, y3};
  Quat<double> acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = {0, 0, 0, 0};

  for (int64_t r0 = r_begin; r0 < r_end; r0 += GR) {
    // load GR rows x GT columns for both column blocks: thread t -> (row t%16, col t/16 (+16))
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int rr = t % GR, cc = t / GR + 16 * h;
        int64_t gr = r0 + rr;
        double vi = 0.0, vj = 0.0;
        if (gr < r_end) {
          if (i0 + cc < l) vi = to_d(yp[c][gr + (int64_t)(i0 + cc) * ld]);
          if (j0 + cc < l) vj = to_d(yp[c][gr + (int64_t)(j0 + cc) * ld]);
        }
        Yi[c][rr][cc] = vi;
        Yj[c][rr][cc] = vj;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < GR; ++rr) {
      Quat<double> a[2], b[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int ci = tx + 16 * h, cj = ty + 16 * h;
        a[h] = {Yi[0][rr][ci], Yi[1][rr][ci], Yi[2][rr][ci], Yi[3][rr][ci]};
        b[h] = {Yj[0][rr][cj], Yj[1][rr][cj], Yj[2][rr][cj], Yj[3][rr][cj]};
      }
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int z = 0; z < 2; ++z) {
          Quat<double> p = qcmul(a[x], b[z]);
          acc[x][z].w += p.w; acc[x][z].x += p.x; acc[x][z].y += p.y; acc[x][z].z += p.z;
        }
    }
    __syncthreads();
  }
  double* P = part + (size_t)blockIdx.y * 4 * l * l;
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int z = 0; z < 2; ++z) {
      int i = i0 + tx + 16 * x, j = j0 + ty + 16 * z;
      if (i < l && j < l) st_small(P, l, i, j, acc[x][z]);
    }
}

// Sum the chunk partials in a fixed order; write the full Hermitian matrix.
__global__ void gram_reduce_kernel(const double* __restrict__ part, int nchunks, int l, double* __restrict__ G) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)l * l) return;
  int i = (int)(idx % l), j = (int)(idx / l);
  if (i > j) return;
  Quat<double> s = {0, 0, 0, 0};
  for (int c = 0; c < nchunks; ++c) {
    Quat<double> q = ld_small(part + (size_t)c * 4 * l * l, l, i, j);
    s.w += q.w; s.x += q.x; s.y += q.y; s.z += q.z;
  }
  if (i == j) { s.x = s.y = s.z = 0.0; }
  st_small(G, l, i, j, s);
  if (i != j) st_small(G, l, j, i, {s.w, -s.x, -s.y, -s.z});
}

// ---------------------------------------------------------------------------------------
// Right-looking quaternion Cholesky G = R^H R in FP64, one CTA.  R is worked in place (upper
// triangle).  shift_coef > 0 adds shift_coef * trace(G) to the diagonal first (shifted CholQR).
__global__ void __launch_bounds__(1024) chol_kernel(const double* __restrict__ G, double* __restrict__ R, int l,
                                                     double shift_coef, int* err) {
  __shared__ double s_piv, s_shift;
  const int t = threadIdx.x, nt = blockDim.x;
  const size_t ll = (size_t)l * l;
  if (t == 0) {
    double tr = 0.0;
    for (int i = 0; i < l; ++i) tr += G[(size_t)i * l + i];
    s_shift = shift_coef * tr;
  }
  for (size_t e = t; e < ll; e += nt) {
    int i = (int)(e % l), j = (int)(e / l);
    for (int c = 0; c < 4; ++c) R[c * ll + e] = (i <= j) ? G[c * ll + e] : 0.0;
  }
  __syncthreads();
  for (int i = t; i < l; i += nt) R[(size_t)i * l + i] += s_shift;
  __syncthreads();
  double maxdiag = 0.0;
  for (int i = 0; i < l; ++i) maxdiag = fmax(maxdiag, R[(size_t)i * l + i]);
  for (int j = 0; j < l; ++j) {
    if (t == 0) {
      double d2 = R[(size_t)j * l + j];
      if (!(d2 > 0.0)) {
        qlr_set_error(err, QLR_ENOTPD);
        d2 = fmax(maxdiag, 1.0) * 1e-300;
      }
      double d = sqrt(d2);
      s_piv = d;
      R[(size_t)j * l + j] = d;
      R[ll + (size_t)j * l + j] = 0.0;
      R[2 * ll + (size_t)j * l + j] = 0.0;
      R[3 * ll + (size_t)j * l + j] = 0.0;
    }
    __syncthreads();
    const double inv = 1.0 / s_piv;
    for (int k = j + 1 + t; k < l; k += nt) {
      size_t o = (size_t)k * l + j;
      for (int c = 0; c < 4; ++c) R[c * ll + o] *= inv;
    }
    __syncthreads();
    // trailing update of the upper triangle: R[i][k] -= conj(R[j][i]) R[j][k], j < i <= k
    const int rem = l - j - 1;
    const int64_t npairs = (int64_t)rem * (rem + 1) / 2;
    for (int64_t p = t; p < npairs; p += nt) {
      // map p -> (ii, kk) with 0 <= ii <= kk < rem, column-major over the upper triangle
      int kk = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
      while ((int64_t)kk * (kk + 1) / 2 > p) --kk;
      while ((int64_t)(kk + 1) * (kk + 2) / 2 <= p) ++kk;
      int ii = (int)(p - (int64_t)kk * (kk + 1) / 2);
      int i = j + 1 + ii, k = j + 1 + kk;
      Quat<double> a = ld_small(R, l, j, i), b = ld_small(R, l, j, k), r = ld_small(R, l, i, k);
      Quat<double> pr = qcmul(a, b);
      r.w -= pr.w; r.x -= pr.x; r.y -= pr.y; r.z -= pr.z;
      st_small(R, l, i, k, r);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Inverse of an upper-triangular quaternion matrix with real diagonal: one warp per column,
// back substitution x_i = -(sum_{t=i+1..j} R_it x_t) / R_ii.
constexpr int TI_WARPS = 4, TI_MAXL = 512;

__global__ void __launch_bounds__(32 * TI_WARPS) tri_inv_kernel(const double* __restrict__ R, double* __restrict__ X, int l) {
  extern __shared__ double sx[];  // TI_WARPS * 4 * l
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int j = blockIdx.x * TI_WARPS + warp;
  if (j >= l) return;
  double* x = sx + (size_t)warp * 4 * l;
  for (int i = lane; i < l; i += 32) x[i] = x[l + i] = x[2 * l + i] = x[3 * l + i] = 0.0;
  __syncwarp();
  if (lane == 0) x[j] = 1.0 / R[(size_t)j * l + j];
  __syncwarp();
  for (int i = j - 1; i >= 0; --i) {
    Quat<double> s = {0, 0, 0, 0};
    for (int t = i + 1 + lane; t <= j; t += 32) {
      Quat<double> p = qmul(ld_small(R, l, i, t), Quat<double>{x[t], x[l + t], x[2 * l + t], x[3 * l + t]});
      s.w += p.w; s.x += p.x; s.y += p.y; s.z += p.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s.w += __shfl_xor_sync(0xffffffffu, s.w, o);
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      s.z += __shfl_xor_sync(0xffffffffu, s.z, o);
    }
    if (lane == 0) {
      double inv = -1.0 / R[(size_t)i * l + i];
      x[i] = s.w * inv; x[l + i] = s.x * inv; x[2 * l + i] = s.y * inv; x[3 * l + i] = s.z * inv;
    }
    __syncwarp();
  }
  const size_t ll = (size_t)l * l;
  for (int i = lane; i < l; i += 32)
    for (int c = 0; c < 4; ++c) X[c * ll + (size_t)j * l + i] = x[(size_t)c * l + i];
}

// C = A B for small l x l quaternion matrices (FP64), A and B upper triangular.
__global__ void small_matmul_kernel(const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C,
                                    int l) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)l * l) return;
  int i = (int)(idx % l), j = (int)(idx / l);
  Quat<double> s = {0, 0, 0, 0};
  for (int t = i; t <= j; ++t) {
    Quat<double> p = qmul(ld_small(A, l, i, t), ld_small(B, l, t, j));
    s.w += p.w; s.x += p.x; s.y += p.y; s.z += p.z;
  }
  st_small(C, l, i, j, s);
}

}  // namespace

namespace qlr {

int gram(qlr_ctx* ctx, const qlr_qmat& Y, double* G, WsArena& ws) {
  const int l = (int)Y.cols;
  const int64_t m = Y.rows;
  if (l == 0) return QLR_OK;
  const int nt = (l + GT - 1) / GT;
  std::vector<int2> tiles;
  for (int b = 0; b < nt; ++b)
    for (int a = 0; a <= b; ++a) tiles.push_back(make_int2(a, b));
  int target = 2 * (ctx->num_sms > 0 ? ctx->num_sms : 148);
  int64_t chunks = (target + (int64_t)tiles.size() - 1) / (int64_t)tiles.size();
  chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, (m + 63) / 64));
  chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, ((int64_t)64 << 20) / ((int64_t)32 * l * l)));
  int64_t rpc = ((m + chunks - 1) / chunks + GR - 1) / GR * GR;
  if (rpc == 0) rpc = GR;
  chunks = (m + rpc - 1) / rpc;
  if (chunks == 0) chunks = 1;
  size_t mark = ws.off;
  int2* d_tiles = ws.take<int2>(tiles.size());
  double* part = ws.take<double>((size_t)chunks * 4 * l * l);
  if (!ws.ok) return QLR_ENOMEM;
  QLR_CUDA_TRY(cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, ctx->stream));
  dim3 grid((unsigned)tiles.size(), (unsigned)chunks);
  KTimer kt(ctx, QLR_KID_GRAM);
  if (Y.dtype == QLR_F64) {
    const double* p[4];
    for (int c = 0; c < 4; ++c) p[c] = static_cast<const double*>(Y.plane[c]);
    gram_partial_kernel<double><<<grid, 256, 0, ctx->stream>>>(p[0], p[1], p[2], p[3], m, l, Y.ld, rpc, d_tiles, part);
  } else if (Y.dtype == QLR_F32) {
    const float* p[4];
    for (int c = 0; c < 4; ++c) p[c] = static_cast<const float*>(Y.plane[c]);
    gram_partial_kernel<float><<<grid, 256, 0, ctx->stream>>>(p[0], p[1], p[2], p[3], m, l, Y.ld, rpc, d_tiles, part);
  } else {
    return QLR_EINVAL;
  }
  QLR_CUDA_TRY(cudaGetLastError());
  int64_t tot = (int64_t)l * l;
  gram_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(part, (int)chunks, l, G);
  QLR_CUDA_TRY(cudaGetLastError());
  ws.off = mark;  // partials are dead once the reduction is enqueued (stream order)
  return QLR_OK;
}

int chol(qlr_ctx* ctx, int l, const double* G, double* R, double shift_coef) {
  if (l == 0) return QLR_OK;
  KTimer kt(ctx, QLR_KID_CHOL);
  chol_kernel<<<1, 1024, 0, ctx->stream>>>(G, R, l, shift_coef, ctx->d_err);
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

int tri_inv(qlr_ctx* ctx, int l, const double* R, double* Rinv) {
  if (l == 0) return QLR_OK;
  if (l > TI_MAXL) return QLR_EUNSUPPORTED;
  size_t smem = (size_t)TI_WARPS * 4 * l * sizeof(double);
  if (smem > 48 * 1024) QLR_CUDA_TRY(cudaFuncSetAttribute(tri_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  KTimer kt(ctx, QLR_KID_TRIINV);
  tri_inv_kernel<<<(l + TI_WARPS - 1) / TI_WARPS, 32 * TI_WARPS, smem, ctx->stream>>>(R, Rinv, l);
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

int small_matmul(qlr_ctx* ctx, int l, const double* A, const double* B, double* C) {
  int64_t tot = (int64_t)l * l;
  KTimer kt(ctx, QLR_KID_MISC);
  small_matmul_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, ctx->stream>>>(A, B, C, l);
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

// Q = Y * Rinv (Rinv FP64 small, column-major, l x l)
static int apply_rinv(qlr_ctx* ctx, const qlr_qmat& Y, const double* Rinv, qlr_qmat& Q) {
  GemmArgs g{};
  for (int c = 0; c < 4; ++c) {
    g.a[c] = Y.plane[c];
    g.b[c] = Rinv + (size_t)c * Y.cols * Y.cols;
    g.c[c] = Q.plane[c];
  }
  g.sa_i = 1; g.sa_k = Y.ld; g.a_dtype = Y.dtype; g.conj_a = false; g.i_contig = true;
  g.ldb = Y.cols; g.b_dtype = QLR_F64;
  g.ldc = Q.ld; g.c_dtype = Q.dtype;
  g.M = Y.rows; g.N = Y.cols; g.K = Y.cols;
  g.alpha = 1.0; g.beta = 0.0;
  g.acc64 = (Y.dtype == QLR_F64);
  return gemm_simt(ctx, g);
}

int cholqr(qlr_ctx* ctx, const qlr_qmat& Y, qlr_qmat& Q, double* R, int orth, WsArena& ws) {
  const int l = (int)Y.cols;
  const int64_t m = Y.rows;
  if (l == 0 || m == 0) return QLR_OK;
  const size_t ll4 = (size_t)4 * l * l;
  const size_t esz = qlr_dtype_size(Y.dtype);
  size_t mark = ws.off;
  double* G = ws.take<double>(ll4);
  double* Rs = ws.take<double>(ll4);
  double* P1 = ws.take<double>(ll4);
  double* P2 = ws.take<double>(ll4);
  double* Rinv = ws.take<double>(ll4);
  char* tbuf = ws.take<char>((size_t)4 * m * l * esz);
  if (!ws.ok) return QLR_ENOMEM;
  qlr_qmat T = Y;
  T.ld = m;
  T.layout = QLR_COL_MAJOR;
  for (int c = 0; c < 4; ++c) T.plane[c] = tbuf + (size_t)c * m * l * esz;

  // CholeskyQR2: Y -> T -> Q.  Shifted CholeskyQR3: Y -> Q -> T -> Q.
  const int steps = (orth == QLR_ORTH_SCHOLQR3) ? 3 : 2;
  const qlr_qmat* seq2[3] = {&Y, &T, &Q};
  const qlr_qmat* seq3[4] = {&Y, &Q, &T, &Q};
  const qlr_qmat* const* seq = (steps == 3) ? seq3 : seq2;
  // shift s = 11 (m l + l (l + 1)) u ||Y||_2^2 with u = 2^-53 (FP64 Gram and Cholesky);
  // ||Y||_2^2 is bounded by trace(G), which the Cholesky kernel multiplies in.
  const double shift = (orth == QLR_ORTH_SCHOLQR3) ? 11.0 * ((double)m * l + (double)l * (l + 1)) * 1.1102230246251565e-16 : 0.0;
  double* Rprod = P1;
  double* Rnext = P2;
  for (int s = 0; s < steps; ++s) {
    const qlr_qmat& src = *seq[s];
    qlr_qmat& dst = const_cast<qlr_qmat&>(*seq[s + 1]);
    double* Rcur = (s == 0) ? Rprod : Rs;
    QLR_TRY(gram(ctx, src, G, ws));
    QLR_TRY(chol(ctx, l, G, Rcur, (s == 0) ? shift : 0.0));
    QLR_TRY(tri_inv(ctx, l, Rcur, Rinv));
    QLR_TRY(apply_rinv(ctx, src, Rinv, dst));
    if (s > 0) {   // R_total <- R_s * R_total
      QLR_TRY(small_matmul(ctx, l, Rs, Rprod, Rnext));
      double* sw = Rprod; Rprod = Rnext; Rnext = sw;
    }
  }
  if (R) QLR_CUDA_TRY(cudaMemcpyAsync(R, Rprod, ll4 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  ws.off = mark;
  return QLR_OK;
}

}  // namespace qlr
