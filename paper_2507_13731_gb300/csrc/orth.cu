// Orthonormalisation of thin quaternion sketches: the "QR" step after every pass of
// Algorithms 1-4 (Def. 1, eq. QQR).  CholeskyQR2: G = Y^H Y and R1 = chol(G) in FP64-class
// arithmetic (FP64 for FP64 sketches; for FP32 sketches the tensor-core Gram of gram_tc.cu and a
// double-FP32 Cholesky and triangular inverse), Q' = Y R1^{-1}, then once more on Q' (where Q'^H Q'
// is close to I, the second factor and its inverse come from a series); R = R2 R1.  Shifted CholeskyQR3 (Fukaya, Kannan,
// Nakatsukasa, Zhang and Yamamoto, SISC 2020) adds s I to the first Gram matrix so the
// Cholesky factorisation exists for ill-conditioned input (Algorithm 4's stacked basis).
#include <cooperative_groups.h>
#include <mutex>

#include "qlr_internal.h"

namespace cg = cooperative_groups;

namespace {

// Position (a, b), a <= b, of entry e in the column-by-column listing of an upper triangle
// (0,0), (0,1), (1,1), (0,2), ...: b is the largest integer with b (b + 1) / 2 <= e.
__device__ __forceinline__ int2 upper_tri_entry(int e) {
  int b = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (b > 0 && b * (b + 1) / 2 > e) --b;
  while ((b + 1) * (b + 2) / 2 <= e) ++b;
  return make_int2(e - b * (b + 1) / 2, b);
}

// ---------------------------------------------------------------------------------------
// Gram partial sums: part[chunk] = sum over the chunk's rows r of conj(y_ri) y_rj, for tiles
// (ti <= tj) of the upper triangle.  32 x 32 quaternion tiles, 256 threads, 2 x 2 per thread.
constexpr int GT = 32, GR = 16;

template <class TY>
__global__ void __launch_bounds__(256) gram_partial_kernel(const TY* __restrict__ y0, const TY* __restrict__ y1,
                                                           const TY* __restrict__ y2, const TY* __restrict__ y3,
                                                           int64_t m, int l, int64_t ld, int64_t rows_per_chunk,
                                                           double* __restrict__ part) {
  __shared__ double Yi[4][GR][GT + 1];
  __shared__ double Yj[4][GR][GT + 1];
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int2 tile = upper_tri_entry((int)blockIdx.x);
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

// C = A B for small l x l quaternion matrices (FP64), A and B upper triangular.
constexpr int MM_SPLIT = 16;   // lanes sharing one output entry of small_matmul_kernel

__global__ void __launch_bounds__(128) small_matmul_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                                            double* __restrict__ C, int l) {
  // C = A B for upper-triangular A, B: only entries i <= j, each the sum over i <= t <= j split
  // across MM_SPLIT lanes so the FP64 work is spread evenly over all SMs; C's lower part is zero.
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ent = gt / MM_SPLIT;
  const int part = (int)(gt % MM_SPLIT);
  const int64_t nent = (int64_t)l * (l + 1) / 2;
  const bool valid = ent < nent;
  int i = 0, j = 0;
  if (valid) {
    const int2 ij = upper_tri_entry((int)ent);
    i = ij.x;
    j = ij.y;
  }
  Quat<double> s = {0, 0, 0, 0};
  if (valid) {
#pragma unroll 4
    for (int t = i + part; t <= j; t += MM_SPLIT) {
      const Quat<double> p = qmul(ld_small(A, l, i, t), ld_small(B, l, t, j));
      s.w += p.w; s.x += p.x; s.y += p.y; s.z += p.z;
    }
  }
#pragma unroll
  for (int o = MM_SPLIT / 2; o > 0; o >>= 1) {
    s.w += __shfl_xor_sync(0xffffffffu, s.w, o);
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    s.z += __shfl_xor_sync(0xffffffffu, s.z, o);
  }
  if (!valid || part != 0) return;
  st_small(C, l, i, j, s);
  if (i < j) st_small(C, l, j, i, Quat<double>{0, 0, 0, 0});
}

// ---------------------------------------------------------------------------------------
// FP64-class Gram of FP32 data on the FP32 pipes (GB300 runs FP64 at 1/64 of the FP32 rate).
// The real symmetric W = Yh^T Yh of the plane-stacked Yh = [Y0 Y1 Y2 Y3] (m x 4l) is accumulated
// in double-FP32: every product a*b is split exactly into hi + lo with an FMA, hi is added with
// a branch-free two-sum (Knuth) into (S, C), lo goes into C.  The result S + C has a relative
// error of about 2^-48 of sum |a b|.  Upper 64 x 64 tiles only (on diagonal tiles, the entries on or
// above the diagonal); row chunks give partial sums
// that a second kernel adds in FP64 and combines into the quaternion Gram:
//   G0 = W00 + W11 + W22 + W33,  G1 = W01 - W10 - W23 + W32,
//   G2 = W02 + W13 - W20 - W31,  G3 = W03 - W12 + W21 - W30   (W_cd = Y_c^T Y_d).
constexpr int WT = 64, WR = 16;

// The _rn intrinsics keep the compiler from contracting these steps into FMAs.
__device__ __forceinline__ void df_add(float& S, float& C, float a, float b) {
  const float hi = __fmul_rn(a, b);
  const float lo = fmaf(a, b, -hi);
  const float s = __fadd_rn(S, hi);
  const float v = __fsub_rn(s, S);
  const float e = __fadd_rn(__fsub_rn(S, __fsub_rn(s, v)), __fsub_rn(hi, v));
  S = s;
  C = __fadd_rn(C, __fadd_rn(e, lo));
}

// One 64 x 64 tile (I0, J0) of W over rows [r_begin, r_end): thread (tx, ty) accumulates the
// entries (I0 + tx + 16 x, J0 + ty + 16 z) into (S, C).  On a diagonal tile (DIAG, I0 == J0) the
// pairs x > z lie strictly below the diagonal (I - J >= 16 - 15) and are skipped: W is symmetric
// and its readers take entry (I, J) with I <= J.
__device__ __forceinline__ const float* plane_of(const float* y0, const float* y1, const float* y2, const float* y3, int c) {
  return c == 0 ? y0 : (c == 1 ? y1 : (c == 2 ? y2 : y3));
}
template <bool DIAG>
__device__ __forceinline__ void gram_df_tile(const float* y0, const float* y1, const float* y2, const float* y3, int l,
                                             int64_t ld, int64_t r_begin, int64_t r_end, int I0, int J0,
                                             float (&S)[4][4], float (&C)[4][4]) {
  __shared__ float Ya[WR][WT];
  __shared__ float Yb[WR][WT];
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int L4 = 4 * l;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) S[a][b] = C[a][b] = 0.f;
  // loader mapping: 256 threads x 4 loads = 16 rows x 64 columns per operand
  for (int64_t r0 = r_begin; r0 < r_end; r0 += WR) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int rr = t % WR, cc = t / WR + 16 * h;
      const int64_t gr = r0 + rr;
      float va = 0.f, vb = 0.f;
      if (gr < r_end) {
        const int Ia = I0 + cc, Ib = J0 + cc;
        if (Ia < L4) va = plane_of(y0, y1, y2, y3, Ia / l)[gr + (int64_t)(Ia % l) * ld];
        if (Ib < L4) vb = plane_of(y0, y1, y2, y3, Ib / l)[gr + (int64_t)(Ib % l) * ld];
      }
      Ya[rr][cc] = va;
      Yb[rr][cc] = vb;
    }
    __syncthreads();
#pragma unroll 2
    for (int rr = 0; rr < WR; ++rr) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = Ya[rr][tx + 16 * q]; b[q] = Yb[rr][ty + 16 * q]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int z = 0; z < 4; ++z)
          if (!DIAG || x <= z) df_add(S[x][z], C[x][z], a[x], b[z]);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) gram_df_partial_kernel(const float* __restrict__ y0, const float* __restrict__ y1,
                                                               const float* __restrict__ y2, const float* __restrict__ y3,
                                                               int64_t m, int l, int64_t ld, int64_t rows_per_chunk,
                                                               double* __restrict__ part) {
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int2 tile = upper_tri_entry((int)blockIdx.x);
  const int I0 = tile.x * WT, J0 = tile.y * WT;
  const int L4 = 4 * l;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r_end = min(m, r_begin + rows_per_chunk);
  float S[4][4], C[4][4];
  const bool diag = (tile.x == tile.y);
  if (diag) gram_df_tile<true>(y0, y1, y2, y3, l, ld, r_begin, r_end, I0, J0, S, C);
  else gram_df_tile<false>(y0, y1, y2, y3, l, ld, r_begin, r_end, I0, J0, S, C);
  double* P = part + (size_t)blockIdx.y * L4 * L4;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int z = 0; z < 4; ++z) {
      const int I = I0 + tx + 16 * x, J = J0 + ty + 16 * z;
      if (I < L4 && J < L4 && !(diag && x > z)) P[(size_t)J * L4 + I] = (double)S[x][z] + (double)C[x][z];
    }
}

// Sum the chunk partials of W (upper tiles) in a fixed order, coalesced, into part[0].
__global__ void gram_df_reduce_kernel(double* __restrict__ part, int nchunks, int L4) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)L4 * L4) return;
  const int I = (int)(e % L4), J = (int)(e / L4);
  if ((I / WT) > (J / WT)) return;
  double s = part[e];
  for (int c = 1; c < nchunks; ++c) s += part[(size_t)c * L4 * L4 + e];
  part[e] = s;
}

__device__ __forceinline__ double w_at(const double* __restrict__ W, int L4, int I, int J) {
  if (I > J) { int t = I; I = J; J = t; }     // only entries on or above the diagonal were computed
  return W[(size_t)J * L4 + I];
}

__global__ void gram_df_combine_kernel(const double* __restrict__ part, int l, double* __restrict__ G) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)l * l) return;
  const int i = (int)(idx % l), j = (int)(idx / l);
  if (i > j) return;
  const int L4 = 4 * l;
  double w[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int d = 0; d < 4; ++d) w[c][d] = w_at(part, L4, c * l + i, d * l + j);
  Quat<double> g;
  g.w = w[0][0] + w[1][1] + w[2][2] + w[3][3];
  g.x = w[0][1] - w[1][0] - w[2][3] + w[3][2];
  g.y = w[0][2] + w[1][3] - w[2][0] - w[3][1];
  g.z = w[0][3] - w[1][2] + w[2][1] - w[3][0];
  if (i == j) g.x = g.y = g.z = 0.0;
  st_small(G, l, i, j, g);
  if (i != j) st_small(G, l, j, i, {g.w, -g.x, -g.y, -g.z});
}


// ---------------------------------------------------------------------------------------
// Blocked right-looking quaternion Cholesky in FP64 over many SMs.  Wm holds the upper triangle
// of the working matrix (initially G, plus the shift); R receives the factor.  For each panel
// [j0, j0 + CB): (1) one CTA factors the diagonal block and inverts it; (2) the panel rows
// R[j0:j1, k] = R_jj^{-H} Wm[j0:j1, k] are formed column-parallel; (3) the trailing upper
// triangle is updated tile-parallel: Wm[i, k] -= sum_t conj(R[t, i]) R[t, k].
constexpr int CB = 16;      // panel width
constexpr int CT = 8;       // trailing-update tile

__global__ void chol_init_kernel(const double* __restrict__ G, double* __restrict__ Wm, double* __restrict__ R, int l,
                                 double shift_coef, const int* run_if) {
  __shared__ double s_tr;
  if (run_if && *run_if == 0) return;
  const size_t ll = (size_t)l * l;
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int i = 0; i < l; ++i) tr += G[(size_t)i * l + i];
    s_tr = shift_coef * tr;
  }
  __syncthreads();
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < ll; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % l), j = (int)(e / l);
    for (int c = 0; c < 4; ++c) {
      Wm[c * ll + e] = (i <= j) ? G[c * ll + e] + ((c == 0 && i == j) ? s_tr : 0.0) : 0.0;
      R[c * ll + e] = 0.0;
    }
  }
}

// Factor the diagonal block [j0, j0+b) of Wm into R (upper, real positive diagonal) and write its
// inverse into Dinv (b x b x 4, column-major).
__global__ void __launch_bounds__(256) chol_diag_kernel(double* __restrict__ Wm, double* __restrict__ R, int l, int j0,
                                                         int b, double* __restrict__ Dinv, int* err, const int* run_if) {
  // FP64 issues at a small fraction of the FP32 rate, so every FP64 instruction here is issued by
  // warps whose lanes all carry work: the active (row, column) pairs of each step are enumerated
  // densely, and pivots and their reciprocals are computed once.
  if (run_if && *run_if == 0) return;
  __shared__ double D[4][CB][CB];
  __shared__ double X[4][CB][CB];
  __shared__ double rpiv[CB];
  const int t = threadIdx.x;
  const size_t ll = (size_t)l * l;
  for (int e = t; e < CB * CB; e += blockDim.x) {
    const int i = e % CB, j = e / CB;
    for (int c = 0; c < 4; ++c) {
      D[c][i][j] = (i < b && j < b && i <= j) ? Wm[c * ll + (size_t)(j0 + j) * l + j0 + i] : 0.0;
      X[c][i][j] = 0.0;
    }
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (t == 0) {
      double d2 = D[0][j][j];
      if (!(d2 > 0.0)) {
        qlr_set_error(err, QLR_ENOTPD);
        d2 = 1e-300;
      }
      const double piv = sqrt(d2);
      D[0][j][j] = piv;
      D[1][j][j] = D[2][j][j] = D[3][j][j] = 0.0;
      rpiv[j] = 1.0 / piv;
    }
    __syncthreads();
    const int n = b - j - 1;                  // row j right of the pivot: n entries x 4 planes
    if (t < 4 * n) {
      const int c = t / n, k = j + 1 + t % n;
      D[c][j][k] *= rpiv[j];
    }
    __syncthreads();
    // trailing update D[i][k] -= conj(D[j][i]) D[j][k] for j < i <= k < b: n (n + 1) / 2 pairs
    const int npairs = n * (n + 1) / 2;
    for (int e = t; e < npairs; e += blockDim.x) {
      const int2 ik = upper_tri_entry(e);
      const int i = j + 1 + ik.x, k = j + 1 + ik.y;
      Quat<double> pr = qcmul(Quat<double>{D[0][j][i], D[1][j][i], D[2][j][i], D[3][j][i]},
                              Quat<double>{D[0][j][k], D[1][j][k], D[2][j][k], D[3][j][k]});
      D[0][i][k] -= pr.w; D[1][i][k] -= pr.x; D[2][i][k] -= pr.y; D[3][i][k] -= pr.z;
    }
    __syncthreads();
  }
  // inverse X = D^{-1} by column-oriented back substitution on all right-hand sides at once:
  // for i = b-1 .. 0: X[i, i:] = Y[i, i:] / d_i, then Y[0:i, i:] -= D[0:i, i] X[i, i:]  (Y starts as I;
  // row i of X is zero left of the diagonal)
  for (int e = t; e < b; e += blockDim.x) X[0][e][e] = 1.0;
  __syncthreads();
  for (int i = b - 1; i >= 0; --i) {
    const int w = b - i;
    if (t < 4 * w) {
      const int c = t / w, j = i + t % w;
      X[c][i][j] *= rpiv[i];
    }
    __syncthreads();
    for (int e = t; e < i * w; e += blockDim.x) {   // rows r < i, columns j >= i
      const int r = e % i, j = i + e / i;
      Quat<double> pr = qmul(Quat<double>{D[0][r][i], D[1][r][i], D[2][r][i], D[3][r][i]},
                             Quat<double>{X[0][i][j], X[1][i][j], X[2][i][j], X[3][i][j]});
      X[0][r][j] -= pr.w; X[1][r][j] -= pr.x; X[2][r][j] -= pr.y; X[3][r][j] -= pr.z;
    }
    __syncthreads();
  }
  for (int e = t; e < b * b; e += blockDim.x) {
    const int i = e % b, j = e / b;
    for (int c = 0; c < 4; ++c) {
      R[c * ll + (size_t)(j0 + j) * l + j0 + i] = (i <= j) ? D[c][i][j] : 0.0;
      Dinv[(size_t)c * b * b + (size_t)j * b + i] = (i <= j) ? X[c][i][j] : 0.0;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Cholesky factorisation of the whole l x l FP64 Gram in one thread-block cluster (NC CTAs,
// 8 or 16).  FP64 runs at a small fraction of the FP32 rate on every SM, so the work has to be
// spread over several SMs, and a chain of one launch per block column spends most of its time
// between kernels.  Here the upper triangle stays in shared memory, column k owned by CTA k mod NC
// (rows 0..k, quaternions stored plane-interleaved).  Column step j: every CTA scales row j, which
// the column owners pushed into its shared memory during step j - 1, by 1/r_jj (this is row j of
// R); it then updates row j + 1 of its own columns and pushes those entries to every CTA through
// distributed shared memory, and the owner of column j + 1 takes and pushes that pivot.  The CTAs
// then arrive at the cluster barrier and do the rest of the rank-1 update (rows >= j + 2) before
// waiting on it, so the bulk FP64 work overlaps the barrier and no remote load sits on the path.  At the end each CTA inverts some of
// the CB x CB diagonal blocks of R for the blocked triangular inverse.
constexpr int CC_THREADS = 256;

__host__ __device__ __forceinline__ int cc_nown(int l, int nc, int c) { return c < l ? (l - c + nc - 1) / nc : 0; }
// Offset (in quaternions) of the first stored row of column k = c + idx * nc in CTA c.
__host__ __device__ __forceinline__ int cc_colstart(int nc, int c, int idx) { return idx * (c + 1) + nc * idx * (idx - 1) / 2; }
__host__ __device__ __forceinline__ size_t cc_smem(int l, int nc) {
  int mx = 0;
  for (int c = 0; c < nc; ++c) {
    const int n = cc_nown(l, nc, c);
    const int tot = cc_colstart(nc, c, n);
    mx = tot > mx ? tot : mx;
  }
  return (size_t)mx * 32 + (size_t)4 * l * 32 + 128;   // columns, h, three receive slots, pivots, mbarriers
}

__device__ __forceinline__ void cluster_arrive_release() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait_acquire() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

// X = D^{-1} for an upper-triangular b x b quaternion block D with real positive diagonal (dense
// lanes, column-oriented back substitution on all right-hand sides; X starts as the identity).
__device__ void cc_block_inverse(double (&D)[4][CB][CB], double (&X)[4][CB][CB], double* rpiv, int b) {
  const int t = threadIdx.x;
  for (int e = t; e < CB * CB; e += blockDim.x) {
    const int i = e % CB, j = e / CB;
    X[0][i][j] = (i == j && i < b) ? 1.0 : 0.0;
    X[1][i][j] = X[2][i][j] = X[3][i][j] = 0.0;
  }
  if (t < b) rpiv[t] = 1.0 / D[0][t][t];
  __syncthreads();
  for (int i = b - 1; i >= 0; --i) {
    const int w = b - i;
    if (t < 4 * w) {
      const int c = t / w, j = i + t % w;
      X[c][i][j] *= rpiv[i];
    }
    __syncthreads();
    for (int e = t; e < i * w; e += blockDim.x) {
      const int r = e % i, j = i + e / i;
      Quat<double> pr = qmul(Quat<double>{D[0][r][i], D[1][r][i], D[2][r][i], D[3][r][i]},
                             Quat<double>{X[0][i][j], X[1][i][j], X[2][i][j], X[3][i][j]});
      X[0][r][j] -= pr.w; X[1][r][j] -= pr.x; X[2][r][j] -= pr.y; X[3][r][j] -= pr.z;
    }
    __syncthreads();
  }
}

// w - conj(a) b for quaternions stored as (real, i, j, k) in double4, four fused multiply-adds
// per component.
__device__ __forceinline__ double4 qcfms(double4 w, const double4 a, const double4 b) {
  w.x = fma(-a.x, b.x, w.x); w.x = fma(-a.y, b.y, w.x); w.x = fma(-a.z, b.z, w.x); w.x = fma(-a.w, b.w, w.x);
  w.y = fma(-a.x, b.y, w.y); w.y = fma(a.y, b.x, w.y);  w.y = fma(a.z, b.w, w.y);  w.y = fma(-a.w, b.z, w.y);
  w.z = fma(-a.x, b.z, w.z); w.z = fma(-a.y, b.w, w.z); w.z = fma(a.z, b.x, w.z);  w.z = fma(a.w, b.y, w.z);
  w.w = fma(-a.x, b.w, w.w); w.w = fma(a.y, b.z, w.w);  w.w = fma(-a.z, b.y, w.w); w.w = fma(a.w, b.x, w.w);
  return w;
}

// 1 / sqrt(d) in FP64: the FP32 hardware estimate refined by Newton-Raphson steps
// y <- y (3 - d y^2) / 2, each squaring the relative error (2^-22 -> 2^-43 -> below FP64
// rounding).  FP64 instructions are slow on this part and the pivot sits on the Cholesky's
// critical path, so the factorisation takes one step (relative error ~2^-43 ~ 1e-13, a uniform
// scaling of row j of R and column j of its inverse) and the other uses take two.
__device__ __forceinline__ double rsqrt_newton(double d, int steps = 2) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf((float)d);
  y = y * fma(-0.5 * d * y, y, 1.5);
  if (steps > 1) y = y * fma(-0.5 * d * y, y, 1.5);
  return y;
}

// Distributed shared memory data flow: st.async writes into another CTA's shared memory and
// completes bytes on that CTA's mbarrier; the receiver waits on its own mbarrier phase.
__device__ __forceinline__ uint32_t cc_smem32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t cc_remote(uint32_t local, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void cc_st_async2(uint32_t raddr, double a, double b, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(raddr), "d"(a),
               "d"(b), "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void cc_st_async1(uint32_t raddr, double a, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(raddr), "d"(a),
               "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void cc_arm(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cc_smem32(bar)), "r"(bytes) : "memory");
}
// Bounded wait on a phase (1.5 s); false on timeout (QLR_ETIMEOUT recorded).
__device__ __forceinline__ bool cc_wait(uint64_t* bar, uint32_t parity, int* err) {
  const uint32_t a = cc_smem32(bar);
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    uint64_t now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (it == 0) t0 = now;
    else if (now - t0 > 1500000000ull) {
      qlr_set_error(err, QLR_ETIMEOUT);
      return false;
    }
  }
}

__global__ void __launch_bounds__(CC_THREADS, 1) chol_cluster_kernel(const double* __restrict__ G, double* __restrict__ R,
                                                                     double* __restrict__ Dinv_all, int l, double shift_coef,
                                                                     int* err, const int* run_if) {
  if (run_if && *run_if == 0) return;           // the same decision in every CTA of the cluster
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int nc = (int)cluster.num_blocks();
  const int c = (int)cluster.block_rank();
  const int t = threadIdx.x, lane = t % 32, warp = t / 32, nwarps = CC_THREADS / 32;
  const size_t ll = (size_t)l * l;
  const int nown = cc_nown(l, nc, c);
  int mxtot = 0;
  for (int cc = 0; cc < nc; ++cc) mxtot = max(mxtot, cc_colstart(nc, cc, cc_nown(l, nc, cc)));
  double4* Wc = reinterpret_cast<double4*>(smem_raw);       // own columns (rows 0..k)
  double4* h = Wc + mxtot;                                    // h_k of the own columns (below)
  // Three receive slots: slot j mod 3 gets row j of W (entries k > j) from the column owners and
  // 1 / r_jj from the pivot owner during step j - 1, with an mbarrier counting the bytes.  A CTA
  // can only start step j once every CTA has pushed its part of row j (made after its step j - 1
  // look-ahead, hence after its step j - 2 bulk), so a slot is never written while still read.
  double4* slot_row = h + l;                                  // [3][l]
  double* slot_rp = reinterpret_cast<double*>(slot_row + 3 * l);   // [3] (+ padding)
  uint64_t* slot_bar = reinterpret_cast<uint64_t*>(slot_rp + 4);   // [3]
  auto bytes_of = [&](int j) -> uint32_t { return (uint32_t)(8 + 32 * (l - j - 1)); };
  cluster.sync();   // every CTA of the cluster is running before any distributed shared memory access
  if (t == 0) {
    for (int s = 0; s < 3; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cc_smem32(&slot_bar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // shift s = shift_coef * trace(G) on the diagonal
  __shared__ double s_shift;
  if (warp == 0) {
    double tr = 0.0;
    for (int i = lane; i < l; i += 32) tr += G[(size_t)i * l + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (lane == 0) s_shift = shift_coef * tr;
  }
  __syncthreads();
  for (int idx = warp; idx < nown; idx += nwarps) {
    const int k = c + idx * nc;
    double4* col = Wc + cc_colstart(nc, c, idx);
    for (int i = lane; i <= k; i += 32) {
      const size_t o = (size_t)k * l + i;
      double4 q = make_double4(G[o], G[ll + o], G[2 * ll + o], G[3 * ll + o]);
      if (i == k) q.x += s_shift;
      col[i] = q;
    }
    for (int i = k + 1 + lane; i < l; i += 32)   // lower part of R is zero
      for (int cp = 0; cp < 4; ++cp) R[cp * ll + (size_t)k * l + i] = 0.0;
  }
  __syncthreads();
  cluster.sync();   // every mbarrier initialised before any remote completion
  if (t == 0)
    for (int s = 0; s < 3 && s < l; ++s) cc_arm(&slot_bar[s], bytes_of(s));

  // R is built in place: once row j has been pushed, W[j][k] of an own column is dead and its slot
  // takes R[j][k]; R goes to global memory once at the end.
  // Pivot of column j by its owner (one thread): R[j][j] and 1 / r_jj to every CTA's slot.
  auto take_pivot = [&](int j) {
    double4& wjj = Wc[cc_colstart(nc, c, j / nc) + j];
    double d = wjj.x;
    if (!(d > 0.0)) {
      qlr_set_error(err, QLR_ENOTPD);
      d = 1e-300;
    }
    const double rp = rsqrt_newton(d, 1);
    const int s = j % 3;
    const uint32_t la = cc_smem32(&slot_rp[s]), lb = cc_smem32(&slot_bar[s]);
    for (int r = 0; r < nc; ++r) cc_st_async1(cc_remote(la, r), rp, cc_remote(lb, r));
    wjj = make_double4(d * rp, 0.0, 0.0, 0.0);
  };
  // Entries k > j of row j of the own columns to every CTA's slot (items e < ncol * nc).
  auto push_row = [&](int j) {
    const int s = j % 3;
    const int idx0 = (j + 1 - c + nc - 1) / nc;   // first own column with k > j
    const int ncol = nown - idx0;
    const uint32_t lb = cc_smem32(&slot_bar[s]);
    for (int e = t; e < ncol * nc; e += CC_THREADS) {
      const int idx = idx0 + e / nc, r = e % nc, k = c + idx * nc;
      const double4 w = Wc[cc_colstart(nc, c, idx) + j];
      const uint32_t la = cc_smem32(&slot_row[s * l + k]);
      const uint32_t ra = cc_remote(la, r), rb = cc_remote(lb, r);
      cc_st_async2(ra, w.x, w.y, rb);
      cc_st_async2(ra + 16, w.z, w.w, rb);
    }
  };
  if (c == 0 && t == 0 && l > 0) take_pivot(0);
  if (l > 1) push_row(0);

  bool ok = true;
  for (int j = 0; j < l && ok; ++j) {
    const int s = j % 3;
    ok = cc_wait(&slot_bar[s], (uint32_t)(j / 3) & 1u, err);
    if (!ok) break;
    const double rp = slot_rp[s];
    const double4* row = slot_row + s * l;
    const int j1 = j + 1;
    const int idx0 = (j1 - c + nc - 1) / nc;   // first own column index with k >= j + 1
    const int nact = nown - idx0;
    // look-ahead row j + 1 (on the critical path of every step): one lane per quaternion
    // component of each own column, so each FP64 instruction serves up to eight columns --
    // h_k = W[j][k] / r_jj^2 component-wise, the other three components by shuffles, then
    // W[j+1][k] -= conj(W[j][j+1]) h_k for this lane's component
    const int nlane = 32 * ((4 * nact + 31) / 32);   // whole warps: every lane takes part in the shuffles
    if (t < nlane) {
      const int ci = t >> 2, comp = t & 3;
      const bool act = ci < nact;
      const int idx = idx0 + (act ? ci : 0), k = c + idx * nc;
      const double rp2 = rp * rp;
      const double* qk = reinterpret_cast<const double*>(&row[act ? k : j1]);
      const double hc = qk[comp] * rp2;
      const int base = (t & 31) & ~3;
      const double h0 = __shfl_sync(0xffffffffu, hc, base + 0), h1 = __shfl_sync(0xffffffffu, hc, base + 1);
      const double h2 = __shfl_sync(0xffffffffu, hc, base + 2), h3 = __shfl_sync(0xffffffffu, hc, base + 3);
      if (act) {
        reinterpret_cast<double*>(&h[k])[comp] = hc;
        const double4 a = row[j1];
        double* wp = reinterpret_cast<double*>(&Wc[cc_colstart(nc, c, idx) + j1]) + comp;
        double w = *wp;
        if (comp == 0) {
          w = fma(-a.x, h0, w); w = fma(-a.y, h1, w); w = fma(-a.z, h2, w); w = fma(-a.w, h3, w);
        } else if (comp == 1) {
          w = fma(-a.x, h1, w); w = fma(a.y, h0, w); w = fma(a.z, h3, w); w = fma(-a.w, h2, w);
        } else if (comp == 2) {
          w = fma(-a.x, h2, w); w = fma(-a.y, h3, w); w = fma(a.z, h0, w); w = fma(a.w, h1, w);
        } else {
          w = fma(-a.x, h3, w); w = fma(a.y, h2, w); w = fma(-a.z, h1, w); w = fma(a.w, h0, w);
        }
        *wp = w;
      }
    }
    __syncthreads();
    if (j1 < l) {
      if (c == j1 % nc && t == 0) take_pivot(j1);
      push_row(j1);
    }
    if (t < nact) {                            // R[j][k] of the own columns (off the critical path)
      const int k = c + (idx0 + t) * nc;
      const double4 q = row[k];
      Wc[cc_colstart(nc, c, idx0 + t) + j] = make_double4(q.x * rp, q.y * rp, q.z * rp, q.w * rp);
    }
    // bulk of the rank-1 update: rows j + 2 .. k of the own columns k >= j + 2, the (column, row)
    // items numbered consecutively over all threads so FP64 warps run full.  Column m (from the
    // first one, k_0 >= j + 2) has L_0 + m nc rows; item e lies in the column m with
    // P(m) <= e < P(m + 1), P(m) = m L_0 + nc m (m - 1) / 2.
    const int j2 = j + 2;
    if (j2 < l) {
      const int jdx0 = (j2 - c + nc - 1) / nc;
      const int ncol = nown - jdx0;
      if (ncol > 0) {
        const int L0 = c + jdx0 * nc - j2 + 1;
        const int total = ncol * L0 + nc * ncol * (ncol - 1) / 2;
        const float hb = (float)L0 - 0.5f * (float)nc;
        for (int e = t; e < total; e += CC_THREADS) {
          int m = (int)((-hb + sqrtf(hb * hb + 2.0f * (float)nc * (float)e)) / (float)nc);
          m = max(0, min(m, ncol - 1));
          while (m > 0 && m * L0 + nc * m * (m - 1) / 2 > e) --m;
          while (m + 1 < ncol && (m + 1) * L0 + nc * (m + 1) * m / 2 <= e) ++m;
          const int i = j2 + e - (m * L0 + nc * m * (m - 1) / 2);
          const int idx = jdx0 + m, k = c + idx * nc;
          double4& w = Wc[cc_colstart(nc, c, idx) + i];
          w = qcfms(w, row[i], h[k]);
        }
      }
    }
    __syncthreads();                           // slot s and h are free again
    if (t == 0 && j + 3 < l) cc_arm(&slot_bar[s], bytes_of(j + 3));
  }
  cluster.sync();   // last distributed shared memory access done before any CTA moves on
  for (int idx = warp; idx < nown; idx += nwarps) {
    const int k = c + idx * nc;
    const double4* col = Wc + cc_colstart(nc, c, idx);
    for (int i = lane; i <= k; i += 32) {
      const double4 r = col[i];
      const size_t o = (size_t)k * l + i;
      R[o] = r.x; R[ll + o] = r.y; R[2 * ll + o] = r.z; R[3 * ll + o] = r.w;
    }
  }
  __threadfence();
  cluster.sync();
  // inverses of the diagonal blocks (block J = rows / columns [J CB, J CB + b))
  __shared__ double D[4][CB][CB];
  __shared__ double X[4][CB][CB];
  __shared__ double rpv[CB];
  const int nblk = (l + CB - 1) / CB;
  for (int J = c; J < nblk; J += nc) {
    const int j0 = J * CB, b = min(CB, l - j0);
    for (int e = t; e < CB * CB; e += blockDim.x) {
      const int i = e % CB, jj = e / CB;
      for (int cp = 0; cp < 4; ++cp)
        D[cp][i][jj] = (i < b && jj < b && i <= jj) ? __ldcg(R + cp * ll + (size_t)(j0 + jj) * l + j0 + i) : 0.0;
    }
    __syncthreads();
    cc_block_inverse(D, X, rpv, b);
    double* Dinv = Dinv_all + (size_t)J * 4 * CB * CB;
    for (int e = t; e < b * b; e += blockDim.x) {
      const int i = e % b, jj = e / b;
      for (int cp = 0; cp < 4; ++cp) Dinv[(size_t)cp * b * b + (size_t)jj * b + i] = (i <= jj) ? X[cp][i][jj] : 0.0;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// The same cluster Cholesky in double-FP32 arithmetic (an unevaluated sum hi + lo of two floats,
// about 48 significant bits), for Grams of FP32 sketches, which the Gram kernel already forms in
// double-FP32: the factorisation then matches the Gram's precision, while every step runs on the
// FP32 pipes (FP64 instructions issue slowly here and a dependent one takes ~200 cycles, which
// put the FP64 column step's look-ahead and pivot near 3000 cycles).  The operations are Knuth's
// two-sum and the fused-multiply-add exact product (Dekker), renormalised after each operation;
// 1 / sqrt uses the FP32 estimate and two Newton-Raphson steps in double-FP32.
struct d32 {
  float h, l;
};
__device__ __forceinline__ d32 d32_add(d32 a, d32 b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ d32 d32_mul(d32 a, d32 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
__device__ __forceinline__ d32 d32_neg(d32 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ d32 d32_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double d32_to(d32 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ d32 d32_rsqrt(d32 d) {
  d32 y = {rsqrtf(d.h), 0.f};
  for (int it = 0; it < 2; ++it) {   // y <- y + y (1 - d y^2) / 2
    const d32 r = d32_add({1.f, 0.f}, d32_neg(d32_mul(d32_mul(d, y), y)));
    y = d32_add(y, d32_mul(y, {0.5f * r.h, 0.5f * r.l}));
  }
  return y;
}
// A quaternion of double-FP32 numbers: components (real, i, j, k) of the high and low parts.
struct dq {
  float4 h, l;
};
__device__ __forceinline__ d32 dq_get(const dq& q, int c) {
  return {reinterpret_cast<const float*>(&q.h)[c], reinterpret_cast<const float*>(&q.l)[c]};
}
__device__ __forceinline__ void dq_set(dq& q, int c, d32 v) {
  reinterpret_cast<float*>(&q.h)[c] = v.h;
  reinterpret_cast<float*>(&q.l)[c] = v.l;
}
// Component c of w - conj(a) b (the signs of conj(a) b per component).
__device__ __forceinline__ d32 dq_cfms_comp(d32 w, const d32 (&a)[4], const d32 (&b)[4], int c) {
  auto sub = [&](d32 x, d32 p, d32 q) { return d32_add(x, d32_neg(d32_mul(p, q))); };
  auto add = [&](d32 x, d32 p, d32 q) { return d32_add(x, d32_mul(p, q)); };
  if (c == 0) { w = sub(w, a[0], b[0]); w = sub(w, a[1], b[1]); w = sub(w, a[2], b[2]); return sub(w, a[3], b[3]); }
  if (c == 1) { w = sub(w, a[0], b[1]); w = add(w, a[1], b[0]); w = add(w, a[2], b[3]); return sub(w, a[3], b[2]); }
  if (c == 2) { w = sub(w, a[0], b[2]); w = sub(w, a[1], b[3]); w = add(w, a[2], b[0]); return add(w, a[3], b[1]); }
  w = sub(w, a[0], b[3]); w = add(w, a[1], b[2]); w = sub(w, a[2], b[1]); return add(w, a[3], b[0]);
}
__device__ __forceinline__ dq dq_cfms(dq w, const dq& a, const dq& b) {
  d32 av[4], bv[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) { av[c] = dq_get(a, c); bv[c] = dq_get(b, c); }
  dq r;
#pragma unroll
  for (int c = 0; c < 4; ++c) dq_set(r, c, dq_cfms_comp(dq_get(w, c), av, bv, c));
  return r;
}
__device__ __forceinline__ void cc_st_async4f(uint32_t raddr, float4 v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(raddr),
               "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void cc_st_async2f(uint32_t raddr, float a, float b, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr), "f"(a),
               "f"(b), "r"(rbar)
               : "memory");
}

__global__ void __launch_bounds__(CC_THREADS, 1) chol_cluster_df_kernel(const double* __restrict__ G, double* __restrict__ R,
                                                                        double* __restrict__ Dinv_all, int l,
                                                                        double shift_coef, int* err, const int* run_if) {
  if (run_if && *run_if == 0) return;           // the same decision in every CTA of the cluster
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int nc = (int)cluster.num_blocks();
  const int c = (int)cluster.block_rank();
  const int t = threadIdx.x, lane = t % 32, warp = t / 32, nwarps = CC_THREADS / 32;
  const size_t ll = (size_t)l * l;
  const int nown = cc_nown(l, nc, c);
  int mxtot = 0;
  for (int cc = 0; cc < nc; ++cc) mxtot = max(mxtot, cc_colstart(nc, cc, cc_nown(l, nc, cc)));
  dq* Wc = reinterpret_cast<dq*>(smem_raw);                  // own columns (rows 0..k)
  dq* h = Wc + mxtot;                                         // h_k of the own columns
  dq* slot_row = h + l;                                       // [3][l] received rows (see the FP64 kernel)
  d32* slot_rp = reinterpret_cast<d32*>(slot_row + 3 * l);   // [3][2]: 1 / r_jj and its square
  uint64_t* slot_bar = reinterpret_cast<uint64_t*>(slot_rp + 6);   // [3]
  auto bytes_of = [&](int j) -> uint32_t { return (uint32_t)(16 + 32 * (l - j - 1)); };
  cluster.sync();   // every CTA of the cluster is running before any distributed shared memory access
  if (t == 0) {
    for (int s = 0; s < 3; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cc_smem32(&slot_bar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __shared__ double s_shift;
  if (warp == 0) {
    double tr = 0.0;
    for (int i = lane; i < l; i += 32) tr += G[(size_t)i * l + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (lane == 0) s_shift = shift_coef * tr;
  }
  __syncthreads();
  for (int idx = warp; idx < nown; idx += nwarps) {
    const int k = c + idx * nc;
    dq* col = Wc + cc_colstart(nc, c, idx);
    for (int i = lane; i <= k; i += 32) {
      const size_t o = (size_t)k * l + i;
      dq q;
      for (int cp = 0; cp < 4; ++cp) dq_set(q, cp, d32_from(G[cp * ll + o] + ((cp == 0 && i == k) ? s_shift : 0.0)));
      col[i] = q;
    }
    for (int i = k + 1 + lane; i < l; i += 32)   // lower part of R is zero
      for (int cp = 0; cp < 4; ++cp) R[cp * ll + (size_t)k * l + i] = 0.0;
  }
  __syncthreads();
  cluster.sync();   // every mbarrier initialised before any remote completion
  if (t == 0)
    for (int s = 0; s < 3 && s < l; ++s) cc_arm(&slot_bar[s], bytes_of(s));

  // Pivot of column j from its (updated) diagonal d, computed by one lane (`me`) of a full warp:
  // R[j][j] in place, and (1 / r_jj, 1 / r_jj^2) to every CTA's slot, one lane per CTA.
  auto take_pivot = [&](int j, d32 d, bool me) {
    d32 rp = {0.f, 0.f}, rp2 = {0.f, 0.f};
    if (me) {
      if (!(d.h > 0.f)) {
        qlr_set_error(err, QLR_ENOTPD);
        d = {1e-30f, 0.f};
      }
      rp = d32_rsqrt(d);
      rp2 = d32_mul(rp, rp);
      const d32 piv = d32_mul(d, rp);
      dq z;
      z.h = make_float4(piv.h, 0.f, 0.f, 0.f);
      z.l = make_float4(piv.l, 0.f, 0.f, 0.f);
      Wc[cc_colstart(nc, c, j / nc) + j] = z;
    }
    const unsigned src = __ffs(__ballot_sync(0xffffffffu, me)) - 1;
    rp.h = __shfl_sync(0xffffffffu, rp.h, src); rp.l = __shfl_sync(0xffffffffu, rp.l, src);
    rp2.h = __shfl_sync(0xffffffffu, rp2.h, src); rp2.l = __shfl_sync(0xffffffffu, rp2.l, src);
    const int ln = threadIdx.x & 31;
    if (ln < nc) {
      const int s = j % 3;
      const uint32_t rb = cc_remote(cc_smem32(&slot_bar[s]), ln);
      const uint32_t ra = cc_remote(cc_smem32(&slot_rp[2 * s]), ln);
      cc_st_async2f(ra, rp.h, rp.l, rb);
      cc_st_async2f(ra + 8, rp2.h, rp2.l, rb);
    }
  };
  auto push_row = [&](int j) {
    const int s = j % 3;
    const int idx0 = (j + 1 - c + nc - 1) / nc;
    const int ncol = nown - idx0;
    const uint32_t lb = cc_smem32(&slot_bar[s]);
    for (int e = t; e < ncol * nc; e += CC_THREADS) {
      const int idx = idx0 + e / nc, r = e % nc, k = c + idx * nc;
      const dq w = Wc[cc_colstart(nc, c, idx) + j];
      const uint32_t ra = cc_remote(cc_smem32(&slot_row[s * l + k]), r), rb = cc_remote(lb, r);
      cc_st_async4f(ra, w.h, rb);
      cc_st_async4f(ra + 16, w.l, rb);
    }
  };
  if (c == 0 && warp == 0 && l > 0) take_pivot(0, dq_get(Wc[0], 0), lane == 0);
  if (l > 1) push_row(0);

  bool ok = true;
  for (int j = 0; j < l && ok; ++j) {
    const int s = j % 3;
    ok = cc_wait(&slot_bar[s], (uint32_t)(j / 3) & 1u, err);
    if (!ok) break;
    const d32 rp = slot_rp[2 * s], rp2 = slot_rp[2 * s + 1];
    const dq* row = slot_row + s * l;
    const int j1 = j + 1;
    const int idx0 = (j1 - c + nc - 1) / nc;
    const int nact = nown - idx0;
    // look-ahead row j + 1, one lane per quaternion component of each own column: h_k =
    // W[j][k] / r_jj^2 (all four components, independent products), the four signed products
    // of this lane's component of conj(W[j][j+1]) h_k summed as a tree, subtracted from W[j+1][k].
    // The lane holding the diagonal of column j + 1 takes the pivot at once.
    const int nlane = 32 * ((4 * nact + 31) / 32);
    const bool own_next = (j1 < l && c == j1 % nc);
    if (t < nlane) {
      const int ci = t >> 2, comp = t & 3;
      const bool act = ci < nact;
      const int idx = idx0 + (act ? ci : 0), k = c + idx * nc;
      d32 piv_d = {0.f, 0.f};
      if (act) {
        // component `comp` of conj(a) h is sum_q (-1)^neg(comp, q) a_q h_{comp xor q}, with the
        // negative (comp, q) pairs the set bits of 0xAC60 at 4 comp + q
        const dq* qk = &row[k];
        const dq* ap = &row[j1];
        d32 p[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const d32 hq = d32_mul(dq_get(*qk, comp ^ q), rp2);
          if (q == 0) dq_set(h[k], comp, hq);
          const d32 aq = dq_get(*ap, q);
          const float sgn = ((0xAC60u >> (4 * comp + q)) & 1u) ? -1.f : 1.f;
          p[q] = d32_mul({sgn * aq.h, sgn * aq.l}, hq);
        }
        const d32 sum = d32_add(d32_add(p[0], p[1]), d32_add(p[2], p[3]));
        dq& w = Wc[cc_colstart(nc, c, idx) + j1];
        const d32 nv = d32_add(dq_get(w, comp), d32_neg(sum));
        dq_set(w, comp, nv);
        piv_d = nv;
      }
      if (own_next && warp == 0) take_pivot(j1, piv_d, act && k == j1 && comp == 0);
    }
    __syncthreads();
    if (j1 < l) push_row(j1);
    if (t < nact) {                            // R[j][k] of the own columns
      const int k = c + (idx0 + t) * nc;
      const dq q = row[k];
      dq r;
      for (int cp = 0; cp < 4; ++cp) dq_set(r, cp, d32_mul(dq_get(q, cp), rp));
      Wc[cc_colstart(nc, c, idx0 + t) + j] = r;
    }
    const int j2 = j + 2;
    if (j2 < l) {
      const int jdx0 = (j2 - c + nc - 1) / nc;
      const int ncol = nown - jdx0;
      if (ncol > 0) {
        const int L0 = c + jdx0 * nc - j2 + 1;
        const int total = ncol * L0 + nc * ncol * (ncol - 1) / 2;
        const float hb = (float)L0 - 0.5f * (float)nc;
        for (int e = t; e < total; e += CC_THREADS) {
          int m = (int)((-hb + sqrtf(hb * hb + 2.0f * (float)nc * (float)e)) / (float)nc);
          m = max(0, min(m, ncol - 1));
          while (m > 0 && m * L0 + nc * m * (m - 1) / 2 > e) --m;
          while (m + 1 < ncol && (m + 1) * L0 + nc * (m + 1) * m / 2 <= e) ++m;
          const int i = j2 + e - (m * L0 + nc * m * (m - 1) / 2);
          const int idx = jdx0 + m, k = c + idx * nc;
          dq& w = Wc[cc_colstart(nc, c, idx) + i];
          w = dq_cfms(w, row[i], h[k]);
        }
      }
    }
    __syncthreads();
    if (t == 0 && j + 3 < l) cc_arm(&slot_bar[s], bytes_of(j + 3));
  }
  cluster.sync();   // last distributed shared memory access done before any CTA moves on
  for (int idx = warp; idx < nown; idx += nwarps) {
    const int k = c + idx * nc;
    const dq* col = Wc + cc_colstart(nc, c, idx);
    for (int i = lane; i <= k; i += 32) {
      const dq r = col[i];
      const size_t o = (size_t)k * l + i;
      for (int cp = 0; cp < 4; ++cp) R[cp * ll + o] = d32_to(dq_get(r, cp));
    }
  }
  __threadfence();
  cluster.sync();
  __shared__ double D[4][CB][CB];
  __shared__ double X[4][CB][CB];
  __shared__ double rpv[CB];
  const int nblk = (l + CB - 1) / CB;
  for (int J = c; J < nblk; J += nc) {
    const int j0 = J * CB, b = min(CB, l - j0);
    for (int e = t; e < CB * CB; e += blockDim.x) {
      const int i = e % CB, jj = e / CB;
      for (int cp = 0; cp < 4; ++cp)
        D[cp][i][jj] = (i < b && jj < b && i <= jj) ? __ldcg(R + cp * ll + (size_t)(j0 + jj) * l + j0 + i) : 0.0;
    }
    __syncthreads();
    cc_block_inverse(D, X, rpv, b);
    double* Dinv = Dinv_all + (size_t)J * 4 * CB * CB;
    for (int e = t; e < b * b; e += blockDim.x) {
      const int i = e % b, jj = e / b;
      for (int cp = 0; cp < 4; ++cp) Dinv[(size_t)cp * b * b + (size_t)jj * b + i] = (i <= jj) ? X[cp][i][jj] : 0.0;
    }
    __syncthreads();
  }
}

// Panel rows: R[j0+r, k] = sum_{s <= r} conj(Dinv[s, r]) Wm[j0+s, k], one warp per column k >= j1.
__global__ void chol_panel_kernel(const double* __restrict__ Wm, double* __restrict__ R, int l, int j0, int b,
                                  const double* __restrict__ Dinv, const int* run_if) {
  if (run_if && *run_if == 0) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  const int j1 = j0 + b;
  const int k = j1 + warp;
  if (k >= l || lane >= b) return;
  const size_t ll = (size_t)l * l, bb = (size_t)b * b;
  const int r = lane;
  Quat<double> acc = {0, 0, 0, 0};
  for (int sidx = 0; sidx <= r; ++sidx) {
    Quat<double> dv = {Dinv[(size_t)r * b + sidx], Dinv[bb + (size_t)r * b + sidx], Dinv[2 * bb + (size_t)r * b + sidx],
                       Dinv[3 * bb + (size_t)r * b + sidx]};
    const size_t o = (size_t)k * l + j0 + sidx;
    Quat<double> w = {Wm[o], Wm[ll + o], Wm[2 * ll + o], Wm[3 * ll + o]};
    Quat<double> pr = qcmul(dv, w);
    acc.w += pr.w; acc.x += pr.x; acc.y += pr.y; acc.z += pr.z;
  }
  const size_t o = (size_t)k * l + j0 + r;
  R[o] = acc.w; R[ll + o] = acc.x; R[2 * ll + o] = acc.y; R[3 * ll + o] = acc.z;
}

// Trailing update of the upper triangle: Wm[i, k] -= sum_{t in panel} conj(R[t, i]) R[t, k].
__global__ void __launch_bounds__(64) chol_update_kernel(double* __restrict__ Wm, const double* __restrict__ R, int l,
                                                          int j0, int b, const int* run_if) {
  if (run_if && *run_if == 0) return;
  __shared__ double Pi[4][CB][CT];
  __shared__ double Pk[4][CB][CT];
  const int j1 = j0 + b;
  const int2 tl = upper_tri_entry((int)blockIdx.x);
  const int i0 = j1 + tl.x * CT, k0 = j1 + tl.y * CT;
  const size_t ll = (size_t)l * l;
  const int t = threadIdx.x;
  for (int e = t; e < CB * CT; e += blockDim.x) {
    const int r = e % CB, c0 = e / CB;
    for (int c = 0; c < 4; ++c) {
      Pi[c][r][c0] = (r < b && i0 + c0 < l) ? R[c * ll + (size_t)(i0 + c0) * l + j0 + r] : 0.0;
      Pk[c][r][c0] = (r < b && k0 + c0 < l) ? R[c * ll + (size_t)(k0 + c0) * l + j0 + r] : 0.0;
    }
  }
  __syncthreads();
  const int ii = t % CT, kk = t / CT;
  const int i = i0 + ii, k = k0 + kk;
  if (i >= l || k >= l || i > k) return;
  Quat<double> acc = {0, 0, 0, 0};
  for (int r = 0; r < b; ++r) {
    Quat<double> pr = qcmul(Quat<double>{Pi[0][r][ii], Pi[1][r][ii], Pi[2][r][ii], Pi[3][r][ii]},
                            Quat<double>{Pk[0][r][kk], Pk[1][r][kk], Pk[2][r][kk], Pk[3][r][kk]});
    acc.w += pr.w; acc.x += pr.x; acc.y += pr.y; acc.z += pr.z;
  }
  const size_t o = (size_t)k * l + i;
  Wm[o] -= acc.w; Wm[ll + o] -= acc.x; Wm[2 * ll + o] -= acc.y; Wm[3 * ll + o] -= acc.z;
}

// Inverse of an upper-triangular quaternion matrix, one CTA per column j (back substitution
// with block-wide dot products).
__global__ void __launch_bounds__(256) tri_inv_col_kernel(const double* __restrict__ R, double* __restrict__ X, int l) {
  extern __shared__ double xs[];   // 4 * l
  __shared__ double red[4][8];
  const int j = blockIdx.x, t = threadIdx.x, lane = t % 32, warp = t / 32, nw = blockDim.x / 32;
  const size_t ll = (size_t)l * l;
  for (int i = t; i < l; i += blockDim.x) xs[i] = xs[l + i] = xs[2 * l + i] = xs[3 * l + i] = 0.0;
  __syncthreads();
  if (t == 0) xs[j] = 1.0 / R[(size_t)j * l + j];
  __syncthreads();
  for (int i = j - 1; i >= 0; --i) {
    Quat<double> sacc = {0, 0, 0, 0};
    for (int q = i + 1 + t; q <= j; q += blockDim.x) {
      Quat<double> pr = qmul(ld_small(R, l, i, q), Quat<double>{xs[q], xs[l + q], xs[2 * l + q], xs[3 * l + q]});
      sacc.w += pr.w; sacc.x += pr.x; sacc.y += pr.y; sacc.z += pr.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sacc.w += __shfl_xor_sync(0xffffffffu, sacc.w, o);
      sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, o);
      sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, o);
      sacc.z += __shfl_xor_sync(0xffffffffu, sacc.z, o);
    }
    if (lane == 0) { red[0][warp] = sacc.w; red[1][warp] = sacc.x; red[2][warp] = sacc.y; red[3][warp] = sacc.z; }
    __syncthreads();
    if (t == 0) {
      Quat<double> s = {0, 0, 0, 0};
      for (int w = 0; w < nw; ++w) { s.w += red[0][w]; s.x += red[1][w]; s.y += red[2][w]; s.z += red[3][w]; }
      const double ninv = -1.0 / R[(size_t)i * l + i];
      xs[i] = s.w * ninv; xs[l + i] = s.x * ninv; xs[2 * l + i] = s.y * ninv; xs[3 * l + i] = s.z * ninv;
    }
    __syncthreads();
  }
  for (int i = t; i < l; i += blockDim.x)
    for (int c = 0; c < 4; ++c) X[c * ll + (size_t)j * l + i] = xs[(size_t)c * l + i];
}


// Inverse of the upper-triangular R from its diagonal-block inverses (Dinv_I, one per panel of
// width CB): column j of X = R^{-1} by block back substitution, one CTA per column:
//   x_J = Dinv_J e_j,   x_I = -Dinv_I (sum_{q in blocks I+1..J} R[I, q] x_q)   for I = J-1 .. 0.
__global__ void __launch_bounds__(256) tri_inv_blocked_kernel(const double* __restrict__ R, const double* __restrict__ Dinv,
                                                               double* __restrict__ X, int l, const int* run_if) {
  // Column j of X = R^{-1} by block back substitution, x_I = -Dinv_I sum_{q > block I} R[I, q] x_q.
  // FP64 results take ~200 cycles each on this part, so every sum is a shuffle tree over 16 lanes
  // (depth 4) instead of a serial chain: lane ch of row r's half-warp takes q = q0 + ch, q0 + ch +
  // 16, ...; the 16 x 16 triangular product with Dinv_I runs as lane (r, q).
  if (run_if && *run_if == 0) return;
  extern __shared__ double xs[];          // 4 * l
  __shared__ double tsum[4][CB];
  const int j = blockIdx.x, t = threadIdx.x;
  const size_t ll = (size_t)l * l;
  const int J = j / CB;
  const int r = t >> 4, ch = t & 15;      // 16 rows x 16 lanes = 256 threads
  for (int i = t; i < l; i += blockDim.x) xs[i] = xs[l + i] = xs[2 * l + i] = xs[3 * l + i] = 0.0;
  __syncthreads();
  {   // x_J = Dinv_J[:, j - J*CB]
    const int bJ = min(CB, l - J * CB), jj = j - J * CB;
    const double* D = Dinv + (size_t)J * 4 * CB * CB;
    const size_t bb = (size_t)bJ * bJ;
    if (t < bJ && t <= jj) {
      const size_t o = (size_t)jj * bJ + t;
      xs[J * CB + t] = D[o]; xs[l + J * CB + t] = D[bb + o]; xs[2 * l + J * CB + t] = D[2 * bb + o];
      xs[3 * l + J * CB + t] = D[3 * bb + o];
    }
  }
  __syncthreads();
  for (int I = J - 1; I >= 0; --I) {
    const int i0 = I * CB, q0 = (I + 1) * CB;
    Quat<double> acc = {0, 0, 0, 0};
    for (int q = q0 + ch; q <= j; q += 16) {
      const Quat<double> pr = qmul(ld_small(R, l, i0 + r, q), Quat<double>{xs[q], xs[l + q], xs[2 * l + q], xs[3 * l + q]});
      acc.w += pr.w; acc.x += pr.x; acc.y += pr.y; acc.z += pr.z;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {      // the 16 lanes of row r are one half-warp
      acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
    }
    if (ch == 0) { tsum[0][r] = acc.w; tsum[1][r] = acc.x; tsum[2][r] = acc.y; tsum[3][r] = acc.z; }
    __syncthreads();
    // x_I[r] = -sum_{q >= r} Dinv_I[r][q] T[q]: lane (r, q)
    {
      const double* D = Dinv + (size_t)I * 4 * CB * CB;
      const size_t bb = (size_t)CB * CB;
      const int q = ch;
      Quat<double> pr = {0, 0, 0, 0};
      if (q >= r) {
        const size_t o = (size_t)q * CB + r;
        pr = qmul(Quat<double>{D[o], D[bb + o], D[2 * bb + o], D[3 * bb + o]},
                  Quat<double>{tsum[0][q], tsum[1][q], tsum[2][q], tsum[3][q]});
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        pr.w += __shfl_xor_sync(0xffffffffu, pr.w, o);
        pr.x += __shfl_xor_sync(0xffffffffu, pr.x, o);
        pr.y += __shfl_xor_sync(0xffffffffu, pr.y, o);
        pr.z += __shfl_xor_sync(0xffffffffu, pr.z, o);
      }
      if (ch == 0) { xs[i0 + r] = -pr.w; xs[l + i0 + r] = -pr.x; xs[2 * l + i0 + r] = -pr.y; xs[3 * l + i0 + r] = -pr.z; }
    }
    __syncthreads();
  }
  for (int i = t; i < l; i += blockDim.x)
    for (int c = 0; c < 4; ++c) X[c * ll + (size_t)j * l + i] = xs[(size_t)c * l + i];
}


// ---------------------------------------------------------------------------------------
// Second CholeskyQR step by series.  After the first step Q' = Y R1^{-1} is orthonormal up to
// E = Q'^H Q' - I with |E| of order u32 kappa(Y).  The Cholesky factor of I + E is I + F with F
// upper triangular and real diagonal; (I + F)^H (I + F) = I + E is equivalent to
// F = Phi(E - F^H F), Phi(X) = strict upper part of X plus half its (real) diagonal, a fixed point
// reached by iterating from F = Phi(E) (the error shrinks like |E|^(n+1)).  The inverse is
// (I + F)^{-1} = I + D with D = -F - F D (the Neumann series I - F + F^2 - ...), iterated from
// D = 0.  Each step is a triangular product spread over all SMs -- no serial pivots.  Both
// iterations contract with rate of order |E|, so a step whose predecessor changed no entry by
// more than SERIES_TOL (far below the FP64 resolution of I + F) only copies its input forward.
// The init kernel raises `use_chol` when l * max|E_ij| exceeds SERIES_MAX; the blocked Cholesky
// kernels then run instead (they are predicated on that flag, so no host synchronisation is
// needed).
//
// Both products, F^H F and F D, are products of two matrices of order |E|, and their sums are
// subtracted from E (or -F) in FP64.  For FP32 sketches they are accumulated in FP32 (TAcc =
// float): the absolute error is of order l |E|^2 2^-24 (below 4e-15 at the SERIES_MAX limit,
// under the 2^-45-class error of the Gram itself), and the steps stop being FP64-bound.  FP64
// sketches accumulate in FP64.
constexpr double SERIES_MAX = 5e-3;
constexpr double SERIES_TOL = 1e-18;
constexpr int SERIES_ITERS = 6, NEUMANN_ITERS = 7;
constexpr int SPLIT = 16;   // lanes per entry: sums as short per-lane chains plus a shuffle tree

__global__ void series_init_kernel(const double* __restrict__ G, double* __restrict__ E, double* __restrict__ F, int l,
                                   unsigned long long* __restrict__ emax_bits) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)l * l) return;
  const int i = (int)(idx % l), j = (int)(idx / l);
  Quat<double> e = ld_small(G, l, i, j);
  if (i == j) e.w -= 1.0;
  st_small(E, l, i, j, e);
  Quat<double> f = {0, 0, 0, 0};
  if (i < j) f = e;
  else if (i == j) f.w = 0.5 * e.w;
  st_small(F, l, i, j, f);
  const double mx = fmax(fmax(fabs(e.w), fabs(e.x)), fmax(fabs(e.y), fabs(e.z)));
  atomicMax(emax_bits, (unsigned long long)__double_as_longlong(mx));
}

__global__ void series_decide_kernel(const unsigned long long* __restrict__ emax_bits, int l, int* use_chol) {
  const double emax = __longlong_as_double((long long)*emax_bits);
  *use_chol = (!(emax * l <= SERIES_MAX)) ? 1 : 0;
}

template <class TA>
__device__ __forceinline__ Quat<TA> ld_small_as(const double* M, int l, int i, int j) {
  const Quat<double> q = ld_small(M, l, i, j);
  return {(TA)q.w, (TA)q.x, (TA)q.y, (TA)q.z};
}

// out(i, j) for i <= j with SPLIT threads per entry:
//   mode 0 (series):  Phi(E - F^H F)(i, j),  (F^H F)_ij = sum_{t <= i} conj(F_ti) F_tj
//   mode 1 (Neumann): (-F - F D)_ij,          (F D)_ij  = sum_{i <= t <= j} F_it D_tj
// The largest change against the step's
// input (F in mode 0, D in mode 1) goes to *delta; when the previous step's change *prev_delta is
// at most SERIES_TOL the input is copied unchanged.  `add_identity` stores I + out (the last
// Neumann step writes R2^{-1} = I + D).
template <class TA>
__global__ void __launch_bounds__(128) series_step_kernel(const double* __restrict__ E, const double* __restrict__ F,
                                                           const double* __restrict__ D, double* __restrict__ out, int l,
                                                           int mode, int nentries, int add_identity,
                                                           const unsigned long long* __restrict__ prev_delta,
                                                           unsigned long long* __restrict__ delta) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ent = gt / SPLIT;
  const int part = (int)(gt % SPLIT);
  const bool valid = ent < nentries;
  const double* in = (mode == 0) ? F : D;
  int i = 0, j = 0;
  if (valid) {
    const int2 ij = upper_tri_entry((int)ent);
    i = ij.x;
    j = ij.y;
  }
  if (prev_delta && __longlong_as_double((long long)*prev_delta) <= SERIES_TOL) {
    if (valid && part == 0) {
      Quat<double> o = ld_small(in, l, i, j);
      if (add_identity && i == j) o.w += 1.0;
      st_small(out, l, i, j, o);
    }
    return;
  }
  Quat<TA> acc = {0, 0, 0, 0};
  if (valid) {
    if (mode == 0) {
#pragma unroll 4
      for (int t = part; t <= i; t += SPLIT) {
        Quat<TA> pr = qcmul(ld_small_as<TA>(F, l, t, i), ld_small_as<TA>(F, l, t, j));
        acc.w += pr.w; acc.x += pr.x; acc.y += pr.y; acc.z += pr.z;
      }
    } else {
#pragma unroll 4
      for (int t = i + part; t <= j; t += SPLIT) {
        Quat<TA> pr = qmul(ld_small_as<TA>(F, l, i, t), ld_small_as<TA>(D, l, t, j));
        acc.w += pr.w; acc.x += pr.x; acc.y += pr.y; acc.z += pr.z;
      }
    }
  }
#pragma unroll
  for (int o = SPLIT / 2; o > 0; o >>= 1) {
    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
  }
  double ch = 0.0;
  if (valid && part == 0) {
    Quat<double> r;
    if (mode == 0) {
      const Quat<double> e = ld_small(E, l, i, j);
      if (i < j) r = {e.w - (double)acc.w, e.x - (double)acc.x, e.y - (double)acc.y, e.z - (double)acc.z};
      else r = {0.5 * (e.w - (double)acc.w), 0.0, 0.0, 0.0};
    } else {
      const Quat<double> f = ld_small(F, l, i, j);
      r = {-f.w - (double)acc.w, -f.x - (double)acc.x, -f.y - (double)acc.y, -f.z - (double)acc.z};
    }
    const Quat<double> o = ld_small(in, l, i, j);
    ch = fmax(fmax(fabs(r.w - o.w), fabs(r.x - o.x)), fmax(fabs(r.y - o.y), fabs(r.z - o.z)));
    if (add_identity && i == j) r.w += 1.0;
    st_small(out, l, i, j, r);
  }
  // warp maximum, one atomic per warp (non-negative doubles order like their bit patterns)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ch = fmax(ch, __shfl_xor_sync(0xffffffffu, ch, o));
  if ((threadIdx.x & 31) == 0) atomicMax(delta, (unsigned long long)__double_as_longlong(ch));
}

// R2 = I + F (full matrix written; lower part zero)
__global__ void series_form_kernel(const double* __restrict__ F, double* __restrict__ R2, int l) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)l * l) return;
  const int i = (int)(idx % l), j = (int)(idx / l);
  Quat<double> f = (i <= j) ? ld_small(F, l, i, j) : Quat<double>{0, 0, 0, 0};
  if (i == j) f.w += 1.0;
  st_small(R2, l, i, j, f);
}

// ---------------------------------------------------------------------------------------
// Grouped steps of batch plans: one launch runs one orthonormalisation step for every problem
// of the plan (item tables map each CTA to its problem and tile).  The small operands are FP32
// or double-FP32 throughout, so no FP64 instruction runs on this path.

// s + e += a b for double-FP32 a = ah + al, b = bh + bl: the high product is split exactly by an
// FMA, its rounded part added into s by a two-sum (Knuth), and every low-order term collected in
// e (renormalised once per entry, after four products).
__device__ __forceinline__ void d32_acc(float& s, float& e, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -p);
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  const float t = __fadd_rn(s, p);
  const float v = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, v)), __fsub_rn(p, v));
  s = t;
  e = __fadd_rn(e, __fadd_rn(err, pe));
}
__device__ __forceinline__ void d32_renorm(float s, float e, float& h, float& l) {
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// A double-FP32 quaternion in shared memory: high and low parts, components (real, i, j, k) in
// (x, y, z, w).
struct DQ {
  float4 h, l;
};

// w <- w - conj(a) b (component signs of conj(a) b as in qcmul).
__device__ __forceinline__ void dq_fms_conj(DQ& w, const DQ& a, const DQ& b) {
  float s, e;
  s = w.h.x; e = w.l.x;
  d32_acc(s, e, -a.h.x, -a.l.x, b.h.x, b.l.x); d32_acc(s, e, -a.h.y, -a.l.y, b.h.y, b.l.y);
  d32_acc(s, e, -a.h.z, -a.l.z, b.h.z, b.l.z); d32_acc(s, e, -a.h.w, -a.l.w, b.h.w, b.l.w);
  d32_renorm(s, e, w.h.x, w.l.x);
  s = w.h.y; e = w.l.y;
  d32_acc(s, e, -a.h.x, -a.l.x, b.h.y, b.l.y); d32_acc(s, e, a.h.y, a.l.y, b.h.x, b.l.x);
  d32_acc(s, e, a.h.z, a.l.z, b.h.w, b.l.w); d32_acc(s, e, -a.h.w, -a.l.w, b.h.z, b.l.z);
  d32_renorm(s, e, w.h.y, w.l.y);
  s = w.h.z; e = w.l.z;
  d32_acc(s, e, -a.h.x, -a.l.x, b.h.z, b.l.z); d32_acc(s, e, -a.h.y, -a.l.y, b.h.w, b.l.w);
  d32_acc(s, e, a.h.z, a.l.z, b.h.x, b.l.x); d32_acc(s, e, a.h.w, a.l.w, b.h.y, b.l.y);
  d32_renorm(s, e, w.h.z, w.l.z);
  s = w.h.w; e = w.l.w;
  d32_acc(s, e, -a.h.x, -a.l.x, b.h.w, b.l.w); d32_acc(s, e, a.h.y, a.l.y, b.h.z, b.l.z);
  d32_acc(s, e, -a.h.z, -a.l.z, b.h.y, b.l.y); d32_acc(s, e, a.h.w, a.l.w, b.h.x, b.l.x);
  d32_renorm(s, e, w.h.w, w.l.w);
}

__device__ __forceinline__ Quat<float> q_of(const float4& v) { return {v.x, v.y, v.z, v.w}; }

// s + e += a b for double-FP32 quaternions a = ah + al, b = bh + bl (Hamilton product, eq. 1),
// components (real, i, j, k) at indices 0..3.
__device__ __forceinline__ void dq_mul_acc(float (&s)[4], float (&e)[4], const float (&ah)[4], const float (&al)[4],
                                           const float (&bh)[4], const float (&bl)[4]) {
  d32_acc(s[0], e[0], ah[0], al[0], bh[0], bl[0]); d32_acc(s[0], e[0], -ah[1], -al[1], bh[1], bl[1]);
  d32_acc(s[0], e[0], -ah[2], -al[2], bh[2], bl[2]); d32_acc(s[0], e[0], -ah[3], -al[3], bh[3], bl[3]);
  d32_acc(s[1], e[1], ah[0], al[0], bh[1], bl[1]); d32_acc(s[1], e[1], ah[1], al[1], bh[0], bl[0]);
  d32_acc(s[1], e[1], ah[2], al[2], bh[3], bl[3]); d32_acc(s[1], e[1], -ah[3], -al[3], bh[2], bl[2]);
  d32_acc(s[2], e[2], ah[0], al[0], bh[2], bl[2]); d32_acc(s[2], e[2], -ah[1], -al[1], bh[3], bl[3]);
  d32_acc(s[2], e[2], ah[2], al[2], bh[0], bl[0]); d32_acc(s[2], e[2], ah[3], al[3], bh[1], bl[1]);
  d32_acc(s[3], e[3], ah[0], al[0], bh[3], bl[3]); d32_acc(s[3], e[3], ah[1], al[1], bh[2], bl[2]);
  d32_acc(s[3], e[3], -ah[2], -al[2], bh[1], bl[1]); d32_acc(s[3], e[3], ah[3], al[3], bh[0], bl[0]);
}

// Renormalise the four (s, e) sums and add them over the 16 lanes of a half-warp (all 32 lanes
// of the warp take part in the shuffles).
__device__ __forceinline__ void dq_halfwarp_sum(const float (&s)[4], const float (&e)[4], d32 (&v)[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) d32_renorm(s[c], e[c], v[c].h, v[c].l);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const d32 w = {__shfl_xor_sync(0xffffffffu, v[c].h, o), __shfl_xor_sync(0xffffffffu, v[c].l, o)};
      v[c] = d32_add(v[c], w);
    }
  }
}

// FP64 values split into double-FP32 pairs: hi = fl32(x), lo = fl32(x - hi), for two arrays in
// one launch (a triangular factor and its diagonal-block inverses).
__global__ void split_d32_kernel(const double* __restrict__ a, float* __restrict__ ah, float* __restrict__ al, int64_t na,
                                 const double* __restrict__ b, float* __restrict__ bh, float* __restrict__ bl, int64_t nb,
                                 const int* run_if) {
  if (run_if && *run_if == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = (i < na) ? a[i] : b[i - na];
    const float h = __double2float_rn(x);
    const float lo = __double2float_rn(x - (double)h);
    if (i < na) { ah[i] = h; al[i] = lo; } else { bh[i - na] = h; bl[i - na] = lo; }
  }
}

// Double-FP32 form of tri_inv_blocked_kernel (same block back substitution, same lane layout) for
// the factors of FP32 sketches' Grams, whose Cholesky already ran in double-FP32: R and the
// diagonal-block inverses come as high/low FP32 planes, every product is an exact FMA product
// summed by two-sums, so no FP64 instruction issues in the loops (the FP64 form is bound by the
// FP64 pipe's few DFMA per clock per SM).
__global__ void __launch_bounds__(256) tri_inv_blocked_df_kernel(const float* __restrict__ Rh, const float* __restrict__ Rl,
                                                                  const float* __restrict__ Dh, const float* __restrict__ Dl,
                                                                  double* __restrict__ X, int l, const int* run_if) {
  if (run_if && *run_if == 0) return;
  extern __shared__ float xsf[];          // 8 * l: high parts of the four planes of x, then low parts
  float* xh = xsf;
  float* xl = xsf + 4 * l;
  __shared__ float th[4][CB], tl[4][CB];
  const int j = blockIdx.x, t = threadIdx.x;
  const size_t ll = (size_t)l * l;
  const int J = j / CB;
  const int r = t >> 4, ch = t & 15;      // 16 rows x 16 lanes = 256 threads
  for (int i = t; i < 4 * l; i += blockDim.x) xh[i] = xl[i] = 0.f;
  __syncthreads();
  {   // x_J = Dinv_J[:, j - J*CB]
    const int bJ = min(CB, l - J * CB), jj = j - J * CB;
    const size_t base = (size_t)J * 4 * CB * CB;
    const size_t bb = (size_t)bJ * bJ;
    if (t < bJ && t <= jj) {
      const size_t o = base + (size_t)jj * bJ + t;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        xh[c * l + J * CB + t] = Dh[o + c * bb];
        xl[c * l + J * CB + t] = Dl[o + c * bb];
      }
    }
  }
  __syncthreads();
  for (int I = J - 1; I >= 0; --I) {
    const int i0 = I * CB, q0 = (I + 1) * CB;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
    for (int q = q0 + ch; q <= j; q += 16) {
      const size_t o = (size_t)q * l + i0 + r;
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        ah[c] = Rh[c * ll + o]; al[c] = Rl[c * ll + o];
        bh[c] = xh[c * l + q]; bl[c] = xl[c * l + q];
      }
      dq_mul_acc(s, e, ah, al, bh, bl);
    }
    d32 v[4];
    dq_halfwarp_sum(s, e, v);
    if (ch == 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) { th[c][r] = v[c].h; tl[c][r] = v[c].l; }
    }
    __syncthreads();
    // x_I[r] = -sum_{q >= r} Dinv_I[r][q] T[q]: lane (r, q)
    {
      const size_t base = (size_t)I * 4 * CB * CB;
      const size_t bb = (size_t)CB * CB;
      const int q = ch;
      float s2[4] = {0.f, 0.f, 0.f, 0.f}, e2[4] = {0.f, 0.f, 0.f, 0.f};
      if (q >= r) {
        const size_t o = base + (size_t)q * CB + r;
        float ah[4], al[4], bh[4], bl[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          ah[c] = Dh[o + c * bb]; al[c] = Dl[o + c * bb];
          bh[c] = th[c][q]; bl[c] = tl[c][q];
        }
        dq_mul_acc(s2, e2, ah, al, bh, bl);
      }
      d32 w[4];
      dq_halfwarp_sum(s2, e2, w);
      if (ch == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) { xh[c * l + i0 + r] = -w[c].h; xl[c * l + i0 + r] = -w[c].l; }
      }
    }
    __syncthreads();
  }
  for (int i = t; i < l; i += blockDim.x)
    for (int c = 0; c < 4; ++c) X[c * ll + (size_t)j * l + i] = (double)xh[c * l + i] + (double)xl[c * l + i];
}

// One CTA per problem: the whole quaternion Cholesky factorisation of G (+ shift I) in
// double-FP32, right-looking over the packed upper triangle in shared memory (column k at offset
// k (k + 1) / 2), with the rank-1 updates' entries enumerated densely over all threads.  Then,
// from the factor's high parts, R^{-1} in FP32 (columns are independent: one warp per column
// solves R x = e_j by column-oriented back substitution) and R Rprev (or R) in FP32.
constexpr int CG_THREADS = 512;

__global__ void __launch_bounds__(CG_THREADS) chol_df_grouped_kernel(const qlr::CholGroupArgs* __restrict__ args,
                                                                    int* err) {
  const qlr::CholGroupArgs& a = args[blockIdx.x];
  const int l = a.l;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DQ* W = reinterpret_cast<DQ*>(smem_raw);
  const int ntri = l * (l + 1) / 2;
  float* rdiag_inv = reinterpret_cast<float*>(W + ntri);   // 1 / r_jj
  __shared__ float s_trace;
  __shared__ d32 s_rp;
  const int t = threadIdx.x, lane = t % 32, warp = t / 32, nwarps = CG_THREADS / 32;
  auto at = [&](int i, int k) -> DQ& { return W[k * (k + 1) / 2 + i]; };
  for (int e = t; e < ntri; e += CG_THREADS) {
    const int2 ik = upper_tri_entry(e);
    const float4* g = reinterpret_cast<const float4*>(a.G + 8 * ((size_t)ik.y * l + ik.x));
    W[e].h = g[0];
    W[e].l = g[1];
  }
  __syncthreads();
  if (a.shift_coef != 0.f) {   // shift s = shift_coef * trace(G) on the diagonal
    if (warp == 0) {
      float tr = 0.f;
      for (int i = lane; i < l; i += 32) tr += at(i, i).h.x;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
      if (lane == 0) s_trace = tr;
    }
    __syncthreads();
    const float sh = a.shift_coef * s_trace;
    for (int i = t; i < l; i += CG_THREADS) {
      DQ& d = at(i, i);
      const d32 v = d32_add({d.h.x, d.l.x}, {sh, 0.f});
      d.h.x = v.h;
      d.l.x = v.l;
    }
    __syncthreads();
  }
  for (int j = 0; j < l; ++j) {
    if (t == 0) {
      DQ& dj = at(j, j);
      d32 d = {dj.h.x, dj.l.x};
      if (!(d.h > 0.f)) {
        qlr_set_error(err, QLR_ENOTPD);
        d = {1e-30f, 0.f};
      }
      const d32 rp = d32_rsqrt(d);
      s_rp = rp;
      const d32 r = d32_mul(d, rp);
      dj.h = make_float4(r.h, 0.f, 0.f, 0.f);
      dj.l = make_float4(r.l, 0.f, 0.f, 0.f);
      rdiag_inv[j] = 1.f / r.h;
    }
    __syncthreads();
    const d32 rp = s_rp;
    for (int k = j + 1 + t; k < l; k += CG_THREADS) {   // row j of R
      DQ& w = at(j, k);
      d32 v;
      v = d32_mul({w.h.x, w.l.x}, rp); w.h.x = v.h; w.l.x = v.l;
      v = d32_mul({w.h.y, w.l.y}, rp); w.h.y = v.h; w.l.y = v.l;
      v = d32_mul({w.h.z, w.l.z}, rp); w.h.z = v.h; w.l.z = v.l;
      v = d32_mul({w.h.w, w.l.w}, rp); w.h.w = v.h; w.l.w = v.l;
    }
    __syncthreads();
    const int n = l - j - 1;
    const int npairs = n * (n + 1) / 2;
    for (int e = t; e < npairs; e += CG_THREADS) {
      const int2 ik = upper_tri_entry(e);
      const int i = j + 1 + ik.x, k = j + 1 + ik.y;
      dq_fms_conj(at(i, k), at(j, i), at(j, k));
    }
    __syncthreads();
  }
  const size_t ll = (size_t)l * l;
  float* Rinv = a.Rinv;
  if (Rinv) {
    for (int j = warp; j < l; j += nwarps) {
      Quat<float> x[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) x[u] = {(lane + 32 * u == j) ? 1.f : 0.f, 0.f, 0.f, 0.f};
      for (int i = j; i >= 0; --i) {
        const int src = i & 31, slot = i >> 5;
        Quat<float> xi = (slot == 0) ? x[0] : (slot == 1 ? x[1] : x[2]);
        const float ri = rdiag_inv[i];
        xi.w = __shfl_sync(0xffffffffu, xi.w, src) * ri;
        xi.x = __shfl_sync(0xffffffffu, xi.x, src) * ri;
        xi.y = __shfl_sync(0xffffffffu, xi.y, src) * ri;
        xi.z = __shfl_sync(0xffffffffu, xi.z, src) * ri;
        if (lane == src) {
          if (slot == 0) x[0] = xi;
          else if (slot == 1) x[1] = xi;
          else x[2] = xi;
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int r = lane + 32 * u;
          if (r < i) {
            const Quat<float> pr = qmul(q_of(at(r, i).h), xi);
            x[u].w -= pr.w; x[u].x -= pr.x; x[u].y -= pr.y; x[u].z -= pr.z;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int r = lane + 32 * u;
        if (r < l) {
          const bool up = (r <= j);
          const size_t o = (size_t)j * l + r;
          Rinv[o] = up ? x[u].w : 0.f;
          Rinv[ll + o] = up ? x[u].x : 0.f;
          Rinv[2 * ll + o] = up ? x[u].y : 0.f;
          Rinv[3 * ll + o] = up ? x[u].z : 0.f;
        }
      }
    }
  }
  float* Rout = a.Rout;
  const float* Rprev = a.Rprev;
  if (Rout) {
    for (int e = t; e < (int)ll; e += CG_THREADS) {
      const int i = e % l, j = e / l;
      Quat<float> acc = {0.f, 0.f, 0.f, 0.f};
      if (i <= j) {
        if (Rprev) {
          for (int tt = i; tt <= j; ++tt) {
            const size_t o = (size_t)j * l + tt;
            const Quat<float> pr = qmul(q_of(at(i, tt).h), Quat<float>{Rprev[o], Rprev[ll + o], Rprev[2 * ll + o], Rprev[3 * ll + o]});
            acc.w += pr.w; acc.x += pr.x; acc.y += pr.y; acc.z += pr.z;
          }
        } else {
          acc = q_of(at(i, j).h);
        }
      }
      Rout[e] = acc.w; Rout[ll + e] = acc.x; Rout[2 * ll + e] = acc.y; Rout[3 * ll + e] = acc.z;
    }
  }
}

// The same grouped factorisation in plain FP32 (a packed upper triangle of float4 quaternions),
// for the Gram of the last CholeskyQR2 step, which is formed in FP32 (its input is already nearly
// orthonormal, so its factor is well conditioned): a quarter of the shared memory and a fraction
// of the instructions of the double-FP32 form, 256 threads, several problems per SM.
constexpr int CF_THREADS = 256;

__global__ void __launch_bounds__(CF_THREADS) chol_f32_grouped_kernel(const qlr::CholGroupArgs* __restrict__ args,
                                                                     int* err) {
  const qlr::CholGroupArgs& a = args[blockIdx.x];
  const int l = a.l;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* W = reinterpret_cast<float4*>(smem_raw);
  const int ntri = l * (l + 1) / 2;
  float* rdiag_inv = reinterpret_cast<float*>(W + ntri);
  __shared__ float s_rp;
  const int t = threadIdx.x, lane = t % 32, warp = t / 32, nwarps = CF_THREADS / 32;
  auto at = [&](int i, int k) -> float4& { return W[k * (k + 1) / 2 + i]; };
  for (int e = t; e < ntri; e += CF_THREADS) {
    const int2 ik = upper_tri_entry(e);
    W[e] = *reinterpret_cast<const float4*>(a.G + 8 * ((size_t)ik.y * l + ik.x));
  }
  __syncthreads();
  if (a.shift_coef != 0.f) {   // shift s = shift_coef * trace(G) on the diagonal
    if (warp == 0) {
      float tr = 0.f;
      for (int i = lane; i < l; i += 32) tr += at(i, i).x;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
      if (lane == 0) s_rp = tr;
    }
    __syncthreads();
    const float sh = a.shift_coef * s_rp;
    __syncthreads();
    for (int i = t; i < l; i += CF_THREADS) at(i, i).x += sh;
    __syncthreads();
  }
  for (int j = 0; j < l; ++j) {
    if (t == 0) {
      float d = at(j, j).x;
      if (!(d > 0.f)) {
        qlr_set_error(err, QLR_ENOTPD);
        d = 1e-30f;
      }
      const float r = sqrtf(d);
      at(j, j) = make_float4(r, 0.f, 0.f, 0.f);
      s_rp = 1.f / r;
      rdiag_inv[j] = 1.f / r;
    }
    __syncthreads();
    const float rp = s_rp;
    for (int k = j + 1 + t; k < l; k += CF_THREADS) {   // row j of R
      float4& w = at(j, k);
      w.x *= rp; w.y *= rp; w.z *= rp; w.w *= rp;
    }
    __syncthreads();
    const int n = l - j - 1;
    const int npairs = n * (n + 1) / 2;
    for (int e = t; e < npairs; e += CF_THREADS) {
      const int2 ik = upper_tri_entry(e);
      const int i = j + 1 + ik.x, k = j + 1 + ik.y;
      const Quat<float> pr = qcmul(q_of(at(j, i)), q_of(at(j, k)));
      float4& w = at(i, k);
      w.x -= pr.w; w.y -= pr.x; w.z -= pr.y; w.w -= pr.z;
    }
    __syncthreads();
  }
  const size_t ll = (size_t)l * l;
  float* Rinv = a.Rinv;
  if (Rinv) {
    for (int j = warp; j < l; j += nwarps) {
      Quat<float> x[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) x[u] = {(lane + 32 * u == j) ? 1.f : 0.f, 0.f, 0.f, 0.f};
      for (int i = j; i >= 0; --i) {
        const int src = i & 31, slot = i >> 5;
        Quat<float> xi = (slot == 0) ? x[0] : (slot == 1 ? x[1] : x[2]);
        const float ri = rdiag_inv[i];
        xi.w = __shfl_sync(0xffffffffu, xi.w, src) * ri;
        xi.x = __shfl_sync(0xffffffffu, xi.x, src) * ri;
        xi.y = __shfl_sync(0xffffffffu, xi.y, src) * ri;
        xi.z = __shfl_sync(0xffffffffu, xi.z, src) * ri;
        if (lane == src) {
          if (slot == 0) x[0] = xi;
          else if (slot == 1) x[1] = xi;
          else x[2] = xi;
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int r = lane + 32 * u;
          if (r < i) {
            const Quat<float> pr = qmul(q_of(at(r, i)), xi);
            x[u].w -= pr.w; x[u].x -= pr.x; x[u].y -= pr.y; x[u].z -= pr.z;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int r = lane + 32 * u;
        if (r < l) {
          const bool up = (r <= j);
          const size_t o = (size_t)j * l + r;
          Rinv[o] = up ? x[u].w : 0.f;
          Rinv[ll + o] = up ? x[u].x : 0.f;
          Rinv[2 * ll + o] = up ? x[u].y : 0.f;
          Rinv[3 * ll + o] = up ? x[u].z : 0.f;
        }
      }
    }
  }
  float* Rout = a.Rout;
  const float* Rprev = a.Rprev;
  if (Rout) {
    for (int e = t; e < (int)ll; e += CF_THREADS) {
      const int i = e % l, j = e / l;
      Quat<float> acc = {0.f, 0.f, 0.f, 0.f};
      if (i <= j) {
        if (Rprev) {
          for (int tt = i; tt <= j; ++tt) {
            const size_t o = (size_t)j * l + tt;
            const Quat<float> pr = qmul(q_of(at(i, tt)), Quat<float>{Rprev[o], Rprev[ll + o], Rprev[2 * ll + o], Rprev[3 * ll + o]});
            acc.w += pr.w; acc.x += pr.x; acc.y += pr.y; acc.z += pr.z;
          }
        } else {
          acc = q_of(at(i, j));
        }
      }
      Rout[e] = acc.w; Rout[ll + e] = acc.x; Rout[2 * ll + e] = acc.y; Rout[3 * ll + e] = acc.z;
    }
  }
}

}  // namespace

namespace qlr {

// ---------------------------------------------------------------------------------------
// grouped steps of batch plans

size_t chol_df_grouped_smem(int lmax) { return (size_t)lmax * (lmax + 1) / 2 * sizeof(DQ) + (size_t)lmax * 4 + 64; }

size_t chol_f32_grouped_smem(int lmax) { return (size_t)lmax * (lmax + 1) / 2 * sizeof(float4) + (size_t)lmax * 4 + 64; }

int chol_f32_grouped(qlr_ctx* ctx, const CholGroupArgs* d_args, int count, int lmax) {
  if (count <= 0) return QLR_OK;
  if (lmax > kBatchMaxL) return QLR_EUNSUPPORTED;
  const size_t smem = chol_f32_grouped_smem(lmax);
  QLR_CUDA_TRY(cudaFuncSetAttribute(chol_f32_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  KTimer kt(ctx, QLR_KID_CHOL);
  chol_f32_grouped_kernel<<<count, CF_THREADS, smem, ctx->stream>>>(d_args, ctx->d_err);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

int chol_df_grouped(qlr_ctx* ctx, const CholGroupArgs* d_args, int count, int lmax) {
  if (count <= 0) return QLR_OK;
  if (lmax > kBatchMaxL) return QLR_EUNSUPPORTED;
  const size_t smem = chol_df_grouped_smem(lmax);
  QLR_CUDA_TRY(cudaFuncSetAttribute(chol_df_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  KTimer kt(ctx, QLR_KID_CHOL);
  chol_df_grouped_kernel<<<count, CG_THREADS, smem, ctx->stream>>>(d_args, ctx->d_err);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

static int gram_df32(qlr_ctx* ctx, const qlr_qmat& Y, double* G, WsArena& ws) {
  const int l = (int)Y.cols;
  const int64_t m = Y.rows;
  const int L4 = 4 * l;
  const int nt = (L4 + WT - 1) / WT;
  const int64_t ntiles = (int64_t)nt * (nt + 1) / 2;
  const int target = 3 * (ctx->num_sms > 0 ? ctx->num_sms : 148);
  int64_t chunks = (target + ntiles - 1) / ntiles;
  chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, (m + 63) / 64));
  chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, ((int64_t)64 << 20) / ((int64_t)8 * L4 * L4)));
  int64_t rpc = ((m + chunks - 1) / chunks + WR - 1) / WR * WR;
  chunks = (m + rpc - 1) / rpc;
  size_t mark = ws.off;
  double* part = ws.take<double>((size_t)chunks * L4 * L4);
  if (!ws.ok) return QLR_ENOMEM;
  {
    KTimer kt(ctx, QLR_KID_GRAM);
    dim3 grid((unsigned)ntiles, (unsigned)chunks);
    gram_df_partial_kernel<<<grid, 256, 0, ctx->stream>>>(
        static_cast<const float*>(Y.plane[0]), static_cast<const float*>(Y.plane[1]), static_cast<const float*>(Y.plane[2]),
        static_cast<const float*>(Y.plane[3]), m, l, Y.ld, rpc, part);
    qlr_count_launch();
    QLR_CUDA_TRY(cudaGetLastError());
  }
  {
    KTimer kt(ctx, QLR_KID_GRAM);
    const int64_t tw = (int64_t)L4 * L4;
    if (chunks > 1) {
      gram_df_reduce_kernel<<<(unsigned)((tw + 255) / 256), 256, 0, ctx->stream>>>(part, (int)chunks, L4);
      qlr_count_launch();
    }
    const int64_t tot = (int64_t)l * l;
    gram_df_combine_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, ctx->stream>>>(part, l, G);
    qlr_count_launch();
    QLR_CUDA_TRY(cudaGetLastError());
  }
  ws.off = mark;
  return QLR_OK;
}

int gram(qlr_ctx* ctx, const qlr_qmat& Y, double* G, WsArena& ws) {
  if (Y.dtype == QLR_F32 && Y.cols > 0 && Y.rows > 0) {
    // tensor cores when the workspace holds the slices, else the double-FP32 SIMT Gram
    if (gram_tc_supported(Y) && ws.cap - ws.off >= gram_tc_ws(Y.rows, (int)Y.cols)) return gram_tc(ctx, Y, G, ws);
    return gram_df32(ctx, Y, G, ws);
  }
  const int l = (int)Y.cols;
  const int64_t m = Y.rows;
  if (l == 0) return QLR_OK;
  const int nt = (l + GT - 1) / GT;
  const int64_t ntiles = (int64_t)nt * (nt + 1) / 2;
  int target = 2 * (ctx->num_sms > 0 ? ctx->num_sms : 148);
  int64_t chunks = (target + ntiles - 1) / ntiles;
  chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, (m + 63) / 64));
  chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, ((int64_t)64 << 20) / ((int64_t)32 * l * l)));
  int64_t rpc = ((m + chunks - 1) / chunks + GR - 1) / GR * GR;
  if (rpc == 0) rpc = GR;
  chunks = (m + rpc - 1) / rpc;
  if (chunks == 0) chunks = 1;
  size_t mark = ws.off;
  double* part = ws.take<double>((size_t)chunks * 4 * l * l);
  if (!ws.ok) return QLR_ENOMEM;
  dim3 grid((unsigned)ntiles, (unsigned)chunks);
  KTimer kt(ctx, QLR_KID_GRAM);
  if (Y.dtype == QLR_F64) {
    const double* p[4];
    for (int c = 0; c < 4; ++c) p[c] = static_cast<const double*>(Y.plane[c]);
    gram_partial_kernel<double><<<grid, 256, 0, ctx->stream>>>(p[0], p[1], p[2], p[3], m, l, Y.ld, rpc, part);
    qlr_count_launch();
  } else if (Y.dtype == QLR_F32) {
    const float* p[4];
    for (int c = 0; c < 4; ++c) p[c] = static_cast<const float*>(Y.plane[c]);
    gram_partial_kernel<float><<<grid, 256, 0, ctx->stream>>>(p[0], p[1], p[2], p[3], m, l, Y.ld, rpc, part);
    qlr_count_launch();
  } else {
    return QLR_EINVAL;
  }
  QLR_CUDA_TRY(cudaGetLastError());
  int64_t tot = (int64_t)l * l;
  gram_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(part, (int)chunks, l, G);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  ws.off = mark;  // partials are dead once the reduction is enqueued (stream order)
  return QLR_OK;
}

// Cluster size for chol_cluster_kernel at this shared-memory size: 16 (non-portable) when the
// device can co-schedule it, else 8; 0 when neither fits.
static int cluster_chol_size(int device, int l) {
  static std::mutex mu;
  static std::vector<std::pair<int64_t, int>> cache;   // (device << 32 | l) -> cluster size
  std::lock_guard<std::mutex> lk(mu);
  const int64_t key = ((int64_t)device << 32) | (uint32_t)l;
  for (const auto& e : cache)
    if (e.first == key) return e.second;
  const bool allowed =
      cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(chol_cluster_df_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  cudaGetLastError();
  int pick = 0;
  for (int nc : {16, 8}) {
    if (nc == 16 && !allowed) continue;
    const size_t smem = cc_smem(l, nc);
    if (smem > 200 * 1024) continue;
    if (cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(chol_cluster_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc, 1, 1);
    cfg.blockDim = dim3(CC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, chol_cluster_kernel, &cfg) == cudaSuccess && ncl > 0) {
      pick = nc;
      break;
    }
    cudaGetLastError();
  }
  cache.emplace_back(key, pick);
  return pick;
}

int chol(qlr_ctx* ctx, int l, const double* G, double* R, double shift_coef, WsArena& ws, double* Dinv_all,
         const int* run_if, bool df) {
  if (l == 0) return QLR_OK;
  const size_t ll4 = (size_t)4 * l * l;
  const int nc = (l > CB) ? cluster_chol_size(ctx->device, l) : 0;
  if (nc > 0 && Dinv_all != nullptr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc, 1, 1);
    cfg.blockDim = dim3(CC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = cc_smem(l, nc);
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    KTimer kt(ctx, QLR_KID_CHOL);
    QLR_CUDA_TRY(cudaLaunchKernelEx(&cfg, df ? chol_cluster_df_kernel : chol_cluster_kernel, G, R, Dinv_all, l, shift_coef,
                                    ctx->d_err, run_if));
    qlr_count_launch();
    return QLR_OK;
  }
  size_t mark = ws.off;
  double* Wm = ws.take<double>(ll4);
  const int npan = (l + CB - 1) / CB;
  if (Dinv_all == nullptr) Dinv_all = ws.take<double>((size_t)npan * 4 * CB * CB);
  if (!ws.ok) return QLR_ENOMEM;
  KTimer kt(ctx, QLR_KID_CHOL);
  chol_init_kernel<<<std::max(1, std::min(64, (int)((ll4 / 4 + 255) / 256))), 256, 0, ctx->stream>>>(G, Wm, R, l, shift_coef, run_if);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  for (int j0 = 0; j0 < l; j0 += CB) {
    const int b = std::min(CB, l - j0);
    double* Dinv = Dinv_all + (size_t)(j0 / CB) * 4 * CB * CB;
    chol_diag_kernel<<<1, 256, 0, ctx->stream>>>(Wm, R, l, j0, b, Dinv, ctx->d_err, run_if);
    qlr_count_launch();
    QLR_CUDA_TRY(cudaGetLastError());
    const int rem = l - j0 - b;
    if (rem <= 0) break;
    chol_panel_kernel<<<(rem * 32 + 127) / 128, 128, 0, ctx->stream>>>(Wm, R, l, j0, b, Dinv, run_if);
    qlr_count_launch();
    QLR_CUDA_TRY(cudaGetLastError());
    // tiles (a <= b) of the trailing triangle, coordinates relative to j0 + b
    const int nt = (rem + CT - 1) / CT;
    const int ntiles = nt * (nt + 1) / 2;
    chol_update_kernel<<<ntiles, 64, 0, ctx->stream>>>(Wm, R, l, j0, b, run_if);
    qlr_count_launch();
    QLR_CUDA_TRY(cudaGetLastError());
  }
  ws.off = mark;
  return QLR_OK;
}

int tri_inv(qlr_ctx* ctx, int l, const double* R, double* Rinv, const double* Dinv_all, const int* run_if,
            float* d32buf) {
  if (l == 0) return QLR_OK;
  KTimer kt(ctx, QLR_KID_TRIINV);
  const size_t smem = (size_t)4 * l * sizeof(double);
  if (Dinv_all && d32buf) {
    const int64_t nr = (int64_t)4 * l * l;
    const int64_t nd = (int64_t)((l + CB - 1) / CB) * 4 * CB * CB;
    float* Rh = d32buf;
    float* Rl = Rh + nr;
    float* Dh = Rl + nr;
    float* Dl = Dh + nd;
    const unsigned gs = (unsigned)std::min<int64_t>((nr + nd + 255) / 256, 1024);
    split_d32_kernel<<<gs, 256, 0, ctx->stream>>>(R, Rh, Rl, nr, Dinv_all, Dh, Dl, nd, run_if);
    qlr_count_launch();
    // 8 l floats: the same bytes as the FP64 form's 4 l doubles
    QLR_CUDA_TRY(cudaFuncSetAttribute(tri_inv_blocked_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tri_inv_blocked_df_kernel<<<l, 256, smem, ctx->stream>>>(Rh, Rl, Dh, Dl, Rinv, l, run_if);
    qlr_count_launch();
  } else if (Dinv_all) {
    // static shared memory comes on top of the dynamic size: always opt in
    QLR_CUDA_TRY(cudaFuncSetAttribute(tri_inv_blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tri_inv_blocked_kernel<<<l, 256, smem, ctx->stream>>>(R, Dinv_all, Rinv, l, run_if);
    qlr_count_launch();
  } else {
    // static shared memory comes on top of the dynamic size: always opt in
    QLR_CUDA_TRY(cudaFuncSetAttribute(tri_inv_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tri_inv_col_kernel<<<l, 256, smem, ctx->stream>>>(R, Rinv, l);
    qlr_count_launch();
  }
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

int small_matmul(qlr_ctx* ctx, int l, const double* A, const double* B, double* C) {
  const int64_t thr = (int64_t)l * (l + 1) / 2 * MM_SPLIT;
  KTimer kt(ctx, QLR_KID_MISC);
  small_matmul_kernel<<<(unsigned)((thr + 127) / 128), 128, 0, ctx->stream>>>(A, B, C, l);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

// Q = Y * Rinv (Rinv FP64 small, column-major, l x l)
static int apply_rinv(qlr_ctx* ctx, const qlr_qmat& Y, const double* Rinv, qlr_qmat& Q, WsArena& ws) {
  return thin_times_small(ctx, Y, Rinv, (int)Y.cols, (int)Y.cols, Q, ws, true);
}

// Cholesky factor R2 = I + F of a near-identity Gram matrix G and its inverse by series; sets
// *use_chol_out to a device flag that is non-zero when G is too far from I for the series.
// f32acc: accumulate the small products in FP32 (Grams of FP32 sketches).
static int series_factor(qlr_ctx* ctx, int l, const double* G, double* R2, double* R2inv, WsArena& ws,
                         int** use_chol_out, bool f32acc) {
  const size_t ll4 = (size_t)4 * l * l;
  double* E = ws.take<double>(ll4);
  double* Fa = ws.take<double>(ll4);
  double* Fb = ws.take<double>(ll4);
  double* Xa = ws.take<double>(ll4);
  double* Xb = ws.take<double>(ll4);
  unsigned long long* emax = ws.take<unsigned long long>(1 + SERIES_ITERS + NEUMANN_ITERS);
  unsigned long long* deltas = emax + 1;
  int* use_chol = ws.take<int>(1);
  const int nent = l * (l + 1) / 2;
  if (!ws.ok) return QLR_ENOMEM;
  QLR_CUDA_TRY(cudaMemsetAsync(emax, 0, (1 + SERIES_ITERS + NEUMANN_ITERS) * sizeof(unsigned long long), ctx->stream));
  KTimer kt(ctx, QLR_KID_SERIES);
  const int64_t tot = (int64_t)l * l;
  const unsigned gsq = (unsigned)((tot + 127) / 128);
  const unsigned gst = (unsigned)(((int64_t)nent * SPLIT + 127) / 128);
  series_init_kernel<<<gsq, 128, 0, ctx->stream>>>(G, E, Fa, l, emax);
  qlr_count_launch();
  series_decide_kernel<<<1, 1, 0, ctx->stream>>>(emax, l, use_chol);
  qlr_count_launch();
  auto step = f32acc ? series_step_kernel<float> : series_step_kernel<double>;
  double* Fc = Fa;
  double* Fn = Fb;
  for (int it = 0; it < SERIES_ITERS; ++it) {
    step<<<gst, 128, 0, ctx->stream>>>(E, Fc, nullptr, Fn, l, 0, nent, 0, it ? deltas + it - 1 : nullptr, deltas + it);
    qlr_count_launch();
    std::swap(Fc, Fn);
  }
  series_form_kernel<<<gsq, 128, 0, ctx->stream>>>(Fc, R2, l);
  qlr_count_launch();
  // the Neumann iteration runs on D = X - I from D = 0; its last step writes I + D
  QLR_CUDA_TRY(cudaMemsetAsync(Xa, 0, ll4 * sizeof(double), ctx->stream));
  double* Xc = Xa;
  double* Xn = Xb;
  unsigned long long* nd = deltas + SERIES_ITERS;
  for (int it = 0; it < NEUMANN_ITERS; ++it) {
    const bool last = (it == NEUMANN_ITERS - 1);
    step<<<gst, 128, 0, ctx->stream>>>(nullptr, Fc, Xc, last ? R2inv : Xn, l, 1, nent, last ? 1 : 0,
                                       it ? nd + it - 1 : nullptr, nd + it);
    qlr_count_launch();
    std::swap(Xc, Xn);
  }
  QLR_CUDA_TRY(cudaGetLastError());
  *use_chol_out = use_chol;
  return QLR_OK;
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
  double* Dinv_all = ws.take<double>((size_t)((l + CB - 1) / CB) * 4 * CB * CB);
  // double-FP32 copies of R and Dinv for the triangular inverse of FP32 sketches' factors
  float* d32buf = (Y.dtype == QLR_F32) ? ws.take<float>(2 * ((size_t)4 * l * l + (size_t)((l + CB - 1) / CB) * 4 * CB * CB))
                                       : nullptr;
  const int64_t tld = (m + 3) / 4 * 4;   // 16-byte multiple pitch (tensor-core thin products)
  char* tbuf = ws.take<char>((size_t)4 * tld * l * esz);
  if (!ws.ok) return QLR_ENOMEM;
  qlr_qmat T = Y;
  T.ld = tld;
  T.layout = QLR_COL_MAJOR;
  for (int c = 0; c < 4; ++c) T.plane[c] = tbuf + (size_t)c * tld * l * esz;

  // CholeskyQR2: Y -> T -> Q.  Shifted CholeskyQR3: Y -> Q -> T -> Q.  Span only: Y -> Q (shifted).
  const int steps = (orth == QLR_ORTH_SCHOLQR3) ? 3 : (orth == ORTH_SPAN || orth == ORTH_ONE) ? 1 : 2;
  // FP32 sketches: the Gram is double-FP32, and the Cholesky runs in the same arithmetic
  const bool df = (Y.dtype == QLR_F32);
  const qlr_qmat* seq1[2] = {&Y, &Q};
  const qlr_qmat* seq2[3] = {&Y, &T, &Q};
  const qlr_qmat* seq3[4] = {&Y, &Q, &T, &Q};
  const qlr_qmat* const* seq = (steps == 3) ? seq3 : (steps == 1) ? seq1 : seq2;
  // shift s = 11 (m l + l (l + 1)) u ||Y||_2^2 with u = 2^-53 (FP64 Gram and Cholesky);
  // ||Y||_2^2 is bounded by trace(G), which the Cholesky kernel multiplies in.
  const double shift = (orth == QLR_ORTH_SCHOLQR3 || orth == ORTH_SPAN) ? 11.0 * ((double)m * l + (double)l * (l + 1)) * 1.1102230246251565e-16 : 0.0;
  double* Rprod = P1;
  double* Rnext = P2;
  for (int s = 0; s < steps; ++s) {
    const qlr_qmat& src = *seq[s];
    qlr_qmat& dst = const_cast<qlr_qmat&>(*seq[s + 1]);
    double* Rcur = (s == 0) ? Rprod : Rs;
    QLR_TRY(gram(ctx, src, G, ws));
    if (s == 1 && orth == QLR_ORTH_CHOLQR2) {
      int* use_chol = nullptr;
      QLR_TRY(series_factor(ctx, l, G, Rcur, Rinv, ws, &use_chol, df));
      QLR_TRY(chol(ctx, l, G, Rcur, 0.0, ws, Dinv_all, use_chol, df));     // only if the series test failed
      QLR_TRY(tri_inv(ctx, l, Rcur, Rinv, Dinv_all, use_chol, d32buf));
    } else {
      QLR_TRY(chol(ctx, l, G, Rcur, (s == 0) ? shift : 0.0, ws, Dinv_all, nullptr, df));
      QLR_TRY(tri_inv(ctx, l, Rcur, Rinv, Dinv_all, nullptr, d32buf));
    }
    QLR_TRY(apply_rinv(ctx, src, Rinv, dst, ws));
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
