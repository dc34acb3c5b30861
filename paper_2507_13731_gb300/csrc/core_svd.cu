// Core truncated QSVD of the small l x l factor R: the "Truncated SVD(R, k)" step of
// Algorithms 1, 2 and 4 (QSVD of Def. 1, eq. qsvd).
//
// The QSVD of R is computed through its complex adjoint chi(R) (2l x 2l).  chi(R)'s columns
// come in structured pairs: column l + j is determined by column j (it is J conj(col_j)), and
// the leading l columns are exactly the quaternion columns of R written in complex form.  A
// one-sided (Hestenes) Jacobi that only uses right rotations of the form chi(G) for 2 x 2
// quaternion unitaries G keeps that structure, so it suffices to store and rotate the l leading
// columns -- equivalently, the quaternion columns of W = R.  For a pair of columns (p, q) with
// alpha = |w_p|^2, beta = |w_q|^2 and gamma = w_p^H w_q = |gamma| mu (mu a unit quaternion),
// w_q <- w_q mu* makes the 2 x 2 Gram real, and a real Jacobi rotation then orthogonalises the
// pair.  At convergence W = U diag(sigma); each quaternion singular value of R is one of the
// doubled singular values of chi(R).
//
// The right rotations are accumulated into V (R V = U diag(sigma)), so both vector sets are
// orthonormal to the working precision.  Precision: the sweeps run in T (float or double); a final
// FP64 step evaluates every kept singular value as the two-sided Rayleigh quotient
// sigma = Re(u^H R v) / (|u| |v|) from the FP64 R, whose error is second order in the vectors'.
#include "qlr_internal.h"

namespace {

constexpr int JT = 1024;  // threads of the Jacobi CTA

template <class T>
__device__ __forceinline__ Quat<T> ldw(const T* W, int l, int i, int j) {
  size_t s = (size_t)l * l, o = (size_t)j * l + i;
  return {W[o], W[s + o], W[2 * s + o], W[3 * s + o]};
}
template <class T>
__device__ __forceinline__ void stw(T* W, int l, int i, int j, const Quat<T>& q) {
  size_t s = (size_t)l * l, o = (size_t)j * l + i;
  W[o] = q.w; W[s + o] = q.x; W[2 * s + o] = q.y; W[3 * s + o] = q.z;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Round-robin (circle method) pairing of lp (even) players: round r, pair i.
__device__ __forceinline__ void rr_pair(int lp, int r, int i, int& p, int& q) {
  if (i == 0) {
    p = r % (lp - 1);
    q = lp - 1;
  } else {
    p = (r + i) % (lp - 1);
    q = (r + lp - 1 - i) % (lp - 1);
  }
}

template <class T>
__global__ void __launch_bounds__(JT) jacobi_kernel(const double* __restrict__ R, int l, T* __restrict__ Wout,
                                                     T* __restrict__ Vout, bool w_smem, bool v_smem, int max_sweeps,
                                                     T tol, T* __restrict__ sig_out, int* __restrict__ sweeps_out,
                                                     int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot;
  T* W = w_smem ? reinterpret_cast<T*>(smem_raw) : Wout;
  T* V = v_smem ? reinterpret_cast<T*>(smem_raw) + (w_smem ? 4 * (size_t)l * l : 0) : Vout;
  const int t = threadIdx.x, lane = t % 32, warp = t / 32, nwarps = JT / 32;
  const size_t ll = (size_t)l * l;
  for (size_t e = t; e < 4 * ll; e += JT) {
    W[e] = (T)R[e];
    V[e] = (e < ll && (e % l) == (e / l)) ? (T)1 : (T)0;   // V = I
  }
  __syncthreads();
  const int lp = l + (l & 1);
  int sweep = 0;
  bool converged = (l < 2);
  for (; sweep < max_sweeps && !converged; ++sweep) {
    if (t == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < lp - 1; ++r) {
      for (int pi = warp; pi < lp / 2; pi += nwarps) {
        int p, q;
        rr_pair(lp, r, pi, p, q);
        if (p >= l || q >= l) continue;
        T a = 0, b = 0;
        Quat<T> g = {0, 0, 0, 0};
        for (int i = lane; i < l; i += 32) {
          Quat<T> wp = ldw(W, l, i, p), wq = ldw(W, l, i, q);
          a += qnorm2(wp);
          b += qnorm2(wq);
          Quat<T> pr = qcmul(wp, wq);
          g.w += pr.w; g.x += pr.x; g.y += pr.y; g.z += pr.z;
        }
        a = warp_sum(a); b = warp_sum(b);
        g.w = warp_sum(g.w); g.x = warp_sum(g.x); g.y = warp_sum(g.y); g.z = warp_sum(g.z);
        T gn = sqrt(qnorm2(g));
        if (!(gn > tol * sqrt(a * b)) || gn == (T)0) continue;
        if (lane == 0) s_rot = 1;
        Quat<T> mu = {g.w / gn, g.x / gn, g.y / gn, g.z / gn};
        T zeta = (b - a) / (2 * gn);
        T tt = (zeta >= 0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
        T c = (T)1 / sqrt((T)1 + tt * tt), s = c * tt;
        for (int i = lane; i < l; i += 32) {
          Quat<T> wp = ldw(W, l, i, p), wq = qmulc(ldw(W, l, i, q), mu);   // w_q mu*
          Quat<T> np = {c * wp.w - s * wq.w, c * wp.x - s * wq.x, c * wp.y - s * wq.y, c * wp.z - s * wq.z};
          Quat<T> nq = {s * wp.w + c * wq.w, s * wp.x + c * wq.x, s * wp.y + c * wq.y, s * wp.z + c * wq.z};
          stw(W, l, i, p, np);
          stw(W, l, i, q, nq);
          Quat<T> vp = ldw(V, l, i, p), vq = qmulc(ldw(V, l, i, q), mu);
          stw(V, l, i, p, {c * vp.w - s * vq.w, c * vp.x - s * vq.x, c * vp.y - s * vq.y, c * vp.z - s * vq.z});
          stw(V, l, i, q, {s * vp.w + c * vq.w, s * vp.x + c * vq.x, s * vp.y + c * vq.y, s * vp.z + c * vq.z});
        }
      }
      __syncthreads();
    }
    converged = (s_rot == 0);
    __syncthreads();
  }
  if (t == 0) {
    *sweeps_out = sweep;
    if (!converged) qlr_set_error(err, QLR_ENOCONV);
  }
  // column norms -> sigma (T precision), columns normalised in place
  for (int j = warp; j < l; j += nwarps) {
    T a = 0;
    for (int i = lane; i < l; i += 32) a += qnorm2(ldw(W, l, i, j));
    a = sqrt(warp_sum(a));
    if (lane == 0) sig_out[j] = a;
    T inv = a > (T)0 ? (T)1 / a : (T)0;
    for (int i = lane; i < l; i += 32) {
      Quat<T> w = ldw(W, l, i, j);
      stw(W, l, i, j, {w.w * inv, w.x * inv, w.y * inv, w.z * inv});
    }
  }
  __syncthreads();
  for (size_t e = t; e < 4 * ll; e += JT) {
    if (w_smem) Wout[e] = W[e];
    if (v_smem) Vout[e] = V[e];
  }
}

// Rank of each column by descending sigma (ties broken by index): order[rank] = column.  A NaN
// sigma sorts last, so the keys are totally ordered and `order` is always a permutation.
template <class T>
__device__ __forceinline__ T rank_key(T x) { return isnan(x) ? -INFINITY : x; }

template <class T>
__global__ void rank_kernel(const T* __restrict__ sig, int l, int* __restrict__ order) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= l) return;
  const T sj = rank_key(sig[j]);
  int rank = 0;
  for (int i = 0; i < l; ++i) {
    const T si = rank_key(sig[i]);
    rank += (si > sj) || (si == sj && i < j);
  }
  order[rank] = j;
}

// FP64 evaluation of kept triplet r (one CTA per column):  x = R v,
// sigma = Re(u^H x) / (|u| |v|); L[:, r] = u / |u|, Rt[:, r] = v / |v|.
template <class T>
__global__ void __launch_bounds__(256) refine_kernel(const double* __restrict__ R, int l, const T* __restrict__ U,
                                                      const T* __restrict__ Vm, const int* __restrict__ order, int k,
                                                      double* __restrict__ L, double* __restrict__ S,
                                                      double* __restrict__ Rt) {
  extern __shared__ double sh[];  // 8 * l doubles: u (4l), v (4l)
  __shared__ double red[3][8];
  double* u = sh;
  double* v = sh + 4 * l;
  const int r = blockIdx.x, t = threadIdx.x;
  const int j = min(max(order[r], 0), l - 1);
  for (int i = t; i < l; i += blockDim.x) {
    Quat<T> a = ldw(U, l, i, j), b = ldw(Vm, l, i, j);
    u[i] = (double)a.w; u[l + i] = (double)a.x; u[2 * l + i] = (double)a.y; u[3 * l + i] = (double)a.z;
    v[i] = (double)b.w; v[l + i] = (double)b.x; v[2 * l + i] = (double)b.y; v[3 * l + i] = (double)b.z;
  }
  __syncthreads();
  double rq = 0.0, nu = 0.0, nv = 0.0;
  for (int i = t; i < l; i += blockDim.x) {
    Quat<double> x = {0, 0, 0, 0};
    for (int tt = 0; tt < l; ++tt) {
      Quat<double> pr = qmul(ld_small(R, l, i, tt), Quat<double>{v[tt], v[l + tt], v[2 * l + tt], v[3 * l + tt]});
      x.w += pr.w; x.x += pr.x; x.y += pr.y; x.z += pr.z;
    }
    Quat<double> ui = {u[i], u[l + i], u[2 * l + i], u[3 * l + i]};
    rq += qcmul(ui, x).w;
    nu += qnorm2(ui);
    nv += v[i] * v[i] + v[l + i] * v[l + i] + v[2 * l + i] * v[2 * l + i] + v[3 * l + i] * v[3 * l + i];
  }
  rq = warp_sum(rq); nu = warp_sum(nu); nv = warp_sum(nv);
  if (t % 32 == 0) { red[0][t / 32] = rq; red[1][t / 32] = nu; red[2][t / 32] = nv; }
  __syncthreads();
  double srq = 0.0, snu = 0.0, snv = 0.0;
  for (int w = 0; w < (int)(blockDim.x / 32); ++w) { srq += red[0][w]; snu += red[1][w]; snv += red[2][w]; }
  snu = sqrt(snu); snv = sqrt(snv);
  const double iu = snu > 0.0 ? 1.0 / snu : 0.0, iv = snv > 0.0 ? 1.0 / snv : 0.0;
  const size_t lk = (size_t)l * k;
  for (int i = t; i < l; i += blockDim.x) {
    const size_t o = (size_t)r * l + i;
    for (int c = 0; c < 4; ++c) {
      L[c * lk + o] = u[c * l + i] * iu;
      Rt[c * lk + o] = v[c * l + i] * iv;
    }
  }
  if (t == 0) S[r] = fabs(srq) * iu * iv;
}

}  // namespace

namespace qlr {

template <class T>
static int core_tsvd_t(qlr_ctx* ctx, int l, const double* R, int k, double* L, double* S, double* Rt, WsArena& ws) {
  const size_t ll4 = (size_t)4 * l * l;
  T* W = ws.take<T>(ll4);
  T* V = ws.take<T>(ll4);
  T* sig = ws.take<T>(l);
  int* order = ws.take<int>(l);
  int* sweeps = ws.take<int>(1);
  if (!ws.ok) return QLR_ENOMEM;
  const size_t one = ll4 * sizeof(T);
  const bool w_smem = one <= 200 * 1024;
  const bool v_smem = w_smem && 2 * one <= 200 * 1024;
  const size_t smem = (w_smem ? one : 0) + (v_smem ? one : 0);
  if (smem > 0)
    QLR_CUDA_TRY(cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const T eps = (sizeof(T) == 4) ? (T)5.9604645e-08 : (T)1.1102230246251565e-16;
  const T tol = (T)8 * eps * (T)sqrt((double)l);   // above the rounding noise of the dot products
  { KTimer kt(ctx, QLR_KID_JACOBI);
  jacobi_kernel<T><<<1, JT, smem, ctx->stream>>>(R, l, W, V, w_smem, v_smem, 60, tol, sig, sweeps, ctx->d_err); }
  QLR_CUDA_TRY(cudaGetLastError());
  { KTimer kt(ctx, QLR_KID_REFINE); rank_kernel<T><<<(l + 127) / 128, 128, 0, ctx->stream>>>(sig, l, order); }
  QLR_CUDA_TRY(cudaGetLastError());
  const size_t rsm = (size_t)8 * l * sizeof(double);
  if (rsm > 48 * 1024)
    QLR_CUDA_TRY(cudaFuncSetAttribute(refine_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
  { KTimer kt(ctx, QLR_KID_REFINE); refine_kernel<T><<<k, 256, rsm, ctx->stream>>>(R, l, W, V, order, k, L, S, Rt); }
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

int core_tsvd(qlr_ctx* ctx, int l, const double* R, int k, double* L, double* S, double* Rt, int prec, WsArena& ws) {
  if (k <= 0) return QLR_OK;
  if (k > l || l > 4096) return QLR_ESHAPE;
  size_t mark = ws.off;
  int rc = (prec == QLR_F64) ? core_tsvd_t<double>(ctx, l, R, k, L, S, Rt, ws)
                             : core_tsvd_t<float>(ctx, l, R, k, L, S, Rt, ws);
  ws.off = mark;
  return rc;
}

}  // namespace qlr
