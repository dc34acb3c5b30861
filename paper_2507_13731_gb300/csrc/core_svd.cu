// Core truncated QSVD of the small l x l factor R: the "Truncated SVD(R, k)" step of
// Algorithms 1, 2 and 4 (QSVD of Def. 1, eq. qsvd).
//
// The QSVD of R is computed through its complex adjoint chi(R) (2l x 2l).  chi(R)'s columns
// come in structured pairs: column l + j is determined by column j (it is J conj(col_j)), and
// the leading l columns are exactly the quaternion columns of R written in complex form.  A
// one-sided (Hestenes) Jacobi that only uses right rotations of the form chi(G) for 2 x 2
// quaternion unitaries G keeps that structure, so it suffices to store and rotate the l leading
// columns -- equivalently, the quaternion columns of the matrix W that is swept.  W = R^H (the
// same singular values; one-sided Jacobi on the conjugate transpose of a triangular factor needs
// fewer sweeps).  For a pair of columns (p, q) with alpha = |w_p|^2, beta = |w_q|^2 and
// gamma = w_p^H w_q = |gamma| mu (mu a unit quaternion), w_q <- w_q mu* makes the 2 x 2 Gram real,
// and a real Jacobi rotation then orthogonalises the pair.  At convergence W V_W = U_W diag(sigma);
// each quaternion singular value of R is one of the doubled singular values of chi(R).
//
// The right rotations make up V_W, and R = V_W diag(sigma) U_W^H: R's left singular vectors are
// V_W, its right ones U_W.  The sweep kernel works on W alone (in shared memory when it fits) and
// logs every rotation (c, s, mu); a second kernel replays the log on V_W = I.  The rows of V_W
// transform independently under right rotations, so the replay runs row-parallel on many SMs.
// Both vector sets are orthonormal to the working precision.  Precision: the sweeps run in T
// (float or double); a final FP64 step evaluates every kept singular value as the two-sided
// Rayleigh quotient sigma = Re(u^H R v) / (|u| |v|) from the FP64 R, whose error is second order
// in the vectors'.
#include <cooperative_groups.h>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "qlr_internal.h"

namespace cg = cooperative_groups;

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

// Reciprocal and reciprocal square root for the rotation parameters: the hardware approximations
// in float (a few ulp; every rotation is applied to W and V, or logged and replayed, exactly as
// computed, so the vectors stay orthonormal to the working precision), correctly rounded in
// double.
__device__ __forceinline__ float jrsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double jrsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float jrcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double jrcp(double x) { return 1.0 / x; }

// Rotation parameters of a column pair (alpha = |w_p|^2, beta = |w_q|^2, gamma = w_p^H w_q with
// |gamma|^2 = gn2 > 0): mu = gamma / |gamma| and the real Jacobi rotation (c, s) that
// orthogonalises (w_p, w_q mu*): t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// zeta = (beta - alpha) / (2 |gamma|), c = 1 / sqrt(1 + t^2), s = c t.
template <class T>
__device__ __forceinline__ void jacobi_rotation(T alpha, T beta, const Quat<T>& g, T gn2, Quat<T>& mu, T& c, T& s) {
  const T ign = jrsqrt(gn2);
  mu = {g.w * ign, g.x * ign, g.y * ign, g.z * ign};
  const T zeta = (beta - alpha) * ((T)0.5 * ign);
  const T az = fabs(zeta);
  const T x = (T)1 + az * az;
  const T den = (az < (T)1e18) ? az + x * jrsqrt(x) : (T)2 * az;
  const T tt = (zeta >= 0 ? (T)1 : (T)-1) * jrcp(den);
  c = jrsqrt((T)1 + tt * tt);
  s = c * tt;
}

// Element e (plane-major, column-major planes) of W = R^H, the matrix the sweeps orthogonalise:
// W(i, j) = conj(R(j, i)).  One-sided Jacobi on R^H rather than R converges in fewer sweeps on
// the triangular factors of CholeskyQR (Drmac and Veselic's preconditioning); the roles of the
// vectors swap: R = V_W Sigma U_W^H, so R's left vectors are W's accumulated rotations V_W and its
// right vectors W's normalised columns U_W.
template <class S>
__device__ __forceinline__ S rh_elem(const S* __restrict__ R, int l, size_t ll, size_t e) {
  const size_t c = e / ll, o = e % ll;
  const size_t i = o % l, j = o / l;
  const S v = R[c * ll + i * l + j];
  return c == 0 ? v : -v;
}

// Cyclic (round-robin) one-sided Jacobi sweeps by one CTA of JT threads on W (l x l, planes of
// l * l, column-major), with the same right rotations applied to Vs when it is set; otherwise
// every rotation is logged to rlog.  Returns the number of sweeps run; *converged is set when
// the last sweep rotated no pair.
template <class T>
__device__ int jacobi_sweeps(T* W, T* Vs, int l, int max_sweeps, T tol, T* rlog, bool* converged_out) {
  __shared__ int s_rot;
  const int t = threadIdx.x, lane = t % 32, warp = t / 32, nwarps = JT / 32;
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
        const T gn2 = qnorm2(g);
        T* lg = Vs ? nullptr : rlog + (((size_t)sweep * (lp - 1) + r) * (lp / 2) + pi) * 6;
        if (!(gn2 > (tol * tol * a) * b)) {      // pair already orthogonal to the tolerance
          if (lane == 0 && lg) { lg[0] = (T)1; lg[1] = (T)0; lg[2] = (T)1; lg[3] = lg[4] = lg[5] = (T)0; }
          continue;
        }
        if (lane == 0) s_rot = 1;
        Quat<T> mu;
        T c, s;
        jacobi_rotation(a, b, g, gn2, mu, c, s);
        if (lane == 0 && lg) { lg[0] = c; lg[1] = s; lg[2] = mu.w; lg[3] = mu.x; lg[4] = mu.y; lg[5] = mu.z; }
        for (int i = lane; i < l; i += 32) {
          Quat<T> wp = ldw(W, l, i, p), wq = qmulc(ldw(W, l, i, q), mu);   // w_q mu*
          Quat<T> np = {c * wp.w - s * wq.w, c * wp.x - s * wq.x, c * wp.y - s * wq.y, c * wp.z - s * wq.z};
          Quat<T> nq = {s * wp.w + c * wq.w, s * wp.x + c * wq.x, s * wp.y + c * wq.y, s * wp.z + c * wq.z};
          stw(W, l, i, p, np);
          stw(W, l, i, q, nq);
          if (Vs) {                              // the same right rotation on V
            Quat<T> vp = ldw(Vs, l, i, p), vq = qmulc(ldw(Vs, l, i, q), mu);
            stw(Vs, l, i, p, {c * vp.w - s * vq.w, c * vp.x - s * vq.x, c * vp.y - s * vq.y, c * vp.z - s * vq.z});
            stw(Vs, l, i, q, {s * vp.w + c * vq.w, s * vp.x + c * vq.x, s * vp.y + c * vq.y, s * vp.z + c * vq.z});
          }
        }
      }
      __syncthreads();
    }
    converged = (s_rot == 0);
    __syncthreads();
  }
  *converged_out = converged;
  return sweep;
}

// One CTA: W = R (in shared memory when it fits), the rotations logged for the replay on V.
template <class T>
__global__ void __launch_bounds__(JT) jacobi_kernel(const double* __restrict__ R, int l, T* __restrict__ Wout,
                                                     bool w_smem, int max_sweeps, T tol, T* __restrict__ sig_out,
                                                     int* __restrict__ sweeps_out, T* __restrict__ rlog, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* W = w_smem ? reinterpret_cast<T*>(smem_raw) : Wout;
  const int t = threadIdx.x, lane = t % 32, warp = t / 32, nwarps = JT / 32;
  const size_t ll = (size_t)l * l;
  for (size_t e = t; e < 4 * ll; e += JT) W[e] = (T)rh_elem(R, l, ll, e);
  __syncthreads();
  bool converged = false;
  const int sweep = jacobi_sweeps<T>(W, (T*)nullptr, l, max_sweeps, tol, rlog, &converged);
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
  if (w_smem)
    for (size_t e = t; e < 4 * ll; e += JT) Wout[e] = W[e];
}

template <class T>
__device__ __forceinline__ T rank_key(T x) { return isnan(x) ? -INFINITY : x; }

// Batch plans: one CTA per problem, W = R^H and V = I in shared memory (FP32, each quaternion
// stored as one float4).  A column pair is handled by a group of g lanes (8 for l <= 48, 16 up to
// 80), each lane holding up to JG_RMAX rows of both columns in registers between the dot products
// and the rotation, so a warp works on 32 / g pairs at once and no lane idles on a short column;
// the group's dot products are reduced with log2(g) shuffle steps.  After the sweeps
// sigma_j = |w_j| and u_j = w_j / sigma_j; the k largest sigma (descending, ties by column) go to
// S and their u, v columns to U, V (times the upper-triangular Lleft, Lright when given: the
// carried inverse factors of the plan's last two passes).  Without the FP64 Rayleigh step of the
// single-problem path:
// the plan's sketches and bases are BF16 / FP32, and the column norms carry the FP32 accuracy of
// the rotated columns.
constexpr int JG_THREADS = 640;   // 40 groups of 16 lanes: every pair of a round at once (l <= 80)
constexpr int JG_RMAX = 6;        // rows per lane: l <= 8 * 6 (groups of 8), l <= 16 * 5 (of 16)

__device__ __forceinline__ Quat<float> q_of4(const float4 v) { return {v.x, v.y, v.z, v.w}; }
__device__ __forceinline__ float4 f4_of(const Quat<float>& q) { return make_float4(q.w, q.x, q.y, q.z); }

__global__ void __launch_bounds__(JG_THREADS) jacobi_grouped_kernel(const qlr::JacobiGroupArgs* __restrict__ args,
                                                                   int max_sweeps, int* err) {
  const qlr::JacobiGroupArgs& a = args[blockIdx.x];
  const int l = a.l, k = a.k;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t ll = (size_t)l * l;
  float4* W = reinterpret_cast<float4*>(smem_raw);   // W(i, j) at W[j l + i]
  float4* Vs = W + ll;
  float* sig = reinterpret_cast<float*>(Vs + ll);
  int* ord = reinterpret_cast<int*>(sig + l);
  __shared__ int s_rot;
  const int t = threadIdx.x, lane = t % 32, warp = t / 32, nwarps = JG_THREADS / 32;
  const float* R = a.R;
  for (size_t e = t; e < ll; e += JG_THREADS) {   // W(i, j) = conj(R(j, i))
    const size_t i = e % l, j = e / l, src = i * l + j;
    W[e] = make_float4(R[src], -R[ll + src], -R[2 * ll + src], -R[3 * ll + src]);
    Vs[e] = make_float4(i == j ? 1.f : 0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  const float tol = 8.f * 5.9604645e-08f * sqrtf((float)l);   // above the rounding noise of the dot products
  const int g = (l <= 8 * JG_RMAX) ? 8 : 16;
  const int grp = t / g, sub = t % g, ngroups = JG_THREADS / g;
  const int lp = l + (l & 1), npairs = lp / 2;
  bool converged = (l < 2);
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    if (t == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < lp - 1; ++r) {
      for (int base = 0; base < npairs; base += ngroups) {
        const int pi = base + grp;
        int p = 0, q = 0;
        bool valid = pi < npairs;
        if (valid) {
          rr_pair(lp, r, pi, p, q);
          valid = p < l && q < l;
        }
        Quat<float> wp[JG_RMAX], wq[JG_RMAX];
        float al = 0.f, be = 0.f;
        Quat<float> ga = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int u = 0; u < JG_RMAX; ++u) {
          const int i = sub + u * g;
          if (valid && i < l) {
            wp[u] = q_of4(W[(size_t)p * l + i]);
            wq[u] = q_of4(W[(size_t)q * l + i]);
            al += qnorm2(wp[u]);
            be += qnorm2(wq[u]);
            const Quat<float> pr = qcmul(wp[u], wq[u]);
            ga.w += pr.w; ga.x += pr.x; ga.y += pr.y; ga.z += pr.z;
          }
        }
        for (int o = g / 2; o > 0; o >>= 1) {   // within the group (every lane of the warp takes part)
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga.w += __shfl_xor_sync(0xffffffffu, ga.w, o);
          ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
          ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
          ga.z += __shfl_xor_sync(0xffffffffu, ga.z, o);
        }
        const float gn2 = qnorm2(ga);
        if (valid && gn2 > (tol * tol * al) * be) {
          if (sub == 0) s_rot = 1;
          Quat<float> mu;
          float c, s;
          jacobi_rotation(al, be, ga, gn2, mu, c, s);
#pragma unroll
          for (int u = 0; u < JG_RMAX; ++u) {
            const int i = sub + u * g;
            if (i < l) {
              const Quat<float> wqm = qmulc(wq[u], mu);   // w_q mu*
              W[(size_t)p * l + i] = make_float4(c * wp[u].w - s * wqm.w, c * wp[u].x - s * wqm.x,
                                                 c * wp[u].y - s * wqm.y, c * wp[u].z - s * wqm.z);
              W[(size_t)q * l + i] = make_float4(s * wp[u].w + c * wqm.w, s * wp[u].x + c * wqm.x,
                                                 s * wp[u].y + c * wqm.y, s * wp[u].z + c * wqm.z);
              const Quat<float> vp = q_of4(Vs[(size_t)p * l + i]), vq = qmulc(q_of4(Vs[(size_t)q * l + i]), mu);
              Vs[(size_t)p * l + i] = make_float4(c * vp.w - s * vq.w, c * vp.x - s * vq.x, c * vp.y - s * vq.y,
                                                  c * vp.z - s * vq.z);
              Vs[(size_t)q * l + i] = make_float4(s * vp.w + c * vq.w, s * vp.x + c * vq.x, s * vp.y + c * vq.y,
                                                  s * vp.z + c * vq.z);
            }
          }
        }
      }
      __syncthreads();
    }
    converged = (s_rot == 0);
    __syncthreads();
  }
  if (t == 0 && !converged) qlr_set_error(err, QLR_ENOCONV);
  for (int j = warp; j < l; j += nwarps) {
    float s2 = 0.f;
    for (int i = lane; i < l; i += 32) s2 += qnorm2(q_of4(W[(size_t)j * l + i]));
    s2 = sqrtf(warp_sum(s2));
    if (lane == 0) sig[j] = s2;
    const float inv = s2 > 0.f ? 1.f / s2 : 0.f;
    for (int i = lane; i < l; i += 32) {
      const float4 w = W[(size_t)j * l + i];
      W[(size_t)j * l + i] = make_float4(w.x * inv, w.y * inv, w.z * inv, w.w * inv);
    }
  }
  __syncthreads();
  for (int j = t; j < l; j += JG_THREADS) {
    const float sj = rank_key(sig[j]);
    int rank = 0;
    for (int i = 0; i < l; ++i) {
      const float si = rank_key(sig[i]);
      rank += (si > sj) || (si == sj && i < j);
    }
    ord[rank] = j;
  }
  __syncthreads();
  for (int r = t; r < k; r += JG_THREADS) a.S[r] = (double)sig[ord[r]];
  const size_t lk = (size_t)l * k;
  float* U = a.U;
  float* V = a.V;
  const float* Ll = a.Lleft;
  const float* Lr = a.Lright;
  for (size_t e = t; e < lk; e += JG_THREADS) {
    const int r = (int)(e / l), i = (int)(e % l);
    const size_t col = (size_t)ord[r] * l;
    // R's left vectors: the rotations of W = R^H; right: W's normalised columns
    Quat<float> u = q_of4(Vs[col + i]), v = q_of4(W[col + i]);
    if (Ll) {
      u = {0.f, 0.f, 0.f, 0.f};
      for (int tt = i; tt < l; ++tt) {
        const size_t o = (size_t)tt * l + i;
        const Quat<float> pr = qmul(Quat<float>{Ll[o], Ll[ll + o], Ll[2 * ll + o], Ll[3 * ll + o]}, q_of4(Vs[col + tt]));
        u.w += pr.w; u.x += pr.x; u.y += pr.y; u.z += pr.z;
      }
    }
    if (Lr) {
      v = {0.f, 0.f, 0.f, 0.f};
      for (int tt = i; tt < l; ++tt) {
        const size_t o = (size_t)tt * l + i;
        const Quat<float> pr = qmul(Quat<float>{Lr[o], Lr[ll + o], Lr[2 * ll + o], Lr[3 * ll + o]}, q_of4(W[col + tt]));
        v.w += pr.w; v.x += pr.x; v.y += pr.y; v.z += pr.z;
      }
    }
    U[e] = u.w; U[lk + e] = u.x; U[2 * lk + e] = u.y; U[3 * lk + e] = u.z;
    V[e] = v.w; V[lk + e] = v.x; V[2 * lk + e] = v.y; V[3 * lk + e] = v.z;
  }
}

// Replay the logged rotations on V = I, one warp per row of V (rows are independent under right
// rotations); the pairs of one round are disjoint, so the lanes apply them concurrently.
template <class T>
__global__ void __launch_bounds__(128) jacobi_replay_kernel(int l, const T* __restrict__ rlog, const int* __restrict__ nsweeps,
                                                             T* __restrict__ Vout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int row = blockIdx.x * 4 + warp;
  T* vr = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 4 * l;   // this row: 4 planes x l
  if (row >= l) return;
  for (int j = lane; j < l; j += 32) {
    vr[j] = (j == row) ? (T)1 : (T)0;
    vr[l + j] = vr[2 * l + j] = vr[3 * l + j] = (T)0;
  }
  __syncwarp();
  const int lp = l + (l & 1);
  const int ns = *nsweeps;
  for (int sw = 0; sw < ns; ++sw) {
    for (int r = 0; r < lp - 1; ++r) {
      const T* lg0 = rlog + (((size_t)sw * (lp - 1) + r) * (lp / 2)) * 6;
      for (int pi = lane; pi < lp / 2; pi += 32) {
        int p, q;
        rr_pair(lp, r, pi, p, q);
        if (p >= l || q >= l) continue;
        const T* lg = lg0 + (size_t)pi * 6;
        const T c = lg[0], s = lg[1];
        if (s == (T)0) continue;
        const Quat<T> mu = {lg[2], lg[3], lg[4], lg[5]};
        Quat<T> vp = {vr[p], vr[l + p], vr[2 * l + p], vr[3 * l + p]};
        Quat<T> vq = qmulc(Quat<T>{vr[q], vr[l + q], vr[2 * l + q], vr[3 * l + q]}, mu);
        vr[p] = c * vp.w - s * vq.w; vr[l + p] = c * vp.x - s * vq.x; vr[2 * l + p] = c * vp.y - s * vq.y; vr[3 * l + p] = c * vp.z - s * vq.z;
        vr[q] = s * vp.w + c * vq.w; vr[l + q] = s * vp.x + c * vq.x; vr[2 * l + q] = s * vp.y + c * vq.y; vr[3 * l + q] = s * vp.z + c * vq.z;
      }
      __syncwarp();
    }
  }
  const size_t ll = (size_t)l * l;
  for (int j = lane; j < l; j += 32)
    for (int c = 0; c < 4; ++c) Vout[c * ll + (size_t)j * l + row] = vr[(size_t)c * l + j];
}

// ---------------------------------------------------------------------------------------
// Cluster block Jacobi for larger l: the l columns of W are split into NB = 2 * P blocks
// (P = cluster size).  A sweep is NB - 1 block rounds; in block round br, CTA p takes the block
// pair rr_pair(NB, br, p) (disjoint across CTAs), loads the union of the two blocks into shared
// memory, runs one local round-robin sweep over its columns and writes them back; a cluster
// barrier ends the round.  W stays in global memory (L2).  Every local round is one "stage" of
// the rotation log: P x BW records (p, q, c, s, mu), disjoint columns, identity-padded, so the
// replay can apply a whole stage in parallel.
constexpr int JP = 8;                 // portable cluster size (16 when the GPU can co-schedule it)
constexpr int JP_MAX = 16;
constexpr int JB_THREADS = 256;      // threads of a cluster CTA (FP64, or at most 8 pairs per local round)
constexpr int JB_THREADS_WIDE = 384; // FP32 with 9..16 pairs per local round: one warp per pair up to 12
constexpr int REC = 8;                // floats per log record: p, q, c, s, mu(4)

// Stage index of local round lr in block round br: block round 0 runs the full round-robin over
// the 2 bw columns of its block pair (U - 1 rounds, covering the pairs inside each block); later
// block rounds only pair columns across the two blocks (bw rounds: a_i with b_{(i + lr) mod bw}).
__host__ __device__ __forceinline__ int jb_stages_per_sweep(int bw, int jp) { return (2 * bw - 1) + (2 * jp - 2) * bw; }
__host__ __device__ __forceinline__ int jb_stage(int br, int lr, int bw) { return br == 0 ? lr : (2 * bw - 1) + (br - 1) * bw + lr; }


// Rows per lane RPL: the two columns of a pair stay in registers between the dot products and
// the rotation (l <= 32 RPL).
template <class T, int RPL, int NT>
__global__ void __launch_bounds__(NT, 1) jacobi_block_kernel(const double* __restrict__ R, int l, int bw,
                                                                   T* __restrict__ W, int max_sweeps, T tol,
                                                                   T* __restrict__ rlog, int* __restrict__ flags,
                                                                   int* __restrict__ sweeps_out, T* __restrict__ sig_out,
                                                                   int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);          // [4][2 bw][l]: plane, local column, row
  cg::cluster_group cluster = cg::this_cluster();
  const int p = (int)cluster.block_rank();
  const int t = threadIdx.x, lane = t % 32, warp = t / 32, nwarps = NT / 32;
  const size_t ll = (size_t)l * l;
  const int JPR = (int)gridDim.x;                 // cluster size: one cluster of JPR CTAs
  const int NB = 2 * JPR;
  const int U = 2 * bw;
  const int sps = jb_stages_per_sweep(bw, JPR);
  const int stage_cap = JPR * bw;
  const T tol2 = tol * tol;
  for (size_t e = (size_t)p * NT + t; e < 4 * ll; e += (size_t)JPR * NT) W[e] = (T)rh_elem(R, l, ll, e);
  if (p == 0)
    for (int i = t; i < max_sweeps; i += NT) flags[i] = 0;
  __threadfence();
  cluster.sync();
  int sweep = 0;
  bool converged = (l < 2);
  __shared__ int s_rot;
  __shared__ int gcol[64];
  auto col = [&](int c, int lc) { return S + ((size_t)c * U + lc) * l; };
  for (; sweep < max_sweeps && !converged; ++sweep) {
    if (t == 0) s_rot = 0;
    for (int br = 0; br < NB - 1; ++br) {
      int ba, bb;
      rr_pair(NB, br, p, ba, bb);
      if (t < U) {
        const int blk = (t < bw) ? ba : bb, off = (t < bw) ? t : t - bw;
        const int g = blk * bw + off;
        gcol[t] = (g < l) ? g : -1;
      }
      __syncthreads();
      for (int lc = warp; lc < U; lc += nwarps) {   // one warp per local column, coalesced rows
        const int g = gcol[lc];
        T v[4][RPL];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int i = lane + 32 * u;
            v[c][u] = (g >= 0 && i < l) ? W[c * ll + (size_t)g * l + i] : (T)0;
          }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int i = lane + 32 * u;
            if (i < l) col(c, lc)[i] = v[c][u];
          }
      }
      __syncthreads();
      if (br > 0 && bw <= nwarps) {
        // cross-block rounds: warp pi keeps column a_pi in registers for all bw local rounds and
        // only the b column it meets this round goes through shared memory
        const int pi = warp;
        const int ga = (pi < bw) ? gcol[pi] : -1;
        Quat<T> wa[RPL];
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int i = lane + 32 * u;
          wa[u] = (ga >= 0 && i < l) ? Quat<T>{col(0, pi)[i], col(1, pi)[i], col(2, pi)[i], col(3, pi)[i]}
                                     : Quat<T>{0, 0, 0, 0};
        }
        for (int lr = 0; lr < bw; ++lr) {
          if (pi < bw) {
            T* lg = rlog + ((size_t)sweep * sps + jb_stage(br, lr, bw)) * stage_cap * REC + ((size_t)p * bw + pi) * REC;
            const int b = bw + (pi + lr) % bw;
            const int gb = gcol[b];
            if (ga < 0 || gb < 0) {
              if (lane == 0) { lg[0] = (T)-1; lg[1] = (T)-1; lg[2] = (T)1; lg[3] = (T)0; }
            } else {
              T* B0 = col(0, b); T* B1 = col(1, b); T* B2 = col(2, b); T* B3 = col(3, b);
              Quat<T> wq[RPL];
              T aa = 0, bb2 = 0;
              Quat<T> g = {0, 0, 0, 0};
#pragma unroll
              for (int u = 0; u < RPL; ++u) {
                const int i = lane + 32 * u;
                wq[u] = (i < l) ? Quat<T>{B0[i], B1[i], B2[i], B3[i]} : Quat<T>{0, 0, 0, 0};
                aa += qnorm2(wa[u]);
                bb2 += qnorm2(wq[u]);
                const Quat<T> pr = qcmul(wa[u], wq[u]);
                g.w += pr.w; g.x += pr.x; g.y += pr.y; g.z += pr.z;
              }
              aa = warp_sum(aa); bb2 = warp_sum(bb2);
              g.w = warp_sum(g.w); g.x = warp_sum(g.x); g.y = warp_sum(g.y); g.z = warp_sum(g.z);
              const T gn2 = qnorm2(g);
              if (!(gn2 > (tol2 * aa) * bb2)) {
                if (lane == 0) { lg[0] = (T)ga; lg[1] = (T)gb; lg[2] = (T)1; lg[3] = (T)0; }
              } else {
                if (lane == 0) s_rot = 1;
                Quat<T> mu;
                T c, sn;
                jacobi_rotation(aa, bb2, g, gn2, mu, c, sn);
                if (lane == 0) {
                  lg[0] = (T)ga; lg[1] = (T)gb; lg[2] = c; lg[3] = sn;
                  lg[4] = mu.w; lg[5] = mu.x; lg[6] = mu.y; lg[7] = mu.z;
                }
#pragma unroll
                for (int u = 0; u < RPL; ++u) {
                  const int i = lane + 32 * u;
                  const Quat<T> q = qmulc(wq[u], mu);
                  const Quat<T> np = {c * wa[u].w - sn * q.w, c * wa[u].x - sn * q.x, c * wa[u].y - sn * q.y,
                                      c * wa[u].z - sn * q.z};
                  if (i < l) {
                    B0[i] = sn * wa[u].w + c * q.w; B1[i] = sn * wa[u].x + c * q.x;
                    B2[i] = sn * wa[u].y + c * q.y; B3[i] = sn * wa[u].z + c * q.z;
                  }
                  wa[u] = np;
                }
              }
            }
          }
          __syncthreads();
        }
        if (ga >= 0) {
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int i = lane + 32 * u;
            if (i < l) { col(0, pi)[i] = wa[u].w; col(1, pi)[i] = wa[u].x; col(2, pi)[i] = wa[u].y; col(3, pi)[i] = wa[u].z; }
          }
        }
        __syncthreads();
      }
      const int nlr = (br == 0) ? U - 1 : ((bw <= nwarps) ? 0 : bw);
      for (int lr = 0; lr < nlr; ++lr) {
        T* lg_stage = rlog + ((size_t)sweep * sps + jb_stage(br, lr, bw)) * stage_cap * REC;
        for (int pi = warp; pi < bw; pi += nwarps) {
          int a, b;
          if (br == 0) rr_pair(U, lr, pi, a, b);
          else { a = pi; b = bw + (pi + lr) % bw; }
          T* lg = lg_stage + ((size_t)p * bw + pi) * REC;
          const int ga = gcol[a], gb = gcol[b];
          if (ga < 0 || gb < 0) {
            if (lane == 0) { lg[0] = (T)-1; lg[1] = (T)-1; lg[2] = (T)1; lg[3] = (T)0; }
            continue;
          }
          T* A0 = col(0, a); T* A1 = col(1, a); T* A2 = col(2, a); T* A3 = col(3, a);
          T* B0 = col(0, b); T* B1 = col(1, b); T* B2 = col(2, b); T* B3 = col(3, b);
          Quat<T> wp[RPL], wq[RPL];
          T aa = 0, bb2 = 0;
          Quat<T> g = {0, 0, 0, 0};
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int i = lane + 32 * u;
            if (i < l) {
              wp[u] = {A0[i], A1[i], A2[i], A3[i]};
              wq[u] = {B0[i], B1[i], B2[i], B3[i]};
            } else {
              wp[u] = {0, 0, 0, 0};
              wq[u] = {0, 0, 0, 0};
            }
            aa += qnorm2(wp[u]);
            bb2 += qnorm2(wq[u]);
            const Quat<T> pr = qcmul(wp[u], wq[u]);
            g.w += pr.w; g.x += pr.x; g.y += pr.y; g.z += pr.z;
          }
          aa = warp_sum(aa); bb2 = warp_sum(bb2);
          g.w = warp_sum(g.w); g.x = warp_sum(g.x); g.y = warp_sum(g.y); g.z = warp_sum(g.z);
          const T gn2 = qnorm2(g);
          if (!(gn2 > (tol2 * aa) * bb2)) {      // pair already orthogonal to the tolerance
            if (lane == 0) { lg[0] = (T)ga; lg[1] = (T)gb; lg[2] = (T)1; lg[3] = (T)0; }
            continue;
          }
          if (lane == 0) s_rot = 1;
          Quat<T> mu;
          T c, sn;
          jacobi_rotation(aa, bb2, g, gn2, mu, c, sn);
          if (lane == 0) {
            lg[0] = (T)ga; lg[1] = (T)gb; lg[2] = c; lg[3] = sn;
            lg[4] = mu.w; lg[5] = mu.x; lg[6] = mu.y; lg[7] = mu.z;
          }
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int i = lane + 32 * u;
            if (i < l) {
              const Quat<T> q = qmulc(wq[u], mu);
              A0[i] = c * wp[u].w - sn * q.w; A1[i] = c * wp[u].x - sn * q.x;
              A2[i] = c * wp[u].y - sn * q.y; A3[i] = c * wp[u].z - sn * q.z;
              B0[i] = sn * wp[u].w + c * q.w; B1[i] = sn * wp[u].x + c * q.x;
              B2[i] = sn * wp[u].y + c * q.y; B3[i] = sn * wp[u].z + c * q.z;
            }
          }
        }
        __syncthreads();
      }
      for (int lc = warp; lc < U; lc += nwarps) {
        const int g = gcol[lc];
        if (g < 0) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int i = lane + 32 * u;
            if (i < l) W[c * ll + (size_t)g * l + i] = col(c, lc)[i];
          }
      }
      cluster.sync();   // arrive.release / wait.acquire at cluster scope: W's columns visible to all CTAs
    }
    if (t == 0 && s_rot) atomicOr(&flags[sweep], 1);
    cluster.sync();
    converged = (*(volatile int*)&flags[sweep] == 0);
    cluster.sync();
  }
  if (p == 0 && t == 0) {
    *sweeps_out = sweep;
    if (!converged) qlr_set_error(err, QLR_ENOCONV);
  }
  for (int j = p * nwarps + warp; j < l; j += JPR * nwarps) {
    T a = 0;
    for (int i = lane; i < l; i += 32) a += qnorm2(ldw(W, l, i, j));
    a = sqrt(warp_sum(a));
    if (lane == 0) sig_out[j] = a;
    const T inv = a > (T)0 ? (T)1 / a : (T)0;
    for (int i = lane; i < l; i += 32) {
      Quat<T> w = ldw(W, l, i, j);
      stw(W, l, i, j, {w.w * inv, w.x * inv, w.y * inv, w.z * inv});
    }
  }
}

// Replay of the staged rotation log on V = I, one warp per row of V.  The log is read in chunks
// of RCH stages that the CTA's four warps share: each chunk is copied to shared memory with
// cp.async while the previous one is applied.
constexpr int RCH = 8;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <class T>
__device__ __forceinline__ void ld_rec(const T* r, T (&v)[REC]) {
#pragma unroll
  for (int f = 0; f < REC; ++f) v[f] = r[f];
}
template <>
__device__ __forceinline__ void ld_rec<float>(const float* r, float (&v)[REC]) {
  const float4 a = reinterpret_cast<const float4*>(r)[0], b = reinterpret_cast<const float4*>(r)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

size_t jb_replay_smem(int l, int bw, int jp, size_t esz) {
  return (size_t)2 * RCH * jp * bw * REC * esz + (size_t)4 * 4 * l * esz;
}

template <class T>
__global__ void __launch_bounds__(128) jacobi_block_replay_kernel(int l, int bw, int jp, const T* __restrict__ rlog,
                                                                   const int* __restrict__ nsweeps, T* __restrict__ Vout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int cap = jp * bw;
  const size_t stage_elems = (size_t)cap * REC;
  T* logbuf = reinterpret_cast<T*>(smem_raw);                    // [2][RCH][cap][REC]
  T* vr = logbuf + 2 * RCH * stage_elems + (size_t)warp * 4 * l;  // this warp's row of V, 4 planes
  const int row = blockIdx.x * 4 + warp;
  const bool active = row < l;
  if (active)
    for (int j = lane; j < l; j += 32) {
      vr[j] = (j == row) ? (T)1 : (T)0;
      vr[l + j] = vr[2 * l + j] = vr[3 * l + j] = (T)0;
    }
  const size_t nst = (size_t)(*nsweeps) * jb_stages_per_sweep(bw, jp);
  const size_t nchunks = (nst + RCH - 1) / RCH;
  auto stage_chunk = [&](size_t ch) {
    const size_t s0 = ch * RCH;
    const size_t ns = (nst - s0 < (size_t)RCH) ? nst - s0 : (size_t)RCH;
    const size_t bytes = ns * stage_elems * sizeof(T);
    const char* src = reinterpret_cast<const char*>(rlog + s0 * stage_elems);
    char* dst = reinterpret_cast<char*>(logbuf + (ch & 1) * RCH * stage_elems);
    for (size_t o = (size_t)threadIdx.x * 16; o < bytes; o += (size_t)blockDim.x * 16) cp_async16(dst + o, src + o);
    cp_async_commit();
  };
  if (nchunks > 0) stage_chunk(0);
  for (size_t ch = 0; ch < nchunks; ++ch) {
    if (ch + 1 < nchunks) {
      stage_chunk(ch + 1);     // fills the other buffer, released by the barrier that ended chunk ch - 1
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const T* lb = logbuf + (ch & 1) * RCH * stage_elems;
    const int ns = (int)((nst - ch * RCH < (size_t)RCH) ? nst - ch * RCH : (size_t)RCH);
    if (active) {
      for (int st = 0; st < ns; ++st) {
        // two records per lane and iteration, loaded and applied side by side (a stage's pairs are
        // disjoint, so the two rotations touch different entries of the row)
        for (int k0 = 0; k0 < cap; k0 += 64) {
          T r[2][REC];
          int pp[2], qq[2];
          bool on[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int k = k0 + 32 * h + lane;
            if (k < cap) ld_rec(lb + ((size_t)st * cap + k) * REC, r[h]);
            else r[h][3] = (T)0;
            on[h] = (r[h][3] != (T)0);
            pp[h] = on[h] ? (int)r[h][0] : 0;
            qq[h] = on[h] ? (int)r[h][1] : 0;
          }
          Quat<T> vp[2], vq[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            vp[h] = {vr[pp[h]], vr[l + pp[h]], vr[2 * l + pp[h]], vr[3 * l + pp[h]]};
            vq[h] = {vr[qq[h]], vr[l + qq[h]], vr[2 * l + qq[h]], vr[3 * l + qq[h]]};
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (!on[h]) continue;
            const T c = r[h][2], sn = r[h][3];
            const Quat<T> q = qmulc(vq[h], Quat<T>{r[h][4], r[h][5], r[h][6], r[h][7]});
            const int a = pp[h], b = qq[h];
            vr[a] = c * vp[h].w - sn * q.w; vr[l + a] = c * vp[h].x - sn * q.x; vr[2 * l + a] = c * vp[h].y - sn * q.y;
            vr[3 * l + a] = c * vp[h].z - sn * q.z;
            vr[b] = sn * vp[h].w + c * q.w; vr[l + b] = sn * vp[h].x + c * q.x; vr[2 * l + b] = sn * vp[h].y + c * q.y;
            vr[3 * l + b] = sn * vp[h].z + c * q.z;
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if (!active) return;
  const size_t ll = (size_t)l * l;
  for (int j = lane; j < l; j += 32)
    for (int c = 0; c < 4; ++c) Vout[c * ll + (size_t)j * l + row] = vr[(size_t)c * l + j];
}

// Rank of each column by descending sigma (ties broken by index): order[rank] = column.  A NaN
// sigma sorts last, so the keys are totally ordered and `order` is always a permutation.

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

constexpr int JMAX_SWEEPS = 30;
constexpr int JBLOCK_MIN_L = 48;     // from this size on, the cluster block Jacobi is used

// The cluster block Jacobi holds two column blocks per CTA in shared memory and gives each replay
// lane at most four records per stage; larger cores run the single-CTA sweep.
static bool use_block_jacobi(int l, size_t esz) {
  const int bw = (l + 2 * JP - 1) / (2 * JP);
  return l >= JBLOCK_MIN_L && l <= 256 && (size_t)4 * l * 2 * bw * esz <= 220 * 1024 && JP * bw <= 128;
}

size_t jacobi_log_floats(int l) {
  size_t blk = 0;
  for (int jp : {JP, JP_MAX}) {
    const int bw = (l + 2 * jp - 1) / (2 * jp);
    blk = std::max(blk, (size_t)JMAX_SWEEPS * jb_stages_per_sweep(bw, jp) * jp * bw * REC + REC);
  }
  const int lp = l + (l & 1);
  const size_t one = (size_t)JMAX_SWEEPS * (lp - 1) * (lp / 2) * 6 + 6;
  return blk > one ? blk : one;
}

// Cluster size of the block Jacobi for this l: 16 when the device allows the non-portable size
// and can co-schedule 16 CTAs of the kernel, else 8 (decided once per device and l).
template <class T>
static int block_jacobi_cluster(int device, int l) {
  static std::mutex mu;
  static std::vector<std::pair<int64_t, int>> cache;
  std::lock_guard<std::mutex> lk(mu);
  const int64_t key = ((int64_t)device << 32) | (uint32_t)l;
  for (const auto& e : cache)
    if (e.first == key) return e.second;
  int pick = JP;
  const int bw = (l + 2 * JP_MAX - 1) / (2 * JP_MAX);
  auto kern = (l <= 128) ? jacobi_block_kernel<T, 4, JB_THREADS> : jacobi_block_kernel<T, 8, JB_THREADS>;
  const size_t smem = (size_t)4 * l * 2 * bw * sizeof(T);
  if (bw <= JB_THREADS / 32 &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(JP_MAX, 1, 1);
    cfg.blockDim = dim3(JB_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = JP_MAX;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) == cudaSuccess && ncl > 0) pick = JP_MAX;
  }
  cudaGetLastError();
  cache.emplace_back(key, pick);
  return pick;
}

template <class T>
static int core_tsvd_t(qlr_ctx* ctx, int l, const double* R, int k, double* L, double* S, double* Rt, WsArena& ws) {
  const size_t ll4 = (size_t)4 * l * l;
  T* W = ws.take<T>(ll4);
  T* V = ws.take<T>(ll4);
  T* rlog = ws.take<T>(jacobi_log_floats(l));
  T* sig = ws.take<T>(l);
  int* order = ws.take<int>(l);
  int* sweeps = ws.take<int>(1);
  int* flags = ws.take<int>(JMAX_SWEEPS);
  if (!ws.ok) return QLR_ENOMEM;
  const T eps = (sizeof(T) == 4) ? (T)5.9604645e-08 : (T)1.1102230246251565e-16;
  const T tol = (T)8 * eps * (T)sqrt((double)l);   // above the rounding noise of the dot products
  const bool blockj = use_block_jacobi(l, sizeof(T));
  if (blockj) {
    // FP32 sweeps spread over a 16-CTA cluster where the GPU can co-schedule one (the sweeps are
    // bound by the FMA issue of the cluster's SMs), else over 8 CTAs
    const int jp = (sizeof(T) == 4) ? block_jacobi_cluster<T>(ctx->device, l) : JP;
    const int bw = (l + 2 * jp - 1) / (2 * jp);
    const size_t smem = (size_t)4 * l * 2 * bw * sizeof(T);
    // FP32 sweeps with more than 8 pairs per local round: a warp for every pair (up to 12), so a
    // local round is one pair rotation deep (the register budget of 384 threads still holds the
    // kernel's working set without spilling)
    const bool wide = sizeof(T) == 4 && bw > JB_THREADS / 32;
    auto kern = (l <= 128) ? jacobi_block_kernel<T, 4, JB_THREADS> : jacobi_block_kernel<T, 8, JB_THREADS>;
    if constexpr (sizeof(T) == 4) {
      if (wide) kern = (l <= 128) ? jacobi_block_kernel<T, 4, JB_THREADS_WIDE> : jacobi_block_kernel<T, 8, JB_THREADS_WIDE>;
    }
    QLR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    if (jp > JP) QLR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cfg.gridDim = dim3(jp, 1, 1);
    cfg.blockDim = dim3(wide ? JB_THREADS_WIDE : JB_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = jp;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    {
      KTimer kt(ctx, QLR_KID_JACOBI);
      QLR_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, R, l, bw, W, (int)JMAX_SWEEPS, tol, rlog, flags, sweeps, sig,
                                      ctx->d_err));
      qlr_count_launch();
    }
    {
      KTimer kt(ctx, QLR_KID_JACOBI);
      const size_t rs = jb_replay_smem(l, bw, jp, sizeof(T));
      // static shared memory comes on top of the dynamic size: always opt in
      QLR_CUDA_TRY(cudaFuncSetAttribute(jacobi_block_replay_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs));
      jacobi_block_replay_kernel<T><<<(l + 3) / 4, 128, rs, ctx->stream>>>(l, bw, jp, rlog, sweeps, V);
      qlr_count_launch();
      QLR_CUDA_TRY(cudaGetLastError());
    }
  } else {
    const size_t one = ll4 * sizeof(T);
    const bool w_smem = one <= 220 * 1024;
    const size_t smem = w_smem ? one : 0;
    if (smem > 0)
      QLR_CUDA_TRY(cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
      KTimer kt(ctx, QLR_KID_JACOBI);
      jacobi_kernel<T><<<1, JT, smem, ctx->stream>>>(R, l, W, w_smem, JMAX_SWEEPS, tol, sig, sweeps, rlog, ctx->d_err);
      qlr_count_launch();
    }
    QLR_CUDA_TRY(cudaGetLastError());
    {
      KTimer kt(ctx, QLR_KID_JACOBI);
      const size_t rs = (size_t)4 * 4 * l * sizeof(T);
      // static shared memory comes on top of the dynamic size: always opt in
      QLR_CUDA_TRY(cudaFuncSetAttribute(jacobi_replay_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs));
      jacobi_replay_kernel<T><<<(l + 3) / 4, 128, rs, ctx->stream>>>(l, rlog, sweeps, V);
      qlr_count_launch();
    }
  }
  QLR_CUDA_TRY(cudaGetLastError());
  if (std::getenv("QLR_DEBUG_JACOBI")) {   // diagnostics only: synchronises the stream
    int hs = -1;
    cudaMemcpyAsync(&hs, sweeps, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    std::fprintf(stderr, "qlr jacobi: l=%d sweeps=%d %s\n", l, hs, blockj ? "cluster" : "single-CTA");
  }
  { KTimer kt(ctx, QLR_KID_REFINE); rank_kernel<T><<<(l + 127) / 128, 128, 0, ctx->stream>>>(sig, l, order); qlr_count_launch(); }
  QLR_CUDA_TRY(cudaGetLastError());
  const size_t rsm = (size_t)8 * l * sizeof(double);
  // static shared memory comes on top of the dynamic size: always opt in
  QLR_CUDA_TRY(cudaFuncSetAttribute(refine_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
  {   // R's left vectors are the replayed rotations V, its right vectors W's columns (W = R^H)
    KTimer kt(ctx, QLR_KID_REFINE);
    refine_kernel<T><<<k, 256, rsm, ctx->stream>>>(R, l, V, W, order, k, L, S, Rt);
    qlr_count_launch();
  }
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

size_t jacobi_grouped_smem(int lmax) { return (size_t)2 * 4 * lmax * lmax * 4 + (size_t)lmax * 8 + 64; }

int jacobi_grouped(qlr_ctx* ctx, const JacobiGroupArgs* d_args, int count, int lmax) {
  if (count <= 0) return QLR_OK;
  if (lmax > kBatchMaxL) return QLR_EUNSUPPORTED;
  const size_t smem = jacobi_grouped_smem(lmax);
  QLR_CUDA_TRY(cudaFuncSetAttribute(jacobi_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  KTimer kt(ctx, QLR_KID_JACOBI);
  jacobi_grouped_kernel<<<count, JG_THREADS, smem, ctx->stream>>>(d_args, JMAX_SWEEPS, ctx->d_err);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

size_t core_tsvd_ws(int l) {
  return (size_t)2 * 4 * l * l * 8 + jacobi_log_floats(l) * 8 + (size_t)16 * l + JMAX_SWEEPS * 4 + 8 * 256;
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
