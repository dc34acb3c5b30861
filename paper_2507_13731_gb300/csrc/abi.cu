// C ABI: context, argument validation, and the pass scheduler for Algorithms 2 and 4.
//
// Algorithm 2 (arbitrary passes): Q2 <- Omega; for i = 1..v: odd i: [Q1, R1] = QR(X Q2),
// even i: [Q2, R2] = QR(X^H Q1); TSVD of R2 (even v: [V_hat, S, U_hat]) or R1 (odd v:
// [U_hat, S, V_hat]); V = Q2 V_hat, U = Q1 U_hat.
// Algorithm 4 (flexible block Krylov): the same alternation, with the per-pass bases of one side
// stacked into K, a QR of K, one final wide pass and the TSVD of its R.
// Section 6: the algorithm may run on X = A or on X = A^H; on A^H the two sketch operators swap
// and the outputs swap back (A ~= V' S U'^H).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "qlr_internal.h"

namespace qlr {
size_t gram_ws_bound(int64_t rows, int64_t l) {
  size_t per = (size_t)32 * l * l;
  size_t cap = std::max<size_t>(per, (size_t)64 << 20);
  const size_t tc = (l <= 1024) ? gram_tc_ws(rows, (int)l) : 0;
  return std::max(cap, tc) + (size_t)8 * ((l + 31) / 32) * ((l + 31) / 32) + 4096;
}

size_t cholqr_ws_bound(int64_t rows, int64_t l, size_t esz) {
  // + the double-FP32 copies of R and the diagonal-block inverses (FP32 sketches)
  return (size_t)12 * 32 * l * l + (size_t)8 * l * l + (size_t)4 * (rows + 4) * l * esz + (size_t)16 * l * l +
         gram_ws_bound(rows, l) + (size_t)32 * l * l + (size_t)8 * 1024 * ((l + 15) / 16) + 17 * 256;
}

size_t tsvd_ws_bound(int64_t l) { return core_tsvd_ws((int)l) + 16384; }

}  // namespace qlr

using qlr::cholqr_ws_bound;
using qlr::gram_ws_bound;
using qlr::tsvd_ws_bound;

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool valid_dtype(int d) { return d == QLR_F64 || d == QLR_F32 || d == QLR_BF16; }

int check_qmat(const qlr_qmat* q, int layout, bool allow_pure) {
  if (!q) return QLR_EINVAL;
  if (q->layout != layout || !valid_dtype(q->dtype)) return QLR_EINVAL;
  if (q->rows < 0 || q->cols < 0) return QLR_ESHAPE;
  const int64_t inner = (layout == QLR_ROW_MAJOR) ? q->cols : q->rows;
  if (q->ld < std::max<int64_t>(1, inner)) return QLR_ESHAPE;
  for (int c = 0; c < 4; ++c)
    if (q->plane[c] == nullptr && !(c == 0 && allow_pure) && q->rows > 0 && q->cols > 0) return QLR_EINVAL;
  return QLR_OK;
}

int resolve_compute(int compute, int a_dtype) {
  if (compute != QLR_COMPUTE_AUTO) return compute;
  if (a_dtype == QLR_F64) return QLR_COMPUTE_F64;
  if (a_dtype == QLR_BF16) return QLR_COMPUTE_BF16;
  return QLR_COMPUTE_TF32X3;
}

bool valid_compute(int c) { return (c >= QLR_COMPUTE_F64 && c <= QLR_COMPUTE_BF16) || c == QLR_COMPUTE_TF32_RN; }
bool tf32_family(int c) {
  return c == QLR_COMPUTE_TF32 || c == QLR_COMPUTE_TF32X3 || c == QLR_COMPUTE_TF32_RN || c == QLR_COMPUTE_TF32_MIXED;
}

// Mixed modes: the products that only feed later bases run one TF32 product; the last pass runs
// 3xTF32 (TF32_MIXED) or one TF32 product of rounded operands with chunked sums (TF32_RN).
int final_compute(int c) { return c == QLR_COMPUTE_TF32_MIXED ? QLR_COMPUTE_TF32X3 : c; }
int mid_compute(int c) { return (c == QLR_COMPUTE_TF32_MIXED || c == QLR_COMPUTE_TF32_RN) ? QLR_COMPUTE_TF32 : c; }

// Thin-matrix dtype used by the scheduler for a compute mode.
int thin_dtype(int compute) { return compute == QLR_COMPUTE_F64 ? QLR_F64 : QLR_F32; }

// ---------------------------------------------------------------------------------------
struct Sched {
  qlr_ctx* ctx;
  WsArena* ws;
  const qlr_qmat* A;
  int compute;      // arithmetic of the products that form the returned R (the last pass)
  int compute_mid;  // arithmetic of the products that only feed a later basis or Krylov block
  int tdt;          // thin dtype
  int op_fwd, op_bwd;
  int64_t rows_fwd, rows_bwd;   // X is rows_fwd x rows_bwd
  bool allow_simt_fallback = false;

  // a product whose result only feeds a later basis (mixed mode: one TF32 product)
  int sketch_mid(int op, const qlr_qmat& B, qlr_qmat& Y) {
    if (compute_mid == compute) return sketch(op, B, Y);
    Sched s2 = *this;
    s2.compute = compute_mid;
    return s2.sketch(op, B, Y);
  }

  int sketch(int op, const qlr_qmat& B, qlr_qmat& Y) {
    if (compute == QLR_COMPUTE_F64 || compute == QLR_COMPUTE_F32) {
      qlr::GemmArgs g{};
      for (int c = 0; c < 4; ++c) { g.a[c] = A->plane[c]; g.b[c] = B.plane[c]; g.c[c] = Y.plane[c]; }
      g.a_dtype = A->dtype; g.b_dtype = B.dtype; g.c_dtype = Y.dtype;
      g.ldb = B.ld; g.ldc = Y.ld;
      if (op == QLR_OP_N) { g.sa_i = A->ld; g.sa_k = 1; g.i_contig = false; g.conj_a = false; g.M = A->rows; g.K = A->cols; }
      else { g.sa_i = 1; g.sa_k = A->ld; g.i_contig = true; g.conj_a = true; g.M = A->cols; g.K = A->rows; }
      g.N = B.cols; g.alpha = 1.0; g.beta = 0.0;
      g.acc64 = (compute == QLR_COMPUTE_F64);
      g.kid = QLR_KID_SKETCH_SIMT;
      return qlr::gemm_simt(ctx, g);
    }
    if (!qlr::sketch_tc_supported(op, *A, B, compute)) {
      if (!allow_simt_fallback) return QLR_EUNSUPPORTED;
      Sched s2 = *this;                 // documented AUTO behaviour: SIMT FP32 for unsupported shapes
      s2.compute = s2.compute_mid = QLR_COMPUTE_F32;
      return s2.sketch(op, B, Y);
    }
    return qlr::sketch_tc(ctx, op, *A, B, Y, compute, *ws);
  }

  // column pitch a multiple of 4 elements (16 bytes in FP32): the tensor-core thin x small
  // products read these through TMA
  qlr_qmat thin(int64_t rows, int64_t cols, int dt = -1) {
    qlr_qmat q{};
    q.rows = rows; q.cols = cols; q.ld = std::max<int64_t>((rows + 3) / 4 * 4, 1);
    q.layout = QLR_COL_MAJOR; q.dtype = dt < 0 ? tdt : dt;
    size_t esz = qlr_dtype_size(q.dtype);
    char* p = ws->take<char>((size_t)4 * q.ld * cols * esz);
    for (int c = 0; c < 4; ++c) q.plane[c] = p ? p + (size_t)c * q.ld * cols * esz : nullptr;
    return q;
  }
};

qlr_qmat col_slice(const qlr_qmat& q, int64_t c0, int64_t nc) {
  qlr_qmat s = q;
  size_t esz = qlr_dtype_size(q.dtype);
  for (int c = 0; c < 4; ++c) s.plane[c] = q.plane[c] ? static_cast<char*>(q.plane[c]) + (size_t)c0 * q.ld * esz : nullptr;
  s.cols = nc;
  return s;
}

// Common argument checks for the algorithm entry points; resolves compute and side.
int prepare(qlr_ctx* ctx, const qlr_qmat* A, int k, int p, int passes, const qlr_qmat* omega, const qlr_opts* opts,
            int& compute, int& side, bool& auto_compute) {
  if (!ctx) return QLR_EINVAL;
  QLR_TRY(check_qmat(A, QLR_ROW_MAJOR, true));
  QLR_TRY(check_qmat(omega, QLR_COL_MAJOR, false));
  if (opts && (opts->flags & ~(QLR_FLAG_QR_EVERY_PASS | QLR_FLAG_NO_GRAPH)) != 0) return QLR_EINVAL;
  if (k < 1 || p < 0 || passes < 2) return QLR_ESHAPE;
  const int64_t l = (int64_t)k + p;
  if (l > std::min(A->rows, A->cols)) return QLR_ESHAPE;
  auto_compute = (opts == nullptr || opts->compute == QLR_COMPUTE_AUTO);
  compute = resolve_compute(opts ? opts->compute : QLR_COMPUTE_AUTO, A->dtype);
  if (!valid_compute(compute) && compute != QLR_COMPUTE_TF32_MIXED) return QLR_EINVAL;
  if (compute == QLR_COMPUTE_BF16 && A->dtype != QLR_BF16) return QLR_EINVAL;
  if (tf32_family(compute) && A->dtype != QLR_F32) return QLR_EINVAL;
  side = opts ? opts->side : QLR_SIDE_AUTO;
  if (side == QLR_SIDE_AUTO) side = (passes % 2 == 0 && A->cols > A->rows) ? QLR_SIDE_XH : QLR_SIDE_X;
  if (side != QLR_SIDE_X && side != QLR_SIDE_XH) return QLR_EINVAL;
  const int64_t om_rows = (side == QLR_SIDE_X) ? A->cols : A->rows;
  if (omega->rows != om_rows || omega->cols != l) return QLR_ESHAPE;
  if (omega->dtype == QLR_BF16) return QLR_EINVAL;
  return QLR_OK;
}

void init_sched(Sched& S, qlr_ctx* ctx, WsArena* ws, const qlr_qmat* A, int compute, int side) {
  S.ctx = ctx; S.ws = ws; S.A = A; S.compute = final_compute(compute); S.compute_mid = mid_compute(compute);
  S.tdt = thin_dtype(compute);
  S.op_fwd = (side == QLR_SIDE_X) ? QLR_OP_N : QLR_OP_H;
  S.op_bwd = (side == QLR_SIDE_X) ? QLR_OP_H : QLR_OP_N;
  S.rows_fwd = (side == QLR_SIDE_X) ? A->rows : A->cols;
  S.rows_bwd = (side == QLR_SIDE_X) ? A->cols : A->rows;
}

// Omega in the scheduler's thin dtype (copy only when the dtype differs).
int omega_in(Sched& S, const qlr_qmat* omega, qlr_qmat& out) {
  if (omega->dtype == S.tdt) { out = *omega; return QLR_OK; }
  out = S.thin(omega->rows, omega->cols);
  if (!S.ws->ok) return QLR_ENOMEM;
  return qlr::convert_qmat(S.ctx, *omega, out);
}

// Orthonormalisation of a basis that only feeds the next pass: opts.orth when every pass should
// run it, else one shifted CholeskyQR step (same column space, R discarded).
int mid_orth(const qlr_opts* opts, int orth) {
  return (opts && (opts->flags & QLR_FLAG_QR_EVERY_PASS)) ? orth : qlr::ORTH_SPAN;
}

// Algorithm 2's v passes.  Q1: rows_fwd x l, Q2: rows_bwd x l, R: last R (FP64 l x l x 4).
// Passes 1..v-2 only feed the next pass; passes v-1 and v give Q1, Q2 and R.
int run_alg2(Sched& S, int l, int v, const qlr_qmat& om, qlr_qmat& Q1, qlr_qmat& Q2, double* R, int orth, int orth_mid) {
  qlr_qmat Y = S.thin(S.rows_fwd, l), Z = S.thin(S.rows_bwd, l);
  if (!S.ws->ok) return QLR_ENOMEM;
  const qlr_qmat* q2 = &om;
  for (int i = 1; i <= v; ++i) {
    if (i % 2 == 1) {
      QLR_TRY(i == v ? S.sketch(S.op_fwd, *q2, Y) : S.sketch_mid(S.op_fwd, *q2, Y));   // X Q2
      QLR_TRY(qlr::cholqr(S.ctx, Y, Q1, i == v ? R : nullptr, i >= v - 1 ? orth : orth_mid, *S.ws));   // [Q1, R1] = QR(.)
    } else {
      QLR_TRY(i == v ? S.sketch(S.op_bwd, Q1, Z) : S.sketch_mid(S.op_bwd, Q1, Z));     // X^H Q1
      QLR_TRY(qlr::cholqr(S.ctx, Z, Q2, i == v ? R : nullptr, i >= v - 1 ? orth : orth_mid, *S.ws));   // [Q2, R2] = QR(.)
      q2 = &Q2;
    }
  }
  return QLR_OK;
}

// Block classical Gram-Schmidt of the newest block of a stack against the blocks before it:
// the slot (columns [c0, c0 + l) of K) becomes Y - B (B^H Y), B = K's columns [0, c0), once.
// B^H Y is the off-diagonal block of the FP64-class Gram of K's first c0 + l columns; the
// product B (B^H Y) accumulates in FP32.  The span of the stack is unchanged.  One pass suffices
// here: the coefficients are FP64-class and B is orthonormal to FP32 rounding, so what a second
// pass would remove (the FP32 rounding of Y along B) leaves the stack's condition number within
// ~1e-5 of 1, and the stack gets its own QR at the end.
int deflate_block(Sched& S, qlr_qmat& K, int64_t c0, int l) {
  if (c0 == 0) return QLR_OK;
  const int64_t w = c0 + l;
  const size_t mark = S.ws->off;
  double* G = S.ws->take<double>((size_t)4 * w * w);
  if (!S.ws->ok) return QLR_ENOMEM;
  const qlr_qmat KB = col_slice(K, 0, w);
  const qlr_qmat slot = col_slice(K, c0, l);
  {
    QLR_TRY(qlr::gram(S.ctx, KB, G, *S.ws));
    qlr::GemmArgs g{};
    for (int c = 0; c < 4; ++c) {
      g.a[c] = K.plane[c];                          // B(i, t) at plane + i + t ld
      g.b[c] = G + (size_t)c * w * w + (size_t)c0 * w;   // (B^H Y)(t, j) = G(t, c0 + j)
      g.c[c] = slot.plane[c];
    }
    g.sa_i = 1; g.sa_k = K.ld; g.i_contig = true; g.conj_a = false; g.a_dtype = K.dtype;
    g.ldb = w; g.b_dtype = QLR_F64;
    g.ldc = K.ld; g.c_dtype = K.dtype;
    g.M = K.rows; g.N = l; g.K = c0;
    g.alpha = -1.0; g.beta = 1.0; g.acc64 = (K.dtype == QLR_F64);
    g.kid = QLR_KID_APPLY;
    QLR_TRY(qlr::gemm_simt(S.ctx, g));
  }
  S.ws->off = mark;
  return QLR_OK;
}

// One Krylov block of Algorithm 4: slot j of the stack K receives QR(sketch of `in`), first
// deflated against the stack's earlier blocks.  In exact arithmetic the deflation changes the
// blocks that feed later views but not the span of [K_1 ... K_j] (every block's span grows by
// the same new directions), so QR(K) -- hence Q1 / Q2, R, U, S, V -- is unchanged; in floating
// point it keeps the new directions of each view, which in the plain stack sit below the FP32
// rounding of the dominant ones.
int krylov_block(Sched& S, int op, const qlr_qmat& in, qlr_qmat& K, int j, int l, qlr_qmat& tmp, int orth_mid) {
  qlr_qmat slot = col_slice(K, (int64_t)j * l, l);
  QLR_TRY(S.sketch_mid(op, in, slot));
  QLR_TRY(deflate_block(S, K, (int64_t)j * l, l));
  QLR_TRY(qlr::cholqr(S.ctx, slot, tmp, nullptr, orth_mid, *S.ws));
  const size_t esz = qlr_dtype_size(K.dtype);
  for (int c = 0; c < 4; ++c)
    QLR_CUDA_TRY(cudaMemcpy2DAsync(slot.plane[c], K.ld * esz, tmp.plane[c], tmp.ld * esz, K.rows * esz, l,
                                   cudaMemcpyDeviceToDevice, S.ctx->stream));
  return QLR_OK;
}

// Algorithm 4.  On return Q1 (rows_fwd x L), Q2 (rows_bwd x L), R (L x L) with L the stacked width.
// The per-view blocks of each side are kept in a stack (K1: range side, K2: co-range side), each
// new block deflated against the blocks before it; the stack Algorithm 4 names (K1 for even v, K2
// for odd v) then gets its QR, the other only serves the deflation.  That QR's R is discarded, but
// its Q is the final basis (it forms the last product and the lifts), so it must be orthonormal to
// working precision; the deflated stack is already well conditioned, so one plain CholeskyQR step
// does that (the plain stack needed the shifted CholeskyQR3).
int run_alg4(Sched& S, int l, int v, const qlr_qmat& om, qlr_qmat& Q1, qlr_qmat& Q2, double* R, int orth, int orth_mid) {
  const int s = (v - 1) / 2;
  const bool even = (v % 2 == 0);
  const int n1 = even ? v / 2 : s, n2 = s;          // blocks on the range / co-range side
  qlr_qmat K1 = S.thin(S.rows_fwd, (int64_t)std::max(n1, 1) * l);
  qlr_qmat K2 = S.thin(S.rows_bwd, (int64_t)std::max(n2, 1) * l);
  qlr_qmat t1 = S.thin(S.rows_fwd, l), t2 = S.thin(S.rows_bwd, l);
  if (!S.ws->ok) return QLR_ENOMEM;
  const qlr_qmat* q2prev = &om;                 // Q2_0 = Omega
  qlr_qmat q2j{};
  for (int j = 1; j <= s; ++j) {
    if (2 * j - 1 < v) {                        // odd view: Q1_j = QR(X Q2_{j-1})
      QLR_TRY(krylov_block(S, S.op_fwd, *q2prev, K1, j - 1, l, t1, orth_mid));
    }
    if (2 * j < v) {                            // even view: Q2_j = QR(X^H Q1_j)
      const qlr_qmat q1j = col_slice(K1, (int64_t)(j - 1) * l, l);
      QLR_TRY(krylov_block(S, S.op_bwd, q1j, K2, j - 1, l, t2, orth_mid));
      q2j = col_slice(K2, (int64_t)(j - 1) * l, l);
      q2prev = &q2j;
    }
  }
  const int64_t Lw = (int64_t)(even ? n1 : n2) * l;
  // the deflated stack is orthonormal up to rounding (condition number ~1): one plain CholeskyQR
  // step makes its Q orthonormal to working precision
  const int korth = (orth == QLR_ORTH_SCHOLQR3) ? orth : qlr::ORTH_ONE;
  if (even) {
    QLR_TRY(krylov_block(S, S.op_fwd, *q2prev, K1, s, l, t1, orth_mid));          // Q1_{s+1}
    QLR_TRY(qlr::cholqr(S.ctx, K1, Q1, nullptr, korth, *S.ws));                    // [Q1, ~] = QR(K1)
    qlr_qmat W = S.thin(S.rows_bwd, Lw);
    if (!S.ws->ok) return QLR_ENOMEM;
    QLR_TRY(S.sketch(S.op_bwd, Q1, W));                                             // X^H Q1
    QLR_TRY(qlr::cholqr(S.ctx, W, Q2, R, orth, *S.ws));                             // [Q2, R2]
  } else {
    QLR_TRY(qlr::cholqr(S.ctx, K2, Q2, nullptr, korth, *S.ws));                    // [Q2, ~] = QR(K2)
    qlr_qmat W = S.thin(S.rows_fwd, Lw);
    if (!S.ws->ok) return QLR_ENOMEM;
    QLR_TRY(S.sketch(S.op_fwd, Q2, W));                                             // X Q2
    QLR_TRY(qlr::cholqr(S.ctx, W, Q1, R, orth, *S.ws));                             // [Q1, R1]
  }
  return QLR_OK;
}

int64_t stacked_width(int algo, int l, int v) {
  if (algo != QLR_ALG4 && algo != QLR_ALG3) return l;
  return (int64_t)((v % 2 == 0) ? v / 2 : (v - 1) / 2) * l;
}

size_t lowrank_ws(int64_t m, int64_t n, int k, int p, int v, int algo, int compute) {
  const int64_t l = k + p;
  const int64_t L = std::max<int64_t>(l, stacked_width(algo, (int)l, v));
  const size_t esz = (compute == QLR_COMPUTE_F64) ? 8 : 4;
  const int64_t rows = std::max(m, n);
  size_t b = 0;
  b += (size_t)4 * esz * (m + n + 8) * l * 4;    // Y, Z, q1cur, q2cur (pitch padded to 4 rows)
  b += (size_t)4 * esz * (rows + 4) * L * 3;     // K, W, Q1/Q2 (stacked)
  b += (size_t)4 * esz * (m + n + 8) * L;        // Q1, Q2 when not caller-provided
  b += (size_t)4 * esz * (rows + 4) * l;         // omega conversion
  b += (size_t)32 * L * L * 3 + (size_t)64 * L * k + 8 * k;   // + the Gram of a deflated stack
  b += cholqr_ws_bound(rows, L, esz) + tsvd_ws_bound(L);
  b += qlr::sketch_tc_ws(rows, L, 160);           // tensor-core operand staging + stream-K partials
  return b + ((size_t)4 << 20);
}

}  // namespace

// ========================================================================================
static cudaEvent_t pool_get(qlr_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

static thread_local KTimer* tl_ktimer = nullptr;

void qlr_count_launch() {
  if (tl_ktimer) tl_ktimer->count += 1;
}

KTimer::KTimer(qlr_ctx* c, int k) : ctx(c), kid(k) {
  prev = tl_ktimer;
  tl_ktimer = this;
  if (ctx->timing) {
    e0 = pool_get(ctx);
    e1 = pool_get(ctx);
    if (e0) cudaEventRecord(e0, ctx->stream);
  }
}
KTimer::~KTimer() {
  tl_ktimer = prev;
  ctx->launches[kid] += count;
  if (e0 && e1) {
    cudaEventRecord(e1, ctx->stream);
    ctx->ev_pending.push_back({kid, {e0, e1}});
  }
}

static void resolve_pending(qlr_ctx* ctx) {
  for (auto& pe : ctx->ev_pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pe.second.first, pe.second.second) == cudaSuccess) ctx->ms[pe.first] += t;
    else cudaGetLastError();
    ctx->ev_pool.push_back(pe.second.first);
    ctx->ev_pool.push_back(pe.second.second);
  }
  ctx->ev_pending.clear();
}

int qlr_ensure_ws(qlr_ctx* ctx, size_t bytes) {
  if (ctx->ws_bytes >= bytes) return QLR_OK;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) return QLR_ENOMEM;
  QLR_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (ctx->ws) { cudaFree(ctx->ws); ctx->ws = nullptr; ctx->ws_bytes = 0; }
  size_t want = std::max(bytes, ctx->ws_bytes * 2);
  if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&ctx->ws, bytes) != cudaSuccess) { cudaGetLastError(); ctx->ws = nullptr; return QLR_ENOMEM; }
    want = bytes;
  }
  ctx->ws_bytes = want;
  return QLR_OK;
}

extern "C" {

int qlr_create(qlr_ctx** out, int device, void* stream) {
  if (!out) return QLR_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) { cudaGetLastError(); return QLR_ECUDA; }
  DeviceGuard g(device);
  qlr_ctx* c = new qlr_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess) { delete c; return QLR_ECUDA; }
  if (cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) { cudaFree(c->d_err); delete c; return QLR_ECUDA; }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  *out = c;
  return QLR_OK;
}

int qlr_set_timing(qlr_ctx* ctx, int enable) {
  if (!ctx) return QLR_EINVAL;
  ctx->timing = enable != 0;
  return QLR_OK;
}

int qlr_reset_stats(qlr_ctx* ctx) {
  if (!ctx) return QLR_EINVAL;
  DeviceGuard g(ctx->device);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return QLR_ECUDA;
  resolve_pending(ctx);
  for (int i = 0; i < QLR_KID_COUNT; ++i) { ctx->launches[i] = 0; ctx->ms[i] = 0.0; }
  return QLR_OK;
}

int qlr_stats(qlr_ctx* ctx, int kid, int64_t* launches, double* total_ms) {
  if (!ctx || kid < 0 || kid >= QLR_KID_COUNT) return QLR_EINVAL;
  DeviceGuard g(ctx->device);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return QLR_ECUDA;
  resolve_pending(ctx);
  if (launches) *launches = ctx->launches[kid];
  if (total_ms) *total_ms = ctx->ms[kid];
  return QLR_OK;
}

int qlr_destroy(qlr_ctx* ctx) {
  if (!ctx) return QLR_OK;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  resolve_pending(ctx);
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_err) cudaFree(ctx->d_err);
  delete ctx;
  return QLR_OK;
}

int qlr_set_stream(qlr_ctx* ctx, void* stream) {
  if (!ctx) return QLR_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return QLR_OK;
}

int qlr_reserve(qlr_ctx* ctx, size_t bytes) {
  if (!ctx) return QLR_EINVAL;
  DeviceGuard g(ctx->device);
  return qlr_ensure_ws(ctx, bytes);
}

size_t qlr_workspace_size(int64_t m, int64_t n, int k, int p, int passes, int algo, int compute) {
  return lowrank_ws(m, n, k, p, passes, algo, compute);
}

int qlr_sync(qlr_ctx* ctx) {
  if (!ctx) return QLR_EINVAL;
  DeviceGuard g(ctx->device);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return QLR_ECUDA;
  int h = 0;
  if (cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return QLR_ECUDA;
  if (h != 0) cudaMemset(ctx->d_err, 0, sizeof(int));
  return h;
}

const char* qlr_strerror(int code) {
  switch (code) {
    case QLR_OK: return "success";
    case QLR_EINVAL: return "invalid argument";
    case QLR_ESHAPE: return "inconsistent sizes (or k + p > min(m, n))";
    case QLR_ENOTPD: return "Cholesky breakdown: Gram matrix not numerically positive definite";
    case QLR_ENOCONV: return "core Jacobi QSVD did not converge";
    case QLR_ETIMEOUT: return "bounded device wait timed out";
    case QLR_ECUDA: return "CUDA error";
    case QLR_ENOMEM: return "workspace too small";
    case QLR_EUNSUPPORTED: return "unsupported combination";
  }
  return "unknown error";
}

int qlr_qsketch(qlr_ctx* ctx, int op, const qlr_qmat* A, const qlr_qmat* X, qlr_qmat* Y, int compute) {
  if (!ctx) return QLR_EINVAL;
  QLR_TRY(check_qmat(A, QLR_ROW_MAJOR, true));
  QLR_TRY(check_qmat(X, QLR_COL_MAJOR, false));
  QLR_TRY(check_qmat(Y, QLR_COL_MAJOR, false));
  if (op != QLR_OP_N && op != QLR_OP_H) return QLR_EINVAL;
  compute = resolve_compute(compute, A->dtype);
  if (!valid_compute(compute)) return QLR_EINVAL;
  const int64_t inner = (op == QLR_OP_N) ? A->cols : A->rows, outer = (op == QLR_OP_N) ? A->rows : A->cols;
  if (X->rows != inner || Y->rows != outer || Y->cols != X->cols) return QLR_ESHAPE;
  const int ydt = (compute == QLR_COMPUTE_F64) ? QLR_F64 : QLR_F32;
  if (Y->dtype != ydt) return QLR_EINVAL;
  if (compute == QLR_COMPUTE_F64 && X->dtype != QLR_F64) return QLR_EINVAL;
  if ((compute == QLR_COMPUTE_F32 || tf32_family(compute)) && X->dtype != QLR_F32) return QLR_EINVAL;
  if (compute == QLR_COMPUTE_BF16 && !(X->dtype == QLR_F32 || X->dtype == QLR_BF16)) return QLR_EINVAL;
  if (compute == QLR_COMPUTE_BF16 && A->dtype != QLR_BF16) return QLR_EINVAL;
  if (tf32_family(compute) && A->dtype != QLR_F32) return QLR_EINVAL;
  DeviceGuard g(ctx->device);
  if (outer == 0 || X->cols == 0) return QLR_OK;                        // Y is empty
  if (inner == 0) return qlr::zero_qmat(ctx, *Y);                       // empty sums: Y = 0
  if (compute >= QLR_COMPUTE_TF32) QLR_TRY(qlr_ensure_ws(ctx, qlr::sketch_tc_ws(X->rows, X->cols, ctx->num_sms)));
  WsArena ws(ctx->ws, ctx->ws_bytes);
  Sched S{};
  init_sched(S, ctx, &ws, A, compute, QLR_SIDE_X);
  return S.sketch(op, *X, *Y);
}

int qlr_qgram(qlr_ctx* ctx, const qlr_qmat* Y, double* G) {
  if (!ctx || !G) return QLR_EINVAL;
  QLR_TRY(check_qmat(Y, QLR_COL_MAJOR, false));
  if (Y->dtype == QLR_BF16) return QLR_EINVAL;
  DeviceGuard g(ctx->device);
  QLR_TRY(qlr_ensure_ws(ctx, gram_ws_bound(Y->rows, Y->cols)));
  WsArena ws(ctx->ws, ctx->ws_bytes);
  return qlr::gram(ctx, *Y, G, ws);
}

int qlr_qchol(qlr_ctx* ctx, int l, const double* G, double* R) {
  if (!ctx || !G || !R || l < 0) return QLR_EINVAL;
  if (G == R) return QLR_EINVAL;
  DeviceGuard g(ctx->device);
  QLR_TRY(qlr_ensure_ws(ctx, (size_t)40 * l * l + 65536));
  WsArena ws(ctx->ws, ctx->ws_bytes);
  return qlr::chol(ctx, l, G, R, 0.0, ws);
}

int qlr_cholqr(qlr_ctx* ctx, const qlr_qmat* Y, qlr_qmat* Q, double* R, int orth) {
  if (!ctx) return QLR_EINVAL;
  QLR_TRY(check_qmat(Y, QLR_COL_MAJOR, false));
  QLR_TRY(check_qmat(Q, QLR_COL_MAJOR, false));
  if (Y->dtype == QLR_BF16 || Q->dtype != Y->dtype) return QLR_EINVAL;
  if (Q->rows != Y->rows || Q->cols != Y->cols) return QLR_ESHAPE;
  if (Y->cols > Y->rows) return QLR_ESHAPE;
  if (orth != QLR_ORTH_CHOLQR2 && orth != QLR_ORTH_SCHOLQR3) return QLR_EINVAL;
  for (int c = 0; c < 4; ++c)
    if (Q->plane[c] == Y->plane[c]) return QLR_EINVAL;
  DeviceGuard g(ctx->device);
  QLR_TRY(qlr_ensure_ws(ctx, cholqr_ws_bound(Y->rows, Y->cols, qlr_dtype_size(Y->dtype))));
  WsArena ws(ctx->ws, ctx->ws_bytes);
  return qlr::cholqr(ctx, *Y, *Q, R, orth, ws);
}

int qlr_qtsvd(qlr_ctx* ctx, int l, const double* R, int k, double* L, double* S, double* Rt, int prec) {
  if (!ctx || !R || !L || !S || !Rt) return QLR_EINVAL;
  if (l < 1 || k < 1 || k > l) return QLR_ESHAPE;
  if (prec != QLR_F64 && prec != QLR_F32) return QLR_EINVAL;
  DeviceGuard g(ctx->device);
  QLR_TRY(qlr_ensure_ws(ctx, tsvd_ws_bound(l)));
  WsArena ws(ctx->ws, ctx->ws_bytes);
  return qlr::core_tsvd(ctx, l, R, k, L, S, Rt, prec, ws);
}

int qlr_qrangefinder(qlr_ctx* ctx, const qlr_qmat* A, int k, int p, int passes, const qlr_qmat* omega,
                     const qlr_opts* opts, qlr_qmat* Q1, qlr_qmat* Q2, double* R, int* side_used) {
  int compute, side;
  bool autoc;
  QLR_TRY(prepare(ctx, A, k, p, passes, omega, opts, compute, side, autoc));
  QLR_TRY(check_qmat(Q1, QLR_COL_MAJOR, false));
  QLR_TRY(check_qmat(Q2, QLR_COL_MAJOR, false));
  if (!R) return QLR_EINVAL;
  const int l = k + p;
  const int tdt = thin_dtype(compute);
  const int64_t rf = (side == QLR_SIDE_X) ? A->rows : A->cols, rb = (side == QLR_SIDE_X) ? A->cols : A->rows;
  if (Q1->rows != rf || Q1->cols != l || Q2->rows != rb || Q2->cols != l) return QLR_ESHAPE;
  if (Q1->dtype != tdt || Q2->dtype != tdt) return QLR_EINVAL;
  const int orth = opts ? opts->orth : QLR_ORTH_CHOLQR2;
  DeviceGuard g(ctx->device);
  QLR_TRY(qlr_ensure_ws(ctx, lowrank_ws(A->rows, A->cols, k, p, passes, QLR_ALG2, compute)));
  WsArena ws(ctx->ws, ctx->ws_bytes);
  Sched S{};
  init_sched(S, ctx, &ws, A, compute, side);
  S.allow_simt_fallback = autoc;
  qlr_qmat om;
  QLR_TRY(omega_in(S, omega, om));
  QLR_TRY(run_alg2(S, l, passes, om, *Q1, *Q2, R, orth, mid_orth(opts, orth)));
  if (side_used) *side_used = side;
  return QLR_OK;
}

// Algorithms 1 and 3 take 2q + 2 passes and, for the same Omega, give the results of Algorithm 2
// and Algorithm 4 with that (even) number of passes (Sections 3 and 5): they run those schedules
// with a QR after every product, as the classical methods orthonormalise every power step.
static int canonical_algo(int algo, int passes, const qlr_opts* opts, int& algo_out, qlr_opts& o) {
  o = opts ? *opts : qlr_opts{QLR_COMPUTE_AUTO, QLR_SIDE_AUTO, QLR_ORTH_CHOLQR2, 0};
  if (algo == QLR_ALG2 || algo == QLR_ALG4) {
    algo_out = algo;
    return QLR_OK;
  }
  if (algo != QLR_ALG1 && algo != QLR_ALG3) return QLR_EINVAL;
  if (passes < 2 || passes % 2 != 0) return QLR_ESHAPE;
  algo_out = (algo == QLR_ALG1) ? QLR_ALG2 : QLR_ALG4;
  o.flags |= QLR_FLAG_QR_EVERY_PASS;
  return QLR_OK;
}

static int lowrank_impl(qlr_ctx* ctx, const qlr_qmat* A, int k, int p, int passes, int algo_in,
                        const qlr_qmat* omega, const qlr_opts* opts_in, qlr_qmat* U, double* S_out, qlr_qmat* V) {
  int algo = QLR_ALG2;
  qlr_opts opts_c;
  QLR_TRY(canonical_algo(algo_in, passes, opts_in, algo, opts_c));
  const qlr_opts* opts = &opts_c;
  int compute, side;
  bool autoc;
  QLR_TRY(prepare(ctx, A, k, p, passes, omega, opts, compute, side, autoc));
  QLR_TRY(check_qmat(U, QLR_COL_MAJOR, false));
  QLR_TRY(check_qmat(V, QLR_COL_MAJOR, false));
  if (!S_out) return QLR_EINVAL;
  if (U->rows != A->rows || U->cols != k || V->rows != A->cols || V->cols != k) return QLR_ESHAPE;
  if (U->dtype == QLR_BF16 || V->dtype == QLR_BF16) return QLR_EINVAL;
  const int l = k + p;
  const int64_t L = stacked_width(algo, l, passes);
  if (L > std::min(A->rows, A->cols)) return QLR_ESHAPE;
  const int orth = opts ? opts->orth : QLR_ORTH_CHOLQR2;
  DeviceGuard g(ctx->device);
  QLR_TRY(qlr_ensure_ws(ctx, lowrank_ws(A->rows, A->cols, k, p, passes, algo, compute)));
  WsArena ws(ctx->ws, ctx->ws_bytes);
  Sched S{};
  init_sched(S, ctx, &ws, A, compute, side);
  S.allow_simt_fallback = autoc;
  qlr_qmat om;
  QLR_TRY(omega_in(S, omega, om));
  qlr_qmat Q1 = S.thin(S.rows_fwd, L), Q2 = S.thin(S.rows_bwd, L);
  double* R = ws.take<double>((size_t)4 * L * L);
  double* Lm = ws.take<double>((size_t)4 * L * k);
  double* Rt = ws.take<double>((size_t)4 * L * k);
  if (!ws.ok) return QLR_ENOMEM;
  if (algo == QLR_ALG2) QLR_TRY(run_alg2(S, l, passes, om, Q1, Q2, R, orth, mid_orth(opts, orth)));
  else QLR_TRY(run_alg4(S, l, passes, om, Q1, Q2, R, orth, mid_orth(opts, orth)));
  const int prec = (compute == QLR_COMPUTE_F64) ? QLR_F64 : QLR_F32;
  QLR_TRY(qlr::core_tsvd(ctx, (int)L, R, k, Lm, S_out, Rt, prec, ws));
  // even v: [V_hat, S, U_hat] = TSVD(R2); odd v: [U_hat, S, V_hat] = TSVD(R1)
  const double* Uhat = (passes % 2 == 0) ? Rt : Lm;
  const double* Vhat = (passes % 2 == 0) ? Lm : Rt;
  qlr_qmat* UX = (side == QLR_SIDE_X) ? U : V;   // U of the algorithm's X
  qlr_qmat* VX = (side == QLR_SIDE_X) ? V : U;
  QLR_TRY(qlr::thin_times_small(ctx, Q1, Uhat, (int)L, k, *UX, ws));   // U = Q1 U_hat
  QLR_TRY(qlr::thin_times_small(ctx, Q2, Vhat, (int)L, k, *VX, ws));   // V = Q2 V_hat
  return QLR_OK;
}

int qlr_qbasis(qlr_ctx* ctx, const qlr_qmat* A, int k, int p, int passes, int algo_in, const qlr_qmat* omega,
               const qlr_opts* opts_in, qlr_qmat* Q1, qlr_qmat* Q2, double* R, int* side_used) {
  int algo = QLR_ALG2;
  qlr_opts opts_c;
  QLR_TRY(canonical_algo(algo_in, passes, opts_in, algo, opts_c));
  const qlr_opts* opts = &opts_c;
  int compute, side;
  bool autoc;
  QLR_TRY(prepare(ctx, A, k, p, passes, omega, opts, compute, side, autoc));
  QLR_TRY(check_qmat(Q1, QLR_COL_MAJOR, false));
  QLR_TRY(check_qmat(Q2, QLR_COL_MAJOR, false));
  if (!R) return QLR_EINVAL;
  const int l = k + p;
  const int64_t L = stacked_width(algo, l, passes);
  if (L > std::min(A->rows, A->cols)) return QLR_ESHAPE;
  const int tdt = thin_dtype(compute);
  const int64_t rf = (side == QLR_SIDE_X) ? A->rows : A->cols, rb = (side == QLR_SIDE_X) ? A->cols : A->rows;
  if (Q1->rows != rf || Q1->cols != L || Q2->rows != rb || Q2->cols != L) return QLR_ESHAPE;
  if (Q1->dtype != tdt || Q2->dtype != tdt) return QLR_EINVAL;
  const int orth = opts->orth;
  DeviceGuard g(ctx->device);
  QLR_TRY(qlr_ensure_ws(ctx, lowrank_ws(A->rows, A->cols, k, p, passes, algo, compute)));
  WsArena ws(ctx->ws, ctx->ws_bytes);
  Sched S{};
  init_sched(S, ctx, &ws, A, compute, side);
  S.allow_simt_fallback = autoc;
  qlr_qmat om;
  QLR_TRY(omega_in(S, omega, om));
  if (algo == QLR_ALG2) QLR_TRY(run_alg2(S, l, passes, om, *Q1, *Q2, R, orth, mid_orth(opts, orth)));
  else QLR_TRY(run_alg4(S, l, passes, om, *Q1, *Q2, R, orth, mid_orth(opts, orth)));
  if (side_used) *side_used = side;
  return QLR_OK;
}

int qlr_qsvd_lowrank(qlr_ctx* ctx, const qlr_qmat* A, int k, int p, int passes, int algo, const qlr_qmat* omega,
                     const qlr_opts* opts, qlr_qmat* U, double* S, qlr_qmat* V) {
  return lowrank_impl(ctx, A, k, p, passes, algo, omega, opts, U, S, V);
}

int qlr_qblock_krylov(qlr_ctx* ctx, const qlr_qmat* A, int k, int b, int passes, const qlr_qmat* omega,
                      const qlr_opts* opts, qlr_qmat* U, double* S, qlr_qmat* V) {
  if (b < k) return QLR_ESHAPE;
  return lowrank_impl(ctx, A, k, b - k, passes, QLR_ALG4, omega, opts, U, S, V);
}

// Checks of the masked completion update's operands (k = 0: U, S, V unused).
static int complete_args(const qlr_qmat* M, const uint8_t* mask, int64_t mask_ld, const qlr_qmat* U, const double* S,
                         const qlr_qmat* V, int k, const qlr_qmat* C, qlr::CompleteArgs& a) {
  QLR_TRY(check_qmat(M, QLR_ROW_MAJOR, true));
  QLR_TRY(check_qmat(C, QLR_ROW_MAJOR, false));
  if (M->dtype != C->dtype || (C->dtype != QLR_F32 && C->dtype != QLR_F64)) return QLR_EINVAL;
  if (M->rows != C->rows || M->cols != C->cols || k < 0) return QLR_ESHAPE;
  if (!mask && C->rows > 0 && C->cols > 0) return QLR_EINVAL;
  if (mask_ld < std::max<int64_t>(1, C->cols)) return QLR_ESHAPE;
  a = qlr::CompleteArgs{};
  if (k > 0) {
    QLR_TRY(check_qmat(U, QLR_COL_MAJOR, false));
    QLR_TRY(check_qmat(V, QLR_COL_MAJOR, false));
    if (!S) return QLR_EINVAL;
    if (U->dtype != C->dtype || V->dtype != C->dtype) return QLR_EINVAL;
    if (U->rows != C->rows || V->rows != C->cols || U->cols < k || V->cols < k) return QLR_ESHAPE;
    for (int c = 0; c < 4; ++c) { a.U[c] = U->plane[c]; a.V[c] = V->plane[c]; }
    a.ldu = U->ld;
    a.ldv = V->ld;
    a.S = S;
  }
  for (int c = 0; c < 4; ++c) { a.M[c] = M->plane[c]; a.C[c] = C->plane[c]; }
  a.ldm = M->ld;
  a.ldc = C->ld;
  a.mask = mask;
  a.ldk = mask_ld;
  a.m = C->rows;
  a.n = C->cols;
  a.k = k;
  return QLR_OK;
}

int qlr_qcomplete_update(qlr_ctx* ctx, const qlr_qmat* M, const uint8_t* mask, int64_t mask_ld, const qlr_qmat* U,
                         const double* S, const qlr_qmat* V, int k, qlr_qmat* C) {
  if (!ctx) return QLR_EINVAL;
  qlr::CompleteArgs a;
  QLR_TRY(complete_args(M, mask, mask_ld, U, S, V, k, C, a));
  DeviceGuard g(ctx->device);
  return qlr::complete_update(ctx, a, C->dtype);
}

int qlr_qcomplete(qlr_ctx* ctx, const qlr_qmat* M, const uint8_t* mask, int64_t mask_ld, int k, int p, int passes,
                  int algo, int iters, const qlr_qmat* omega, const qlr_opts* opts, qlr_qmat* C, qlr_qmat* U,
                  double* S, qlr_qmat* V) {
  if (!ctx) return QLR_EINVAL;
  if (iters < 1 || k < 1) return QLR_ESHAPE;
  qlr::CompleteArgs start, update;
  QLR_TRY(complete_args(M, mask, mask_ld, nullptr, nullptr, nullptr, 0, C, start));
  QLR_TRY(complete_args(M, mask, mask_ld, U, S, V, k, C, update));
  DeviceGuard g(ctx->device);
  QLR_TRY(qlr::complete_update(ctx, start, C->dtype));                        // C = P_Omega(M)
  for (int it = 0; it < iters; ++it) {
    QLR_TRY(lowrank_impl(ctx, C, k, p, passes, algo, omega, opts, U, S, V));   // eq. Step1
    QLR_TRY(qlr::complete_update(ctx, update, C->dtype));                     // eq. Step2
  }
  return QLR_OK;
}

int qlr_selftest_wait_timeout(qlr_ctx* ctx) {
  if (!ctx) return QLR_EINVAL;
  DeviceGuard g(ctx->device);
  return qlr::selftest_wait_timeout(ctx);
}

int qlr_qsvd_lowrank_batched(qlr_ctx* ctx, int count, const qlr_qmat* A, const int* k, const int* p, int passes,
                             const qlr_qmat* omega, const qlr_opts* opts, qlr_qmat* U, double* const* S, qlr_qmat* V) {
  if (!ctx || count < 0 || (count > 0 && (!A || !k || !p || !omega || !U || !S || !V))) return QLR_EINVAL;
  if (count == 0) return QLR_OK;
  qlr_batch* b = nullptr;
  const int rc = qlr::batch_create(ctx, count, A, k, p, passes, omega, opts, U, S, V, false, false, &b);
  if (rc == QLR_OK) return qlr_batch_destroy(b);   // the plan's creation ran it once
  if (rc != QLR_EUNSUPPORTED && rc != QLR_EINVAL) return rc;
  for (int i = 0; i < count; ++i)
    QLR_TRY(lowrank_impl(ctx, &A[i], k[i], p[i], passes, QLR_ALG2, &omega[i], opts, &U[i], S[i], &V[i]));
  return QLR_OK;
}

// Largest eigenvalue of an n x n quaternion Hermitian matrix G (four column-major FP64 planes,
// host) by power iteration with Rayleigh quotients; n is the handful of vectors of a block.
static double herm_lmax(const std::vector<double>& g, int64_t n) {
  const size_t nn = (size_t)n * n;
  std::vector<double> x((size_t)4 * n), y((size_t)4 * n);
  for (int64_t i = 0; i < n; ++i) {     // a start with components along every direction
    x[i] = 1.0;
    x[n + i] = 0.25 + 0.125 * (double)(i % 5);
    x[2 * n + i] = -0.5 + 0.0625 * (double)(i % 7);
    x[3 * n + i] = 0.375 - 0.03125 * (double)(i % 3);
  }
  double lam = 0.0;
  for (int it = 0; it < 5000; ++it) {
    double xx = 0.0, xy = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double acc[4] = {0, 0, 0, 0};
      for (int64_t j = 0; j < n; ++j) {   // y_i = sum_j G_ij x_j (Hamilton product, eq. 1)
        const size_t o = (size_t)j * n + i;
        const double a0 = g[o], a1 = g[nn + o], a2 = g[2 * nn + o], a3 = g[3 * nn + o];
        const double b0 = x[j], b1 = x[n + j], b2 = x[2 * n + j], b3 = x[3 * n + j];
        acc[0] += a0 * b0 - a1 * b1 - a2 * b2 - a3 * b3;
        acc[1] += a0 * b1 + a1 * b0 + a2 * b3 - a3 * b2;
        acc[2] += a0 * b2 - a1 * b3 + a2 * b0 + a3 * b1;
        acc[3] += a0 * b3 + a1 * b2 - a2 * b1 + a3 * b0;
      }
      for (int c = 0; c < 4; ++c) {
        y[(size_t)c * n + i] = acc[c];
        xx += x[(size_t)c * n + i] * x[(size_t)c * n + i];
        xy += x[(size_t)c * n + i] * acc[c];       // Re(x^H y)
      }
    }
    const double lnew = xx > 0.0 ? xy / xx : 0.0;
    double yy = 0.0;
    for (double v : y) yy += v * v;
    if (!(yy > 0.0)) return lnew;
    const double inv = 1.0 / std::sqrt(yy);
    for (size_t e = 0; e < y.size(); ++e) x[e] = y[e] * inv;
    const bool done = it > 8 && std::fabs(lnew - lam) <= 1e-15 * std::fabs(lnew);
    lam = lnew;
    if (done) break;
  }
  return lam;
}

int qlr_residual_norm(qlr_ctx* ctx, const qlr_qmat* A, const qlr_qmat* Q, int side, const qlr_qmat* start, int iters,
                      double* out) {
  if (!ctx || !out) return QLR_EINVAL;
  QLR_TRY(check_qmat(A, QLR_ROW_MAJOR, true));
  QLR_TRY(check_qmat(Q, QLR_COL_MAJOR, false));
  QLR_TRY(check_qmat(start, QLR_COL_MAJOR, false));
  if (side != QLR_SIDE_X && side != QLR_SIDE_XH) return QLR_EINVAL;
  if (Q->dtype != start->dtype || Q->dtype == QLR_BF16) return QLR_EINVAL;
  const int64_t qrows = (side == QLR_SIDE_X) ? A->rows : A->cols;
  if (Q->rows != qrows || start->rows != A->cols || iters < 1 || start->cols < 1) return QLR_ESHAPE;
  DeviceGuard g(ctx->device);
  const int64_t nv = start->cols, l = Q->cols;
  const int cmp = (Q->dtype == QLR_F64) ? QLR_COMPUTE_F64 : QLR_COMPUTE_F32;
  size_t esz = qlr_dtype_size(Q->dtype);
  QLR_TRY(qlr_ensure_ws(ctx, (size_t)4 * esz * (A->rows + A->cols) * nv * 3 + (size_t)4 * esz * l * nv +
                                 cholqr_ws_bound(A->cols, nv, esz) + ((size_t)1 << 20)));
  WsArena ws(ctx->ws, ctx->ws_bytes);
  Sched S{};
  init_sched(S, ctx, &ws, A, cmp, QLR_SIDE_X);
  qlr_qmat x = S.thin(A->cols, nv), xt = S.thin(A->cols, nv), y = S.thin(A->rows, nv), h = S.thin(l, nv);
  if (!ws.ok) return QLR_ENOMEM;
  QLR_TRY(qlr::convert_qmat(ctx, *start, x));
  // P z = z - Q (Q^H z)
  auto project = [&](qlr_qmat& z) -> int {
    qlr::GemmArgs g1{};
    for (int c = 0; c < 4; ++c) { g1.a[c] = Q->plane[c]; g1.b[c] = z.plane[c]; g1.c[c] = h.plane[c]; }
    g1.sa_i = Q->ld; g1.sa_k = 1; g1.i_contig = false; g1.conj_a = true; g1.a_dtype = Q->dtype;
    g1.ldb = z.ld; g1.b_dtype = z.dtype; g1.ldc = h.ld; g1.c_dtype = h.dtype;
    g1.M = l; g1.N = nv; g1.K = Q->rows; g1.alpha = 1.0; g1.beta = 0.0; g1.acc64 = (cmp == QLR_COMPUTE_F64);
    QLR_TRY(qlr::gemm_simt(ctx, g1));
    qlr::GemmArgs g2{};
    for (int c = 0; c < 4; ++c) { g2.a[c] = Q->plane[c]; g2.b[c] = h.plane[c]; g2.c[c] = z.plane[c]; }
    g2.sa_i = 1; g2.sa_k = Q->ld; g2.i_contig = true; g2.conj_a = false; g2.a_dtype = Q->dtype;
    g2.ldb = h.ld; g2.b_dtype = h.dtype; g2.ldc = z.ld; g2.c_dtype = z.dtype;
    g2.M = Q->rows; g2.N = nv; g2.K = l; g2.alpha = -1.0; g2.beta = 1.0; g2.acc64 = (cmp == QLR_COMPUTE_F64);
    return qlr::gemm_simt(ctx, g2);
  };
  double* norms = ws.take<double>((size_t)4 * nv * nv);
  if (!ws.ok) return QLR_ENOMEM;
  double best = 0.0;
  for (int it = 0; it < iters; ++it) {
    QLR_TRY(qlr::cholqr(ctx, x, xt, nullptr, QLR_ORTH_SCHOLQR3, ws));   // orthonormal block
    if (side == QLR_SIDE_XH) QLR_TRY(project(xt));
    QLR_TRY(S.sketch(QLR_OP_N, xt, y));        // y = A x
    if (side == QLR_SIDE_X) QLR_TRY(project(y));
    // ||E x|| per column (Gram diagonal) -> lower bound on ||E||_2
    QLR_TRY(qlr::gram(ctx, y, norms, ws));
    std::vector<double> hg((size_t)4 * nv * nv);
    QLR_CUDA_TRY(cudaMemcpyAsync(hg.data(), norms, hg.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    QLR_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    // Rayleigh-Ritz: ||E x_block||_2 = sqrt(lambda_max(Y^H Y)) for the orthonormal block x
    best = std::max(best, std::sqrt(std::max(0.0, herm_lmax(hg, nv))));
    QLR_TRY(S.sketch(QLR_OP_H, y, x));         // x = A^H y (= E^H y for side X)
    if (side == QLR_SIDE_XH) QLR_TRY(project(x));
  }
  *out = best;
  return QLR_OK;
}

}  // extern "C"
