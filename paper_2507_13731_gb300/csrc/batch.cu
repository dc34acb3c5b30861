// Batched Algorithm 2 over many independent problems (image patches / frames of uneven sizes).
//
// One plan per problem set.  Every pass is one grouped tensor-core sketch launch over all the
// problems' output tiles (sketch_tc.cu), preceded by one grouped staging launch of their thin
// operands.  Between passes the per-problem orthonormalisations (and after the last pass the core
// QSVDs and lifts) run on a set of side streams ("lanes"), problems dealt round-robin, so that
// the many small latency-bound kernels of different problems overlap on the GPU.  The whole
// sequence is captured once into a CUDA graph and replayed by every run.  At plan time a small
// autotuner times the grouped sketch's tile orders and keeps the faster one.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "qlr_internal.h"

struct qlr_batch {
  struct Prob {
    qlr_qmat A, om, U, V, Y, Z, Q1, Q2;
    double* S;
    double *R, *Lm, *Rt;
    int k, p, l;
  };
  qlr_ctx* ctx = nullptr;
  qlr_ctx main_ctx;                         // issues the grouped launches, untimed: on ctx->stream, or
                                            // on cap_stream while the graph is captured
  cudaStream_t cap_stream = nullptr;        // capture needs a stream other than the legacy default
  int count = 0, passes = 0, compute = 0, orth = 0, mid = 0, lanes = 0;
  std::vector<Prob> pr;
  std::vector<cudaStream_t> ls;
  std::vector<qlr_ctx> lctx;
  std::vector<char*> lws;
  size_t lws_bytes = 0;
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  qlr::GroupedSketch gs[3];                 // (N, Omega -> Y), (H, Q1 -> Z), (N, Q2 -> Y)
  char* gdev[3] = {nullptr, nullptr, nullptr};
  size_t gbytes[3] = {0, 0, 0};
  void* dev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int order = 1;                            // chosen grouped-sketch variant (bit 0 order, bit 1 persistent)
  float tune_ms[4] = {0.f, 0.f, 0.f, 0.f};
  int64_t launches_per_run = 0;
};

namespace {

// Side streams: enough that the per-problem chains of small, latency-bound kernels fill the GPU
// (the hardware runs up to 128 kernels at once).
constexpr int kMaxLanes = 128;

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int check_q(const qlr_qmat* q, int layout, int dtype, bool allow_pure) {
  if (!q || q->layout != layout || q->dtype != dtype) return QLR_EINVAL;
  if (q->rows <= 0 || q->cols <= 0) return QLR_ESHAPE;
  const int64_t inner = (layout == QLR_ROW_MAJOR) ? q->cols : q->rows;
  if (q->ld < inner) return QLR_ESHAPE;
  for (int c = 0; c < 4; ++c)
    if (q->plane[c] == nullptr && !(c == 0 && allow_pure)) return QLR_EINVAL;
  return QLR_OK;
}

// Column-major FP32 thin matrix with a 16-byte multiple column pitch (the tensor-core thin x
// small products read it through TMA).
qlr_qmat thin_at(char*& cur, int64_t rows, int64_t cols) {
  qlr_qmat q{};
  q.rows = rows; q.cols = cols; q.ld = (rows + 3) / 4 * 4; q.layout = QLR_COL_MAJOR; q.dtype = QLR_F32;
  const size_t plane = (size_t)q.ld * cols * 4;
  for (int c = 0; c < 4; ++c) q.plane[c] = cur + (size_t)c * plane;
  cur += (4 * plane + 255) / 256 * 256;
  return q;
}

double* small_at(char*& cur, size_t doubles) {
  double* p = reinterpret_cast<double*>(cur);
  cur += (doubles * 8 + 255) / 256 * 256;
  return p;
}

const qlr::GroupedSketch& plan_of(const qlr_batch* b, int pass) {
  return pass == 1 ? b->gs[0] : (pass % 2 == 0 ? b->gs[1] : b->gs[2]);
}

// The whole batched QSVD, enqueued on main_ctx.stream (and the lanes, forked from and joined to it).
int enqueue(qlr_batch* b) {
  const int v = b->passes;
  cudaStream_t ms = b->main_ctx.stream;
  int64_t launches = 0;
  for (int i = 1; i <= v; ++i) {
    QLR_TRY(qlr::sketch_tc_grouped_run(&b->main_ctx, plan_of(b, i)));
    launches += 2;
    QLR_CUDA_TRY(cudaEventRecord(b->fork_ev, ms));
    for (int L = 0; L < b->lanes; ++L) QLR_CUDA_TRY(cudaStreamWaitEvent(b->ls[L], b->fork_ev, 0));
    for (int j = 0; j < b->count; ++j) {
      const int L = j % b->lanes;
      qlr_ctx* lc = &b->lctx[L];
      WsArena ws(b->lws[L], b->lws_bytes);
      qlr_batch::Prob& P = b->pr[j];
      const int orth = (i >= v - 1) ? b->orth : b->mid;
      if (i % 2 == 1) QLR_TRY(qlr::cholqr(lc, P.Y, P.Q1, i == v ? P.R : nullptr, orth, ws));
      else QLR_TRY(qlr::cholqr(lc, P.Z, P.Q2, i == v ? P.R : nullptr, orth, ws));
      if (i == v) {
        ws.off = 0;
        QLR_TRY(qlr::core_tsvd(lc, P.l, P.R, P.k, P.Lm, P.S, P.Rt, QLR_F32, ws));
        // even v: [V_hat, S, U_hat] = TSVD(R2); odd v: [U_hat, S, V_hat] = TSVD(R1)
        const double* Uhat = (v % 2 == 0) ? P.Rt : P.Lm;
        const double* Vhat = (v % 2 == 0) ? P.Lm : P.Rt;
        QLR_TRY(qlr::thin_times_small(lc, P.Q1, Uhat, P.l, P.k, P.U, ws));
        QLR_TRY(qlr::thin_times_small(lc, P.Q2, Vhat, P.l, P.k, P.V, ws));
      }
    }
    for (int L = 0; L < b->lanes; ++L) {
      QLR_CUDA_TRY(cudaEventRecord(b->join_ev[L], b->ls[L]));
      QLR_CUDA_TRY(cudaStreamWaitEvent(ms, b->join_ev[L], 0));
    }
  }
  int64_t lane_launches = 0;
  for (auto& lc : b->lctx) {
    for (int kk = 0; kk < QLR_KID_COUNT; ++kk) lane_launches += lc.launches[kk];
    std::fill(std::begin(lc.launches), std::end(lc.launches), 0);
  }
  std::fill(std::begin(b->main_ctx.launches), std::end(b->main_ctx.launches), 0);
  b->launches_per_run = launches + lane_launches;
  return QLR_OK;
}

int plan_sketches(qlr_batch* b, int order) {
  std::vector<qlr_qmat> A(b->count), X(b->count), Y(b->count);
  for (int pass = 0; pass < 3; ++pass) {
    const int op = (pass == 1) ? QLR_OP_H : QLR_OP_N;
    for (int j = 0; j < b->count; ++j) {
      const qlr_batch::Prob& P = b->pr[j];
      A[j] = P.A;
      X[j] = pass == 0 ? P.om : (pass == 1 ? P.Q1 : P.Q2);
      Y[j] = pass == 1 ? P.Z : P.Y;
    }
    QLR_TRY(qlr::sketch_tc_grouped_plan(b->ctx, op, b->count, A.data(), X.data(), Y.data(), b->compute, order,
                                        b->gdev[pass], b->gbytes[pass], b->gs[pass]));
  }
  return QLR_OK;
}

// Autotuner: time the grouped sketch variants -- tile order (problem order / longest reduction
// first) x schedule (one CTA per tile / one persistent CTA per SM) -- on passes N and H, best of
// three after a warm-up, and keep the fastest.
int autotune(qlr_batch* b) {
  cudaEvent_t e0, e1;
  QLR_CUDA_TRY(cudaEventCreate(&e0));
  QLR_CUDA_TRY(cudaEventCreate(&e1));
  int rc = QLR_OK;
  for (int order = 0; order < 4 && rc == QLR_OK; ++order) {
    rc = plan_sketches(b, order);
    if (rc != QLR_OK) break;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && rc == QLR_OK; ++rep) {
      cudaEventRecord(e0, b->ctx->stream);
      rc = qlr::sketch_tc_grouped_run(&b->main_ctx, b->gs[0]);
      if (rc == QLR_OK) rc = qlr::sketch_tc_grouped_run(&b->main_ctx, b->gs[1]);
      cudaEventRecord(e1, b->ctx->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = QLR_ECUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, ms);
    }
    b->tune_ms[order] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  QLR_TRY(rc);
  b->order = (int)(std::min_element(b->tune_ms, b->tune_ms + 4) - b->tune_ms);
  return plan_sketches(b, b->order);
}

void release(qlr_batch* b) {
  if (!b) return;
  if (b->ctx) cudaStreamSynchronize(b->ctx->stream);
  for (auto s : b->ls) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (auto e : b->join_ev) cudaEventDestroy(e);
  if (b->dev) cudaFree(b->dev);
  delete b;
}

}  // namespace

namespace qlr {

int batch_create(qlr_ctx* ctx, int count, const qlr_qmat* A, const int* k, const int* p, int passes,
                 const qlr_qmat* omega, const qlr_opts* opts, qlr_qmat* U, double* const* S, qlr_qmat* V,
                 bool tune, bool use_graph, qlr_batch** out) {
  if (!ctx || !out || count <= 0 || !A || !k || !p || !omega || !U || !S || !V) return QLR_EINVAL;
  *out = nullptr;
  if (passes < 2) return QLR_ESHAPE;
  if (opts && (opts->flags & ~(QLR_FLAG_QR_EVERY_PASS | QLR_FLAG_NO_GRAPH)) != 0) return QLR_EINVAL;
  if (opts && opts->side == QLR_SIDE_XH) return QLR_EINVAL;
  const int req = opts ? opts->compute : QLR_COMPUTE_AUTO;
  const int compute = (req == QLR_COMPUTE_AUTO) ? (A[0].dtype == QLR_BF16 ? QLR_COMPUTE_BF16 : QLR_COMPUTE_TF32X3) : req;
  if (compute != QLR_COMPUTE_BF16 && compute != QLR_COMPUTE_TF32 && compute != QLR_COMPUTE_TF32X3) return QLR_EUNSUPPORTED;
  const int adt = (compute == QLR_COMPUTE_BF16) ? QLR_BF16 : QLR_F32;
  const int orth = opts ? opts->orth : QLR_ORTH_CHOLQR2;
  if (orth != QLR_ORTH_CHOLQR2 && orth != QLR_ORTH_SCHOLQR3) return QLR_EINVAL;
  if (opts && (opts->flags & QLR_FLAG_NO_GRAPH)) use_graph = false;
  for (int j = 0; j < count; ++j) {
    QLR_TRY(check_q(&A[j], QLR_ROW_MAJOR, adt, true));
    const int l = k[j] + p[j];
    if (k[j] < 1 || p[j] < 0 || l > std::min(A[j].rows, A[j].cols)) return QLR_ESHAPE;
    QLR_TRY(check_q(&omega[j], QLR_COL_MAJOR, QLR_F32, false));
    QLR_TRY(check_q(&U[j], QLR_COL_MAJOR, QLR_F32, false));
    QLR_TRY(check_q(&V[j], QLR_COL_MAJOR, QLR_F32, false));
    if (omega[j].rows != A[j].cols || omega[j].cols != l) return QLR_ESHAPE;
    if (U[j].rows != A[j].rows || U[j].cols != k[j] || V[j].rows != A[j].cols || V[j].cols != k[j]) return QLR_ESHAPE;
    if (!S[j]) return QLR_EINVAL;
    if (!qlr::sketch_tc_supported(QLR_OP_N, A[j], omega[j], compute)) return QLR_EUNSUPPORTED;
  }
  DevGuard g(ctx->device);
  qlr_batch* b = new qlr_batch();
  b->ctx = ctx;
  b->count = count;
  b->passes = passes;
  b->compute = compute;
  b->orth = orth;
  b->mid = (opts && (opts->flags & QLR_FLAG_QR_EVERY_PASS)) ? orth : ORTH_SPAN;
  b->lanes = std::min(count, kMaxLanes);
  b->main_ctx.device = ctx->device;
  b->main_ctx.stream = ctx->stream;
  b->main_ctx.d_err = ctx->d_err;
  b->main_ctx.num_sms = ctx->num_sms;
  b->pr.resize(count);

  // sizes: per-problem thin and small buffers, the three grouped plans, the lane workspaces
  size_t bytes = 0, lane_need = 0;
  int64_t maxl = 0;
  for (int j = 0; j < count; ++j) {
    const int64_t m = A[j].rows, n = A[j].cols, l = k[j] + p[j];
    const int64_t mp = (m + 3) / 4 * 4, np = (n + 3) / 4 * 4;
    bytes += 2 * ((4 * (size_t)mp * l * 4 + 255) / 256 * 256) + 2 * ((4 * (size_t)np * l * 4 + 255) / 256 * 256);
    bytes += ((size_t)4 * l * l * 8 + 255) / 256 * 256 + 2 * (((size_t)4 * l * k[j] * 8 + 255) / 256 * 256);
    lane_need = std::max(lane_need, cholqr_ws_bound(std::max(m, n), l, 4) + tsvd_ws_bound(l));
    maxl = std::max(maxl, l);
  }
  (void)maxl;
  // thin operands of the grouped plans are described before their buffers exist: sizes only
  std::vector<qlr_qmat> Av(A, A + count), Xn(count), Xh(count);
  for (int j = 0; j < count; ++j) {
    const int l = k[j] + p[j];
    Xn[j] = omega[j];
    Xh[j] = omega[j];
    Xh[j].rows = A[j].rows;
    Xh[j].ld = A[j].rows;
    Xn[j].cols = Xh[j].cols = l;
  }
  b->gbytes[0] = b->gbytes[2] = sketch_tc_grouped_bytes(QLR_OP_N, count, Av.data(), Xn.data(), compute);
  b->gbytes[1] = sketch_tc_grouped_bytes(QLR_OP_H, count, Av.data(), Xh.data(), compute);
  b->lws_bytes = (lane_need + 255) / 256 * 256;
  const size_t total = bytes + b->gbytes[0] + b->gbytes[1] + b->gbytes[2] + (size_t)b->lanes * b->lws_bytes + 4096;
  if (cudaMalloc(&b->dev, total) != cudaSuccess) {
    cudaGetLastError();
    release(b);
    return QLR_ENOMEM;
  }
  char* cur = static_cast<char*>(b->dev);
  for (int j = 0; j < count; ++j) {
    qlr_batch::Prob& P = b->pr[j];
    P.A = A[j]; P.om = omega[j]; P.U = U[j]; P.V = V[j]; P.S = S[j];
    P.k = k[j]; P.p = p[j]; P.l = k[j] + p[j];
    P.Y = thin_at(cur, A[j].rows, P.l);
    P.Q1 = thin_at(cur, A[j].rows, P.l);
    P.Z = thin_at(cur, A[j].cols, P.l);
    P.Q2 = thin_at(cur, A[j].cols, P.l);
    P.R = small_at(cur, (size_t)4 * P.l * P.l);
    P.Lm = small_at(cur, (size_t)4 * P.l * P.k);
    P.Rt = small_at(cur, (size_t)4 * P.l * P.k);
  }
  for (int s = 0; s < 3; ++s) { b->gdev[s] = cur; cur += (b->gbytes[s] + 255) / 256 * 256; }
  for (int L = 0; L < b->lanes; ++L) { b->lws.push_back(cur); cur += b->lws_bytes; }
  int rc = cudaMemsetAsync(b->dev, 0, bytes, ctx->stream) == cudaSuccess ? QLR_OK : QLR_ECUDA;

  // lanes: streams, untimed contexts sharing the error word, an even share of the SMs
  b->lctx.resize(b->lanes);
  b->join_ev.resize(b->lanes, nullptr);
  if (rc == QLR_OK && cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess) rc = QLR_ECUDA;
  for (int L = 0; L < b->lanes && rc == QLR_OK; ++L) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { rc = QLR_ECUDA; break; }
    b->ls.push_back(s);
    if (cudaEventCreateWithFlags(&b->join_ev[L], cudaEventDisableTiming) != cudaSuccess) { rc = QLR_ECUDA; break; }
    qlr_ctx& lc = b->lctx[L];
    lc.device = ctx->device;
    lc.stream = s;
    lc.d_err = ctx->d_err;
    lc.num_sms = std::max(4, 2 * ctx->num_sms / b->lanes);
    lc.small_mode = true;
  }
  // QLR_BATCH_VARIANT=0..3 in the environment fixes the grouped sketch variant (no tuning)
  const char* force = std::getenv("QLR_BATCH_VARIANT");
  if (rc == QLR_OK && force && force[0] >= '0' && force[0] <= '3' && force[1] == 0) {
    b->order = force[0] - '0';
    rc = plan_sketches(b, b->order);
  } else if (rc == QLR_OK) {
    rc = tune ? autotune(b) : plan_sketches(b, b->order);
  }
  // one eager run: every lazily configured kernel attribute is set before any capture
  if (rc == QLR_OK) rc = enqueue(b);
  if (rc == QLR_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = QLR_ECUDA;
  if (rc == QLR_OK && use_graph) {
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) rc = QLR_ECUDA;
    if (rc == QLR_OK && cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) rc = QLR_ECUDA;
    if (rc == QLR_OK) {
      b->main_ctx.stream = b->cap_stream;
      const int erc = enqueue(b);
      b->main_ctx.stream = ctx->stream;
      cudaGraph_t gr = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &gr);
      if (erc != QLR_OK) rc = erc;
      else if (ce != cudaSuccess || !gr) rc = QLR_ECUDA;
      b->graph = gr;
    }
    if (rc == QLR_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) rc = QLR_ECUDA;
    if (rc != QLR_OK) cudaGetLastError();
  }
  if (rc != QLR_OK) {
    release(b);
    return rc;
  }
  *out = b;
  return QLR_OK;
}

}  // namespace qlr

extern "C" int qlr_batch_create(qlr_ctx* ctx, int count, const qlr_qmat* A, const int* k, const int* p, int passes,
                                const qlr_qmat* omega, const qlr_opts* opts, qlr_qmat* U, double* const* S, qlr_qmat* V,
                                qlr_batch** out) {
  return qlr::batch_create(ctx, count, A, k, p, passes, omega, opts, U, S, V, true, true, out);
}

extern "C" int qlr_batch_run(qlr_batch* b) {
  if (!b) return QLR_EINVAL;
  DevGuard g(b->ctx->device);
  if (b->exec) {
    QLR_CUDA_TRY(cudaGraphLaunch(b->exec, b->ctx->stream));
    return QLR_OK;
  }
  return enqueue(b);
}

extern "C" int qlr_batch_info(const qlr_batch* b, qlr_batch_stats* st) {
  if (!b || !st) return QLR_EINVAL;
  st->lanes = b->lanes;
  st->graph = b->exec ? 1 : 0;
  st->tile_order = b->order;
  for (int i = 0; i < 4; ++i) st->tune_ms[i] = b->tune_ms[i];
  st->sketch_launches = 2 * b->passes;
  st->launches_per_run = b->launches_per_run;
  return QLR_OK;
}

extern "C" int qlr_batch_destroy(qlr_batch* b) {
  if (!b) return QLR_OK;
  DevGuard g(b->ctx->device);
  release(b);
  return QLR_OK;
}
