// Batched Algorithm 2 over many independent problems (image patches / frames of uneven sizes).
//
// One plan per problem set, and one launch per step for all the problems: every sketch pass is
// a grouped tensor-core launch over all the problems' output tiles (sketch_tc.cu), preceded by
// one grouped staging launch of their thin operands; every orthonormalisation step is a grouped
// tensor-core Gram (slicing, MMA and combine launches, gram_tc.cu), a grouped double-FP32
// Cholesky launch (one CTA per problem, which also forms R^{-1} and the running product of the R
// factors) and a grouped thin x small product; after the last pass one grouped Jacobi launch
// computes every core QSVD and one grouped product lifts all U and V.  A run is a few dozen
// launches, whatever the problem count, and each launch spreads the problems' CTAs over the whole
// GPU.  The sequence is captured once into a CUDA graph and replayed by every run.  At plan time a
// small autotuner times the grouped sketch's tile orders and keeps the faster one.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "qlr_internal.h"

namespace {

constexpr int kBatchVariants = 16;   // grouped sketch variants (see autotune)

// One orthonormalisation step of one pass (device tables, one entry per problem).
struct StepTables {
  const void* gram = nullptr;               // tensor-core Gram records (FP64-class steps)
  const qlr::GramF32Args* gram32 = nullptr; // FP32 Gram arguments (last step of a QR)
  const qlr::CholGroupArgs* chol = nullptr;
  const qlr::GemmArgs* apply = nullptr;
};

}  // namespace

struct qlr_batch {
  struct Prob {
    qlr_qmat A, om, U, V, Y, Z, Q1, Q2, T;
    double* S;
    char* gsc;        // tensor-core Gram scratch (slices, exponents, chunk partials)
    float* G;         // Gram, double-FP32 upper triangle
    float* Rinv;      // R^{-1} of the current step (FP32)
    float* Rp[2];     // running products of the last pass's R factors (FP32)
    float* Sinv[2];   // inverse last factors of passes v - 1 ([0]) and v ([1]), carried (see layout)
    float* Uh;        // core QSVD: left vectors (l x k)
    float* Vh;        // core QSVD: right vectors (l x k)
    int k, p, l;
  };
  qlr_ctx* ctx = nullptr;
  qlr_ctx main_ctx;                         // issues the launches (timed only in eager runs): on ctx->stream, or
                                            // on cap_stream while the graph is captured
  cudaStream_t cap_stream = nullptr;        // capture needs a stream other than the legacy default
  int count = 0, passes = 0, compute = 0, orth = 0, mid = 0, lmax = 0;
  std::vector<Prob> pr;
  qlr::GroupedSketch gs[3];                 // (N, Omega -> Y), (H, Q1 -> Z), (N, Q2 -> Y)
  char* gdev[3] = {nullptr, nullptr, nullptr};
  size_t gbytes[3] = {0, 0, 0};
  std::vector<std::vector<StepTables>> steps;   // [pass - 1][step]
  const int4* slice_items[2] = {nullptr, nullptr};  // [0]: rows m (odd passes), [1]: rows n
  const int4* gram_items[2] = {nullptr, nullptr};
  const int4* comb_items[2] = {nullptr, nullptr};
  const int4* apply_items[2] = {nullptr, nullptr};
  int n_slice[2] = {0, 0}, n_gram[2] = {0, 0}, n_comb[2] = {0, 0}, n_apply[2] = {0, 0};
  const int4* gf_items = nullptr;           // FP32 Gram tiles (independent of the row count)
  int n_gf = 0;
  const qlr::JacobiGroupArgs* jac = nullptr;
  const qlr::GemmArgs* lift = nullptr;
  const int4* lift_items = nullptr;
  int n_lift = 0;
  void* dev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int order = 1;                            // chosen grouped-sketch variant (bit 0 order, bit 1 persistent,
                                            // bit 2 128-byte stage rows, bit 3 column blocks <= 64)
  float tune_ms[kBatchVariants] = {};
  int64_t launches_per_run = 0;
};

namespace {

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

size_t rup(size_t b) { return (b + 255) / 256 * 256; }

// Column-major FP32 thin matrix with a 16-byte multiple column pitch (TMA reads it as the next
// pass's sketch operand).
qlr_qmat thin_at(char*& cur, int64_t rows, int64_t cols) {
  qlr_qmat q{};
  q.rows = rows; q.cols = cols; q.ld = (rows + 3) / 4 * 4; q.layout = QLR_COL_MAJOR; q.dtype = QLR_F32;
  const size_t plane = (size_t)q.ld * cols * 4;
  for (int c = 0; c < 4; ++c) q.plane[c] = cur + (size_t)c * plane;
  cur += rup(4 * plane);
  return q;
}

template <class T>
T* take(char*& cur, size_t count) {
  T* p = reinterpret_cast<T*>(cur);
  cur += rup(count * sizeof(T));
  return p;
}

qlr::GemmArgs thin_small_args(const qlr_qmat& T, const float* S, int l, int k, const qlr_qmat& C) {
  qlr::GemmArgs g{};
  for (int c = 0; c < 4; ++c) {
    g.a[c] = T.plane[c];
    g.b[c] = S + (size_t)c * l * k;
    g.c[c] = C.plane[c];
  }
  g.sa_i = 1; g.sa_k = T.ld; g.a_dtype = QLR_F32; g.conj_a = false; g.a_pure = false; g.i_contig = true;
  g.ldb = l; g.b_dtype = QLR_F32;
  g.ldc = C.ld; g.c_dtype = QLR_F32;
  g.M = T.rows; g.N = k; g.K = l;
  g.alpha = 1.0; g.beta = 0.0;
  g.acc64 = false;
  return g;
}

int orth_steps(int orth) { return orth == QLR_ORTH_SCHOLQR3 ? 3 : (orth == qlr::ORTH_SPAN ? 1 : 2); }

// The last step of CholeskyQR2 (and of shifted CholeskyQR3) factors the Gram of a basis whose
// previous, unshifted step left it nearly orthonormal: its Gram is formed in FP32.  Every other
// step (a sketch's first step, the step after a shifted one) keeps the FP64-class Gram.
bool fp32_gram_step(int orth, int s) {
  return (orth == QLR_ORTH_CHOLQR2 && s == 1) || (orth == QLR_ORTH_SCHOLQR3 && s == 2);
}

const qlr::GroupedSketch& plan_of(const qlr_batch* b, int pass) {
  return pass == 1 ? b->gs[0] : (pass % 2 == 0 ? b->gs[1] : b->gs[2]);
}

// The whole batched QSVD, enqueued on main_ctx.stream.
int enqueue(qlr_batch* b) {
  const int v = b->passes;
  qlr_ctx* mc = &b->main_ctx;
  std::fill(std::begin(mc->launches), std::end(mc->launches), 0);
  for (int i = 1; i <= v; ++i) {
    QLR_TRY(qlr::sketch_tc_grouped_run(mc, plan_of(b, i)));
    const int par = (i % 2 == 1) ? 0 : 1;
    for (const StepTables& st : b->steps[i - 1]) {
      if (st.gram32)
        QLR_TRY(qlr::gram_f32_grouped(mc, st.gram32, b->gf_items, b->n_gf));
      else
        QLR_TRY(qlr::gram_tc_grouped(mc, st.gram, b->slice_items[par], b->n_slice[par], b->gram_items[par],
                                     b->n_gram[par], b->comb_items[par], b->n_comb[par]));
      if (st.gram32) QLR_TRY(qlr::chol_f32_grouped(mc, st.chol, b->count, b->lmax));
      else QLR_TRY(qlr::chol_df_grouped(mc, st.chol, b->count, b->lmax));
      if (st.apply) QLR_TRY(qlr::thin_small_grouped(mc, st.apply, b->apply_items[par], b->n_apply[par]));
    }
  }
  QLR_TRY(qlr::jacobi_grouped(mc, b->jac, b->count, b->lmax));
  QLR_TRY(qlr::thin_small_grouped(mc, b->lift, b->lift_items, b->n_lift));
  int64_t n = 0;
  for (int kk = 0; kk < QLR_KID_COUNT; ++kk) n += mc->launches[kk];
  b->launches_per_run = n;
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

// Whether the autotuner times variant v: the tile shapes (bits 2, 3) only apply to the persistent
// schedule, and 128-byte stage rows not to 3xTF32 (its stages are 32-byte rows).
bool tuned_variant(int v, int compute) {
  if (!((v >> 1) & 1) && (v & 12)) return false;
  if (compute == QLR_COMPUTE_TF32X3 && ((v >> 2) & 1)) return false;
  return true;
}

// Autotuner: time the grouped sketch variants -- tile order (problem order / longest reduction
// first) x schedule (one CTA per tile / one persistent CTA per SM) x, for the persistent schedule,
// tile shape (K elements per stage: 64-byte or 128-byte rows; column blocks of at most 128 or 64)
// -- on passes N and H, best of three after a warm-up, and keep the fastest.
int autotune(qlr_batch* b) {
  cudaEvent_t e0, e1;
  QLR_CUDA_TRY(cudaEventCreate(&e0));
  QLR_CUDA_TRY(cudaEventCreate(&e1));
  int rc = QLR_OK;
  for (int order = 0; order < kBatchVariants && rc == QLR_OK; ++order) {
    if (!tuned_variant(order, b->compute)) continue;
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
  int best = -1;
  for (int v = 0; v < kBatchVariants; ++v)
    if (tuned_variant(v, b->compute) && (best < 0 || b->tune_ms[v] < b->tune_ms[best])) best = v;
  b->order = best;
  return plan_sketches(b, b->order);
}

void release(qlr_batch* b) {
  if (!b) return;
  if (b->ctx) cudaStreamSynchronize(b->ctx->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->dev) cudaFree(b->dev);
  delete b;
}

// Host images of the device tables, appended to one byte buffer (256-byte aligned entries).
struct TableBuf {
  std::vector<char> host;
  std::vector<size_t> offs;
  void add_raw(const std::vector<char>& v) { add(v); }
  template <class T>
  void add(const std::vector<T>& v) {
    const size_t off = rup(host.size());
    host.resize(off + rup(v.size() * sizeof(T) + 1));
    if (!v.empty()) std::memcpy(host.data() + off, v.data(), v.size() * sizeof(T));
    offs.push_back(off);
  }
};

// Lays out every problem's buffers from `base` (returns the bytes used) and records the host
// images of the step tables in tb, in the order batch_create reads them back; *rc receives the
// first failure to encode a tensor map (the dry run from a dummy base ignores it).
size_t layout(qlr_batch* b, const qlr_qmat* A, const int* k, const int* p, const qlr_qmat* omega, qlr_qmat* U,
              double* const* S, qlr_qmat* V, char* base, TableBuf& tb, int* rc) {
  using namespace qlr;
  const int count = b->count, passes = b->passes;
  char* cur = base;
  for (int j = 0; j < count; ++j) {
    qlr_batch::Prob& P = b->pr[j];
    P.A = A[j]; P.om = omega[j]; P.U = U[j]; P.V = V[j]; P.S = S[j];
    P.k = k[j]; P.p = p[j]; P.l = k[j] + p[j];
    const int64_t m = A[j].rows, n = A[j].cols;
    P.Y = thin_at(cur, m, P.l);
    P.Q1 = thin_at(cur, m, P.l);
    P.Z = thin_at(cur, n, P.l);
    P.Q2 = thin_at(cur, n, P.l);
    P.T = thin_at(cur, std::max(m, n), P.l);
    P.gsc = take<char>(cur, gram_tc_ws(std::max(m, n), P.l));
    P.G = take<float>(cur, (size_t)8 * P.l * P.l);
    P.Rinv = take<float>(cur, (size_t)4 * P.l * P.l);
    P.Rp[0] = take<float>(cur, (size_t)4 * P.l * P.l);
    P.Rp[1] = take<float>(cur, (size_t)4 * P.l * P.l);
    P.Sinv[0] = take<float>(cur, (size_t)4 * P.l * P.l);
    P.Sinv[1] = take<float>(cur, (size_t)4 * P.l * P.l);
    P.Uh = take<float>(cur, (size_t)4 * P.l * P.k);
    P.Vh = take<float>(cur, (size_t)4 * P.l * P.k);
  }
  // items: Gram tiles, combine blocks and product tiles for row count m (odd passes) or n, the
  // problems with the most rows first (their CTAs run longest)
  for (int par = 0; par < 2; ++par) {
    std::vector<int4> si, gi, ci, ai;
    std::vector<int> heavy(count);
    for (int j = 0; j < count; ++j) heavy[j] = j;
    auto rows_of = [&](int j) { return par == 0 ? b->pr[j].A.rows : b->pr[j].A.cols; };
    std::stable_sort(heavy.begin(), heavy.end(), [&](int x, int y) { return rows_of(x) > rows_of(y); });
    for (int j : heavy) {
      const qlr_batch::Prob& P = b->pr[j];
      const int64_t rows = par == 0 ? P.A.rows : P.A.cols;
      gram_tc_grouped_items(rows, P.l, j, si, gi, ci);
      thin_small_items(rows, P.l, j, ai);
    }
    b->n_slice[par] = (int)si.size();
    b->n_gram[par] = (int)gi.size();
    b->n_comb[par] = (int)ci.size();
    b->n_apply[par] = (int)ai.size();
    tb.add(si);
    tb.add(gi);
    tb.add(ci);
    tb.add(ai);
  }
  {
    std::vector<int4> gf;
    for (int j = 0; j < count; ++j) gram_f32_items(b->pr[j].l, j, gf);
    b->n_gf = (int)gf.size();
    tb.add(gf);
  }
  const size_t rec = gram_tc_record_bytes();
  // steps of every pass: Y (odd) or Z (even) -> Q1 or Q2, through T.
  // The last two passes carry their last CholeskyQR factor S instead of applying it: their basis
  // buffer keeps B = Q S (the previous step's output) and S^{-1} is kept in Sinv.  The last pass
  // then sketches with B_{v-1} = Q_{v-1} S_{v-1}, so its own factorisation B_v R' of that sketch
  // gives the core factor R = R' S_{v-1}^{-1} (the chain's first Rprev), and the lifts take
  // Q_v U_hat = B_v (S_v^{-1} U_hat), Q_{v-1} V_hat = B_{v-1} (S_{v-1}^{-1} V_hat) (the factors
  // applied to the core's vectors in the Jacobi launch).  The same factorisations in exact
  // arithmetic, without two thin x small products per run.
  for (int i = 1; i <= passes; ++i) {
    const int o = (i >= passes - 1) ? b->orth : b->mid;
    const int ns = orth_steps(o);
    const bool carry = (i >= passes - 1);
    for (int s = 0; s < ns; ++s) {
      const bool no_apply = carry && (s == ns - 1);
      const bool g32 = fp32_gram_step(o, s);
      std::vector<char> ga(g32 ? 0 : (size_t)count * rec);
      std::vector<GramF32Args> gfa(g32 ? count : 0);
      std::vector<CholGroupArgs> ca(count);
      std::vector<GemmArgs> aa(count);
      for (int j = 0; j < count; ++j) {
        qlr_batch::Prob& P = b->pr[j];
        const qlr_qmat& src = (i % 2 == 1) ? P.Y : P.Z;
        const qlr_qmat& dst = (i % 2 == 1) ? P.Q1 : P.Q2;
        qlr_qmat T = P.T;
        T.rows = dst.rows;
        T.ld = dst.ld;
        // 1 step: src -> dst; 2: src -> T -> dst; 3: src -> dst -> T -> dst; carried (the last
        // step factors only): 2: src -> dst, 3: src -> T -> dst
        const qlr_qmat* seq[4] = {&src, &dst, nullptr, nullptr};
        if (carry) {
          if (ns == 3) { seq[1] = &T; seq[2] = &dst; }
        } else {
          if (ns == 2) { seq[1] = &T; seq[2] = &dst; }
          if (ns == 3) { seq[2] = &T; seq[3] = &dst; }
        }
        const qlr_qmat& from = *seq[s];
        if (g32) {
          GramF32Args& G = gfa[j];
          for (int c = 0; c < 4; ++c) G.y[c] = static_cast<const float*>(from.plane[c]);
          G.ld = from.ld;
          G.m = from.rows;
          G.l = P.l;
          G.G = P.G;
        } else {
          const int grc = gram_tc_record(ga.data() + (size_t)j * rec, from, P.gsc, P.G, b->ctx->d_err);
          if (grc != QLR_OK && *rc == QLR_OK) *rc = grc;
        }
        CholGroupArgs& C = ca[j];
        C.G = P.G;
        C.Rinv = no_apply ? P.Sinv[i == passes ? 1 : 0] : P.Rinv;
        C.l = P.l;
        // shifted first step (span steps, shifted CholeskyQR3): s = 11 (m l + l (l + 1)) u trace(G),
        // u = 2^-48 for the double-FP32 Gram and Cholesky
        const bool shifted = (s == 0) && (o == QLR_ORTH_SCHOLQR3 || o == ORTH_SPAN);
        C.shift_coef = shifted ? (float)(11.0 * ((double)from.rows * P.l + (double)P.l * (P.l + 1)) * 3.552713678800501e-15)
                               : 0.f;
        // the last pass keeps R = R_s ... R_0 S_{v-1}^{-1} for the core QSVD
        C.Rout = (i == passes) ? P.Rp[s % 2] : nullptr;
        C.Rprev = (i == passes) ? (s > 0 ? P.Rp[(s - 1) % 2] : P.Sinv[0]) : nullptr;
        if (!no_apply) {
          aa[j] = thin_small_args(from, P.Rinv, P.l, P.l, *seq[s + 1]);
          aa[j].b_upper = true;   // R^{-1} is upper triangular
        }
      }
      if (no_apply) aa.clear();
      if (g32) tb.add(gfa);
      else tb.add_raw(ga);
      tb.add(ca);
      tb.add(aa);
    }
  }
  // core QSVDs and lifts U = Q1 U_hat, V = Q2 V_hat; even v: [V_hat, S, U_hat] = TSVD(R2),
  // odd v: [U_hat, S, V_hat] = TSVD(R1)
  const int nlast = orth_steps(b->orth);
  std::vector<JacobiGroupArgs> ja(count);
  std::vector<GemmArgs> la(2 * count);
  std::vector<int4> li;
  for (int j = 0; j < count; ++j) {
    qlr_batch::Prob& P = b->pr[j];
    ja[j] = {P.Rp[(nlast - 1) % 2], P.Uh, P.Vh, P.S, P.l, P.k, P.Sinv[1], P.Sinv[0]};
    const float* Uhat = (passes % 2 == 0) ? P.Vh : P.Uh;
    const float* Vhat = (passes % 2 == 0) ? P.Uh : P.Vh;
    la[j] = thin_small_args(P.Q1, Uhat, P.l, P.k, P.U);
    la[count + j] = thin_small_args(P.Q2, Vhat, P.l, P.k, P.V);
    thin_small_items(P.A.rows, P.k, j, li);
  }
  for (int j = 0; j < count; ++j) thin_small_items(b->pr[j].A.cols, b->pr[j].k, count + j, li);
  b->n_lift = (int)li.size();
  // the largest cores first: CTAs are dispatched in order as SMs free up (longest job first)
  std::stable_sort(ja.begin(), ja.end(), [](const JacobiGroupArgs& x, const JacobiGroupArgs& y) { return x.l > y.l; });
  tb.add(ja);
  tb.add(la);
  tb.add(li);
  return (size_t)(cur - base);
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
  int lmax = 0;
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
    if (l > kBatchMaxL) return QLR_EUNSUPPORTED;
    if (!qlr::sketch_tc_supported(QLR_OP_N, A[j], omega[j], compute)) return QLR_EUNSUPPORTED;
    lmax = std::max(lmax, l);
  }
  DevGuard g(ctx->device);
  qlr_batch* b = new qlr_batch();
  b->ctx = ctx;
  b->count = count;
  b->passes = passes;
  b->compute = compute;
  b->orth = orth;
  b->mid = (opts && (opts->flags & QLR_FLAG_QR_EVERY_PASS)) ? orth : ORTH_SPAN;
  b->lmax = lmax;
  b->main_ctx.device = ctx->device;
  b->main_ctx.stream = ctx->stream;
  b->main_ctx.d_err = ctx->d_err;
  b->main_ctx.num_sms = ctx->num_sms;
  b->pr.resize(count);

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
  // a dry layout from a dummy base gives the sizes of the buffers and of the tables
  size_t bytes = 0, tbytes = 0;
  {
    TableBuf dry;
    char* dummy = reinterpret_cast<char*>((uintptr_t)256);
    int dry_rc = QLR_OK;
    bytes = rup(layout(b, A, k, p, omega, U, S, V, dummy, dry, &dry_rc));
    tbytes = rup(dry.host.size());
  }
  const size_t total = bytes + rup(b->gbytes[0]) + rup(b->gbytes[1]) + rup(b->gbytes[2]) + tbytes;
  if (cudaMalloc(&b->dev, total) != cudaSuccess) {
    cudaGetLastError();
    release(b);
    return QLR_ENOMEM;
  }
  char* base = static_cast<char*>(b->dev);
  TableBuf tb;
  int rc = QLR_OK;
  layout(b, A, k, p, omega, U, S, V, base, tb, &rc);
  char* cur = base + bytes;
  for (int s = 0; s < 3; ++s) { b->gdev[s] = cur; cur += rup(b->gbytes[s]); }
  char* tdev = cur;
  if (rc == QLR_OK && cudaMemsetAsync(b->dev, 0, bytes, ctx->stream) != cudaSuccess) rc = QLR_ECUDA;
  if (rc == QLR_OK && cudaMemcpyAsync(tdev, tb.host.data(), tb.host.size(), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    rc = QLR_ECUDA;
  if (rc == QLR_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = QLR_ECUDA;   // tb is pageable
  if (rc == QLR_OK) {
    size_t q = 0;
    auto next = [&]() { return tdev + tb.offs[q++]; };
    for (int par = 0; par < 2; ++par) {
      b->slice_items[par] = reinterpret_cast<const int4*>(next());
      b->gram_items[par] = reinterpret_cast<const int4*>(next());
      b->comb_items[par] = reinterpret_cast<const int4*>(next());
      b->apply_items[par] = reinterpret_cast<const int4*>(next());
    }
    b->gf_items = reinterpret_cast<const int4*>(next());
    b->steps.resize(passes);
    for (int i = 1; i <= passes; ++i) {
      const int ns = orth_steps((i >= passes - 1) ? b->orth : b->mid);
      const int o = (i >= passes - 1) ? b->orth : b->mid;
      for (int s = 0; s < ns; ++s) {
        StepTables st;
        if (fp32_gram_step(o, s)) st.gram32 = reinterpret_cast<const GramF32Args*>(next());
        else st.gram = next();
        st.chol = reinterpret_cast<const CholGroupArgs*>(next());
        st.apply = reinterpret_cast<const GemmArgs*>(next());
        if (i >= passes - 1 && s == ns - 1) st.apply = nullptr;   // carried factor (see layout)
        b->steps[i - 1].push_back(st);
      }
    }
    b->jac = reinterpret_cast<const JacobiGroupArgs*>(next());
    b->lift = reinterpret_cast<const GemmArgs*>(next());
    b->lift_items = reinterpret_cast<const int4*>(next());
  }
  // QLR_BATCH_VARIANT=0..15 in the environment fixes the grouped sketch variant (no tuning)
  const char* force = std::getenv("QLR_BATCH_VARIANT");
  char* fend = nullptr;
  const long fv = force ? std::strtol(force, &fend, 10) : -1;
  if (rc == QLR_OK && force && fend != force && *fend == 0 && fv >= 0 && fv < kBatchVariants) {
    b->order = (int)fv;
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
  // eager run: with timing enabled on the caller's context, every kernel class of the run is
  // bracketed by events and counted there (a graph replay is one launch and is not broken down)
  qlr_ctx* c = b->ctx;
  b->main_ctx.timing = c->timing;
  const int rc = enqueue(b);
  b->main_ctx.timing = false;
  for (auto& pe : b->main_ctx.ev_pending) c->ev_pending.push_back(pe);
  b->main_ctx.ev_pending.clear();
  if (c->timing)
    for (int kk = 0; kk < QLR_KID_COUNT; ++kk) c->launches[kk] += b->main_ctx.launches[kk];
  return rc;
}

extern "C" int qlr_batch_info(const qlr_batch* b, qlr_batch_stats* st) {
  if (!b || !st) return QLR_EINVAL;
  st->lanes = 1;
  st->graph = b->exec ? 1 : 0;
  st->tile_order = b->order;
  for (int i = 0; i < kBatchVariants; ++i) st->tune_ms[i] = b->tune_ms[i];
  const qlr::GroupedSketch& g = b->gs[0];   // the first pass's plan (op N)
  st->stage_k = g.stage_k;
  st->col_block_max = g.nb_max;
  st->ring_stages = g.stages;
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
