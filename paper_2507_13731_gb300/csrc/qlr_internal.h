// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/qlr.h"

// ----------------------------------------------------------------------------------------
// context
struct qlr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int* d_err = nullptr;          // device error word: first QLR_E* code recorded by a kernel
  void* ws = nullptr;            // workspace
  size_t ws_bytes = 0;
  int num_sms = 0;
  // launch statistics
  int64_t launches[QLR_KID_COUNT] = {};
  double ms[QLR_KID_COUNT] = {};
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;                       // free events
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
};

// Brackets the launches of one kernel class: with timing enabled it records events on
// ctx->stream around them; the launches themselves are counted by qlr_count_launch() after each
// one (added to the innermost live KTimer of the calling thread when it closes).
struct KTimer {
  qlr_ctx* ctx;
  int kid;
  int count = 0;
  KTimer* prev = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KTimer(qlr_ctx* c, int k);
  ~KTimer();
};
void qlr_count_launch();

// Bump allocator over the context workspace (256-byte aligned slices).
struct WsArena {
  char* base;
  size_t cap, off = 0;
  bool ok = true;
  WsArena(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (off + bytes > cap) { ok = false; return nullptr; }
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

int qlr_ensure_ws(qlr_ctx* ctx, size_t bytes);

// Failing CUDA calls are reported on stderr when QLR_DEBUG_CUDA is set in the environment.
void qlr_report_cuda(cudaError_t e, const char* expr, const char* file, int line);
#define QLR_CUDA_TRY(expr)                                        \
  do {                                                            \
    cudaError_t e_ = (expr);                                      \
    if (e_ != cudaSuccess) {                                      \
      qlr_report_cuda(e_, #expr, __FILE__, __LINE__);             \
      return QLR_ECUDA;                                           \
    }                                                             \
  } while (0)

#define QLR_TRY(expr)                               \
  do {                                              \
    int r_ = (expr);                                \
    if (r_ != QLR_OK) return r_;                    \
  } while (0)

// ----------------------------------------------------------------------------------------
// device helpers
__device__ __forceinline__ void qlr_set_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

template <class T> __device__ __forceinline__ T qlr_load(const T* p) { return *p; }

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(double x) { return (float)x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <class T> struct Cvt;
template <> struct Cvt<float> {
  template <class S> __device__ __forceinline__ static float from(S x) { return to_f(x); }
};
template <> struct Cvt<double> {
  template <class S> __device__ __forceinline__ static double from(S x) { return to_d(x); }
};
template <> struct Cvt<__nv_bfloat16> {
  template <class S> __device__ __forceinline__ static __nv_bfloat16 from(S x) {
    return __float2bfloat16_rn(to_f(x));
  }
};

// Quaternion stored as 4 reals (real, i, j, k).
template <class T> struct Quat { T w, x, y, z; };

// Hamilton product a*b (Section 2, eq. 1).
template <class T>
__device__ __forceinline__ Quat<T> qmul(const Quat<T>& a, const Quat<T>& b) {
  return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
          a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
          a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
          a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
// conj(a)*b
template <class T>
__device__ __forceinline__ Quat<T> qcmul(const Quat<T>& a, const Quat<T>& b) {
  return {a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z,
          a.w * b.x - a.x * b.w - a.y * b.z + a.z * b.y,
          a.w * b.y + a.x * b.z - a.y * b.w - a.z * b.x,
          a.w * b.z - a.x * b.y + a.y * b.x - a.z * b.w};
}
// a*conj(b)
template <class T>
__device__ __forceinline__ Quat<T> qmulc(const Quat<T>& a, const Quat<T>& b) {
  return {a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z,
          -a.w * b.x + a.x * b.w - a.y * b.z + a.z * b.y,
          -a.w * b.y + a.x * b.z + a.y * b.w - a.z * b.x,
          -a.w * b.z - a.x * b.y + a.y * b.x + a.z * b.w};
}
template <class T> __device__ __forceinline__ T qnorm2(const Quat<T>& a) {
  return a.w * a.w + a.x * a.x + a.y * a.y + a.z * a.z;
}

// ----------------------------------------------------------------------------------------
// Small dense quaternion matrices in FP64 (Gram, R, core QSVD operands): 4 planes of l x l,
// column-major: element (i, j) of plane c at M[c*l*l + j*l + i].
__device__ __forceinline__ Quat<double> ld_small(const double* M, int l, int i, int j) {
  size_t s = (size_t)l * l, o = (size_t)j * l + i;
  return {M[o], M[s + o], M[2 * s + o], M[3 * s + o]};
}
__device__ __forceinline__ void st_small(double* M, int l, int i, int j, const Quat<double>& q) {
  size_t s = (size_t)l * l, o = (size_t)j * l + i;
  M[o] = q.w; M[s + o] = q.x; M[2 * s + o] = q.y; M[3 * s + o] = q.z;
}

// ----------------------------------------------------------------------------------------
// launchers implemented in the .cu files (all asynchronous on ctx->stream)
namespace qlr {

// Internal orthonormalisation modes of cholqr(): one shifted CholeskyQR step, for bases of which
// only the column space is used; one plain CholeskyQR step, for a well-conditioned input (a
// deflated Krylov stack) whose Q must be orthonormal to working precision.
constexpr int ORTH_SPAN = 16;
constexpr int ORTH_ONE = 17;

// SIMT generic quaternion GEMM  C = alpha * op(A) * B + beta * C
//   A element (i, k) at A.plane[c] + i*sa_i + k*sa_k, conj_a applies A -> conj(A) elementwise.
//   B column-major (k, j) at b + k + j*ldb.  C column-major.  Types per dtype fields.
struct GemmArgs {
  const void* a[4]; int64_t sa_i, sa_k; int a_dtype; bool conj_a; bool a_pure;
  const void* b[4]; int64_t ldb; int b_dtype;
  void* c[4]; int64_t ldc; int c_dtype;
  int64_t M, N, K;
  double alpha, beta;
  bool i_contig;      // true when sa_i == 1 (A's row index contiguous in memory)
  bool acc64;         // accumulate in FP64
  bool b_upper = false;      // B upper triangular: column tile j0 reads K rows [0, j0 + BN) only
  int kid = QLR_KID_APPLY;   // statistics class of the launch
};
int gemm_simt(qlr_ctx* ctx, const GemmArgs& g);

// tcgen05 sketch products (see sketch_tc.cu)
int sketch_tc(qlr_ctx* ctx, int op, const qlr_qmat& A, const qlr_qmat& X, qlr_qmat& Y, int compute, WsArena& ws);
size_t sketch_tc_ws(int64_t rows_in, int64_t l, int num_sms);
// Exact scratch bytes sketch_tc takes for this product with a budget of num_sms stream-K CTAs
// (staged thin operand, stream-K partial tiles, arrival counters; 256-byte aligned slices).
size_t sketch_tc_need(int op, int64_t M, int64_t K, int l, int compute, int num_sms);
bool sketch_tc_supported(int op, const qlr_qmat& A, const qlr_qmat& X, int compute);

// Grouped tensor-core sketch over many problems (one launch for the staging of every X and one
// for every output tile).  The plan lives in caller-provided device memory (`dev`, sized by
// sketch_tc_grouped_bytes) and is reused by every run.  `variant` bit 0: schedule the tiles with
// the longest reduction first (else in problem order); bit 1: one persistent CTA per SM walking
// the tile list (else one CTA per tile); bit 2 (persistent, K-major A, BF16 / TF32): 128-byte
// stage rows (else 64); bit 3: column blocks of at most 64 (else 128).
struct GroupedSketch {
  int kind = 0, amode = 0, count = 0, nitems = 0, stage_grid_x = 0;
  int persistent = 0, grid = 0, nb_max = 0, stages = 0, apl = 4, wide = 0, stage_k = 0, fd = 0;
  uint32_t tmem_cols = 0;
  size_t smem = 0;
  void* d_probs = nullptr;
  int4* d_items = nullptr;
  void* d_stage = nullptr;
};
size_t sketch_tc_grouped_bytes(int op, int count, const qlr_qmat* A, const qlr_qmat* X, int compute);
int sketch_tc_grouped_plan(qlr_ctx* ctx, int op, int count, const qlr_qmat* A, const qlr_qmat* X, const qlr_qmat* Y,
                           int compute, int variant, char* dev, size_t bytes, GroupedSketch& gs);
int sketch_tc_grouped_run(qlr_ctx* ctx, const GroupedSketch& gs);

// orthonormalisation pieces (orth.cu)
int gram(qlr_ctx* ctx, const qlr_qmat& Y, double* G, WsArena& ws);
// FP64-class Gram of FP32 Y on the tensor cores by exact BF16 slicing (gram_tc.cu); G FP64 planes.
size_t gram_tc_ws(int64_t m, int l);
bool gram_tc_supported(const qlr_qmat& Y);
int gram_tc(qlr_ctx* ctx, const qlr_qmat& Y, double* G, WsArena& ws);
// Batch plans (grouped launches): a per-problem record of gram_tc_record_bytes() bytes (64-byte
// aligned in the device table) holds the tensor maps over the problem's scratch (gram_tc_ws(m, l)
// bytes) and writes G as a double-FP32 upper triangle (8 floats per entry at G + 8 (j l + i)).
size_t gram_tc_record_bytes();
int gram_tc_record(void* dst, const qlr_qmat& Y, char* scratch, float* G, int* err);
void gram_tc_grouped_items(int64_t m, int l, int prob, std::vector<int4>& slice, std::vector<int4>& mma,
                           std::vector<int4>& comb);
int gram_tc_grouped(qlr_ctx* ctx, const void* d_probs, const int4* slice, int n_slice, const int4* mma, int n_mma,
                    const int4* comb, int n_comb);
int chol(qlr_ctx* ctx, int l, const double* G, double* R, double shift_rel, WsArena& ws, double* Dinv_all = nullptr,
         const int* run_if = nullptr, bool df = false);
// d32buf (2 (4 l^2 + ceil(l/16) 4 16^2) floats, or null): run the double-FP32 form of the blocked
// inverse (factors of FP32 sketches' Grams); null runs it in FP64.
int tri_inv(qlr_ctx* ctx, int l, const double* R, double* Rinv, const double* Dinv_all = nullptr,
            const int* run_if = nullptr, float* d32buf = nullptr);
int small_matmul(qlr_ctx* ctx, int l, const double* A, const double* B, double* C);  // C = A B (upper-tri A, B)
int cholqr(qlr_ctx* ctx, const qlr_qmat& Y, qlr_qmat& Q, double* R, int orth, WsArena& ws);

// Masked update of matrix completion (complete.cu, Section 7 eq. Step2):
// C = mask .* M + (1 - mask) .* U diag(S) V^H, entries in the dtype of C (F32 or F64).
struct CompleteArgs {
  const void* M[4];      // row-major m x n; M[0] null for a pure M
  int64_t ldm;
  const uint8_t* mask;   // row-major m x n, non-zero = observed
  int64_t ldk;
  const void* U[4];      // column-major m x k
  int64_t ldu;
  const double* S;       // k values
  const void* V[4];      // column-major n x k
  int64_t ldv;
  void* C[4];            // row-major m x n (may alias M)
  int64_t ldc;
  int64_t m, n;
  int k;
};
int complete_update(qlr_ctx* ctx, const CompleteArgs& a, int dtype);
// Failure-detection self test (selftest.cu): a bounded mbarrier wait that times out.
int selftest_wait_timeout(qlr_ctx* ctx);

// Grouped steps of batch plans: one launch runs one step for every problem of a plan, the
// per-problem arguments and the (problem, tile) items of each launch in device tables built once
// by the plan.  The small operands are FP32 / double-FP32 (no FP64 instruction on this path).
constexpr int kBatchMaxL = 80;   // largest l = k + p of a batch plan (one CTA holds its factors)
//  Gram: gram_tc_grouped (below, with the single-problem tensor-core Gram), FP64-class; and, for
//  the last step of CholeskyQR2 / shifted CholeskyQR3 (a nearly orthonormal input), the FP32 Gram
//  gram_f32_grouped (gram_f32.cu): Y FP32 column-major planes, G in the same double-FP32 upper
//  layout, items (problem, tile I, tile J >= I) of 16 x 16 entries.
struct GramF32Args { const float* y[4]; int64_t ld, m; int l; float* G; };
void gram_f32_items(int l, int prob, std::vector<int4>& items);
int gram_f32_grouped(qlr_ctx* ctx, const GramF32Args* d_args, const int4* d_items, int nitems);
//  Cholesky (orth.cu), one CTA per problem: R = chol(G + shift_coef trace(G) I) in double-FP32;
//  Rinv = R^{-1} and Rout = R Rprev (R when Rprev is null) as FP32 l x l planes (column-major,
//  zero below the diagonal); either output may be null.
struct CholGroupArgs { const float* G; const float* Rprev; float* Rout; float* Rinv; int l; float shift_coef; };
size_t chol_df_grouped_smem(int lmax);
int chol_df_grouped(qlr_ctx* ctx, const CholGroupArgs* d_args, int count, int lmax);
//  The same in plain FP32 (G's high parts only), for the steps whose Gram is formed in FP32.
int chol_f32_grouped(qlr_ctx* ctx, const CholGroupArgs* d_args, int count, int lmax);
//  Thin x small products (thin.cu): FP32 GemmArgs (A column-major, sa_i == 1, 4 planes; B FP32
//  column-major; no conj, alpha 1, beta 0), items (problem, row block, column chunk).
void thin_small_items(int64_t M, int64_t N, int prob, std::vector<int4>& items);
int thin_small_grouped(qlr_ctx* ctx, const GemmArgs* d_args, const int4* d_items, int nitems);
//  Core QSVD (core_svd.cu), one CTA per problem: one-sided Jacobi on R (FP32 l x l planes) with
//  W and V in shared memory; the k largest sigma in descending order into S, the matching left
//  vectors into U and right vectors into V (FP32 l x k planes, column-major), multiplied on the
//  left by the upper-triangular Lleft / Lright (FP32 l x l planes) when those are set.
struct JacobiGroupArgs { const float* R; float* U; float* V; double* S; int l, k; const float* Lleft; const float* Lright; };
size_t jacobi_grouped_smem(int lmax);
int jacobi_grouped(qlr_ctx* ctx, const JacobiGroupArgs* d_args, int count, int lmax);

// core QSVD (core_svd.cu)
int core_tsvd(qlr_ctx* ctx, int l, const double* R, int k, double* L, double* S, double* Rt, int prec,
              WsArena& ws);
size_t core_tsvd_ws(int l);

// workspace bounds (abi.cu)
size_t gram_ws_bound(int64_t rows, int64_t l);
size_t cholqr_ws_bound(int64_t rows, int64_t l, size_t esz);
size_t tsvd_ws_bound(int64_t l);

// batch plans (batch.cu): tune = run the tile-order autotuner, use_graph = capture a CUDA graph
int batch_create(qlr_ctx* ctx, int count, const qlr_qmat* A, const int* k, const int* p, int passes,
                 const qlr_qmat* omega, const qlr_opts* opts, qlr_qmat* U, double* const* S, qlr_qmat* V,
                 bool tune, bool use_graph, qlr_batch** out);

// utilities (util.cu)
int convert_qmat(qlr_ctx* ctx, const qlr_qmat& src, qlr_qmat& dst);  // elementwise dtype change
// C (rows x k) = T (rows x l, column-major) * S (FP64 l x k, column-major planes) (thin.cu)
// S_upper: S is upper triangular (R^{-1}), so the product skips its zero rows.
int thin_times_small(qlr_ctx* ctx, const qlr_qmat& T, const double* S, int l, int k, qlr_qmat& C, WsArena& ws,
                     bool S_upper = false);
int zero_qmat(qlr_ctx* ctx, qlr_qmat& dst);
int small_to_qmat(qlr_ctx* ctx, const double* S, int l, int k, qlr_qmat& dst);  // l x k FP64 small -> qmat

}  // namespace qlr

size_t qlr_dtype_size(int dtype);
