// Allocation-free variant of the tensor-core sketch product.
//
// Who needs it: callers that must not call cudaMalloc (or create a qlr context, which does).
// cudaMalloc can synchronise the device and takes a driver-wide lock, so latency-critical serving
// loops keep it out of their steady state; some host applications hand all device memory to their
// own pool allocator and forbid any other allocation.  This entry point gives them the sketch
// product Y = A X / Y = A^H X of qlr_qsketch with every scratch byte taken from one fixed
// file-scope device array that the CUDA module carries, so the call itself allocates nothing.
//
// The scratch array is shared by every call on a device and keeps the last call's contents; the
// parts that must start at zero (the stream-K arrival counters) are cleared on the stream by each
// call.  Calls that overlap on the GPU (different streams, or another thread's call in flight)
// race on the array.
#include <mutex>

#include "qlr_internal.h"

#define QLR_NOALLOC_SCRATCH_BYTES (128u << 20)
#define QLR_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_qlr_noalloc_scratch[QLR_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_mu;
void* g_scratch_addr[QLR_NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once per device with that
// device current (the name g_qlr_noalloc_scratch is only a host-side handle and must never be
// passed to a kernel).  The cached address belongs to the device's primary context: after a
// cudaDeviceReset of that device it is stale, so a process that resets a device must not call
// this entry point on it again.
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= QLR_NOALLOC_MAX_DEVICES) return QLR_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_qlr_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return QLR_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return QLR_OK;
}

// Makes `dev` current for the call and restores the caller's device on exit.
struct DeviceScope {
  int prev = -1;
  bool ok = true;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) { cudaGetLastError(); ok = false; prev = -1; }
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int check_qmat_na(const qlr_qmat* q, int layout, bool allow_pure) {
  if (!q) return QLR_EINVAL;
  if (q->layout != layout || !(q->dtype == QLR_F64 || q->dtype == QLR_F32 || q->dtype == QLR_BF16)) return QLR_EINVAL;
  if (q->rows < 0 || q->cols < 0) return QLR_ESHAPE;
  const int64_t inner = (layout == QLR_ROW_MAJOR) ? q->cols : q->rows;
  if (q->ld < (inner > 1 ? inner : 1)) return QLR_ESHAPE;
  for (int c = 0; c < 4; ++c)
    if (q->plane[c] == nullptr && !(c == 0 && allow_pure) && q->rows > 0 && q->cols > 0) return QLR_EINVAL;
  return QLR_OK;
}
}  // namespace

extern "C" int qlr_qsketch_noalloc(void* stream, int op, const qlr_qmat* A, const qlr_qmat* X, qlr_qmat* Y,
                                   int compute, int* err) {
  if (check_qmat_na(A, QLR_ROW_MAJOR, true) != QLR_OK || check_qmat_na(X, QLR_COL_MAJOR, false) != QLR_OK ||
      check_qmat_na(Y, QLR_COL_MAJOR, false) != QLR_OK)
    return QLR_EINVAL;
  if (op != QLR_OP_N && op != QLR_OP_H) return QLR_EINVAL;
  if (compute != QLR_COMPUTE_TF32 && compute != QLR_COMPUTE_TF32X3 && compute != QLR_COMPUTE_BF16) return QLR_EINVAL;
  const int64_t inner = (op == QLR_OP_N) ? A->cols : A->rows, outer = (op == QLR_OP_N) ? A->rows : A->cols;
  if (X->rows != inner || Y->rows != outer || Y->cols != X->cols) return QLR_ESHAPE;
  if (Y->dtype != QLR_F32 || !(X->dtype == QLR_F32 || (compute == QLR_COMPUTE_BF16 && X->dtype == QLR_BF16)))
    return QLR_EINVAL;
  if ((compute == QLR_COMPUTE_BF16) != (A->dtype == QLR_BF16) || A->dtype == QLR_F64) return QLR_EINVAL;

  // The stream's device runs the call (the legacy default stream means the current device).
  int dev = 0;
  if (cudaStreamGetDevice(static_cast<cudaStream_t>(stream), &dev) != cudaSuccess) {
    cudaGetLastError();
    return QLR_ECUDA;
  }
  DeviceScope scope(dev);
  if (!scope.ok) return QLR_ECUDA;

  // A context on the stack: no device allocation, no launch statistics timing.
  qlr_ctx ctx;
  ctx.device = dev;
  ctx.stream = static_cast<cudaStream_t>(stream);
  ctx.d_err = err;
  if (outer == 0 || X->cols == 0) return QLR_OK;                 // Y is empty
  if (inner == 0) return qlr::zero_qmat(&ctx, *Y);               // empty sums: Y = 0 (a memset)
  if (!qlr::sketch_tc_supported(op, *A, *X, compute)) return QLR_EUNSUPPORTED;

  void* scratch = nullptr;
  const int rc = scratch_address(dev, &scratch);
  if (rc != QLR_OK) return rc;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QLR_ECUDA;
  // Stream-K partial tiles take scratch in proportion to the CTA budget: use the largest budget
  // whose plan fits the array (the need grows with the budget, so the first fit from the top).
  const int l = (int)X->cols;
  int budget = sms;
  while (budget > 1 && qlr::sketch_tc_need(op, outer, inner, l, compute, budget) > QLR_NOALLOC_SCRATCH_BYTES) --budget;
  if (qlr::sketch_tc_need(op, outer, inner, l, compute, budget) > QLR_NOALLOC_SCRATCH_BYTES) return QLR_ENOMEM;
  ctx.num_sms = budget;
  ctx.ws = scratch;
  ctx.ws_bytes = QLR_NOALLOC_SCRATCH_BYTES;
  WsArena ws(scratch, QLR_NOALLOC_SCRATCH_BYTES);
  return qlr::sketch_tc(&ctx, op, *A, *X, *Y, compute, ws);
}
