// Failure-detection self test (the paper has no counterpart): one CTA waits on an mbarrier that
// nothing arrives at, through the bounded wait every tensor-core pipeline uses (limit WAIT_NS,
// 1.5 s).  The wait gives up, records QLR_ETIMEOUT in the context's device error word, and the
// kernel returns normally, so the context stays usable.  Nothing faults, traps or spins without
// a limit.
#include "tc_common.cuh"

namespace {

__global__ void wait_timeout_selftest_kernel(int* err) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    qlr_tc::mbar_init(&bar, 1);
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) qlr_tc::mbar_wait(&bar, 0, &abort_flag, err);   // phase 0 never completes
}

}  // namespace

namespace qlr {

int selftest_wait_timeout(qlr_ctx* ctx) {
  KTimer kt(ctx, QLR_KID_MISC);
  wait_timeout_selftest_kernel<<<1, 32, 0, ctx->stream>>>(ctx->d_err);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

}  // namespace qlr
