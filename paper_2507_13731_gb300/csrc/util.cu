// Elementwise helpers on quaternion matrices: dtype conversion / copy, zero fill.
#include <cstdio>
#include <cstdlib>

#include "qlr_internal.h"

void qlr_report_cuda(cudaError_t e, const char* expr, const char* file, int line) {
  static const bool on = std::getenv("QLR_DEBUG_CUDA") != nullptr;
  if (on) std::fprintf(stderr, "qlr: %s failed at %s:%d: %s\n", expr, file, line, cudaGetErrorString(e));
}

size_t qlr_dtype_size(int dtype) {
  switch (dtype) {
    case QLR_F64: return 8;
    case QLR_F32: return 4;
    case QLR_BF16: return 2;
    default: return 0;
  }
}

namespace {

template <class S, class D>
__global__ void convert_kernel(const S* __restrict__ s, int64_t lds, D* __restrict__ d, int64_t ldd, int64_t inner,
                               int64_t outer) {
  int64_t tot = inner * outer;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % inner, o = e / inner;
    d[o * ldd + i] = Cvt<D>::from(s ? s[o * lds + i] : S(0));
  }
}

template <class S, class D>
int launch_convert(qlr_ctx* ctx, const void* s, int64_t lds, void* d, int64_t ldd, int64_t inner, int64_t outer) {
  int64_t tot = inner * outer;
  if (tot == 0) return QLR_OK;
  int blocks = (int)std::min<int64_t>((tot + 255) / 256, 4096);
  KTimer kt(ctx, QLR_KID_MISC);
  convert_kernel<S, D><<<blocks, 256, 0, ctx->stream>>>(static_cast<const S*>(s), lds, static_cast<D*>(d), ldd, inner,
                                                         outer);
  qlr_count_launch();
  QLR_CUDA_TRY(cudaGetLastError());
  return QLR_OK;
}

template <class S>
int convert_from(qlr_ctx* ctx, const void* s, int64_t lds, int ddt, void* d, int64_t ldd, int64_t inner, int64_t outer) {
  switch (ddt) {
    case QLR_F64: return launch_convert<S, double>(ctx, s, lds, d, ldd, inner, outer);
    case QLR_F32: return launch_convert<S, float>(ctx, s, lds, d, ldd, inner, outer);
    case QLR_BF16: return launch_convert<S, __nv_bfloat16>(ctx, s, lds, d, ldd, inner, outer);
  }
  return QLR_EINVAL;
}

}  // namespace

namespace qlr {

// Copy src into dst (same shape and layout), converting the element type.  A NULL source plane
// (pure quaternion) writes zeros.
int convert_qmat(qlr_ctx* ctx, const qlr_qmat& src, qlr_qmat& dst) {
  if (src.rows != dst.rows || src.cols != dst.cols || src.layout != dst.layout) return QLR_ESHAPE;
  const bool col = (src.layout == QLR_COL_MAJOR);
  const int64_t inner = col ? src.rows : src.cols, outer = col ? src.cols : src.rows;
  for (int c = 0; c < 4; ++c) {
    if (dst.plane[c] == nullptr) continue;
    int rc;
    switch (src.dtype) {
      case QLR_F64: rc = convert_from<double>(ctx, src.plane[c], src.ld, dst.dtype, dst.plane[c], dst.ld, inner, outer); break;
      case QLR_F32: rc = convert_from<float>(ctx, src.plane[c], src.ld, dst.dtype, dst.plane[c], dst.ld, inner, outer); break;
      case QLR_BF16:
        rc = convert_from<__nv_bfloat16>(ctx, src.plane[c], src.ld, dst.dtype, dst.plane[c], dst.ld, inner, outer);
        break;
      default: return QLR_EINVAL;
    }
    if (rc != QLR_OK) return rc;
  }
  return QLR_OK;
}

int zero_qmat(qlr_ctx* ctx, qlr_qmat& dst) {
  const bool col = (dst.layout == QLR_COL_MAJOR);
  const int64_t inner = col ? dst.rows : dst.cols, outer = col ? dst.cols : dst.rows;
  const size_t esz = qlr_dtype_size(dst.dtype);
  for (int c = 0; c < 4; ++c) {
    if (dst.plane[c] == nullptr || inner == 0 || outer == 0) continue;
    QLR_CUDA_TRY(cudaMemset2DAsync(dst.plane[c], dst.ld * esz, 0, inner * esz, outer, ctx->stream));
  }
  return QLR_OK;
}

}  // namespace qlr
