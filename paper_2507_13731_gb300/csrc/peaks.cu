// Throughput probes for the roofline denominators (measurement support; the paper has no
// counterpart).  Each probe keeps one pipe busy on every SM and is timed by CUDA events:
//  - tcgen05 MMA loops: one CTA per SM accumulates 128 x 256 tiles in TMEM from operands staged
//    once in shared memory (M = 128, N = 256, K = 8 for kind::tf32, K = 16 for kind::f16 with BF16
//    operands), the issuing thread keeping the tensor pipe fed back to back;
//  - FMA loops on the CUDA cores in FP32 and FP64: every thread runs eight independent chains of
//    fused multiply-adds.
// The operands are zero (the values do not change the issue rate), and the results go to a sink
// the host never reads unless a chain produced a non-zero value, so nothing is optimised away.
#include <cstdint>

#include "qlr_internal.h"
#include "tc_common.cuh"

namespace {

using namespace qlr_tc;

constexpr int PM = 128, PN = 256;
constexpr int MMAS_PER_ROUND = 8;

// KIND 0: kind::tf32 (K = 8 per MMA); KIND 1: kind::f16 with BF16 operands (K = 16 per MMA).
// Both operands use 32-byte rows (one K step), the 32-byte swizzled K-major layout.  N = PN
// (256: the dense rate) or 64 (the rate of the narrow MMAs of thin sketches: an MMA of M = 128
// takes about the same time for every N up to ~100).
template <int KIND, int NN = PN>
__global__ void __launch_bounds__(128, 1) mma_peak_kernel(int64_t rounds, int* err, float* sink) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* a = smem;                 // 128 rows x 32 bytes
  unsigned char* b = smem + PM * 32;       // 256 rows x 32 bytes
  uint64_t* done = reinterpret_cast<uint64_t*>(smem + (PM + PN) * 32);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x / 32;
  for (int i = threadIdx.x; i < (PM + PN) * 32 / 16; i += blockDim.x) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)PN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (threadIdx.x == 0) {
    const uint64_t ad = make_desc(smem_u32(a), 16, 8 * 32, 6);
    const uint64_t bd = make_desc(smem_u32(b), 16, 8 * 32, 6);
    const uint32_t fmt = (KIND == 0) ? 2u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(PM >> 4) << 24);
    for (int64_t r = 0; r < rounds; ++r) {
#pragma unroll
      for (int j = 0; j < MMAS_PER_ROUND; ++j) {
        const uint32_t acc = (r > 0 || j > 0) ? 1u : 0u;
        if (KIND == 0)
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        else
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
      }
    }
    umma_commit(done);
  }
  __syncwarp();
  // every thread waits (bounded) for the last MMA, then warp 0 reads one accumulator row
  const bool ok = mbar_wait(done, 0, abort_flag, err);
  tc_fence_after();
  if (warp == 0 && ok) {
    float v[16];
    tmem_ld16(tmem, v);
    if (v[0] != 0.0f) sink[threadIdx.x] = v[0];
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)PN) : "memory");
  }
}

template <class T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int64_t iters, T x, T y, T* sink) {
  T a0 = (T)threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int64_t i = 0; i < iters; ++i) {
    a0 = fma(a0, x, y); a1 = fma(a1, x, y); a2 = fma(a2, x, y); a3 = fma(a3, x, y);
    a4 = fma(a4, x, y); a5 = fma(a5, x, y); a6 = fma(a6, x, y); a7 = fma(a7, x, y);
  }
  const T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == (T)-12345.0) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" int qlr_peak_probe(int kind, int device, int64_t iters, double* flops, float* ms) {
  if (!flops || !ms || iters < 1 || kind < QLR_PEAK_TF32_MMA || kind > QLR_PEAK_BF16_MMA_N64) return QLR_EINVAL;
  const bool mma = kind == QLR_PEAK_TF32_MMA || kind == QLR_PEAK_BF16_MMA || kind == QLR_PEAK_TF32_MMA_N64 ||
                   kind == QLR_PEAK_BF16_MMA_N64;
  if (mma && iters > 400000) return QLR_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); return QLR_ECUDA; }
  if (prev != device && cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return QLR_ECUDA; }
  int sms = 0;
  int rc = QLR_OK;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* scratch = nullptr;   // error word + sink
  float t = 0.f;
  do {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&scratch, 4096) != cudaSuccess ||
        cudaMemsetAsync(scratch, 0, 4096, st) != cudaSuccess) {
      rc = QLR_ECUDA;
      break;
    }
    int* err = static_cast<int*>(scratch);
    char* sink = static_cast<char*>(scratch) + 256;
    double f = 0.0;
    cudaEventRecord(e0, st);
    if (mma) {
      const size_t smem = (size_t)(PM + PN) * 32 + 64 + 1024;
      const bool tf32 = kind == QLR_PEAK_TF32_MMA || kind == QLR_PEAK_TF32_MMA_N64;
      const bool n64 = kind == QLR_PEAK_TF32_MMA_N64 || kind == QLR_PEAK_BF16_MMA_N64;
      auto kern = tf32 ? (n64 ? mma_peak_kernel<0, 64> : mma_peak_kernel<0>) : (n64 ? mma_peak_kernel<1, 64> : mma_peak_kernel<1>);
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        rc = QLR_ECUDA;
        break;
      }
      kern<<<sms, 128, smem, st>>>(iters, err, reinterpret_cast<float*>(sink));
      const double k = tf32 ? 8.0 : 16.0;
      f = (double)sms * (double)iters * MMAS_PER_ROUND * 2.0 * PM * (n64 ? 64 : PN) * k;
    } else {
      const int blocks = sms * 8;
      if (kind == QLR_PEAK_FP32_FMA)
        fma_peak_kernel<float><<<blocks, 256, 0, st>>>(iters, 0.999f, 1e-3f, reinterpret_cast<float*>(sink));
      else
        fma_peak_kernel<double><<<blocks, 256, 0, st>>>(iters, 0.999, 1e-3, reinterpret_cast<double*>(sink));
      f = (double)blocks * 256.0 * (double)iters * 8.0 * 2.0;
    }
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      rc = QLR_ECUDA;
      break;
    }
    int h = 0;
    if (cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) { rc = QLR_ECUDA; break; }
    if (h != 0) { rc = h; break; }
    *flops = f;
    *ms = t;
  } while (false);
  if (rc == QLR_ECUDA) cudaGetLastError();
  if (scratch) cudaFree(scratch);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}
