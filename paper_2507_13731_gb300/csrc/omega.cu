// The Gaussian quaternion test matrix Omega (Def. 2) from a seed, on the host.
//
// Def. 2 asks for a quaternion matrix whose four components are independent standard normal
// entries; the paper fixes no generator.  This library uses a counter-based SplitMix64 (Steele,
// Lea and Flood, OOPSLA 2014) with the Box-Muller transform, so that a C caller can reproduce the
// test matrix the tests and benchmarks hand to both the GPU path and the FP64 oracle:
//   draw t of the stream with seed s is mix(s + (t + 1) * 0x9E3779B97F4A7C15), mix being
//   SplitMix64's finaliser; a uniform is the draw's top 53 bits times 2^-53; normal 2p and 2p + 1
//   come from the uniforms u = draw 2p and w = draw 2p + 1 as r cos(2 pi w) and r sin(2 pi w) with
//   r = sqrt(-2 ln(1 - u)); entry (c, i, j) of an r x s quaternion matrix (plane c, row i, column
//   j) is normal number c r s + j r + i (plane-major, column-major).
#include <cmath>
#include <cstring>
#include <vector>

#include "qlr_internal.h"

namespace {

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

inline double uniform53(uint64_t seed, uint64_t t) {
  return (double)(mix64(seed + (t + 1) * 0x9E3779B97F4A7C15ull) >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace

extern "C" uint64_t qlr_splitmix64(uint64_t seed, uint64_t counter) {
  return mix64(seed + (counter + 1) * 0x9E3779B97F4A7C15ull);
}

extern "C" int qlr_gaussian_qmat_host(uint64_t seed, int64_t rows, int64_t cols, int real_only, double* out) {
  if (!out || rows < 0 || cols < 0) return QLR_EINVAL;
  const int64_t per = rows * cols;
  const int planes = real_only ? 1 : 4;
  const double two_pi = 2.0 * 3.141592653589793;
  const int64_t count = planes * per;
  for (int64_t p = 0; 2 * p < count; ++p) {
    const double u1 = 1.0 - uniform53(seed, (uint64_t)(2 * p));
    const double u2 = uniform53(seed, (uint64_t)(2 * p + 1));
    const double r = std::sqrt(-2.0 * std::log(u1));
    out[2 * p] = r * std::cos(two_pi * u2);
    if (2 * p + 1 < count) out[2 * p + 1] = r * std::sin(two_pi * u2);
  }
  if (real_only) std::memset(out + per, 0, sizeof(double) * (size_t)(3 * per));
  return QLR_OK;
}

extern "C" int qlr_fill_omega(qlr_ctx* ctx, uint64_t seed, int real_only, qlr_qmat* omega) {
  if (!ctx || !omega || omega->layout != QLR_COL_MAJOR) return QLR_EINVAL;
  if (omega->dtype != QLR_F64 && omega->dtype != QLR_F32) return QLR_EINVAL;
  const int64_t r = omega->rows, s = omega->cols;
  if (r < 0 || s < 0 || omega->ld < (r > 1 ? r : 1)) return QLR_ESHAPE;
  if (r == 0 || s == 0) return QLR_OK;
  for (int c = 0; c < 4; ++c)
    if (!omega->plane[c]) return QLR_EINVAL;
  std::vector<double> h((size_t)4 * r * s);
  QLR_TRY(qlr_gaussian_qmat_host(seed, r, s, real_only, h.data()));
  const bool f32 = omega->dtype == QLR_F32;
  std::vector<float> hf(f32 ? h.size() : 0);
  for (size_t e = 0; e < hf.size(); ++e) hf[e] = (float)h[e];
  const size_t esz = f32 ? 4 : 8;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); return QLR_ECUDA; }
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) { cudaGetLastError(); return QLR_ECUDA; }
  int rc = QLR_OK;
  for (int c = 0; c < 4 && rc == QLR_OK; ++c) {
    const void* src = f32 ? (const void*)(hf.data() + (size_t)c * r * s) : (const void*)(h.data() + (size_t)c * r * s);
    if (cudaMemcpy2DAsync(omega->plane[c], (size_t)omega->ld * esz, src, (size_t)r * esz, (size_t)r * esz, (size_t)s,
                          cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
      rc = QLR_ECUDA;
  }
  if (rc == QLR_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = QLR_ECUDA;
  if (rc != QLR_OK) cudaGetLastError();
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return rc;
}
