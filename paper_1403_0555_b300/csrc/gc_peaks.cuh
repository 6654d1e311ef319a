// Throughput probes of the arithmetic units the enumerator's kernels are bound
// by: FP32 FMA, packed f32x2 FMA, FP64 FMA (all lanes, and one lane per warp:
// whether an FP64 warp instruction costs the pipe by its active lanes) and the
// special-function unit's reciprocal square root.  They give the roofline
// denominators measured on the GPU that runs the library (the paper has no
// counterpart).  Every thread runs eight independent dependency chains of one
// instruction kind, unrolled eight times, so the probe measures the unit's
// throughput rather than its latency, and loop overhead is under 5 % of the
// issued instructions.
#pragma once
#include <cuda_runtime.h>

namespace gc {

enum { kPeakFFMA = 0, kPeakFFMA2 = 1, kPeakDFMA = 2, kPeakRSQ = 3, kPeakDFMA1 = 4 };

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

__device__ __forceinline__ float rsq_approx(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// m and c are runtime values (the host passes m = 1 - 2^-20, c = 2^-21), so
// the chains cannot be folded; each thread stores one sum so none is dead.
template <int KIND>
__global__ void __launch_bounds__(256) peak_probe_kernel(float* out, int iters, float m, float c) {
  const float seed = (float)(threadIdx.x + 1) * 1e-3f;
  float r = 0.f;
  if constexpr (KIND == kPeakFFMA) {
    float a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = seed + (float)u;
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = fmaf(a[u], m, c);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) r += a[u];
  } else if constexpr (KIND == kPeakFFMA2) {
    float2 a[8];
    const float2 mm = make_float2(m, m), cc = make_float2(c, c);
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = make_float2(seed + (float)u, seed - (float)u);
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = ffma2(a[u], mm, cc);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) r += a[u].x + a[u].y;
  } else if constexpr (KIND == kPeakDFMA || KIND == kPeakDFMA1) {
    // kPeakDFMA1: only lane 0 of each warp runs the chains
    double a[8];
    const double md = (double)m, cd = (double)c;
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = (double)seed + (double)u;
    if (KIND == kPeakDFMA || (threadIdx.x & 31) == 0) {
#pragma unroll 8
      for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = fma(a[u], md, cd);
      }
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u];
    r = (float)s;
  } else {
    float a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = seed + (float)(u + 1);
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = rsq_approx(a[u]);   // tends to the fixed point 1
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) r += a[u];
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace gc
