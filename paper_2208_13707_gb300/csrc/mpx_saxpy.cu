// Listing 4's user compute kernel (§6): y[i] = a * x[i] + y[i], one fused
// multiply-add per element (single rounding).  Exported so that programs and
// tests can interleave compute with enqueued communication in stream order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpx.h"

namespace {

__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(__fmaf_rn(a, x.x, y.x), __fmaf_rn(a, x.y, y.y), __fmaf_rn(a, x.z, y.z),
                     __fmaf_rn(a, x.w, y.w));
}

// Grid-stride over 16-byte vectors, four vectors of x and four of y in flight
// per thread (independent loads) so that a few CTAs per SM cover HBM latency.
__global__ void __launch_bounds__(256) saxpy_kernel(int64_t n, float a, const float* __restrict__ x,
                                                    float* __restrict__ y) {
  const int64_t n4 = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool aligned = ((((uintptr_t)x) | ((uintptr_t)y)) & 15) == 0;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (aligned) {
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4* y4 = reinterpret_cast<float4*>(y);
    int64_t k = i;
    for (; k + 3 * stride < n4; k += 4 * stride) {
      float4 xv[4], yv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xv[u] = x4[k + u * stride];
        yv[u] = y4[k + u * stride];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) y4[k + u * stride] = fma4(a, xv[u], yv[u]);
    }
    for (; k < n4; k += stride) y4[k] = fma4(a, x4[k], y4[k]);
    for (int64_t q = (n4 << 2) + i; q < n; q += stride) y[q] = __fmaf_rn(a, x[q], y[q]);
  } else {
    for (int64_t q = i; q < n; q += stride) y[q] = __fmaf_rn(a, x[q], y[q]);
  }
}

}  // namespace

extern "C" int mpxi_saxpy_preload(void) {
  cudaFuncAttributes a;
  return cudaFuncGetAttributes(&a, saxpy_kernel) == cudaSuccess ? 0 : 1;
}

extern "C" int mpx_saxpy_enqueue(int64_t n, float a, const float* x, float* y,
                                 mpx_cuda_stream_t stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return MPX_ERR_ARG;
  if (n == 0) return MPX_SUCCESS;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = ((n >> 2) + 1023) / 1024;  // about four vectors per thread
  const int64_t cap = (int64_t)nsm * 4;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  saxpy_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, a, x, y);
  return cudaGetLastError() == cudaSuccess ? MPX_SUCCESS : MPX_ERR_CUDA;
}
