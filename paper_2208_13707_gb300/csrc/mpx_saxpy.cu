// Listing 4's user compute kernel (§6): y[i] = a * x[i] + y[i], one fused
// multiply-add per element (single rounding).  Exported so that programs and
// tests can interleave compute with enqueued communication in stream order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpx.h"

namespace {

__global__ void saxpy_kernel(int64_t n, float a, const float* __restrict__ x, float* __restrict__ y) {
  const int64_t n4 = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool aligned = ((((uintptr_t)x) | ((uintptr_t)y)) & 15) == 0;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (aligned) {
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4* y4 = reinterpret_cast<float4*>(y);
    for (int64_t k = i; k < n4; k += stride) {
      float4 xv = x4[k], yv = y4[k];
      yv.x = __fmaf_rn(a, xv.x, yv.x);
      yv.y = __fmaf_rn(a, xv.y, yv.y);
      yv.z = __fmaf_rn(a, xv.z, yv.z);
      yv.w = __fmaf_rn(a, xv.w, yv.w);
      y4[k] = yv;
    }
    for (int64_t k = (n4 << 2) + i; k < n; k += stride) y[k] = __fmaf_rn(a, x[k], y[k]);
  } else {
    for (int64_t k = i; k < n; k += stride) y[k] = __fmaf_rn(a, x[k], y[k]);
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
  int64_t blocks = ((n >> 2) + 255) / 256;
  const int64_t cap = (int64_t)nsm * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  saxpy_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, a, x, y);
  return cudaGetLastError() == cudaSuccess ? MPX_SUCCESS : MPX_ERR_CUDA;
}
