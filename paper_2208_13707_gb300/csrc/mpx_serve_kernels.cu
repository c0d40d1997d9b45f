// Small device helpers of the serving loop (mpx_serve_run): deterministic
// payload fill, an order-independent digest of a buffer, and a probe of the
// device clock that completion times are reported in.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  // splitmix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom
  // number generators", 2014)
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// as_f32: two floats in [-1, 1) per word (the top 24 bits of each half),
// else raw bits
__global__ void fill_kernel(uint64_t* p, int64_t nwords, uint64_t seed, int as_f32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t z = mix64(seed ^ mix64((uint64_t)i));
    if (as_f32) {
      const float lo = (float)((uint32_t)z >> 8) * (1.0f / 8388608.0f) - 1.0f;
      const float hi = (float)((uint32_t)(z >> 32) >> 8) * (1.0f / 8388608.0f) - 1.0f;
      p[i] = ((uint64_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
    } else {
      p[i] = z;
    }
  }
}

// sum over bytes b_i of mix64((i << 8) | b_i), wrapping: equal buffers give
// equal digests, and any byte change changes one term
__global__ void digest_kernel(const uint8_t* p, int64_t n, unsigned long long* out) {
  uint64_t acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += mix64(((uint64_t)i << 8) | p[i]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)acc);
}

__global__ void clock_kernel(volatile uint64_t* out) {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *out = t;
}

}  // namespace

extern "C" int mpxi_fill(void* p, int64_t bytes, uint64_t seed, int as_f32, void* stream) {
  if (bytes <= 0) return 0;
  fill_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>((uint64_t*)p, bytes / 8, seed, as_f32);
  return (int)cudaGetLastError();
}

extern "C" int mpxi_digest(const void* p, int64_t bytes, void* out_dev, void* stream) {
  cudaError_t e = cudaMemsetAsync(out_dev, 0, 8, (cudaStream_t)stream);
  if (e != cudaSuccess) return (int)e;
  if (bytes <= 0) return 0;
  int blocks = (int)((bytes + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  digest_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>((const uint8_t*)p, bytes,
                                                          (unsigned long long*)out_dev);
  return (int)cudaGetLastError();
}

extern "C" int mpxi_clock_probe(void* out_mapped, void* stream) {
  clock_kernel<<<1, 1, 0, (cudaStream_t)stream>>>((volatile uint64_t*)out_mapped);
  return (int)cudaGetLastError();
}
