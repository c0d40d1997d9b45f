// Device-side publication of a recorded step (mpx_step_create): the kernel
// that a step's CUDA graph runs before its engine pass.  It writes the step's
// descriptors and waitall lists into the streams' submission rings exactly as
// host enqueue calls would, with sequence numbers and waitlist indices taken
// from per-stream counters kept in device memory, then releases each ring's
// tail.  One block per stream of the step.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpx_internal.h"

namespace mpxi {
namespace {

__device__ __forceinline__ void st_vol16(void* p, uint4 v) {
  asm volatile("st.volatile.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ uint64_t ld_vol64(const void* p) {
  uint64_t v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(256) step_post_kernel(EngineParams P, const Desc* tmpl,
                                                        const int64_t* tmpl_wl,
                                                        const StepStream* ss, uint64_t* cnt_seq,
                                                        uint64_t* cnt_wl, int32_t* err) {
  const StepStream S = ss[blockIdx.x];
  const int g = S.g;
  __shared__ int ok;
  const uint64_t base = cnt_seq[g];  // last sequence number published on stream g
  const uint64_t wlb = cnt_wl[g];    // next waitlist index of stream g
  const uint64_t slots = 1ull << P.slots_log2, wl_slots = 1ull << P.wl_log2;
  if (threadIdx.x == 0) {
    // the previous step's operations are retired once its engine pass ended
    const uint64_t retired = ld_vol64(&P.sctl[g].retired);
    const uint64_t wl_retired = ld_vol64(&P.sctl[g].wl_retired);
    ok = (base + (uint64_t)S.nops - retired <= slots) &&
         (wlb + (uint64_t)S.nwl - wl_retired <= wl_slots);
    if (!ok) atomicCAS(err, 0, 12 /* MPX_ERR_NO_MEM */);
  }
  __syncthreads();
  if (!ok) return;
  Desc* ring = const_cast<Desc*>(P.rings) + ((size_t)g << P.slots_log2);
  for (int i = threadIdx.x; i < S.nops; i += blockDim.x) {
    Desc d = tmpl[S.op0 + i];
    const uint32_t kind = kw_kind(d.kw);
    if (kind == K_WAITALL) d.aux = wlb + d.aux;        // relative waitlist offset
    else if (kind == K_WAIT) d.aux = base + d.aux;     // relative sequence number
    const uint64_t seq = base + 1 + (uint64_t)i;
    const uint4* src = reinterpret_cast<const uint4*>(&d);
    uint4* dst = reinterpret_cast<uint4*>(ring + ((seq - 1) & (slots - 1)));
    for (int k = 0; k < 4; ++k) st_vol16(dst + k, src[k]);
  }
  int64_t* wl = const_cast<int64_t*>(P.waitlists) + ((size_t)g << P.wl_log2);
  for (int k = threadIdx.x; k < S.nwl; k += blockDim.x) {
    const int64_t rel = tmpl_wl[S.wl0 + k];
    wl[(wlb + (uint64_t)k) & (wl_slots - 1)] = rel == 0 ? 0 : (int64_t)(base + (uint64_t)rel);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // descriptors and lists before the tail the engine acquires
    __threadfence_system();
    const uint64_t tail = base + (uint64_t)S.nops;
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(&P.sctl[g].tail), "l"(tail) : "memory");
    cnt_seq[g] = tail;
    cnt_wl[g] = wlb + (uint64_t)S.nwl;
  }
}

}  // namespace
}  // namespace mpxi

extern "C" int mpxi_step_post_launch(const mpxi::EngineParams* P, const void* tmpl,
                                     const void* tmpl_wl, const void* streams, int nstreams,
                                     uint64_t* cnt_seq, uint64_t* cnt_wl, int32_t* err,
                                     void* cuda_stream) {
  if (nstreams <= 0) return 0;
  mpxi::step_post_kernel<<<nstreams, 256, 0, (cudaStream_t)cuda_stream>>>(
      *P, (const mpxi::Desc*)tmpl, (const int64_t*)tmpl_wl, (const mpxi::StepStream*)streams,
      cnt_seq, cnt_wl, err);
  return (int)cudaGetLastError();
}

extern "C" int mpxi_step_preload(void) {
  cudaFuncAttributes a;
  return cudaFuncGetAttributes(&a, mpxi::step_post_kernel) == cudaSuccess ? 0 : 1;
}
