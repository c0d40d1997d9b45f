// Host runtime of libmpx: worlds, streams (endpoints), stream communicators,
// datatypes, the lock-free enqueue path and the engine's life cycle.
//
// Enqueue path (§3.4; §5.2 names the better design: a progress agent plus
// triggers enqueued in the GPU stream):
//   1. validate the call,
//   2. write a 64-byte descriptor into the stream's submission ring (pinned
//      host memory) and publish the ring tail with a release store -- no lock,
//      the stream is a serial context (§3.1),
//   3. put a stream-ordered doorbell (cuStreamWriteValue64) on the user's
//      CUDA stream, telling the engine that earlier work on the stream is done
//      and the buffer may be read or written,
//   4. for calls that block in stream order (send, recv, wait, waitall,
//      allreduce) put cuStreamWaitValue64(done >= seq) on the stream: work
//      enqueued afterwards starts once the engine has completed the call,
//   5. make sure the engine kernel is running (persistent mode).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mpx.h"
#include "mpx_internal.h"
#include "mpx_plain.h"

using namespace mpxi;

extern "C" int mpxi_engine_max_ctas_per_sm(int nthreads);
extern "C" int mpxi_engine_regs(void);
extern "C" int mpxi_engine_preload(void);
extern "C" int mpxi_saxpy_preload(void);
extern "C" int mpxi_step_preload(void);
extern "C" int mpxi_static_preload(void);
extern "C" int mpxi_plain_preload(void);
extern "C" int mpxi_step_post_launch(const mpxi::EngineParams* P, const void* tmpl,
                                     const void* tmpl_wl, const void* streams, int nstreams,
                                     uint64_t* cnt_seq, uint64_t* cnt_wl, int32_t* err,
                                     void* cuda_stream);

// A cuStreamWaitValue64 that is not yet satisfied stalls the hardware queue
// its CUDA stream is mapped to, and every other stream sharing that queue.
// CUDA maps streams onto CUDA_DEVICE_MAX_CONNECTIONS queues (default 8), so
// a doorbell of one virtual rank could sit behind another rank's blocked
// wait.  Ask for the maximum (32) when the library is loaded before CUDA is
// initialised; an explicit user setting is kept.
__attribute__((constructor)) static void mpxi_default_connections() {
  setenv("CUDA_DEVICE_MAX_CONNECTIONS", "32", 0);
}

// MPX_DEBUG=1 traces host-side steps to stderr.
static bool debug_on() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("MPX_DEBUG");
    v = (e && *e && *e != '0') ? 1 : 0;
  }
  return v == 1;
}
#define MPX_TRACE(...)                    \
  do {                                    \
    if (debug_on()) {                     \
      fprintf(stderr, "[mpx] " __VA_ARGS__); \
      fprintf(stderr, "\n");              \
      fflush(stderr);                     \
    }                                     \
  } while (0)

// Stream memory operations come from the driver; they are looked up through
// the runtime so the library loads (and its symbols can be inspected) on a
// machine without a driver.
namespace {
typedef CUresult (*PfnMemop64)(CUstream, CUdeviceptr, cuuint64_t, unsigned int);
PfnMemop64 g_write64 = nullptr;
PfnMemop64 g_wait64 = nullptr;
std::once_flag g_memops_once;

bool memops_ready() {
  std::call_once(g_memops_once, [] {
    void* fp = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue64", &fp, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_write64 = (PfnMemop64)fp;
    fp = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuStreamWaitValue64", &fp, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_wait64 = (PfnMemop64)fp;
  });
  return g_write64 && g_wait64;
}
}  // namespace

// ---------------------------------------------------------------------------
// datatypes (process-wide, append-only table; reads need no lock)
// ---------------------------------------------------------------------------
namespace {

struct TypeRec {
  int32_t alive;
  int32_t base;
  int32_t vcount, blocklen, stride;
};

constexpr int kMaxTypes = 1 << 16;
constexpr int64_t kMaxTypeExtent = 1ll << 48;  // bytes of one instance of a derived type
constexpr int64_t kMaxSpan = 1ll << 60;        // bytes one call may span
constexpr int kFirstDerived = 16;
TypeRec g_types[kMaxTypes];
std::mutex g_types_mu;
int g_types_next = kFirstDerived;
std::vector<int> g_types_free;

struct TypeInit {
  TypeInit() {
    for (int b = 0; b <= MPX_DOUBLE; ++b) g_types[b] = TypeRec{1, b, 1, 1, 1};
  }
} g_type_init;

const TypeRec* type_get(mpx_datatype_t t) {
  if (t < 0 || t >= kMaxTypes) return nullptr;
  const TypeRec* r = &g_types[t];
  if (!__atomic_load_n(&r->alive, __ATOMIC_ACQUIRE)) return nullptr;
  return r;
}

// `count` instances of type t span at most kMaxSpan bytes (so the packed size,
// the extent and every offset the engine derives from them fit in int64).
// Checked by division before anything multiplies the count.
bool span_ok(const TypeRec* t, int64_t count) {
  const int64_t ext = base_size((uint32_t)t->base) * ((int64_t)(t->vcount - 1) * t->stride + t->blocklen);
  return count >= 0 && (count == 0 || count <= kMaxSpan / (ext > 0 ? ext : 1));
}

int64_t now_ms() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000 + ts.tv_nsec / 1000000;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int log2i(int64_t v) {
  int l = 0;
  while ((1ll << l) < v) ++l;
  return l;
}

}  // namespace

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------
struct mpx_world_s;

struct mpx_stream_s {
  mpx_world_s* w;
  int id;
  int rank;
  cudaStream_t cs;
  unsigned flags;
  uint64_t next_seq;  // next sequence number to publish
  uint64_t wl_next;   // next waitlist index
  uint64_t retired_seen;  // last value read of the engine's retirement word
  mpx_step_s* step;   // recorded step that owns the stream's sequence numbers, or null
  uint64_t owed;      // a batch wrote descriptors up to here without releasing the tail
                      // and ringing the doorbell (0 = none)
  int ncomms;         // communicators using this stream
  bool owns_cs;       // the library created cs (MPI_INFO_NULL) and destroys it at free
};

struct CommShared {
  std::atomic<int> handles;
  int id;
  int reduce_mode;
  // multiplex stream communicator (§3.5): member (rank r, local index i) is
  // mux_off[r] + i; empty for a communicator with one stream per rank
  std::vector<int> mux_off;
  int mux_max = 0;  // most streams any rank attached
  bool mux() const { return !mux_off.empty(); }
};

struct mpx_comm_s {
  mpx_world_s* w;
  CommShared* shared;
  int rank;
  int size;
  mpx_stream_s* stream;              // the rank's stream (multiplex: its index 0)
  std::vector<mpx_stream_s*> local;  // multiplex: the rank's streams by local index
};

struct mpx_world_s {
  int widx;
  int nranks;
  mpx_world_config_t cfg;
  int device;
  int nsm;
  int slots_log2, wl_log2, qcap_log2, tq_log2, sr_log2, iw;
  // submission side: pinned host memory, or managed memory kept on the
  // device (rings_managed) that the host reaches through the coherent link
  Desc* rings;
  int64_t* waitlists;
  StreamCtl* sctl;
  bool rings_managed;
  WorldCtl* wctl;     // pinned host memory
  // device memory (one block; see layout in world_create)
  void* dev_block;
  size_t dev_bytes;
  EngineParams params;
  cudaStream_t engine_stream;
  int engine_ctas, engine_threads;
  std::mutex mu;                    // stream/comm creation
  std::vector<mpx_stream_s*> streams;
  std::vector<uint64_t> slot_seq;   // per endpoint: last sequence number used
  int comms_used;
  int live_comm_handles;
  plain::PlainWorld* plain;
};

// Requests name (world index, endpoint, sequence number):
// bits 56..62 world, 40..55 endpoint, 0..39 sequence number.
namespace {
constexpr int kMaxWorlds = 128;
mpx_world_s* g_world_table[kMaxWorlds];
std::mutex g_worlds_mu;
}  // namespace

static mpx_request_t make_request(mpx_stream_s* s, uint64_t seq);

// ---------------------------------------------------------------------------
// configuration
// ---------------------------------------------------------------------------
static int64_t env_i64(const char* name, int64_t dflt) {
  const char* v = getenv(name);
  if (!v || !*v) return dflt;
  return strtoll(v, nullptr, 0);
}

extern "C" int mpx_world_config_init(mpx_world_config_t* c) {
  if (!c) return MPX_ERR_ARG;
  memset(c, 0, sizeof(*c));
  c->engine_mode = (int32_t)env_i64("MPX_ENGINE_MODE", MPX_ENGINE_PERSISTENT);
  c->max_streams = (int32_t)env_i64("MPX_MAX_STREAMS", 64);
  c->ring_slots = (int32_t)env_i64("MPX_RING_SLOTS", 4096);
  c->max_comms = (int32_t)env_i64("MPX_MAX_COMMS", 8);
  c->queue_slots = (int32_t)env_i64("MPX_QUEUE_SLOTS", 4096);
  c->task_slots = (int32_t)env_i64("MPX_TASK_SLOTS", 16384);
  c->engine_ctas = (int32_t)env_i64("MPX_ENGINE_CTAS", 0);
  c->engine_threads = (int32_t)env_i64("MPX_ENGINE_THREADS", 256);
  c->tile_bytes = (int32_t)env_i64("MPX_TILE_BYTES", 65536);
  c->bulk_min_bytes = (int32_t)env_i64("MPX_BULK_MIN_BYTES", 32768);
  c->reduce_mode = (int32_t)env_i64("MPX_REDUCE_MODE", MPX_REDUCE_FIXED);
  c->mover_schedule = (int32_t)env_i64("MPX_MOVER_SCHEDULE", MPX_MOVERS_WORKLIST);
  c->staging_bytes = env_i64("MPX_STAGING_BYTES", 256ll << 20);
  c->budget_bytes = env_i64("MPX_BUDGET_BYTES", 0);
  c->watchdog_ns = env_i64("MPX_WATCHDOG_NS", 10ll * 1000 * 1000 * 1000);
  c->idle_exit_ns = env_i64("MPX_IDLE_EXIT_NS", 100ll * 1000 * 1000);
  c->stage_delay_ns = env_i64("MPX_STAGE_DELAY_NS", 20000);
  c->ring_placement = (int32_t)env_i64("MPX_RING_PLACEMENT", MPX_RINGS_HOST);
  return MPX_SUCCESS;
}

// ---------------------------------------------------------------------------
// world
// ---------------------------------------------------------------------------
static mpx_request_t make_request(mpx_stream_s* s, uint64_t seq) {
  return (mpx_request_t)(((uint64_t)s->w->widx << 56) | ((uint64_t)s->id << 40) | seq);
}

static void world_release(mpx_world_s* w) {
  if (!w) return;
  if (w->widx >= 0) {
    std::lock_guard<std::mutex> g(g_worlds_mu);
    g_world_table[w->widx] = nullptr;
  }
  if (w->plain) plain::destroy(w->plain);
  if (w->engine_stream) cudaStreamDestroy(w->engine_stream);
  if (w->dev_block) cudaFree(w->dev_block);
  for (void* p : {(void*)w->rings, (void*)w->waitlists, (void*)w->sctl}) {
    if (!p) continue;
    if (w->rings_managed) cudaFree(p);
    else cudaFreeHost(p);
  }
  if (w->wctl) cudaFreeHost(w->wctl);
  delete w;
}

// Diagnostic: one attribute of the current device (cudaDeviceAttr numbering).
extern "C" int mpxi_device_attr(int attr, int* value) {
  int dev = 0;
  if (!value || cudaGetDevice(&dev) != cudaSuccess) return MPX_ERR_CUDA;
  return cudaDeviceGetAttribute(value, (cudaDeviceAttr)attr, dev) == cudaSuccess ? MPX_SUCCESS : MPX_ERR_CUDA;
}

// Device-resident submission side: managed memory whose preferred location
// is the device, mapped for direct host access (on a coherent chip-to-chip
// link the host's loads and stores reach device memory without migrating
// pages), moved to the device before anyone touches it and zeroed there.
static int alloc_device_rings(mpx_world_s* w, size_t ring_b, size_t wl_b, size_t sctl_b) {
  int direct = 0, concurrent = 0;
  if (cudaDeviceGetAttribute(&direct, cudaDevAttrDirectManagedMemAccessFromHost, w->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&concurrent, cudaDevAttrConcurrentManagedAccess, w->device) != cudaSuccess)
    return MPX_ERR_CUDA;
  if (!direct || !concurrent) return MPX_ERR_UNSUPPORTED;
  cudaMemLocation dev{};
  dev.type = cudaMemLocationTypeDevice;
  dev.id = w->device;
  cudaMemLocation host{};
  host.type = cudaMemLocationTypeHost;
  host.id = 0;
  w->rings_managed = true;
  void** dst[3] = {(void**)&w->rings, (void**)&w->waitlists, (void**)&w->sctl};
  const size_t bytes[3] = {ring_b, wl_b, sctl_b};
  for (int k = 0; k < 3; ++k) {
    if (cudaMallocManaged(dst[k], bytes[k], cudaMemAttachGlobal) != cudaSuccess) return MPX_ERR_NO_MEM;
    if (cudaMemAdvise(*dst[k], bytes[k], cudaMemAdviseSetPreferredLocation, dev) != cudaSuccess ||
        cudaMemAdvise(*dst[k], bytes[k], cudaMemAdviseSetAccessedBy, host) != cudaSuccess ||
        cudaMemAdvise(*dst[k], bytes[k], cudaMemAdviseSetAccessedBy, dev) != cudaSuccess ||
        cudaMemPrefetchAsync(*dst[k], bytes[k], dev, 0, 0) != cudaSuccess ||
        cudaMemsetAsync(*dst[k], 0, bytes[k], 0) != cudaSuccess)
      return MPX_ERR_CUDA;
  }
  return cudaStreamSynchronize(0) == cudaSuccess ? MPX_SUCCESS : MPX_ERR_CUDA;
}

extern "C" int mpx_world_create(int nranks, const mpx_world_config_t* cfg_in, mpx_world_t* out) {
  if (!out || nranks < 1 || nranks > 4096) return MPX_ERR_ARG;
  *out = nullptr;
  mpx_world_config_t cfg;
  if (cfg_in) cfg = *cfg_in;
  else mpx_world_config_init(&cfg);
  if (cfg.max_streams < 1 || cfg.max_streams > 1024) return MPX_ERR_ARG;
  if (!is_pow2(cfg.ring_slots) || cfg.ring_slots < 16) return MPX_ERR_ARG;
  if (!is_pow2(cfg.queue_slots) || cfg.queue_slots < 32) return MPX_ERR_ARG;
  if (!is_pow2(cfg.task_slots) || cfg.task_slots < 64) return MPX_ERR_ARG;
  if (cfg.max_comms < 1 || cfg.max_comms > 65535) return MPX_ERR_ARG;
  if (cfg.tile_bytes < 256 || (cfg.tile_bytes & 15)) return MPX_ERR_ARG;
  if (cfg.engine_threads < 64 || cfg.engine_threads > 512 || (cfg.engine_threads & 31))
    return MPX_ERR_ARG;
  if (cfg.engine_mode < MPX_ENGINE_PERSISTENT || cfg.engine_mode > MPX_ENGINE_PLAIN) return MPX_ERR_ARG;
  if (cfg.staging_bytes < 4096) return MPX_ERR_ARG;
  if (cfg.mover_schedule != MPX_MOVERS_WORKLIST && cfg.mover_schedule != MPX_MOVERS_PER_CTA)
    return MPX_ERR_ARG;
  if (cfg.ring_placement != MPX_RINGS_HOST && cfg.ring_placement != MPX_RINGS_DEVICE) return MPX_ERR_ARG;

  mpx_world_s* w = new (std::nothrow) mpx_world_s();
  if (!w) return MPX_ERR_NO_MEM;
  w->widx = -1;
  {
    std::lock_guard<std::mutex> g(g_worlds_mu);
    for (int i = 0; i < kMaxWorlds; ++i)
      if (!g_world_table[i]) { g_world_table[i] = w; w->widx = i; break; }
  }
  if (w->widx < 0) { delete w; return MPX_ERR_NO_MEM; }
  w->nranks = nranks;
  w->cfg = cfg;
  w->plain = nullptr;
  w->comms_used = 0;
  w->live_comm_handles = 0;
  if (cudaGetDevice(&w->device) != cudaSuccess) { world_release(w); return MPX_ERR_CUDA; }
  cudaDeviceGetAttribute(&w->nsm, cudaDevAttrMultiProcessorCount, w->device);
  // make sure the runtime's primary context exists, and the driver's stream
  // memory operations are available
  MPX_TRACE("world_create: nranks=%d mode=%d", nranks, cfg.engine_mode);
  cudaFree(0);
  MPX_TRACE("world_create: context ready");
  if (cfg.engine_mode != MPX_ENGINE_PLAIN && !memops_ready()) { world_release(w); return MPX_ERR_CUDA; }
  // load every kernel of the library before any engine runs (lazy loading of
  // a module can wait for running kernels, and a resident engine is one)
  if (mpxi_engine_preload() || mpxi_saxpy_preload() || mpxi_step_preload() || mpxi_static_preload() ||
      mpxi_plain_preload()) {
    world_release(w);
    return MPX_ERR_CUDA;
  }
  MPX_TRACE("world_create: memops and kernels loaded");
  const int S = cfg.max_streams;
  w->slots_log2 = log2i(cfg.ring_slots);
  w->wl_log2 = log2i((int64_t)cfg.ring_slots * 4);
  w->qcap_log2 = log2i(cfg.queue_slots);
  w->tq_log2 = log2i(cfg.task_slots);
  w->sr_log2 = 16;
  w->iw = 32;
  const size_t slots = (size_t)1 << w->slots_log2;
  const size_t ndom = (size_t)cfg.max_comms * nranks;

  // submission rings, waitlists, stream control lines: pinned host memory,
  // or device memory written by the host through the coherent link
  const size_t ring_b = (size_t)S * slots * sizeof(Desc);
  const size_t wl_b = ((size_t)S << w->wl_log2) * sizeof(int64_t);
  const size_t sctl_b = (size_t)S * sizeof(StreamCtl);
  if (cfg.ring_placement == MPX_RINGS_DEVICE) {
    const int rc = alloc_device_rings(w, ring_b, wl_b, sctl_b);
    if (rc) { world_release(w); return rc; }
  } else if (cudaHostAlloc((void**)&w->rings, ring_b, cudaHostAllocMapped) != cudaSuccess ||
             cudaHostAlloc((void**)&w->waitlists, wl_b, cudaHostAllocMapped) != cudaSuccess ||
             cudaHostAlloc((void**)&w->sctl, sctl_b, cudaHostAllocMapped) != cudaSuccess) {
    world_release(w);
    return MPX_ERR_NO_MEM;
  } else {
    memset(w->sctl, 0, sctl_b);
  }
  if (cudaHostAlloc((void**)&w->wctl, sizeof(WorldCtl), cudaHostAllocMapped) != cudaSuccess) {
    world_release(w);
    return MPX_ERR_NO_MEM;
  }
  memset(w->wctl, 0, sizeof(WorldCtl));
  w->slot_seq.assign(S, 0);
  w->streams.assign(S, nullptr);

  if (cfg.engine_mode == MPX_ENGINE_PLAIN) {
    w->plain = plain::create(nranks, cfg.max_streams, cfg.staging_bytes);
    if (!w->plain) { world_release(w); return MPX_ERR_NO_MEM; }
    plain::set_world_index(w->plain, w->widx);
    if (mpxi_saxpy_preload() || mpxi_static_preload() || mpxi_plain_preload()) {
      world_release(w);
      return MPX_ERR_CUDA;
    }
    *out = w;
    return MPX_SUCCESS;
  }

  // device memory, carved from one allocation
  struct Part { size_t bytes; void** dst; };
  EngineParams& P = w->params;
  memset(&P, 0, sizeof(P));
  const size_t iwn = (size_t)cfg.max_comms * w->iw;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t o = (off + 255) & ~(size_t)255;
    off = o + bytes;
    return o;
  };
  const size_t o_door = carve(S * 8), o_done = carve(S * 8);
  const size_t o_ops = carve((size_t)S * slots * sizeof(DOp));
  const size_t o_ss = carve(S * sizeof(SState));
  const size_t o_post = carve((size_t)S * slots * sizeof(PostRec));
  const size_t o_pq = carve((ndom << w->qcap_log2) * sizeof(QEntry));
  const size_t o_uq = carve((ndom << w->qcap_log2) * sizeof(QEntry));
  const size_t o_pqh = carve(ndom * sizeof(QHead)), o_uqh = carve(ndom * sizeof(QHead));
  const size_t o_tasks = carve(((size_t)1 << w->tq_log2) * sizeof(Task));
  const size_t o_cq = carve(((size_t)2 << w->tq_log2) * sizeof(uint64_t));
  const size_t o_sh = carve(sizeof(Shared));
  const size_t o_srec = carve(((size_t)1 << w->sr_log2) * sizeof(StageRec));
  const size_t o_inst = carve(iwn * sizeof(InstSlot));
  const size_t o_irefs = carve(iwn * nranks * 8);
  const size_t o_ninst = carve((size_t)cfg.max_comms * nranks * 8);
  const size_t o_rptr = carve(iwn * 2 * nranks * 8);
  const size_t o_wl = carve(((size_t)S << w->wl_log2) * sizeof(int64_t));
  // counting-sort scratch for large rounds (skipped for very large worlds,
  // which then match by scanning)
  const bool sort_ok = (size_t)S * ndom <= ((size_t)16 << 20);
  const size_t o_cnt2 = sort_ok ? carve((size_t)S * ndom * 4) : 0;
  const size_t o_dtot = sort_ok ? carve(ndom * 4) : 0;
  const size_t o_dbase = sort_ok ? carve(ndom * 8) : 0;
  const size_t o_dlist = sort_ok ? carve((size_t)S * slots * sizeof(PostRec)) : 0;
  size_t cand_cap = 1;  // a power of two at least the operations in flight
  while (cand_cap < (size_t)S * slots) cand_cap <<= 1;
  const size_t o_cand = carve(cand_cap * 8);
  const int64_t trace_cap = env_i64("MPX_ENGINE_TRACE", 0);  // diagnostic tile trace records
  const size_t o_trace = trace_cap > 0 ? carve((size_t)trace_cap * 32 + 8) : 0;
  const size_t o_stage = carve((size_t)cfg.staging_bytes);
  w->dev_bytes = off;
  if (cfg.budget_bytes > 0 && (int64_t)off > cfg.budget_bytes) { world_release(w); return MPX_ERR_NO_MEM; }
  MPX_TRACE("world_create: device block %zu bytes", off);
  if (cudaMalloc(&w->dev_block, off) != cudaSuccess) { world_release(w); return MPX_ERR_NO_MEM; }
  uint8_t* base = (uint8_t*)w->dev_block;
  // zero everything except the staging arena
  if (cudaMemset(base, 0, o_stage) != cudaSuccess) { world_release(w); return MPX_ERR_CUDA; }
  std::vector<SState> ss(S);
  for (auto& x : ss) {
    memset(&x, 0, sizeof(x));
    x.cursor = 1;
    x.pc = 1;
    x.sched = 1;
  }
  if (cudaMemcpy(base + o_ss, ss.data(), S * sizeof(SState), cudaMemcpyHostToDevice) != cudaSuccess) {
    world_release(w);
    return MPX_ERR_CUDA;
  }

  P.nranks = nranks;
  P.max_streams = S;
  P.slots_log2 = w->slots_log2;
  P.max_comms = cfg.max_comms;
  P.qcap_log2 = w->qcap_log2;
  P.tq_log2 = w->tq_log2;
  P.iw = w->iw;
  P.mode = 0;
  P.wl_log2 = w->wl_log2;
  P.sr_log2 = w->sr_log2;
  P.ctl_ctas = 1;
  P.movers_per_cta = cfg.mover_schedule == MPX_MOVERS_PER_CTA ? 1 : 0;
  // per-phase timers of the control CTA (diagnostic; reported through
  // mpx_world_get_counters); MPX_ENGINE_TIMING=0 leaves them out
  P.timing = env_i64("MPX_ENGINE_TIMING", 1) != 0 ? 1 : 0;
  P.watchdog_ns = cfg.watchdog_ns;
  P.idle_ns = cfg.idle_exit_ns;
  P.stage_delay_ns = cfg.stage_delay_ns;
  P.tile_bytes = cfg.tile_bytes;
  P.bulk_min = cfg.bulk_min_bytes;
  P.stage_bytes = cfg.staging_bytes;
  void* dp;
  if (w->rings_managed) {  // one address for host and device
    P.rings = w->rings;
    P.waitlists = w->waitlists;
    P.sctl = w->sctl;
  } else {
    cudaHostGetDevicePointer(&dp, w->rings, 0); P.rings = (const Desc*)dp;
    cudaHostGetDevicePointer(&dp, w->waitlists, 0); P.waitlists = (const int64_t*)dp;
    cudaHostGetDevicePointer(&dp, w->sctl, 0); P.sctl = (StreamCtl*)dp;
  }
  cudaHostGetDevicePointer(&dp, w->wctl, 0); P.wctl = (WorldCtl*)dp;
  P.doorbell = (uint64_t*)(base + o_door);
  P.done = (uint64_t*)(base + o_done);
  P.ops = (DOp*)(base + o_ops);
  P.ss = (SState*)(base + o_ss);
  P.postbuf = (PostRec*)(base + o_post);
  P.pq = (QEntry*)(base + o_pq);
  P.uq = (QEntry*)(base + o_uq);
  P.pqh = (QHead*)(base + o_pqh);
  P.uqh = (QHead*)(base + o_uqh);
  P.tasks = (Task*)(base + o_tasks);
  P.cq = (uint64_t*)(base + o_cq);
  P.sh = (Shared*)(base + o_sh);
  P.srec = (StageRec*)(base + o_srec);
  P.inst = (InstSlot*)(base + o_inst);
  P.inst_refs = (uint64_t*)(base + o_irefs);
  P.next_inst = (int64_t*)(base + o_ninst);
  P.reduce_ptrs = (uint64_t*)(base + o_rptr);
  P.stage = base + o_stage;
  P.wl_dev = (int64_t*)(base + o_wl);
  P.cnt2 = sort_ok ? (int32_t*)(base + o_cnt2) : nullptr;
  P.dtot = sort_ok ? (int32_t*)(base + o_dtot) : nullptr;
  P.dbase = sort_ok ? (int64_t*)(base + o_dbase) : nullptr;
  P.dlist = sort_ok ? (PostRec*)(base + o_dlist) : nullptr;
  P.cand = (uint64_t*)(base + o_cand);
  P.cand_cap = (int64_t)cand_cap;
  P.trace = trace_cap > 0 ? (uint64_t*)(base + o_trace) : nullptr;
  P.trace_pos = trace_cap > 0 ? (uint64_t*)(base + o_trace + (size_t)trace_cap * 32) : nullptr;
  P.trace_cap = trace_cap > 0 ? trace_cap : 0;

  if (cudaStreamCreateWithFlags(&w->engine_stream, cudaStreamNonBlocking) != cudaSuccess) {
    world_release(w);
    return MPX_ERR_CUDA;
  }
  w->engine_threads = cfg.engine_threads;
  if (cfg.engine_mode == MPX_ENGINE_PERSISTENT) {
    // a resident engine leaves at least half of each SM's registers to the
    // application's kernels: with all of them taken, a kernel enqueued before
    // a send never runs, its doorbell never rings and the engine waits for it
    const int regs = mpxi_engine_regs();
    const int cap = regs > 0 ? std::max(64, (32768 / regs) & ~31) : 256;
    w->engine_threads = std::min(w->engine_threads, cap);
  }
  int per_sm = mpxi_engine_max_ctas_per_sm(w->engine_threads);
  if (per_sm < 1) { world_release(w); return MPX_ERR_CUDA; }
  int ctas = cfg.engine_ctas > 0 ? cfg.engine_ctas : w->nsm;
  ctas = std::min(ctas, per_sm * w->nsm);
  w->engine_ctas = std::max(1, ctas);
  P.nctas = w->engine_ctas;
  MPX_TRACE("world_create: done, engine %d x %d (per_sm %d)", w->engine_ctas, w->engine_threads, per_sm);
  *out = w;
  return MPX_SUCCESS;
}

static int launch_engine(mpx_world_s* w, cudaStream_t s, int mode, bool limits = true) {
  EngineParams P = w->params;
  P.mode = mode;
  P.nlimit = 0;
  if (mode == 1) {
    P.idle_ns = std::min<int64_t>(w->cfg.idle_exit_ns, 200000);
    // a pass drains what was published before it was enqueued
    if (limits && w->cfg.max_streams <= kMaxDrainLimits) {
      P.nlimit = w->cfg.max_streams;
      for (int g = 0; g < P.nlimit; ++g) P.limit[g] = __atomic_load_n(&w->sctl[g].tail, __ATOMIC_ACQUIRE);
    }
  }
  MPX_TRACE("launch_engine: mode %d", mode);
  int e = mpxi_engine_launch(&P, w->engine_ctas, w->engine_threads, (void*)s, 1);
  MPX_TRACE("launch_engine: rc %d", e);
  return e == 0 ? MPX_SUCCESS : MPX_ERR_CUDA;
}

// Persistent mode: launch the engine if it is not running (see the exit
// protocol in the engine: it re-checks the rings after announcing EXITING).
static int ensure_engine(mpx_world_s* w) {
  if (w->cfg.engine_mode != MPX_ENGINE_PERSISTENT) return MPX_SUCCESS;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  const int64_t t0 = now_ms();
  for (;;) {
    int st = __atomic_load_n(&w->wctl->state, __ATOMIC_ACQUIRE);
    if (st == ENG_RUNNING) return MPX_SUCCESS;
    if (st == ENG_STOPPED) {
      int expected = ENG_STOPPED;
      if (__atomic_compare_exchange_n(&w->wctl->state, &expected, ENG_RUNNING, false,
                                      __ATOMIC_ACQ_REL, __ATOMIC_ACQUIRE)) {
        int rc = launch_engine(w, w->engine_stream, 0);
        if (rc != MPX_SUCCESS) __atomic_store_n(&w->wctl->state, ENG_STOPPED, __ATOMIC_RELEASE);
        return rc;
      }
      continue;
    }
    if (now_ms() - t0 > 5000) return MPX_ERR_STATE;
    std::this_thread::yield();
  }
}

extern "C" int mpx_world_start(mpx_world_t w) {
  if (!w) return MPX_ERR_ARG;
  if (w->cfg.engine_mode != MPX_ENGINE_PERSISTENT) return MPX_ERR_STATE;
  return ensure_engine(w);
}

extern "C" int mpx_world_stop(mpx_world_t w, int timeout_ms) {
  if (!w) return MPX_ERR_ARG;
  if (w->cfg.engine_mode != MPX_ENGINE_PERSISTENT) return MPX_SUCCESS;
  __atomic_store_n(&w->wctl->stop, 1, __ATOMIC_RELEASE);
  const int64_t t0 = now_ms();
  int rc = MPX_SUCCESS;
  while (__atomic_load_n(&w->wctl->state, __ATOMIC_ACQUIRE) != ENG_STOPPED) {
    if (now_ms() - t0 > timeout_ms) { rc = MPX_ERR_TIMEOUT; break; }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  // the kernel has announced its exit; wait (bounded) until it has left the GPU
  while (rc == MPX_SUCCESS) {
    cudaError_t q = cudaStreamQuery(w->engine_stream);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) { rc = MPX_ERR_CUDA; break; }
    if (now_ms() - t0 > timeout_ms) { rc = MPX_ERR_TIMEOUT; break; }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  __atomic_store_n(&w->wctl->stop, 0, __ATOMIC_RELEASE);
  return rc;
}

extern "C" int mpx_world_progress(mpx_world_t w, mpx_cuda_stream_t stream) {
  if (!w) return MPX_ERR_ARG;
  if (w->cfg.engine_mode == MPX_ENGINE_PLAIN) return plain::progress(w->plain);
  if (w->cfg.engine_mode != MPX_ENGINE_DRAIN) return MPX_ERR_STATE;
  return launch_engine(w, (cudaStream_t)stream, 1);
}

// Failure recovery: mark the world failed (a running engine then releases
// every waiter with MPX_ERR_TIMEOUT and moves no more data) and write every
// completion word from the host, so no CUDA stream stays blocked on one.
extern "C" int mpx_world_abort(mpx_world_t w) {
  if (!w) return MPX_ERR_ARG;
  if (w->plain) return MPX_SUCCESS;
  __atomic_store_n(&w->wctl->error, MPX_ERR_TIMEOUT, __ATOMIC_RELEASE);
  __atomic_store_n(&w->wctl->failed, 1, __ATOMIC_RELEASE);
  const int S = w->cfg.max_streams;
  uint64_t* hv = nullptr;
  if (cudaHostAlloc((void**)&hv, (size_t)S * 8, cudaHostAllocDefault) != cudaSuccess) return MPX_ERR_NO_MEM;
  for (int g = 0; g < S; ++g) hv[g] = __atomic_load_n(&w->sctl[g].tail, __ATOMIC_ACQUIRE);
  cudaStream_t s;
  int rc = MPX_SUCCESS;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFreeHost(hv);
    return MPX_ERR_CUDA;
  }
  if (cudaMemcpyAsync(w->params.done, hv, (size_t)S * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    rc = MPX_ERR_CUDA;
  cudaStreamDestroy(s);
  cudaFreeHost(hv);
  return rc;
}

// Diagnostic: print the engine's per-stream cursors and task-ring state to
// stderr.  Reads device memory through a private non-blocking stream with a
// bounded wait, so it is safe while the engine runs.
extern "C" int mpx_world_debug_dump(mpx_world_t w) {
  if (!w || w->plain) return MPX_ERR_ARG;
  const int S = w->cfg.max_streams;
  std::vector<SState> ss(S);
  Shared sh;
  std::vector<uint64_t> door(S), done(S);
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return MPX_ERR_CUDA;
  cudaMemcpyAsync(ss.data(), w->params.ss, S * sizeof(SState), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&sh, w->params.sh, sizeof(Shared), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(door.data(), w->params.doorbell, S * 8, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(done.data(), w->params.done, S * 8, cudaMemcpyDeviceToHost, st);
  const int64_t t0 = now_ms();
  while (cudaStreamQuery(st) == cudaErrorNotReady && now_ms() - t0 < 2000)
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  const bool ok = cudaStreamQuery(st) == cudaSuccess;
  cudaStreamDestroy(st);
  if (!ok) return MPX_ERR_TIMEOUT;
  fprintf(stderr, "[mpx dump] state %d failed %d error %d tasks head %llu alloc %llu retire %llu round %llu"
          " cq head %llu tail %llu\n",
          w->wctl->state, w->wctl->failed, w->wctl->error, (unsigned long long)sh.task_head,
          (unsigned long long)sh.task_alloc, (unsigned long long)sh.task_retire,
          (unsigned long long)sh.round, (unsigned long long)sh.cq_head, (unsigned long long)sh.cq_tail);
  // the live tasks: how many are unfinished, and where their tiles stand
  const uint64_t cap = 1ull << w->tq_log2;
  if (sh.task_alloc > sh.task_retire && sh.task_alloc - sh.task_retire <= cap) {
    std::vector<Task> tk(cap);
    if (cudaMemcpy(tk.data(), w->params.tasks, cap * sizeof(Task), cudaMemcpyDeviceToHost) == cudaSuccess) {
      uint64_t open = 0, unclaimed = 0, ran = 0, shown = 0;
      for (uint64_t id = sh.task_retire; id < sh.task_alloc; ++id) {
        const Task& t = tk[id & (cap - 1)];
        if (t.type == 0) continue;
        ++open;
        const uint32_t nx = claim_next(t.claim), nt = claim_ntiles(t.claim);
        if (nx < nt) ++unclaimed;
        if (t.tiles_done >= t.ntiles) ++ran;
        if (shown++ < 8)
          fprintf(stderr,
                  "[mpx dump]   task %llu type %u action %u bytes %lld tile %lld ntiles %u done %u claim idp %u"
                  " nt %u next %u (tag %u) chunk %lld unit %u\n",
                  (unsigned long long)id, t.type, t.action, (long long)t.bytes, (long long)t.tile, t.ntiles,
                  t.tiles_done, claim_idp(t.claim), nt, nx, id_tag(id), (long long)t.chunk, t.unit);
      }
      fprintf(stderr, "[mpx dump]   open tasks %llu: tiles unclaimed %llu, all tiles counted done %llu\n",
              (unsigned long long)open, (unsigned long long)unclaimed, (unsigned long long)ran);
    }
  }
  for (int g = 0; g < S; ++g) {
    const StreamCtl& c = w->sctl[g];
    if (!c.flags && !c.tail) continue;
    const SState& x = ss[g];
    fprintf(stderr,
            "[mpx dump] g%d tail %llu retired %llu | ing %llu cur %llu pc %llu ret %llu sched %llu done %llu "
            "reached %llu door %llu dn %llu stall %lld flags %d err %d\n",
            g, (unsigned long long)c.tail, (unsigned long long)c.retired, (unsigned long long)x.ingested,
            (unsigned long long)x.cursor, (unsigned long long)x.pc, (unsigned long long)x.retire,
            (unsigned long long)x.sched, (unsigned long long)x.done, (unsigned long long)x.reached,
            (unsigned long long)door[g], (unsigned long long)done[g], (long long)x.stall_t0, x.flags, c.error);
    // the operations at the logical cursor and at the physical scan position
    const uint64_t at[2] = {x.cursor, x.pc};
    for (int k = 0; k < 2; ++k) {
      if (at[k] == 0 || at[k] > x.ingested) continue;
      DOp o;
      const size_t idx = ((size_t)g << w->slots_log2) + ((at[k] - 1) & ((1ull << w->slots_log2) - 1));
      if (cudaMemcpy(&o, w->params.ops + idx, sizeof(DOp), cudaMemcpyDeviceToHost) != cudaSuccess) break;
      fprintf(stderr,
              "[mpx dump]   %s seq %llu kind %u peer %d tag %d count %lld lstate %d lround %d pflags %#x "
              "partner %#llx n32 %d wscan %u pscan %u\n",
              k ? "pc" : "cursor", (unsigned long long)at[k], kw_kind(o.d.kw), o.d.peer, o.d.tag,
              (long long)o.d.count, o.lstate, o.lround, o.pflags, (unsigned long long)o.partner, o.d.n32,
              o.wscan, o.pscan);
    }
  }
  fflush(stderr);
  return MPX_SUCCESS;
}

extern "C" int mpx_world_get_error(mpx_world_t w, int* err) {
  if (!w || !err) return MPX_ERR_ARG;
  if (w->plain) { *err = plain::error(w->plain); return MPX_SUCCESS; }
  *err = __atomic_load_n(&w->wctl->error, __ATOMIC_ACQUIRE);
  return MPX_SUCCESS;
}

// Diagnostic: copy up to n tile-trace records (4 words each) into out and
// restart the trace; returns the number of records taken (0 without a trace).
extern "C" int64_t mpxi_world_trace(mpx_world_t w, uint64_t* out, int64_t n) {
  if (!w || w->plain || !w->params.trace || !out) return 0;
  uint64_t pos = 0;
  if (cudaMemcpy(&pos, w->params.trace_pos, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  const int64_t k = std::min<int64_t>({(int64_t)pos, w->params.trace_cap, n});
  if (k > 0 && cudaMemcpy(out, w->params.trace, (size_t)k * 32, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  const uint64_t zero = 0;
  if (cudaMemcpy(w->params.trace_pos, &zero, 8, cudaMemcpyHostToDevice) != cudaSuccess) return -1;
  return k;
}

extern "C" int mpx_world_get_counters(mpx_world_t w, int64_t* outv, int n) {
  if (!w || !outv || n < 0) return MPX_ERR_ARG;
  for (int i = 0; i < n && i < 27; ++i) {
    if (w->plain) outv[i] = i < 19 ? plain::counter(w->plain, i) : 0;
    else if (i < 8) outv[i] = (int64_t)__atomic_load_n(&w->wctl->counters[i], __ATOMIC_ACQUIRE);
    else if (i < 12) outv[i] = (int64_t)__atomic_load_n(&w->wctl->phase[i - 8], __ATOMIC_ACQUIRE);
    else if (i < 19) outv[i] = (int64_t)__atomic_load_n(&w->wctl->tick_ns[i - 12], __ATOMIC_ACQUIRE);
    else if (i < 26) outv[i] = (int64_t)__atomic_load_n(&w->wctl->sub_ns[i - 19], __ATOMIC_ACQUIRE);
    else outv[i] = (int64_t)__atomic_load_n(&w->wctl->sub_ns[7], __ATOMIC_ACQUIRE);
  }
  return MPX_SUCCESS;
}

extern "C" int mpx_world_free(mpx_world_t* pw) {
  if (!pw || !*pw) return MPX_ERR_ARG;
  mpx_world_s* w = *pw;
  {
    std::lock_guard<std::mutex> g(w->mu);
    for (auto* s : w->streams)
      if (s) return MPX_ERR_PENDING;
    if (w->live_comm_handles) return MPX_ERR_PENDING;
  }
  if (w->cfg.engine_mode == MPX_ENGINE_PERSISTENT) {
    if (mpx_world_stop(w, 10000) != MPX_SUCCESS) return MPX_ERR_TIMEOUT;
  }
  // every wait here is bounded: a kernel that does not finish leaves the
  // world allocated and reports MPX_ERR_TIMEOUT
  if (w->engine_stream) {
    const int64_t t0 = now_ms();
    for (;;) {
      cudaError_t q = cudaStreamQuery(w->engine_stream);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady) return MPX_ERR_CUDA;
      if (now_ms() - t0 > 10000) return MPX_ERR_TIMEOUT;
      std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
  }
  world_release(w);
  *pw = nullptr;
  return MPX_SUCCESS;
}

// ---------------------------------------------------------------------------
// streams
// ---------------------------------------------------------------------------
extern "C" int mpx_stream_create(mpx_world_t w, int rank, mpx_cuda_stream_t cs, unsigned flags,
                                 mpx_stream_t* out) {
  if (!w || !out) return MPX_ERR_ARG;
  if (rank < 0 || rank >= w->nranks) return MPX_ERR_RANK;
  if (flags & ~(unsigned)MPX_STREAM_EXCLUSIVE) return MPX_ERR_ARG;
  std::lock_guard<std::mutex> g(w->mu);
  int id = -1;
  for (int i = 0; i < w->cfg.max_streams; ++i)
    if (!w->streams[i]) { id = i; break; }
  if (id < 0) return MPX_ERR_NO_ENDPOINT;
  mpx_stream_s* s = new (std::nothrow) mpx_stream_s();
  if (!s) return MPX_ERR_NO_MEM;
  s->w = w;
  s->id = id;
  s->rank = rank;
  s->cs = (cudaStream_t)cs;
  s->flags = flags;
  s->ncomms = 0;
  if (w->plain) {
    if (plain::stream_create(w->plain, id, rank, (cudaStream_t)cs, (flags & MPX_STREAM_EXCLUSIVE) != 0) != MPX_SUCCESS) { delete s; return MPX_ERR_NO_MEM; }
  } else {
    StreamCtl* c = &w->sctl[id];
    // sequence numbers continue across incarnations of an endpoint so the
    // doorbell and completion words stay monotone
    s->next_seq = __atomic_load_n(&c->tail, __ATOMIC_ACQUIRE) + 1;
    s->wl_next = __atomic_load_n(&c->wl_retired, __ATOMIC_ACQUIRE);
    c->error = 0;
    c->rank = rank;
    __atomic_store_n(&c->flags, SF_ACTIVE | ((flags & MPX_STREAM_EXCLUSIVE) ? SF_EXCLUSIVE : 0),
                     __ATOMIC_RELEASE);
  }
  w->streams[id] = s;
  *out = s;
  return MPX_SUCCESS;
}

static int64_t stream_pending(mpx_stream_s* s) {
  if (s->w->plain) return plain::stream_pending(s->w->plain, s->id);
  StreamCtl* c = &s->w->sctl[s->id];
  return (int64_t)(__atomic_load_n(&c->tail, __ATOMIC_ACQUIRE) - __atomic_load_n(&c->retired, __ATOMIC_ACQUIRE));
}

extern "C" int mpx_stream_free(mpx_stream_t* ps) {
  if (!ps || !*ps) return MPX_ERR_ARG;
  mpx_stream_s* s = *ps;
  mpx_world_s* w = s->w;
  std::lock_guard<std::mutex> g(w->mu);
  if (s->step) return MPX_ERR_STATE;  // free the recorded step first
  if (s->ncomms > 0) return MPX_ERR_PENDING;
  if (stream_pending(s) != 0) return MPX_ERR_PENDING;
  if (w->plain) plain::stream_free(w->plain, s->id);
  else __atomic_store_n(&w->sctl[s->id].flags, 0, __ATOMIC_RELEASE);
  w->streams[s->id] = nullptr;
  if (s->owns_cs) cudaStreamDestroy(s->cs);  // queued work finishes first
  delete s;
  *ps = nullptr;
  return MPX_SUCCESS;
}

extern "C" int mpx_stream_create_info(mpx_world_t w, int rank, mpx_info_t info, mpx_stream_t* out) {
  if (!w || !out) return MPX_ERR_ARG;
  if (!info) {
    // MPI_INFO_NULL: an MPIX stream with a queue of its own
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MPX_ERR_CUDA;
    int rc = mpx_stream_create(w, rank, (mpx_cuda_stream_t)cs, MPX_STREAM_DEFAULT, out);
    if (rc) {
      cudaStreamDestroy(cs);
      return rc;
    }
    (*out)->owns_cs = true;
    return MPX_SUCCESS;
  }
  char type[64];
  int has_type = 0, has_value = 0, has_excl = 0;
  if (mpx_info_get(info, "type", type, (int)sizeof(type), &has_type)) return MPX_ERR_ARG;
  mpx_cuda_stream_t cs = nullptr;
  if (mpx_info_get_hex(info, "value", &cs, (int)sizeof(cs), &has_value)) return MPX_ERR_ARG;
  char excl[8];
  if (mpx_info_get(info, "mpx_exclusive", excl, (int)sizeof(excl), &has_excl)) return MPX_ERR_ARG;
  unsigned flags = MPX_STREAM_DEFAULT;
  if (has_excl) {
    if (strcmp(excl, "true") == 0) flags = MPX_STREAM_EXCLUSIVE;
    else if (strcmp(excl, "false") != 0) return MPX_ERR_ARG;
  }
  // only a CUDA stream can back an MPIX stream here, and it must be given
  if (!has_type || strcmp(type, "cudaStream_t") != 0 || !has_value) return MPX_ERR_ARG;
  return mpx_stream_create(w, rank, cs, flags, out);
}

extern "C" int mpx_stream_get_cuda_stream(mpx_stream_t s, mpx_cuda_stream_t* cs) {
  if (!s || !cs) return MPX_ERR_ARG;
  *cs = (mpx_cuda_stream_t)s->cs;
  return MPX_SUCCESS;
}

extern "C" int mpx_stream_get_id(mpx_stream_t s, int* id) {
  if (!s || !id) return MPX_ERR_ARG;
  *id = s->id;
  return MPX_SUCCESS;
}

extern "C" int mpx_stream_get_error(mpx_stream_t s, int* err) {
  if (!s || !err) return MPX_ERR_ARG;
  if (s->w->plain) { *err = plain::stream_error(s->w->plain, s->id); return MPX_SUCCESS; }
  *err = __atomic_load_n(&s->w->sctl[s->id].error, __ATOMIC_ACQUIRE);
  return MPX_SUCCESS;
}

extern "C" int mpx_stream_pending(mpx_stream_t s, int64_t* pending) {
  if (!s || !pending) return MPX_ERR_ARG;
  *pending = stream_pending(s);
  return MPX_SUCCESS;
}

// ---------------------------------------------------------------------------
// communicators
// ---------------------------------------------------------------------------
extern "C" int mpx_stream_comm_create(mpx_world_t w, int nranks, const mpx_stream_t streams[],
                                      mpx_comm_t comms_out[]) {
  if (!w || !streams || !comms_out) return MPX_ERR_ARG;
  if (nranks != w->nranks) return MPX_ERR_ARG;
  for (int r = 0; r < nranks; ++r) {
    if (!streams[r]) return MPX_ERR_COMM;  // MPIX_STREAM_NULL members are not supported
    if (streams[r]->w != w || streams[r]->rank != r) return MPX_ERR_ARG;
  }
  std::lock_guard<std::mutex> g(w->mu);
  if (w->comms_used >= w->cfg.max_comms) return MPX_ERR_NO_MEM;
  CommShared* sh = new (std::nothrow) CommShared();
  if (!sh) return MPX_ERR_NO_MEM;
  sh->id = w->comms_used++;
  sh->reduce_mode = w->cfg.reduce_mode;
  sh->handles.store(nranks);
  std::vector<mpx_comm_s*> made;
  for (int r = 0; r < nranks; ++r) {
    mpx_comm_s* c = new (std::nothrow) mpx_comm_s();
    if (!c) {
      for (auto* m : made) delete m;
      delete sh;
      return MPX_ERR_NO_MEM;
    }
    c->w = w;
    c->shared = sh;
    c->rank = r;
    c->size = nranks;
    c->stream = streams[r];
    made.push_back(c);
  }
  if (w->plain) plain::comm_create(w->plain, sh->id);
  for (int r = 0; r < nranks; ++r) {
    streams[r]->ncomms++;
    comms_out[r] = made[r];
  }
  w->live_comm_handles += nranks;
  return MPX_SUCCESS;
}

extern "C" int mpx_stream_comm_create_multiple(mpx_world_t w, int nranks, const int counts[],
                                               const mpx_stream_t streams[],
                                               mpx_comm_t comms_out[]) {
  if (!w || !counts || !streams || !comms_out) return MPX_ERR_ARG;
  if (nranks != w->nranks) return MPX_ERR_ARG;
  if (w->plain) return MPX_ERR_UNSUPPORTED;
  std::vector<int> off((size_t)nranks + 1, 0);
  int most = 0;
  for (int r = 0; r < nranks; ++r) {
    if (counts[r] < 1 || counts[r] > 0x7FFE) return MPX_ERR_ARG;
    off[(size_t)r + 1] = off[(size_t)r] + counts[r];
    if (off[(size_t)r + 1] > 0xFFFF) return MPX_ERR_ARG;  // members fit the 16-bit rank field
    most = std::max(most, counts[r]);
  }
  for (int r = 0; r < nranks; ++r) {
    for (int i = 0; i < counts[r]; ++i) {
      mpx_stream_s* st = streams[off[(size_t)r] + i];
      if (!st) return MPX_ERR_COMM;
      if (st->w != w || st->rank != r) return MPX_ERR_ARG;
      for (int k = 0; k < i; ++k)
        if (streams[off[(size_t)r] + k] == st) return MPX_ERR_ARG;
    }
  }
  // every member is a matching domain: ceil(M / nranks) consecutive slots
  const int slots = (off[(size_t)nranks] + nranks - 1) / nranks;
  std::lock_guard<std::mutex> g(w->mu);
  if (w->comms_used + slots > w->cfg.max_comms) return MPX_ERR_NO_MEM;
  CommShared* sh = new (std::nothrow) CommShared();
  if (!sh) return MPX_ERR_NO_MEM;
  sh->id = w->comms_used;
  sh->reduce_mode = w->cfg.reduce_mode;
  sh->handles.store(nranks);
  sh->mux_off = off;
  sh->mux_max = most;
  std::vector<mpx_comm_s*> made;
  for (int r = 0; r < nranks; ++r) {
    mpx_comm_s* c = new (std::nothrow) mpx_comm_s();
    if (!c) {
      for (auto* m : made) delete m;
      delete sh;
      return MPX_ERR_NO_MEM;
    }
    c->w = w;
    c->shared = sh;
    c->rank = r;
    c->size = nranks;
    c->local.assign(streams + off[(size_t)r], streams + off[(size_t)r + 1]);
    c->stream = c->local[0];
    made.push_back(c);
  }
  w->comms_used += slots;
  for (int r = 0; r < nranks; ++r) {
    for (mpx_stream_s* st : made[(size_t)r]->local) st->ncomms++;
    comms_out[r] = made[(size_t)r];
  }
  w->live_comm_handles += nranks;
  return MPX_SUCCESS;
}

extern "C" int mpx_comm_free(mpx_comm_t* pc) {
  if (!pc || !*pc) return MPX_ERR_ARG;
  mpx_comm_s* c = *pc;
  mpx_world_s* w = c->w;
  std::lock_guard<std::mutex> g(w->mu);
  if (c->shared->mux()) {
    for (mpx_stream_s* st : c->local) st->ncomms--;
  } else {
    c->stream->ncomms--;
  }
  w->live_comm_handles--;
  if (c->shared->handles.fetch_sub(1) == 1) delete c->shared;
  delete c;
  *pc = nullptr;
  return MPX_SUCCESS;
}

// For the persistent requests (mpx_persist.cpp): whether a communicator's
// world runs the plain path, which has no nonblocking collectives.
extern "C" int mpxi_comm_is_plain(mpx_comm_t c) { return c && c->w && c->w->plain ? 1 : 0; }

extern "C" int mpx_comm_rank(mpx_comm_t c, int* rank) {
  if (!c || !rank) return MPX_ERR_ARG;
  *rank = c->rank;
  return MPX_SUCCESS;
}

extern "C" int mpx_comm_size(mpx_comm_t c, int* size) {
  if (!c || !size) return MPX_ERR_ARG;
  *size = c->size;
  return MPX_SUCCESS;
}

extern "C" int mpx_comm_set_reduce_mode(mpx_comm_t c, int mode) {
  if (!c || (mode != MPX_REDUCE_FIXED && mode != MPX_REDUCE_TREE)) return MPX_ERR_ARG;
  c->shared->reduce_mode = mode;
  return MPX_SUCCESS;
}

// ---------------------------------------------------------------------------
// datatypes
// ---------------------------------------------------------------------------
extern "C" int mpx_type_vector(int count, int blocklength, int stride, mpx_datatype_t oldtype,
                               mpx_datatype_t* newtype) {
  if (!newtype || count < 1 || blocklength < 1 || stride < blocklength) return MPX_ERR_ARG;
  if (oldtype < 0 || oldtype > MPX_DOUBLE) return MPX_ERR_TYPE;
  // one instance's extent in bytes stays below 2^48, so that byte counts of
  // whole messages can be checked against int64 with one division
  const int64_t ext = ((int64_t)count - 1) * stride + blocklength;  // < 2^62: no overflow
  if (ext > (kMaxTypeExtent >> 3)) return MPX_ERR_ARG;
  std::lock_guard<std::mutex> g(g_types_mu);
  int id;
  if (!g_types_free.empty()) {
    id = g_types_free.back();
    g_types_free.pop_back();
  } else {
    if (g_types_next >= kMaxTypes) return MPX_ERR_NO_MEM;
    id = g_types_next++;
  }
  g_types[id].base = oldtype;
  g_types[id].vcount = count;
  g_types[id].blocklen = blocklength;
  g_types[id].stride = stride;
  __atomic_store_n(&g_types[id].alive, 1, __ATOMIC_RELEASE);
  *newtype = id;
  return MPX_SUCCESS;
}

extern "C" int mpx_type_free(mpx_datatype_t* t) {
  if (!t) return MPX_ERR_ARG;
  if (*t < kFirstDerived || *t >= kMaxTypes) return MPX_ERR_TYPE;
  std::lock_guard<std::mutex> g(g_types_mu);
  if (!g_types[*t].alive) return MPX_ERR_TYPE;
  __atomic_store_n(&g_types[*t].alive, 0, __ATOMIC_RELEASE);
  g_types_free.push_back(*t);
  *t = -1;
  return MPX_SUCCESS;
}

extern "C" int mpx_type_size(mpx_datatype_t t, int64_t* size) {
  const TypeRec* r = type_get(t);
  if (!r || !size) return r ? MPX_ERR_ARG : MPX_ERR_TYPE;
  *size = base_size((uint32_t)r->base) * r->vcount * r->blocklen;
  return MPX_SUCCESS;
}

extern "C" int mpx_type_extent(mpx_datatype_t t, int64_t* extent) {
  const TypeRec* r = type_get(t);
  if (!r || !extent) return r ? MPX_ERR_ARG : MPX_ERR_TYPE;
  *extent = base_size((uint32_t)r->base) * ((int64_t)(r->vcount - 1) * r->stride + r->blocklen);
  return MPX_SUCCESS;
}

// Layout parameters of a datatype, for library code outside this file.
extern "C" int mpxi_type_desc(int32_t t, int32_t* base, int32_t* vcount, int32_t* blocklen,
                              int32_t* stride) {
  const TypeRec* r = type_get(t);
  if (!r) return MPX_ERR_TYPE;
  *base = r->base;
  *vcount = r->vcount;
  *blocklen = r->blocklen;
  *stride = r->stride;
  return MPX_SUCCESS;
}

extern "C" int mpx_get_count(const mpx_status_t* st, mpx_datatype_t t, int64_t* count) {
  if (!st || !count) return MPX_ERR_ARG;
  int64_t sz;
  int rc = mpx_type_size(t, &sz);
  if (rc) return rc;
  *count = (sz > 0 && st->bytes % sz == 0) ? st->bytes / sz : (int64_t)MPX_UNDEFINED;
  return MPX_SUCCESS;
}

extern "C" int mpx_version(void) { return 100; }

extern "C" int mpx_cuda_stream_create(mpx_cuda_stream_t* stream) {
  if (!stream) return MPX_ERR_ARG;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return MPX_ERR_CUDA;
  *stream = (mpx_cuda_stream_t)s;
  return MPX_SUCCESS;
}

extern "C" int mpx_cuda_stream_destroy(mpx_cuda_stream_t stream) {
  return cudaStreamDestroy((cudaStream_t)stream) == cudaSuccess ? MPX_SUCCESS : MPX_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// enqueue
// ---------------------------------------------------------------------------
// Make descriptors up to `seq` visible to the engine (release the ring tail),
// have the engine running, and ring the stream-order doorbell.
static int announce(mpx_stream_s* s, uint64_t seq) {
  mpx_world_s* w = s->w;
  s->owed = 0;
  __atomic_store_n(&w->sctl[s->id].tail, seq, __ATOMIC_RELEASE);
  // launch the engine (persistent mode) before a later wait can stall a
  // hardware queue the engine's stream might share
  int erc = ensure_engine(w);
  if (erc) return erc;
  if (!(s->flags & MPX_STREAM_EXCLUSIVE)) {
    CUdeviceptr db = (CUdeviceptr)(w->params.doorbell + s->id);
    if (g_write64((CUstream)s->cs, db, seq, 0) != CUDA_SUCCESS) return MPX_ERR_CUDA;
  }
  return MPX_SUCCESS;
}

static int flush_owed(mpx_stream_s* s) { return s->owed ? announce(s, s->owed) : MPX_SUCCESS; }

// defer: a batch will publish the next op on this stream right after this
// one, with nothing enqueued on the CUDA stream in between; the descriptor is
// written but the tail release and the doorbell are left to that op (or to
// the batch's flush), so a run of operations costs one of each.
static int publish(mpx_stream_s* s, Desc& d, bool blocking, uint64_t* seq_out,
                   bool defer = false) {
  mpx_world_s* w = s->w;
  StreamCtl* c = &w->sctl[s->id];
  if (__atomic_load_n(&w->wctl->failed, __ATOMIC_ACQUIRE)) return MPX_ERR_STATE;
  if (s->step) return MPX_ERR_STATE;  // a recorded step publishes on this stream
  const uint64_t seq = s->next_seq;
  const uint64_t slots = 1ull << w->slots_log2;
  // read the engine-written retirement word only when the cached one says full
  if (seq - s->retired_seen > slots) s->retired_seen = __atomic_load_n(&c->retired, __ATOMIC_ACQUIRE);
  if (seq - s->retired_seen > slots) {
    // the engine can only retire what it can see
    int rc = flush_owed(s);
    if (rc) return rc;
    if (w->cfg.engine_mode != MPX_ENGINE_PERSISTENT) return MPX_ERR_AGAIN;
    rc = ensure_engine(w);
    if (rc) return rc;
    const int64_t t0 = now_ms();
    while (seq - __atomic_load_n(&c->retired, __ATOMIC_ACQUIRE) > slots) {
      if (now_ms() - t0 > 1000) return MPX_ERR_AGAIN;
      if (__atomic_load_n(&w->wctl->state, __ATOMIC_ACQUIRE) != ENG_RUNNING) ensure_engine(w);
      std::this_thread::yield();
    }
  }
  MPX_TRACE("publish: stream %d seq %llu kind %u blocking %d", s->id, (unsigned long long)seq,
            kw_kind(d.kw), (int)blocking);
  Desc* slot = &w->rings[((size_t)s->id << w->slots_log2) + ((seq - 1) & (slots - 1))];
  memcpy(slot, &d, sizeof(Desc));
  s->next_seq = seq + 1;
  if (seq_out) *seq_out = seq;  // the operation exists from here on
  if (defer && !blocking) {
    s->owed = seq;
    return MPX_SUCCESS;
  }
  int rc = announce(s, seq);
  if (rc) return rc;
  if (blocking) {
    CUdeviceptr dn = (CUdeviceptr)(w->params.done + s->id);
    if (g_wait64((CUstream)s->cs, dn, seq, CU_STREAM_WAIT_VALUE_GEQ) != CUDA_SUCCESS) return MPX_ERR_CUDA;
  }
  MPX_TRACE("publish: memops queued");
  return MPX_SUCCESS;
}

static int fill_p2p(Desc& d, uint32_t kind, const void* buf, int64_t count, mpx_datatype_t dt,
                    int peer, int tag, mpx_comm_s* c, bool is_recv) {
  if (!c || !c->stream || c->shared->mux()) return MPX_ERR_COMM;
  if (count < 0) return MPX_ERR_ARG;
  const TypeRec* t = type_get(dt);
  if (!t) return MPX_ERR_TYPE;
  if (!span_ok(t, count)) return MPX_ERR_ARG;
  if (is_recv) {
    if (peer != MPX_ANY_SOURCE && (peer < 0 || peer >= c->size)) return MPX_ERR_RANK;
    if (tag != MPX_ANY_TAG && (tag < 0 || tag > MPX_TAG_UB)) return MPX_ERR_TAG;
  } else {
    if (peer < 0 || peer >= c->size) return MPX_ERR_RANK;
    if (tag < 0 || tag > MPX_TAG_UB) return MPX_ERR_TAG;
  }
  if (count > 0 && !buf) return MPX_ERR_ARG;
  memset(&d, 0, sizeof(d));
  d.kw = make_kw(kind, (uint32_t)t->base, 0);
  d.comm = (uint16_t)c->shared->id;
  d.rank = (uint16_t)c->rank;
  d.peer = peer;
  d.tag = tag;
  d.buf = (uint64_t)buf;
  d.count = count;
  d.vcount = t->vcount;
  d.blocklen = t->blocklen;
  d.stride = t->stride;
  if (!is_recv) d.n32 = (int32_t)c->rank;  // sender key (rank, local index 0)
  return MPX_SUCCESS;
}

// A point-to-point call on a multiplex stream communicator (§3.5).  The
// engine matches per member: a send's domain is the destination member
// (d.peer), a receive's its own member (d.rank).  A send carries its sender
// key (local index << 16 | rank) in d.n32; a receive carries its source
// pattern in d.peer: MPX_ANY_SOURCE when both rank and index are wildcards,
// else (index or 0x7FFF) << 16 | (rank or 0xFFFF).  Returns the local stream
// the call is enqueued on through *st.
static int fill_mux(Desc& d, uint32_t kind, const void* buf, int64_t count, mpx_datatype_t dt,
                    int peer, int tag, mpx_comm_s* c, int src_idx, int dst_idx,
                    mpx_stream_s** st) {
  if (!c || !c->shared->mux()) return MPX_ERR_COMM;
  const CommShared* sh = c->shared;
  if (count < 0) return MPX_ERR_ARG;
  const TypeRec* t = type_get(dt);
  if (!t) return MPX_ERR_TYPE;
  if (!span_ok(t, count)) return MPX_ERR_ARG;
  auto nloc = [&](int r) { return sh->mux_off[(size_t)r + 1] - sh->mux_off[(size_t)r]; };
  const bool is_recv = kind == K_RECV || kind == K_IRECV;
  int own;
  if (is_recv) {
    if (peer != MPX_ANY_SOURCE && (peer < 0 || peer >= c->size)) return MPX_ERR_RANK;
    if (tag != MPX_ANY_TAG && (tag < 0 || tag > MPX_TAG_UB)) return MPX_ERR_TAG;
    if (dst_idx < 0 || dst_idx >= nloc(c->rank)) return MPX_ERR_ARG;
    if (src_idx != MPX_ANY_INDEX &&
        (src_idx < 0 || src_idx >= (peer == MPX_ANY_SOURCE ? sh->mux_max : nloc(peer))))
      return MPX_ERR_ARG;
    own = dst_idx;
  } else {
    if (peer < 0 || peer >= c->size) return MPX_ERR_RANK;
    if (tag < 0 || tag > MPX_TAG_UB) return MPX_ERR_TAG;
    if (src_idx < 0 || src_idx >= nloc(c->rank)) return MPX_ERR_ARG;
    if (dst_idx < 0 || dst_idx >= nloc(peer)) return MPX_ERR_ARG;
    own = src_idx;
  }
  if (count > 0 && !buf) return MPX_ERR_ARG;
  memset(&d, 0, sizeof(d));
  d.kw = make_kw(kind, (uint32_t)t->base, 0);
  d.comm = (uint16_t)sh->id;
  d.rank = (uint16_t)(sh->mux_off[(size_t)c->rank] + own);
  if (is_recv) {
    if (peer == MPX_ANY_SOURCE && src_idx == MPX_ANY_INDEX) {
      d.peer = MPX_ANY_SOURCE;
    } else {
      const uint32_t pi = src_idx == MPX_ANY_INDEX ? 0x7FFFu : (uint32_t)src_idx;
      const uint32_t pr = peer == MPX_ANY_SOURCE ? 0xFFFFu : (uint32_t)peer;
      d.peer = (int32_t)((pi << 16) | pr);
    }
  } else {
    d.peer = sh->mux_off[(size_t)peer] + dst_idx;
    d.n32 = (int32_t)(((uint32_t)src_idx << 16) | (uint32_t)c->rank);
  }
  d.tag = tag;
  d.buf = (uint64_t)buf;
  d.count = count;
  d.vcount = t->vcount;
  d.blocklen = t->blocklen;
  d.stride = t->stride;
  *st = c->local[(size_t)own];
  return MPX_SUCCESS;
}

extern "C" int mpx_send_enqueue(const void* buf, int64_t count, mpx_datatype_t dt, int dest,
                                int tag, mpx_comm_t c) {
  if (c && c->w->plain) return plain::p2p(c->w->plain, K_SEND, buf, count, dt, dest, tag, c->shared->id, c->rank, c->stream->id, nullptr, nullptr);
  Desc d;
  int rc = fill_p2p(d, K_SEND, buf, count, dt, dest, tag, c, false);
  if (rc) return rc;
  return publish(c->stream, d, true, nullptr);
}

extern "C" int mpx_recv_enqueue(void* buf, int64_t count, mpx_datatype_t dt, int source, int tag,
                                mpx_comm_t c, mpx_status_t* status) {
  if (c && c->w->plain) return plain::p2p(c->w->plain, K_RECV, buf, count, dt, source, tag, c->shared->id, c->rank, c->stream->id, status, nullptr);
  Desc d;
  int rc = fill_p2p(d, K_RECV, buf, count, dt, source, tag, c, true);
  if (rc) return rc;
  d.status = (uint64_t)status;
  return publish(c->stream, d, true, nullptr);
}

static int nb_p2p(uint32_t kind, const void* buf, int64_t count, mpx_datatype_t dt, int peer,
                  int tag, mpx_comm_t c, mpx_request_t* req, bool defer_db) {
  if (!req) return MPX_ERR_ARG;
  if (c && c->w->plain)
    return plain::p2p(c->w->plain, kind, buf, count, dt, peer, tag, c->shared->id, c->rank,
                      c->stream->id, nullptr, req);
  Desc d;
  int rc = fill_p2p(d, kind, buf, count, dt, peer, tag, c, kind == K_IRECV);
  if (rc) return rc;
  uint64_t seq = 0;
  rc = publish(c->stream, d, false, &seq, defer_db);
  if (seq) *req = make_request(c->stream, seq);
  return rc;
}

extern "C" int mpx_isend_enqueue(const void* buf, int64_t count, mpx_datatype_t dt, int dest,
                                 int tag, mpx_comm_t c, mpx_request_t* req) {
  return nb_p2p(K_ISEND, buf, count, dt, dest, tag, c, req, false);
}

extern "C" int mpx_irecv_enqueue(void* buf, int64_t count, mpx_datatype_t dt, int source, int tag,
                                 mpx_comm_t c, mpx_request_t* req) {
  return nb_p2p(K_IRECV, buf, count, dt, source, tag, c, req, false);
}

extern "C" int mpx_stream_send_enqueue(const void* buf, int64_t count, mpx_datatype_t dt, int dest,
                                       int tag, mpx_comm_t c, int src_idx, int dst_idx) {
  Desc d;
  mpx_stream_s* st = nullptr;
  int rc = fill_mux(d, K_SEND, buf, count, dt, dest, tag, c, src_idx, dst_idx, &st);
  if (rc) return rc;
  return publish(st, d, true, nullptr);
}

extern "C" int mpx_stream_recv_enqueue(void* buf, int64_t count, mpx_datatype_t dt, int source,
                                       int tag, mpx_comm_t c, int src_idx, int dst_idx,
                                       mpx_status_t* status) {
  Desc d;
  mpx_stream_s* st = nullptr;
  int rc = fill_mux(d, K_RECV, buf, count, dt, source, tag, c, src_idx, dst_idx, &st);
  if (rc) return rc;
  d.status = (uint64_t)status;
  return publish(st, d, true, nullptr);
}

static int mux_nb(uint32_t kind, const void* buf, int64_t count, mpx_datatype_t dt, int peer,
                  int tag, mpx_comm_t c, int src_idx, int dst_idx, mpx_request_t* req) {
  if (!req) return MPX_ERR_ARG;
  Desc d;
  mpx_stream_s* st = nullptr;
  int rc = fill_mux(d, kind, buf, count, dt, peer, tag, c, src_idx, dst_idx, &st);
  if (rc) return rc;
  uint64_t seq = 0;
  rc = publish(st, d, false, &seq);
  if (seq) *req = make_request(st, seq);
  return rc;
}

extern "C" int mpx_stream_isend_enqueue(const void* buf, int64_t count, mpx_datatype_t dt, int dest,
                                        int tag, mpx_comm_t c, int src_idx, int dst_idx,
                                        mpx_request_t* req) {
  return mux_nb(K_ISEND, buf, count, dt, dest, tag, c, src_idx, dst_idx, req);
}

extern "C" int mpx_stream_irecv_enqueue(void* buf, int64_t count, mpx_datatype_t dt, int source,
                                        int tag, mpx_comm_t c, int src_idx, int dst_idx,
                                        mpx_request_t* req) {
  return mux_nb(K_IRECV, buf, count, dt, source, tag, c, src_idx, dst_idx, req);
}

static mpx_stream_s* request_stream(mpx_request_t r) {
  if (r < 0) return nullptr;
  const int widx = (int)(((uint64_t)r >> 56) & 0x7f);
  const int id = (int)(((uint64_t)r >> 40) & 0xffff);
  mpx_world_s* w = g_world_table[widx];
  if (!w || id >= w->cfg.max_streams) return nullptr;
  return w->streams[id];
}

extern "C" int mpxi_persist_active(mpx_request_t h, mpx_request_t* active);
extern "C" void mpxi_persist_complete(mpx_request_t h);

static int wait_impl(int n, mpx_request_t* reqs, mpx_status_t* statuses, bool single);

// A persistent request (mpx_*_init, values <= -2) stands for the instance its
// last start enqueued, or for nothing when inactive (a wait on it then has the
// empty status).  The wait consumes the instance and leaves the persistent
// handle valid and inactive.
static int wait_common(int n, mpx_request_t* reqs, mpx_status_t* statuses, bool single) {
  bool persistent = false;
  for (int i = 0; i < n && !persistent; ++i) persistent = reqs[i] <= -2;
  if (!persistent) return wait_impl(n, reqs, statuses, single);
  std::vector<mpx_request_t> eff(reqs, reqs + n);
  for (int i = 0; i < n; ++i)
    if (reqs[i] <= -2 && mpxi_persist_active(reqs[i], &eff[i]) != MPX_SUCCESS) return MPX_ERR_REQUEST;
  const int rc = wait_impl(n, eff.data(), statuses, single);
  if (rc != MPX_SUCCESS) return rc;
  for (int i = 0; i < n; ++i) {
    if (reqs[i] <= -2) mpxi_persist_complete(reqs[i]);
    else reqs[i] = MPX_REQUEST_NULL;
  }
  return MPX_SUCCESS;
}

static int wait_impl(int n, mpx_request_t* reqs, mpx_status_t* statuses, bool single) {
  mpx_world_s* w = nullptr;
  mpx_stream_s* s = nullptr;
  int live = 0;
  for (int i = 0; i < n; ++i) {
    if (reqs[i] == MPX_REQUEST_NULL) continue;
    if (reqs[i] < 0) return MPX_ERR_REQUEST;
    mpx_stream_s* si = request_stream(reqs[i]);
    if (!si) return MPX_ERR_REQUEST;
    w = si->w;
    if (s && si != s) return MPX_ERR_STREAM;  // §3.4: one local stream per waitall
    s = si;
    const uint64_t seq = (uint64_t)reqs[i] & ((1ull << 40) - 1);
    // the plain path numbers its own operations and validates them itself
    if (!w->plain && (seq == 0 || seq >= s->next_seq)) return MPX_ERR_REQUEST;
    ++live;
  }
  (void)live;
  if (!s) return MPX_SUCCESS;  // every request is null: nothing to wait for
  if (w->plain) {
    int rc = plain::wait(w->plain, s->id, n, reqs, statuses);
    if (rc == MPX_SUCCESS)
      for (int i = 0; i < n; ++i) reqs[i] = MPX_REQUEST_NULL;
    return rc;
  }
  Desc d;
  memset(&d, 0, sizeof(d));
  d.status = (uint64_t)statuses;
  if (single) {
    d.kw = make_kw(K_WAIT, 0, 0);
    d.aux = (uint64_t)reqs[0] & ((1ull << 40) - 1);
  } else {
    const uint64_t wl_slots = 1ull << w->wl_log2;
    StreamCtl* c = &w->sctl[s->id];
    if (s->wl_next + (uint64_t)n - __atomic_load_n(&c->wl_retired, __ATOMIC_ACQUIRE) > wl_slots)
      return MPX_ERR_AGAIN;
    // statuses are positional: a null request stays in the list as seq 0,
    // which the engine treats as complete with an empty status
    int64_t* wl = w->waitlists + ((size_t)s->id << w->wl_log2);
    uint64_t k = s->wl_next;
    for (int i = 0; i < n; ++i) {
      wl[k & (wl_slots - 1)] =
          reqs[i] == MPX_REQUEST_NULL ? 0 : (int64_t)((uint64_t)reqs[i] & ((1ull << 40) - 1));
      ++k;
    }
    d.kw = make_kw(K_WAITALL, 0, 0);
    d.aux = s->wl_next;
    d.n32 = n;
    s->wl_next = k;
  }
  int rc = publish(s, d, true, nullptr);
  if (rc == MPX_SUCCESS)
    for (int i = 0; i < n; ++i) reqs[i] = MPX_REQUEST_NULL;
  return rc;
}

extern "C" int mpx_wait_enqueue(mpx_request_t* req, mpx_status_t* status) {
  if (!req) return MPX_ERR_ARG;
  return wait_common(1, req, status, true);
}

extern "C" int mpx_waitall_enqueue(int n, mpx_request_t reqs[], mpx_status_t statuses[]) {
  if (n < 0 || (n > 0 && !reqs)) return MPX_ERR_ARG;
  return wait_common(n, reqs, statuses, false);
}

// Descriptor of a collective call (allreduce, bcast, reduce, allgather):
// buf = input, aux = output, peer = root.
// A collective's element count, times the element size and the number of
// ranks (an allgather's receive buffer), stays within kMaxSpan bytes.
static bool coll_count_ok(int64_t count, mpx_comm_t c) {
  return count >= 0 && count <= kMaxSpan / (8 * (int64_t)(c->size > 0 ? c->size : 1));
}

static void fill_collective(Desc& d, uint32_t kind, mpx_datatype_t dt, mpx_comm_t c,
                            const void* in, void* out, int64_t count, int root) {
  memset(&d, 0, sizeof(d));
  d.kw = make_kw(kind, (uint32_t)dt, (uint32_t)c->shared->reduce_mode);
  d.comm = (uint16_t)c->shared->id;
  d.rank = (uint16_t)c->rank;
  d.peer = root;
  d.buf = (uint64_t)in;
  d.aux = (uint64_t)out;
  d.count = count;
  d.vcount = 1;
  d.blocklen = 1;
  d.stride = 1;
}

// Blocking collectives (req == nullptr) stop their stream until complete; a
// nonblocking one (MPI_I*) returns a request at once and carries the
// nonblocking bit in its kind word, so it never forms an instance with a
// blocking call of another rank (MPI: they do not match).
static int publish_collective(mpx_comm_t c, Desc& d, mpx_request_t* req) {
  if (!req) return publish(c->stream, d, true, nullptr);
  d.kw |= kKwNonblocking;
  uint64_t seq = 0;
  const int rc = publish(c->stream, d, false, &seq);
  if (seq) *req = make_request(c->stream, seq);
  return rc;
}

static int bcast_common(void* buf, int64_t count, mpx_datatype_t dt, int root, mpx_comm_t c,
                        mpx_request_t* req) {
  if (!c || !c->stream || c->shared->mux()) return MPX_ERR_COMM;
  if (dt < 0 || dt > MPX_DOUBLE) return MPX_ERR_TYPE;
  if (root < 0 || root >= c->size) return MPX_ERR_RANK;
  if (!coll_count_ok(count, c)) return MPX_ERR_ARG;
  if (count < 0 || (count > 0 && !buf)) return MPX_ERR_ARG;
  if (c->w->plain) return MPX_ERR_UNSUPPORTED;
  Desc d;
  fill_collective(d, K_BCAST, dt, c, buf, buf, count, root);
  return publish_collective(c, d, req);
}

static int reduce_common(const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t dt,
                         int op, int root, mpx_comm_t c, mpx_request_t* req) {
  if (!c || !c->stream || c->shared->mux()) return MPX_ERR_COMM;
  if (op != MPX_SUM) return MPX_ERR_ARG;
  if (dt < 0 || dt > MPX_DOUBLE) return MPX_ERR_TYPE;
  if (root < 0 || root >= c->size) return MPX_ERR_RANK;
  const bool at_root = c->rank == root;
  if (sendbuf == MPX_IN_PLACE) {
    if (!at_root) return MPX_ERR_ARG;
    sendbuf = recvbuf;
  }
  if (!coll_count_ok(count, c)) return MPX_ERR_ARG;
  if (count < 0 || (count > 0 && (!sendbuf || (at_root && !recvbuf)))) return MPX_ERR_ARG;
  if (c->w->plain) return MPX_ERR_UNSUPPORTED;
  Desc d;
  fill_collective(d, K_REDUCE, dt, c, sendbuf, at_root ? recvbuf : nullptr, count, root);
  return publish_collective(c, d, req);
}

static int allgather_common(const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t dt,
                            mpx_comm_t c, mpx_request_t* req) {
  if (!c || !c->stream || c->shared->mux()) return MPX_ERR_COMM;
  if (dt < 0 || dt > MPX_DOUBLE) return MPX_ERR_TYPE;
  if (sendbuf == MPX_IN_PLACE) sendbuf = recvbuf;  // the rank's block is already in place
  if (!coll_count_ok(count, c)) return MPX_ERR_ARG;
  if (count < 0 || (count > 0 && (!sendbuf || !recvbuf))) return MPX_ERR_ARG;
  if (c->w->plain) return MPX_ERR_UNSUPPORTED;
  Desc d;
  fill_collective(d, K_ALLGATHER, dt, c, sendbuf, recvbuf, count, 0);
  return publish_collective(c, d, req);
}

static int allreduce_common(const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t dt,
                            int op, mpx_comm_t c, mpx_request_t* req) {
  if (!c || !c->stream || c->shared->mux()) return MPX_ERR_COMM;
  if (op != MPX_SUM) return MPX_ERR_ARG;
  if (dt < 0 || dt > MPX_DOUBLE) return MPX_ERR_TYPE;
  if (!coll_count_ok(count, c)) return MPX_ERR_ARG;
  if (count < 0 || (count > 0 && !recvbuf)) return MPX_ERR_ARG;
  if (sendbuf == MPX_IN_PLACE) sendbuf = recvbuf;
  if (count > 0 && !sendbuf) return MPX_ERR_ARG;
  if (c->w->plain) {
    if (req) return MPX_ERR_UNSUPPORTED;
    return plain::allreduce(c->w->plain, sendbuf, recvbuf, count, dt, c->shared->reduce_mode,
                            c->shared->id, c->rank, c->stream->id);
  }
  Desc d;
  fill_collective(d, K_ALLREDUCE, dt, c, sendbuf, recvbuf, count, 0);
  return publish_collective(c, d, req);
}

extern "C" int mpx_bcast_enqueue(void* buf, int64_t count, mpx_datatype_t dt, int root,
                                 mpx_comm_t c) {
  return bcast_common(buf, count, dt, root, c, nullptr);
}

extern "C" int mpx_reduce_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                                  mpx_datatype_t dt, int op, int root, mpx_comm_t c) {
  return reduce_common(sendbuf, recvbuf, count, dt, op, root, c, nullptr);
}

extern "C" int mpx_allgather_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                                     mpx_datatype_t dt, mpx_comm_t c) {
  return allgather_common(sendbuf, recvbuf, count, dt, c, nullptr);
}

extern "C" int mpx_barrier_enqueue(mpx_comm_t c) {
  // an allreduce of no elements: complete once every rank has arrived
  return allreduce_common(nullptr, nullptr, 0, MPX_BYTE, MPX_SUM, c, nullptr);
}

extern "C" int mpx_allreduce_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                                     mpx_datatype_t dt, int op, mpx_comm_t c) {
  return allreduce_common(sendbuf, recvbuf, count, dt, op, c, nullptr);
}

extern "C" int mpx_iallreduce_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                                      mpx_datatype_t dt, int op, mpx_comm_t c,
                                      mpx_request_t* req) {
  if (!req) return MPX_ERR_ARG;
  return allreduce_common(sendbuf, recvbuf, count, dt, op, c, req);
}

extern "C" int mpx_ibcast_enqueue(void* buf, int64_t count, mpx_datatype_t dt, int root,
                                  mpx_comm_t c, mpx_request_t* req) {
  if (!req) return MPX_ERR_ARG;
  return bcast_common(buf, count, dt, root, c, req);
}

extern "C" int mpx_ireduce_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                                   mpx_datatype_t dt, int op, int root, mpx_comm_t c,
                                   mpx_request_t* req) {
  if (!req) return MPX_ERR_ARG;
  return reduce_common(sendbuf, recvbuf, count, dt, op, root, c, req);
}

extern "C" int mpx_iallgather_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                                      mpx_datatype_t dt, mpx_comm_t c, mpx_request_t* req) {
  if (!req) return MPX_ERR_ARG;
  return allgather_common(sendbuf, recvbuf, count, dt, c, req);
}

extern "C" int mpx_ibarrier_enqueue(mpx_comm_t c, mpx_request_t* req) {
  if (!req) return MPX_ERR_ARG;
  return allreduce_common(nullptr, nullptr, 0, MPX_BYTE, MPX_SUM, c, req);
}


// ---------------------------------------------------------------------------
// batch submission
// ---------------------------------------------------------------------------
static mpx_stream_s* batch_op_stream(const mpx_op_t& o) {
  switch (o.kind) {
    case MPX_OP_SEND: case MPX_OP_RECV: case MPX_OP_ISEND: case MPX_OP_IRECV:
    case MPX_OP_ALLREDUCE: case MPX_OP_BCAST: case MPX_OP_REDUCE: case MPX_OP_ALLGATHER:
    case MPX_OP_BARRIER:
      return o.comm ? o.comm->stream : nullptr;
    case MPX_OP_WAIT: case MPX_OP_WAITALL:
      if (!o.requests) return nullptr;
      for (int64_t i = 0; i < (o.kind == MPX_OP_WAIT ? 1 : o.count); ++i)
        if (o.requests[i] != MPX_REQUEST_NULL) return request_stream(o.requests[i]);
      return nullptr;
    default:
      return nullptr;
  }
}

extern "C" int mpx_enqueue_batch(int n, const mpx_op_t ops[], int* done) {
  if (done) *done = 0;
  if (n < 0 || (n > 0 && !ops)) return MPX_ERR_ARG;
  // At most one stream owes an announcement at a time: a run is deferred
  // only while the next op goes to the same stream.
  mpx_stream_s* owing = nullptr;
  int rc = MPX_SUCCESS, i = 0;
  mpx_stream_s* st = n > 0 ? batch_op_stream(ops[0]) : nullptr;
  for (; i < n; ++i) {
    const mpx_op_t& o = ops[i];
    mpx_stream_s* next = i + 1 < n ? batch_op_stream(ops[i + 1]) : nullptr;
    const bool defer = st && next == st && !st->w->plain;
    switch (o.kind) {
      case MPX_OP_SEND:
        rc = mpx_send_enqueue(o.buf, o.count, o.datatype, o.peer, o.tag, o.comm);
        break;
      case MPX_OP_RECV:
        rc = mpx_recv_enqueue((void*)o.buf, o.count, o.datatype, o.peer, o.tag, o.comm, o.status);
        break;
      case MPX_OP_ISEND:
        rc = nb_p2p(K_ISEND, o.buf, o.count, o.datatype, o.peer, o.tag, o.comm, o.requests, defer);
        break;
      case MPX_OP_IRECV:
        rc = nb_p2p(K_IRECV, o.buf, o.count, o.datatype, o.peer, o.tag, o.comm, o.requests, defer);
        break;
      case MPX_OP_WAIT:
        rc = mpx_wait_enqueue(o.requests, o.status);
        break;
      case MPX_OP_WAITALL:
        rc = o.count > INT32_MAX ? MPX_ERR_ARG
                                 : mpx_waitall_enqueue((int)o.count, o.requests, o.status);
        break;
      case MPX_OP_ALLREDUCE:
        rc = mpx_allreduce_enqueue(o.buf, o.recvbuf, o.count, o.datatype, o.op, o.comm);
        break;
      case MPX_OP_BCAST:
        rc = mpx_bcast_enqueue((void*)o.buf, o.count, o.datatype, o.peer, o.comm);
        break;
      case MPX_OP_REDUCE:
        rc = mpx_reduce_enqueue(o.buf, o.recvbuf, o.count, o.datatype, o.op, o.peer, o.comm);
        break;
      case MPX_OP_ALLGATHER:
        rc = mpx_allgather_enqueue(o.buf, o.recvbuf, o.count, o.datatype, o.comm);
        break;
      case MPX_OP_BARRIER:
        rc = mpx_barrier_enqueue(o.comm);
        break;
      default:
        rc = MPX_ERR_ARG;
    }
    if (rc != MPX_SUCCESS) break;
    owing = st && st->owed ? st : nullptr;
    if (owing && next != st) {  // the run ends here
      rc = flush_owed(owing);
      owing = nullptr;
      if (rc != MPX_SUCCESS) {
        ++i;
        break;
      }
    }
    st = next;
  }
  // an op that failed validation leaves its predecessor's run unannounced
  if (owing) {
    const int frc = flush_owed(owing);
    if (rc == MPX_SUCCESS) rc = frc;
  }
  if (done) *done = i;
  return rc;
}

// ---------------------------------------------------------------------------
// recorded steps: one CUDA graph per step (device-side publication, then one
// engine pass)
// ---------------------------------------------------------------------------
struct mpx_step_s {
  mpx_world_s* w;
  std::vector<mpx_stream_s*> streams;  // streams the step publishes on
  uint8_t* dmem;                       // templates, per-stream records, counters, error word
  uint64_t* cnt_seq;                   // [max_streams] device: last published sequence number
  uint64_t* cnt_wl;                    // [max_streams] device: next waitlist index
  int32_t* err;                        // device: first publication error
  cudaStream_t cap;                    // stream the graph was captured on
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

static void step_release(mpx_step_s* st) {
  if (!st) return;
  if (st->exec) cudaGraphExecDestroy(st->exec);
  if (st->graph) cudaGraphDestroy(st->graph);
  if (st->cap) cudaStreamDestroy(st->cap);
  if (st->dmem) cudaFree(st->dmem);
  delete st;
}

extern "C" int mpx_step_create(mpx_world_t w, int n, const mpx_op_t ops[], mpx_step_t* out) {
  if (!w || !out || n < 0 || (n > 0 && !ops)) return MPX_ERR_ARG;
  if (w->cfg.engine_mode != MPX_ENGINE_DRAIN) return MPX_ERR_STATE;
  const int S = w->cfg.max_streams;
  // 1. per stream, its operations in order; a request slot -> (stream, relative seq)
  std::vector<std::vector<int>> per(S);
  std::unordered_map<const mpx_request_t*, std::pair<int, int64_t>> reqmap;
  std::vector<mpx_stream_s*> sof(n, nullptr);
  for (int i = 0; i < n; ++i) {
    const mpx_op_t& o = ops[i];
    mpx_stream_s* st = nullptr;
    switch (o.kind) {
      case MPX_OP_SEND: case MPX_OP_RECV: case MPX_OP_ISEND: case MPX_OP_IRECV:
      case MPX_OP_ALLREDUCE: case MPX_OP_BCAST: case MPX_OP_REDUCE: case MPX_OP_ALLGATHER:
      case MPX_OP_BARRIER:
        if (!o.comm || !o.comm->stream || o.comm->shared->mux()) return MPX_ERR_COMM;
        if (o.comm->w != w) return MPX_ERR_ARG;
        st = o.comm->stream;
        break;
      case MPX_OP_WAIT: case MPX_OP_WAITALL: {
        const int64_t m = o.kind == MPX_OP_WAIT ? 1 : o.count;
        if (m < 0 || (m > 0 && !o.requests)) return MPX_ERR_ARG;
        for (int64_t k = 0; k < m; ++k) {
          auto it = reqmap.find(o.requests + k);
          if (it == reqmap.end()) return MPX_ERR_REQUEST;  // must name an op of this step
          mpx_stream_s* sk = w->streams[it->second.first];
          if (st && sk != st) return MPX_ERR_STREAM;
          st = sk;
        }
        if (!st) return MPX_ERR_ARG;
        break;
      }
      default:
        return MPX_ERR_ARG;
    }
    if (!(st->flags & MPX_STREAM_EXCLUSIVE)) return MPX_ERR_STREAM;  // no doorbells in a graph
    if (st->step) return MPX_ERR_STATE;
    sof[i] = st;
    per[st->id].push_back(i);
    if (o.kind == MPX_OP_ISEND || o.kind == MPX_OP_IRECV) {
      if (!o.requests) return MPX_ERR_ARG;
      reqmap[o.requests] = {st->id, (int64_t)per[st->id].size()};
    }
  }
  // 2. templates
  std::vector<Desc> tmpl;
  std::vector<int64_t> tmpl_wl;
  std::vector<StepStream> recs;
  for (int g = 0; g < S; ++g) {
    if (per[g].empty()) continue;
    StepStream r;
    memset(&r, 0, sizeof(r));
    r.g = g;
    r.op0 = (int64_t)tmpl.size();
    r.wl0 = (int64_t)tmpl_wl.size();
    for (int i : per[g]) {
      const mpx_op_t& o = ops[i];
      Desc d;
      memset(&d, 0, sizeof(d));
      int rc = MPX_SUCCESS;
      switch (o.kind) {
        case MPX_OP_SEND: case MPX_OP_ISEND:
          rc = fill_p2p(d, o.kind == MPX_OP_SEND ? K_SEND : K_ISEND, o.buf, o.count, o.datatype,
                        o.peer, o.tag, o.comm, false);
          break;
        case MPX_OP_RECV: case MPX_OP_IRECV:
          rc = fill_p2p(d, o.kind == MPX_OP_RECV ? K_RECV : K_IRECV, o.buf, o.count, o.datatype,
                        o.peer, o.tag, o.comm, true);
          if (o.kind == MPX_OP_RECV) d.status = (uint64_t)o.status;
          break;
        case MPX_OP_WAIT:
          d.kw = make_kw(K_WAIT, 0, 0);
          d.aux = (uint64_t)reqmap[o.requests].second;
          d.status = (uint64_t)o.status;
          break;
        case MPX_OP_WAITALL:
          d.kw = make_kw(K_WAITALL, 0, 0);
          d.aux = (uint64_t)(tmpl_wl.size() - (size_t)r.wl0);
          d.n32 = (int32_t)o.count;
          d.status = (uint64_t)o.status;
          for (int64_t k = 0; k < o.count; ++k) tmpl_wl.push_back(reqmap[o.requests + k].second);
          break;
        case MPX_OP_ALLREDUCE: case MPX_OP_BARRIER: {
          const bool bar = o.kind == MPX_OP_BARRIER;
          const int64_t cnt = bar ? 0 : o.count;
          if (!bar && o.op != MPX_SUM) return MPX_ERR_ARG;
          if (!bar && (o.datatype < 0 || o.datatype > MPX_DOUBLE)) return MPX_ERR_TYPE;
          const void* sb = o.buf == MPX_IN_PLACE ? o.recvbuf : o.buf;
          if (cnt < 0 || (cnt > 0 && (!o.recvbuf || !sb))) return MPX_ERR_ARG;
          fill_collective(d, K_ALLREDUCE, bar ? MPX_BYTE : o.datatype, o.comm, bar ? nullptr : sb,
                          bar ? nullptr : o.recvbuf, cnt, 0);
          break;
        }
        case MPX_OP_BCAST: case MPX_OP_REDUCE: case MPX_OP_ALLGATHER: {
          if (o.datatype < 0 || o.datatype > MPX_DOUBLE) return MPX_ERR_TYPE;
          if (o.kind != MPX_OP_ALLGATHER && (o.peer < 0 || o.peer >= o.comm->size)) return MPX_ERR_RANK;
          if (o.kind == MPX_OP_REDUCE && o.op != MPX_SUM) return MPX_ERR_ARG;
          const bool at_root = o.comm->rank == o.peer;
          const void* in = o.buf == MPX_IN_PLACE ? o.recvbuf : o.buf;
          void* outp = o.kind == MPX_OP_BCAST ? (void*)o.buf
                       : (o.kind == MPX_OP_REDUCE && !at_root ? nullptr : o.recvbuf);
          if (o.count < 0 || (o.count > 0 && (!in || (o.kind != MPX_OP_BCAST && o.kind != MPX_OP_REDUCE && !outp))))
            return MPX_ERR_ARG;
          const uint32_t kind = o.kind == MPX_OP_BCAST ? K_BCAST : o.kind == MPX_OP_REDUCE ? K_REDUCE : K_ALLGATHER;
          fill_collective(d, kind, o.datatype, o.comm, in, outp, o.count, o.kind == MPX_OP_ALLGATHER ? 0 : o.peer);
          break;
        }
      }
      if (rc) return rc;
      tmpl.push_back(d);
    }
    r.nops = (int32_t)per[g].size();
    r.nwl = (int32_t)(tmpl_wl.size() - (size_t)r.wl0);
    if ((uint64_t)r.nops > (1ull << w->slots_log2) || (uint64_t)r.nwl > (1ull << w->wl_log2))
      return MPX_ERR_NO_MEM;  // a step must fit one stream's ring
    recs.push_back(r);
  }
  // 3. device memory: templates, records, counters, error word
  mpx_step_s* st = new (std::nothrow) mpx_step_s();
  if (!st) return MPX_ERR_NO_MEM;
  st->w = w;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t o_t = 0, o_wl = al(tmpl.size() * sizeof(Desc));
  const size_t o_r = o_wl + al(tmpl_wl.size() * 8 + 8);
  const size_t o_cs = o_r + al(recs.size() * sizeof(StepStream) + 8);
  const size_t o_cw = o_cs + al((size_t)S * 8);
  const size_t o_e = o_cw + al((size_t)S * 8);
  const size_t total = o_e + 256;
  if (cudaMalloc((void**)&st->dmem, total) != cudaSuccess) { step_release(st); return MPX_ERR_NO_MEM; }
  std::vector<uint64_t> cs((size_t)S, 0), cw((size_t)S, 0);
  for (int g = 0; g < S; ++g) {
    if (per[g].empty()) continue;
    mpx_stream_s* sg = w->streams[g];
    cs[(size_t)g] = sg->next_seq - 1;
    cw[(size_t)g] = sg->wl_next;
    st->streams.push_back(sg);
  }
  st->cnt_seq = (uint64_t*)(st->dmem + o_cs);
  st->cnt_wl = (uint64_t*)(st->dmem + o_cw);
  st->err = (int32_t*)(st->dmem + o_e);
  bool ok = cudaMemset(st->dmem, 0, total) == cudaSuccess;
  ok = ok && (tmpl.empty() || cudaMemcpy(st->dmem + o_t, tmpl.data(), tmpl.size() * sizeof(Desc), cudaMemcpyHostToDevice) == cudaSuccess);
  ok = ok && (tmpl_wl.empty() || cudaMemcpy(st->dmem + o_wl, tmpl_wl.data(), tmpl_wl.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess);
  ok = ok && (recs.empty() || cudaMemcpy(st->dmem + o_r, recs.data(), recs.size() * sizeof(StepStream), cudaMemcpyHostToDevice) == cudaSuccess);
  ok = ok && cudaMemcpy(st->cnt_seq, cs.data(), (size_t)S * 8, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(st->cnt_wl, cw.data(), (size_t)S * 8, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&st->cap, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) { step_release(st); return MPX_ERR_CUDA; }
  // 4. capture: publication kernel, then one engine pass over everything visible
  if (cudaStreamBeginCapture(st->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    step_release(st);
    return MPX_ERR_CUDA;
  }
  int rc1 = mpxi_step_post_launch(&w->params, st->dmem + o_t, st->dmem + o_wl, st->dmem + o_r,
                                  (int)recs.size(), st->cnt_seq, st->cnt_wl, st->err, st->cap);
  int rc2 = launch_engine(w, st->cap, 1, false);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(st->cap, &graph);
  st->graph = graph;
  if (rc1 || rc2 != MPX_SUCCESS || ce != cudaSuccess || !graph ||
      cudaGraphInstantiate(&st->exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    step_release(st);
    return MPX_ERR_CUDA;
  }
  for (mpx_stream_s* sg : st->streams) sg->step = st;
  *out = st;
  return MPX_SUCCESS;
}

extern "C" int mpx_step_launch(mpx_step_t st, mpx_cuda_stream_t stream) {
  if (!st || !st->exec) return MPX_ERR_ARG;
  if (__atomic_load_n(&st->w->wctl->failed, __ATOMIC_ACQUIRE)) return MPX_ERR_STATE;
  return cudaGraphLaunch(st->exec, (cudaStream_t)stream) == cudaSuccess ? MPX_SUCCESS : MPX_ERR_CUDA;
}

extern "C" int mpx_step_get_error(mpx_step_t st, int* err) {
  if (!st || !err) return MPX_ERR_ARG;
  int32_t v = 0;
  if (cudaMemcpy(&v, st->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return MPX_ERR_CUDA;
  *err = v;
  return MPX_SUCCESS;
}

extern "C" int mpx_step_free(mpx_step_t* pst) {
  if (!pst || !*pst) return MPX_ERR_ARG;
  mpx_step_s* st = *pst;
  mpx_world_s* w = st->w;
  // hand the streams' sequence numbers back to host enqueue
  const int S = w->cfg.max_streams;
  std::vector<uint64_t> cs((size_t)S), cw((size_t)S);
  if (cudaMemcpy(cs.data(), st->cnt_seq, (size_t)S * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(cw.data(), st->cnt_wl, (size_t)S * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return MPX_ERR_CUDA;
  for (mpx_stream_s* sg : st->streams) {
    sg->next_seq = cs[(size_t)sg->id] + 1;
    sg->wl_next = cw[(size_t)sg->id];
    sg->retired_seen = 0;
    sg->step = nullptr;
  }
  step_release(st);
  *pst = nullptr;
  return MPX_SUCCESS;
}

// ---------------------------------------------------------------------------
// internal accessors for the serving loop (mpx_serve.cpp)
// ---------------------------------------------------------------------------
extern "C" uint64_t mpxi_stream_last_seq(mpx_stream_t s) { return s ? s->next_seq - 1 : 0; }

extern "C" int mpxi_stream_done(mpx_stream_t s, uint64_t* done, uint64_t* done_t) {
  if (!s || s->w->plain) return MPX_ERR_ARG;
  StreamCtl* c = &s->w->sctl[s->id];
  *done = __atomic_load_n(&c->done, __ATOMIC_ACQUIRE);
  *done_t = __atomic_load_n(&c->done_t, __ATOMIC_ACQUIRE);
  return MPX_SUCCESS;
}
