// Internal layout shared by the host runtime and the device engine of libmpx.
// Nothing here is part of the public ABI (include/mpx.h).
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace mpxi {

// ---------------------------------------------------------------------------
// operation descriptor: one 64-byte record per enqueued call, written by the
// host into the stream's submission ring (pinned host memory) and copied by
// the engine into its device-resident operation table.
// ---------------------------------------------------------------------------
enum OpKind : uint32_t {
  K_SEND = 0, K_RECV = 1, K_ISEND = 2, K_IRECV = 3, K_WAIT = 4, K_WAITALL = 5, K_ALLREDUCE = 6,
  K_BCAST = 7, K_REDUCE = 8, K_ALLGATHER = 9
};

// kind word: bits 0-7 kind, 8-11 base type (MPX_BYTE..MPX_DOUBLE),
// 12-13 reduce mode, 14 nonblocking collective (completed by a wait)
__host__ __device__ inline uint32_t kw_kind(uint32_t kw) { return kw & 0xffu; }
__host__ __device__ inline uint32_t kw_base(uint32_t kw) { return (kw >> 8) & 0xfu; }
__host__ __device__ inline uint32_t kw_mode(uint32_t kw) { return (kw >> 12) & 0x3u; }
constexpr uint32_t kKwNonblocking = 1u << 14;
__host__ __device__ inline bool kw_nonblocking(uint32_t kw) { return (kw & kKwNonblocking) != 0; }
__host__ __device__ inline uint32_t make_kw(uint32_t kind, uint32_t base, uint32_t mode) {
  return kind | (base << 8) | (mode << 12);
}
__host__ __device__ inline int64_t base_size(uint32_t base) {
  return base == 0 ? 1 : (base == 1 ? 4 : (base == 2 ? 8 : (base == 3 ? 4 : 8)));
}

struct alignas(64) Desc {
  uint32_t kw;        // kind word
  uint16_t comm;      // communicator slot
  uint16_t rank;      // issuing stream's rank in the communicator
  int32_t peer;       // dest (send) / source or ANY_SOURCE (recv)
  int32_t tag;        // tag / ANY_TAG
  uint64_t buf;       // send or receive buffer; allreduce send buffer
  int64_t count;      // datatype instances; allreduce elements
  int32_t vcount;     // vector layout of one instance, in base elements
  int32_t blocklen;   // (1, 1, 1 for a predefined type)
  int32_t stride;
  int32_t n32;        // waitall: number of requests
  uint64_t aux;       // allreduce: receive buffer; wait: request seq; waitall: waitlist index
  uint64_t status;    // mpx_status_t* (device-accessible) or 0
};
static_assert(sizeof(Desc) == 64, "descriptor is 64 bytes");

// ---------------------------------------------------------------------------
// host <-> engine control words (pinned host memory, one cache line each)
// ---------------------------------------------------------------------------
// Host-written and engine-written words sit on different 128-byte lines: the
// host stores a tail per batch run while the engine polls it, and the engine
// stores retirement while the host reads it; sharing a line would bounce it
// across the chip-to-chip link on every access.
struct alignas(128) StreamCtl {
  uint64_t tail;        // H->D  last published sequence number
  int32_t flags;        // H->D  bit0 active, bit1 exclusive  (tail, flags, rank: one 16-byte load)
  int32_t rank;         // H->D  world rank of the stream
  uint64_t wl_tail;     // H->D  waitlist entries published
  int32_t pad0[26];
  uint64_t retired;     // D->H  every op with seq <= retired is finished
  uint64_t wl_retired;  // D->H  waitlist entries no longer read
  uint64_t done;        // D->H  mirror of the completion word
  int32_t error;        // D->H  first asynchronous error
  int32_t pad1a;
  uint64_t done_t;      // D->H  %globaltimer when `done` last advanced
  int32_t pad1[22];
};
static_assert(sizeof(StreamCtl) == 256, "stream control: two lines");
static_assert(offsetof(StreamCtl, retired) == 128, "engine-written line");

enum { SF_ACTIVE = 1, SF_EXCLUSIVE = 2 };
enum { ENG_STOPPED = 0, ENG_RUNNING = 1, ENG_EXITING = 2 };

struct alignas(128) WorldCtl {
  int32_t state;      // ENG_*
  int32_t stop;       // H->D exit when idle
  int32_t error;      // D->H first world error
  int32_t failed;     // D->H watchdog fired: operations are released without data
  int32_t pad0[28];   // the engine updates the words below all the time
  uint64_t counters[8];
  uint64_t heartbeat;  // D->H globaltimer of the last engine tick
  // D->H phase times summed over launches (ns): start->first task,
  // first task->all tasks done, last task->exit; [3] ticks
  uint64_t phase[4];
  // D->H control-tick time by phase, summed (ns): ingest, rounds, finished
  // tasks, per-stream completion, scheduling, decision, own data movement
  uint64_t tick_ns[8];
  // D->H finer split, summed (ns unless noted): stream advance, matching,
  // collectives (inside rounds); per-stream scheduling, reductions and staging
  // (inside scheduling); [5] rounds run, [6] ticks that ran rounds
  uint64_t sub_ns[8];
};
static_assert(offsetof(WorldCtl, counters) == 128, "engine-updated words on their own lines");

// ---------------------------------------------------------------------------
// device-side state
// ---------------------------------------------------------------------------
// physical flags of an operation
enum : int32_t {
  PF_MATCHED = 1,     // logical partner known
  PF_SCHED = 2,       // a data task has been created
  PF_STAGED = 4,      // send payload is in the staging arena
  PF_DELIVERED = 8,   // payload is in the receive buffer (send or recv side)
  PF_COMPLETE = 16,   // completion visible to the stream (send: staged or delivered)
  PF_WAITED = 32,     // a completed wait covered this request
  PF_STAGING = 64,    // staging task in flight
  PF_CAND = 128       // receive: listed for this tick's delivery scheduling
};

struct alignas(64) DOp {
  Desc d;             // copy of the descriptor
  uint64_t partner;   // ref (stream << 40 | seq) of the matched partner
  int64_t bytes;      // recv: bytes delivered; send: packed bytes
  uint64_t stage;     // staging arena offset + 1 when staged
  int32_t lstate;     // 0 new, 1 posted, 2 logically complete
  int32_t lround;     // round of logical completion
  int32_t pflags;     // PF_*
  int32_t err;        // status error
  int32_t msrc;       // recv: matched source rank
  int32_t mtag;       // recv: matched tag
  uint32_t wscan;     // waitall: logical scan position
  uint32_t pscan;     // waitall: physical scan position
  int64_t t_ingest;   // globaltimer at ingest
};
static_assert(sizeof(DOp) == 128, "device op record");

struct SState {
  uint64_t ingested;   // last seq copied from the ring
  uint64_t cursor;     // next seq the logical advance looks at
  uint64_t pc;         // next seq the physical completion scan looks at
  uint64_t retire;     // last retired seq
  uint64_t sched;      // next seq the scheduler looks at
  uint64_t done;       // last completion word value written
  uint64_t reached;    // stream has executed up to this seq (doorbell)
  uint64_t wl_retired; // waitlist entries finished
  uint64_t sreach;     // the scheduler has seen this stream reach every seq up to here
  int64_t stall_t0;    // globaltimer when the current physical stall began (0: none)
  int32_t flags;       // copy of StreamCtl.flags
  int32_t rank;
  int32_t nposts;      // posts of the current round
  int32_t pad;
};

struct QEntry {
  uint64_t ref;   // 0 = tombstone
  int32_t src;    // send: sender key; recv: source pattern or ANY_SOURCE
  int32_t tag;    // send: tag; recv: tag or ANY_TAG
  int64_t bytes;  // send: packed bytes; recv: capacity
};

// One post of a logical round: what matching needs of the operation, so
// that matching and pairing read no operation record.
struct PostRec {
  uint64_t ref;     // make_ref(stream, seq)
  int32_t key;      // send: sender key; recv: source pattern or ANY_SOURCE
  int32_t tag;      // send: tag; recv: tag or ANY_TAG
  int64_t bytes;    // send: packed bytes; recv: capacity
  uint32_t dom;     // matching domain (comm slot * ranks + member)
  uint32_t send;    // 1: a send, 0: a receive
};
static_assert(sizeof(PostRec) == 32, "post record");

struct QHead {
  uint32_t head, tail;
};

struct Layout {
  uint64_t base;     // address of instance 0
  int64_t seg;       // contiguous bytes per segment (whole message when contiguous)
  int64_t stride;    // bytes between segment starts within an instance
  int64_t per;       // segments per instance
  int64_t extent;    // bytes between instance starts
};

enum TaskType : uint32_t { T_COPY = 1, T_REDUCE = 2 };
enum TaskAction : uint32_t { A_DELIVER = 1, A_STAGE = 2, A_DELIVER_STAGED = 3, A_REDUCE = 4 };

// Task claim word: bits 40..63 (id+1) mod 2^24 (0: never published),
// 20..39 number of tiles, 0..19 next unclaimed tile (fetch-and-add).
__host__ __device__ inline uint64_t claim_word(uint64_t id, uint32_t ntiles) {
  return (((id + 1) & 0xFFFFFFull) << 40) | ((uint64_t)(ntiles & 0xFFFFF) << 20);
}
__host__ __device__ inline uint32_t claim_idp(uint64_t c) { return (uint32_t)(c >> 40); }
__host__ __device__ inline uint32_t claim_ntiles(uint64_t c) { return (uint32_t)((c >> 20) & 0xFFFFF); }
__host__ __device__ inline uint32_t claim_next(uint64_t c) { return (uint32_t)(c & 0xFFFFF); }
__host__ __device__ inline uint32_t id_tag(uint64_t id) { return (uint32_t)((id + 1) & 0xFFFFFF); }

struct alignas(128) Task {
  uint64_t claim;       // claim_word(id, ntiles) + tiles handed out
  uint32_t tiles_done;  // tiles finished
  uint32_t ntiles;
  uint32_t type;        // TaskType
  uint32_t action;      // TaskAction
  int64_t bytes;        // COPY: packed bytes; REDUCE: elements
  int64_t tile;         // COPY: packed bytes per tile; REDUCE: elements per tile
  Layout src, dst;      // COPY
  uint64_t ref_s, ref_r;  // COPY: send / recv ops; REDUCE: instance slot
  uint32_t nr, dtype, mode, unit;   // unit: bytes moved per access (16/8/4/2/1)
  uint64_t ptrs;        // REDUCE: device array: inputs at [0, nin), outputs at [nr, nr + nout)
  uint32_t nin, nout;   // REDUCE: inputs and outputs used
  uint32_t cop, pad_c;  // REDUCE: CO_SUM, CO_COPY (one input) or CO_GATHER (input e / gcount)
  int64_t gcount;       // REDUCE, CO_GATHER: elements per input
  int64_t chunk;        // COPY: bytes contiguous on both sides (kContig = whole tile)
};
static_assert(sizeof(Task) <= 256, "task record");
enum CollOp : uint32_t { CO_SUM = 0, CO_COPY = 1, CO_GATHER = 2 };
__host__ __device__ inline bool is_collective_kind(uint32_t k) {
  return k == K_ALLREDUCE || k == K_BCAST || k == K_REDUCE || k == K_ALLGATHER;
}

struct InstSlot {
  uint64_t k1;      // instance number + 1, 0 = free
  int32_t arrived;  // arrivals so far
  int32_t state;    // 0 collecting, 1 logically complete, 2 task created
  int32_t err;
  int32_t pad;
};

struct StageRec {
  uint64_t off;     // arena offset
  uint64_t size;    // bytes reserved (0 = free slot)
  int32_t freed;
  int32_t pad;
};

struct alignas(128) Shared {
  // task ring
  uint64_t task_head;    // lowest task id that may have unclaimed tiles (movers)
  uint64_t task_alloc;   // next task id to allocate (control)
  uint64_t task_retire;  // tasks below this are finished and processed
  uint64_t pad0[13];
  // control
  uint64_t round;
  int64_t last_progress;
  int32_t exit_flag;     // control -> movers: leave now
  int32_t epoch;         // launch epoch
  int32_t ctl_error;
  int32_t pad1;
  // staging ring allocator (control-owned)
  uint64_t st_head, st_tail;     // arena byte offsets (monotone)
  uint64_t sr_head, sr_tail;     // StageRec ring indices
  uint64_t cand_h, cand_t;       // delivery-scheduling list (EngineParams.cand), kept across launches
  uint64_t pad2[4];
  // completion queue: the CTA that finishes a task's last tile appends the
  // task's slot (movers: cq_tail); the control CTA consumes (cq_head)
  uint64_t cq_head;
  uint64_t pad3[15];
  uint64_t cq_tail;
  uint64_t pad4[15];
  // grid barrier for the control group
  uint32_t bar_count, bar_gen;
};

constexpr int kMaxDrainLimits = 256;

// One stream's part of a recorded step (mpx_step_create): its descriptors are
// tmpl[op0, op0 + nops), its waitall lists tmpl_wl[wl0, wl0 + nwl).  In the
// templates a waitall's aux is its offset into the step's lists, a wait's aux
// and every list entry are sequence numbers relative to the step (1-based;
// 0 = null request).
struct StepStream {
  int32_t g;
  int32_t nops;
  int32_t nwl;
  int32_t pad;
  int64_t op0;
  int64_t wl0;
};

// Kernel argument: pointers into world-owned memory plus configuration.
struct EngineParams {
  int32_t nranks, max_streams, slots_log2, max_comms;
  int32_t qcap_log2, tq_log2, iw, mode;   // mode: 0 persistent, 1 drain
  int32_t wl_log2, sr_log2, ctl_ctas, nctas;
  int32_t movers_per_cta;     // MPX_MOVERS_PER_CTA: mover m owns the task ids = m mod movers
  int32_t timing;             // control CTA times its phases (WorldCtl tick_ns, sub_ns)
  int64_t watchdog_ns, idle_ns, stage_delay_ns;
  int64_t tile_bytes, bulk_min;
  int64_t stage_bytes;
  const Desc* rings;          // [max_streams << slots_log2]   pinned
  const int64_t* waitlists;   // [max_streams << wl_log2]      pinned
  int64_t* wl_dev;            // [max_streams << wl_log2]      device copy of waitall lists
  uint64_t* cq;               // [2 << tq_log2] completion queue entries (slot + 1; 0 empty)
  int32_t* cnt2;              // [max_streams * ndomains] posts per (stream, domain), or null
  int32_t* dtot;              // [ndomains] posts per domain this round
  int64_t* dbase;             // [ndomains] start of each domain's list
  PostRec* dlist;             // [max_streams << slots_log2] this round's posts sorted by domain
  uint64_t* cand;             // [cand_cap] FIFO of receives whose delivery may have become possible
  int64_t cand_cap;           // a power of two
  StreamCtl* sctl;            // [max_streams]                 pinned
  WorldCtl* wctl;             //                                pinned
  uint64_t* doorbell;         // [max_streams] device (written by stream memops)
  uint64_t* done;             // [max_streams] device (waited on by stream memops)
  DOp* ops;                   // [max_streams << slots_log2]
  SState* ss;                 // [max_streams]
  PostRec* postbuf;           // [max_streams << slots_log2] this round's posts
  QEntry* pq;                 // posted receives [ndomains << qcap_log2]
  QEntry* uq;                 // unexpected sends
  QHead* pqh;                 // [ndomains]
  QHead* uqh;
  Task* tasks;                // [1 << tq_log2]
  Shared* sh;
  uint8_t* stage;             // staging arena
  StageRec* srec;             // [1 << sr_log2]
  InstSlot* inst;             // [max_comms * iw]
  uint64_t* inst_refs;        // [max_comms * iw * nranks]
  int64_t* next_inst;         // [max_comms * nranks]
  uint64_t* reduce_ptrs;      // [max_comms * iw * 2 * nranks]
  // diagnostic tile trace (MPX_ENGINE_TRACE entries, or null): one record of
  // 4 words per tile run by a mover: start and end %globaltimer, task slot <<
  // 32 | tile, bytes << 8 | unit (bit 7: bulk-copy path)
  uint64_t* trace;
  uint64_t* trace_pos;        // next record (atomic)
  int64_t trace_cap;
  // drain pass: ingest stream g only up to limit[g] (the operations published
  // when the pass was enqueued); nlimit = 0 means no limit
  int32_t nlimit, pad2;
  uint64_t limit[kMaxDrainLimits];
};

constexpr int64_t kContig = (int64_t)1 << 62;

__host__ __device__ inline uint64_t make_ref(int g, uint64_t seq) {
  return ((uint64_t)g << 40) | seq;
}
__host__ __device__ inline int ref_stream(uint64_t ref) { return (int)(ref >> 40); }
__host__ __device__ inline uint64_t ref_seq(uint64_t ref) { return ref & ((1ull << 40) - 1); }

}  // namespace mpxi

// engine launch entry (mpx_engine.cu)
extern "C" int mpxi_engine_launch(const mpxi::EngineParams* p, int nctas, int nthreads,
                                  void* cuda_stream, int cooperative);
extern "C" int mpxi_engine_smem_bytes(void);
