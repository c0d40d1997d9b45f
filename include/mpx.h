/*
 * mpx.h -- MPI communication enqueued on CUDA streams, among R virtual ranks
 * that share one GPU.  C ABI of libmpx.so.
 *
 * The operations follow "MPIX Stream: An Explicit Solution to Hybrid MPI+X
 * Programming" (Zhou, Raffenetti, Guo, Thakur; EuroMPI/USA'22):
 *   - MPIX stream: a local serial execution context, here a cudaStream_t bound
 *     to one virtual rank (§3.1, MPIX_Stream_create / MPIX_Stream_free).
 *   - stream communicator: one stream per rank (§3.3, MPIX_Stream_comm_create).
 *   - enqueue operations with the MPI signatures (§3.4, MPIX_Send_enqueue,
 *     MPIX_Recv_enqueue, MPIX_Isend_enqueue, MPIX_Irecv_enqueue,
 *     MPIX_Wait_enqueue, MPIX_Waitall_enqueue) and their extension to
 *     collectives (§3.4, last paragraph), here SUM allreduce.
 * The paper's process ranks become virtual ranks of one world living on one
 * GPU; the "network" is the GPU's own memory.  A device-resident engine
 * (one cooperative kernel) ingests operations from per-stream submission
 * rings, matches them, moves payloads with its own copy kernels and releases
 * each CUDA stream in stream order, so the host never synchronises per
 * message (§2.4, §5.2).
 *
 * Conventions for every call:
 *   - Return value: MPX_SUCCESS (0) or an MPX_ERR_* code.  Errors detected at
 *     enqueue time are returned synchronously and nothing is enqueued.
 *     Errors found while an operation executes on the GPU go to its status
 *     (if one was given) and to the sticky error of the stream and world
 *     (mpx_stream_get_error / mpx_world_get_error).
 *   - Buffers are device-accessible memory the caller owns (cudaMalloc,
 *     PyTorch tensors, or mapped pinned host memory).  A buffer must stay valid
 *     and unmodified (send) or untouched (receive) until its operation has
 *     completed in stream order.
 *   - mpx_status_t pointers passed to enqueue calls must be device-accessible
 *     (device memory or mapped pinned host memory) and stay valid until the
 *     operation completes; NULL (MPX_STATUS_IGNORE) discards the status.
 *   - A stream (and everything enqueued through it) is used by at most one
 *     host thread at a time (§3.1: the user guarantees serial use, so the
 *     enqueue path takes no lock).  Different streams may be used from
 *     different threads concurrently.
 *   - Nothing here allocates per message.  Library memory is allocated at
 *     mpx_world_create and mpx_stream_create.
 *   - Blocking calls put cuStreamWaitValue64 on the caller's stream.  An
 *     unsatisfied wait stalls the hardware queue the stream is mapped to, and
 *     so every stream sharing it; CUDA maps streams onto
 *     CUDA_DEVICE_MAX_CONNECTIONS queues.  Loading the library sets that
 *     variable to 32 unless it is already set (it only takes effect if CUDA
 *     is not initialised yet).  In PERSISTENT mode the engine is resident
 *     before any wait is enqueued, so the number of streams is not limited
 *     by this.  In DRAIN mode the pass that would satisfy a wait is itself
 *     launched on a stream: keep the streams that can sit at a blocking call
 *     at the same time, plus the pass's stream, within that many queues.
 */
#ifndef MPX_H
#define MPX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;                       /* cudaStream_t is a CUstream_st* */
typedef struct CUstream_st* mpx_cuda_stream_t;

typedef struct mpx_world_s* mpx_world_t;   /* R virtual ranks on this GPU (stands in for MPI_COMM_WORLD) */
typedef struct mpx_stream_s* mpx_stream_t; /* MPIX_Stream */
typedef struct mpx_comm_s* mpx_comm_t;     /* one rank's handle of a stream communicator */
typedef struct mpx_step_s* mpx_step_t;     /* a recorded step replayed as one CUDA graph */
typedef int64_t mpx_request_t;             /* opaque: (world << 56) | (stream << 40) | seq; MPX_REQUEST_NULL = -1 */
typedef int32_t mpx_datatype_t;
typedef struct mpx_info_s* mpx_info_t;     /* MPI_Info: (key, value) string hints; NULL = MPI_INFO_NULL */

typedef struct {
  int32_t source; /* sender's rank in the communicator */
  int32_t tag;    /* sender's tag */
  int32_t error;  /* MPX_SUCCESS, MPX_ERR_TRUNCATE, MPX_ERR_TIMEOUT, ... */
  int32_t source_index; /* multiplex stream communicator: the sender's local stream index; else 0 */
  int64_t bytes;  /* bytes delivered */
} mpx_status_t;   /* 24 bytes */

#define MPX_STATUS_IGNORE ((mpx_status_t*)0)
#define MPX_STATUSES_IGNORE ((mpx_status_t*)0)
#define MPX_IN_PLACE ((const void*)1)
#define MPX_REQUEST_NULL ((mpx_request_t)-1)

enum {
  MPX_ANY_SOURCE = -2,
  MPX_ANY_TAG = -1,
  MPX_ANY_INDEX = -1,   /* MPIX_ANY_INDEX: any local stream of the source (multiplex comms) */
  MPX_TAG_UB = (1 << 30) - 1,
  MPX_MAX_INFO_KEY = 255,   /* MPI_MAX_INFO_KEY */
  MPX_MAX_INFO_VAL = 1024,  /* MPI_MAX_INFO_VAL */
  MPX_UNDEFINED = -32766
};

/* predefined datatypes; derived ones come from mpx_type_vector */
enum {
  MPX_BYTE = 0, MPX_UINT8 = 0,
  MPX_INT32 = 1,
  MPX_INT64 = 2,
  MPX_FLOAT = 3,
  MPX_DOUBLE = 4
};

enum { MPX_SUM = 0 };

/* allreduce summation order */
enum {
  MPX_REDUCE_FIXED = 0, /* left fold (((x0+x1)+x2)+...) in rank order: bit-reproducible */
  MPX_REDUCE_TREE = 1   /* pairwise tree over ranks: tighter error bound */
};

/* stream flags */
enum {
  MPX_STREAM_DEFAULT = 0,
  /* The caller promises that no other work is enqueued on the CUDA stream
   * between these operations and that buffers are ready at enqueue time;
   * the per-operation stream-order doorbell is then omitted. */
  MPX_STREAM_EXCLUSIVE = 1
};

/* how the engine's mover CTAs take copy and reduction tiles
 * (mpx_world_config_t.mover_schedule) */
enum {
  MPX_MOVERS_WORKLIST = 0, /* every mover takes the next tile of the oldest task (large messages
                              spread over all CTAs) */
  MPX_MOVERS_PER_CTA = 1   /* mover m owns the tasks whose id is m modulo the mover count and
                              moves all their tiles (no shared claim point; small messages) */
};

/* where the submission rings live (mpx_world_config_t.ring_placement) */
enum {
  MPX_RINGS_HOST = 0,   /* pinned host memory: the host writes locally, the engine reads across
                           the chip-to-chip link */
  MPX_RINGS_DEVICE = 1  /* device memory that the host writes through the coherent chip-to-chip
                           mapping (managed memory kept on the device); needs a device on which
                           the host can access managed memory directly, else MPX_ERR_UNSUPPORTED */
};

/* engine modes (mpx_world_config_t.engine_mode) */
enum {
  MPX_ENGINE_PERSISTENT = 0, /* one cooperative engine kernel stays resident; relaunched on demand */
  MPX_ENGINE_DRAIN = 1,      /* the engine runs only inside mpx_world_progress(), in stream order */
  MPX_ENGINE_PLAIN = 2       /* no engine: host matching, one copy or kernel per operation, host sync per wait */
};

enum {
  MPX_SUCCESS = 0,
  MPX_ERR_ARG = 1,         /* invalid argument */
  MPX_ERR_RANK = 2,        /* destination/source rank out of range */
  MPX_ERR_TAG = 3,         /* tag out of range */
  MPX_ERR_TYPE = 4,        /* invalid datatype */
  MPX_ERR_COMM = 5,        /* not a stream communicator with a GPU stream (§3.4) */
  MPX_ERR_NO_ENDPOINT = 6, /* stream pool exhausted (§3.1) */
  MPX_ERR_AGAIN = 7,       /* submission ring or request space full; retry */
  MPX_ERR_STREAM = 8,      /* waitall requests on different streams (§3.4) */
  MPX_ERR_PENDING = 9,     /* object still has operations in flight (§3.1, MPIX_Stream_free) */
  MPX_ERR_CUDA = 10,       /* a CUDA runtime/driver call failed */
  MPX_ERR_REQUEST = 11,    /* invalid request handle */
  MPX_ERR_NO_MEM = 12,     /* allocation failed / budget exceeded / staging exhausted */
  MPX_ERR_STATE = 13,      /* engine in a state that does not allow the call */
  MPX_ERR_INTERN = 14,     /* internal error (device-side consistency check) */
  MPX_ERR_TRUNCATE = 15,   /* message longer than the receive buffer: capacity delivered */
  MPX_ERR_TIMEOUT = 16,    /* watchdog: no progress within watchdog_ns */
  MPX_ERR_UNSUPPORTED = 17
};

typedef struct {
  int32_t engine_mode;     /* MPX_ENGINE_* (default PERSISTENT) */
  int32_t max_streams;     /* stream (endpoint) pool size, <= 1024 (default 64) */
  int32_t ring_slots;      /* operations in flight per stream, power of two (default 4096) */
  int32_t max_comms;       /* stream communicators created over the world's life (default 8) */
  int32_t queue_slots;     /* matching queue capacity per (comm, rank) domain, power of two (default 4096) */
  int32_t task_slots;      /* engine task ring, power of two (default 16384) */
  int32_t engine_ctas;     /* engine CTAs; 0 = one per SM */
  int32_t engine_threads;  /* threads per engine CTA, multiple of 32, <= 512 (default 256); a
                              PERSISTENT engine uses at most as many as leave half of each SM's
                              registers to other kernels (256 in this build) */
  int32_t tile_bytes;      /* copy tile, multiple of 16 (default 65536) */
  int32_t bulk_min_bytes;  /* contiguous tiles at least this large move by TMA bulk copy (default 32768; 0 = never) */
  int32_t reduce_mode;     /* default allreduce order, MPX_REDUCE_* (default FIXED) */
  int32_t mover_schedule;  /* MPX_MOVERS_* (default WORKLIST) */
  int64_t staging_bytes;   /* eager-send staging arena (default 256 MiB) */
  int64_t budget_bytes;    /* cap on library device memory; 0 = no cap */
  int64_t watchdog_ns;     /* pending work with no progress this long fails with MPX_ERR_TIMEOUT (default 10 s) */
  int64_t idle_exit_ns;    /* persistent engine exits after this long with nothing to do (default 100 ms) */
  int64_t stage_delay_ns;  /* a stalled stream's undeliverable send is staged after this long (default 20 us) */
  int32_t ring_placement;  /* MPX_RINGS_* : submission rings, waitall lists and stream control
                              lines (default HOST) */
  int32_t reserved0;       /* 0 */
} mpx_world_config_t;

/* Fill *cfg with defaults, then apply MPX_* environment overrides. */
int mpx_world_config_init(mpx_world_config_t* cfg);

/* Create a world of `nranks` virtual ranks on the current CUDA device.
 * cfg may be NULL (defaults).  Allocates the submission rings, waitall lists
 * and stream control words where cfg->ring_placement says (pinned host
 * memory by default), the world control words in pinned host memory, and the
 * engine state, matching queues and staging arena in device memory.
 * Errors: MPX_ERR_ARG, MPX_ERR_NO_MEM, MPX_ERR_CUDA, MPX_ERR_UNSUPPORTED
 * (MPX_RINGS_DEVICE on a device without direct host access to managed
 * memory). */
int mpx_world_create(int nranks, const mpx_world_config_t* cfg, mpx_world_t* world);

/* Stop the engine and free everything.  MPX_ERR_PENDING if streams or
 * communicators are still alive (nothing is freed then). */
int mpx_world_free(mpx_world_t* world);

/* PERSISTENT mode: launch the engine now if it is not running (enqueue calls
 * also do this on demand).  Errors: MPX_ERR_STATE in other modes. */
int mpx_world_start(mpx_world_t world);

/* PERSISTENT mode: ask the engine to exit once idle and wait (host side, at
 * most timeout_ms) until it has exited.  MPX_ERR_TIMEOUT if it did not. */
int mpx_world_stop(mpx_world_t world, int timeout_ms);

/* DRAIN mode: enqueue one engine pass on `stream` (stream-ordered).  The pass
 * ingests the operations published before this call (for worlds of at most
 * 256 streams; larger worlds ingest everything visible when the pass runs),
 * moves every payload whose both ends are ready, and returns once all of
 * them are finished or nothing has progressed for 200 us.  A pass must not
 * overlap another engine pass of the same world (enqueue them on one
 * stream).  PLAIN mode: run host progress until nothing more can complete. */
int mpx_world_progress(mpx_world_t world, mpx_cuda_stream_t stream);

/* Failure recovery: mark the world failed and release every CUDA stream that
 * waits on an operation of this world (from the host, without the engine).
 * Pending operations complete with MPX_ERR_TIMEOUT and move no data; later
 * enqueue calls return MPX_ERR_STATE.  Use it when a deadline passes.  The
 * engine writes the released operations' statuses and retires them: a
 * running persistent engine at once, in DRAIN mode the next
 * mpx_world_progress pass (streams can be freed after that). */
int mpx_world_abort(mpx_world_t world);

/* Diagnostic: print the engine's per-stream cursors and task-ring state to
 * stderr (bounded wait; safe while the engine runs). */
int mpx_world_debug_dump(mpx_world_t world);

/* Sticky first asynchronous error of the world (MPX_SUCCESS if none). */
int mpx_world_get_error(mpx_world_t world, int* first_error);

/* Engine counters: [0] launches, [1] ticks, [2] messages completed,
 * [3] payload bytes moved, [4] tasks, [5] staged sends, [6] rounds,
 * [7] allreduce instances; summed over launches, in ns: [8] launch to first
 * data task, [9] first task to all tasks done, [10] last task to exit;
 * [11] control ticks; control-tick time by phase in ns: [12] ingest,
 * [13] logical rounds, [14] finished tasks, [15] per-stream completion,
 * [16] scheduling, [17] decisions, [18] the control CTA's own data movement;
 * finer, in ns: [19] stream advance, [20] matching, [21] collectives (parts
 * of [13]), [22] per-stream scheduling, [23] reductions and staging (parts of
 * [16]); [24] logical rounds run, [25] ticks that ran rounds; [26] the
 * domain sort of large rounds (part of [20]).
 * n is the array length (<= 27 filled). */
int mpx_world_get_counters(mpx_world_t world, int64_t* out, int n);

/* MPIX_Stream_create (§3.1) for virtual rank `rank`, backed by a CUDA
 * stream the caller owns and keeps alive until mpx_stream_free.  Claims a
 * dedicated endpoint (submission ring, doorbell and completion word) from
 * the world's pool; MPX_ERR_NO_ENDPOINT when the pool is exhausted.
 * flags: MPX_STREAM_DEFAULT or MPX_STREAM_EXCLUSIVE. */
int mpx_stream_create(mpx_world_t world, int rank, mpx_cuda_stream_t cuda_stream, unsigned flags,
                      mpx_stream_t* stream);

/* MPIX_Stream_create(info, &stream) (§3.1, §3.2; Listing 4): the queue
 * comes from info hints.  "type" = "cudaStream_t" with "value" = the
 * cudaStream_t handle as written by mpx_info_set_hex binds that CUDA stream
 * (the caller keeps it alive until mpx_stream_free); the optional hint
 * "mpx_exclusive" = "true" or "false" selects MPX_STREAM_EXCLUSIVE.  info =
 * NULL (MPI_INFO_NULL): the library creates a non-blocking CUDA stream for
 * the MPIX stream, owns it and destroys it in mpx_stream_free
 * (mpx_stream_get_cuda_stream returns it).  MPX_ERR_ARG for another "type",
 * a "value" that is not 8 bytes of hex, a "value" without "type", or an
 * exclusive hint other than "true"/"false"; otherwise as mpx_stream_create. */
int mpx_stream_create_info(mpx_world_t world, int rank, mpx_info_t info, mpx_stream_t* stream);

/* The CUDA stream an MPIX stream's operations are enqueued on. */
int mpx_stream_get_cuda_stream(mpx_stream_t stream, mpx_cuda_stream_t* cuda_stream);

/* MPIX_Stream_free (§3.1): fails with MPX_ERR_PENDING while operations
 * enqueued on the stream have not completed; *stream is then unchanged. */
int mpx_stream_free(mpx_stream_t* stream);

/* MPI_Info objects and MPIX_Info_set_hex (§3.2).  Keys are 1..MPX_MAX_INFO_KEY
 * characters, values at most MPX_MAX_INFO_VAL; setting a key again replaces
 * its value; keys keep their insertion order.  mpx_info_set_hex stores vallen
 * bytes as 2 * vallen lowercase hexadecimal digits, bytes in memory order
 * (the paper leaves the encoding to the implementation); mpx_info_get_hex
 * reverses it (MPX_ERR_ARG when the value is not 2 * vallen hex digits).
 * mpx_info_get copies at most buflen - 1 characters and a terminating NUL.
 * *flag = 1 when the key is present, else 0 (the output is then untouched).
 * Host-only: these need no GPU.  Errors: MPX_ERR_ARG for a null object, a key
 * out of bounds, a value too long, n out of range; MPX_ERR_NO_MEM. */
int mpx_info_create(mpx_info_t* info);
int mpx_info_free(mpx_info_t* info);
int mpx_info_set(mpx_info_t info, const char* key, const char* value);
int mpx_info_get(mpx_info_t info, const char* key, char* value, int buflen, int* flag);
int mpx_info_get_valuelen(mpx_info_t info, const char* key, int* valuelen, int* flag);
int mpx_info_get_nkeys(mpx_info_t info, int* nkeys);
int mpx_info_get_nthkey(mpx_info_t info, int n, char* key, int buflen);
int mpx_info_set_hex(mpx_info_t info, const char* key, const void* value, int vallen);
int mpx_info_get_hex(mpx_info_t info, const char* key, void* value, int vallen, int* flag);

/* Endpoint id of the stream (the order key used for matching ties). */
int mpx_stream_get_id(mpx_stream_t stream, int* id);

/* Sticky first asynchronous error of operations on this stream. */
int mpx_stream_get_error(mpx_stream_t stream, int* first_error);

/* Number of operations enqueued on the stream that have not completed. */
int mpx_stream_pending(mpx_stream_t stream, int64_t* pending);

/* MPIX_Stream_comm_create (§3.3), done for all R ranks at once because the
 * ranks share one process: streams[r] is rank r's stream; comms_out[r]
 * receives rank r's handle.  Each stream may serve in several comms. */
int mpx_stream_comm_create(mpx_world_t parent, int nranks, const mpx_stream_t streams[],
                           mpx_comm_t comms_out[]);

/* MPIX_Stream_comm_create_multiple (§3.5): a multiplex stream communicator
 * in which rank r attaches counts[r] >= 1 of its own streams, addressed by
 * their local index 0..counts[r]-1.  streams[] lists rank 0's streams in
 * index order, then rank 1's, ... (sum of counts entries; no stream twice
 * within one rank).  comms_out[r] receives rank r's handle.  It carries the
 * mpx_stream_* point-to-point calls below only: the plain p2p calls and the
 * collectives answer MPX_ERR_COMM on it, and so do mpx_enqueue_batch and
 * mpx_step_create.  Every member (rank, index) is a matching domain: a
 * communicator of M = sum(counts) members takes ceil(M / nranks) of the
 * world's max_comms slots (MPX_ERR_NO_MEM when they are used up).  M is at
 * most 65535 and counts[r] at most 32766.  MPX_ERR_UNSUPPORTED on the plain
 * path (MPX_ENGINE_PLAIN). */
int mpx_stream_comm_create_multiple(mpx_world_t parent, int nranks, const int counts[],
                                    const mpx_stream_t streams[], mpx_comm_t comms_out[]);

/* Free one rank's handle; the communicator dies with its last handle. */
int mpx_comm_free(mpx_comm_t* comm);
int mpx_comm_rank(mpx_comm_t comm, int* rank);
int mpx_comm_size(mpx_comm_t comm, int* size);
/* Summation order for allreduce on this communicator (all ranks' handles). */
int mpx_comm_set_reduce_mode(mpx_comm_t comm, int mode);

/* MPI_Type_vector(count, blocklength, stride, oldtype): `count` blocks of
 * `blocklength` old elements whose starts are `stride` elements apart.  One
 * instance spans ((count-1)*stride+blocklength) elements (its extent);
 * instance i of a message starts at i*extent.  oldtype must be predefined.
 * Process-wide handle; stays valid until mpx_type_free.  MPX_ERR_ARG when an
 * instance's extent exceeds 2^48 bytes.  Every call that takes a count of a
 * datatype rejects, with MPX_ERR_ARG, a count whose instances would span more
 * than 2^60 bytes (collectives: count * 8 * communicator size), so no byte
 * count derived from it can overflow. */
int mpx_type_vector(int count, int blocklength, int stride, mpx_datatype_t oldtype,
                    mpx_datatype_t* newtype);
int mpx_type_free(mpx_datatype_t* type);
/* bytes of data in one instance (gaps excluded) */
int mpx_type_size(mpx_datatype_t type, int64_t* size);
/* bytes from the start of one instance to the start of the next */
int mpx_type_extent(mpx_datatype_t type, int64_t* extent);

/* MPIX_Send_enqueue (§3.4): blocking in stream order.  Work enqueued on the
 * stream after it runs once the send buffer may be reused (the payload was
 * delivered or copied to the staging arena: eager protocol).  The buffer is
 * read only after the work enqueued before the call has completed. */
int mpx_send_enqueue(const void* buf, int64_t count, mpx_datatype_t datatype, int dest, int tag,
                     mpx_comm_t comm);

/* MPIX_Recv_enqueue (§3.4): blocking in stream order.  Work enqueued after it
 * sees the received data; no cudaStreamSynchronize is needed.  source may be
 * MPX_ANY_SOURCE, tag may be MPX_ANY_TAG.  A longer message delivers the
 * buffer's capacity and reports MPX_ERR_TRUNCATE in the status. */
int mpx_recv_enqueue(void* buf, int64_t count, mpx_datatype_t datatype, int source, int tag,
                     mpx_comm_t comm, mpx_status_t* status);

/* MPIX_Isend_enqueue / MPIX_Irecv_enqueue (§3.4): start in stream order and
 * let later enqueued work proceed; complete with mpx_wait(all)_enqueue. */
int mpx_isend_enqueue(const void* buf, int64_t count, mpx_datatype_t datatype, int dest, int tag,
                      mpx_comm_t comm, mpx_request_t* request);
int mpx_irecv_enqueue(void* buf, int64_t count, mpx_datatype_t datatype, int source, int tag,
                      mpx_comm_t comm, mpx_request_t* request);

/* MPIX_Stream_send / recv / isend / irecv (§3.5) on a multiplex stream
 * communicator, in enqueue form: a send is enqueued on the caller's local
 * stream src_idx and addresses stream dst_idx of rank dest; a receive is
 * enqueued on the caller's local stream dst_idx and accepts a message from
 * stream src_idx of rank source, where source may be MPX_ANY_SOURCE and
 * src_idx MPX_ANY_INDEX.  Messages between one (rank, index) pair and
 * another do not overtake; matching is otherwise as for the plain calls.
 * Requests belong to the local stream the call was enqueued on (wait for
 * them there).  status->source / source_index give the sender's rank and
 * local index.  Errors: MPX_ERR_COMM (not a multiplex handle), MPX_ERR_RANK,
 * MPX_ERR_TAG, MPX_ERR_ARG (an index out of range: src_idx on a receive is
 * checked against the source's stream count, or the largest count when
 * source is MPX_ANY_SOURCE), MPX_ERR_TYPE, and those of the plain calls. */
int mpx_stream_send_enqueue(const void* buf, int64_t count, mpx_datatype_t datatype, int dest,
                            int tag, mpx_comm_t comm, int src_idx, int dst_idx);
int mpx_stream_recv_enqueue(void* buf, int64_t count, mpx_datatype_t datatype, int source,
                            int tag, mpx_comm_t comm, int src_idx, int dst_idx,
                            mpx_status_t* status);
int mpx_stream_isend_enqueue(const void* buf, int64_t count, mpx_datatype_t datatype, int dest,
                             int tag, mpx_comm_t comm, int src_idx, int dst_idx,
                             mpx_request_t* request);
int mpx_stream_irecv_enqueue(void* buf, int64_t count, mpx_datatype_t datatype, int source,
                             int tag, mpx_comm_t comm, int src_idx, int dst_idx,
                             mpx_request_t* request);

/* MPIX_Wait_enqueue (§3.4): enqueued on the request's stream; work enqueued
 * after it runs once the request completed.  *request becomes
 * MPX_REQUEST_NULL at enqueue time (a null request is a no-op). */
int mpx_wait_enqueue(mpx_request_t* request, mpx_status_t* status);

/* MPIX_Waitall_enqueue (§3.4): all non-null requests must belong to one
 * stream (else MPX_ERR_STREAM).  statuses may be NULL, else n entries. */
int mpx_waitall_enqueue(int n, mpx_request_t requests[], mpx_status_t statuses[]);

/* Enqueued MPI_Allreduce (§3.4, last paragraph), op = MPX_SUM over a
 * predefined datatype.  The k-th call on a communicator from every rank forms
 * instance k.  Every rank's recvbuf receives the result; sendbuf may be
 * MPX_IN_PLACE.  Blocking in stream order.  Integer sums wrap; float sums use
 * the communicator's reduce mode. */
int mpx_allreduce_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                          mpx_datatype_t datatype, int op, mpx_comm_t comm);

/* One operation of mpx_enqueue_batch.  Fields a kind does not use are ignored. */
enum {
  MPX_OP_SEND = 0,      /* mpx_send_enqueue(buf, count, datatype, peer, tag, comm) */
  MPX_OP_RECV = 1,      /* mpx_recv_enqueue(buf, count, datatype, peer, tag, comm, status) */
  MPX_OP_ISEND = 2,     /* mpx_isend_enqueue(buf, count, datatype, peer, tag, comm, requests) */
  MPX_OP_IRECV = 3,     /* mpx_irecv_enqueue(buf, count, datatype, peer, tag, comm, requests) */
  MPX_OP_WAIT = 4,      /* mpx_wait_enqueue(requests, status) */
  MPX_OP_WAITALL = 5,   /* mpx_waitall_enqueue(count, requests, status) */
  MPX_OP_ALLREDUCE = 6, /* mpx_allreduce_enqueue(buf, recvbuf, count, datatype, op, comm) */
  MPX_OP_BCAST = 7,     /* mpx_bcast_enqueue(buf, count, datatype, peer = root, comm) */
  MPX_OP_REDUCE = 8,    /* mpx_reduce_enqueue(buf, recvbuf, count, datatype, op, peer = root, comm) */
  MPX_OP_ALLGATHER = 9, /* mpx_allgather_enqueue(buf, recvbuf, count, datatype, comm) */
  MPX_OP_BARRIER = 10   /* mpx_barrier_enqueue(comm) */
};

typedef struct {
  int32_t kind;             /* MPX_OP_* */
  mpx_datatype_t datatype;
  int32_t peer;             /* destination (send kinds) or source (receive kinds) */
  int32_t tag;
  int64_t count;            /* elements; for MPX_OP_WAITALL the number of requests */
  const void* buf;          /* message buffer; allreduce send buffer (or MPX_IN_PLACE) */
  void* recvbuf;            /* allreduce receive buffer */
  mpx_comm_t comm;
  mpx_request_t* requests;  /* isend/irecv: receives the request; wait/waitall: the request(s) */
  mpx_status_t* status;     /* recv/wait: one status; waitall: `count` statuses; may be NULL */
  int32_t op;               /* allreduce: MPX_SUM */
  int32_t pad;
} mpx_op_t;                 /* 72 bytes */

/* Batch submission: enqueue ops[0..n) in array order, each exactly as its
 * single call would (same validation, same semantics, same stream order),
 * and stop at the first one that fails.  *done (may be NULL) receives the
 * number of operations enqueued; the return value is the failing
 * operation's error, else MPX_SUCCESS.  Nothing is enqueued on a CUDA stream
 * by anyone else during the call, so consecutive non-blocking operations of
 * one non-exclusive stream share one stream-order doorbell (the last one's);
 * doorbells still owed when the batch stops are written before it returns.
 * The host cost per operation is that of filling one descriptor. */
int mpx_enqueue_batch(int n, const mpx_op_t ops[], int* done);

/* Recorded steps: the CUDA-graph form of batch submission, for a step that
 * repeats (the same operations on the same buffers every iteration, like
 * MPI persistent requests started together).  mpx_step_create validates
 * ops[0..n) as mpx_enqueue_batch would and records them instead of
 * enqueueing them; it then captures one CUDA graph with two nodes: a kernel
 * that publishes the step's descriptors and waitall lists into the streams'
 * submission rings from device memory (sequence numbers continue from the
 * streams' own), and one engine pass that matches, moves and completes
 * everything the step published.  mpx_step_launch replays that graph on
 * `stream`: the host cost of a step is one cudaGraphLaunch, whatever its
 * number of messages, and work enqueued on `stream` after the launch sees
 * the step complete.
 * Requirements: the world is in MPX_ENGINE_DRAIN mode (the graph carries its
 * engine pass); every stream of the step is MPX_STREAM_EXCLUSIVE
 * (MPX_ERR_STREAM otherwise; nothing else orders it); wait and waitall
 * operations name request slots that isend/irecv operations of the same step
 * write (MPX_ERR_REQUEST otherwise); a stream's part of a step fits its ring.
 * While the step exists its streams accept no other enqueue calls
 * (MPX_ERR_STATE) and belong to no other step.  Launches of one step, and
 * engine passes of its world, must not overlap: launch them on one stream.
 * Request values written during creation are placeholders: the step's waits
 * consume them internally.  Errors: those of the single calls, MPX_ERR_STATE
 * (world not in DRAIN mode), MPX_ERR_NO_MEM, MPX_ERR_CUDA (capture failed). */
int mpx_step_create(mpx_world_t world, int n, const mpx_op_t ops[], mpx_step_t* step);
int mpx_step_launch(mpx_step_t step, mpx_cuda_stream_t stream);
/* First error of the step's publication kernel (MPX_ERR_NO_MEM when a launch
 * found a ring still holding an earlier step's operations); synchronous. */
int mpx_step_get_error(mpx_step_t step, int* first_error);
/* Free the step and return its streams to host enqueue.  Every launch of the
 * step must have completed (synchronize the launch stream first). */
int mpx_step_free(mpx_step_t* step);

/* Serving loop: `nthreads` host threads, one MPIX stream (exclusive) and one
 * virtual rank each, submit enqueue requests open-loop (Poisson arrivals)
 * to one world; each request's receive or result buffer is admitted against
 * a device-memory budget (each thread owns budget/nthreads of it) and is
 * released when the request completes, so requests arriving while others
 * are on the GPU start as memory frees up.  A reaper thread reads the
 * streams' completion words and their device timestamps; latencies run
 * from a request's arrival (p50_us/p99_us) and from its enqueue call
 * (svc_p50_us/svc_p99_us) to its completion.  engine_mode
 * MPX_ENGINE_PLAIN runs the same requests through the plain path, where a
 * thread's blocking calls return only when complete.
 * Workload: every thread makes requests/nthreads calls; a share p_allreduce
 * of them are fp32 SUM allreduce participations over all threads (the same
 * instance list everywhere), the rest are isends and irecvs of messages
 * with uniform source, uniform other destination and Zipf(zipf_s) sizes over
 * the powers of two 2^min_log2..2^max_log2 (allreduce sizes likewise); the
 * calls between two allreduce instances form an epoch that each thread ends
 * with a waitall.  Items are numbered: messages first, then allreduce
 * instances.  digests (length ndigests, may be NULL) receives, for every
 * sampled item (item % sample_every == 0, or only_item), a digest of the
 * delivered bytes (rank 0's result for an allreduce); source_digests (may be
 * NULL; needs digests) receives, for every sampled message, the same digest
 * of the payload as its sender holds it, taken after the run; only_item >= 0
 * runs that item alone, without pacing, so that its digest can be compared
 * with the mix.  Errors: MPX_ERR_ARG, MPX_ERR_NO_MEM, and those of the calls
 * it makes. */
typedef struct {
  int32_t nthreads;
  int32_t engine_mode;   /* MPX_ENGINE_PERSISTENT or MPX_ENGINE_PLAIN */
  int64_t requests;
  double mean_gap_us;    /* mean Poisson gap per thread (0: no pacing) */
  double zipf_s;
  int32_t min_log2, max_log2;
  double p_allreduce;
  int64_t budget_bytes;
  uint64_t seed;
  int64_t sample_every;
  int64_t only_item;
} mpx_serve_config_t;

typedef struct {
  int64_t completed;       /* requests completed */
  int64_t items;           /* messages + allreduce instances in the schedule */
  double seconds;          /* first arrival to last completion */
  double msgs_per_s;       /* completed requests per second */
  double gbs;              /* delivered payload bytes per second / 1e9 */
  double p50_us, p99_us;   /* arrival -> completion */
  double svc_p50_us, svc_p99_us;  /* enqueue call -> completion */
  int64_t admission_waits; /* requests that waited for budget */
  int64_t peak_bytes;      /* peak budget in use (sum over threads) */
} mpx_serve_result_t;

/* Defaults: 32 threads, persistent engine, 10^6 requests, 2 us mean gap,
 * Zipf 1.2 over 64 B..16 MB, 30% allreduce, 40 GiB budget. */
int mpx_serve_config_init(mpx_serve_config_t* cfg);
int mpx_serve_run(const mpx_serve_config_t* cfg, mpx_serve_result_t* result, uint64_t* digests,
                  uint64_t* source_digests, int64_t ndigests);

/* The serving loop over a schedule the caller supplies instead of the one
 * generated from cfg (zipf_s, min/max_log2, p_allreduce, requests, seed and
 * sample_every are then unused; nthreads, engine_mode, mean_gap_us,
 * budget_bytes keep their meaning), so that the same requests can be run
 * through an independent implementation and compared item by item.
 * Thread t issues calls[call_lo[t] .. call_lo[t+1]) in order:
 *  - MPX_SERVE_SEND: isend of `bytes` bytes (MPX_BYTE) at regions[t] + off
 *    to thread `peer` with `tag`;
 *  - MPX_SERVE_RECV: irecv of `bytes` bytes from thread `peer` with `tag`
 *    into a buffer admitted from the thread's budget share;
 *  - MPX_SERVE_WAITALL: waitall over the thread's requests since its last
 *    waitall (blocking); its statuses go to statuses[capture ...] when
 *    capture >= 0 and statuses is not NULL;
 *  - MPX_SERVE_ALLREDUCE: blocking fp32 SUM allreduce of bytes/4 elements at
 *    regions[t] + off over all threads into a budget buffer.
 * A RECV or ALLREDUCE call with capture >= 0 has its delivered bytes copied
 * to (char*)capture + capture, in stream order after the blocking call that
 * covers it and before its buffer returns to the budget.  Calls of one item
 * (a message's send and receive, an instance's allreduces) share `item`.
 * Ownership: every array is the caller's; regions, capture and statuses are
 * device memory (statuses may be mapped pinned host memory).  Errors:
 * MPX_ERR_ARG (a call out of range: kind, peer, bytes, offsets, capture or
 * status ranges, or call_lo not monotone), MPX_ERR_NO_MEM, and those of the
 * calls it makes.  `result` as for mpx_serve_run. */
enum { MPX_SERVE_SEND = 0, MPX_SERVE_RECV = 1, MPX_SERVE_WAITALL = 2, MPX_SERVE_ALLREDUCE = 3 };
typedef struct {
  int32_t kind;      /* MPX_SERVE_* */
  int32_t peer;      /* send: destination thread; recv: source thread */
  int32_t tag;
  int32_t pad;
  int64_t item;      /* message or allreduce instance the call belongs to (>= 0) */
  int64_t bytes;     /* payload bytes; an allreduce's are a multiple of 4 */
  int64_t off;       /* send, allreduce: payload offset in the thread's source region */
  int64_t capture;   /* see above; -1: none */
} mpx_serve_call_t;  /* 48 bytes */
typedef struct {
  const mpx_serve_call_t* calls;
  const int64_t* call_lo;   /* nthreads + 1 entries */
  void* const* regions;     /* nthreads device source regions of region_bytes each */
  int64_t region_bytes;
  void* capture;            /* device memory of capture_bytes, or NULL */
  int64_t capture_bytes;
  mpx_status_t* statuses;   /* nstatuses device-accessible statuses, or NULL */
  int64_t nstatuses;
} mpx_serve_schedule_t;
int mpx_serve_run_schedule(const mpx_serve_config_t* cfg, const mpx_serve_schedule_t* sched,
                           mpx_serve_result_t* result);

/* Further enqueued collectives (§3.4, last paragraph: collectives take the
 * enqueue form).  Like allreduce, every collective call on a communicator is
 * blocking in stream order, and the k-th collective call of every rank, of
 * whatever kind, forms instance k: the ranks must call the same kinds in the
 * same order with the same count, datatype and root (else MPX_ERR_ARG in
 * the status and the sticky errors).  Predefined datatypes only.  The plain
 * path (MPX_ENGINE_PLAIN) has allreduce only: these return
 * MPX_ERR_UNSUPPORTED there.
 *  - mpx_bcast_enqueue: MPI_Bcast; the root's count elements of buf replace
 *    every other rank's.
 *  - mpx_reduce_enqueue: MPI_Reduce with op = MPX_SUM; the root's recvbuf
 *    receives the sum (recvbuf is ignored elsewhere and may be NULL);
 *    sendbuf may be MPX_IN_PLACE at the root.  Floating-point order as for
 *    allreduce (the communicator's reduce mode).
 *  - mpx_allgather_enqueue: MPI_Allgather; recvbuf holds nranks blocks of
 *    count elements, block s receives rank s's sendbuf; sendbuf may be
 *    MPX_IN_PLACE (the rank's block of recvbuf is its contribution).
 *  - mpx_barrier_enqueue: MPI_Barrier; work enqueued after it on any rank's
 *    stream runs once every rank's stream has reached it. */
int mpx_bcast_enqueue(void* buf, int64_t count, mpx_datatype_t datatype, int root, mpx_comm_t comm);
int mpx_reduce_enqueue(const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t datatype,
                       int op, int root, mpx_comm_t comm);
int mpx_allgather_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                          mpx_datatype_t datatype, mpx_comm_t comm);
int mpx_barrier_enqueue(mpx_comm_t comm);

/* Nonblocking collectives (MPI_Iallreduce, MPI_Ibcast, MPI_Ireduce,
 * MPI_Iallgather, MPI_Ibarrier) in enqueue form (§3.4): the call returns a
 * request at once and the stream goes on; the collective completes once
 * every rank has called it (and, for data, once each rank's stream has
 * reached its call), and mpx_wait(all)_enqueue on the request orders later
 * work on the stream after it.  Arguments, buffers and results are those of
 * the blocking call; the buffers must not be touched until the wait.
 * Blocking and nonblocking calls share one instance order per communicator
 * but never match each other: an instance that mixes them completes with
 * MPX_ERR_ARG (as a kind mismatch).  *request receives the request
 * (MPX_ERR_ARG when request is NULL).  MPX_ERR_UNSUPPORTED on the plain path
 * (MPX_ENGINE_PLAIN). */
int mpx_iallreduce_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                           mpx_datatype_t datatype, int op, mpx_comm_t comm,
                           mpx_request_t* request);
int mpx_ibcast_enqueue(void* buf, int64_t count, mpx_datatype_t datatype, int root,
                       mpx_comm_t comm, mpx_request_t* request);
int mpx_ireduce_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                        mpx_datatype_t datatype, int op, int root, mpx_comm_t comm,
                        mpx_request_t* request);
int mpx_iallgather_enqueue(const void* sendbuf, void* recvbuf, int64_t count,
                           mpx_datatype_t datatype, mpx_comm_t comm, mpx_request_t* request);
int mpx_ibarrier_enqueue(mpx_comm_t comm, mpx_request_t* request);

/* Persistent collectives (§3.4 last paragraph: collectives, nonblocking and
 * persistent ones included, take the enqueue form; MPI-4's
 * MPI_Allreduce_init, MPI_Bcast_init, MPI_Reduce_init, MPI_Allgather_init,
 * MPI_Barrier_init with MPI_Start / MPI_Startall and MPI_Request_free).
 * mpx_*_init records the call's arguments (those of the nonblocking call,
 * checked as far as they can be without enqueueing) in a persistent request
 * and enqueues nothing; *request receives a handle that is never
 * MPX_REQUEST_NULL and never equal to an operation's request.
 * mpx_start_enqueue starts one instance: exactly the nonblocking call
 * (mpx_i*_enqueue) with the recorded arguments, enqueued on the
 * communicator's stream at this point, so the buffers are read and written
 * when the stream reaches the start.  mpx_wait_enqueue / mpx_waitall_enqueue
 * on the handle complete the started instance (statuses as for the
 * nonblocking call) and leave the handle valid and inactive for the next
 * start; a wait on an inactive handle completes at once with the empty
 * status.  Starting an active handle gives MPX_ERR_STATE; mpx_startall_enqueue
 * starts n handles in array order and stops at the first error.
 * mpx_request_free frees an inactive persistent request and sets *request to
 * MPX_REQUEST_NULL (MPX_ERR_PENDING while started and not waited for;
 * MPX_ERR_REQUEST for any other request, which completes by a wait).  A
 * persistent request is used by one host thread at a time, like its stream.
 * Errors: those of the nonblocking calls; MPX_ERR_UNSUPPORTED on the plain
 * path. */
int mpx_allreduce_init(const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t datatype,
                       int op, mpx_comm_t comm, mpx_request_t* request);
int mpx_bcast_init(void* buf, int64_t count, mpx_datatype_t datatype, int root, mpx_comm_t comm,
                   mpx_request_t* request);
int mpx_reduce_init(const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t datatype,
                    int op, int root, mpx_comm_t comm, mpx_request_t* request);
int mpx_allgather_init(const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t datatype,
                       mpx_comm_t comm, mpx_request_t* request);
int mpx_barrier_init(mpx_comm_t comm, mpx_request_t* request);
int mpx_start_enqueue(mpx_request_t* request);
int mpx_startall_enqueue(int n, mpx_request_t requests[]);
int mpx_request_free(mpx_request_t* request);

/* Host-thread message rate (§5.3, Fig. 3, on host cores): `threads` pairs of
 * host threads, sender t sending `messages` 8-byte messages to receiver t
 * over a channel of its own (a per-thread communicator), `window` sends or
 * receives per wait.  The mode picks the discipline around each channel's
 * matching state: MPX_HOSTRATE_GLOBAL_LOCK (one mutex for every channel, a
 * global critical section), MPX_HOSTRATE_ENDPOINT_LOCK (a mutex per channel,
 * taken by every send, receive post and completion poll) or
 * MPX_HOSTRATE_STREAM (the MPIX stream serial-context guarantee: one
 * producer and one consumer per channel, a lock-free ring).  No GPU is used.
 * result: wall seconds from the release of all threads to the last join,
 * messages per second over all pairs, and payloads received out of order
 * (0 when correct).  MPX_ERR_ARG: threads outside 1..512, messages < 1,
 * window outside 1..1024, an unknown mode. */
enum { MPX_HOSTRATE_GLOBAL_LOCK = 0, MPX_HOSTRATE_ENDPOINT_LOCK = 1, MPX_HOSTRATE_STREAM = 2 };

typedef struct {
  int32_t threads;   /* sender/receiver pairs (default 1) */
  int32_t mode;      /* MPX_HOSTRATE_* (default STREAM) */
  int64_t messages;  /* per pair (default 2^20) */
  int32_t window;    /* operations per wait (default 64) */
  int32_t pad;
} mpx_hostrate_config_t;

typedef struct {
  double seconds;
  double msgs_per_s;
  int64_t errors;
} mpx_hostrate_result_t;

int mpx_hostrate_config_init(mpx_hostrate_config_t* cfg);
int mpx_hostrate_run(const mpx_hostrate_config_t* cfg, mpx_hostrate_result_t* result);

/* MPI_Get_count: elements of `datatype` in status->bytes, or MPX_UNDEFINED. */
int mpx_get_count(const mpx_status_t* status, mpx_datatype_t datatype, int64_t* count);

/* Listing 4's user compute kernel, for programs that interleave compute with
 * enqueued communication: y[i] = a*x[i] + y[i] (fused multiply-add, one
 * rounding) for i < n, launched on `stream`.  Not an MPI call. */
int mpx_saxpy_enqueue(int64_t n, float a, const float* x, float* y, mpx_cuda_stream_t stream);

/* Staged point-to-point copy that allocates nothing.  The paper has no
 * counterpart; it is for callers that cannot call cudaMalloc: code on
 * latency-critical paths that must not risk the implicit device-wide
 * synchronization an allocation or a free may bring, and processes whose
 * device memory is entirely carved up in advance.  In stream order on
 * `stream`, the message described by (sendbuf, sendcount, sendtype) is
 * packed into a staging area and unpacked into (recvbuf, recvcount,
 * recvtype); like a matched send/receive it delivers min(message, receive
 * capacity) bytes, and *bytes_delivered (host memory, may be NULL) is set to
 * that number before the call returns.  The staging area is a 16 MiB array
 * in the library's device memory (a file-scope __device__ array that every
 * GPU which loads the library holds until the process exits); the call
 * returns MPX_ERR_NO_MEM when more than 16 MiB would be delivered, and
 * allocates nothing itself.  Each device has its own copy of the array.  Its
 * device address is looked up once per device (cudaGetSymbolAddress, with
 * that device current) by mpx_world_create or by the first call on the
 * device, whichever comes first.  The address is kept for the life of the
 * process: after a cudaDeviceReset it is stale, and the function must not be
 * called again.  Every call on one device shares that device's array, which
 * keeps the last call's bytes, so calls that overlap on the same device (on
 * different streams) race: order them in one stream.  Counts whose byte span
 * exceeds 2^60 are rejected with MPX_ERR_ARG.  Errors: MPX_ERR_TYPE,
 * MPX_ERR_ARG, MPX_ERR_NO_MEM, MPX_ERR_CUDA. */
int mpx_sendrecv_static(const void* sendbuf, int64_t sendcount, mpx_datatype_t sendtype,
                        void* recvbuf, int64_t recvcount, mpx_datatype_t recvtype,
                        mpx_cuda_stream_t stream, int64_t* bytes_delivered);

/* Convenience: create / destroy a non-blocking CUDA stream (each call makes a
 * new stream).  Not an MPI call. */
int mpx_cuda_stream_create(mpx_cuda_stream_t* stream);
int mpx_cuda_stream_destroy(mpx_cuda_stream_t stream);

/* Library version (major*100+minor). */
int mpx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MPX_H */
