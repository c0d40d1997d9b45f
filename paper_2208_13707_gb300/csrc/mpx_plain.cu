// Plain path of libmpx (MPX_ENGINE_PLAIN): the baseline the device engine is
// measured against.  It does what a GPU-aware MPI does without stream
// integration (§2.4): a call on a non-exclusive stream first synchronizes the
// caller's CUDA stream (the full CPU/GPU synchronization the paper names as
// the penalty; an exclusive stream promises its buffers are ready), matching
// runs on the host under one world-wide lock, each match moves its payload
// with one cudaMemcpyAsync or one copy kernel on the world's copy stream, and
// every blocking call (recv, send, wait, waitall, allreduce) synchronizes the
// host with that copy stream before it returns.  Blocking calls that cannot
// complete yet return MPX_ERR_AGAIN (a progress loop retries them).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <deque>
#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "mpx_internal.h"
#include "mpx_plain.h"

extern "C" int mpxi_type_desc(int32_t type, int32_t* base, int32_t* vcount, int32_t* blocklen,
                              int32_t* stride);
extern "C" int mpxi_copy_typed(const void* src, int64_t scount, int32_t stype, void* dst,
                               int64_t dcount, int32_t dtype, int64_t n, void* stream);

namespace plain {
namespace {

__global__ void reduce_kernel(const uint64_t* ptrs, int nr, int64_t n, int dtype, int mode) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    switch (dtype) {
      case MPX_BYTE: {
        uint8_t a = ((const uint8_t*)ptrs[0])[i];
        for (int r = 1; r < nr; ++r) a = (uint8_t)(a + ((const uint8_t*)ptrs[r])[i]);
        for (int r = 0; r < nr; ++r) ((uint8_t*)ptrs[nr + r])[i] = a;
        break;
      }
      case MPX_INT32: {
        uint32_t a = ((const uint32_t*)ptrs[0])[i];
        for (int r = 1; r < nr; ++r) a += ((const uint32_t*)ptrs[r])[i];
        for (int r = 0; r < nr; ++r) ((uint32_t*)ptrs[nr + r])[i] = a;
        break;
      }
      case MPX_INT64: {
        uint64_t a = ((const uint64_t*)ptrs[0])[i];
        for (int r = 1; r < nr; ++r) a += ((const uint64_t*)ptrs[r])[i];
        for (int r = 0; r < nr; ++r) ((uint64_t*)ptrs[nr + r])[i] = a;
        break;
      }
      case MPX_FLOAT: {
        float a;
        if (mode == MPX_REDUCE_TREE) {
          // pairwise over ranks, leftovers folded from the top (as the engine)
          float stack[16];
          int depth[16], sp = 0;
          for (int r = 0; r < nr; ++r) {
            float cur = ((const float*)ptrs[r])[i];
            int d = 0;
            while (sp > 0 && depth[sp - 1] == d) {
              cur = __fadd_rn(stack[sp - 1], cur);
              --sp;
              ++d;
            }
            stack[sp] = cur;
            depth[sp] = d;
            ++sp;
          }
          a = stack[sp - 1];
          for (int k = sp - 2; k >= 0; --k) a = __fadd_rn(stack[k], a);
        } else {
          a = ((const float*)ptrs[0])[i];
          for (int r = 1; r < nr; ++r) a = __fadd_rn(a, ((const float*)ptrs[r])[i]);
        }
        for (int r = 0; r < nr; ++r) ((float*)ptrs[nr + r])[i] = a;
        break;
      }
      default: {
        double a = ((const double*)ptrs[0])[i];
        for (int r = 1; r < nr; ++r) a = __dadd_rn(a, ((const double*)ptrs[r])[i]);
        for (int r = 0; r < nr; ++r) ((double*)ptrs[nr + r])[i] = a;
        break;
      }
    }
  }
}

int64_t type_bytes(int32_t t) {
  int32_t b, v, bl, st;
  if (mpxi_type_desc(t, &b, &v, &bl, &st)) return -1;
  return mpxi::base_size((uint32_t)b) * v * bl;
}

// `count` instances of type t span at most 2^60 bytes (the engine path's rule):
// checked by division, before anything multiplies the count.
bool span_ok(int32_t t, int64_t count) {
  int32_t b, v, bl, st;
  if (mpxi_type_desc(t, &b, &v, &bl, &st)) return false;
  const int64_t ext = mpxi::base_size((uint32_t)b) * ((int64_t)(v - 1) * st + bl);
  return count >= 0 && (count == 0 || count <= (1ll << 60) / (ext > 0 ? ext : 1));
}

struct Msg {
  int stream;
  uint64_t seq;
  int src;
  int tag;
  const void* buf;  // send buffer, or the staging copy (then type BYTE)
  int64_t count;
  int32_t type;
  int64_t bytes;
  int64_t stage_off;  // >= 0 when staged
};

struct Recv {
  int stream;
  uint64_t seq;
  int src;  // pattern
  int tag;  // pattern
  void* buf;
  int64_t count;
  int32_t type;
  mpx_status_t* status;
};

struct Req {
  bool complete;
  bool is_recv;
  mpx_status_t st;
};

struct Stream {
  bool alive = false;
  bool exclusive = false;
  int rank = 0;
  cudaStream_t cs = nullptr;
  uint64_t next_seq = 1;
  std::unordered_map<uint64_t, Req> reqs;
  int err = 0;
  // the blocking call waiting to be retried (allreduce arrival)
  bool ar_pending = false;
  int64_t ar_instance = -1;
};

struct Instance {
  std::vector<const void*> send;
  std::vector<void*> recv;
  std::vector<int> arrived;
  int64_t count = 0;
  int32_t type = 0;
  int mode = 0;
  int narrived = 0;
  int nreturned = 0;
  bool done = false;
};

}  // namespace

struct PlainWorld {
  int nranks;
  int widx;
  std::mutex mu;  // one lock for the whole world: the baseline's critical section
  std::vector<Stream> streams;
  std::map<std::pair<int, int>, std::deque<Msg>> unexpected;  // (comm, dst) -> arrived sends
  std::map<std::pair<int, int>, std::deque<Recv>> posted;     // (comm, dst) -> posted receives
  std::map<int, std::map<int64_t, Instance>> inst;            // comm -> instance -> arrivals
  std::map<std::pair<int, int>, int64_t> next_inst;           // (comm, rank) -> next instance
  uint8_t* stage = nullptr;
  int64_t stage_bytes = 0;
  int64_t stage_head = 0;
  int64_t staged_live = 0;
  uint64_t* dptrs = nullptr;  // device array of allreduce pointers
  int dptrs_cap = 0;
  cudaStream_t copy_stream = nullptr;
  int error = 0;
  int64_t counters[19] = {0};
};

namespace {

int sync_stream(cudaStream_t s) { return cudaStreamSynchronize(s) == cudaSuccess ? MPX_SUCCESS : MPX_ERR_CUDA; }

bool accepts(const Recv& r, int src, int tag) {
  return (r.src == MPX_ANY_SOURCE || r.src == src) && (r.tag == MPX_ANY_TAG || r.tag == tag);
}

mpx_status_t make_status(int src, int tag, int err, int64_t bytes) {
  mpx_status_t st;
  st.source = src;
  st.tag = tag;
  st.error = err;
  st.source_index = 0;
  st.bytes = bytes;
  return st;
}

// Move a matched message into the receive buffer; host-synchronized.
int deliver(PlainWorld* pw, const Msg& m, const Recv& r, mpx_status_t* out) {
  const int64_t cap = r.count * type_bytes(r.type);
  const int64_t n = m.bytes < cap ? m.bytes : cap;
  // the copy is stream-ordered on the copy stream; a later staging copy into
  // the same arena space queues behind it
  int rc = mpxi_copy_typed(m.buf, m.count, m.type, r.buf, r.count, r.type, n, pw->copy_stream);
  if (rc) return rc;
  if (m.stage_off >= 0 && --pw->staged_live == 0) pw->stage_head = 0;
  *out = make_status(m.src, m.tag, m.bytes > cap ? MPX_ERR_TRUNCATE : 0, n);
  if (out->error) {
    if (!pw->error) pw->error = out->error;
    if (!pw->streams[r.stream].err) pw->streams[r.stream].err = out->error;
  }
  pw->counters[2] += 1;
  pw->counters[3] += n;
  pw->counters[4] += 1;
  return MPX_SUCCESS;
}

int write_statuses(mpx_status_t* dst, const mpx_status_t* st, int n) {
  if (!dst || n <= 0) return MPX_SUCCESS;
  return cudaMemcpy(dst, st, sizeof(*st) * (size_t)n, cudaMemcpyDefault) == cudaSuccess
             ? MPX_SUCCESS
             : MPX_ERR_CUDA;
}

}  // namespace

PlainWorld* create(int nranks, int max_streams, int64_t staging_bytes) {
  PlainWorld* pw = new PlainWorld();
  pw->nranks = nranks;
  pw->widx = 0;
  pw->streams.resize(max_streams);
  pw->stage_bytes = staging_bytes;
  if (cudaMalloc(&pw->stage, (size_t)staging_bytes) != cudaSuccess ||
      cudaStreamCreateWithFlags(&pw->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
    destroy(pw);
    return nullptr;
  }
  return pw;
}

void set_world_index(PlainWorld* pw, int widx) { pw->widx = widx; }

void destroy(PlainWorld* pw) {
  if (!pw) return;
  if (pw->copy_stream) cudaStreamDestroy(pw->copy_stream);
  if (pw->stage) cudaFree(pw->stage);
  if (pw->dptrs) cudaFree(pw->dptrs);
  delete pw;
}

int progress(PlainWorld*) { return MPX_SUCCESS; }  // everything happens inside the calls

int error(PlainWorld* pw) { return pw->error; }

int64_t counter(PlainWorld* pw, int i) { return (i >= 0 && i < 19) ? pw->counters[i] : 0; }

int stream_create(PlainWorld* pw, int id, int rank, cudaStream_t cs, bool exclusive) {
  std::lock_guard<std::mutex> g(pw->mu);
  Stream& s = pw->streams[id];
  const uint64_t keep = s.next_seq;
  s = Stream();
  s.alive = true;
  s.exclusive = exclusive;
  s.rank = rank;
  s.cs = cs;
  s.next_seq = keep;
  return MPX_SUCCESS;
}

void stream_free(PlainWorld* pw, int id) {
  std::lock_guard<std::mutex> g(pw->mu);
  pw->streams[id].alive = false;
  pw->streams[id].reqs.clear();
}

int64_t stream_pending(PlainWorld* pw, int id) {
  std::lock_guard<std::mutex> g(pw->mu);
  return (int64_t)pw->streams[id].reqs.size() + (pw->streams[id].ar_pending ? 1 : 0);
}

int stream_error(PlainWorld* pw, int id) {
  std::lock_guard<std::mutex> g(pw->mu);
  return pw->streams[id].err;
}

void comm_create(PlainWorld*, int) {}

int p2p(PlainWorld* pw, uint32_t kind, const void* buf, int64_t count, mpx_datatype_t dt, int peer,
        int tag, int comm, int rank, int sid, mpx_status_t* status, mpx_request_t* req) {
  const int64_t tb = type_bytes(dt);
  if (tb < 0) return MPX_ERR_TYPE;
  if (count < 0 || !span_ok(dt, count)) return MPX_ERR_ARG;
  const bool is_send = kind == mpxi::K_SEND || kind == mpxi::K_ISEND;
  if (is_send) {
    if (peer < 0 || peer >= pw->nranks) return MPX_ERR_RANK;
    if (tag < 0 || tag > MPX_TAG_UB) return MPX_ERR_TAG;
  } else {
    if (peer != MPX_ANY_SOURCE && (peer < 0 || peer >= pw->nranks)) return MPX_ERR_RANK;
    if (tag != MPX_ANY_TAG && (tag < 0 || tag > MPX_TAG_UB)) return MPX_ERR_TAG;
  }
  std::lock_guard<std::mutex> g(pw->mu);
  Stream& S = pw->streams[sid];
  // the buffer is ready only once the work enqueued before the call is done
  int rc = S.exclusive ? MPX_SUCCESS : sync_stream(S.cs);
  if (rc) return rc;
  if (is_send) {
    Msg m{sid, S.next_seq, rank, tag, buf, count, dt, count * tb, -1};
    auto& q = pw->posted[{comm, peer}];
    bool matched = false;
    for (auto it = q.begin(); it != q.end(); ++it) {
      if (!accepts(*it, rank, tag)) continue;
      Recv r = *it;
      q.erase(it);
      mpx_status_t st;
      rc = deliver(pw, m, r, &st);
      if (rc) return rc;
      Stream& RS = pw->streams[r.stream];
      auto rq = RS.reqs.find(r.seq);
      if (rq != RS.reqs.end()) {
        rq->second.complete = true;
        rq->second.st = st;
      }
      matched = true;
      break;
    }
    // no receive yet: stage the payload (eager)
    if (!matched && m.bytes > 0) {
      const int64_t need = (m.bytes + 255) & ~(int64_t)255;
      if (pw->stage_head + need > pw->stage_bytes) return MPX_ERR_AGAIN;
      uint8_t* dst = pw->stage + pw->stage_head;
      rc = mpxi_copy_typed(buf, count, dt, dst, m.bytes, MPX_BYTE, m.bytes, pw->copy_stream);
      if (rc) return rc;
      m.buf = dst;
      m.count = m.bytes;
      m.type = MPX_BYTE;
      m.stage_off = pw->stage_head;
      pw->stage_head += need;
      pw->staged_live++;
      pw->counters[5] += 1;
    }
    if (!matched) pw->unexpected[{comm, peer}].push_back(m);
    if (kind == mpxi::K_SEND) {  // blocking: the buffer is reusable on return
      rc = sync_stream(pw->copy_stream);
      if (rc) return rc;
    }
    const uint64_t seq = S.next_seq++;
    if (kind == mpxi::K_ISEND && req) {
      Req r0{true, false, make_status(MPX_ANY_SOURCE, MPX_ANY_TAG, 0, 0)};
      S.reqs[seq] = r0;
      *req = (mpx_request_t)(((uint64_t)pw->widx << 56) | ((uint64_t)sid << 40) | seq);
    }
    return MPX_SUCCESS;
  }
  // receive: take the first arrived send it accepts, else post (irecv) or retry later (recv)
  Recv r{sid, S.next_seq, peer, tag, (void*)buf, count, dt, status};
  auto& uq = pw->unexpected[{comm, rank}];
  for (auto it = uq.begin(); it != uq.end(); ++it) {
    if (!accepts(r, it->src, it->tag)) continue;
    Msg m = *it;
    uq.erase(it);
    mpx_status_t st;
    rc = deliver(pw, m, r, &st);
    if (rc) return rc;
    const uint64_t seq = S.next_seq++;
    if (kind == mpxi::K_IRECV && req) {
      S.reqs[seq] = Req{true, true, st};
      *req = (mpx_request_t)(((uint64_t)pw->widx << 56) | ((uint64_t)sid << 40) | seq);
      return MPX_SUCCESS;
    }
    rc = sync_stream(pw->copy_stream);  // blocking receive: data in place on return
    if (rc) return rc;
    return write_statuses(status, &st, 1);
  }
  if (kind == mpxi::K_RECV) return MPX_ERR_AGAIN;  // nothing to receive yet: retry
  const uint64_t seq = S.next_seq++;
  r.seq = seq;
  pw->posted[{comm, rank}].push_back(r);
  S.reqs[seq] = Req{false, true, make_status(0, 0, 0, 0)};
  if (req) *req = (mpx_request_t)(((uint64_t)pw->widx << 56) | ((uint64_t)sid << 40) | seq);
  return MPX_SUCCESS;
}

int wait(PlainWorld* pw, int sid, int n, const mpx_request_t* reqs, mpx_status_t* statuses) {
  std::lock_guard<std::mutex> g(pw->mu);
  Stream& S = pw->streams[sid];
  for (int i = 0; i < n; ++i) {
    if (reqs[i] == MPX_REQUEST_NULL) continue;
    const uint64_t seq = (uint64_t)reqs[i] & ((1ull << 40) - 1);
    auto it = S.reqs.find(seq);
    if (it == S.reqs.end()) return MPX_ERR_REQUEST;
    if (!it->second.complete) return MPX_ERR_AGAIN;
  }
  // one host synchronization per wait: every copy of these requests is done
  int rc = sync_stream(pw->copy_stream);
  if (rc) return rc;
  std::vector<mpx_status_t> sts((size_t)n);
  for (int i = 0; i < n; ++i) {
    mpx_status_t st = make_status(MPX_ANY_SOURCE, MPX_ANY_TAG, 0, 0);
    if (reqs[i] != MPX_REQUEST_NULL) {
      const uint64_t seq = (uint64_t)reqs[i] & ((1ull << 40) - 1);
      auto it = S.reqs.find(seq);
      st = it->second.st;
      S.reqs.erase(it);
    }
    sts[(size_t)i] = st;
  }
  return write_statuses(statuses, sts.data(), n);
}

int allreduce(PlainWorld* pw, const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t dt,
              int mode, int comm, int rank, int sid) {
  std::lock_guard<std::mutex> g(pw->mu);
  Stream& S = pw->streams[sid];
  if (!S.ar_pending) {
    int rc = sync_stream(S.cs);
    if (rc) return rc;
    const int64_t k = pw->next_inst[{comm, rank}]++;
    Instance& I = pw->inst[comm][k];
    if (I.arrived.empty()) {
      I.send.assign(pw->nranks, nullptr);
      I.recv.assign(pw->nranks, nullptr);
      I.arrived.assign(pw->nranks, 0);
    }
    I.send[rank] = sendbuf;
    I.recv[rank] = recvbuf;
    I.arrived[rank] = 1;
    I.count = count;
    I.type = dt;
    I.mode = mode;
    I.narrived++;
    S.ar_pending = true;
    S.ar_instance = k;
    if (I.narrived == pw->nranks && count > 0) {
      // the last arrival runs the one reduction kernel and waits for it
      const int nr = pw->nranks;
      if (pw->dptrs_cap < 2 * nr) {
        if (pw->dptrs) cudaFree(pw->dptrs);
        if (cudaMalloc(&pw->dptrs, (size_t)2 * nr * 8) != cudaSuccess) return MPX_ERR_NO_MEM;
        pw->dptrs_cap = 2 * nr;
      }
      std::vector<uint64_t> hp(2 * nr);
      for (int r = 0; r < nr; ++r) {
        hp[r] = (uint64_t)I.send[r];
        hp[nr + r] = (uint64_t)I.recv[r];
      }
      if (cudaMemcpy(pw->dptrs, hp.data(), hp.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) return MPX_ERR_CUDA;
      reduce_kernel<<<1024, 256, 0, pw->copy_stream>>>(pw->dptrs, nr, count, dt, mode);
      rc = sync_stream(pw->copy_stream);
      if (rc) return rc;
      I.done = true;
      pw->counters[7] += 1;
      pw->counters[3] += 2 * nr * count * type_bytes(dt);
    } else if (I.narrived == pw->nranks) {
      I.done = true;
    }
  }
  auto& per_comm = pw->inst[comm];
  auto it = per_comm.find(S.ar_instance);
  if (it == per_comm.end()) return MPX_ERR_INTERN;
  if (!it->second.done) return MPX_ERR_AGAIN;
  S.ar_pending = false;
  if (++it->second.nreturned == pw->nranks) per_comm.erase(it);
  return MPX_SUCCESS;
}

}  // namespace plain

// Load the plain path's reduction kernel now (its copies use the library's
// standalone copy kernel, which mpxi_static_preload loads).
extern "C" int mpxi_plain_preload(void) {
  cudaFuncAttributes a;
  return cudaFuncGetAttributes(&a, plain::reduce_kernel) == cudaSuccess ? 0 : 1;
}
