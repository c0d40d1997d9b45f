// Persistent collective requests of libmpx (MPI-4 persistent collectives:
// MPI_Allreduce_init and friends, MPI_Start), in enqueue form.
//
// A persistent request fixes a collective's arguments once.  Each
// mpx_start_enqueue starts one instance of it: exactly the nonblocking
// collective (mpx_i*_enqueue) with those arguments, enqueued on the
// communicator's stream at that point of stream order, so its buffers are
// read and written when the stream reaches the start (§3.4).  A wait on the
// persistent handle completes the active instance and leaves the handle
// inactive but valid for the next start; mpx_request_free releases it.
//
// Handles: a persistent request is MPX_REQUEST_NULL - 1 - k for table slot k
// (every value <= -2), so it never collides with an operation's request
// (non-negative) or with MPX_REQUEST_NULL.  The table is append-only with
// per-slot alive flags; like a stream, a persistent request is used by one
// host thread at a time.
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/mpx.h"

extern "C" int mpxi_comm_is_plain(mpx_comm_t c);

namespace {

enum PKind { P_ALLREDUCE, P_BCAST, P_REDUCE, P_ALLGATHER, P_BARRIER };

struct PReq {
  std::atomic<int> alive{0};
  int kind = 0;
  const void* sendbuf = nullptr;
  void* recvbuf = nullptr;
  int64_t count = 0;
  mpx_datatype_t dt = 0;
  int op = 0;
  int root = 0;
  mpx_comm_t comm = nullptr;
  mpx_request_t active = MPX_REQUEST_NULL;  // the started instance, or NULL when inactive
};

constexpr int kMaxPersistent = 1 << 16;
PReq g_preq[kMaxPersistent];
std::mutex g_preq_mu;
int g_preq_next = 0;
std::vector<int> g_preq_free;

PReq* lookup(mpx_request_t h) {
  if (h > -2) return nullptr;
  const int64_t k = -2 - h;
  if (k >= kMaxPersistent) return nullptr;
  PReq* p = &g_preq[k];
  return p->alive.load(std::memory_order_acquire) ? p : nullptr;
}

int create(const PReq& args, mpx_request_t* out) {
  if (!out) return MPX_ERR_ARG;
  if (!args.comm) return MPX_ERR_COMM;
  if (mpxi_comm_is_plain(args.comm)) return MPX_ERR_UNSUPPORTED;  // no nonblocking collectives there
  int rc;
  if (args.count < 0) return MPX_ERR_ARG;
  if (args.kind != P_BARRIER && (args.dt < 0 || args.dt > MPX_DOUBLE)) return MPX_ERR_TYPE;
  if ((args.kind == P_ALLREDUCE || args.kind == P_REDUCE) && args.op != MPX_SUM) return MPX_ERR_ARG;
  int size = 0;
  rc = mpx_comm_size(args.comm, &size);
  if (rc) return rc;
  if ((args.kind == P_BCAST || args.kind == P_REDUCE) && (args.root < 0 || args.root >= size))
    return MPX_ERR_RANK;
  std::lock_guard<std::mutex> g(g_preq_mu);
  int k;
  if (!g_preq_free.empty()) {
    k = g_preq_free.back();
    g_preq_free.pop_back();
  } else {
    if (g_preq_next >= kMaxPersistent) return MPX_ERR_NO_MEM;
    k = g_preq_next++;
  }
  PReq& p = g_preq[k];
  p.kind = args.kind;
  p.sendbuf = args.sendbuf;
  p.recvbuf = args.recvbuf;
  p.count = args.count;
  p.dt = args.dt;
  p.op = args.op;
  p.root = args.root;
  p.comm = args.comm;
  p.active = MPX_REQUEST_NULL;
  p.alive.store(1, std::memory_order_release);
  *out = (mpx_request_t)(-2 - (int64_t)k);
  return MPX_SUCCESS;
}

int start_one(PReq* p) {
  if (p->active != MPX_REQUEST_NULL) return MPX_ERR_STATE;  // MPI: starting an active request
  mpx_request_t r = MPX_REQUEST_NULL;
  int rc;
  switch (p->kind) {
    case P_ALLREDUCE:
      rc = mpx_iallreduce_enqueue(p->sendbuf, p->recvbuf, p->count, p->dt, p->op, p->comm, &r);
      break;
    case P_BCAST: rc = mpx_ibcast_enqueue(p->recvbuf, p->count, p->dt, p->root, p->comm, &r); break;
    case P_REDUCE:
      rc = mpx_ireduce_enqueue(p->sendbuf, p->recvbuf, p->count, p->dt, p->op, p->root, p->comm, &r);
      break;
    case P_ALLGATHER: rc = mpx_iallgather_enqueue(p->sendbuf, p->recvbuf, p->count, p->dt, p->comm, &r); break;
    default: rc = mpx_ibarrier_enqueue(p->comm, &r); break;
  }
  if (rc == MPX_SUCCESS) p->active = r;
  return rc;
}

}  // namespace

// Wait support for the host runtime: the request a persistent handle stands
// for (MPX_REQUEST_NULL when inactive), and its return to inactive.
extern "C" int mpxi_persist_active(mpx_request_t h, mpx_request_t* active) {
  PReq* p = lookup(h);
  if (!p) return MPX_ERR_REQUEST;
  *active = p->active;
  return MPX_SUCCESS;
}

extern "C" void mpxi_persist_complete(mpx_request_t h) {
  PReq* p = lookup(h);
  if (p) p->active = MPX_REQUEST_NULL;
}

extern "C" int mpx_allreduce_init(const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t dt,
                                  int op, mpx_comm_t comm, mpx_request_t* request) {
  PReq a;
  a.kind = P_ALLREDUCE;
  a.sendbuf = sendbuf;
  a.recvbuf = recvbuf;
  a.count = count;
  a.dt = dt;
  a.op = op;
  a.comm = comm;
  return create(a, request);
}

extern "C" int mpx_bcast_init(void* buf, int64_t count, mpx_datatype_t dt, int root, mpx_comm_t comm,
                              mpx_request_t* request) {
  PReq a;
  a.kind = P_BCAST;
  a.recvbuf = buf;
  a.count = count;
  a.dt = dt;
  a.root = root;
  a.comm = comm;
  return create(a, request);
}

extern "C" int mpx_reduce_init(const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t dt,
                               int op, int root, mpx_comm_t comm, mpx_request_t* request) {
  PReq a;
  a.kind = P_REDUCE;
  a.sendbuf = sendbuf;
  a.recvbuf = recvbuf;
  a.count = count;
  a.dt = dt;
  a.op = op;
  a.root = root;
  a.comm = comm;
  return create(a, request);
}

extern "C" int mpx_allgather_init(const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t dt,
                                  mpx_comm_t comm, mpx_request_t* request) {
  PReq a;
  a.kind = P_ALLGATHER;
  a.sendbuf = sendbuf;
  a.recvbuf = recvbuf;
  a.count = count;
  a.dt = dt;
  a.comm = comm;
  return create(a, request);
}

extern "C" int mpx_barrier_init(mpx_comm_t comm, mpx_request_t* request) {
  PReq a;
  a.kind = P_BARRIER;
  a.comm = comm;
  return create(a, request);
}

extern "C" int mpx_start_enqueue(mpx_request_t* request) {
  if (!request) return MPX_ERR_ARG;
  PReq* p = lookup(*request);
  if (!p) return MPX_ERR_REQUEST;
  return start_one(p);
}

extern "C" int mpx_startall_enqueue(int n, mpx_request_t requests[]) {
  if (n < 0 || (n > 0 && !requests)) return MPX_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!lookup(requests[i])) return MPX_ERR_REQUEST;
  for (int i = 0; i < n; ++i) {
    const int rc = start_one(lookup(requests[i]));
    if (rc) return rc;
  }
  return MPX_SUCCESS;
}

extern "C" int mpx_request_free(mpx_request_t* request) {
  if (!request) return MPX_ERR_ARG;
  PReq* p = lookup(*request);
  if (!p) return MPX_ERR_REQUEST;  // only persistent requests are freed; others complete by a wait
  if (p->active != MPX_REQUEST_NULL) return MPX_ERR_PENDING;
  std::lock_guard<std::mutex> g(g_preq_mu);
  p->alive.store(0, std::memory_order_release);
  g_preq_free.push_back((int)(-2 - *request));
  *request = MPX_REQUEST_NULL;
  return MPX_SUCCESS;
}
