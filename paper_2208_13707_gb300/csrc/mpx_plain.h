// Plain path of libmpx: host matching, one cudaMemcpyAsync or one kernel per
// operation, a host synchronization at every blocking call and wait.  It is the
// baseline the device engine is measured against (MPX_ENGINE_PLAIN).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpx.h"

namespace plain {

struct PlainWorld;

PlainWorld* create(int nranks, int max_streams, int64_t staging_bytes);
void destroy(PlainWorld* pw);
void set_world_index(PlainWorld* pw, int widx);
int progress(PlainWorld* pw);
int error(PlainWorld* pw);
int64_t counter(PlainWorld* pw, int i);
int stream_create(PlainWorld* pw, int id, int rank, cudaStream_t cs, bool exclusive);
void stream_free(PlainWorld* pw, int id);
int64_t stream_pending(PlainWorld* pw, int id);
int stream_error(PlainWorld* pw, int id);
void comm_create(PlainWorld* pw, int comm);
// kind: mpxi::K_SEND/K_RECV/K_ISEND/K_IRECV
int p2p(PlainWorld* pw, uint32_t kind, const void* buf, int64_t count, mpx_datatype_t dt, int peer,
        int tag, int comm, int rank, int stream_id, mpx_status_t* status, mpx_request_t* req);
int wait(PlainWorld* pw, int stream_id, int n, const mpx_request_t* reqs, mpx_status_t* statuses);
int allreduce(PlainWorld* pw, const void* sendbuf, void* recvbuf, int64_t count, mpx_datatype_t dt,
              int mode, int comm, int rank, int stream_id);

}  // namespace plain
