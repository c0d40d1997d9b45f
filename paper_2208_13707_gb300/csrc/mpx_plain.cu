// Plain path (see mpx_plain.h).  Filled in below the engine path.
#include "mpx_plain.h"

namespace plain {
struct PlainWorld {
  int nranks;
};
PlainWorld* create(int nranks, int, int64_t) { return new PlainWorld{nranks}; }
void destroy(PlainWorld* pw) { delete pw; }
int progress(PlainWorld*) { return MPX_ERR_UNSUPPORTED; }
int error(PlainWorld*) { return 0; }
int64_t counter(PlainWorld*, int) { return 0; }
int stream_create(PlainWorld*, int, int, cudaStream_t) { return MPX_SUCCESS; }
void stream_free(PlainWorld*, int) {}
int64_t stream_pending(PlainWorld*, int) { return 0; }
int stream_error(PlainWorld*, int) { return 0; }
void comm_create(PlainWorld*, int) {}
int p2p(PlainWorld*, uint32_t, const void*, int64_t, mpx_datatype_t, int, int, int, int, int,
        mpx_status_t*, mpx_request_t*) {
  return MPX_ERR_UNSUPPORTED;
}
int wait(PlainWorld*, int, int, const mpx_request_t*, mpx_status_t*) { return MPX_ERR_UNSUPPORTED; }
int allreduce(PlainWorld*, const void*, void*, int64_t, mpx_datatype_t, int, int, int, int) {
  return MPX_ERR_UNSUPPORTED;
}
}  // namespace plain
