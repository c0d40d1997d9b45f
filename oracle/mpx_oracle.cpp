/*
 * CPU oracle for stream-enqueued MPI point-to-point and allreduce semantics.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file.  It shares no code, header or constant
 * table with the CUDA library; it is a plain, single-threaded, deliberately
 * slow restatement of what an enqueued traffic program computes.
 *
 * What it follows (MPIX Stream paper, Zhou et al., EuroMPI/USA'22):
 *  - §2.1: MPI is an outcome-dictated serial model.  Delivery order is not an
 *    outcome; matching order is: two sends from one sender that both match a
 *    receive are matched in issue order (non-overtaking).  Matching is
 *    independent per communicator.
 *  - §3.1: an MPIX stream is a local serial execution context.
 *  - §3.3: a stream communicator binds one stream per process (here: per
 *    virtual rank); operations on it run in that stream's order.
 *  - §3.4: an enqueued operation processes its buffer only after the
 *    operations enqueued before it on the same stream have completed; an
 *    Isend/Irecv lets later enqueued work go on until the matching Wait;
 *    data received is visible to work enqueued after the completing call.
 *  - §3.4 (last paragraph): collectives take the same enqueue form; here
 *    SUM allreduce, bcast, reduce and allgather, blocking or nonblocking.  A
 *    nonblocking one lets the stream go on at once and completes through a
 *    wait; as in MPI it never forms an instance with a blocking call.
 *  - §3.5: a multiplex stream communicator attaches several local streams
 *    per process, addressed by index; a send names its own stream (src_idx)
 *    and the destination's (dst_idx), a receive its own stream (dst_idx) and
 *    the sender's (src_idx, or any index).  A communicator with one stream
 *    per rank is the case where every index is 0, so one rule covers both:
 *    matching is per (comm, destination rank, destination index), and a
 *    receive accepts a sender whose rank and index both fit its pattern.
 *
 * Readings where the paper is silent:
 *  - Posting is logical and proceeds in rounds.  In round k every stream, in
 *    ascending stream id g, advances past each operation that is not blocked;
 *    sends and receives it passes are posted with key (k, g, program index).
 *    Posts are then matched in ascending key order: a send takes the first
 *    posted receive of its (comm, destination) domain whose source and tag
 *    accept it, a receive takes the first unexpected send of its domain that it
 *    accepts.  Completions made in round k unblock streams in round k+1.
 *  - Sends are eager: a send completes when posted and its bytes are taken at
 *    that moment.
 *  - A receive shorter than the message takes its capacity and reports
 *    TRUNCATE; bytes are matched regardless of datatype signature.
 *  - Allreduce FIXED mode is the left fold (((x0+x1)+x2)+...) in the element
 *    type with round-to-nearest and no contraction; integer sums wrap.  TREE
 *    mode leaves the summation order to the implementation; this oracle
 *    writes the double-precision rank-order sum rounded once, and the tests
 *    bound the difference.
 *  - The user compute op AXPY (Listing 4's saxpy) is y = a*x + y with a
 *    single rounding (fused multiply-add).
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <list>
#include <map>
#include <tuple>
#include <utility>
#include <vector>

namespace {

enum Kind { SEND = 0, RECV, ISEND, IRECV, WAIT, WAITALL, ALLREDUCE, AXPY, BCAST, REDUCE, ALLGATHER,
            IALLREDUCE, IBCAST, IREDUCE, IALLGATHER };
// nonblocking collectives: the call returns a request at once, a wait completes it
bool is_nonblocking_collective(int k) { return k >= IALLREDUCE && k <= IALLGATHER; }
// the blocking kind a collective computes like
int collective_base(int k) {
  switch (k) {
    case IALLREDUCE: return ALLREDUCE;
    case IBCAST: return BCAST;
    case IREDUCE: return REDUCE;
    case IALLGATHER: return ALLGATHER;
    default: return k;
  }
}
bool is_collective(int k) {
  const int b = collective_base(k);
  return b == ALLREDUCE || b == BCAST || b == REDUCE || b == ALLGATHER;
}
constexpr int kAnySource = -2;
constexpr int kAnyTag = -1;
constexpr int kAnyIndex = -1;
constexpr int kInPlace = -3;
constexpr int kErrTruncate = 15;
enum BasicType { T_BYTE = 0, T_INT32, T_INT64, T_FLOAT, T_DOUBLE };
enum Mode { FIXED = 0, TREE = 1 };

struct Op {
  int32_t stream, kind, comm, peer, tag, type;
  int64_t count;
  int32_t buf, buf2;
  int64_t off, off2;
  int32_t req_lo, req_n, status, mode;
  float alpha;
  int32_t sidx, didx;  // multiplex comm: sender's / receiver's local stream index
  int32_t pad;
};
static_assert(sizeof(Op) == 88, "op record is 88 bytes");

struct Type {
  int32_t kind, base, elem, vcount, blocklen, stride;
};
static_assert(sizeof(Type) == 24, "type record is 24 bytes");

struct Status {
  int32_t source, tag, error, source_index;
  int64_t bytes;
};
static_assert(sizeof(Status) == 24, "status record is 24 bytes");

}  // namespace

extern "C" {

struct OracleProgram {
  int32_t nranks, nstreams, ncomms, ntypes;
  int64_t nops, nbufs, nreq, nstatus;
  const int32_t* stream_rank;   // [nstreams]
  const int32_t* comm_stream;   // [ncomms * nranks]: stream of rank r in comm c
  const int64_t* stream_op_lo;  // [nstreams + 1]: ops of stream g are [lo[g], lo[g+1])
  const Op* ops;                // [nops]
  const Type* types;            // [ntypes]
  uint8_t* const* bufs;         // [nbufs] mutated in place
  const int64_t* buf_size;      // [nbufs]
  const int64_t* reqlist;       // [nreq]
  // multiplex comms (§3.5): the local streams of rank r in comm c are
  // mux_stream[mux_off[c * nranks + r] .. mux_off[c * nranks + r + 1]);
  // an empty range marks a comm with one stream per rank.  Both may be null.
  const int64_t* mux_off;       // [ncomms * nranks + 1]
  const int32_t* mux_stream;
};

struct OracleResult {
  int64_t* match;       // [nops] partner op of a send/receive, or -1
  int32_t* post_round;  // [nops]
  int32_t* done_round;  // [nops]
  Status* status;       // [nstatus]
  int32_t* stuck_op;    // [nstreams] op under the cursor at a deadlock, or -1
  int32_t rounds, deadlock, error, pad;
};

}  // extern "C"

namespace {

struct Layout {
  int64_t elem, vcount, blocklen, stride, extent, size;
};

Layout layout_of(const OracleProgram& p, int t) {
  const Type& ty = p.types[t];
  Layout L;
  L.elem = ty.elem;
  if (ty.kind == 0) {
    L.vcount = 1; L.blocklen = 1; L.stride = 1;
  } else {
    L.vcount = ty.vcount; L.blocklen = ty.blocklen; L.stride = ty.stride;
  }
  // MPI_Type_vector: block b, element j of instance i sits at
  // i*extent + (b*stride + j)*elem, extent = ((vcount-1)*stride + blocklen)*elem.
  L.extent = ((L.vcount - 1) * L.stride + L.blocklen) * L.elem;
  L.size = L.vcount * L.blocklen * L.elem;
  return L;
}

// Byte offset (from the buffer start) of the p-th byte of the packed stream.
int64_t packed_byte_offset(const Layout& L, int64_t p) {
  int64_t e = p / L.elem;
  int64_t within = p % L.elem;
  int64_t per_inst = L.vcount * L.blocklen;
  int64_t i = e / per_inst;
  int64_t rem = e % per_inst;
  int64_t b = rem / L.blocklen;
  int64_t j = rem % L.blocklen;
  return i * L.extent + (b * L.stride + j) * L.elem + within;
}

struct Oracle {
  const OracleProgram& p;
  OracleResult& r;
  int err = 0;

  // per-op state
  std::vector<std::vector<uint8_t>> snapshot;  // eager send payloads
  std::vector<Status> op_status;               // status of completed receives
  std::vector<int32_t> op_rank;                // comm rank of the issuing stream
  std::vector<int32_t> op_index;               // its local stream index in the comm
  // matching domains, one per (comm, destination rank, destination index)
  using Domain = std::tuple<int, int, int>;
  std::map<Domain, std::list<int64_t>> posted;      // receives waiting, in post order
  std::map<Domain, std::list<int64_t>> unexpected;  // sends waiting, in post order
  // collectives: per (comm, rank) next instance; per (comm, instance) arrivals
  std::vector<int64_t> next_instance;
  std::map<std::pair<int, int64_t>, std::vector<int64_t>> instances;

  Oracle(const OracleProgram& prog, OracleResult& res) : p(prog), r(res) {}

  int rank_in_comm(int c, int g) const {
    for (int k = 0; k < p.nranks; ++k)
      if (p.comm_stream[(int64_t)c * p.nranks + k] == g) return k;
    return -1;
  }

  // streams rank r attached to multiplex comm c (0: not a multiplex comm)
  int64_t mux_count(int c, int r) const {
    if (!p.mux_off) return 0;
    const int64_t i = (int64_t)c * p.nranks + r;
    return p.mux_off[i + 1] - p.mux_off[i];
  }
  bool is_mux(int c) const {
    for (int r = 0; r < p.nranks; ++r)
      if (mux_count(c, r) > 0) return true;
    return false;
  }
  // (rank, index) of stream g in comm c; rank -1 when g is not a member
  std::pair<int, int> member(int c, int g) const {
    if (!is_mux(c)) return {rank_in_comm(c, g), 0};
    for (int r = 0; r < p.nranks; ++r) {
      const int64_t a = p.mux_off[(int64_t)c * p.nranks + r];
      for (int64_t k = 0; k < mux_count(c, r); ++k)
        if (p.mux_stream[a + k] == g) return {r, (int)k};
    }
    return {-1, 0};
  }
  // how many streams a rank attached (1 on a plain stream comm)
  int64_t streams_of(int c, int r) const { return is_mux(c) ? mux_count(c, r) : 1; }

  bool in_bounds(int buf, int64_t off, int64_t nbytes_span) const {
    if (nbytes_span == 0) return true;  // nothing is read or written (MPI: count 0)
    if (buf < 0 || buf >= p.nbufs) return false;
    return off >= 0 && off + nbytes_span <= p.buf_size[buf];
  }

  // address of a buffer offset; null for a buffer id that names none, which
  // callers reach only for spans of zero bytes (MPI: a count of 0 moves nothing)
  uint8_t* at(int buf, int64_t off) const {
    return buf >= 0 && buf < p.nbufs ? p.bufs[buf] + off : nullptr;
  }

  // bytes spanned in memory by `count` instances of layout L
  static int64_t span(const Layout& L, int64_t count) {
    return count <= 0 ? 0 : (count - 1) * L.extent + L.extent;
  }

  std::vector<uint8_t> pack(int buf, int64_t off, int type, int64_t count) {
    Layout L = layout_of(p, type);
    int64_t n = L.size * count;
    std::vector<uint8_t> out((size_t)n);
    if (n == 0) return out;
    if (!in_bounds(buf, off, span(L, count))) { err = 2; return out; }
    const uint8_t* base = p.bufs[buf] + off;
    for (int64_t q = 0; q < n; ++q) out[(size_t)q] = base[packed_byte_offset(L, q)];
    return out;
  }

  void unpack(const std::vector<uint8_t>& data, int64_t n, int buf, int64_t off, int type,
              int64_t count) {
    Layout L = layout_of(p, type);
    if (count == 0) return;
    if (!in_bounds(buf, off, span(L, count))) { err = 3; return; }
    uint8_t* base = p.bufs[buf] + off;
    for (int64_t q = 0; q < n; ++q) base[packed_byte_offset(L, q)] = data[(size_t)q];
  }

  static bool accepts(const Op& recv, int src_rank, int src_index, int tag) {
    bool src_ok = recv.peer == kAnySource || recv.peer == src_rank;
    bool idx_ok = recv.sidx == kAnyIndex || recv.sidx == src_index;
    bool tag_ok = recv.tag == kAnyTag || recv.tag == tag;
    return src_ok && idx_ok && tag_ok;
  }

  void deliver(int64_t s, int64_t q, int round) {
    const Op& so = p.ops[s];
    const Op& ro = p.ops[q];
    const std::vector<uint8_t>& data = snapshot[(size_t)s];
    int64_t sent = (int64_t)data.size();
    int64_t cap = layout_of(p, ro.type).size * ro.count;
    int64_t n = sent < cap ? sent : cap;
    unpack(data, n, ro.buf, ro.off, ro.type, ro.count);
    r.match[s] = q;
    r.match[q] = s;
    r.done_round[q] = round;
    Status st{};
    st.source = op_rank[(size_t)s];
    st.source_index = op_index[(size_t)s];
    st.tag = so.tag;
    st.error = sent > cap ? kErrTruncate : 0;
    st.bytes = n;
    op_status[(size_t)q] = st;
    if (ro.kind == RECV && ro.status >= 0) r.status[ro.status] = st;
  }

  void match_send(int64_t s, int round) {
    const Op& so = p.ops[s];
    const Domain d{so.comm, so.peer, so.didx};
    auto& lst = posted[d];
    for (auto it = lst.begin(); it != lst.end(); ++it) {
      if (accepts(p.ops[*it], op_rank[(size_t)s], op_index[(size_t)s], so.tag)) {
        int64_t q = *it;
        lst.erase(it);
        deliver(s, q, round);
        return;
      }
    }
    unexpected[d].push_back(s);
  }

  void match_recv(int64_t q, int round) {
    const Op& ro = p.ops[q];
    const Domain d{ro.comm, op_rank[(size_t)q], op_index[(size_t)q]};
    auto& lst = unexpected[d];
    for (auto it = lst.begin(); it != lst.end(); ++it) {
      const Op& so = p.ops[*it];
      if (accepts(ro, op_rank[(size_t)*it], op_index[(size_t)*it], so.tag)) {
        int64_t s = *it;
        lst.erase(it);
        deliver(s, q, round);
        return;
      }
    }
    posted[d].push_back(q);
  }

  void run_axpy(const Op& o) {
    int64_t n = o.count;
    if (!in_bounds(o.buf, o.off, 4 * n) || !in_bounds(o.buf2, o.off2, 4 * n)) { err = 4; return; }
    const uint8_t* xb = p.bufs[o.buf] + o.off;
    uint8_t* yb = p.bufs[o.buf2] + o.off2;
    for (int64_t i = 0; i < n; ++i) {
      float x, y;
      std::memcpy(&x, xb + 4 * i, 4);
      std::memcpy(&y, yb + 4 * i, 4);
      y = std::fma(o.alpha, x, y);
      std::memcpy(yb + 4 * i, &y, 4);
    }
  }

  template <typename T>
  static T load(const uint8_t* b, int64_t i) { T v; std::memcpy(&v, b + sizeof(T) * i, sizeof(T)); return v; }
  template <typename T>
  static void store(uint8_t* b, int64_t i, T v) { std::memcpy(b + sizeof(T) * i, &v, sizeof(T)); }

  // SUM over the R arrivals of one allreduce instance; writes every receive buffer.
  // The k-th collective call on a communicator from every rank forms one
  // instance (§3.4: collectives take the enqueue form; MPI: collective calls
  // on a communicator are ordered).  All arrivals must be the same kind.
  void run_collective(const std::vector<int64_t>& arr, int round) {
    const int call = p.ops[arr[0]].kind;
    for (int64_t j : arr)
      if (p.ops[j].kind != call) { err = 5; return; }
    const int kind = collective_base(call);
    if (kind == ALLREDUCE) run_allreduce(arr, round);
    else if (kind == REDUCE) run_allreduce(arr, round, p.ops[arr[0]].peer);
    else if (kind == BCAST) run_bcast(arr, round);
    else run_allgather(arr, round);
  }

  // MPI_Bcast: the root's count elements replace every other rank's buffer.
  void run_bcast(const std::vector<int64_t>& arr, int round) {
    const Op& o0 = p.ops[arr[0]];
    const int64_t n = o0.count;
    for (int64_t j : arr) {
      const Op& o = p.ops[j];
      if (o.count != n || o.type != o0.type || o.peer != o0.peer) { err = 5; return; }
    }
    const int64_t bytes = p.types[o0.type].elem * n;
    const Op& root = p.ops[arr[(size_t)o0.peer]];
    if (!in_bounds(root.buf, root.off, bytes)) { err = 6; return; }
    for (size_t k = 0; k < arr.size(); ++k) {
      if ((int)k == o0.peer) continue;
      const Op& o = p.ops[arr[k]];
      if (!in_bounds(o.buf, o.off, bytes)) { err = 6; return; }
      if (bytes) std::memcpy(at(o.buf, o.off), at(root.buf, root.off), (size_t)bytes);
    }
    for (int64_t j : arr) r.done_round[j] = round;
  }

  // MPI_Allgather: rank s's count elements land at block s of every rank's
  // receive buffer (in place: rank s's block is already there).
  void run_allgather(const std::vector<int64_t>& arr, int round) {
    const Op& o0 = p.ops[arr[0]];
    const int64_t n = o0.count;
    for (int64_t j : arr) {
      const Op& o = p.ops[j];
      if (o.count != n || o.type != o0.type) { err = 5; return; }
    }
    const size_t R = arr.size();
    const int64_t bytes = p.types[o0.type].elem * n;
    std::vector<std::vector<uint8_t>> block(R);
    for (size_t s = 0; s < R; ++s) {  // read every contribution before writing any
      const Op& o = p.ops[arr[s]];
      const int sb = o.buf == kInPlace ? o.buf2 : o.buf;
      const int64_t so = o.buf == kInPlace ? o.off2 + (int64_t)s * bytes : o.off;
      if (!in_bounds(sb, so, bytes)) { err = 6; return; }
      if (bytes) block[s].assign(at(sb, so), at(sb, so) + bytes);
    }
    for (size_t k = 0; k < R; ++k) {
      const Op& o = p.ops[arr[k]];
      if (!in_bounds(o.buf2, o.off2, bytes * (int64_t)R)) { err = 6; return; }
      for (size_t s = 0; s < R; ++s)
        if (bytes) std::memcpy(at(o.buf2, o.off2) + (int64_t)s * bytes, block[s].data(), (size_t)bytes);
    }
    for (int64_t j : arr) r.done_round[j] = round;
  }

  // MPI_Allreduce (root < 0) or MPI_Reduce to `root`: the SUM is written to
  // every rank's receive buffer, or to the root's only.
  void run_allreduce(const std::vector<int64_t>& arr, int round, int root = -1) {
    const Op& o0 = p.ops[arr[0]];
    int64_t n = o0.count;
    int type = o0.type;
    int mode = o0.mode;
    for (int64_t j : arr) {
      const Op& o = p.ops[j];
      if (o.count != n || o.type != type || o.mode != mode) { err = 5; return; }
    }
    int64_t esz = p.types[type].elem;
    size_t R = arr.size();
    std::vector<const uint8_t*> in(R);
    std::vector<uint8_t*> out(R);
    for (size_t k = 0; k < R; ++k) {
      const Op& o = p.ops[arr[k]];
      if (root >= 0 && o.peer != root) { err = 5; return; }
      const bool writes = root < 0 || (int)k == root;
      int sb = o.buf == kInPlace ? o.buf2 : o.buf;
      int64_t so = o.buf == kInPlace ? o.off2 : o.off;
      if (!in_bounds(sb, so, esz * n) || (writes && !in_bounds(o.buf2, o.off2, esz * n))) { err = 6; return; }
      in[k] = at(sb, so);
      out[k] = writes ? at(o.buf2, o.off2) : nullptr;
    }
    // inputs are read in full before any output is written (a root reducing
    // in place reads its own receive buffer)
    std::vector<std::vector<uint8_t>> copy(R);
    for (size_t k = 0; k < R; ++k) {
      copy[k].assign(in[k], in[k] + esz * n);
      in[k] = copy[k].data();
    }
    // non-writing ranks store into a scratch row
    std::vector<uint8_t> scratch((size_t)(esz * n));
    for (size_t k = 0; k < R; ++k)
      if (!out[k]) out[k] = scratch.data();
    for (int64_t i = 0; i < n; ++i) {
      switch (type) {
        case T_BYTE: {
          uint8_t acc = load<uint8_t>(in[0], i);
          for (size_t k = 1; k < R; ++k) acc = (uint8_t)(acc + load<uint8_t>(in[k], i));
          for (size_t k = 0; k < R; ++k) store<uint8_t>(out[k], i, acc);
          break;
        }
        case T_INT32: {
          uint32_t acc = load<uint32_t>(in[0], i);
          for (size_t k = 1; k < R; ++k) acc += load<uint32_t>(in[k], i);
          for (size_t k = 0; k < R; ++k) store<uint32_t>(out[k], i, acc);
          break;
        }
        case T_INT64: {
          uint64_t acc = load<uint64_t>(in[0], i);
          for (size_t k = 1; k < R; ++k) acc += load<uint64_t>(in[k], i);
          for (size_t k = 0; k < R; ++k) store<uint64_t>(out[k], i, acc);
          break;
        }
        case T_FLOAT: {
          float res;
          if (mode == FIXED) {
            float acc = load<float>(in[0], i);
            for (size_t k = 1; k < R; ++k) acc = acc + load<float>(in[k], i);
            res = acc;
          } else {
            double acc = 0.0;
            for (size_t k = 0; k < R; ++k) acc += (double)load<float>(in[k], i);
            res = (float)acc;
          }
          for (size_t k = 0; k < R; ++k) store<float>(out[k], i, res);
          break;
        }
        case T_DOUBLE: {
          double acc = load<double>(in[0], i);
          for (size_t k = 1; k < R; ++k) acc = acc + load<double>(in[k], i);
          for (size_t k = 0; k < R; ++k) store<double>(out[k], i, acc);
          break;
        }
        default:
          err = 7;
          return;
      }
    }
    for (int64_t j : arr) r.done_round[j] = round;
  }

  // Arguments an enqueue call would reject up front.
  bool valid(const Op& o, int64_t j) const {
    bool p2p = o.kind == SEND || o.kind == ISEND || o.kind == RECV || o.kind == IRECV;
    if (p2p || is_collective(o.kind)) {
      if (o.comm < 0 || o.comm >= p.ncomms || op_rank[(size_t)j] < 0) return false;
      if (o.type < 0 || o.type >= p.ntypes || o.count < 0) return false;
    }
    // a multiplex comm carries point-to-point traffic only (§3.5)
    if (is_collective(o.kind)) {
      const int b = collective_base(o.kind);
      return !is_mux(o.comm) && (b == ALLREDUCE || b == ALLGATHER || (o.peer >= 0 && o.peer < p.nranks));
    }
    if (o.kind == SEND || o.kind == ISEND)
      return o.peer >= 0 && o.peer < p.nranks && o.tag >= 0 && o.sidx == op_index[(size_t)j] &&
             o.didx >= 0 && o.didx < streams_of(o.comm, o.peer);
    if (o.kind == RECV || o.kind == IRECV) {
      if (!(o.peer == kAnySource || (o.peer >= 0 && o.peer < p.nranks))) return false;
      if (!(o.tag == kAnyTag || o.tag >= 0) || o.didx != op_index[(size_t)j]) return false;
      if (o.sidx == kAnyIndex) return is_mux(o.comm);  // ANY_INDEX only on a multiplex comm
      if (o.peer != kAnySource) return o.sidx >= 0 && o.sidx < streams_of(o.comm, o.peer);
      int64_t most = 0;
      for (int r = 0; r < p.nranks; ++r) most = std::max(most, streams_of(o.comm, r));
      return o.sidx >= 0 && o.sidx < most;
    }
    if (o.kind == WAIT || o.kind == WAITALL) {
      for (int k = 0; k < o.req_n; ++k) {
        int64_t q = p.reqlist[o.req_lo + k];
        if (q < 0 || q >= p.nops || p.ops[q].stream != o.stream) return false;
      }
    }
    return true;
  }

  bool complete_before(int64_t j, int round) const {
    return r.done_round[j] >= 0 && r.done_round[j] < round;
  }

  void write_wait_status(const Op& w) {
    if (w.status < 0) return;
    for (int k = 0; k < w.req_n; ++k) {
      int64_t q = p.reqlist[w.req_lo + k];
      Status st{};
      int kind = p.ops[q].kind;
      if (kind == IRECV || kind == RECV) {
        st = op_status[(size_t)q];
      } else {
        st.source = kAnySource;  // empty status for send requests
        st.tag = kAnyTag;
        st.error = 0;
        st.bytes = 0;
      }
      r.status[w.status + k] = st;
    }
  }

  int run() {
    const int64_t nops = p.nops;
    snapshot.assign((size_t)nops, {});
    op_status.assign((size_t)nops, Status{});
    op_rank.assign((size_t)nops, -1);
    op_index.assign((size_t)nops, 0);
    for (int64_t j = 0; j < nops; ++j) {
      r.match[j] = -1;
      r.post_round[j] = -1;
      r.done_round[j] = -1;
      const Op& o = p.ops[j];
      if (o.comm >= 0 && o.comm < p.ncomms) {
        const std::pair<int, int> m = member(o.comm, o.stream);
        op_rank[(size_t)j] = m.first;
        op_index[(size_t)j] = m.second;
      }
    }
    for (int64_t s = 0; s < p.nstatus; ++s) r.status[s] = Status{};
    posted.clear();
    unexpected.clear();
    next_instance.assign((size_t)p.ncomms * p.nranks, 0);
    std::vector<int64_t> cursor(p.nstreams);
    for (int g = 0; g < p.nstreams; ++g) cursor[g] = p.stream_op_lo[g];
    r.deadlock = 0;
    int round = 0;
    for (;;) {
      ++round;
      bool progress = false;
      std::vector<int64_t> posts;
      std::vector<std::pair<int, int64_t>> arrived_now;
      for (int g = 0; g < p.nstreams; ++g) {
        const int64_t hi = p.stream_op_lo[g + 1];
        while (cursor[g] < hi && !err) {
          const int64_t j = cursor[g];
          const Op& o = p.ops[j];
          if (!valid(o, j)) { err = 9; break; }
          if (o.kind == SEND || o.kind == ISEND) {
            snapshot[(size_t)j] = pack(o.buf, o.off, o.type, o.count);
            r.post_round[j] = round;
            r.done_round[j] = round;  // eager
            posts.push_back(j);
            ++cursor[g];
            progress = true;
          } else if (o.kind == IRECV) {
            r.post_round[j] = round;
            posts.push_back(j);
            ++cursor[g];
            progress = true;
          } else if (o.kind == RECV) {
            if (r.post_round[j] < 0) {
              r.post_round[j] = round;
              posts.push_back(j);
              progress = true;
              break;
            }
            if (complete_before(j, round)) { ++cursor[g]; progress = true; continue; }
            break;
          } else if (o.kind == WAIT || o.kind == WAITALL) {
            bool all = true;
            for (int k = 0; k < o.req_n; ++k)
              if (!complete_before(p.reqlist[o.req_lo + k], round)) { all = false; break; }
            if (!all) break;
            r.post_round[j] = round;
            r.done_round[j] = round;
            write_wait_status(o);
            ++cursor[g];
            progress = true;
          } else if (is_collective(o.kind)) {
            if (r.post_round[j] < 0) {
              r.post_round[j] = round;
              int rk = op_rank[(size_t)j];
              int64_t k = next_instance[(size_t)o.comm * p.nranks + rk]++;
              auto& v = instances[{o.comm, k}];
              if (v.empty()) v.assign((size_t)p.nranks, -1);
              v[(size_t)rk] = j;
              arrived_now.push_back({o.comm, k});
              progress = true;
              if (is_nonblocking_collective(o.kind)) {  // the stream goes on; a wait completes it
                ++cursor[g];
                continue;
              }
              break;
            }
            if (complete_before(j, round)) { ++cursor[g]; progress = true; continue; }
            break;
          } else if (o.kind == AXPY) {
            run_axpy(o);
            r.post_round[j] = round;
            r.done_round[j] = round;
            ++cursor[g];
            progress = true;
          } else {
            err = 8;
            break;
          }
        }
        if (err) break;
      }
      if (err) break;
      // match this round's posts in ascending post key (round, g, program index)
      for (int64_t j : posts) {
        const Op& o = p.ops[j];
        if (o.kind == SEND || o.kind == ISEND) match_send(j, round);
        else match_recv(j, round);
        if (err) break;
      }
      if (err) break;
      // collectives whose arrivals are all present, in (comm, instance) order
      for (auto& kv : instances) {
        auto& v = kv.second;
        bool full = true, pending = false;
        for (int64_t j : v) {
          if (j < 0) { full = false; break; }
          if (r.done_round[j] < 0) pending = true;
        }
        if (full && pending) run_collective(v, round);
        if (err) break;
      }
      if (err) break;
      bool finished = true;
      for (int g = 0; g < p.nstreams; ++g)
        if (cursor[g] < p.stream_op_lo[g + 1]) finished = false;
      if (finished) break;
      if (!progress) {
        r.deadlock = 1;
        break;
      }
    }
    for (int g = 0; g < p.nstreams; ++g)
      r.stuck_op[g] = cursor[g] < p.stream_op_lo[g + 1] ? (int32_t)cursor[g] : -1;
    r.rounds = round;
    r.error = err;
    return err;
  }
};

}  // namespace

extern "C" {

int oracle_run(const OracleProgram* prog, OracleResult* res) {
  Oracle o(*prog, *res);
  return o.run();
}

// Exact-as-possible reference for a float32 SUM over R inputs: the rank-order
// double sum and the sum of magnitudes, used to bound a tree-order result.
void oracle_sum_f32_ref(int32_t nranks, int64_t n, const float* const* xs, double* sum,
                        double* abssum) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0, a = 0.0;
    for (int k = 0; k < nranks; ++k) {
      double v = (double)xs[k][i];
      s += v;
      a += std::fabs(v);
    }
    sum[i] = s;
    abssum[i] = a;
  }
}

int oracle_abi_version(void) { return 2; }

}  // extern "C"
