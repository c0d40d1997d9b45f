// Serving loop of libmpx (mpx_serve_run): many host threads, one MPIX stream
// each (the paper's thread-to-endpoint mapping, §3.1), submit enqueue
// requests open-loop; a device-memory budget admits them (continuous
// batching: a request that arrives while others are on the GPU starts as soon
// as completions free enough of the budget); match and queue state stay on
// the device in the resident engine; a reaper thread turns the streams'
// completion words into per-request enqueue-to-complete latencies and
// releases the requests' memory.  The same loop runs over the plain path for
// comparison (there every blocking call synchronizes its host thread).
//
// Workload (one item = one p2p message or one allreduce instance):
//   * every thread makes `requests / nthreads` calls; a share p_allreduce of
//     them are allreduce participations (fp32 SUM over all threads, the same
//     instance list on every thread), the rest are p2p sends and receives;
//   * each message has a uniform source, a uniform other destination and a
//     Zipf(s) power-of-two size; its tag counts the messages of its
//     (source, destination) pair, so matching is exact (no wildcards);
//   * the calls between two allreduce instances form an epoch: a thread
//     isends and irecvs its messages of the epoch in a seeded order, waits
//     for all of them (waitall) and then joins the epoch's allreduce, so no
//     blocking call waits on a message sent after it;
//   * payloads are slices of per-thread source regions filled from a seed;
//     receive and result buffers come from the budget.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mpx.h"

extern "C" uint64_t mpxi_stream_last_seq(mpx_stream_t s);
extern "C" int mpxi_stream_done(mpx_stream_t s, uint64_t* done, uint64_t* done_t);
extern "C" int mpxi_fill(void* p, int64_t bytes, uint64_t seed, int as_f32, void* stream);
extern "C" int mpxi_digest_store(const void* p, int64_t bytes, void* out_mapped, void* stream);
extern "C" int mpxi_clock_probe(void* out_mapped, void* stream);
extern "C" int mpxi_serve_preload(void);

namespace {

uint64_t mix64(uint64_t z) {  // splitmix64 finaliser (Steele, Lea, Flood 2014)
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Rng {  // counter-based: draw k of stream (seed, key) is mix64(seed, key, k)
  uint64_t base, k = 0;
  Rng(uint64_t seed, uint64_t key) : base(mix64(seed ^ mix64(key))) {}
  uint64_t u64() { return mix64(base + 0x9E3779B97F4A7C15ull * ++k); }
  double uniform() { return (double)(u64() >> 11) * (1.0 / 9007199254740992.0); }
  int64_t below(int64_t n) { return (int64_t)(u64() % (uint64_t)n); }
};

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// --- budget: first-fit arena over one thread's share of the device budget --
// Each thread admits its requests against its own share (budget / threads).
// A shared pool could deadlock under overload: threads that ran ahead could
// hold the whole budget with receives of later epochs while a thread still
// needs memory for a receive of the oldest epoch, which the others' later
// requests wait on.  With shares, a thread blocked on admission holds only
// memory of the oldest unfinished epoch and of finished ones being released.
class Budget {
 public:
  void init(uint8_t* base, int64_t bytes) {
    base_ = base;
    cap_ = bytes & ~(int64_t)255;
    free_[0] = cap_;
  }
  // wait until `bytes` fit; false if `stop` was raised meanwhile
  void* admit(int64_t bytes, bool* waited, const std::atomic<bool>& stop) {
    const int64_t need = (std::max<int64_t>(bytes, 1) + 255) & ~(int64_t)255;
    std::unique_lock<std::mutex> g(mu_);
    *waited = false;
    for (;;) {
      for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second < need) continue;
        const int64_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > need) free_[off + need] = len - need;
        used_ += need;
        peak_ = std::max(peak_, used_);
        sizes_[off] = need;
        return base_ + off;
      }
      if (need > cap_ || stop.load()) return nullptr;
      *waited = true;
      cv_.wait_for(g, std::chrono::milliseconds(1));
    }
  }
  void release(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(mu_);
    const int64_t off = (uint8_t*)p - base_;
    auto sz = sizes_.find(off);
    if (sz == sizes_.end()) return;
    int64_t start = off, len = sz->second;
    sizes_.erase(sz);
    used_ -= len;
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + len) {
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = len;
    cv_.notify_all();
  }
  int64_t peak() const { return peak_; }

 private:
  uint8_t* base_ = nullptr;
  int64_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<int64_t, int64_t> free_, sizes_;
  std::mutex mu_;
  std::condition_variable cv_;
};

enum CallKind { C_SEND, C_RECV, C_WAITALL, C_ALLREDUCE };
struct Call {
  int kind;
  int peer;
  int tag;
  int64_t item;
  int64_t bytes;
  int64_t off;           // payload offset in the caller's source region
  int64_t capture = -1;  // caller schedules: capture offset (recv, allreduce) or first status (waitall)
};

struct Rec {  // one request in flight
  int64_t t_arr, t_enq;
  int owner;       // thread whose budget share holds buf
  void* buf;
  int64_t bytes;   // payload delivered by this request (for GB/s)
  int64_t item;    // >= 0: digest this buffer
  int64_t capture; // >= 0: copy the delivered bytes to the capture area here
};
struct Batch {  // requests covered by one blocking operation
  uint64_t seq;
  std::vector<Rec> recs;
  cudaEvent_t digested = nullptr;  // digests and captures done (stream-ordered after seq)
};

struct Shared {
  const mpx_serve_config_t* cfg;
  int T;
  std::vector<std::vector<Call>> calls;
  std::vector<uint8_t*> region;
  int64_t region_bytes = 0;
  int64_t nitems = 0;
  uint8_t* pool = nullptr;       // the whole budget (one allocation)
  std::vector<Budget> budget;    // one share per thread
  std::vector<std::mutex> fmu;
  std::vector<std::deque<Batch>> fifo;
  std::atomic<int> running{0};
  std::atomic<bool> stop{false};
  std::atomic<int> error{0};
  std::atomic<int64_t> waits{0};
  int64_t clock_offset = 0;  // device globaltimer - host steady clock
  uint64_t* digests = nullptr;
  int64_t ndigests = 0;
  uint64_t* dig_host = nullptr;  // mapped pinned digest slots [ndigests]
  uint64_t* dig_dev = nullptr;   // their device address
  uint8_t* capture = nullptr;    // caller schedules: where delivered bytes are copied
  mpx_status_t* statuses = nullptr;  // caller schedules: waitall statuses
  bool own_regions = true;       // regions allocated (and filled) here
  // results, per thread (merged at the end)
  std::vector<std::vector<float>> lat, svc;
  std::vector<int64_t> bytes_done, t_last;
  explicit Shared(int n)
      : budget(n), fmu(n), fifo(n), lat(n + 1), svc(n + 1), bytes_done(n + 1, 0), t_last(n + 1, 0) {}
  ~Shared() {
    if (pool) cudaFree(pool);
  }
  int64_t peak() const {
    int64_t p = 0;
    for (const Budget& b : budget) p += b.peak();
    return p;
  }
};

// Digests of a batch's sampled buffers, enqueued on the client's own stream
// right after the blocking operation that covers them: stream order runs
// them once the data is in place, and nothing else waits on them.  (A reaper
// that launched them on a stream of its own could find that stream's
// hardware queue behind a client stream's unsatisfied wait.)
void enqueue_digests(Shared& S, Batch& b, cudaStream_t cs) {
  bool any = false;
  for (const Rec& r : b.recs) {
    if (r.capture >= 0 && S.capture && r.buf && r.bytes > 0) {
      cudaMemcpyAsync(S.capture + r.capture, r.buf, (size_t)r.bytes, cudaMemcpyDeviceToDevice, cs);
      any = true;
    }
    if (r.item < 0 || !S.dig_dev || r.item >= S.ndigests || !r.buf) continue;
    mpxi_digest_store(r.buf, r.bytes, S.dig_dev + r.item, cs);
    any = true;
  }
  if (any && cudaEventCreateWithFlags(&b.digested, cudaEventDisableTiming) == cudaSuccess)
    cudaEventRecord(b.digested, cs);
}

void finish_batch(Shared& S, int slot, Batch& b, int64_t t_c) {
  for (Rec& r : b.recs) {
    S.lat[(size_t)slot].push_back((float)((t_c - r.t_arr) / 1e3));
    S.svc[(size_t)slot].push_back((float)((t_c - r.t_enq) / 1e3));
    S.bytes_done[(size_t)slot] += r.bytes;
    if (r.item >= 0 && S.dig_host && r.item < S.ndigests)
      S.digests[r.item] = *(volatile uint64_t*)&S.dig_host[r.item];
    if (r.buf) S.budget[(size_t)r.owner].release(r.buf);
  }
  if (b.digested) cudaEventDestroy(b.digested);
  b.digested = nullptr;
  S.t_last[(size_t)slot] = std::max(S.t_last[(size_t)slot], t_c);
}

// Build every thread's call list (deterministic in the seed).
void build_schedule(Shared& S) {
  const mpx_serve_config_t& c = *S.cfg;
  const int T = S.T;
  const int64_t per = std::max<int64_t>(1, c.requests / T);
  const int64_t nar = std::llround(c.p_allreduce * (double)per);
  const int64_t p2p_calls = (per - nar) * T;
  const int64_t M = p2p_calls / 2;
  const int nb = c.max_log2 - c.min_log2 + 1;
  std::vector<double> cdf((size_t)nb);
  double z = 0;
  for (int k = 0; k < nb; ++k) z += 1.0 / std::pow((double)(k + 1), c.zipf_s);
  double acc = 0;
  for (int k = 0; k < nb; ++k) {
    acc += 1.0 / std::pow((double)(k + 1), c.zipf_s) / z;
    cdf[(size_t)k] = acc;
  }
  auto zipf_bytes = [&](Rng& r) {
    const double u = r.uniform();
    int k = 0;
    while (k < nb - 1 && u > cdf[(size_t)k]) ++k;
    return (int64_t)1 << (c.min_log2 + k);
  };
  const int64_t maxb = (int64_t)1 << c.max_log2;
  S.region_bytes = 2 * maxb;
  auto slice = [&](uint64_t key, int64_t bytes) {
    const int64_t room = S.region_bytes - bytes + 1;
    return (int64_t)(mix64(c.seed ^ key) % (uint64_t)room) & ~(int64_t)255;
  };
  // messages: (epoch, src, dst, bytes, tag)
  struct Msg { int64_t epoch; int src, dst; int64_t bytes; int tag; };
  std::vector<Msg> msgs((size_t)M);
  std::vector<int> pair_count((size_t)T * T, 0);
  Rng rm(c.seed, 1);
  for (int64_t m = 0; m < M; ++m) {
    Msg& g = msgs[(size_t)m];
    g.src = (int)rm.below(T);
    g.dst = (int)rm.below(T - 1);
    if (g.dst >= g.src) ++g.dst;
    g.epoch = rm.below(nar + 1);
    g.bytes = zipf_bytes(rm);
    g.tag = pair_count[(size_t)g.src * T + g.dst]++;
  }
  std::vector<int64_t> ar_bytes((size_t)nar);
  Rng ra(c.seed, 2);
  for (int64_t e = 0; e < nar; ++e) ar_bytes[(size_t)e] = zipf_bytes(ra) & ~(int64_t)3;
  S.nitems = M + nar;
  // per thread, per epoch: its sends and receives, shuffled; waitall; allreduce
  std::vector<std::vector<std::vector<Call>>> ep((size_t)T, std::vector<std::vector<Call>>((size_t)nar + 1));
  const bool alone = c.only_item >= 0;
  for (int64_t m = 0; m < M; ++m) {
    if (alone && c.only_item != m) continue;
    const Msg& g = msgs[(size_t)m];
    ep[(size_t)g.src][(size_t)g.epoch].push_back(Call{C_SEND, g.dst, g.tag, m, g.bytes, slice((uint64_t)m, g.bytes)});
    ep[(size_t)g.dst][(size_t)g.epoch].push_back(Call{C_RECV, g.src, g.tag, m, g.bytes, 0});
  }
  S.calls.assign((size_t)T, {});
  for (int t = 0; t < T; ++t) {
    Rng rs(c.seed, 100 + (uint64_t)t);
    for (int64_t e = 0; e <= nar; ++e) {
      auto& v = ep[(size_t)t][(size_t)e];
      for (size_t i = v.size(); i > 1; --i) std::swap(v[i - 1], v[(size_t)rs.below((int64_t)i)]);
      for (const Call& x : v) S.calls[(size_t)t].push_back(x);
      if (!v.empty()) S.calls[(size_t)t].push_back(Call{C_WAITALL, 0, 0, -1, 0, 0});
      if (e < nar && (!alone || c.only_item == M + e)) {
        const int64_t b = ar_bytes[(size_t)e];
        S.calls[(size_t)t].push_back(Call{C_ALLREDUCE, 0, 0, M + e, b,
                                          slice(0x5A5A0000ull + (uint64_t)e, b)});
      }
    }
  }
}

struct ThreadCtx {
  int t;
  mpx_stream_t stream;
  mpx_comm_t comm;
  cudaStream_t cs;
};

void client_thread(Shared& S, ThreadCtx ctx, bool plain, int64_t t0) {
  const mpx_serve_config_t& c = *S.cfg;
  const int t = ctx.t;
  Rng arr(c.seed, 200 + (uint64_t)t);
  const bool paced = c.only_item < 0 && c.mean_gap_us > 0;
  int64_t t_arr = t0;
  while (now_ns() < t0) std::this_thread::yield();  // every thread starts together
  std::vector<mpx_request_t> reqs;
  std::vector<Rec> open;
  uint8_t* src = S.region[(size_t)t];
  auto fail = [&](int rc) {
    int z = 0;
    S.error.compare_exchange_strong(z, rc);
    S.stop = true;
  };
  for (const Call& x : S.calls[(size_t)t]) {
    if (S.stop.load()) break;
    if (x.kind != C_WAITALL) {
      if (paced) {
        t_arr += (int64_t)(-std::log(1.0 - arr.uniform()) * c.mean_gap_us * 1e3);
        while (now_ns() < t_arr) std::this_thread::yield();
      } else {
        t_arr = now_ns();
      }
    }
    int rc = MPX_SUCCESS;
    if (x.kind == C_SEND) {
      const int64_t te = now_ns();
      mpx_request_t r = MPX_REQUEST_NULL;
      do rc = mpx_isend_enqueue(src + x.off, x.bytes, MPX_BYTE, x.peer, x.tag, ctx.comm, &r);
      while (rc == MPX_ERR_AGAIN && !S.stop.load());
      if (rc) { fail(rc); break; }
      reqs.push_back(r);
      open.push_back(Rec{t_arr, te, t, nullptr, 0, -1, -1});
    } else if (x.kind == C_RECV) {
      bool waited = false;
      void* buf = S.budget[(size_t)t].admit(x.bytes, &waited, S.stop);
      if (!buf) { fail(MPX_ERR_NO_MEM); break; }
      if (waited) S.waits++;
      const int64_t te = now_ns();
      mpx_request_t r = MPX_REQUEST_NULL;
      do rc = mpx_irecv_enqueue(buf, x.bytes, MPX_BYTE, x.peer, x.tag, ctx.comm, &r);
      while (rc == MPX_ERR_AGAIN && !S.stop.load());
      if (rc) { fail(rc); break; }
      reqs.push_back(r);
      const bool sample = c.only_item >= 0 || (c.sample_every > 0 && x.item % c.sample_every == 0);
      open.push_back(Rec{t_arr, te, t, buf, x.bytes, sample ? x.item : -1, x.capture});
    } else {
      // a blocking call: waitall over the epoch's requests, or an allreduce
      Batch b;
      if (x.kind == C_WAITALL) {
        // engine: MPX_ERR_AGAIN only while the waitlist is full; plain path:
        // until the requests complete (the host thread waits here)
        mpx_status_t* sts = x.capture >= 0 && S.statuses ? S.statuses + x.capture : nullptr;
        do rc = mpx_waitall_enqueue((int)reqs.size(), reqs.data(), sts);
        while (rc == MPX_ERR_AGAIN && !S.stop.load());
        if (rc) { fail(rc); break; }
        b.recs.swap(open);
        reqs.clear();
      } else {
        bool waited = false;
        void* buf = S.budget[(size_t)t].admit(x.bytes, &waited, S.stop);
        if (!buf) { fail(MPX_ERR_NO_MEM); break; }
        if (waited) S.waits++;
        const int64_t te = now_ns();
        const int64_t n = x.bytes / 4;
        do rc = mpx_allreduce_enqueue(src + x.off, buf, n, MPX_FLOAT, MPX_SUM, ctx.comm);
        while (rc == MPX_ERR_AGAIN && !S.stop.load());
        if (rc) { fail(rc); break; }
        const bool sample = t == 0 && (c.only_item >= 0 || (c.sample_every > 0 && x.item % c.sample_every == 0));
        b.recs.push_back(Rec{t_arr, te, t, buf, x.bytes, sample ? x.item : -1, x.capture});
      }
      if (plain) {
        const int64_t t_c = now_ns();  // the blocking call returned: complete
        enqueue_digests(S, b, ctx.cs);
        if (b.digested) cudaEventSynchronize(b.digested);
        finish_batch(S, t, b, t_c);
      } else {
        b.seq = mpxi_stream_last_seq(ctx.stream);
        enqueue_digests(S, b, ctx.cs);
        std::lock_guard<std::mutex> g(S.fmu[(size_t)t]);
        S.fifo[(size_t)t].push_back(std::move(b));
      }
    }
  }
  S.running--;
}

void reaper_thread(Shared& S, std::vector<ThreadCtx>& ctx) {
  const int T = S.T;
  const int slot = T;  // the reaper's result slot
  for (;;) {
    bool pending = false;
    for (int t = 0; t < T; ++t) {
      uint64_t done = 0, done_t = 0;
      mpxi_stream_done(ctx[(size_t)t].stream, &done, &done_t);
      for (;;) {
        Batch b;
        {
          std::lock_guard<std::mutex> g(S.fmu[(size_t)t]);
          auto& q = S.fifo[(size_t)t];
          if (q.empty()) break;
          if (q.front().seq > done ||
              (q.front().digested && cudaEventQuery(q.front().digested) == cudaErrorNotReady)) {
            pending = true;
            break;
          }
          b = std::move(q.front());
          q.pop_front();
        }
        finish_batch(S, slot, b, (int64_t)done_t - S.clock_offset);
      }
    }
    if (!pending && S.running.load() == 0) {
      bool empty = true;
      for (int t = 0; t < T; ++t) {
        std::lock_guard<std::mutex> g(S.fmu[(size_t)t]);
        empty = empty && S.fifo[(size_t)t].empty();
      }
      if (empty) break;
    }
    if (S.stop.load() && S.running.load() == 0) break;
  }
}

double pct(std::vector<float>& v, double q) {
  if (v.empty()) return 0;
  const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
  std::nth_element(v.begin(), v.begin() + (long)k, v.end());
  return v[k];
}

}  // namespace

extern "C" int mpx_serve_config_init(mpx_serve_config_t* c) {
  if (!c) return MPX_ERR_ARG;
  memset(c, 0, sizeof(*c));
  c->nthreads = 32;
  c->engine_mode = MPX_ENGINE_PERSISTENT;
  c->requests = 1000000;
  c->mean_gap_us = 2.0;
  c->zipf_s = 1.2;
  c->min_log2 = 6;
  c->max_log2 = 24;
  c->p_allreduce = 0.3;
  c->budget_bytes = 40ll << 30;
  c->seed = 0x220813707ull + 4;
  c->sample_every = 0;
  c->only_item = -1;
  return MPX_SUCCESS;
}

namespace {

// A caller's schedule into the threads' call lists, every call checked
// against the thread count and the regions, capture and status ranges.
int load_schedule(Shared& S, const mpx_serve_schedule_t& q, int64_t* max_buf) {
  const int T = S.T;
  if (!q.calls || !q.call_lo || !q.regions || q.region_bytes < 0 || q.call_lo[0] != 0) return MPX_ERR_ARG;
  if ((q.capture_bytes > 0 && !q.capture) || (q.nstatuses > 0 && !q.statuses)) return MPX_ERR_ARG;
  S.calls.assign((size_t)T, {});
  S.nitems = 0;
  *max_buf = 0;
  for (int t = 0; t < T; ++t) {
    if (q.call_lo[t + 1] < q.call_lo[t] || !q.regions[t]) return MPX_ERR_ARG;
    int64_t nreq = 0;
    for (int64_t i = q.call_lo[t]; i < q.call_lo[t + 1]; ++i) {
      const mpx_serve_call_t& x = q.calls[i];
      const bool p2p = x.kind == MPX_SERVE_SEND || x.kind == MPX_SERVE_RECV;
      if (x.kind < MPX_SERVE_SEND || x.kind > MPX_SERVE_ALLREDUCE || x.item < 0) return MPX_ERR_ARG;
      if (x.kind != MPX_SERVE_WAITALL && (x.bytes < 0 || x.bytes > q.region_bytes)) return MPX_ERR_ARG;
      if (p2p && (x.peer < 0 || x.peer >= T || x.tag < 0 || x.tag > MPX_TAG_UB)) return MPX_ERR_ARG;
      if ((x.kind == MPX_SERVE_SEND || x.kind == MPX_SERVE_ALLREDUCE) &&
          (x.off < 0 || x.off > q.region_bytes - x.bytes))
        return MPX_ERR_ARG;
      if (x.kind == MPX_SERVE_ALLREDUCE && (x.bytes & 3)) return MPX_ERR_ARG;
      if ((x.kind == MPX_SERVE_RECV || x.kind == MPX_SERVE_ALLREDUCE) && x.capture >= 0 &&
          (!q.capture || x.capture > q.capture_bytes - x.bytes))
        return MPX_ERR_ARG;
      if (x.kind == MPX_SERVE_WAITALL && x.capture >= 0 &&
          (!q.statuses || x.capture > q.nstatuses - nreq))
        return MPX_ERR_ARG;
      if (x.kind == MPX_SERVE_WAITALL) nreq = 0;
      else if (p2p) ++nreq;
      if (x.kind == MPX_SERVE_RECV || x.kind == MPX_SERVE_ALLREDUCE) *max_buf = std::max(*max_buf, x.bytes);
      Call y{x.kind == MPX_SERVE_SEND ? C_SEND : x.kind == MPX_SERVE_RECV ? C_RECV
             : x.kind == MPX_SERVE_WAITALL ? C_WAITALL : C_ALLREDUCE,
             x.peer, x.tag, x.item, x.bytes, x.off};
      y.capture = x.capture;
      S.calls[(size_t)t].push_back(y);
      S.nitems = std::max(S.nitems, x.item + 1);
    }
  }
  S.region_bytes = q.region_bytes;
  S.region.assign((size_t)T, nullptr);
  for (int t = 0; t < T; ++t) S.region[(size_t)t] = (uint8_t*)q.regions[t];
  S.own_regions = false;
  S.capture = (uint8_t*)q.capture;
  S.statuses = q.statuses;
  return MPX_SUCCESS;
}

int serve(const mpx_serve_config_t* cfg, const mpx_serve_schedule_t* sched, mpx_serve_result_t* res,
          uint64_t* digests, uint64_t* source_digests, int64_t ndigests) {
  if (!cfg || !res) return MPX_ERR_ARG;
  const mpx_serve_config_t& c = *cfg;
  if (c.nthreads < 2 || c.nthreads > 1024 || c.budget_bytes <= 0 ||
      (c.engine_mode != MPX_ENGINE_PERSISTENT && c.engine_mode != MPX_ENGINE_PLAIN))
    return MPX_ERR_ARG;
  if (!sched && (c.requests < 1 || c.min_log2 < 2 || c.max_log2 < c.min_log2 || c.max_log2 > 30 ||
                 c.p_allreduce < 0 || c.p_allreduce > 1))
    return MPX_ERR_ARG;
  memset(res, 0, sizeof(*res));
  const int T = c.nthreads;
  const bool plain = c.engine_mode == MPX_ENGINE_PLAIN;
  Shared S(T);
  S.cfg = cfg;
  S.T = T;
  S.digests = digests;
  S.ndigests = ndigests;
  int64_t max_buf = 0;
  if (sched) {
    const int lrc = load_schedule(S, *sched, &max_buf);
    if (lrc) return lrc;
  } else {
    max_buf = (int64_t)1 << c.max_log2;
    build_schedule(S);
  }
  res->items = S.nitems;
  if (mpxi_serve_preload()) return MPX_ERR_CUDA;
  struct HostSlots {
    uint64_t* p = nullptr;
    ~HostSlots() {
      if (p) cudaFreeHost(p);
    }
  } slots;
  if (digests && ndigests > 0) {
    if (cudaHostAlloc((void**)&slots.p, (size_t)ndigests * 8, cudaHostAllocMapped) != cudaSuccess)
      return MPX_ERR_NO_MEM;
    memset(slots.p, 0, (size_t)ndigests * 8);
    void* dp = nullptr;
    cudaHostGetDevicePointer(&dp, slots.p, 0);
    S.dig_host = slots.p;
    S.dig_dev = (uint64_t*)dp;
  }
  if (cudaMalloc((void**)&S.pool, (size_t)c.budget_bytes) != cudaSuccess) return MPX_ERR_NO_MEM;
  const int64_t share = (c.budget_bytes / T) & ~(int64_t)255;
  if (share < max_buf) return MPX_ERR_ARG;  // a request must fit a share
  for (int t = 0; t < T; ++t) S.budget[(size_t)t].init(S.pool + (size_t)t * (size_t)share, share);
  // world, streams, comm
  mpx_world_config_t wc;
  mpx_world_config_init(&wc);
  wc.engine_mode = c.engine_mode;
  wc.max_streams = std::max(wc.max_streams, T);
  wc.watchdog_ns = 3000000000ll;
  mpx_world_t w = nullptr;
  int rc = mpx_world_create(T, &wc, &w);
  if (rc) return rc;
  std::vector<ThreadCtx> ctx((size_t)T);
  std::vector<mpx_stream_t> ms((size_t)T);
  std::vector<mpx_comm_t> comm((size_t)T);
  if (S.own_regions) S.region.assign((size_t)T, nullptr);
  for (int t = 0; t < T && rc == 0; ++t) {
    ctx[(size_t)t].t = t;
    if (cudaStreamCreateWithFlags(&ctx[(size_t)t].cs, cudaStreamNonBlocking) != cudaSuccess) rc = MPX_ERR_CUDA;
    if (!rc) rc = mpx_stream_create(w, t, (mpx_cuda_stream_t)ctx[(size_t)t].cs, MPX_STREAM_EXCLUSIVE, &ms[(size_t)t]);
    ctx[(size_t)t].stream = ms[(size_t)t];
    if (!S.own_regions) continue;  // the caller's regions hold the caller's data
    if (!rc && cudaMalloc((void**)&S.region[(size_t)t], (size_t)S.region_bytes) != cudaSuccess) rc = MPX_ERR_NO_MEM;
    // first half raw bytes (messages), second half fp32 (allreduce inputs) would
    // split the region; instead every slice is valid fp32 data and raw bytes alike
    if (!rc) rc = mpxi_fill(S.region[(size_t)t], S.region_bytes, c.seed ^ (0x1000ull + (uint64_t)t), 1, ctx[(size_t)t].cs) ? MPX_ERR_CUDA : 0;
  }
  if (!rc) rc = mpx_stream_comm_create(w, T, ms.data(), comm.data());
  for (int t = 0; t < T; ++t) ctx[(size_t)t].comm = comm[(size_t)t];
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = MPX_ERR_CUDA;
  // device clock vs host clock: a kernel writes %globaltimer to mapped memory
  uint64_t* probe = nullptr;
  if (!rc && cudaHostAlloc((void**)&probe, 8, cudaHostAllocMapped) == cudaSuccess) {
    *(volatile uint64_t*)probe = 0;
    void* dp = nullptr;
    cudaHostGetDevicePointer(&dp, probe, 0);
    if (mpxi_clock_probe(dp, ctx[0].cs) == 0) {
      const int64_t t_dl = now_ns() + 1000000000ll;
      while (*(volatile uint64_t*)probe == 0 && now_ns() < t_dl) {
      }
      const int64_t h = now_ns();
      S.clock_offset = (int64_t)*(volatile uint64_t*)probe - h;
    }
    cudaStreamSynchronize(ctx[0].cs);
    cudaFreeHost(probe);
  }
  if (!rc && !plain) rc = mpx_world_start(w);
  if (!rc) {
    S.running = T;
    const int64_t t0 = now_ns() + 2000000;  // let every thread start first
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back(client_thread, std::ref(S), ctx[(size_t)t], plain, t0);
    std::thread reaper;
    if (!plain) reaper = std::thread(reaper_thread, std::ref(S), std::ref(ctx));
    for (auto& x : th) x.join();
    if (!plain) reaper.join();
    rc = S.error.load();
    // the sampled messages' payloads as their senders hold them (a check that
    // the bytes were delivered unchanged: equal digests)
    if (!rc && source_digests && S.dig_dev) {
      for (int t = 0; t < T; ++t) {
        for (const Call& x : S.calls[(size_t)t]) {
          if (x.kind != C_SEND || x.item < 0 || x.item >= ndigests || !digests[x.item]) continue;
          mpxi_digest_store(S.region[(size_t)t] + x.off, x.bytes, S.dig_dev + x.item, ctx[0].cs);
        }
      }
      cudaStreamSynchronize(ctx[0].cs);
      for (int64_t i = 0; i < ndigests; ++i)
        source_digests[i] = digests[i] && i < S.nitems ? S.dig_host[i] : 0;
    }
    int64_t t_end = 0, completed = 0, bytes = 0;
    std::vector<float> lat, svc;
    for (int k = 0; k <= T; ++k) {
      t_end = std::max(t_end, S.t_last[(size_t)k]);
      completed += (int64_t)S.lat[(size_t)k].size();
      bytes += S.bytes_done[(size_t)k];
      lat.insert(lat.end(), S.lat[(size_t)k].begin(), S.lat[(size_t)k].end());
      svc.insert(svc.end(), S.svc[(size_t)k].begin(), S.svc[(size_t)k].end());
    }
    const double secs = std::max(1e-9, (double)(t_end - t0) / 1e9);
    res->completed = completed;
    res->seconds = secs;
    res->msgs_per_s = (double)completed / secs;
    res->gbs = (double)bytes / secs / 1e9;
    res->p50_us = pct(lat, 0.5);
    res->p99_us = pct(lat, 0.99);
    res->svc_p50_us = pct(svc, 0.5);
    res->svc_p99_us = pct(svc, 0.99);
    res->admission_waits = S.waits.load();
    res->peak_bytes = S.peak();
  }
  int err = 0;
  if (w && !plain && mpx_world_get_error(w, &err) == MPX_SUCCESS && err && !rc) rc = err;
  if (rc && w && !plain) {
    fprintf(stderr, "[mpx_serve_run] failed with %d (world error %d)\n", rc, err);
    mpx_world_debug_dump(w);
  }
  if (w && !plain) mpx_world_stop(w, 10000);
  for (int t = 0; t < T; ++t) {
    if (comm[(size_t)t]) mpx_comm_free(&comm[(size_t)t]);
  }
  for (int t = 0; t < T; ++t) {
    if (ctx[(size_t)t].cs) cudaStreamSynchronize(ctx[(size_t)t].cs);
    if (ms[(size_t)t]) mpx_stream_free(&ms[(size_t)t]);
    if (ctx[(size_t)t].cs) cudaStreamDestroy(ctx[(size_t)t].cs);
    if (S.own_regions && S.region[(size_t)t]) cudaFree(S.region[(size_t)t]);
  }
  if (w) mpx_world_free(&w);
  return rc;
}

}  // namespace

extern "C" int mpx_serve_run(const mpx_serve_config_t* cfg, mpx_serve_result_t* res,
                             uint64_t* digests, uint64_t* source_digests, int64_t ndigests) {
  return serve(cfg, nullptr, res, digests, source_digests, ndigests);
}

extern "C" int mpx_serve_run_schedule(const mpx_serve_config_t* cfg, const mpx_serve_schedule_t* sched,
                                      mpx_serve_result_t* res) {
  if (!sched) return MPX_ERR_ARG;
  return serve(cfg, sched, res, nullptr, nullptr, 0);
}
