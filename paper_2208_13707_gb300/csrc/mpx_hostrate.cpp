// Host-thread message rate under three locking disciplines (the experiment of
// §5.3, Fig. 3, on host cores).  N pairs of host threads: sender t sends
// 8-byte messages to receiver t over a channel of its own (a per-thread
// communicator).  Each side works in windows: the sender issues `window`
// sends, the receiver posts `window` receives and then waits for all of them.
//
//  - GLOBAL_LOCK: every channel's matching state sits behind one mutex, taken
//    by every send, every receive post and every completion poll (a global
//    critical section).
//  - ENDPOINT_LOCK: each channel has its own mutex (a per-endpoint critical
//    section); the calls take the same locks as above, but only their own
//    channel's, so threads never contend, yet every call still locks.
//  - STREAM: the serial-context guarantee of an MPIX stream (§3.1): a channel
//    has one producer and one consumer, so sends publish into a
//    single-producer ring with a release store and the receiver matches its
//    own posted receives without any lock.
//
// The matching work is the same in all three.  A channel carries one tag, so
// a send completes the oldest posted receive or joins the unexpected queue,
// and a receive post takes the oldest unexpected message or joins the posted
// queue (in STREAM the receiver pairs ring entries with its receives in
// order).  Payload k of pair t is (t << 40 | k); receivers count payloads
// that arrive out of order as errors.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "mpx.h"

namespace {

constexpr uint32_t kCap = 1024;  // queue capacity per channel (power of two)

struct alignas(64) Recv {
  uint64_t value;
  std::atomic<int32_t> done;
};

// Matching state of one channel for the locked disciplines.
struct LockedChan {
  alignas(64) std::mutex own;          // ENDPOINT_LOCK
  uint64_t unexp[kCap];                // unexpected payloads
  uint32_t uh = 0, ut = 0;
  Recv* posted[kCap];                  // posted receives
  uint32_t ph = 0, pt = 0;
};

// One single-producer single-consumer ring per channel for STREAM.
struct StreamChan {
  alignas(64) std::atomic<uint64_t> tail{0};  // written by the sender
  alignas(64) std::atomic<uint64_t> head{0};  // written by the receiver
  alignas(64) uint64_t slot[kCap];
};

struct Shared {
  int mode;
  int window;
  int64_t messages;
  std::mutex global;
  std::vector<std::unique_ptr<LockedChan>> lc;
  std::vector<std::unique_ptr<StreamChan>> sc;
  std::atomic<int> ready{0};
  std::atomic<bool> go{false};
  std::atomic<int64_t> errors{0};
};

std::mutex& lock_of(Shared& S, LockedChan& c) {
  return S.mode == MPX_HOSTRATE_GLOBAL_LOCK ? S.global : c.own;
}

// send (locked disciplines): complete the oldest posted receive, else queue
// as unexpected; false when the unexpected queue is full (retry later)
bool locked_send(Shared& S, LockedChan& c, uint64_t v) {
  std::lock_guard<std::mutex> g(lock_of(S, c));
  if (c.ph != c.pt) {
    Recv* r = c.posted[c.ph++ & (kCap - 1)];
    r->value = v;
    r->done.store(1, std::memory_order_release);
    return true;
  }
  if (c.ut - c.uh >= kCap) return false;
  c.unexp[c.ut++ & (kCap - 1)] = v;
  return true;
}

void locked_post(Shared& S, LockedChan& c, Recv* r) {
  std::lock_guard<std::mutex> g(lock_of(S, c));
  if (c.uh != c.ut) {
    r->value = c.unexp[c.uh++ & (kCap - 1)];
    r->done.store(1, std::memory_order_relaxed);
    return;
  }
  c.posted[c.pt++ & (kCap - 1)] = r;
}

// completion poll: a progress call under the lock, as a locked library makes
bool locked_test(Shared& S, LockedChan& c, Recv* r) {
  std::lock_guard<std::mutex> g(lock_of(S, c));
  return r->done.load(std::memory_order_acquire) != 0;
}

void wait_start(Shared& S) {
  S.ready.fetch_add(1);
  while (!S.go.load(std::memory_order_acquire)) std::this_thread::yield();
}

void sender(Shared& S, int t) {
  wait_start(S);
  const uint64_t base = (uint64_t)t << 40;
  for (int64_t k0 = 0; k0 < S.messages; k0 += S.window) {
    const int64_t k1 = std::min<int64_t>(S.messages, k0 + S.window);
    for (int64_t k = k0; k < k1; ++k) {
      const uint64_t v = base | (uint64_t)k;
      if (S.mode == MPX_HOSTRATE_STREAM) {
        StreamChan& c = *S.sc[(size_t)t];
        const uint64_t tl = c.tail.load(std::memory_order_relaxed);
        while (tl - c.head.load(std::memory_order_acquire) >= kCap) std::this_thread::yield();
        c.slot[tl & (kCap - 1)] = v;
        c.tail.store(tl + 1, std::memory_order_release);
      } else {
        LockedChan& c = *S.lc[(size_t)t];
        while (!locked_send(S, c, v)) std::this_thread::yield();
      }
    }
  }
}

void receiver(Shared& S, int t) {
  std::vector<Recv> win((size_t)S.window);
  wait_start(S);
  const uint64_t base = (uint64_t)t << 40;
  int64_t errors = 0;
  for (int64_t k0 = 0; k0 < S.messages; k0 += S.window) {
    const int n = (int)std::min<int64_t>(S.window, S.messages - k0);
    if (S.mode == MPX_HOSTRATE_STREAM) {
      // the receiver is the ring's only consumer: post and match locally
      StreamChan& c = *S.sc[(size_t)t];
      uint64_t hd = c.head.load(std::memory_order_relaxed);
      for (int i = 0; i < n; ++i) {
        while (c.tail.load(std::memory_order_acquire) == hd) std::this_thread::yield();
        win[(size_t)i].value = c.slot[hd & (kCap - 1)];
        ++hd;
        c.head.store(hd, std::memory_order_release);
      }
    } else {
      LockedChan& c = *S.lc[(size_t)t];
      for (int i = 0; i < n; ++i) {
        win[(size_t)i].done.store(0, std::memory_order_relaxed);
        locked_post(S, c, &win[(size_t)i]);
      }
      for (int i = 0; i < n; ++i)
        while (!locked_test(S, c, &win[(size_t)i])) std::this_thread::yield();
    }
    for (int i = 0; i < n; ++i)
      if (win[(size_t)i].value != (base | (uint64_t)(k0 + i))) ++errors;
  }
  S.errors.fetch_add(errors);
}

}  // namespace

extern "C" int mpx_hostrate_config_init(mpx_hostrate_config_t* cfg) {
  if (!cfg) return MPX_ERR_ARG;
  memset(cfg, 0, sizeof(*cfg));
  cfg->threads = 1;
  cfg->mode = MPX_HOSTRATE_STREAM;
  cfg->messages = 1 << 20;
  cfg->window = 64;
  return MPX_SUCCESS;
}

extern "C" int mpx_hostrate_run(const mpx_hostrate_config_t* cfg, mpx_hostrate_result_t* res) {
  if (!cfg || !res) return MPX_ERR_ARG;
  if (cfg->threads < 1 || cfg->threads > 512 || cfg->messages < 1 || cfg->window < 1 ||
      cfg->window > (int)kCap)
    return MPX_ERR_ARG;
  if (cfg->mode != MPX_HOSTRATE_GLOBAL_LOCK && cfg->mode != MPX_HOSTRATE_ENDPOINT_LOCK &&
      cfg->mode != MPX_HOSTRATE_STREAM)
    return MPX_ERR_ARG;
  Shared S;
  S.mode = cfg->mode;
  S.window = cfg->window;
  S.messages = cfg->messages;
  for (int t = 0; t < cfg->threads; ++t) {
    if (S.mode == MPX_HOSTRATE_STREAM) S.sc.emplace_back(new StreamChan());
    else S.lc.emplace_back(new LockedChan());
  }
  std::vector<std::thread> th;
  th.reserve((size_t)cfg->threads * 2);
  for (int t = 0; t < cfg->threads; ++t) {
    th.emplace_back(receiver, std::ref(S), t);
    th.emplace_back(sender, std::ref(S), t);
  }
  while (S.ready.load() < 2 * cfg->threads) std::this_thread::yield();
  const auto t0 = std::chrono::steady_clock::now();
  S.go.store(true, std::memory_order_release);
  for (auto& x : th) x.join();
  const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  res->seconds = sec;
  res->msgs_per_s = sec > 0 ? (double)cfg->messages * cfg->threads / sec : 0.0;
  res->errors = S.errors.load();
  return MPX_SUCCESS;
}
