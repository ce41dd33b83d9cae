// hostcache.cu -- the parse stage of the load pipeline and the second-level
// (host) cache (Sec. III stage 2, Sec. IV-A-2), for out-of-core vector sets
// whose items arrive encoded.
//
// Codec AP_CODEC_XOR_VARINT (lossless): value k of a row is stored as the
// bits of x_k XOR the bits of x_(k-1) (x_(-1) = +0), written as an unsigned
// LEB128 varint (7 bits a byte, high bit = more follows).  Decoding is a
// branchy byte loop on the CPU, the stand-in for parsing a file.
//
// The cache holds decoded 256-item macros in page-locked host slots.  A
// request for a macro that is not there takes an empty slot or the least
// recently used one nobody holds, and a pool of host threads decodes the
// macro's rows into it; requests wait until the slot is ready.  A slot is
// held while its host-to-device copy is in flight and released by a host
// function queued on the copy stream behind it.  The run announces its
// schedule up front so the threads decode ahead of the copies.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ap_internal.h"

namespace ap {

int64_t xor_varint_encode(const float *x, int64_t dim, uint8_t *out, uint64_t cap) {
  uint32_t prev = 0;
  uint64_t o = 0;
  for (int64_t k = 0; k < dim; ++k) {
    uint32_t b;
    memcpy(&b, x + k, 4);
    uint32_t u = b ^ prev;
    prev = b;
    do {
      if (o >= cap) return -1;
      const uint8_t byte = (uint8_t)(u & 0x7Fu);
      u >>= 7;
      out[o++] = (uint8_t)(byte | (u ? 0x80u : 0u));
    } while (u);
  }
  return (int64_t)o;
}

bool xor_varint_decode(const uint8_t *in, uint64_t len, int64_t dim, float *x) {
  uint32_t prev = 0;
  uint64_t o = 0;
  for (int64_t k = 0; k < dim; ++k) {
    uint32_t u = 0;
    int shift = 0;
    for (;;) {
      if (o >= len || shift > 28) return false;
      const uint8_t byte = in[o++];
      u |= (uint32_t)(byte & 0x7Fu) << shift;
      if (!(byte & 0x80u)) break;
      shift += 7;
    }
    prev ^= u;
    memcpy(x + k, &prev, 4);
  }
  return o == len;
}

struct HostCache::Impl {
  struct Slot {
    int64_t macro = -1;
    int state = 0;          // 0 empty, 1 decoding, 2 ready
    int pins = 0;
    bool reserved = false;  // pinned ahead of its request by the prefetcher
    bool reserved_hit = false;   // ... while it was already in the cache
    int pending = 0;        // row jobs of the macro still decoding
    uint64_t last_use = 0;
  };
  std::mutex mu;
  std::condition_variable cv;
  std::vector<Slot> slots;
  std::unordered_map<int64_t, int> where;
  struct Job {
    int64_t macro;
    int slot;
    int64_t r0, r1;        // rows of the macro
  };
  std::deque<Job> jobs;
  std::vector<int64_t> plan;      // announced requests, in order
  size_t plan_pos = 0;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t clock = 0;
};

struct HostCacheRelease {
  HostCache *cache;
  int slot;
};

HostCache::~HostCache() {
  if (impl) {
    {
      std::lock_guard<std::mutex> g(impl->mu);
      impl->stop = true;
    }
    impl->cv.notify_all();
    for (std::thread &t : impl->workers) t.join();
    delete impl;
  }
  if (pinned) cudaFreeHost(pinned);
  delete[] release_args;
}

ap_status HostCache::init(int64_t n_items, int64_t dim_, const uint8_t *const *blobs_,
                          const uint64_t *bytes_, int32_t codec_, int64_t slots, int threads) {
  n = n_items;
  dim = dim_;
  blobs = blobs_;
  blob_bytes = bytes_;
  codec = codec_;
  n_slots = std::max<int64_t>(2, slots);
  slot_floats = (size_t)kOocMacroItems * dim;
  if (cudaHostAlloc(reinterpret_cast<void **>(&pinned), (size_t)n_slots * slot_floats * 4,
                    cudaHostAllocDefault) != cudaSuccess) {
    pinned = nullptr;
    return AP_ERR_OOM;
  }
  impl = new Impl();
  impl->slots.resize(n_slots);
  release_args = new HostCacheRelease[n_slots];
  for (int64_t s = 0; s < n_slots; ++s) release_args[s] = {this, (int)s};
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
  for (int t = 0; t < threads; ++t) impl->workers.emplace_back([this] { worker(); });
  return AP_OK;
}

// rows of a macro decoded per job, so that all threads share one macro
constexpr int64_t kRowsPerJob = 8;

void HostCache::worker() {
  for (;;) {
    Impl::Job job;
    {
      std::unique_lock<std::mutex> g(impl->mu);
      impl->cv.wait(g, [this] { return impl->stop || !impl->jobs.empty(); });
      if (impl->stop) return;
      job = impl->jobs.front();
      impl->jobs.pop_front();
    }
    const int64_t g0 = job.macro * kOocMacroItems;
    float *dst = pinned + (size_t)job.slot * slot_floats;
    bool ok = true;
    for (int64_t r = job.r0; r < job.r1; ++r)
      ok = ok && xor_varint_decode(blobs[g0 + r], blob_bytes[g0 + r], dim, dst + (size_t)r * dim);
    bool done;
    {
      std::lock_guard<std::mutex> g(impl->mu);
      Impl::Slot &sl = impl->slots[job.slot];
      done = --sl.pending == 0;
      if (done) sl.state = 2;
      parsed_rows += job.r1 - job.r0;
      if (!ok) bad_input = true;
    }
    if (done) impl->cv.notify_all();
  }
}

// queue the row jobs of `macro` into slot s (caller holds the lock)
static void queue_macro(HostCache::Impl *impl, int64_t n, int64_t macro, int s) {
  const int64_t rows = std::min<int64_t>(kOocMacroItems, n - macro * kOocMacroItems);
  int pending = 0;
  for (int64_t r0 = 0; r0 < rows; r0 += kRowsPerJob) {
    impl->jobs.push_back({macro, s, r0, std::min<int64_t>(rows, r0 + kRowsPerJob)});
    ++pending;
  }
  impl->slots[s].pending = pending;
  if (pending == 0) impl->slots[s].state = 2;
}

// a slot for `macro` (caller holds the lock): an empty one, else the least
// recently used one nobody holds; -1 if all are held
static int pick_victim(std::vector<HostCache::Impl::Slot> &slots) {
  int best = -1;
  for (int s = 0; s < (int)slots.size(); ++s) {
    if (slots[s].pins > 0) continue;
    if (slots[s].macro < 0) return s;
    if (best < 0 || slots[s].last_use < slots[best].last_use) best = s;
  }
  return best;
}

// reserve and start decoding announced requests while a slot stays free
// for requests that were not announced (caller holds the lock)
void HostCache::pump() {
  int held = 0;
  for (const Impl::Slot &sl : impl->slots) held += sl.pins > 0;
  while (impl->plan_pos < impl->plan.size() && held < (int)n_slots - 1) {
    const int64_t m = impl->plan[impl->plan_pos];
    auto it = impl->where.find(m);
    if (it != impl->where.end()) {
      Impl::Slot &sl = impl->slots[it->second];
      if (sl.reserved) break;                 // already ahead of its request
      ++sl.pins;
      sl.reserved = true;
      sl.reserved_hit = true;
      ++held;
      ++impl->plan_pos;
      continue;
    }
    const int v = pick_victim(impl->slots);
    if (v < 0) break;
    Impl::Slot &sl = impl->slots[v];
    if (sl.macro >= 0) impl->where.erase(sl.macro);
    sl.macro = m;
    sl.state = 1;
    sl.pins = 1;
    sl.reserved = true;
    sl.reserved_hit = false;
    sl.last_use = ++impl->clock;
    impl->where[m] = v;
    queue_macro(impl, n, m, v);
    ++held;
    ++impl->plan_pos;
  }
  impl->cv.notify_all();
}

void HostCache::announce(const std::vector<int64_t> &macros) {
  std::lock_guard<std::mutex> g(impl->mu);
  for (Impl::Slot &sl : impl->slots)          // holds of an earlier plan not taken up
    if (sl.reserved) {
      sl.reserved = false;
      --sl.pins;
    }
  impl->plan = macros;
  impl->plan_pos = 0;
  pump();
}

int HostCache::acquire(int64_t macro) {
  std::unique_lock<std::mutex> g(impl->mu);
  for (;;) {
    auto it = impl->where.find(macro);
    if (it != impl->where.end()) {
      const int s = it->second;
      Impl::Slot &sl = impl->slots[s];
      if (sl.reserved) {
        sl.reserved = false;                  // the prefetcher's hold becomes ours
        if (sl.reserved_hit) ++hits;
        else ++misses;                        // decoded for this request
      } else {
        ++sl.pins;
        ++hits;
      }
      sl.last_use = ++impl->clock;
      if (impl->plan_pos < impl->plan.size() && impl->plan[impl->plan_pos] == macro)
        ++impl->plan_pos;                     // an announced request met before its turn
      impl->cv.wait(g, [&] { return impl->slots[s].state == 2; });
      pump();
      return s;
    }
    const int v = pick_victim(impl->slots);
    if (v >= 0) {
      Impl::Slot &sl = impl->slots[v];
      if (sl.macro >= 0) impl->where.erase(sl.macro);
      sl.macro = macro;
      sl.state = 1;
      sl.pins = 1;
      sl.reserved = false;
      sl.last_use = ++impl->clock;
      impl->where[macro] = v;
      queue_macro(impl, n, macro, v);
      ++misses;
      impl->cv.notify_all();
      impl->cv.wait(g, [&] { return impl->slots[v].state == 2; });
      pump();
      return v;
    }
    impl->cv.wait(g);                         // every slot held: wait for a release
  }
}

void HostCache::release(int slot) {
  {
    std::lock_guard<std::mutex> g(impl->mu);
    --impl->slots[slot].pins;
    pump();
  }
  impl->cv.notify_all();
}

void CUDART_CB HostCache::release_cb(void *arg) {
  HostCacheRelease *r = static_cast<HostCacheRelease *>(arg);
  r->cache->release(r->slot);
}

void *HostCache::release_arg(int slot) { return &release_args[slot]; }

}  // namespace ap

using namespace ap;

extern "C" ap_status ap_encode_vector(const float *x, int64_t dim, int32_t codec, uint8_t *out,
                                      uint64_t cap, uint64_t *len) {
  if (!x || dim < 0 || !len || (cap > 0 && !out)) return AP_ERR_INVALID_ARG;
  if (codec != AP_CODEC_XOR_VARINT) return AP_ERR_INVALID_ARG;
  if (!out) {                                 // size query
    *len = (uint64_t)dim * 5;
    return AP_OK;
  }
  const int64_t r = xor_varint_encode(x, dim, out, cap);
  if (r < 0) return AP_ERR_INVALID_ARG;
  *len = (uint64_t)r;
  return AP_OK;
}

extern "C" ap_status ap_decode_vector(const uint8_t *in, uint64_t len, int32_t codec,
                                      int64_t dim, float *x) {
  if ((!in && len > 0) || dim < 0 || (!x && dim > 0)) return AP_ERR_INVALID_ARG;
  if (codec != AP_CODEC_XOR_VARINT) return AP_ERR_INVALID_ARG;
  return xor_varint_decode(in, len, dim, x) ? AP_OK : AP_ERR_INVALID_ARG;
}
