// Launch counter and per-kernel-class event timing (see kprof.cuh).
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kprof.cuh"

namespace bse {

static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_on{false};

struct Rec {
  int k;
  cudaEvent_t a, b;
  double bytes, flops;
  bool done;
};

static std::mutex g_mu;
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_pool;
static double g_ms[K_NUM_CLASSES], g_bytes[K_NUM_CLASSES], g_flops[K_NUM_CLASSES];
static long long g_count[K_NUM_CLASSES];

void kcount(int launches) { g_launches.fetch_add(launches, std::memory_order_relaxed); }
bool kprof_on() { return g_on.load(std::memory_order_relaxed); }

static cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

int kprof_begin(int k, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r;
  r.k = k;
  r.a = take_event();
  r.b = take_event();
  r.bytes = r.flops = 0;
  r.done = false;
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void kprof_end(int slot, cudaStream_t s, double bytes, double flops) {
  std::lock_guard<std::mutex> lk(g_mu);
  Rec& r = g_recs[slot];
  cudaEventRecord(r.b, s);
  r.bytes = bytes;
  r.flops = flops;
  r.done = true;
}

// Fold finished records into the per-class totals (synchronises on each event).
static void drain() {
  for (auto& r : g_recs) {
    if (!r.done) continue;
    cudaEventSynchronize(r.b);
    float ms = 0;
    cudaEventElapsedTime(&ms, r.a, r.b);
    g_ms[r.k] += ms;
    g_bytes[r.k] += r.bytes;
    g_flops[r.k] += r.flops;
    g_count[r.k] += 1;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}

}  // namespace bse

using namespace bse;

extern "C" long long bse_launch_count(void) { return g_launches.load(); }

extern "C" int bse_kprof_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!on) drain();
  for (int k = 0; k < K_NUM_CLASSES; ++k) {
    g_ms[k] = g_bytes[k] = g_flops[k] = 0;
    g_count[k] = 0;
  }
  g_recs.clear();
  g_on.store(on != 0);
  return BSE_OK;
}

extern "C" int bse_kprof_read(int k, long long* launches, double* ms, double* bytes, double* flops) {
  if (k < 0 || k >= K_NUM_CLASSES) return BSE_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  drain();
  if (launches) *launches = g_count[k];
  if (ms) *ms = g_ms[k];
  if (bytes) *bytes = g_bytes[k];
  if (flops) *flops = g_flops[k];
  return BSE_OK;
}

namespace bse {
DevStatus*& current_status() {
  static thread_local DevStatus* cur = nullptr;
  return cur;
}
}  // namespace bse
