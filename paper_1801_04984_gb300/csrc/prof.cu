// Launch counting and optional CUDA-event timing of selected kernels (tracing
// support of the library; disabled by default, on the launching stream when on).
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

namespace biot {

static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_prof{false};
static std::mutex g_mu;
struct EvPair {
  cudaEvent_t a, b;
  int kind;
  double units;
};
static std::vector<EvPair> g_open;   // recorded, not yet collected
static std::vector<EvPair> g_free;   // reusable
static EvPair g_cur[PROF_KINDS];

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }
void prof_enable(bool on) { g_prof.store(on); }
bool prof_enabled() { return g_prof.load(); }

void prof_begin(cudaStream_t st, int kind, double units) {
  if (!g_prof.load()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  EvPair e;
  if (!g_free.empty()) {
    e = g_free.back();
    g_free.pop_back();
  } else {
    cudaEventCreate(&e.a);
    cudaEventCreate(&e.b);
  }
  e.kind = kind;
  e.units = units;
  cudaEventRecord(e.a, st);
  g_cur[kind] = e;
}

void prof_end(cudaStream_t st, int kind) {
  if (!g_prof.load()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  EvPair e = g_cur[kind];
  cudaEventRecord(e.b, st);
  g_open.push_back(e);
}

// sums the recorded launches of `kind` (synchronising on their events) and clears them
void prof_collect(int kind, long long* n, double* ms, double* units) {
  std::lock_guard<std::mutex> lk(g_mu);
  long long cnt = 0;
  double tot = 0, un = 0;
  std::vector<EvPair> keep;
  for (EvPair& e : g_open) {
    if (e.kind != kind) {
      keep.push_back(e);
      continue;
    }
    cudaEventSynchronize(e.b);
    float t = 0;
    cudaEventElapsedTime(&t, e.a, e.b);
    tot += t;
    un += e.units;
    ++cnt;
    g_free.push_back(e);
  }
  g_open.swap(keep);
  if (n) *n = cnt;
  if (ms) *ms = tot;
  if (units) *units = un;
}

}  // namespace biot
