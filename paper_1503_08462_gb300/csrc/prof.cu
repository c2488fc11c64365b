// Launch counter and event-based per-class timing (see prof.cuh).
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "amgeig.h"
#include "prof.cuh"

namespace amgeig {

namespace {
struct DevCache {
  std::mutex mu;
  std::multimap<std::pair<int, size_t>, void*> kept;  // (device, bytes) -> block
  size_t bytes = 0;
};
DevCache& dev_cache() {
  static DevCache* c = new DevCache();  // never destroyed: blocks outlive static destructors safely
  return *c;
}
}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  {
    DevCache& c = dev_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.kept.find({dev, bytes});
    if (it != c.kept.end()) {
      *p = it->second;
      c.kept.erase(it);
      c.bytes -= bytes;
      return cudaSuccess;
    }
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    if (dev_cache_trim() > 0) e = cudaMalloc(p, bytes);
  }
  return e;
}

void dev_release(void* p, size_t bytes) {
  if (!p) return;
  int dev = 0;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) == cudaSuccess) dev = at.device;
  {
    DevCache& c = dev_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.bytes + bytes <= kDevCacheBytes) {
      c.kept.emplace(std::make_pair(dev, bytes), p);
      c.bytes += bytes;
      return;
    }
  }
  cudaFree(p);
}

size_t dev_cache_trim() {
  DevCache& c = dev_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  const size_t freed = c.bytes;
  for (auto& kv : c.kept) cudaFree(kv.second);
  c.kept.clear();
  c.bytes = 0;
  return freed;
}
namespace {

struct Rec {
  int cls;
  int level;  // hierarchy level of the launch (-1: untagged)
  double bytes, flops;
  int kernels;
  cudaEvent_t e0, e1;
};

struct Profiler {
  std::atomic<unsigned long long> launches{0};
  std::atomic<bool> on{false};
  std::mutex mu;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_next = 0;

  cudaEvent_t take() {
    if (pool_next == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[pool_next++];
  }
};

Profiler& prof() {
  static Profiler* p = new Profiler();
  return *p;
}

const char* kNames[P_COUNT] = {"defect", "smooth", "transfer", "coarse_solve", "augment",
                               "gram", "pencil", "recombine", "other", "chain"};

}  // namespace

void ensure_dynamic_smem(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return;
  // the attribute belongs to the current device's copy of the function: one
  // record per (device, function)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[std::make_pair(dev, func)];
  if (bytes <= cur) return;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) ==
      cudaSuccess)
    cur = bytes;
}

thread_local unsigned long long g_thread_launches = 0;  // kernels launched by the calling thread

unsigned long long launch_count() { return prof().launches.load(); }
unsigned long long thread_launch_count() { return g_thread_launches; }
void add_launches(unsigned long long n) { prof().launches += n; }
bool profiling_on() { return prof().on.load(std::memory_order_relaxed); }

thread_local int g_depth = 0;  // nested scopes only count launches; the outermost one is timed
thread_local int g_outer = -1;  // record of the open outermost scope (nested scopes add their kernels to it)
thread_local int g_level = -1;  // level tag of the launches in flight (LevelTag)

LevelTag::LevelTag(int level) : prev_(g_level) { g_level = level; }
LevelTag::~LevelTag() { g_level = prev_; }

ProfScope::ProfScope(cudaStream_t st, int cls, double bytes, double flops, int kernels) : st_(st), slot_(-1) {
  Profiler& p = prof();
  p.launches += static_cast<unsigned long long>(kernels);
  g_thread_launches += static_cast<unsigned long long>(kernels);
  if (g_depth++ > 0) {
    if (g_outer >= 0) {
      std::lock_guard<std::mutex> lk(p.mu);
      if (g_outer < static_cast<int>(p.recs.size())) p.recs[g_outer].kernels += kernels;
    }
    return;
  }
  if (!p.on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(p.mu);
  Rec r{cls, g_level, bytes, flops, kernels, p.take(), p.take()};
  if (!r.e0 || !r.e1) return;
  cudaEventRecord(r.e0, st);
  slot_ = static_cast<int>(p.recs.size());
  p.recs.push_back(r);
  g_outer = slot_;
}

ProfScope::~ProfScope() {
  --g_depth;
  if (slot_ < 0) return;
  g_outer = -1;
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (slot_ < static_cast<int>(p.recs.size())) cudaEventRecord(p.recs[slot_].e1, st_);
}

}  // namespace amgeig

using namespace amgeig;

extern "C" {

int amgeig_profile_enable(int enable) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (enable) {
    p.recs.clear();
    p.pool_next = 0;
  }
  p.on.store(enable != 0);
  return AMGEIG_OK;
}

int amgeig_profile_read(amgeig_prof_entry* out, int max_entries, int* n_entries) {
  if (!out || !n_entries || max_entries < 0) return AMGEIG_EINVAL;
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  constexpr int kLevels = 64;
  std::vector<amgeig_prof_entry> tab(static_cast<size_t>(P_COUNT) * (kLevels + 1));
  std::memset(tab.data(), 0, sizeof(amgeig_prof_entry) * tab.size());
  // slot c: the class total; slot P_COUNT * (1 + l) + c: the class on level l
  for (int c = 0; c < P_COUNT; ++c) {
    std::strncpy(tab[c].name, kNames[c], sizeof(tab[c].name) - 1);
    for (int l = 0; l < kLevels; ++l)
      std::snprintf(tab[P_COUNT * (1 + l) + c].name, sizeof(tab[0].name), "%s@%d", kNames[c], l);
  }
  for (const Rec& r : p.recs) {
    if (cudaEventSynchronize(r.e1) != cudaSuccess) return AMGEIG_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) return AMGEIG_ECUDA;
    for (int slot : {r.cls, (r.level >= 0 && r.level < kLevels) ? P_COUNT * (1 + r.level) + r.cls : -1}) {
      if (slot < 0) continue;
      amgeig_prof_entry& t = tab[slot];
      t.launches += 1;
      t.kernels += r.kernels;
      t.total_ms += ms;
      t.bytes += r.bytes;
      t.flops += r.flops;
    }
  }
  int n = 0;
  for (size_t i = 0; i < tab.size() && n < max_entries; ++i)
    if (tab[i].launches > 0) out[n++] = tab[i];
  *n_entries = n;
  return AMGEIG_OK;
}

uint64_t amgeig_kernel_launches(void) { return prof().launches.load(); }

}  // extern "C"
