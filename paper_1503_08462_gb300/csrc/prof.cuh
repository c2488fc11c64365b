// Launch accounting and optional per-kernel-class CUDA-event timing.
//
// Every launcher wraps its kernel(s) in a ProfScope.  The scope always adds
// its kernel count to a process-wide launch counter; when profiling is
// enabled it also records CUDA events before and after the launch on the
// launching stream, together with the algorithmic bytes and flops of that
// launch, so that achieved GB/s and FLOP/s per kernel class can be computed
// from the event times.
#pragma once

#include <cuda_runtime.h>

namespace amgeig {

enum ProfClass {
  P_DEFECT = 0,   // lambda M u - A u (+ residual norms)
  P_SMOOTH,       // l1-Jacobi sweeps and residuals of the V-cycle
  P_TRANSFER,     // restriction / prolongation SpMM (V-cycle, chains, nested phase)
  P_COARSE,       // coarsest-level solve of the V-cycle
  P_AUGMENT,      // [A V | M V]
  P_GRAM,         // V^T [A V | M V]
  P_PENCIL,       // reduced pencil and its float-float eigensolve
  P_RECOMBINE,    // I_n^k Xc + V Y
  P_OTHER,        // copies, conversions, sign normalisation
  P_CHAIN,        // float64 transfer chains: I_k^n [AV | MV], I_n^k Xc, nested prolongation
  P_COUNT
};

// Raise a kernel's dynamic shared-memory limit to at least `bytes`, never
// lowering it: the limit is one per function for the whole process, so solves
// running on several host threads must not shrink it under each other's
// launches.  Sizes up to 48 KB need no attribute.  The attribute is set on
// the current device, and recorded per (device, function).
void ensure_dynamic_smem(const void* func, size_t bytes);

// Device blocks released by owners (hierarchies, workspaces) are kept, per device
// and size, for the next owner: a load after a free then maps nothing new.
// dev_alloc takes a kept block of exactly `bytes` on the current device or calls
// cudaMalloc (after giving every kept block back to the device once, if that
// fails); dev_release keeps the block while at most kDevCacheBytes are kept, else
// frees it -- the caller guarantees that no work in flight still uses it;
// dev_cache_trim frees every kept block (returns the bytes freed).
constexpr size_t kDevCacheBytes = size_t(16) << 30;
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_release(void* p, size_t bytes);
size_t dev_cache_trim();

// Record `msg` as the calling thread's last failure (amgeig_last_error) and
// return `code`; code == AMGEIG_OK clears the record.
int set_last_error(int code, const char* msg);

// The process-wide kernel count (what amgeig_kernel_launches returns), a way
// to add the kernels of a replayed CUDA graph to it (their ProfScopes ran once,
// when the graph was captured), and whether per-launch event timing is on.
unsigned long long launch_count();
// kernels launched by the calling thread so far (what a capture on this thread records)
unsigned long long thread_launch_count();
void add_launches(unsigned long long n);
bool profiling_on();

// Tags the launches made while it lives with a hierarchy level, so that the
// timing table also reports each class per level.
class LevelTag {
 public:
  explicit LevelTag(int level);
  ~LevelTag();
  LevelTag(const LevelTag&) = delete;
  LevelTag& operator=(const LevelTag&) = delete;

 private:
  int prev_;
};

class ProfScope {
 public:
  ProfScope(cudaStream_t st, int cls, double bytes, double flops, int kernels = 1);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaStream_t st_;
  int slot_;
};

}  // namespace amgeig
