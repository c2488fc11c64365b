// Allocation-free variant of the dense symmetric eigensolver entry point.
//
// Some callers cannot allocate device memory at the time they need the
// eigensolver: code running inside a memory pool that forbids outside
// cudaMalloc/cudaFree, callers that must not synchronise the device (cudaFree
// does), or embedded hosts whose allocator is owned by another runtime.  This
// entry point takes device pointers for its input and outputs and keeps all of
// its scratch in one file-scope __device__ array of fixed size, so it calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The array costs every GPU that loads the library kNoAllocScratchBytes of
// device memory until the process exits.  All calls on a device share it, and
// it keeps the contents of the last call; the eigensolver writes every scratch
// element before reading it, so nothing needs clearing between calls.  Calls
// whose executions overlap on the GPU (different streams, or different host
// threads) race on the array: serialise them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "amgeig.h"
#include "common.cuh"
#include "kernels.cuh"
#include "prof.cuh"

namespace amgeig {
namespace {

constexpr int kNoAllocMaxN = 128;
constexpr int kNoAllocMaxWant = 64;
constexpr size_t kNoAllocScratchBytes = 512 * 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (device < 0 || device >= kMaxDevices) return set_last_error(AMGEIG_EINVAL, "device ordinal beyond 63");
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return set_last_error(AMGEIG_ECUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return AMGEIG_OK;
}

size_t carve(size_t* off, size_t bytes) {
  const size_t at = *off;
  *off = (at + bytes + 255) & ~static_cast<size_t>(255);
  return at;
}

}  // namespace
}  // namespace amgeig

using namespace amgeig;

extern "C" int amgeig_sym_eigh_noalloc(int n, int nwant, const double* H, double* evals, double* evecs,
                                       void* stream) {
  set_last_error(AMGEIG_OK, nullptr);
  if (!H || !evals || !evecs) return set_last_error(AMGEIG_EINVAL, "NULL pointer");
  if (n < 1 || nwant < 1 || nwant > n) return set_last_error(AMGEIG_EINVAL, "need 1 <= nwant <= n");
  if (n > kNoAllocMaxN || nwant > kNoAllocMaxWant)
    return set_last_error(AMGEIG_EINVAL, "n > 128 or nwant > 64: beyond the fixed scratch array");
  int device = 0;
  cudaError_t ge = cudaGetDevice(&device);
  if (ge != cudaSuccess)
    return set_last_error(AMGEIG_ECUDA, (std::string("cudaGetDevice: ") + cudaGetErrorString(ge)).c_str());
  void* base = nullptr;
  int rc = scratch_address(device, &base);
  if (rc) return rc;
  // carve the eigensolver's workspace out of the fixed array
  const size_t nm = static_cast<size_t>(n), nw = static_cast<size_t>(nwant);
  size_t off = 0;
  const size_t oW = carve(&off, sizeof(df) * nm * (nm + 1));
  const size_t oTau = carve(&off, sizeof(df) * nm);
  const size_t oD = carve(&off, sizeof(df) * nm);
  const size_t oE = carve(&off, sizeof(df) * nm);
  const size_t oF = carve(&off, sizeof(df) * 2 * nm * nw);
  const size_t oZ = carve(&off, sizeof(df) * nm * nw);
  const size_t rrn = nw * nw > 4 * nw ? nw * nw : 4 * nw;
  const size_t oR = carve(&off, sizeof(df) * 4 * rrn);
  const size_t oP = carve(&off, sizeof(int) * nw);
  if (off > kNoAllocScratchBytes) return set_last_error(AMGEIG_EINVAL, "scratch layout exceeds 512 KiB");
  unsigned char* b = static_cast<unsigned char*>(base);
  launch_syev_df_into(n, nwant, H, evals, evecs, reinterpret_cast<df*>(b + oW), reinterpret_cast<df*>(b + oTau),
                      reinterpret_cast<df*>(b + oD), reinterpret_cast<df*>(b + oE), reinterpret_cast<df*>(b + oF),
                      reinterpret_cast<df*>(b + oZ), reinterpret_cast<df*>(b + oR), reinterpret_cast<int*>(b + oP),
                      static_cast<cudaStream_t>(stream));
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess)
    return set_last_error(AMGEIG_ECUDA, (std::string("eigensolver launch: ") + cudaGetErrorString(le)).c_str());
  return AMGEIG_OK;
}
