// C ABI of the solve phase: hierarchy loading, the solve driver (Algorithm 3.2
// around Algorithm 3.1) and the request service.  Every arithmetic step of a
// solve runs in the kernels of spmm.cu, dense.cu and pencil.cu; the host only
// validates input, moves data and sequences launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <type_traits>
#include <vector>

#include "amgeig.h"
#include "common.cuh"
#include "kernels.cuh"
#include "prof.cuh"

using namespace amgeig;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CK(expr)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      return fail(e_ == cudaErrorMemoryAllocation ? AMGEIG_ENOMEM : AMGEIG_ECUDA,                  \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                             \
    }                                                                                              \
  } while (0)

// ------------------------------------------------------------------ small kernels

// per-column (max |u|, lowest index) over rows, stage 1: each block scans a slab
// of rows for all q columns (coalesced along the row) and writes its best entry
// per column; stage 2 picks the best slab per column and the sign
__global__ void k_col_best(const double* __restrict__ U, int rows, int ld, int q, int slab, double* __restrict__ bval,
                           int* __restrict__ bidx) {
  __shared__ double sb[8][32];
  __shared__ int si[8][32];
  const int r0 = blockIdx.x * slab, r1 = min(rows, r0 + slab);
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32, nwarp = blockDim.x / 32;
  for (int c0 = 0; c0 < q; c0 += 32) {  // uniform trip count: barriers below are reached by all
    const int c = c0 + lane;
    double best = -1.0;
    int bi = 0x7fffffff;
    if (c < q) {
      for (int i = r0 + wid; i < r1; i += nwarp) {
        const double a = fabs(U[static_cast<long long>(i) * ld + c]);
        if (a > best || (a == best && i < bi)) {
          best = a;
          bi = i;
        }
      }
    }
    sb[wid][lane] = best;
    si[wid][lane] = bi;
    __syncthreads();
    if (wid == 0 && c < q) {
      for (int w = 1; w < nwarp; ++w) {
        const double b2 = sb[w][lane];
        const int i2 = si[w][lane];
        if (b2 > best || (b2 == best && i2 < bi)) {
          best = b2;
          bi = i2;
        }
      }
      bval[static_cast<long long>(blockIdx.x) * q + c] = best;
      bidx[static_cast<long long>(blockIdx.x) * q + c] = bi;
    }
    __syncthreads();
  }
}

// stage 2: one block (kSignThreads) per column; (max |u|, lowest index) is a
// total order, so the pick does not depend on how the slabs are split
constexpr int kSignThreads = 128;
__global__ void k_col_sign2(const double* __restrict__ U, int ld, int q, int nslabs, const double* __restrict__ bval,
                            const int* __restrict__ bidx, double* __restrict__ sign) {
  __shared__ double sb[kSignThreads];
  __shared__ int si[kSignThreads];
  const int c = blockIdx.x, t = threadIdx.x;
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int s = t; s < nslabs; s += kSignThreads) {
    const double b2 = bval[static_cast<long long>(s) * q + c];
    const int i2 = bidx[static_cast<long long>(s) * q + c];
    if (b2 > best || (b2 == best && i2 < bi)) {
      best = b2;
      bi = i2;
    }
  }
  sb[t] = best;
  si[t] = bi;
  __syncthreads();
  for (int o = kSignThreads / 2; o > 0; o >>= 1) {
    if (t < o) {
      const double b2 = sb[t + o];
      const int i2 = si[t + o];
      if (b2 > sb[t] || (b2 == sb[t] && i2 < si[t])) {
        sb[t] = b2;
        si[t] = i2;
      }
    }
    __syncthreads();
  }
  if (t == 0) sign[c] = (si[0] != 0x7fffffff && U[static_cast<long long>(si[0]) * ld + c] < 0.0) ? -1.0 : 1.0;
}

__global__ void k_out_vectors(const double* __restrict__ U, int rows, int ld, int q, const double* __restrict__ sign,
                              double* __restrict__ out) {
  const long long total = static_cast<long long>(rows) * q;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = i / q;
    const int c = static_cast<int>(i % q);
    out[i] = sign[c] * U[r * ld + c];
  }
}

__global__ void k_copy_d(const double* __restrict__ a, int n, double* __restrict__ b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i];
}

// ------------------------------------------------------------------ blob parsing

// A CSR matrix read in place from the hierarchy blob (no copies): the arrays
// are 8-byte aligned inside the blob, which is 8-byte aligned itself (or copied
// once to an aligned buffer).  m is null for transfer operators.
struct CsrView {
  int64_t rows = 0, cols = 0, nnz = 0;
  const int32_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* a = nullptr;
  const double* m = nullptr;
};

struct Reader {
  const uint8_t* p;
  size_t n, off;
  template <typename T>
  bool view(const T** out, size_t count) {
    const size_t bytes = count * sizeof(T);
    if (count > (n / sizeof(T)) || off + bytes > n - 8) return false;
    *out = reinterpret_cast<const T*>(p + off);
    off += bytes;
    off += (8 - off % 8) % 8;
    return true;
  }
};

int host_threads(int64_t rows);
template <class F>
void parallel_for(int T, F f);

bool csr_valid(const CsrView& v) {
  if (v.rp[0] != 0 || v.rp[v.rows] != v.nnz) return false;
  const int T = host_threads(std::max(v.rows, v.nnz));
  std::vector<char> ok(T, 1);
  parallel_for(T, [&](int t) {
    const int64_t r0 = v.rows * t / T, r1 = v.rows * (t + 1) / T;
    for (int64_t i = r0; i < r1; ++i)
      if (v.rp[i + 1] < v.rp[i]) ok[t] = 0;
    const int64_t p0 = v.nnz * t / T, p1 = v.nnz * (t + 1) / T;
    for (int64_t q = p0; q < p1; ++q)
      if (v.ci[q] < 0 || v.ci[q] >= v.cols) ok[t] = 0;
  });
  for (char c : ok)
    if (!c) return false;
  return true;
}

// Host threads for the load-time loops over rows: one per 32k rows, at most 16.
int host_threads(int64_t rows) {
  const unsigned hc = std::thread::hardware_concurrency();
  const int64_t want = rows / 32768 + 1;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>({want, 16, hc ? static_cast<int64_t>(hc) : 1})));
}

// f(t) for t in [0, T) on T threads (the calling thread runs t = 0)
template <class F>
void parallel_for(int T, F f) {
  if (T <= 0) return;
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back([&f, t] { f(t); });
  f(0);
  for (auto& x : th) x.join();
}

// The blob's layout: magic, header and in-place views of every array, each
// bounds-checked against the blob; *base receives the blob or its aligned copy.
// The content (checksum, CSR structure) is checked by validate_blob.
int parse_blob(const void* blob, size_t bytes, std::vector<CsrView>& levels, std::vector<CsrView>& prolong,
               std::vector<uint64_t>& aligned, const uint8_t** base) {
  const uint8_t* b = static_cast<const uint8_t*>(blob);
  if (reinterpret_cast<uintptr_t>(b) % 8 != 0) {
    // the views need 8-byte alignment: one aligned copy of an unaligned blob
    aligned.resize(bytes / 8 + 1);
    std::memcpy(aligned.data(), b, bytes);
    b = reinterpret_cast<const uint8_t*>(aligned.data());
  }
  if (bytes < 24 || bytes % 8 != 0 || std::memcmp(b, "AMGEIGH1", 8) != 0)
    return fail(AMGEIG_ECORRUPT, "not a hierarchy blob (magic/length)");
  *base = b;
  uint32_t version, n;
  std::memcpy(&version, b + 8, 4);
  std::memcpy(&n, b + 12, 4);
  if (version != 1 || n < 1 || n > 64) return fail(AMGEIG_ECORRUPT, "unsupported blob version or level count");
  size_t off = 16;
  if (off + 8ull * (3 * n - 1) > bytes - 8) return fail(AMGEIG_ECORRUPT, "truncated blob header");
  std::vector<uint64_t> rows(n), nnz(n), nnzp(n > 1 ? n - 1 : 0);
  std::memcpy(rows.data(), b + off, 8 * n);
  off += 8 * n;
  std::memcpy(nnz.data(), b + off, 8 * n);
  off += 8 * n;
  if (n > 1) std::memcpy(nnzp.data(), b + off, 8 * (n - 1));
  off += 8 * (n - 1);
  off += (8 - off % 8) % 8;
  for (uint32_t l = 0; l < n; ++l) {
    if (rows[l] == 0 || rows[l] >= (1ull << 31) || nnz[l] >= (1ull << 31)) return fail(AMGEIG_ECORRUPT, "level size out of range");
    if (l > 0 && rows[l] >= rows[l - 1]) return fail(AMGEIG_ECORRUPT, "levels must shrink");
  }
  Reader rd{b, bytes, off};
  levels.assign(n, CsrView());
  prolong.assign(n > 1 ? n - 1 : 0, CsrView());
  for (uint32_t l = 0; l < n; ++l) {
    CsrView& L = levels[l];
    L.rows = L.cols = static_cast<int64_t>(rows[l]);
    L.nnz = static_cast<int64_t>(nnz[l]);
    if (!rd.view(&L.rp, rows[l] + 1) || !rd.view(&L.ci, nnz[l]) || !rd.view(&L.a, nnz[l]) || !rd.view(&L.m, nnz[l]))
      return fail(AMGEIG_ECORRUPT, "truncated level arrays");
  }
  for (uint32_t l = 0; l + 1 < n; ++l) {
    CsrView& P = prolong[l];
    P.rows = static_cast<int64_t>(rows[l]);
    P.cols = static_cast<int64_t>(rows[l + 1]);
    P.nnz = static_cast<int64_t>(nnzp[l]);
    if (nnzp[l] >= (1ull << 31)) return fail(AMGEIG_ECORRUPT, "prolongation size out of range");
    if (!rd.view(&P.rp, rows[l] + 1) || !rd.view(&P.ci, nnzp[l]) || !rd.view(&P.a, nnzp[l]))
      return fail(AMGEIG_ECORRUPT, "truncated prolongation arrays");
  }
  if (rd.off != bytes - 8) return fail(AMGEIG_ECORRUPT, "trailing bytes in blob");
  return AMGEIG_OK;
}

// ------------------------------------------------------------------ device data

// Device memory of one owner (a hierarchy, a solve workspace), released with it.
// Arrays of 64 MiB and more get a cudaMalloc of their own; smaller ones are carved,
// 256-byte aligned, from blocks whose size doubles from 2 MiB up to 64 MiB (a block
// is at least as large as the array that opens it).  A hierarchy holds ~200 arrays
// and each cudaMalloc / cudaFree costs tens of microseconds (a cudaFree synchronises
// the device), so loading and releasing one takes about ten calls, while a small
// owner still holds only a few MiB.
struct DeviceBuffers {
  static constexpr size_t kOwn = size_t(64) << 20, kFirst = size_t(2) << 20, kAlign = 256;
  size_t next_block = kFirst;  // size of the next block of carved arrays
  std::vector<void*> ptrs;  // every block of this owner
  std::vector<size_t> sizes;  // and its size
  size_t held = 0;          // bytes of those allocations
  size_t mallocs = 0;       // allocation calls made (or, when dry, that would be made)
  bool dry = false;         // count the bytes a sequence of allocs would take, allocate nothing
  char* blk = nullptr;      // free tail of the current block of small arrays
  size_t blk_left = 0;
  cudaStream_t st = nullptr;  // the owner's work (and uploads) run on this stream
  // the owner's stream is drained first: the blocks go back to the device cache for the next owner
  ~DeviceBuffers() {
    if (st) cudaStreamSynchronize(st);
    for (size_t i = 0; i < ptrs.size(); ++i) dev_release(ptrs[i], sizes[i]);
  }
  template <typename T>
  cudaError_t alloc(T** out, size_t count) {
    const size_t bytes = (sizeof(T) * (count > 0 ? count : 1) + kAlign - 1) / kAlign * kAlign;
    void* p = nullptr;
    *out = nullptr;
    if (bytes >= kOwn) {
      if (!dry) {
        cudaError_t e = dev_alloc(&p, bytes);
        if (e != cudaSuccess) return e;
        ptrs.push_back(p);
        sizes.push_back(bytes);
      }
      ++mallocs;
      held += bytes;
      *out = static_cast<T*>(p);
      return cudaSuccess;
    }
    if (bytes > blk_left) {
      const size_t block = std::max(next_block, bytes);  // < kOwn
      next_block = std::min(kOwn, 2 * block);
      if (!dry) {
        cudaError_t e = dev_alloc(&p, block);
        if (e != cudaSuccess) return e;
        ptrs.push_back(p);
        sizes.push_back(block);
        blk = static_cast<char*>(p);
      }
      ++mallocs;
      held += block;
      blk_left = block;
    }
    if (!dry) {
      *out = reinterpret_cast<T*>(blk);
      blk += bytes;
    }
    blk_left -= bytes;
    return cudaSuccess;
  }
  template <typename T>
  cudaError_t upload(T** out, const T* src, size_t count) {
    cudaError_t e = alloc(out, count);
    if (e != cudaSuccess) return e;
    if (count) e = cudaMemcpyAsync(*out, src, sizeof(T) * count, cudaMemcpyHostToDevice, st);
    return e;
  }
  template <typename T>
  cudaError_t upload(T** out, const std::vector<T>& v) {
    return upload(out, v.data(), v.size());
  }
};

struct SolveWork;

}  // namespace

struct amgeig_hierarchy_t {
  int device = 0;
  int nlev = 0;
  std::vector<int64_t> sizes;
  std::vector<DevCsr> A;  // v64 = A, m64 = M, v32 = float(A)
  std::vector<double*> dinv64;
  std::vector<float*> dinv32;
  std::vector<DevCsr> P, R;  // v64 and v32
  std::vector<DevCsr> PC;    // PC[k] = I_n^k = P_k ... P_{n-2} (rows_k x d_n), float-float values
  int dn = 0;
  double *An = nullptr, *Mn = nullptr, *Z = nullptr, *theta = nullptr, *Ainv = nullptr;
  // the coarse eigenbasis is computed during the load (amgeig_load_hierarchy_modes)
  // or on the first solve that needs it: modes_ready leading columns of Z (and
  // theta) are valid; cpw keeps the M_n factor and the solver's scratch
  int modes_ready = 0;
  PencilWork* cpw = nullptr;
  float* Ainv32 = nullptr;
  float2* Zdf = nullptr;  // Z as float-float pairs
  int* dstatus = nullptr;
  DeviceBuffers mem;
  std::mutex mu;  // one solve at a time per hierarchy (shared workspace)
  std::unique_ptr<SolveWork> ws;
  // multicolour Gauss-Seidel, built on the first solve that asks for it:
  // per level below the coarsest, the rows sorted by colour (device), the
  // colour offsets (host) and 1 / a_ii
  bool gs_ready = false;
  bool bf16_ready = false;  // bfloat16 copies of the V-cycle's operators (on the first such solve)
  std::vector<int*> gs_rows;
  std::vector<std::vector<int>> gs_off;
  std::vector<double*> gs_dinv64;
  std::vector<float*> gs_dinv32;
  // Algorithm 3.2 step 1 on a level n1 above the coarsest (when q + q_extra
  // exceeds d_n, or the caller asks for it): the dense pencil (A_n1, M_n1), its
  // M_n1 factor's workspace and its `count` lowest eigenpairs, kept for later solves
  struct Initial {
    int level = -1, count = 0, d = 0;
    double *A = nullptr, *M = nullptr, *Z = nullptr, *theta = nullptr;
    PencilWork* pw = nullptr;
  } init;
  // the shifted inner solve (options.shift = sigma): the V-cycle's operators
  // A_l - sigma M_l (same pattern and transfers), their l1-Jacobi diagonals and the
  // exact coarsest solve (A_n - sigma M_n)^-1, made for the last sigma asked for
  struct Shifted {
    bool ready = false;
    double sigma = 0.0;
    std::vector<DevCsr> A;
    std::vector<double*> dinv64;
    std::vector<float*> dinv32;
    double *Bn = nullptr, *L = nullptr, *Linv = nullptr, *Ainv = nullptr;
    float* Ainv32 = nullptr;
  } sh;
  // float32 V-cycle widths (float4 columns) whose launch shapes are tuned, and the tuner's log
  bool tuned_w4[33] = {};
  std::string tune_log;
  cudaStream_t stream = nullptr;
  std::atomic<int> pending{0};
  ~amgeig_hierarchy_t();
};

namespace {

struct SolveWork {
  int smoother = AMGEIG_SMOOTHER_L1_JACOBI;  // of the current solve
  bool shifted = false;                       // the current solve's V-cycle runs on A_l - sigma M_l
  bool bf16 = false;                          // the current solve reads bfloat16 operator values
  int qcap = 0;  // column capacity: the buffers serve any solve with q + q_extra <= qcap
  int bcap = 0;  // augmentation width capacity (qcap, or a Krylov block's 2 (q + q_extra))
  int qt = 0;    // columns of the current solve (every block's row stride)
  int ld32 = 0;  // row stride of the float32 V-cycle blocks: qt rounded up to a multiple of 4
  int precision = -1;
  int vcycles = 1;
  DeviceBuffers mem;
  double *U = nullptr, *Ualt = nullptr, *V = nullptr, *W = nullptr;
  double* K = nullptr;  // the Krylov block [V1 | E] (rows x 2 qt), when the capacity allows one
  std::vector<double*> B64, X64, T64, D64, E64;  // per level (FP64 V-cycle)
  std::vector<float*> B32, X32, T32, D32, E32;   // per level (FP32 V-cycle)
  std::vector<double*> WC, PX;                   // restriction chain [N][2q], prolongation chain [N][q]
  double *partials = nullptr, *sums = nullptr, *relres = nullptr, *lam = nullptr, *mu = nullptr;
  double *C = nullptr, *G = nullptr, *gsc = nullptr, *Xc = nullptr, *Yv = nullptr, *sign = nullptr;
  double* Ydf = nullptr;   // Yv in float-float (two floats per value), streamed by the wide recombination
  int* flags = nullptr;
  int* perm = nullptr;     // output column c is column perm[c] of the iterate (after the refinement)
  bool permuted = false;   // perm applies to the current solve's outputs
  double* refined = nullptr;  // the refined iterate in float64 (U or V)
  int* nfallback = nullptr;  // corrections that needed the dense eigensolver
  PencilWork* pw = nullptr;
  size_t pw_bytes = 0;  // device bytes of pw
  // captured CUDA graphs of launch segments (see run_segment), keyed by the
  // segment, the settings and the buffer roles on entry
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    std::vector<void*> post;  // buffer roles after the segment
    unsigned long long kernels = 0;
  };
  std::map<std::string, Graph> graphs;
  std::map<std::string, int> graph_seen;  // segments run so far without a graph
  ~SolveWork() {
    if (mem.st) cudaStreamSynchronize(mem.st);  // its solves' work is done before its blocks are released
    for (auto& g : graphs)
      if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    pencil_work_destroy(pw);
  }
};

// dry: allocate nothing, only add up in w->mem.held (and pw_bytes) what the
// workspace would hold
int make_workspace(amgeig_hierarchy_t* h, int qt, int precision, int vcycles, std::unique_ptr<SolveWork>& out,
                   bool dry = false, int border = 0) {
  auto w = std::make_unique<SolveWork>();
  w->mem.dry = dry;
  w->mem.st = dry ? nullptr : h->stream;
  // the augmentation's width: the iterate's qt columns, or a Krylov block of up to 2 qt
  const int bw = std::max(qt, border);
  w->bcap = bw;
  w->qcap = qt;
  w->qt = qt;
  w->ld32 = (qt + 3) & ~3;
  w->precision = precision;
  w->vcycles = vcycles;
  const int n = h->nlev;
  const int64_t N0 = h->sizes[0];
  auto& m = w->mem;
  CK(m.alloc(&w->U, N0 * qt));
  CK(m.alloc(&w->Ualt, N0 * qt));
  CK(m.alloc(&w->V, N0 * qt));
  CK(m.alloc(&w->W, N0 * 2 * bw));
  if (bw > qt) CK(m.alloc(&w->K, N0 * bw));
  w->B64.assign(n, nullptr);
  w->X64.assign(n, nullptr);
  w->T64.assign(n, nullptr);
  w->D64.assign(n, nullptr);
  w->E64.assign(n, nullptr);
  w->B32.assign(n, nullptr);
  w->X32.assign(n, nullptr);
  w->T32.assign(n, nullptr);
  w->D32.assign(n, nullptr);
  w->E32.assign(n, nullptr);
  w->WC.assign(n, nullptr);
  w->PX.assign(n, nullptr);
  for (int l = 0; l < n; ++l) {
    const int64_t Nl = h->sizes[l];
    if (precision == AMGEIG_FP64) {
      CK(m.alloc(&w->B64[l], Nl * qt));
      CK(m.alloc(&w->X64[l], Nl * qt));
      CK(m.alloc(&w->T64[l], Nl * qt));
      if (vcycles > 1) {
        CK(m.alloc(&w->D64[l], Nl * qt));
        CK(m.alloc(&w->E64[l], Nl * qt));
      }
    } else {
      CK(m.alloc(&w->B32[l], Nl * w->ld32));
      CK(m.alloc(&w->X32[l], Nl * w->ld32));
      CK(m.alloc(&w->T32[l], Nl * w->ld32));
      if (vcycles > 1) {
        CK(m.alloc(&w->D32[l], Nl * w->ld32));
        CK(m.alloc(&w->E32[l], Nl * w->ld32));
      }
    }
    if (l > 0) CK(m.alloc(&w->WC[l], Nl * 2 * bw));
    CK(m.alloc(&w->PX[l], Nl * qt));
  }
  const int blocks_max = ceil_div(N0, 8) + 1;  // defect launches use >= 8 rows per block
  CK(m.alloc(&w->partials, std::max(static_cast<size_t>(blocks_max) * 2 * qt,
                                     static_cast<size_t>(rayleigh_blocks(qt)) * 7 * qt)));
  CK(m.alloc(&w->sums, 5 * qt));
  CK(m.alloc(&w->relres, qt));
  CK(m.alloc(&w->lam, qt));
  CK(m.alloc(&w->mu, qt));
  CK(m.alloc(&w->C, static_cast<size_t>(h->dn) * 2 * bw));
  CK(m.alloc(&w->G, static_cast<size_t>(bw) * 2 * bw));
  size_t gs = 0;
  for (int l = 0; l < n; ++l)
    for (int qq = 1; qq <= bw; ++qq) {  // any width up to the capacity (the chunking depends on it)
      gs = std::max(gs, gram_scratch_doubles(static_cast<int>(h->sizes[l]), qq, 2 * qq));
      gs = std::max(gs, gram_df_scratch_doubles(static_cast<int>(h->sizes[l]), qq, 2 * qq));
    }
  CK(m.alloc(&w->gsc, gs));
  CK(m.alloc(&w->Xc, static_cast<size_t>(h->dn) * qt));
  CK(m.alloc(&w->Yv, static_cast<size_t>(bw) * qt));
  CK(m.alloc(&w->Ydf, static_cast<size_t>(qt) * qt));
  CK(m.alloc(&w->sign, qt));
  CK(m.alloc(&w->flags, 4));
  CK(m.alloc(&w->perm, qt));
  CK(m.alloc(&w->nfallback, 1));
  w->pw_bytes = pencil_work_bytes(h->dn, bw);
  if (!dry) {
    cudaError_t e;
    w->pw = pencil_work_create(h->dn, bw, &e);
    if (!w->pw) return fail(AMGEIG_ENOMEM, std::string("pencil workspace: ") + cudaGetErrorString(e));
  }
  out = std::move(w);
  return AMGEIG_OK;
}

// Keep a workspace that can hold qt columns: a smaller solve reuses the buffers
// of a larger one (all layouts follow the current qt), so a stream of requests
// with varying q on one hierarchy allocates only when its largest width grows.
int ensure_workspace(amgeig_hierarchy_t* h, int qt, int precision, int vcycles, int border = 0) {
  // the bfloat16 option only swaps the V-cycle's operator values: same workspace
  if (precision == AMGEIG_MIXED_BF16) precision = AMGEIG_MIXED_FP32;
  SolveWork* w = h->ws.get();
  const int bw = std::max(qt, border);
  if (!w || w->qcap < qt || w->bcap < bw || w->precision != precision || w->vcycles < vcycles) {
    const bool same = w && w->precision == precision;
    const int cap = same ? std::max(qt, w->qcap) : qt;
    const int bcap = same ? std::max(bw, w->bcap) : bw;
    const int vc = same ? std::max(vcycles, w->vcycles) : vcycles;
    h->ws.reset();
    const int rc = make_workspace(h, cap, precision, vc, h->ws, false, bcap);
    if (rc) return rc;
    w = h->ws.get();
  }
  w->qt = qt;
  w->ld32 = (qt + 3) & ~3;
  return AMGEIG_OK;
}

// ------------------------------------------------------------------ V-cycle

template <typename T>
struct VBufs;
template <>
struct VBufs<double> {
  static std::vector<double*>& B(SolveWork* w) { return w->B64; }
  static std::vector<double*>& X(SolveWork* w) { return w->X64; }
  static std::vector<double*>& Tm(SolveWork* w) { return w->T64; }
  static std::vector<double*>& D(SolveWork* w) { return w->D64; }
  static std::vector<double*>& E(SolveWork* w) { return w->E64; }
};
template <>
struct VBufs<float> {
  static std::vector<float*>& B(SolveWork* w) { return w->B32; }
  static std::vector<float*>& X(SolveWork* w) { return w->X32; }
  static std::vector<float*>& Tm(SolveWork* w) { return w->T32; }
  static std::vector<float*>& D(SolveWork* w) { return w->D32; }
  static std::vector<float*>& E(SolveWork* w) { return w->E32; }
};

// bf: the float32 path reads the operators' bfloat16 values (AMGEIG_MIXED_BF16)
void presmooth_residual(const DevCsr& A, const double* d, const double* b, int wdt, double* x, double* r, cudaStream_t s, bool = false) { launch_presmooth_residual_f64(A, d, b, wdt, x, r, s); }
void presmooth_residual(const DevCsr& A, const float* d, const float* b, int wdt, float* x, float* r, cudaStream_t s, bool bf = false) { launch_presmooth_residual_f32(A, d, b, wdt, x, r, s, bf); }
void jacobi(const DevCsr& A, const double* d, const double* b, const double* x, int wdt, double* o, cudaStream_t s, bool = false) { launch_jacobi_f64(A, d, b, x, wdt, o, s); }
void jacobi(const DevCsr& A, const float* d, const float* b, const float* x, int wdt, float* o, cudaStream_t s, bool bf = false) { launch_jacobi_f32(A, d, b, x, wdt, o, s, bf); }
void residual(const DevCsr& A, const double* b, const double* x, int wdt, double* r, cudaStream_t s, bool = false) { launch_residual_f64(A, b, x, wdt, r, s); }
void residual(const DevCsr& A, const float* b, const float* x, int wdt, float* r, cudaStream_t s, bool bf = false) { launch_residual_f32(A, b, x, wdt, r, s, bf); }
void spmm(const DevCsr& S, const double* X, int wdt, double* Y, bool acc, cudaStream_t s, bool = false) { launch_spmm_f64(S, X, wdt, Y, acc, s); }
void spmm(const DevCsr& S, const float* X, int wdt, float* Y, bool acc, cudaStream_t s, bool bf = false) { launch_spmm_f32(S, X, wdt, Y, acc, s, bf); }
void jacobi_to_v(const DevCsr& A, const double* d, const double* b, const double* x, int wdt, const double* U, double* V, cudaStream_t s, int) { launch_jacobi_to_v_f64(A, d, b, x, wdt, U, V, s); }
// the float32 V-cycle belongs to the mixed path, whose U and V are float-float
void jacobi_to_v(const DevCsr& A, const float* d, const float* b, const float* x, int wdt, const double* U, double* V, cudaStream_t s, int qv, const float* xadd = nullptr, bool bf = false) { launch_jacobi_to_vdf_f32(A, d, b, x, wdt, reinterpret_cast<const float2*>(U), reinterpret_cast<float2*>(V), s, qv, xadd, bf); }
void add_to_v(const double* U, const double* x, int rows, int q, int, double* V, cudaStream_t s) { launch_add_to_v_f64(U, x, static_cast<long long>(rows) * q, V, s); }
void add_to_v(const double* U, const float* x, int rows, int q, int ldx, double* V, cudaStream_t s) { launch_add_to_vdf(reinterpret_cast<const float2*>(U), x, rows, q, ldx, reinterpret_cast<float2*>(V), s); }
void axpy(const double* x, long long c, double* y, cudaStream_t s) { launch_axpy_f64(x, c, y, s); }
void axpy(const float* x, long long c, float* y, cudaStream_t s) { launch_axpy_f32(x, c, y, s); }
// the V-cycle's operator, l1-Jacobi diagonal and coarsest solve: the
// hierarchy's own, or the shifted ones when the solve asks for a shift
const DevCsr& vop(amgeig_hierarchy_t* h, SolveWork* w, int l) { return w->shifted ? h->sh.A[l] : h->A[l]; }
const double* dinv_of(amgeig_hierarchy_t* h, SolveWork* w, int l, double*) {
  return w->shifted ? h->sh.dinv64[l] : h->dinv64[l];
}
const float* dinv_of(amgeig_hierarchy_t* h, SolveWork* w, int l, float*) {
  return w->shifted ? h->sh.dinv32[l] : h->dinv32[l];
}
void coarse_solve(amgeig_hierarchy_t* h, SolveWork* w, const double* b, int q, double* x, cudaStream_t s) {
  launch_dense_apply(h->dn, q, w->shifted ? h->sh.Ainv : h->Ainv, b, x, s, P_COARSE);
}
void coarse_solve(amgeig_hierarchy_t* h, SolveWork* w, const float* b, int q, float* x, cudaStream_t s) {
  launch_dense_apply(h->dn, q, w->shifted ? h->sh.Ainv32 : h->Ainv32, b, x, s, P_COARSE);
}

// One V-cycle for A_k x = B[k] from x = 0; the result is left in X[k] unless
// to_v, in which case the last sweep on level k writes V = U + x instead.
int width_of(SolveWork* w, double*) { return w->qt; }
int width_of(SolveWork* w, float*) { return w->ld32; }

// First-fit colouring in row order of every level below the coarsest (row i
// takes the smallest colour no neighbour j < i holds; rows of one colour are
// never adjacent), the rows sorted by colour and 1 / a_ii.  Runs once per
// hierarchy, under its lock.
int ensure_gs(amgeig_hierarchy_t* h, cudaStream_t st) {
  if (h->gs_ready) return AMGEIG_OK;
  const int n = h->nlev;
  h->gs_rows.assign(n, nullptr);
  h->gs_off.assign(n, std::vector<int>());
  h->gs_dinv64.assign(n, nullptr);
  h->gs_dinv32.assign(n, nullptr);
  auto& m = h->mem;
  for (int l = 0; l + 1 < n; ++l) {
    const DevCsr& A = h->A[l];
    std::vector<int32_t> rp(static_cast<size_t>(A.rows) + 1), ci(static_cast<size_t>(A.nnz));
    std::vector<double> av(static_cast<size_t>(A.nnz));
    CK(cudaMemcpyAsync(rp.data(), A.rp, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ci.data(), A.ci, sizeof(int32_t) * ci.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(av.data(), A.v64, sizeof(double) * av.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int32_t> col(static_cast<size_t>(A.rows), 0), seen;
    std::vector<double> d64(static_cast<size_t>(A.rows), 0.0);
    for (int32_t i = 0; i < A.rows; ++i) {
      double aii = 0.0;
      for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        const int32_t j = ci[p];
        if (j == i) aii = av[p];
        if (j < i) seen[col[j]] = i;
      }
      int32_t c = 0;
      while (c < static_cast<int32_t>(seen.size()) && seen[c] == i) ++c;
      if (c == static_cast<int32_t>(seen.size())) seen.push_back(-1);
      col[i] = c;
      if (!(aii > 0.0)) return fail(AMGEIG_ECORRUPT, "non-positive diagonal entry in A");
      d64[i] = 1.0 / aii;
    }
    const int nc = static_cast<int>(seen.size());
    std::vector<int>& off = h->gs_off[l];
    off.assign(static_cast<size_t>(nc) + 1, 0);
    for (int32_t i = 0; i < A.rows; ++i) off[col[i] + 1]++;
    for (int c = 0; c < nc; ++c) off[c + 1] += off[c];
    std::vector<int32_t> rows(static_cast<size_t>(A.rows)), pos(off.begin(), off.end() - 1);
    for (int32_t i = 0; i < A.rows; ++i) rows[pos[col[i]]++] = i;
    std::vector<float> d32(d64.begin(), d64.end());
    CK(m.upload(&h->gs_rows[l], rows));
    CK(m.upload(&h->gs_dinv64[l], d64));
    CK(m.upload(&h->gs_dinv32[l], d32));
    CK(cudaStreamSynchronize(m.st));  // the uploads run on the hierarchy's stream
  }
  h->gs_ready = true;
  return AMGEIG_OK;
}

// bfloat16 copies of A_l, R_l and P_l (levels below the coarsest) for
// AMGEIG_MIXED_BF16, rounded from the float32 values on the first such solve.
int ensure_bf16(amgeig_hierarchy_t* h, cudaStream_t st) {
  if (h->bf16_ready) return AMGEIG_OK;
  auto& m = h->mem;
  auto make = [&](DevCsr& D) -> int {
    if (D.vbf || D.nnz == 0) return AMGEIG_OK;
    CK(m.alloc(&D.vbf, static_cast<size_t>(D.nnz)));
    launch_f32_to_bf16(D.v32, D.nnz, D.vbf, st);
    return AMGEIG_OK;
  };
  for (int l = 0; l + 1 < h->nlev; ++l) {
    int rc = make(h->A[l]);
    if (!rc) rc = make(h->R[l]);
    if (!rc) rc = make(h->P[l]);
    if (rc) return rc;
  }
  CK(cudaGetLastError());
  h->bf16_ready = true;
  return AMGEIG_OK;
}

const double* gs_dinv_of(amgeig_hierarchy_t* h, int l, double*) { return h->gs_dinv64[l]; }
const float* gs_dinv_of(amgeig_hierarchy_t* h, int l, float*) { return h->gs_dinv32[l]; }

// One multicolour Gauss-Seidel sweep on level l (colours ascending, or descending)
template <typename T>
void gs_sweep(amgeig_hierarchy_t* h, int l, const T* b, T* x, int ld, bool descending, cudaStream_t st) {
  const DevCsr& A = h->A[l];
  const std::vector<int>& off = h->gs_off[l];
  const int nc = static_cast<int>(off.size()) - 1;
  const double N = A.rows;
  const double sweep = 4.0 * (N + 1) + (4.0 + sizeof(T)) * A.nnz + sizeof(T) * (N + 3.0 * N * ld);
  T* dummy = nullptr;
  for (int k = 0; k < nc; ++k) {
    const int c = descending ? nc - 1 - k : k;
    const int cnt = off[c + 1] - off[c];
    launch_gs_colour(cnt, h->gs_rows[l] + off[c], A, gs_dinv_of(h, l, dummy), b, x, ld, ld, sweep * cnt / N, st);
  }
}

template <typename T>
void vcycle(amgeig_hierarchy_t* h, SolveWork* w, int k, int pre, int post, bool to_v, const double* U, double* V,
            cudaStream_t st, const float* xadd = nullptr) {
  const int q = width_of(w, static_cast<T*>(nullptr));
  const int n = h->nlev;
  auto& B = VBufs<T>::B(w);
  auto& X = VBufs<T>::X(w);
  auto& Tm = VBufs<T>::Tm(w);
  T* dummy = nullptr;
  const bool gs = w->smoother == AMGEIG_SMOOTHER_GAUSS_SEIDEL;
  for (int l = k; l < n - 1; ++l) {
    LevelTag tag(l);
    const DevCsr& A = vop(h, w, l);
    const T* d = dinv_of(h, w, l, dummy);
    if (gs && pre >= 1) {
      // Gauss-Seidel from x = 0, colours ascending; then the residual
      cudaMemsetAsync(X[l], 0, sizeof(T) * h->sizes[l] * q, st);
      for (int s = 0; s < pre; ++s) gs_sweep(h, l, B[l], X[l], q, false, st);
      residual(A, B[l], X[l], q, Tm[l], st);
      spmm(h->R[l], Tm[l], q, B[l + 1], false, st, w->bf16);
    } else if (pre >= 1) {
      presmooth_residual(A, d, B[l], q, X[l], Tm[l], st, w->bf16);
      for (int s = 1; s < pre; ++s) {
        jacobi(A, d, B[l], X[l], q, Tm[l], st, w->bf16);
        std::swap(X[l], Tm[l]);
      }
      if (pre > 1) residual(A, B[l], X[l], q, Tm[l], st, w->bf16);
      spmm(h->R[l], Tm[l], q, B[l + 1], false, st, w->bf16);
    } else {
      cudaMemsetAsync(X[l], 0, sizeof(T) * h->sizes[l] * q, st);
      spmm(h->R[l], B[l], q, B[l + 1], false, st, w->bf16);
    }
  }
  {
    LevelTag tag(n - 1);
    coarse_solve(h, w, B[n - 1], q, X[n - 1], st);
  }
  for (int l = n - 2; l >= k; --l) {
    LevelTag tag(l);
    const DevCsr& A = vop(h, w, l);
    const T* d = dinv_of(h, w, l, dummy);
    spmm(h->P[l], X[l + 1], q, X[l], true, st, w->bf16);
    if (gs) {
      // colours descending after the coarse correction (a symmetric cycle)
      for (int s = 0; s < post; ++s) gs_sweep(h, l, B[l], X[l], q, true, st);
      if (to_v && l == k) {
        if constexpr (std::is_same<T, float>::value)
          if (xadd) axpy(xadd, h->sizes[l] * q, X[l], st);
        add_to_v(U, X[l], static_cast<int>(h->sizes[l]), w->qt, q, V, st);
      }
      continue;
    }
    for (int s = 0; s < post; ++s) {
      if (to_v && l == k && s == post - 1) {
        if constexpr (std::is_same<T, float>::value)
          jacobi_to_v(A, d, B[l], X[l], q, U, V, st, w->qt, xadd, w->bf16);
        else
          jacobi_to_v(A, d, B[l], X[l], q, U, V, st, w->qt);
      } else {
        jacobi(A, d, B[l], X[l], q, Tm[l], st, w->bf16);
        std::swap(X[l], Tm[l]);
      }
    }
    if (to_v && l == k && post == 0) {
      if constexpr (std::is_same<T, float>::value)
        if (xadd) axpy(xadd, h->sizes[l] * q, X[l], st);
      add_to_v(U, X[l], static_cast<int>(h->sizes[l]), w->qt, q, V, st);
    }
  }
}

// m V-cycles in defect-correction form: x_{c+1} = x_c + V(b - A x_c), x_0 = 0;
// the final V = U + x_m.  B[k] holds the defect on entry.
template <typename T>
void amg_correction(amgeig_hierarchy_t* h, SolveWork* w, int k, const amgeig_options& o, const double* U, double* V,
                    cudaStream_t st) {
  const int q = w->qt;
  if (o.v_cycles <= 1) {
    vcycle<T>(h, w, k, o.pre_sweeps, o.post_sweeps, true, U, V, st);
    return;
  }
  auto& B = VBufs<T>::B(w);
  auto& X = VBufs<T>::X(w);
  auto& D = VBufs<T>::D(w);
  auto& E = VBufs<T>::E(w);
  const int wd = width_of(w, static_cast<T*>(nullptr));
  const long long cnt = h->sizes[k] * wd;
  LevelTag tag(k);
  if constexpr (std::is_same<T, float>::value) {
    // the same sums without the copies: the first cycle's result becomes E by a
    // pointer swap, its residual goes to D and trades places with B (D then
    // keeps the original defect), and the last cycle's final sweep writes
    // V = U + (x + E) itself
    vcycle<T>(h, w, k, o.pre_sweeps, o.post_sweeps, false, U, V, st);
    std::swap(X[k], E[k]);
    residual(vop(h, w, k), B[k], E[k], wd, D[k], st, w->bf16);
    std::swap(B[k], D[k]);
    for (int c = 1; c + 1 < o.v_cycles; ++c) {
      vcycle<T>(h, w, k, o.pre_sweeps, o.post_sweeps, false, U, V, st);
      axpy(X[k], cnt, E[k], st);
      residual(vop(h, w, k), D[k], E[k], wd, B[k], st, w->bf16);
    }
    vcycle<T>(h, w, k, o.pre_sweeps, o.post_sweeps, true, U, V, st, E[k]);
    return;
  }
  cudaMemcpyAsync(D[k], B[k], sizeof(T) * cnt, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(E[k], 0, sizeof(T) * cnt, st);
  for (int c = 0; c < o.v_cycles; ++c) {
    vcycle<T>(h, w, k, o.pre_sweeps, o.post_sweeps, false, U, V, st);
    // E += X[k]
    axpy(X[k], cnt, E[k], st);
    if (c + 1 < o.v_cycles) residual(vop(h, w, k), D[k], E[k], wd, B[k], st);
  }
  add_to_v(U, E[k], static_cast<int>(h->sizes[k]), q, wd, V, st);
}

// The correction of m V-cycles for A_k x = B[k] from x = 0 (defect form, as in
// amg_correction, without adding it to an iterate): the pointer to x (row
// stride width_of).  B[k] holds the defect on entry.
template <typename T>
const T* amg_x(amgeig_hierarchy_t* h, SolveWork* w, int k, const amgeig_options& o, cudaStream_t st) {
  auto& B = VBufs<T>::B(w);
  auto& X = VBufs<T>::X(w);
  auto& D = VBufs<T>::D(w);
  auto& E = VBufs<T>::E(w);
  if (o.v_cycles <= 1) {
    vcycle<T>(h, w, k, o.pre_sweeps, o.post_sweeps, false, nullptr, nullptr, st);
    return X[k];
  }
  const int wd = width_of(w, static_cast<T*>(nullptr));
  const long long cnt = h->sizes[k] * wd;
  LevelTag tag(k);
  cudaMemcpyAsync(D[k], B[k], sizeof(T) * cnt, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(E[k], 0, sizeof(T) * cnt, st);
  for (int c = 0; c < o.v_cycles; ++c) {
    vcycle<T>(h, w, k, o.pre_sweeps, o.post_sweeps, false, nullptr, nullptr, st);
    axpy(X[k], cnt, E[k], st);
    if (c + 1 < o.v_cycles) residual(vop(h, w, k), D[k], E[k], wd, B[k], st, w->bf16);
  }
  return E[k];
}

}  // namespace

amgeig_hierarchy_t::~amgeig_hierarchy_t() {
  if (stream) cudaStreamSynchronize(stream);  // nothing in flight uses the blocks released below
  ws.reset();
  pencil_work_destroy(cpw);
  pencil_work_destroy(init.pw);
  mem.st = nullptr;  // drained above; the stream goes before the member buffers are released
  if (stream) cudaStreamDestroy(stream);
}

namespace {

// ------------------------------------------------------------------ one correction (Algorithm 3.1)

// Step 1 (inexact inverse iteration from u_j, in defect form) and step 2
// (augmented pencil on V_n + span(V), its q smallest pairs, recombination).
// On entry U (level k) and lam hold {lambda_j, u_j}; the defect of the current
// pair is already in B[k] (float64 or float32 by precision).
float2* as_df(double* p) { return reinterpret_cast<float2*>(p); }

// Step 2 on the depth-2 Krylov space (the remark after Algorithm 3.1): V_n +
// span(T U, T^2 U) = V_n + span(V1, E) with V1 = T U (step 1) and E the
// correction T V1 - V1 (m V-cycles on the defect of V1 with the same lambda);
// the pencil is taken on the block K = [V1 | E] (Rayleigh-Ritz depends only on
// the span) and its q + q_extra smallest pairs recombined as I_n^k Xc + K Y.
int correction_tail_krylov(amgeig_hierarchy_t* h, SolveWork* w, int k, const amgeig_options& o, cudaStream_t st) {
  const int q = w->qt, nb = 2 * q;
  const int n = h->nlev;
  const int Nk = static_cast<int>(h->sizes[k]);
  const int modes = (o.coarse_modes > 0 && o.coarse_modes < h->dn) ? o.coarse_modes : h->dn;
  int nbk = 0;
  if (o.precision == AMGEIG_FP64) {
    amg_correction<double>(h, w, k, o, w->U, w->V, st);
    launch_defect_f64(h->A[k], w->V, q, w->lam, w->B64[k], nullptr, &nbk, st);
    const double* E = amg_x<double>(h, w, k, o, st);
    launch_pack_krylov_f64(Nk, w->V, E, q, q, w->K, st);
    launch_dual_spmm(h->A[k], w->K, nb, w->W, st);
    launch_gram(Nk, w->K, nb, w->W, 2 * nb, w->gsc, w->G, st, false);
    const double* cur = w->W;
    for (int l = k; l < n - 1; ++l) {
      launch_spmm_f64(h->R[l], cur, 2 * nb, w->WC[l + 1], false, st, P_CHAIN);
      cur = w->WC[l + 1];
    }
    launch_pencil_solve(w->pw, h->dn, modes, nb, cur, nullptr, w->G, h->Zdf, h->theta, w->mu, w->Xc, nullptr,
                        w->Yv, h->dstatus, st, w->nfallback, q);
    const double* px = w->Xc;
    for (int l = n - 2; l >= k; --l) {
      launch_spmm_f64(h->P[l], px, q, w->PX[l], false, st, P_CHAIN);
      px = w->PX[l];
    }
    launch_recombine_wide(Nk, px, w->K, nb, w->Yv, q, w->U, st);
  } else {
    amg_correction<float>(h, w, k, o, w->U, w->V, st);
    launch_defect_df(h->A[k], as_df(w->V), q, w->lam, w->B32[k], w->ld32, nullptr, &nbk, st);
    const float* E = amg_x<float>(h, w, k, o, st);
    launch_pack_krylov_df(Nk, as_df(w->V), E, w->ld32, q, as_df(w->K), st);
    launch_dual_spmm_df(h->A[k], as_df(w->K), nb, as_df(w->W), st);
    launch_gram_df(Nk, as_df(w->K), nb, as_df(w->W), 2 * nb, w->gsc, w->G, st, h->dstatus);
    const float2* cur = as_df(w->W);
    for (int l = k; l < n - 1; ++l) {
      launch_spmm_df(h->R[l], cur, 2 * nb, as_df(w->WC[l + 1]), false, st, P_CHAIN);
      cur = as_df(w->WC[l + 1]);
    }
    launch_pencil_solve(w->pw, h->dn, modes, nb, nullptr, cur, w->G, h->Zdf, h->theta, w->mu, w->Xc,
                        as_df(w->PX[n - 1]), w->Yv, h->dstatus, st, w->nfallback, q);
    const DevCsr& PC = h->PC[k];
    launch_recombine_pc_df(Nk, PC.nnz, PC.rp, PC.ci, PC.d2, as_df(w->PX[n - 1]), as_df(w->K), w->Yv, q,
                           as_df(w->U), st, nb);
  }
  {
    ProfScope ps(st, P_OTHER, 16.0 * q, 0.0);
    k_copy_d<<<1, 128, 0, st>>>(w->mu, q, w->lam);
  }
  CK(cudaGetLastError());
  return AMGEIG_OK;
}

int correction_tail(amgeig_hierarchy_t* h, SolveWork* w, int k, const amgeig_options& o, cudaStream_t st) {
  if (o.krylov == 2) return correction_tail_krylov(h, w, k, o, st);
  const int q = w->qt;
  const int n = h->nlev;
  const int Nk = static_cast<int>(h->sizes[k]);
  const int modes = (o.coarse_modes > 0 && o.coarse_modes < h->dn) ? o.coarse_modes : h->dn;
  if (o.precision == AMGEIG_FP64) {
    amg_correction<double>(h, w, k, o, w->U, w->V, st);
    // augmentation: W = [A_k V | M_k V], G = V^T W, C = I_k^n W
    launch_dual_spmm(h->A[k], w->V, q, w->W, st);
    launch_gram(Nk, w->V, q, w->W, 2 * q, w->gsc, w->G, st, false);
    const double* cur = w->W;
    for (int l = k; l < n - 1; ++l) {
      launch_spmm_f64(h->R[l], cur, 2 * q, w->WC[l + 1], false, st, P_CHAIN);
      cur = w->WC[l + 1];
    }
    launch_pencil_solve(w->pw, h->dn, modes, q, cur, nullptr, w->G, h->Zdf, h->theta, w->mu, w->Xc, nullptr, w->Yv,
                        h->dstatus, st, w->nfallback);
    // recombination: U = I_n^k Xc + V Y
    const double* px = w->Xc;
    for (int l = n - 2; l >= k; --l) {
      launch_spmm_f64(h->P[l], px, q, w->PX[l], false, st, P_CHAIN);
      px = w->PX[l];
    }
    launch_recombine(Nk, px, w->V, w->Yv, q, w->U, st, false);
  } else {
    // mixed path: float32 V-cycle; U, V, W and the chains in float-float
    amg_correction<float>(h, w, k, o, w->U, w->V, st);
    launch_dual_spmm_df(h->A[k], as_df(w->V), q, as_df(w->W), st);
    launch_gram_df(Nk, as_df(w->V), q, as_df(w->W), 2 * q, w->gsc, w->G, st, h->dstatus);
    const float2* cur = as_df(w->W);
    for (int l = k; l < n - 1; ++l) {
      launch_spmm_df(h->R[l], cur, 2 * q, as_df(w->WC[l + 1]), false, st, P_CHAIN);
      cur = as_df(w->WC[l + 1]);
    }
    launch_pencil_solve(w->pw, h->dn, modes, q, nullptr, cur, w->G, h->Zdf, h->theta, w->mu, w->Xc,
                        as_df(w->PX[n - 1]), w->Yv, h->dstatus, st, w->nfallback);
    if (q <= 32) {
      // U = I_n^k Xc + V Y in one pass: the composite prolongation is applied row by row
      const DevCsr& PC = h->PC[k];
      launch_recombine_pc_df(Nk, PC.nnz, PC.rp, PC.ci, PC.d2, as_df(w->PX[n - 1]), as_df(w->V), w->Yv, q,
                             as_df(w->U), st);
      CK(cudaGetLastError());
      {
        ProfScope ps(st, P_OTHER, 16.0 * q, 0.0);
        k_copy_d<<<1, 128, 0, st>>>(w->mu, q, w->lam);
      }
      CK(cudaGetLastError());
      return AMGEIG_OK;
    }
    const float2* px = as_df(w->PX[n - 1]);
    for (int l = n - 2; l >= k; --l) {
      launch_spmm_df(h->P[l], px, q, as_df(w->PX[l]), false, st, P_CHAIN);
      px = as_df(w->PX[l]);
    }
    launch_recombine_df(Nk, px, as_df(w->V), w->Yv, q, as_df(w->U), st, as_df(w->Ydf), h->dstatus);
  }
  {
    ProfScope ps(st, P_OTHER, 16.0 * q, 0.0);
    k_copy_d<<<1, 128, 0, st>>>(w->mu, q, w->lam);
  }
  CK(cudaGetLastError());
  return AMGEIG_OK;
}

int defect(amgeig_hierarchy_t* h, SolveWork* w, int k, const amgeig_options& o, bool norms, cudaStream_t st) {
  const int q = w->qt;
  int nb = 0;
  double* part = norms ? w->partials : nullptr;
  if (o.precision == AMGEIG_FP64)
    launch_defect_f64(h->A[k], w->U, q, w->lam, w->B64[k], part, &nb, st);
  else
    launch_defect_df(h->A[k], as_df(w->U), q, w->lam, w->B32[k], w->ld32, part, &nb, st);
  if (norms) {
    launch_sum_partials(w->partials, nb, 2 * q, w->sums, st);
    CK(cudaMemsetAsync(w->flags, 0, sizeof(int), st));
    launch_relres(w->sums, w->lam, q, w->relres, w->flags, st);
  }
  CK(cudaGetLastError());
  return AMGEIG_OK;
}

int check_options(const amgeig_options& o) {
  if (o.max_corrections < 0 || o.v_cycles < 1 || o.pre_sweeps < 0 || o.post_sweeps < 0 || o.q_extra < 0 ||
      o.fixed_corrections < 0 || o.coarse_modes < 0 ||
      (o.precision != AMGEIG_FP64 && o.precision != AMGEIG_MIXED_FP32 && o.precision != AMGEIG_MIXED_BF16) ||
      (o.smoother != AMGEIG_SMOOTHER_L1_JACOBI && o.smoother != AMGEIG_SMOOTHER_GAUSS_SEIDEL) || o.n1 < -1 ||
      (o.refine < 0 || o.refine > 2) || (o.graphs != 0 && o.graphs != 1) || (o.autotune != 0 && o.autotune != 1) ||
      (o.batch != 0 && o.batch != 1) || !std::isfinite(o.shift) || (o.krylov != 1 && o.krylov != 2) ||
      (o.shift != 0.0 && (o.smoother != AMGEIG_SMOOTHER_L1_JACOBI || o.precision == AMGEIG_MIXED_BF16)))
    return fail(AMGEIG_EINVAL, "invalid options");
  return AMGEIG_OK;
}

// The leading `need` eigenpairs of the coarsest pencil (computed again, all of
// them, when a solve asks for more than are ready).  Under the hierarchy's lock.
int ensure_modes(amgeig_hierarchy_t* h, int need, cudaStream_t st) {
  if (need <= h->modes_ready) return AMGEIG_OK;
  launch_coarse_modes(h->cpw, h->dn, need, h->An, h->Z, h->theta, st);
  launch_f64_to_df(h->Z, static_cast<long long>(h->dn) * h->dn, h->Zdf, st);
  CK(cudaGetLastError());
  h->modes_ready = need;
  return AMGEIG_OK;
}

// ------------------------------------------------------------------ CUDA graphs

// Which buffer plays which role: the workspace swaps buffer pointers between
// launches (the iterate and its copy, smoothing in/out, defect and residual),
// so a captured launch sequence is valid only from the roles it was captured in.
std::vector<void*> roles(SolveWork* w) {
  std::vector<void*> r = {w->U, w->Ualt, w->V, w->W};
  for (auto* v : {&w->B64, &w->X64, &w->T64, &w->D64, &w->E64})
    for (double* p : *v) r.push_back(p);
  for (auto* v : {&w->B32, &w->X32, &w->T32, &w->D32, &w->E32})
    for (float* p : *v) r.push_back(p);
  return r;
}

void set_roles(SolveWork* w, const std::vector<void*>& r) {
  size_t i = 0;
  w->U = static_cast<double*>(r[i++]);
  w->Ualt = static_cast<double*>(r[i++]);
  w->V = static_cast<double*>(r[i++]);
  w->W = static_cast<double*>(r[i++]);
  for (auto* v : {&w->B64, &w->X64, &w->T64, &w->D64, &w->E64})
    for (double*& p : *v) p = static_cast<double*>(r[i++]);
  for (auto* v : {&w->B32, &w->X32, &w->T32, &w->D32, &w->E32})
    for (float*& p : *v) p = static_cast<float*>(r[i++]);
}

// Run the launch sequence `body` on st.  With graphs on (and no profiling, and
// st not already capturing), the second run of a (segment, settings, roles)
// combination captures the sequence as a CUDA graph and later runs replay it:
// one launch instead of the sequence's hundred-odd, with no host work between
// kernels.  body must only enqueue work (no host synchronisation).
template <class F>
int run_segment(SolveWork* w, const amgeig_options& o, const std::string& seg, cudaStream_t st, F body) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!o.graphs || profiling_on() || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone)
    return body();
  std::vector<void*> pre = roles(w);
  std::string key = seg;
  const int cfg[] = {w->qt, w->ld32, o.precision, o.v_cycles, o.pre_sweeps, o.post_sweeps, o.smoother,
                     o.coarse_modes, w->bf16 ? 1 : 0, w->shifted ? 1 : 0, o.krylov};
  key.append(reinterpret_cast<const char*>(cfg), sizeof(cfg));
  key.append(reinterpret_cast<const char*>(&o.shift), sizeof(o.shift));
  key.append(reinterpret_cast<const char*>(pre.data()), sizeof(void*) * pre.size());
  auto it = w->graphs.find(key);
  if (it == w->graphs.end()) {
    // capture only a combination seen before: a one-off solve (a freshly loaded
    // hierarchy solved once) does not pay for capturing and instantiating
    if (w->graph_seen[key]++ == 0) return body();
    const unsigned long long k0 = thread_launch_count();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    const int rc = body();
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &g);
    if (rc != AMGEIG_OK) {
      if (g) cudaGraphDestroy(g);
      set_roles(w, pre);
      return rc;
    }
    if (ec != cudaSuccess) return fail(AMGEIG_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    SolveWork::Graph rec;
    const cudaError_t ei = cudaGraphInstantiate(&rec.exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail(AMGEIG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    rec.post = roles(w);
    // the kernels were counted when captured (on this thread; other threads
    // launch meanwhile); the launch below runs them
    rec.kernels = thread_launch_count() - k0;
    it = w->graphs.emplace(key, std::move(rec)).first;
    CK(cudaGraphLaunch(it->second.exec, st));
    return AMGEIG_OK;
  }
  CK(cudaGraphLaunch(it->second.exec, st));
  add_launches(it->second.kernels);
  set_roles(w, it->second.post);
  return AMGEIG_OK;
}

// The shifted operators for sigma (Algorithm 3.1's remark: a shifted linear
// solve in step 1), made on the GPU: A_l - sigma M_l on every level below the
// coarsest (float64 and float32 values on the shared pattern), their l1
// diagonals, and (A_n - sigma M_n)^-1 from its float64 Cholesky factor.
// EINVAL when A_n - sigma M_n is not positive definite (sigma not below the
// coarsest pencil's lowest eigenvalue).  Under the hierarchy's lock.
int ensure_shift(amgeig_hierarchy_t* h, double sigma, cudaStream_t st) {
  auto& S = h->sh;
  const int n = h->nlev, dn = h->dn;
  if (S.ready && S.sigma == sigma) return AMGEIG_OK;
  auto& m = h->mem;
  if (S.A.empty()) {
    S.A.assign(n > 1 ? n - 1 : 0, DevCsr());
    S.dinv64.assign(n, nullptr);
    S.dinv32.assign(n, nullptr);
    for (int l = 0; l + 1 < n; ++l) {
      const DevCsr& A = h->A[l];
      DevCsr& D = S.A[l];
      D.rows = A.rows;
      D.cols = A.cols;
      D.nnz = A.nnz;
      D.rp = A.rp;
      D.ci = A.ci;
      D.m64 = A.m64;
      CK(m.alloc(&D.v64, static_cast<size_t>(A.nnz)));
      CK(m.alloc(&D.v32, static_cast<size_t>(A.nnz)));
      CK(m.alloc(&S.dinv64[l], static_cast<size_t>(A.rows)));
      CK(m.alloc(&S.dinv32[l], static_cast<size_t>(A.rows)));
    }
    const size_t dd = static_cast<size_t>(dn) * dn;
    CK(m.alloc(&S.Bn, dd));
    CK(m.alloc(&S.L, dd));
    CK(m.alloc(&S.Linv, dd));
    CK(m.alloc(&S.Ainv, dd));
    CK(m.alloc(&S.Ainv32, dd));
  }
  S.ready = false;
  int* flag = h->dstatus + 3;
  CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
  for (int l = 0; l + 1 < n; ++l) {
    DevCsr& D = S.A[l];
    std::memcpy(D.tuned, h->A[l].tuned, sizeof(D.tuned));
    launch_axpby_f64(h->A[l].v64, -sigma, h->A[l].m64, D.nnz, D.v64, st);
    launch_convert_f64_to_f32(D.v64, D.nnz, D.v32, st);
    launch_l1_inv_diag(D, S.dinv64[l], S.dinv32[l], flag, st);
  }
  launch_axpby_f64(h->An, -sigma, h->Mn, static_cast<long long>(dn) * dn, S.Bn, st);
  launch_coarse_inverse(dn, S.Bn, S.L, S.Linv, S.Ainv, flag, st);
  launch_convert_f64_to_f32(S.Ainv, static_cast<long long>(dn) * dn, S.Ainv32, st);
  CK(cudaGetLastError());
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) return fail(AMGEIG_EINVAL, "shift not below the lowest eigenvalue of the coarsest pencil");
  S.sigma = sigma;
  S.ready = true;
  return AMGEIG_OK;
}

// Launch shapes of the float32 V-cycle kernels for this solve's width, tuned on
// its first mixed solve at that width (smoothing on every A_l, restriction R_l
// and prolongation P_l): every lane layout is timed on the level's own
// operator and the fastest is kept in the hierarchy.  Layouts that split a
// row's nonzeros over several lane streams add its terms in another order, so
// tuned solves can differ from untuned ones by float32 rounding in the V-cycle
// (the fixed point is the same); a hierarchy keeps its choice, so its solves
// repeat bit for bit.  Before any capture; under the lock.
// Tuned shapes are also kept per process, keyed by the operator's role, shape
// and nonzero count and the width: a hierarchy loaded again (the same problem)
// takes them without timing anything.
struct TuneKey {
  int role, w4;
  int64_t rows, cols, nnz;
  bool operator<(const TuneKey& o) const {
    return std::tie(role, w4, rows, cols, nnz) < std::tie(o.role, o.w4, o.rows, o.cols, o.nnz);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<unsigned char, TuneResult>> g_tuned;

TuneResult tune_or_reuse(DevCsr& S, int role, int kind, int w4, const float* dinv, const float* x, const float* b,
                         float* out, cudaStream_t st) {
  const TuneKey key{role, w4, S.rows, S.cols, S.nnz};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      S.tuned[w4] = it->second.first;
      return it->second.second;
    }
  }
  const TuneResult r = autotune_f4(S, kind, w4, dinv, x, b, out, st);
  if (S.tuned[w4]) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = std::make_pair(S.tuned[w4], r);
  }
  return r;
}

int ensure_tuned(amgeig_hierarchy_t* h, SolveWork* w, cudaStream_t st) {
  const int w4 = w->ld32 / 4;
  if (w4 < 1 || w4 > 32 || h->tuned_w4[w4]) return AMGEIG_OK;
  const int n = h->nlev;
  for (int l = 0; l + 1 < n; ++l) {
    const size_t cl = static_cast<size_t>(h->sizes[l]) * w->ld32, cn = static_cast<size_t>(h->sizes[l + 1]) * w->ld32;
    CK(cudaMemsetAsync(w->X32[l], 0, sizeof(float) * cl, st));
    CK(cudaMemsetAsync(w->B32[l], 0, sizeof(float) * cl, st));
    CK(cudaMemsetAsync(w->X32[l + 1], 0, sizeof(float) * cn, st));
    const TuneResult a = tune_or_reuse(h->A[l], 0, 0, w4, h->dinv32[l], w->X32[l], w->B32[l], w->T32[l], st);
    const TuneResult r = tune_or_reuse(h->R[l], 1, 1, w4, nullptr, w->T32[l], nullptr, w->B32[l + 1], st);
    const TuneResult p = tune_or_reuse(h->P[l], 2, 1, w4, nullptr, w->X32[l + 1], nullptr, w->T32[l], st);
    char line[512];
    const TuneResult* tr[3] = {&a, &r, &p};
    const char* nm[3] = {"smooth", "restrict", "prolong"};
    for (int i = 0; i < 3; ++i) {
      std::snprintf(line, sizeof(line),
                    "%s{\"level\": %d, \"kernel\": \"%s\", \"w4\": %d, \"G\": %d, \"cpt\": %d, \"S\": %d, "
                    "\"us\": %.2f, \"rule_G\": %d, \"rule_cpt\": %d, \"rule_us\": %.2f}",
                    h->tune_log.empty() ? "" : ", ", l, nm[i], w4, tr[i]->G, tr[i]->cpt, tr[i]->S, tr[i]->us,
                    tr[i]->rule_G, tr[i]->rule_cpt, tr[i]->rule_us);
      h->tune_log += line;
    }
  }
  CK(cudaGetLastError());
  h->tuned_w4[w4] = true;
  return AMGEIG_OK;
}

// The `count` lowest eigenpairs of (A_l, M_l) on level l (above the coarsest),
// Algorithm 3.2 step 1 with n1 = l: the level's dense pencil, the Cholesky
// factor of M_l and the float-float eigensolver of the coarse modes.  Kept for
// later solves; under the hierarchy's lock.
int ensure_initial(amgeig_hierarchy_t* h, int l, int count, cudaStream_t st) {
  auto& I = h->init;
  if (I.level == l && I.count >= count) return AMGEIG_OK;
  const int d = static_cast<int>(h->sizes[l]);
  if (I.level != l) {
    // arrays of an earlier level stay in the hierarchy's allocations until it is freed
    const size_t dd = static_cast<size_t>(d) * d;
    CK(h->mem.alloc(&I.A, dd));
    CK(h->mem.alloc(&I.M, dd));
    CK(h->mem.alloc(&I.Z, dd));
    CK(h->mem.alloc(&I.theta, static_cast<size_t>(d)));
    pencil_work_destroy(I.pw);
    cudaError_t e;
    I.pw = pencil_work_create(d, 1, &e);
    if (!I.pw) {
      I.level = -1;
      return fail(AMGEIG_ENOMEM, std::string("initial-level workspace: ") + cudaGetErrorString(e));
    }
    I.level = l;
    I.d = d;
    I.count = 0;
    const DevCsr& L = h->A[l];
    launch_csr_to_dense(d, L.rp, L.ci, L.v64, L.m64, I.A, I.M, st);
  }
  CK(cudaMemsetAsync(h->dstatus + 2, 0, sizeof(int), st));
  launch_mass_factor(I.pw, d, I.M, h->dstatus + 2, st);
  launch_coarse_modes(I.pw, d, count, I.A, I.Z, I.theta, st);
  CK(cudaGetLastError());
  int stt = 0;
  CK(cudaMemcpyAsync(&stt, h->dstatus + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (stt) {
    I.count = 0;
    return fail(AMGEIG_ENOTSPD, "M on the initial level is not positive definite");
  }
  I.count = count;
  return AMGEIG_OK;
}

// Mixed path, after the last correction: float64 Rayleigh quotients and
// relative residuals of the finest-level vectors with the exact operator values
// (V receives the iterate in float64, W the residual block); lam receives the
// quotients in ascending order, perm the matching columns, relres the residual
// of each column (unpermuted).
int refine_fp64(amgeig_hierarchy_t* h, SolveWork* w, bool compensated, bool fp64_path, cudaStream_t st) {
  const int qt = w->qt;
  const long long cnt = h->sizes[0] * static_cast<long long>(qt);
  double* X = w->U;
  if (!fp64_path) {
    launch_df_to_f64(as_df(w->U), cnt, w->V, st);
    X = w->V;
  }
  launch_rayleigh_f64(h->A[0], X, qt, compensated, w->partials, w->sums, st);
  launch_rq_finish(w->sums, qt, w->mu, w->lam, w->perm, w->relres, w->flags, st);
  int redo = 0;
  CK(cudaMemcpyAsync(&redo, w->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (redo == 2) return fail(AMGEIG_ENAN, "NaN or Inf in the refined Rayleigh quotients");
  if (redo) {
    // small residuals: form them explicitly with the refined quotients
    int nb = 0;
    launch_defect_f64(h->A[0], X, qt, w->mu, w->W, w->partials, &nb, st);
    launch_sum_partials(w->partials, nb, 2 * qt, w->sums, st);
    CK(cudaMemsetAsync(w->flags, 0, sizeof(int), st));
    launch_relres(w->sums, w->mu, qt, w->relres, w->flags, st);
  }
  CK(cudaGetLastError());
  w->refined = X;
  w->permuted = true;
  return AMGEIG_OK;
}

// Algorithm 3.2 on the hierarchy's stream; results stay in the workspace.
int solve_impl(amgeig_hierarchy_t* h, int q, double tol, const amgeig_options& o, amgeig_info* info,
               std::vector<double>& relres_host, cudaStream_t st) {
  const int qt = q + o.q_extra;
  const int n = h->nlev;
  int rc = check_options(o);
  if (rc) return rc;
  if (q < 1 || qt > h->sizes[0]) return fail(AMGEIG_EINVAL, "q + q_extra must be in [1, finest dimension]");
  if (qt > 128) return fail(AMGEIG_EINVAL, "q + q_extra must be at most 128");
  // n1: the coarsest level that holds q + q_extra pairs (n1 = n when d_n suffices)
  int n1 = o.n1;
  if (n1 < 0) {
    n1 = n - 1;
    while (n1 > 0 && h->sizes[n1] < qt) --n1;
  }
  if (n1 >= n || h->sizes[n1] < qt) return fail(AMGEIG_EINVAL, "n1 must be a level with at least q + q_extra rows");
  if (n1 < n - 1 && h->sizes[n1] > 2048)
    return fail(AMGEIG_EINVAL, "the initial level above the coarsest must have at most 2048 rows");
  if (o.krylov == 2 && (2 * qt > 128 || (o.precision != AMGEIG_FP64 && qt > 32)))
    return fail(AMGEIG_EINVAL, "the Krylov space needs 2 (q + q_extra) <= 128 (and q + q_extra <= 32 when mixed)");
  rc = ensure_workspace(h, qt, o.precision, std::max(1, o.v_cycles), o.krylov == 2 ? 2 * qt : 0);
  if (rc) return rc;
  SolveWork* w = h->ws.get();
  w->permuted = false;
  w->smoother = o.smoother;
  if (o.smoother == AMGEIG_SMOOTHER_GAUSS_SEIDEL) {
    rc = ensure_gs(h, st);
    if (rc) return rc;
  }
  w->bf16 = o.precision == AMGEIG_MIXED_BF16;
  if (w->bf16) {
    rc = ensure_bf16(h, st);
    if (rc) return rc;
  }
  w->shifted = o.shift != 0.0;
  if (w->shifted) {
    rc = ensure_shift(h, o.shift, st);
    if (rc) return rc;
  }
  if (o.precision != AMGEIG_FP64 && o.autotune) {
    rc = ensure_tuned(h, w, st);
    if (rc) return rc;
  }
  {
    const int modes = (o.coarse_modes > 0 && o.coarse_modes < h->dn) ? o.coarse_modes : h->dn;
    rc = ensure_modes(h, n1 == n - 1 ? std::max(modes, qt) : modes, st);
    if (rc) return rc;
  }
  // step 1: initial eigenpairs on level n1 (the coarsest unless it is too small)
  const double* Z0 = h->Z;
  const double* theta0 = h->theta;
  int d0 = h->dn;
  if (n1 < n - 1) {
    rc = ensure_initial(h, n1, qt, st);
    if (rc) return rc;
    Z0 = h->init.Z;
    theta0 = h->init.theta;
    d0 = h->init.d;
  }
  if (o.precision == AMGEIG_FP64)
    launch_copy_cols(Z0, d0, d0, qt, w->U, st);
  else
    launch_cols_to_df(Z0, d0, d0, qt, as_df(w->U), st);
  {
    ProfScope ps(st, P_OTHER, 16.0 * qt, 0.0);
    k_copy_d<<<1, 128, 0, st>>>(theta0, qt, w->lam);
  }
  CK(cudaMemsetAsync(w->nfallback, 0, sizeof(int), st));
  // the pencil kernels only ever set the status (Cholesky of the Gram Schur
  // complement failed), so one clear per solve suffices and the nested phase
  // runs without host round trips: its status is read with the first
  // finest-level residual
  CK(cudaMemsetAsync(h->dstatus, 0, sizeof(int), st));
  CK(cudaGetLastError());
  int corrections = 0;
  bool converged = false;
  relres_host.assign(qt, 0.0);
  // step 2: k = n1-1 .. 1 (0-based) one correction each after the prolongation,
  // then the prolongation to the finest level and its first defect (one launch
  // segment), then the finest level's corrections (one segment each: the
  // correction and the next defect) until the stopping test
  if (n1 > 0) {
    rc = run_segment(w, o, "nested " + std::to_string(n1), st, [&]() -> int {
      for (int k = n1 - 1; k >= 0; --k) {
        if (o.precision == AMGEIG_FP64)
          launch_spmm_f64(h->P[k], w->U, qt, w->Ualt, false, st, P_CHAIN);
        else
          launch_spmm_df(h->P[k], as_df(w->U), qt, as_df(w->Ualt), false, st, P_CHAIN);
        std::swap(w->U, w->Ualt);
        int r = defect(h, w, k, o, k == 0, st);
        if (r) return r;
        if (k >= 1) {
          r = correction_tail(h, w, k, o, st);
          if (r) return r;
        }
      }
      return AMGEIG_OK;
    });
    if (rc) return rc;
    for (;;) {
      int flags = 0;
      CK(cudaMemcpyAsync(relres_host.data(), w->relres, sizeof(double) * qt, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(&flags, w->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
      int stt = 0;
      CK(cudaMemcpyAsync(&stt, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (stt == AMGEIG_ECUDA) return fail(stt, "a bulk copy into shared memory did not complete in time");
      if (stt) return fail(stt, "augmented pencil: Gram Schur complement not positive definite");
      if (flags) return fail(AMGEIG_ENAN, "NaN or Inf in the iterates");
      double mx = 0.0;
      for (int j = 0; j < q; ++j) mx = std::max(mx, relres_host[j]);
      if (o.fixed_corrections > 0) {
        if (corrections == o.fixed_corrections) {
          converged = mx <= tol;
          break;
        }
      } else {
        if (mx <= tol) {
          converged = true;
          break;
        }
        if (corrections == o.max_corrections) break;
      }
      rc = run_segment(w, o, "finest", st, [&]() -> int {
        const int r = correction_tail(h, w, 0, o, st);
        if (r) return r;
        return defect(h, w, 0, o, true, st);
      });
      if (rc) return rc;
      ++corrections;
    }
  }
  if (n1 == 0) {
    // the initial level is the finest: its eigenpairs are the answer; report their residual
    rc = defect(h, w, 0, o, true, st);
    if (rc) return rc;
    CK(cudaMemcpyAsync(relres_host.data(), w->relres, sizeof(double) * qt, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double mx = 0.0;
    for (int j = 0; j < q; ++j) mx = std::max(mx, relres_host[j]);
    converged = mx <= tol;
  }
  if (o.refine) {
    // the returned values and residuals: float64 (or compensated float64)
    // Rayleigh quotients of the final vectors; the stopping decision above
    // stands unless the float64 residuals contradict it
    rc = refine_fp64(h, w, o.refine == 2, o.precision == AMGEIG_FP64, st);
    if (rc) return rc;
    std::vector<int> perm(qt);
    std::vector<double> rr(qt);
    int flags = 0;
    CK(cudaMemcpyAsync(rr.data(), w->relres, sizeof(double) * qt, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(perm.data(), w->perm, sizeof(int) * qt, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&flags, w->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flags) return fail(AMGEIG_ENAN, "NaN or Inf in the refined Rayleigh quotients");
    for (int c = 0; c < qt; ++c) relres_host[c] = rr[perm[c]];
    double mx = 0.0;
    for (int j = 0; j < q; ++j) mx = std::max(mx, relres_host[j]);
    converged = mx <= tol;
  }
  if (info) {
    double mx = 0.0;
    for (int j = 0; j < q; ++j) mx = std::max(mx, relres_host[j]);
    int nfb = 0;
    CK(cudaMemcpyAsync(&nfb, w->nfallback, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    info->dense_fallbacks = nfb;
    info->corrections = corrections;
    info->converged = converged ? 1 : 0;
    info->n1 = n1;
    info->max_relres = mx;
    info->status = converged ? AMGEIG_OK : AMGEIG_ENOCONV;
  }
  return converged ? AMGEIG_OK : AMGEIG_ENOCONV;
}

// Copy the q wanted eigenvalues / sign-normalised eigenvectors out.
int write_outputs(amgeig_hierarchy_t* h, int q, double* eigvals, double* eigvecs, int on_device, cudaStream_t st) {
  SolveWork* w = h->ws.get();
  const int qt = w->qt;
  const int N0 = static_cast<int>(h->sizes[0]);
  if (eigvals) CK(cudaMemcpyAsync(eigvals, w->lam, sizeof(double) * q, cudaMemcpyDeviceToHost, st));
  if (eigvecs) {
    const double* src = w->U;
    int ld = qt;
    if (w->permuted) {
      // the refined float64 iterate's columns perm[0..q) gathered into the other
      // of U and V (both free after the solve)
      double* g = w->refined == w->U ? w->V : w->U;
      launch_gather_cols(w->refined, N0, qt, w->perm, q, g, st);
      src = g;
      ld = q;
    } else if (w->precision != AMGEIG_FP64) {
      // float-float iterate -> float64 (V is free after the solve)
      launch_df_to_f64(as_df(w->U), static_cast<long long>(N0) * qt, w->V, st);
      src = w->V;
    }
    double* dst = on_device ? eigvecs : w->Ualt;  // Ualt is free after the solve
    const long long total = static_cast<long long>(N0) * q;
    ProfScope ps(st, P_OTHER, 8.0 * N0 * qt + 16.0 * total, 0.0, 3);
    {
      const int slab = 512, nslabs = ceil_div(N0, slab);
      // the slab results live in W, free after the solve (nslabs * q <= N0 * 2q)
      double* bval = w->W;
      int* bidx = reinterpret_cast<int*>(w->W + static_cast<size_t>(nslabs) * q);
      k_col_best<<<nslabs, 256, 0, st>>>(src, N0, ld, q, slab, bval, bidx);
      k_col_sign2<<<q, kSignThreads, 0, st>>>(src, ld, q, nslabs, bval, bidx, w->sign);
    }
    k_out_vectors<<<static_cast<int>(std::min<long long>((total + 255) / 256, 8LL * kNumSms)), 256, 0, st>>>(
        src, N0, ld, q, w->sign, dst);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpyAsync(eigvecs, dst, sizeof(double) * total, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  return AMGEIG_OK;
}

// ------------------------------------------------------------------ request service

struct Request {
  uint64_t id;
  amgeig_hierarchy_t* h;
  int q;
  double tol;
  amgeig_options opt;
  bool done = false;
  int status = AMGEIG_OK;
  std::vector<double> vals, vecs;
  amgeig_info info{};
  // queued requests on the same hierarchy that share this request's solve
  std::vector<std::shared_ptr<Request>> riders;
};

// Two requests can share one solve when everything but the wanted count, the
// buffer and the tolerance agrees (the shared solve takes the widest of each
// and the tightest tolerance).
bool can_share(const Request& a, const Request& b) {
  const amgeig_options &x = a.opt, &y = b.opt;
  return a.h == b.h && x.batch && y.batch && x.fixed_corrections == 0 && y.fixed_corrections == 0 &&
         x.precision == y.precision && x.v_cycles == y.v_cycles && x.pre_sweeps == y.pre_sweeps &&
         x.post_sweeps == y.post_sweeps && x.coarse_modes == y.coarse_modes && x.smoother == y.smoother &&
         x.n1 == y.n1 && x.refine == y.refine && x.graphs == y.graphs && x.autotune == y.autotune &&
         x.shift == y.shift && x.krylov == y.krylov;
}

// Continuous batching over hierarchies: kWorkers library threads take queued
// requests in arrival order, skipping one whose hierarchy is busy (a hierarchy
// runs one solve at a time on its own stream, so requests on different
// hierarchies overlap on the device).  A request whose workspace does not fit
// in free device memory waits while others run and is admitted when one ends;
// with nothing else running it is tried anyway (and fails with ENOMEM if it
// cannot fit at all).
constexpr int kWorkers = 4;

struct Service {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> table;
  std::vector<amgeig_hierarchy_t*> busy;
  // hierarchies whose workspace the service has used, least recently used first;
  // under a memory limit, idle ones give their workspace back to admit others
  std::vector<amgeig_hierarchy_t*> resident;
  // admitted requests whose workspace is being made: the bytes it will hold
  std::map<amgeig_hierarchy_t*, size_t> reserved;
  size_t mem_limit = 0;  // bytes of resident workspaces the service may hold (0: no limit)
  uint64_t evictions = 0;
  uint64_t next_id = 1;
  int running_solves = 0;
  bool started = false;

  void start() {
    if (started) return;
    started = true;
    for (int i = 0; i < kWorkers; ++i) std::thread([this] { loop(); }).detach();
  }

  bool is_busy(amgeig_hierarchy_t* h) const { return std::find(busy.begin(), busy.end(), h) != busy.end(); }

  // first admissible request (caller holds mu).  A request that cannot fit
  // under the memory limit even with every idle workspace released, while
  // nothing else runs, is refused here with ENOMEM.
  std::shared_ptr<Request> pick() {
    for (auto it = queue.begin(); it != queue.end();) {
      const std::shared_ptr<Request> r = *it;
      if (is_busy(r->h)) {
        ++it;
        continue;
      }
      const int f = fits(r.get());
      if (f == kRefuse && running_solves == 0) {
        it = queue.erase(it);
        r->status = AMGEIG_ENOMEM;
        r->info.status = AMGEIG_ENOMEM;
        r->done = true;
        r->h->pending--;
        continue;
      }
      if (running_solves > 0 && f != kFits) {
        ++it;
        continue;
      }
      queue.erase(it);
      touch(r->h);
      gather_riders(r);
      return r;
    }
    return nullptr;
  }

  // Queued requests on r's hierarchy that can share its solve ride along.  The
  // shared solve takes the group's widest q and q_extra: up to the width of r's
  // workspace (or the one admitted for r), or wider when a workspace of the
  // wider width is admissible now (caller holds mu).
  void gather_riders(const std::shared_ptr<Request>& r) {
    r->riders.clear();
    if (!r->opt.batch) return;
    int width = r->q + r->opt.q_extra;
    {
      std::unique_lock<std::mutex> lk(r->h->mu, std::try_to_lock);
      if (lk.owns_lock() && r->h->ws) width = std::max(width, r->h->ws->qcap);
    }
    {
      // the widest group the queue offers, if its workspace fits
      int wq = 0, we = 0;
      for (const auto& x : queue)
        if (can_share(*r, *x)) {
          wq = std::max(wq, x->q);
          we = std::max(we, x->opt.q_extra);
        }
      const int wide = std::min(128, std::max(r->q, wq) + std::max(r->opt.q_extra, we));
      if (wide > width) {
        Request probe = *r;
        probe.riders.clear();
        probe.q = std::max(r->q, wq);
        probe.opt.q_extra = wide - probe.q;
        if (probe.opt.q_extra >= 0 && fits(&probe) == kFits) width = wide;
      }
    }
    int qm = r->q, qe = r->opt.q_extra;
    for (auto it = queue.begin(); it != queue.end();) {
      const std::shared_ptr<Request>& x = *it;
      if (can_share(*r, *x) && std::max(qm, x->q) + std::max(qe, x->opt.q_extra) <= width) {
        qm = std::max(qm, x->q);
        qe = std::max(qe, x->opt.q_extra);
        r->riders.push_back(x);
        it = queue.erase(it);
      } else {
        ++it;
      }
    }
  }

  static constexpr int kFits = 0, kWait = 1, kRefuse = 2;
  int fits(const Request* r);
  size_t resident_bytes() const;
  void touch(amgeig_hierarchy_t* h) {
    auto it = std::find(resident.begin(), resident.end(), h);
    if (it != resident.end()) resident.erase(it);
    resident.push_back(h);
  }
  void forget(amgeig_hierarchy_t* h) {
    auto it = std::find(resident.begin(), resident.end(), h);
    if (it != resident.end()) resident.erase(it);
  }

  void loop() {
    for (;;) {
      std::shared_ptr<Request> r;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return (r = pick()) != nullptr; });
        busy.push_back(r->h);
        ++running_solves;
      }
      run(r);
      {
        std::lock_guard<std::mutex> lk(mu);
        busy.erase(std::find(busy.begin(), busy.end(), r->h));
        reserved.erase(r->h);
        --running_solves;
        r->h->pending -= 1 + static_cast<int>(r->riders.size());
        r->riders.clear();
      }
      cv.notify_all();
    }
  }

  void run(const std::shared_ptr<Request>& r);
};

Service& service() {
  static Service* s = new Service();  // intentionally never destroyed (detached worker)
  return *s;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

void amgeig_default_options(amgeig_options* opt) {
  if (!opt) return;
  opt->max_corrections = 20;
  opt->v_cycles = 1;
  opt->pre_sweeps = 1;
  opt->post_sweeps = 1;
  opt->q_extra = 0;
  opt->precision = AMGEIG_FP64;
  opt->fixed_corrections = 0;
  opt->coarse_modes = 0;
  opt->smoother = AMGEIG_SMOOTHER_L1_JACOBI;
  opt->n1 = -1;
  opt->refine = 0;
  opt->graphs = 1;
  opt->autotune = 1;
  opt->batch = 1;
  opt->shift = 0.0;
  opt->krylov = 1;
}

const char* amgeig_strerror(int code) {
  switch (code) {
    case AMGEIG_OK: return "ok";
    case AMGEIG_EINVAL: return "invalid argument";
    case AMGEIG_ECORRUPT: return "corrupt hierarchy blob";
    case AMGEIG_ENOMEM: return "out of device memory";
    case AMGEIG_ENOTSPD: return "matrix not positive definite";
    case AMGEIG_ENOCONV: return "not converged within max_corrections";
    case AMGEIG_ENAN: return "NaN or Inf in the iterates";
    case AMGEIG_ECUDA: return "CUDA error";
    case AMGEIG_ENOTFOUND: return "unknown request id";
    default: return "unknown status";
  }
}

const char* amgeig_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

int amgeig::set_last_error(int code, const char* msg) {
  if (code == AMGEIG_OK)
    g_last_error.clear();
  else
    g_last_error = msg ? msg : "";
  return code;
}

extern "C" {

namespace {

// The load behind both entry points.  modes < 0: the coarse eigenbasis waits for the
// first solve; modes >= 0: its `modes` lowest pairs (0 or more than d_n: all) are
// computed during the load.
int load_hierarchy(const void* blob, size_t bytes, int device, int modes, amgeig_hierarchy* out) {
  g_last_error.clear();
  if (!blob || !out) return fail(AMGEIG_EINVAL, "NULL argument");
  *out = nullptr;
  // the blob's layout first (host only: a malformed blob is reported as such
  // whatever the device argument)
  std::vector<CsrView> levels, prolong;
  std::vector<uint64_t> aligned;
  const uint8_t* base = nullptr;
  int rc = parse_blob(blob, bytes, levels, prolong, aligned, &base);
  if (rc) return rc;
  // the coarsest level is checked on its own: its GPU work starts before the
  // rest of the blob is validated
  if (levels.back().rows > 4096) return fail(AMGEIG_EINVAL, "coarsest level larger than 4096");
  if (!csr_valid(levels.back())) return fail(AMGEIG_ECORRUPT, "invalid level CSR");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(AMGEIG_EINVAL, "no such CUDA device");
  CK(cudaSetDevice(device));
  auto h = std::make_unique<amgeig_hierarchy_t>();
  h->device = device;
  h->nlev = static_cast<int>(levels.size());
  const int n = h->nlev;
  for (auto& L : levels) h->sizes.push_back(L.rows);
  h->dn = static_cast<int>(h->sizes[n - 1]);
  {
    // small hierarchies get the higher stream priority: when solves on several
    // hierarchies share the GPU (the request service), the short kernels of a
    // small problem are scheduled ahead of a large problem's long ones, which
    // keeps small requests' latency near their own solve time
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));  // hi is the numerically smallest, the highest priority
    const int64_t N0 = h->sizes[0];
    const int prio = N0 <= 65536 ? hi : (N0 <= 262144 ? (lo + hi) / 2 : lo);
    CK(cudaStreamCreateWithPriority(&h->stream, cudaStreamNonBlocking, prio));
  }
  auto& m = h->mem;
  m.st = h->stream;
  // The coarsest level goes first, on two more streams: the GPU factors M_n
  // (and computes the asked-for lowest eigenpairs, Algorithm 3.2 step 1) on
  // one and inverts A_n on the other while the host validates the blob and
  // prepares the finer levels.  Both are drained before any return.
  struct SideStream {
    cudaStream_t s = nullptr;
    ~SideStream() {
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    }
  } side, side2;
  struct Event {
    cudaEvent_t e = nullptr;
    ~Event() {
      if (e) cudaEventDestroy(e);
    }
  } uploaded, copied;
  CK(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&side2.s, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&uploaded.e, cudaEventDisableTiming));
  // The rest of the blob goes to the device in one copy, first, and its arrays are
  // used in place; its checksum and every CSR structure are checked there, and the
  // results read back (after the coarsest level's work is queued) before any kernel
  // follows one of its column indices.
  uint8_t* dblob = nullptr;
  unsigned long long* dsum = nullptr;
  int* dbad = nullptr;
  CK(m.alloc(&dblob, bytes));
  CK(m.alloc(&dsum, 1));
  CK(m.alloc(&dbad, 2));
  CK(cudaMemcpyAsync(dblob, base, bytes, cudaMemcpyHostToDevice, h->stream));
  CK(cudaEventCreateWithFlags(&copied.e, cudaEventDisableTiming));
  CK(cudaEventRecord(copied.e, h->stream));
  auto dev = [&](const void* hp) { return dblob + (static_cast<const uint8_t*>(hp) - base); };
  CK(cudaMemsetAsync(dsum, 0, sizeof(unsigned long long), h->stream));
  CK(cudaMemsetAsync(dbad, 0, 2 * sizeof(int), h->stream));
  launch_blob_checksum(dblob, bytes - 8, dsum, h->stream);
  for (const CsrView& L : levels)
    launch_csr_check(reinterpret_cast<const int*>(dev(L.rp)), reinterpret_cast<const int*>(dev(L.ci)), L.rows,
                     L.cols, L.nnz, dbad, h->stream);
  for (const CsrView& P : prolong)
    launch_csr_check(reinterpret_cast<const int*>(dev(P.rp)), reinterpret_cast<const int*>(dev(P.ci)), P.rows,
                     P.cols, P.nnz, dbad + 1, h->stream);
  const int dn = h->dn;
  // the coarsest level's dense A_n and M_n, formed on the device from its arrays in the
  // blob (checked on the host above) as soon as the copy has landed
  CK(m.alloc(&h->An, static_cast<size_t>(dn) * dn));
  CK(m.alloc(&h->Mn, static_cast<size_t>(dn) * dn));
  CK(cudaStreamWaitEvent(side.s, copied.e, 0));
  {
    const CsrView& Lc = levels[n - 1];
    launch_csr_to_dense(dn, reinterpret_cast<const int*>(dev(Lc.rp)), reinterpret_cast<const int*>(dev(Lc.ci)),
                        reinterpret_cast<const double*>(dev(Lc.a)), reinterpret_cast<const double*>(dev(Lc.m)),
                        h->An, h->Mn, side.s);
  }
  CK(m.alloc(&h->Z, static_cast<size_t>(dn) * dn));
  CK(m.alloc(&h->theta, dn));
  CK(m.alloc(&h->Ainv, static_cast<size_t>(dn) * dn));
  CK(m.alloc(&h->Ainv32, static_cast<size_t>(dn) * dn));
  CK(m.alloc(&h->Zdf, static_cast<size_t>(dn) * dn));
  CK(m.alloc(&h->dstatus, 4));
  CK(cudaMemsetAsync(h->dstatus, 0, 2 * sizeof(int), side.s));  // [0]: M_n factor, [1]: A_n inverse
  CK(cudaEventRecord(uploaded.e, side.s));
  CK(cudaStreamWaitEvent(side2.s, uploaded.e, 0));
  {
    cudaError_t e;
    h->cpw = pencil_work_create(dn, 1, &e);
    if (!h->cpw) return fail(AMGEIG_ENOMEM, std::string("coarse workspace: ") + cudaGetErrorString(e));
  }
  launch_mass_factor(h->cpw, dn, h->Mn, h->dstatus, side.s);
  const int prefetch = modes < 0 ? 0 : (modes == 0 || modes > dn ? dn : modes);
  if (prefetch > 0) {
    launch_coarse_modes(h->cpw, dn, prefetch, h->An, h->Z, h->theta, side.s);
    launch_f64_to_df(h->Z, static_cast<long long>(dn) * dn, h->Zdf, side.s);
  }
  // the exact coarsest solve of the V-cycle (float64 Cholesky), its two dn x dn
  // scratch matrices stream-ordered on side2
  struct SideTemp {
    double* p = nullptr;
    cudaStream_t s = nullptr;
    ~SideTemp() {
      if (p) cudaFreeAsync(p, s);
    }
  } Lf, Li;
  Lf.s = Li.s = side2.s;
  CK(cudaMallocAsync(reinterpret_cast<void**>(&Lf.p), sizeof(double) * dn * dn, side2.s));
  CK(cudaMallocAsync(reinterpret_cast<void**>(&Li.p), sizeof(double) * dn * dn, side2.s));
  launch_coarse_inverse(dn, h->An, Lf.p, Li.p, h->Ainv, h->dstatus + 1, side2.s);
  launch_convert_f64_to_f32(h->Ainv, static_cast<long long>(dn) * dn, h->Ainv32, side2.s);
  CK(cudaGetLastError());
  // the checks' results (enqueued at the start) are read before any kernel follows a column index
  {
    unsigned long long sum = 0;
    int bad[2] = {0, 0};
    CK(cudaMemcpyAsync(&sum, dsum, sizeof(sum), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(bad, dbad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    uint64_t stored;
    std::memcpy(&stored, base + bytes - 8, 8);
    if (sum != stored) return fail(AMGEIG_ECORRUPT, "hierarchy blob checksum mismatch");
    if (bad[0]) return fail(AMGEIG_ECORRUPT, "invalid level CSR");
    if (bad[1]) return fail(AMGEIG_ECORRUPT, "invalid prolongation CSR");
  }
  h->A.resize(n);
  h->dinv64.assign(n, nullptr);
  h->dinv32.assign(n, nullptr);
  // the float32 and float-float copies of the values and the l1-Jacobi inverse
  // diagonals are made on the device
  int* zero_row = nullptr;
  CK(m.alloc(&zero_row, 1));
  CK(cudaMemsetAsync(zero_row, 0, sizeof(int), h->stream));
  for (int l = 0; l < n; ++l) {
    const CsrView& L = levels[l];
    DevCsr& D = h->A[l];
    D.rows = D.cols = static_cast<int>(L.rows);
    D.nnz = static_cast<int>(L.nnz);
    D.rp = reinterpret_cast<int*>(dev(L.rp));
    D.ci = reinterpret_cast<int*>(dev(L.ci));
    D.v64 = reinterpret_cast<double*>(dev(L.a));
    D.m64 = reinterpret_cast<double*>(dev(L.m));
    CK(m.alloc(&D.v32, static_cast<size_t>(L.nnz)));
    CK(m.alloc(&D.d2, static_cast<size_t>(L.nnz)));
    CK(m.alloc(&D.m2, static_cast<size_t>(L.nnz)));
    launch_convert_f64_to_f32(D.v64, L.nnz, D.v32, h->stream);
    launch_f64_to_df(D.v64, L.nnz, D.d2, h->stream);
    launch_f64_to_df(D.m64, L.nnz, D.m2, h->stream);
    CK(m.alloc(&h->dinv64[l], static_cast<size_t>(L.rows)));
    CK(m.alloc(&h->dinv32[l], static_cast<size_t>(L.rows)));
    launch_l1_inv_diag(D, h->dinv64[l], h->dinv32[l], zero_row, h->stream);
  }
  h->P.resize(n - 1);
  h->R.resize(n - 1);
  // P_l in place; R_l = P_l^T formed on the device (rows in ascending column order)
  int* tscratch = nullptr;
  long long* scan_tmp = nullptr;
  CK(m.alloc(&scan_tmp, 1024));
  if (n > 1) CK(m.alloc(&tscratch, static_cast<size_t>(h->sizes[1])));
  for (int l = 0; l + 1 < n; ++l) {
    const CsrView& P = prolong[l];
    DevCsr& Dp = h->P[l];
    DevCsr& Dr = h->R[l];
    Dp.rows = Dr.cols = static_cast<int>(P.rows);
    Dp.cols = Dr.rows = static_cast<int>(P.cols);
    Dp.nnz = Dr.nnz = static_cast<int>(P.nnz);
    Dp.rp = reinterpret_cast<int*>(dev(P.rp));
    Dp.ci = reinterpret_cast<int*>(dev(P.ci));
    Dp.v64 = reinterpret_cast<double*>(dev(P.a));
    CK(m.alloc(&Dr.rp, static_cast<size_t>(P.cols) + 1));
    CK(m.alloc(&Dr.ci, static_cast<size_t>(P.nnz)));
    CK(m.alloc(&Dr.v64, static_cast<size_t>(P.nnz)));
    launch_transpose_csr(P.rows, P.cols, P.nnz, Dp.rp, Dp.ci, Dp.v64, Dr.rp, Dr.ci, Dr.v64, tscratch, scan_tmp,
                         h->stream);
    for (DevCsr* D : {&Dp, &Dr}) {
      CK(m.alloc(&D->v32, static_cast<size_t>(P.nnz)));
      CK(m.alloc(&D->d2, static_cast<size_t>(P.nnz)));
      launch_convert_f64_to_f32(D->v64, P.nnz, D->v32, h->stream);
      launch_f64_to_df(D->v64, P.nnz, D->d2, h->stream);
    }
  }
  // composite prolongations I_n^k (coarsest -> level k) for the recombination:
  // PC[n-2] = P_{n-2}, PC[k] = P_k PC[k+1] -- sparse products with d_n columns,
  // built on the GPU level by level (count pass, row offsets, fill pass) in
  // float64 and kept as float-float pairs
  h->PC.resize(n > 1 ? n - 1 : 0);
  if (n > 1) {
    const int dn0 = h->dn;
    // PC[n-1] = I (the identity on the coarsest level) starts the recursion
    std::vector<int32_t> irp(static_cast<size_t>(dn0) + 1), ici(static_cast<size_t>(dn0));
    for (int i = 0; i <= dn0; ++i) irp[i] = i;
    for (int i = 0; i < dn0; ++i) ici[i] = i;
    std::vector<double> iv(static_cast<size_t>(dn0), 1.0);
    int *nrp = nullptr, *nci = nullptr;
    double* nv = nullptr;
    CK(m.upload(&nrp, irp));
    CK(m.upload(&nci, ici));
    // float64 values of the level below (freed once the next level is built) and of this level
    // (stream-ordered: a cudaFree would wait for the coarsest level's work on the side stream)
    struct DeviceTemp {
      double* p = nullptr;
      cudaStream_t s = nullptr;
      ~DeviceTemp() {
        if (p) cudaFreeAsync(p, s);
      }
    } prev, cur;
    prev.s = cur.s = h->stream;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&prev.p), sizeof(double) * iv.size(), h->stream));
    CK(cudaMemcpyAsync(prev.p, iv.data(), sizeof(double) * iv.size(), cudaMemcpyHostToDevice, h->stream));
    nv = prev.p;
    int* counts = nullptr;
    long long* dtotal = nullptr;
    CK(m.alloc(&counts, static_cast<size_t>(h->sizes[0])));
    CK(m.alloc(&dtotal, 1));
    for (int k = n - 2; k >= 0; --k) {
      const DevCsr& P = h->P[k];
      DevCsr& D = h->PC[k];
      D.rows = P.rows;
      D.cols = dn0;
      // row counts, their offsets on the device; only the total comes back (to size the arrays)
      launch_composite_rows(P, nrp, nci, nv, dn0, nullptr, counts, nullptr, nullptr, h->stream);
      CK(m.alloc(&D.rp, static_cast<size_t>(P.rows) + 1));
      launch_exclusive_scan(counts, P.rows, D.rp, scan_tmp, dtotal, h->stream);
      long long total = 0;
      CK(cudaMemcpyAsync(&total, dtotal, sizeof(total), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      if (total >= (1LL << 31)) return fail(AMGEIG_ENOMEM, "composite prolongation too large");
      D.nnz = static_cast<int>(total);
      CK(m.alloc(&D.ci, static_cast<size_t>(total)));
      CK(cudaMallocAsync(reinterpret_cast<void**>(&cur.p), sizeof(double) * std::max<int64_t>(total, 1), h->stream));
      launch_composite_rows(P, nrp, nci, nv, dn0, D.rp, nullptr, D.ci, cur.p, h->stream);
      CK(m.alloc(&D.d2, static_cast<size_t>(total)));
      launch_f64_to_df(cur.p, total, D.d2, h->stream);
      CK(cudaFreeAsync(prev.p, h->stream));
      prev.p = cur.p;
      cur.p = nullptr;
      nrp = D.rp;
      nci = D.ci;
      nv = prev.p;
    }
  }
  int stt[2] = {0, 0}, zr = 0;
  cudaError_t e0 = cudaStreamSynchronize(side2.s);
  cudaError_t e1 = cudaStreamSynchronize(side.s);
  cudaError_t e2 = cudaMemcpyAsync(stt, h->dstatus, 2 * sizeof(int), cudaMemcpyDeviceToHost, side.s);
  cudaError_t e3 = cudaMemcpyAsync(&zr, zero_row, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  cudaError_t e4 = cudaStreamSynchronize(h->stream);
  CK(e0);
  CK(e1);
  CK(e2);
  CK(e3);
  CK(e4);
  CK(cudaGetLastError());
  if (zr) return fail(AMGEIG_ECORRUPT, "zero row in A");
  if (stt[0] || stt[1]) return fail(AMGEIG_ENOTSPD, "coarsest M_n or A_n is not positive definite");
  h->modes_ready = prefetch;
  *out = h.release();
  return AMGEIG_OK;
}

}  // namespace

int amgeig_load_hierarchy(const void* blob, size_t bytes, int device, amgeig_hierarchy* out) {
  return load_hierarchy(blob, bytes, device, -1, out);
}

int amgeig_load_hierarchy_modes(const void* blob, size_t bytes, int device, int modes, amgeig_hierarchy* out) {
  if (modes < 0) {
    g_last_error.clear();
    return fail(AMGEIG_EINVAL, "modes must be >= 0");
  }
  return load_hierarchy(blob, bytes, device, modes, out);
}

int amgeig_free_hierarchy(amgeig_hierarchy h) {
  if (!h) return AMGEIG_OK;
  if (h->pending.load() != 0) return fail(AMGEIG_EINVAL, "hierarchy has pending requests");
  {
    Service& s = service();
    std::lock_guard<std::mutex> lk(s.mu);
    s.forget(h);
  }
  cudaSetDevice(h->device);
  delete h;
  return AMGEIG_OK;
}

int amgeig_hierarchy_info(amgeig_hierarchy h, int* n_levels, int64_t* sizes, int max_sizes) {
  if (!h || !n_levels) return fail(AMGEIG_EINVAL, "NULL argument");
  *n_levels = h->nlev;
  if (sizes)
    for (int l = 0; l < std::min(h->nlev, max_sizes); ++l) sizes[l] = h->sizes[l];
  return AMGEIG_OK;
}

int amgeig_solve(amgeig_hierarchy h, int q, double tol, const amgeig_options* opt, double* eigvals, double* eigvecs,
                 int eigvecs_on_device, amgeig_info* info, void* stream) {
  g_last_error.clear();
  if (!h) return fail(AMGEIG_EINVAL, "NULL hierarchy");
  amgeig_options o;
  amgeig_default_options(&o);
  if (opt) o = *opt;
  std::lock_guard<std::mutex> lk(h->mu);
  CK(cudaSetDevice(h->device));
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
  std::vector<double> rr;
  if (info) std::memset(info, 0, sizeof(*info));
  const int rc = solve_impl(h, q, tol, o, info, rr, st);
  if (rc != AMGEIG_OK && rc != AMGEIG_ENOCONV) {
    if (info) info->status = rc;
    return rc;
  }
  const int rc2 = write_outputs(h, q, eigvals, eigvecs, eigvecs_on_device, st);
  if (rc2) return rc2;
  return rc;
}

int amgeig_sym_eigh(int device, int n, int nwant, const double* H, double* evals, double* evecs) {
  g_last_error.clear();
  if (!H || !evals || !evecs || n < 1 || n > 2048 || nwant < 1 || nwant > n)
    return fail(AMGEIG_EINVAL, "invalid argument");
  CK(cudaSetDevice(device));
  cudaError_t e;
  PencilWork* pw = pencil_work_create(n, 1, &e);
  if (!pw) return fail(AMGEIG_ENOMEM, std::string("eigensolver workspace: ") + cudaGetErrorString(e));
  DeviceBuffers m;
  double *dH, *dv, *dV;
  cudaStream_t st;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaError_t e0 = m.alloc(&dH, static_cast<size_t>(n) * n);
  if (e0 == cudaSuccess) e0 = m.alloc(&dv, nwant);
  if (e0 == cudaSuccess) e0 = m.alloc(&dV, static_cast<size_t>(n) * nwant);
  if (e0 == cudaSuccess) e0 = cudaMemcpyAsync(dH, H, sizeof(double) * n * n, cudaMemcpyHostToDevice, st);
  if (e0 == cudaSuccess) {
    launch_syev_df(pw, n, nwant, dH, dv, dV, st);
    e0 = cudaGetLastError();
  }
  if (e0 == cudaSuccess) e0 = cudaMemcpyAsync(evals, dv, sizeof(double) * nwant, cudaMemcpyDeviceToHost, st);
  if (e0 == cudaSuccess)
    e0 = cudaMemcpyAsync(evecs, dV, sizeof(double) * n * nwant, cudaMemcpyDeviceToHost, st);
  cudaError_t e1 = cudaStreamSynchronize(st);
  pencil_work_destroy(pw);
  cudaStreamDestroy(st);
  CK(e0);
  CK(e1);
  return AMGEIG_OK;
}

int amgeig_apply_defect(amgeig_hierarchy h, int level, int width, const amgeig_options* opt, const double* U,
                        const double* lam, double* R, double* relres) {
  g_last_error.clear();
  if (!h || !U || !lam || !R || level < 0 || level >= h->nlev || width < 1 || width > 128)
    return fail(AMGEIG_EINVAL, "invalid argument");
  amgeig_options o;
  amgeig_default_options(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->mu);
  CK(cudaSetDevice(h->device));
  cudaStream_t st = h->stream;
  rc = ensure_workspace(h, width, o.precision, 1);
  if (rc) return rc;
  SolveWork* w = h->ws.get();
  const int Nl = static_cast<int>(h->sizes[level]);
  const long long cnt = static_cast<long long>(Nl) * width;
  CK(cudaMemcpyAsync(w->V, U, sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(w->lam, lam, sizeof(double) * width, cudaMemcpyHostToDevice, st));
  int nb = 0;
  if (o.precision == AMGEIG_FP64) {
    launch_defect_f64(h->A[level], w->V, width, w->lam, w->B64[level], w->partials, &nb, st);
    CK(cudaMemcpyAsync(R, w->B64[level], sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
  } else {
    // the iterate in float-float, the defect rounded to float32 (the V-cycle's right-hand side)
    launch_f64_to_df(w->V, cnt, as_df(w->U), st);
    launch_defect_df(h->A[level], as_df(w->U), width, w->lam, w->B32[level], w->ld32, w->partials, &nb, st);
    launch_f32_to_f64_unpad(w->B32[level], Nl, width, w->ld32, w->Ualt, st);
    CK(cudaMemcpyAsync(R, w->Ualt, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
  }
  launch_sum_partials(w->partials, nb, 2 * width, w->sums, st);
  CK(cudaMemsetAsync(w->flags, 0, sizeof(int), st));
  launch_relres(w->sums, w->lam, width, w->relres, w->flags, st);
  CK(cudaGetLastError());
  if (relres) CK(cudaMemcpyAsync(relres, w->relres, sizeof(double) * width, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return AMGEIG_OK;
}

int amgeig_apply_vcycle(amgeig_hierarchy h, int level, int width, const amgeig_options* opt, const double* b,
                        double* x) {
  g_last_error.clear();
  if (!h || !b || !x || level < 0 || level >= h->nlev || width < 1 || width > 128)
    return fail(AMGEIG_EINVAL, "invalid argument");
  amgeig_options o;
  amgeig_default_options(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->mu);
  CK(cudaSetDevice(h->device));
  cudaStream_t st = h->stream;
  rc = ensure_workspace(h, width, o.precision, 1);
  if (rc) return rc;
  SolveWork* w = h->ws.get();
  w->smoother = o.smoother;
  if (o.smoother == AMGEIG_SMOOTHER_GAUSS_SEIDEL) {
    rc = ensure_gs(h, st);
    if (rc) return rc;
  }
  w->bf16 = o.precision == AMGEIG_MIXED_BF16;
  if (w->bf16) {
    rc = ensure_bf16(h, st);
    if (rc) return rc;
  }
  w->shifted = o.shift != 0.0;
  if (w->shifted) {
    rc = ensure_shift(h, o.shift, st);
    if (rc) return rc;
  }
  const long long cnt = h->sizes[level] * static_cast<long long>(width);
  if (level == h->nlev - 1) {
    // the coarsest level: the exact solve
    CK(cudaMemcpyAsync(w->V, b, sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
    launch_gemm_f64(h->dn, width, h->dn, 1.0, w->shifted ? h->sh.Ainv : h->Ainv, h->dn, false, w->V, width, false,
                    0.0, w->U, width, st);
    CK(cudaMemcpyAsync(x, w->U, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return AMGEIG_OK;
  }
  CK(cudaMemcpyAsync(w->V, b, sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
  if (o.precision == AMGEIG_FP64) {
    CK(cudaMemcpyAsync(w->B64[level], w->V, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st));
    vcycle<double>(h, w, level, o.pre_sweeps, o.post_sweeps, false, nullptr, nullptr, st);
    CK(cudaMemcpyAsync(w->U, w->X64[level], sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st));
  } else {
    launch_f64_to_f32_pad(w->V, static_cast<int>(h->sizes[level]), width, w->ld32, w->B32[level], st);
    vcycle<float>(h, w, level, o.pre_sweeps, o.post_sweeps, false, nullptr, nullptr, st);
    launch_f32_to_f64_unpad(w->X32[level], static_cast<int>(h->sizes[level]), width, w->ld32, w->U, st);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(x, w->U, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return AMGEIG_OK;
}

int amgeig_submit(amgeig_hierarchy h, int q, double tol, const amgeig_options* opt, uint64_t* request_id) {
  if (!h || !request_id) return fail(AMGEIG_EINVAL, "NULL argument");
  amgeig_options o;
  amgeig_default_options(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  if (q < 1 || q + o.q_extra > h->sizes[0] || q + o.q_extra > 128) return fail(AMGEIG_EINVAL, "q out of range");
  auto r = std::make_shared<Request>();
  r->h = h;
  r->q = q;
  r->tol = tol;
  r->opt = o;
  Service& s = service();
  {
    std::lock_guard<std::mutex> lk(s.mu);
    r->id = s.next_id++;
    s.table[r->id] = r;
    s.queue.push_back(r);
    h->pending++;
    s.start();
  }
  s.cv.notify_one();
  *request_id = r->id;
  return AMGEIG_OK;
}

int amgeig_tuning_report(amgeig_hierarchy h, char* buf, size_t len) {
  if (!h || !buf || len == 0) return fail(AMGEIG_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(h->mu);
  const std::string txt = "[" + h->tune_log + "]";
  std::snprintf(buf, len, "%s", txt.c_str());
  if (txt.size() + 1 > len) return fail(AMGEIG_EINVAL, "buffer too small for the tuning report");
  return AMGEIG_OK;
}

int amgeig_service_set_memory_limit(uint64_t bytes) {
  Service& s = service();
  {
    std::lock_guard<std::mutex> lk(s.mu);
    s.mem_limit = static_cast<size_t>(bytes);
  }
  s.cv.notify_all();
  return AMGEIG_OK;
}

int amgeig_service_memory(uint64_t* resident_bytes, uint64_t* evictions) {
  if (!resident_bytes && !evictions) return fail(AMGEIG_EINVAL, "NULL arguments");
  Service& s = service();
  std::lock_guard<std::mutex> lk(s.mu);
  if (resident_bytes) *resident_bytes = s.resident_bytes();
  if (evictions) *evictions = s.evictions;
  return AMGEIG_OK;
}

int amgeig_poll(uint64_t request_id, int* done, double* eigvals, double* eigvecs, amgeig_info* info) {
  if (!done) return fail(AMGEIG_EINVAL, "NULL argument");
  Service& s = service();
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.table.find(request_id);
    if (it == s.table.end()) return fail(AMGEIG_ENOTFOUND, "unknown request id");
    r = it->second;
    if (!r->done) {
      *done = 0;
      return AMGEIG_OK;
    }
    s.table.erase(it);
  }
  *done = 1;
  if (eigvals && !r->vals.empty()) std::memcpy(eigvals, r->vals.data(), sizeof(double) * r->vals.size());
  if (eigvecs && !r->vecs.empty()) std::memcpy(eigvecs, r->vecs.data(), sizeof(double) * r->vecs.size());
  if (info) *info = r->info;
  return r->status;
}

}  // extern "C"

namespace {

// device bytes of the workspace a request needs (the allocations make_workspace
// would make for it, counted without allocating)
size_t workspace_bytes(amgeig_hierarchy_t* h, const Request* r) {
  const int qt = r->q + r->opt.q_extra;
  const int prec = r->opt.precision == AMGEIG_FP64 ? AMGEIG_FP64 : AMGEIG_MIXED_FP32;
  std::unique_ptr<SolveWork> w;
  if (make_workspace(h, qt, prec, std::max(1, r->opt.v_cycles), w, true, r->opt.krylov == 2 ? 2 * qt : 0) !=
          AMGEIG_OK ||
      !w)
    return 0;
  return w->mem.held + w->pw_bytes;
}

size_t ws_held(const amgeig_hierarchy_t* h) { return h->ws ? h->ws->mem.held + h->ws->pw_bytes : 0; }

// Bytes held by the workspaces of the hierarchies the service has used, or
// about to be held by the ones being made for admitted requests (caller holds mu).
size_t Service::resident_bytes() const {
  size_t b = 0;
  for (amgeig_hierarchy_t* x : resident) {
    auto it = reserved.find(x);
    b += it != reserved.end() ? it->second : ws_held(x);
  }
  return b;
}

// Admission (caller holds mu): kFits when the request's workspace is resident or
// can be made (under the memory limit, after releasing idle workspaces of other
// hierarchies, least recently used first, and within free device memory); kWait
// when it may fit once running requests end; kRefuse when it cannot fit under
// the limit at all.
int Service::fits(const Request* r) {
  amgeig_hierarchy_t* h = r->h;
  const int qt = r->q + r->opt.q_extra;
  size_t own = 0;
  {
    // a direct solve on this hierarchy from another thread: not now
    std::unique_lock<std::mutex> lk(h->mu, std::try_to_lock);
    if (!lk.owns_lock()) return kWait;
    const int wp = r->opt.precision == AMGEIG_FP64 ? AMGEIG_FP64 : AMGEIG_MIXED_FP32;
    if (h->ws && h->ws->qcap >= qt && h->ws->precision == wp) return kFits;
    own = ws_held(h);
  }
  const size_t need = workspace_bytes(h, r);
  if (mem_limit > 0) {
    if (need > mem_limit) return kRefuse;
    // the request's own (too small) workspace is replaced, so it does not count
    size_t held = resident_bytes() - std::min(resident_bytes(), own);
    for (size_t i = 0; i < resident.size() && held + need > mem_limit; ++i) {
      amgeig_hierarchy_t* x = resident[i];
      if (x == h || is_busy(x) || reserved.count(x)) continue;
      std::unique_lock<std::mutex> lk(x->mu, std::try_to_lock);
      if (!lk.owns_lock() || !x->ws) continue;
      held -= std::min(held, ws_held(x));
      cudaSetDevice(x->device);
      x->ws.reset();  // its last solve synchronised its stream: nothing in flight
      ++evictions;
    }
    if (held + need > mem_limit) return kWait;
  }
  size_t fr = 0, tot = 0;
  cudaSetDevice(h->device);
  bool ok = cudaMemGetInfo(&fr, &tot) != cudaSuccess || need <= fr;
  if (!ok && dev_cache_trim() > 0) ok = cudaMemGetInfo(&fr, &tot) != cudaSuccess || need <= fr;
  if (!ok) return kWait;
  reserved[h] = need;  // admitted (pick takes it now): counted until its workspace exists
  return kFits;
}

void Service::run(const std::shared_ptr<Request>& r) {
  amgeig_hierarchy_t* h = r->h;
  if (r->riders.empty()) {
    r->vals.assign(r->q, 0.0);
    r->vecs.assign(static_cast<size_t>(h->sizes[0]) * r->q, 0.0);
    int status = amgeig_solve(h, r->q, r->tol, &r->opt, r->vals.data(), r->vecs.data(), 0, &r->info, nullptr);
    if (status != AMGEIG_OK && status != AMGEIG_ENOCONV) {
      r->vals.clear();
      r->vecs.clear();
    }
    r->info.status = status;
    std::lock_guard<std::mutex> lk(mu);
    r->status = status;
    r->done = true;
    return;
  }
  // One solve for the group: the widest wanted count and buffer, the tightest
  // tolerance, the largest correction limit.  Every member wants the lowest
  // eigenpairs of the same pencil, so each takes the leading columns it asked
  // for, with its own residual test over them.
  std::vector<Request*> grp = {r.get()};
  for (auto& x : r->riders) grp.push_back(x.get());
  int qm = 0, qe = 0, mc = 0;
  double tol = r->tol;
  for (Request* x : grp) {
    qm = std::max(qm, x->q);
    qe = std::max(qe, x->opt.q_extra);
    mc = std::max(mc, x->opt.max_corrections);
    tol = std::min(tol, x->tol);
  }
  amgeig_options o = r->opt;
  o.q_extra = qe;
  o.max_corrections = mc;
  const int64_t N0 = h->sizes[0];
  std::vector<double> vals(qm), vecs(static_cast<size_t>(N0) * qm), rr;
  amgeig_info info{};
  int status;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    g_last_error.clear();
    cudaSetDevice(h->device);
    status = solve_impl(h, qm, tol, o, &info, rr, h->stream);
    if (status == AMGEIG_OK || status == AMGEIG_ENOCONV) {
      const int rc2 = write_outputs(h, qm, vals.data(), vecs.data(), 0, h->stream);
      if (rc2) status = rc2;
    }
  }
  for (Request* x : grp) {
    x->info = info;
    if (status == AMGEIG_OK || status == AMGEIG_ENOCONV) {
      x->vals.assign(vals.begin(), vals.begin() + x->q);
      x->vecs.resize(static_cast<size_t>(N0) * x->q);
      for (int64_t i = 0; i < N0; ++i)
        std::memcpy(x->vecs.data() + i * x->q, vecs.data() + i * qm, sizeof(double) * x->q);
      double mx = 0.0;
      for (int j = 0; j < x->q && j < static_cast<int>(rr.size()); ++j) mx = std::max(mx, rr[j]);
      x->info.max_relres = mx;
      x->info.converged = mx <= x->tol ? 1 : 0;
      x->info.status = x->info.converged ? AMGEIG_OK : AMGEIG_ENOCONV;
    } else {
      x->vals.clear();
      x->vecs.clear();
      x->info.status = status;
    }
  }
  std::lock_guard<std::mutex> lk(mu);
  for (Request* x : grp) {
    x->status = x->info.status;
    x->done = true;
  }
}

}  // namespace
