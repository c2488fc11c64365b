// AMG setup of Sec. 2 with its bulk on the GPU: the hierarchy the solve phase
// reads, built from the finest pencil (A, M).
//
// Per level k (Sec. 2.1-2.3):
//   C/F splitting  on the host (the classical Ruge-Stueben passes are a
//                  sequential greedy order; the setup library's own splitting,
//                  strength threshold theta on the negative couplings);
//   interpolation  direct interpolation (Eqs. Interpolation_Def and
//                  Interpolation_Dir) on the GPU, one thread per row: C rows
//                  inject, an F row i takes w_ij = -alpha_i a_ij / (a_ii +
//                  sum of its positive couplings) over its strong negative C
//                  couplings, alpha_i = (sum of its negative couplings) / (the
//                  same over the strong C ones); each sum in row order;
//   coarse ops     A_{k+1} = P^T A_k P and M_{k+1} = P^T M_k P (Eq.
//                  Coarse_Matrices) as two sparse products on the GPU on the
//                  symbolic pattern (no dropping; A and M share it): A P with
//                  both value arrays, then R (A P) with R = P^T.
// The sparse products run one warp per output row: the row's candidate
// (column, value) terms are gathered into shared memory, sorted by column
// (bitonic sort on column and position, so equal columns keep their order) and
// each column's terms summed in that order.
//
// The result is written as the hierarchy blob both the solve path and the
// CPU checker read (layout: the writer in the package's inputs/hierarchy.py).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "amgeig.h"
#include "common.cuh"
#include "kernels.cuh"
#include "prof.cuh"

extern "C" int amgsetup_cf_split(int64_t n, const int32_t* rp, const int32_t* ci, const double* a, double theta,
                                 int8_t* state);

namespace amgeig {
namespace {

constexpr int8_t kC = 1;

// ---------------------------------------------------------------- interpolation

__device__ __forceinline__ double max_neg(const int* rp, const int* ci, const double* a, int i) {
  double mx = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] != i && a[p] < 0.0) mx = fmax(mx, -a[p]);
  return mx;
}

// nonzeros of row i of P: 1 for a C row, the strong negative C couplings otherwise
__global__ void k_interp_count(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                               const double* __restrict__ a, const int8_t* __restrict__ state, double theta,
                               int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (state[i] == kC) {
    cnt[i] = 1;
    return;
  }
  const double thr = theta * max_neg(rp, ci, a, i);
  int c = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    if (j != i && a[p] < 0.0 && -a[p] >= thr && state[j] == kC) ++c;
  }
  cnt[i] = c;
}

__global__ void k_interp_fill(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ a, const int8_t* __restrict__ state,
                              const int* __restrict__ cidx, double theta, const int* __restrict__ prp,
                              int* __restrict__ pci, double* __restrict__ pv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = prp[i];
  if (state[i] == kC) {
    pci[o] = cidx[i];
    pv[o] = 1.0;
    return;
  }
  const double thr = theta * max_neg(rp, ci, a, i);
  double diag = 0.0, neg_all = 0.0, pos_all = 0.0, neg_p = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    const double v = a[p];
    if (j == i) {
      diag = __dadd_rn(diag, v);
      continue;
    }
    if (v < 0.0)
      neg_all = __dadd_rn(neg_all, v);
    else
      pos_all = __dadd_rn(pos_all, v);
    if (v < 0.0 && -v >= thr && state[j] == kC) neg_p = __dadd_rn(neg_p, v);
  }
  const double alpha = __ddiv_rn(neg_all, neg_p);
  const double dd = __dadd_rn(diag, pos_all);  // positive couplings lumped onto the diagonal
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    const double v = a[p];
    if (j != i && v < 0.0 && -v >= thr && state[j] == kC) {
      pci[o] = cidx[j];
      pv[o] = __ddiv_rn(__dmul_rn(-alpha, v), dd);
      ++o;
    }
  }
}

// ---------------------------------------------------------------- sparse products

// candidate terms of row i of X Y: sum over X's row of Y's row lengths
__global__ void k_cand_count(int n, const int* __restrict__ xrp, const int* __restrict__ xci,
                             const int* __restrict__ yrp, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0;
  for (int p = xrp[i]; p < xrp[i + 1]; ++p) {
    const int k = xci[p];
    c += yrp[k + 1] - yrp[k];
  }
  cnt[i] = c;
}

// One warp per output row of C = X Y (two value arrays out: ca = xa . ya and
// cm = xm . ym, a missing xm / ym standing for xa / ya).  cap: power of two >=
// the row's candidate count, the shared staging of each warp.  Pass 1 (crp
// null) counts the row's distinct columns into cnt; pass 2 writes them from
// crp[row] on, sorted, each column's terms summed in candidate order.
__global__ void k_spgemm_rows(int n, const int* __restrict__ xrp, const int* __restrict__ xci,
                              const double* __restrict__ xa, const double* __restrict__ xm,
                              const int* __restrict__ yrp, const int* __restrict__ yci,
                              const double* __restrict__ ya, const double* __restrict__ ym, int cap,
                              int* __restrict__ cnt, const int* __restrict__ crp, int* __restrict__ cci,
                              double* __restrict__ ca, double* __restrict__ cm) {
  extern __shared__ __align__(16) unsigned char sraw[];
  const int warps = blockDim.x / 32;
  const int wid = threadIdx.x / 32, lane = threadIdx.x % 32;
  long long* key = reinterpret_cast<long long*>(sraw) + static_cast<long long>(wid) * cap;
  double* va = reinterpret_cast<double*>(reinterpret_cast<long long*>(sraw) + static_cast<long long>(warps) * cap) +
               static_cast<long long>(wid) * 2 * cap;
  double* vm = va + cap;
  const int row = blockIdx.x * warps + wid;
  if (row >= n) return;  // whole warps leave together
  const bool fill = crp != nullptr;
  {
    // a row beyond the staging capacity is the long-row kernel's (whole warp leaves)
    int total = 0;
    for (int p = xrp[row]; p < xrp[row + 1]; ++p) total += yrp[xci[p] + 1] - yrp[xci[p]];
    if (total > cap) return;
  }
  // gather: the (p, r) loop in order; position m is the candidate's order
  int m0 = 0;
  for (int p = xrp[row]; p < xrp[row + 1]; ++p) {
    const int k = xci[p];
    const double sa = xa[p], sm = xm ? xm[p] : xa[p];
    const int r0 = yrp[k], len = yrp[k + 1] - r0;
    for (int t = lane; t < len; t += 32) {
      const int r = r0 + t, m = m0 + t;
      key[m] = (static_cast<long long>(yci[r]) << 20) | m;
      if (fill) {
        va[m] = sa * ya[r];
        vm[m] = sm * (ym ? ym[r] : ya[r]);
      }
    }
    m0 += len;
  }
  for (int m = m0 + lane; m < cap; m += 32) key[m] = 0x7fffffffffffffffLL;
  __syncwarp();
  // bitonic sort of the keys (column, position)
  for (int k = 2; k <= cap; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < cap; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const long long ki = key[i], kl = key[l];
          const bool up = (i & k) == 0;
          if ((ki > kl) == up) {
            key[i] = kl;
            key[l] = ki;
          }
        }
      }
      __syncwarp();
    }
  }
  // runs of equal columns: each lane takes a contiguous chunk, counts the runs
  // starting in it, and (pass 2) sums each run in order and writes it
  const int chunk = cap / 32;
  const int i0 = lane * chunk, i1 = min(m0, i0 + chunk);
  int starts = 0;
  for (int i = i0; i < i1; ++i)
    if (i == 0 || (key[i] >> 20) != (key[i - 1] >> 20)) ++starts;
  int off = starts;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, off, o);
    if (lane >= o) off += v;
  }
  const int total = __shfl_sync(0xffffffffu, off, 31);
  if (!fill) {
    if (lane == 0) cnt[row] = total;
    return;
  }
  int w = crp[row] + off - starts;
  for (int i = i0; i < i1; ++i) {
    const long long col = key[i] >> 20;
    if (i != 0 && col == (key[i - 1] >> 20)) continue;
    double sa = 0.0, sm = 0.0;
    for (int t = i; t < m0 && (key[t] >> 20) == col; ++t) {
      const int m = static_cast<int>(key[t] & 0xfffff);
      sa = __dadd_rn(sa, va[m]);
      sm = __dadd_rn(sm, vm[m]);
    }
    cci[w] = static_cast<int>(col);
    ca[w] = sa;
    cm[w] = sm;
    ++w;
  }
}

// Rows with more candidate terms than the shared staging holds (dense rows of
// the coarse 3D Galerkin levels): one thread per such row accumulates its terms
// in candidate order into a dense row of scratch (marker, two sums per column of
// C), then walks the columns in order.  Pass 1 (crp null) counts, pass 2
// writes.  Same sums in the same order as the sorted path.
__global__ void k_spgemm_long(int nlong, const int* __restrict__ rows, int ncols, const int* __restrict__ xrp,
                              const int* __restrict__ xci, const double* __restrict__ xa,
                              const double* __restrict__ xm, const int* __restrict__ yrp,
                              const int* __restrict__ yci, const double* __restrict__ ya,
                              const double* __restrict__ ym, int* __restrict__ mark, double* __restrict__ sa,
                              double* __restrict__ sm, int* __restrict__ cnt, const int* __restrict__ crp,
                              int* __restrict__ cci, double* __restrict__ ca, double* __restrict__ cm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlong) return;
  const int row = rows[t];
  int* mk = mark + static_cast<long long>(t) * ncols;
  double* a = sa + static_cast<long long>(t) * ncols;
  double* m = sm + static_cast<long long>(t) * ncols;
  for (int j = 0; j < ncols; ++j) mk[j] = 0;
  for (int p = xrp[row]; p < xrp[row + 1]; ++p) {
    const int k = xci[p];
    const double s1 = xa[p], s2 = xm ? xm[p] : xa[p];
    for (int r = yrp[k]; r < yrp[k + 1]; ++r) {
      const int j = yci[r];
      if (!mk[j]) {
        mk[j] = 1;
        a[j] = 0.0;
        m[j] = 0.0;
      }
      a[j] = __dadd_rn(a[j], s1 * ya[r]);
      m[j] = __dadd_rn(m[j], s2 * (ym ? ym[r] : ya[r]));
    }
  }
  if (!crp) {
    int c = 0;
    for (int j = 0; j < ncols; ++j) c += mk[j];
    cnt[row] = c;
    return;
  }
  int w = crp[row];
  for (int j = 0; j < ncols; ++j)
    if (mk[j]) {
      cci[w] = j;
      ca[w] = a[j];
      cm[w] = m[j];
      ++w;
    }
}

// ---------------------------------------------------------------- host side

struct Csr {
  int64_t rows = 0, cols = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> a, m;
};

struct DevMat {
  int* rp = nullptr;
  int* ci = nullptr;
  double* a = nullptr;
  double* m = nullptr;
};

struct Pool {
  std::vector<void*> ptrs;
  ~Pool() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t alloc(T** out, size_t count) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * (count > 0 ? count : 1));
    if (e == cudaSuccess) ptrs.push_back(p);
    *out = static_cast<T*>(p);
    return e;
  }
  template <typename T>
  cudaError_t upload(T** out, const std::vector<T>& v, cudaStream_t st) {
    cudaError_t e = alloc(out, v.size());
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpyAsync(*out, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
    return e;
  }
};

#define SCK(expr)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (expr);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return set_last_error(e_ == cudaErrorMemoryAllocation ? AMGEIG_ENOMEM : AMGEIG_ECUDA,       \
                            (std::string(#expr) + ": " + cudaGetErrorString(e_)).c_str());        \
  } while (0)

int scan_counts(const std::vector<int32_t>& cnt, std::vector<int32_t>& rp) {
  rp.assign(cnt.size() + 1, 0);
  int64_t t = 0;
  for (size_t i = 0; i < cnt.size(); ++i) {
    t += cnt[i];
    if (t >= (int64_t(1) << 31)) return set_last_error(AMGEIG_ENOMEM, "setup: a matrix beyond 2^31 nonzeros");
    rp[i + 1] = static_cast<int32_t>(t);
  }
  return AMGEIG_OK;
}

// C = X Y on the device (see k_spgemm_rows; rows beyond 8192 candidate terms:
// k_spgemm_long); C's arrays in pool, its row offsets also on the host
// (crp_host).  ncols: the columns of Y.
int spgemm(Pool& pool, int nrows, int ncols, const DevMat& X, const DevMat& Y, DevMat& C,
           std::vector<int32_t>& crp_host, int* d_cnt, cudaStream_t st) {
  if (nrows == 0) return set_last_error(AMGEIG_EINVAL, "setup: empty product");
  {
    ProfScope ps(st, P_OTHER, 0.0, 0.0);
    k_cand_count<<<ceil_div(nrows, 256), 256, 0, st>>>(nrows, X.rp, X.ci, Y.rp, d_cnt);
  }
  std::vector<int32_t> cnt(static_cast<size_t>(nrows));
  SCK(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * nrows, cudaMemcpyDeviceToHost, st));
  SCK(cudaStreamSynchronize(st));
  constexpr int kCap = 8192;
  int mx = 1;
  std::vector<int32_t> longrows;
  for (int i = 0; i < nrows; ++i) {
    if (cnt[i] > kCap)
      longrows.push_back(i);
    else
      mx = std::max(mx, static_cast<int>(cnt[i]));
  }
  int cap = 32;
  while (cap < mx) cap <<= 1;
  int* d_long = nullptr;
  int* d_mark = nullptr;
  double *d_sa = nullptr, *d_sm = nullptr;
  const int nlong = static_cast<int>(longrows.size());
  if (nlong > 0) {
    // dense scratch rows for the long rows (freed with the setup's other arrays)
    const size_t cells = static_cast<size_t>(nlong) * static_cast<size_t>(ncols);
    SCK(pool.upload(&d_long, longrows, st));
    SCK(pool.alloc(&d_mark, cells));
    SCK(pool.alloc(&d_sa, cells));
    SCK(pool.alloc(&d_sm, cells));
  }
  const size_t per_warp = static_cast<size_t>(cap) * (8 + 16);
  const int warps = static_cast<int>(std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_warp)));
  const size_t sm = per_warp * warps;
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_spgemm_rows), sm);
  const int blocks = ceil_div(nrows, warps);
  {
    ProfScope ps(st, P_OTHER, 0.0, 0.0);
    k_spgemm_rows<<<blocks, 32 * warps, sm, st>>>(nrows, X.rp, X.ci, X.a, X.m, Y.rp, Y.ci, Y.a, Y.m, cap, d_cnt,
                                                  nullptr, nullptr, nullptr, nullptr);
  }
  if (nlong > 0) {
    ProfScope ps(st, P_OTHER, 0.0, 0.0);
    k_spgemm_long<<<ceil_div(nlong, 64), 64, 0, st>>>(nlong, d_long, ncols, X.rp, X.ci, X.a, X.m, Y.rp, Y.ci, Y.a,
                                                     Y.m, d_mark, d_sa, d_sm, d_cnt, nullptr, nullptr, nullptr,
                                                     nullptr);
  }
  SCK(cudaGetLastError());
  SCK(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * nrows, cudaMemcpyDeviceToHost, st));
  SCK(cudaStreamSynchronize(st));
  int rc = scan_counts(cnt, crp_host);
  if (rc) return rc;
  const size_t nnz = static_cast<size_t>(crp_host.back());
  SCK(pool.upload(&C.rp, crp_host, st));
  SCK(pool.alloc(&C.ci, nnz));
  SCK(pool.alloc(&C.a, nnz));
  SCK(pool.alloc(&C.m, nnz));
  {
    ProfScope ps(st, P_OTHER, 0.0, 0.0);
    k_spgemm_rows<<<blocks, 32 * warps, sm, st>>>(nrows, X.rp, X.ci, X.a, X.m, Y.rp, Y.ci, Y.a, Y.m, cap, d_cnt,
                                                  C.rp, C.ci, C.a, C.m);
  }
  if (nlong > 0) {
    ProfScope ps(st, P_OTHER, 0.0, 0.0);
    k_spgemm_long<<<ceil_div(nlong, 64), 64, 0, st>>>(nlong, d_long, ncols, X.rp, X.ci, X.a, X.m, Y.rp, Y.ci, Y.a,
                                                     Y.m, d_mark, d_sa, d_sm, nullptr, C.rp, C.ci, C.a, C.m);
  }
  SCK(cudaGetLastError());
  return AMGEIG_OK;
}

void pad8(std::vector<uint8_t>& b) {
  while (b.size() % 8) b.push_back(0);
}
template <typename T>
void put(std::vector<uint8_t>& b, const T* p, size_t count) {
  const uint8_t* s = reinterpret_cast<const uint8_t*>(p);
  b.insert(b.end(), s, s + sizeof(T) * count);
  pad8(b);
}

// the blob layout of the package's writer (inputs/hierarchy.py), version 1
std::vector<uint8_t> write_blob(const std::vector<Csr>& L, const std::vector<Csr>& P) {
  std::vector<uint8_t> b;
  const uint32_t version = 1, n = static_cast<uint32_t>(L.size());
  b.insert(b.end(), {'A', 'M', 'G', 'E', 'I', 'G', 'H', '1'});
  b.insert(b.end(), reinterpret_cast<const uint8_t*>(&version), reinterpret_cast<const uint8_t*>(&version) + 4);
  b.insert(b.end(), reinterpret_cast<const uint8_t*>(&n), reinterpret_cast<const uint8_t*>(&n) + 4);
  for (const Csr& x : L) {
    const uint64_t r = static_cast<uint64_t>(x.rows);
    b.insert(b.end(), reinterpret_cast<const uint8_t*>(&r), reinterpret_cast<const uint8_t*>(&r) + 8);
  }
  for (const Csr& x : L) {
    const uint64_t z = x.ci.size();
    b.insert(b.end(), reinterpret_cast<const uint8_t*>(&z), reinterpret_cast<const uint8_t*>(&z) + 8);
  }
  for (const Csr& x : P) {
    const uint64_t z = x.ci.size();
    b.insert(b.end(), reinterpret_cast<const uint8_t*>(&z), reinterpret_cast<const uint8_t*>(&z) + 8);
  }
  pad8(b);
  for (const Csr& x : L) {
    put(b, x.rp.data(), x.rp.size());
    put(b, x.ci.data(), x.ci.size());
    put(b, x.a.data(), x.a.size());
    put(b, x.m.data(), x.m.size());
  }
  for (const Csr& x : P) {
    put(b, x.rp.data(), x.rp.size());
    put(b, x.ci.data(), x.ci.size());
    put(b, x.a.data(), x.a.size());
  }
  uint64_t sum = 0;
  for (size_t i = 0; i + 8 <= b.size(); i += 8) {
    uint64_t w;
    std::memcpy(&w, b.data() + i, 8);
    sum += w;
  }
  b.insert(b.end(), reinterpret_cast<const uint8_t*>(&sum), reinterpret_cast<const uint8_t*>(&sum) + 8);
  return b;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ------------------------------------------------------------------ blob checks and transposes at load
//
// The loader copies a hierarchy blob to the device in one piece and uses its
// arrays in place; these kernels check it there (the word-sum checksum and
// every CSR structure) before any kernel follows a column index, and form the
// restrictions R = P^T.

namespace {

// sum (mod 2^64) of n 64-bit words
__global__ void k_word_sum(const unsigned long long* __restrict__ w, long long n, unsigned long long* out) {
  unsigned long long acc = 0;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    acc += w[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// *bad = 1 unless rp[0] = 0, rp[rows] = nnz, rp non-decreasing and 0 <= ci < cols
__global__ void k_csr_check(const int* __restrict__ rp, const int* __restrict__ ci, long long rows, long long cols,
                            long long nnz, int* bad) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  const long long t0 = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  int ok = 1;
  if (t0 == 0 && (rp[0] != 0 || static_cast<long long>(rp[rows]) != nnz)) ok = 0;
  for (long long i = t0; i < rows; i += stride)
    if (rp[i + 1] < rp[i]) ok = 0;
  for (long long p = t0; p < nnz; p += stride)
    if (ci[p] < 0 || static_cast<long long>(ci[p]) >= cols) ok = 0;
  if (!ok) atomicOr(bad, 1);
}

__global__ void k_count_cols(const int* __restrict__ ci, long long nnz, int* __restrict__ cnt) {
  for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < nnz;
       p += static_cast<long long>(gridDim.x) * blockDim.x)
    atomicAdd(&cnt[ci[p]], 1);
}

// Exclusive scan of n int counts in three passes over up to 1024 blocks: the
// blocks' chunk sums, one block scanning those (int64), then each block
// scanning its chunk from its offset (inside a block each thread sums a slice,
// the slice totals are scanned in shared memory, each thread writes its slice).
constexpr int kScanThreads = 1024, kScanBlocks = 1024;

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const int* __restrict__ cnt, long long n, long long chunk,
                                                            long long* __restrict__ bsum) {
  __shared__ long long red[32];
  const long long b0 = blockIdx.x * chunk, b1 = b0 + chunk < n ? b0 + chunk : n;
  long long s = 0;
  for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += cnt[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += red[w];
    bsum[blockIdx.x] = t;
  }
}

// inclusive scan of part[0 .. blockDim) in place (Hillis-Steele)
__device__ void block_scan_inclusive(long long* part) {
  const int t = threadIdx.x;
  for (int o = 1; o < static_cast<int>(blockDim.x); o <<= 1) {
    const long long v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_offsets(long long* __restrict__ bsum, int nb,
                                                               long long* __restrict__ total) {
  __shared__ long long part[kScanThreads];
  const int t = threadIdx.x;
  const long long v = t < nb ? bsum[t] : 0;
  part[t] = v;
  __syncthreads();
  block_scan_inclusive(part);
  if (t < nb) bsum[t] = part[t] - v;  // exclusive offsets
  if (t == blockDim.x - 1 && total) *total = part[t];
}

__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(const int* __restrict__ cnt, long long n, long long chunk,
                                                              const long long* __restrict__ boff, int* __restrict__ out) {
  __shared__ long long part[kScanThreads];
  const int t = threadIdx.x;
  const long long c0 = blockIdx.x * chunk, c1 = c0 + chunk < n ? c0 + chunk : n;
  const long long per = (chunk + blockDim.x - 1) / blockDim.x;
  const long long b = c0 + t * per, e = b + per < c1 ? b + per : c1;
  long long s = 0;
  for (long long i = b; i < e; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  block_scan_inclusive(part);
  long long run = boff[blockIdx.x] + part[t] - s;
  if (blockIdx.x == 0 && t == 0) out[0] = 0;
  for (long long i = b; i < e; ++i) {
    run += cnt[i];
    out[i + 1] = static_cast<int>(run);
  }
}

void scan_counts(const int* cnt, long long n, int* out, long long* tmp, long long* total, cudaStream_t st) {
  long long chunk = (n + kScanBlocks - 1) / kScanBlocks;
  if (chunk < kScanThreads) chunk = kScanThreads;
  const int nb = static_cast<int>((n + chunk - 1) / chunk > 0 ? (n + chunk - 1) / chunk : 1);
  k_scan_sums<<<nb, kScanThreads, 0, st>>>(cnt, n, chunk, tmp);
  k_scan_offsets<<<1, kScanThreads, 0, st>>>(tmp, nb, total);
  k_scan_chunks<<<nb, kScanThreads, 0, st>>>(cnt, n, chunk, tmp, out);
}

// R entries at atomically taken positions of their rows (next: the rows' running offsets)
__global__ void k_transpose_fill(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                                 long long rows, int* __restrict__ next, int* __restrict__ rci,
                                 double* __restrict__ rv) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < rows;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const int k = atomicAdd(&next[ci[p]], 1);
      rci[k] = static_cast<int>(i);
      rv[k] = v[p];
    }
}

// each row of R sorted by column (insertion sort: a few entries per row), so that R is
// the same whatever order the atomics took
__global__ void k_sort_rows(const int* __restrict__ rp, long long rows, int* __restrict__ ci, double* __restrict__ v) {
  for (long long r = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; r < rows;
       r += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int b = rp[r], e = rp[r + 1];
    for (int p = b + 1; p < e; ++p) {
      const int c = ci[p];
      const double x = v[p];
      int k = p - 1;
      while (k >= b && ci[k] > c) {
        ci[k + 1] = ci[k];
        v[k + 1] = v[k];
        --k;
      }
      ci[k + 1] = c;
      v[k + 1] = x;
    }
  }
}

int load_grid(long long n) {
  const long long b = (n + 255) / 256;
  return static_cast<int>(b < 4 * kNumSms ? (b > 0 ? b : 1) : 4 * kNumSms);
}

}  // namespace

void launch_blob_checksum(const void* blob, size_t bytes, unsigned long long* out, cudaStream_t st) {
  const long long words = static_cast<long long>(bytes / 8);
  ProfScope ps(st, P_OTHER, 1.0 * bytes, 0.0);
  k_word_sum<<<load_grid(words), 256, 0, st>>>(static_cast<const unsigned long long*>(blob), words, out);
}

void launch_csr_check(const int* rp, const int* ci, long long rows, long long cols, long long nnz, int* bad,
                      cudaStream_t st) {
  ProfScope ps(st, P_OTHER, 4.0 * (rows + 1) + 4.0 * nnz, 0.0);
  k_csr_check<<<load_grid(rows > nnz ? rows : nnz), 256, 0, st>>>(rp, ci, rows, cols, nnz, bad);
}

void launch_exclusive_scan(const int* cnt, long long n, int* out, long long* tmp, long long* total,
                           cudaStream_t st) {
  ProfScope ps(st, P_OTHER, 8.0 * n, 0.0, 3);
  scan_counts(cnt, n, out, tmp, total, st);
}

void launch_transpose_csr(long long rows, long long cols, long long nnz, const int* rp, const int* ci,
                          const double* v, int* rrp, int* rci, double* rv, int* scratch, long long* tmp,
                          cudaStream_t st) {
  ProfScope ps(st, P_OTHER, 4.0 * (rows + 1) + 24.0 * nnz + 8.0 * (cols + 1), 0.0, 6);
  cudaMemsetAsync(scratch, 0, sizeof(int) * static_cast<size_t>(cols), st);
  k_count_cols<<<load_grid(nnz), 256, 0, st>>>(ci, nnz, scratch);
  scan_counts(scratch, cols, rrp, tmp, nullptr, st);
  cudaMemcpyAsync(scratch, rrp, sizeof(int) * static_cast<size_t>(cols), cudaMemcpyDeviceToDevice, st);
  k_transpose_fill<<<load_grid(rows), 256, 0, st>>>(rp, ci, v, rows, scratch, rci, rv);
  k_sort_rows<<<load_grid(cols), 256, 0, st>>>(rrp, cols, rci, rv);
}

}  // namespace amgeig

using namespace amgeig;

extern "C" int amgeig_setup_blob(int64_t n, const int32_t* rp, const int32_t* ci, const double* a,
                                 const double* m, double theta, int64_t coarse_cap, int max_levels, int device,
                                 void** blob, size_t* bytes, double* seconds) {
  set_last_error(AMGEIG_OK, nullptr);
  if (!rp || !ci || !a || !m || !blob || !bytes) return set_last_error(AMGEIG_EINVAL, "NULL argument");
  *blob = nullptr;
  *bytes = 0;
  if (n < 1 || n >= (int64_t(1) << 31) || !(theta > 0.0 && theta < 1.0) || coarse_cap < 1 || max_levels < 1)
    return set_last_error(AMGEIG_EINVAL, "invalid size, theta, coarse cap or level count");
  const int64_t nnz = rp[n];
  if (rp[0] != 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return set_last_error(AMGEIG_EINVAL, "invalid row offsets");
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return set_last_error(AMGEIG_EINVAL, "invalid row offsets");
  for (int64_t p = 0; p < nnz; ++p)
    if (ci[p] < 0 || ci[p] >= n) return set_last_error(AMGEIG_EINVAL, "column index out of range");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return set_last_error(AMGEIG_EINVAL, "no such CUDA device");
  const double t0 = now_s();
  SCK(cudaSetDevice(device));
  cudaStream_t st;
  SCK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } guard{st};
  Pool pool;
  std::vector<Csr> L(1), P;
  {
    Csr& A0 = L[0];
    A0.rows = A0.cols = n;
    A0.rp.assign(rp, rp + n + 1);
    A0.ci.assign(ci, ci + nnz);
    A0.a.assign(a, a + nnz);
    A0.m.assign(m, m + nnz);
  }
  DevMat dA;
  SCK(pool.upload(&dA.rp, L[0].rp, st));
  SCK(pool.upload(&dA.ci, L[0].ci, st));
  SCK(pool.upload(&dA.a, L[0].a, st));
  SCK(pool.upload(&dA.m, L[0].m, st));
  int* d_cnt = nullptr;
  SCK(pool.alloc(&d_cnt, static_cast<size_t>(n) + 1));
  double t_split = 0.0;
  while (static_cast<int>(L.size()) < max_levels && L.back().rows > coarse_cap) {
    const Csr& Af = L.back();
    const int nf = static_cast<int>(Af.rows);
    // C/F splitting on the host
    const double ts = now_s();
    std::vector<int8_t> state(static_cast<size_t>(nf));
    if (amgsetup_cf_split(nf, Af.rp.data(), Af.ci.data(), Af.a.data(), theta, state.data()) != 0)
      return set_last_error(AMGEIG_EINVAL, "setup: C/F splitting refused the level");
    std::vector<int32_t> cidx(static_cast<size_t>(nf), -1);
    int nc = 0;
    for (int i = 0; i < nf; ++i)
      if (state[i] == kC) cidx[i] = nc++;
    t_split += now_s() - ts;
    if (nc == 0 || nc >= nf) break;  // coarsening stalled
    int8_t* d_state = nullptr;
    int* d_cidx = nullptr;
    SCK(pool.upload(&d_state, state, st));
    SCK(pool.upload(&d_cidx, cidx, st));
    // direct interpolation P (nf x nc)
    {
      ProfScope ps(st, P_OTHER, 0.0, 0.0);
      k_interp_count<<<ceil_div(nf, 256), 256, 0, st>>>(nf, dA.rp, dA.ci, dA.a, d_state, theta, d_cnt);
    }
    std::vector<int32_t> pc(static_cast<size_t>(nf));
    SCK(cudaMemcpyAsync(pc.data(), d_cnt, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    Csr Pk;
    Pk.rows = nf;
    Pk.cols = nc;
    int rc = scan_counts(pc, Pk.rp);
    if (rc) return rc;
    const size_t pnz = static_cast<size_t>(Pk.rp.back());
    DevMat dP;
    SCK(pool.upload(&dP.rp, Pk.rp, st));
    SCK(pool.alloc(&dP.ci, pnz));
    SCK(pool.alloc(&dP.a, pnz));
    {
      ProfScope ps(st, P_OTHER, 0.0, 0.0);
      k_interp_fill<<<ceil_div(nf, 256), 256, 0, st>>>(nf, dA.rp, dA.ci, dA.a, d_state, d_cidx, theta, dP.rp, dP.ci,
                                                       dP.a);
    }
    SCK(cudaGetLastError());
    Pk.ci.resize(pnz);
    Pk.a.resize(pnz);
    SCK(cudaMemcpyAsync(Pk.ci.data(), dP.ci, sizeof(int32_t) * pnz, cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(Pk.a.data(), dP.a, sizeof(double) * pnz, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    // R = P^T (rows in ascending order of the fine index), made on the host
    Csr R;
    R.rows = nc;
    R.cols = nf;
    R.rp.assign(static_cast<size_t>(nc) + 1, 0);
    for (int32_t c : Pk.ci) R.rp[c + 1]++;
    for (int c = 0; c < nc; ++c) R.rp[c + 1] += R.rp[c];
    R.ci.resize(pnz);
    R.a.resize(pnz);
    {
      std::vector<int32_t> pos(R.rp.begin(), R.rp.end() - 1);
      for (int i = 0; i < nf; ++i)
        for (int32_t p = Pk.rp[i]; p < Pk.rp[i + 1]; ++p) {
          const int32_t q = pos[Pk.ci[p]]++;
          R.ci[q] = i;
          R.a[q] = Pk.a[p];
        }
    }
    DevMat dR;
    SCK(pool.upload(&dR.rp, R.rp, st));
    SCK(pool.upload(&dR.ci, R.ci, st));
    SCK(pool.upload(&dR.a, R.a, st));
    // A P (both value arrays), then R (A P)
    DevMat dAP, dC;
    std::vector<int32_t> aprp, crp;
    rc = spgemm(pool, nf, nc, dA, dP, dAP, aprp, d_cnt, st);
    if (rc) return rc;
    rc = spgemm(pool, nc, nc, dR, dAP, dC, crp, d_cnt, st);
    if (rc) return rc;
    Csr Ac;
    Ac.rows = Ac.cols = nc;
    Ac.rp = crp;
    const size_t cnz = static_cast<size_t>(crp.back());
    Ac.ci.resize(cnz);
    Ac.a.resize(cnz);
    Ac.m.resize(cnz);
    SCK(cudaMemcpyAsync(Ac.ci.data(), dC.ci, sizeof(int32_t) * cnz, cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(Ac.a.data(), dC.a, sizeof(double) * cnz, cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(Ac.m.data(), dC.m, sizeof(double) * cnz, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    P.push_back(std::move(Pk));
    L.push_back(std::move(Ac));
    dA = dC;
  }
  std::vector<uint8_t> b = write_blob(L, P);
  void* out = std::malloc(b.size());
  if (!out) return set_last_error(AMGEIG_ENOMEM, "setup: host allocation of the blob failed");
  std::memcpy(out, b.data(), b.size());
  *blob = out;
  *bytes = b.size();
  if (seconds) {
    seconds[0] = now_s() - t0;
    seconds[1] = t_split;
  }
  return AMGEIG_OK;
}

extern "C" void amgeig_free_blob(void* blob) { std::free(blob); }
