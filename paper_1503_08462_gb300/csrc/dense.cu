// Small dense kernels: GEMM on coarse-size operands, the tall-skinny Gram
// products V^T W of Algorithm 3.1 step 2 (V^T A_k V and V^T M_k V), fixed-order
// reductions of per-block partial sums, and the residual test.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"
#include "prof.cuh"

namespace amgeig {
namespace {

constexpr int kTile = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, T alpha, const T* __restrict__ A, int lda, int ta,
                                              const T* __restrict__ B, int ldb, int tb, T beta, T* __restrict__ C,
                                              int ldc) {
  __shared__ T As[kTile][kTile + 1];
  __shared__ T Bs[kTile][kTile + 1];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int row = blockIdx.y * kTile + ty, col = blockIdx.x * kTile + tx;
  T acc = T(0);
  for (int k0 = 0; k0 < K; k0 += kTile) {
    {
      const int r = blockIdx.y * kTile + ty, k = k0 + tx;
      As[ty][tx] = (r < M && k < K) ? (ta ? A[static_cast<long long>(k) * lda + r] : A[static_cast<long long>(r) * lda + k])
                                    : T(0);
    }
    {
      const int k = k0 + ty, c = blockIdx.x * kTile + tx;
      Bs[ty][tx] = (k < K && c < N) ? (tb ? B[static_cast<long long>(c) * ldb + k] : B[static_cast<long long>(k) * ldb + c])
                                    : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTile; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (row < M && col < N) {
    T* c = C + static_cast<long long>(row) * ldc + col;
    *c = (beta == T(0)) ? alpha * acc : fma(alpha, acc, beta * *c);
  }
}

// x = A b for a dense n x n row-major A and an n x w row-major block b.  One
// block per output row; its threads are (column, segment) pairs: each sums a
// contiguous segment of k for one column, and the segments are added in a
// fixed order in shared memory.  Short independent chains keep the latency of
// this once-per-V-cycle coarse solve low.
template <typename T>
__global__ void __launch_bounds__(256) k_dense_apply(int n, int w, const T* __restrict__ A, const T* __restrict__ b,
                                                     T* __restrict__ x, int segs) {
  __shared__ T part[256];
  const int c = threadIdx.x % w, sg = threadIdx.x / w;
  const int r = blockIdx.x;
  T s0 = T(0), s1 = T(0);
  if (sg < segs) {
    const int len = (n + segs - 1) / segs, k0 = sg * len, k1 = min(n, k0 + len);
    const T* a = A + static_cast<long long>(r) * n;
    int k = k0;
    for (; k + 2 <= k1; k += 2) {
      s0 = fma(a[k], b[static_cast<long long>(k) * w + c], s0);
      s1 = fma(a[k + 1], b[static_cast<long long>(k + 1) * w + c], s1);
    }
    if (k < k1) s0 = fma(a[k], b[static_cast<long long>(k) * w + c], s0);
    part[threadIdx.x] = s0 + s1;
  }
  __syncthreads();
  if (sg == 0) {
    T s = part[c];
    for (int t = 1; t < segs; ++t) s += part[t * w + c];
    x[static_cast<long long>(r) * w + c] = s;
  }
}

// Gram partials: block (chunk, tile) accumulates out[a][b] = sum_{r in chunk} V[r][a] W[r][b]
// for a 32 x 32 tile of (a, b); each thread owns 4 outputs.
constexpr int kGT = 32;
constexpr int kGramRows = 32;

template <bool DF>
__global__ void __launch_bounds__(256) k_gram_partial(int rows, const double* __restrict__ V, int ldv, int q,
                                                      const double* __restrict__ W, int ldw, int w, int chunk_rows,
                                                      int tiles_w, double* __restrict__ part) {
  // float64 operands; DF = true stages them as float-float pairs and accumulates
  // the products on the float32 pipes with compensated (two-sum) accumulation
  using Stage = typename std::conditional<DF, df, double>::type;
  __shared__ Stage Vs[kGramRows][kGT + 1];
  __shared__ Stage Ws[kGramRows][kGT + 1];
  const int chunk = blockIdx.x;
  const int ta = blockIdx.y / tiles_w, tb = blockIdx.y % tiles_w;
  const int a0 = ta * kGT, b0 = tb * kGT;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // ty in 0..7
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  df_acc facc[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) facc[s] = acc_zero();
  const int r0 = chunk * chunk_rows;
  const int r1 = min(rows, r0 + chunk_rows);
  for (int rb = r0; rb < r1; rb += kGramRows) {
    for (int idx = threadIdx.x; idx < kGramRows * kGT; idx += blockDim.x) {
      const int rr = idx / kGT, cc = idx % kGT;
      const int r = rb + rr;
      const double vv = (r < r1 && a0 + cc < q) ? V[static_cast<long long>(r) * ldv + a0 + cc] : 0.0;
      const double ww = (r < r1 && b0 + cc < w) ? W[static_cast<long long>(r) * ldw + b0 + cc] : 0.0;
      if constexpr (DF) {
        Vs[rr][cc] = df_from_double(vv);
        Ws[rr][cc] = df_from_double(ww);
      } else {
        Vs[rr][cc] = vv;
        Ws[rr][cc] = ww;
      }
    }
    __syncthreads();
    const int nr = min(kGramRows, r1 - rb);
    for (int rr = 0; rr < nr; ++rr) {
      const Stage wv = Ws[rr][tx];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if constexpr (DF)
          facc[s].fma(Vs[rr][ty * 4 + s], wv);
        else
          acc[s] = fma(Vs[rr][ty * 4 + s], wv, acc[s]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int a = a0 + ty * 4 + s, b = b0 + tx;
    double val = acc[s];
    if constexpr (DF) val = df_to_double(facc[s].value());
    if (a < q && b < w) part[(static_cast<long long>(chunk) * q + a) * w + b] = val;
  }
}

__global__ void k_sum_partials(const double* __restrict__ part, int nparts, int len, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < len; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[static_cast<long long>(b) * len + j];
    out[j] = s;
  }
}

// many parts: one block per output, strided partial sums then a fixed-shape tree
__global__ void __launch_bounds__(256) k_sum_partials_wide(const double* __restrict__ part, int nparts, int len,
                                                           double* __restrict__ out) {
  __shared__ double sh[256];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[static_cast<long long>(b) * len + j];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = sh[0];
}

__global__ void k_relres(const double* __restrict__ sums, const double* __restrict__ lam, int q,
                         double* __restrict__ relres, int* __restrict__ flags) {
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    const double r = sqrt(sums[j]) / (fabs(lam[j]) * sqrt(sums[q + j]));
    relres[j] = r;
    if (!isfinite(r) || !isfinite(lam[j])) atomicOr(flags, 1);
  }
}

__global__ void k_copy_cols(const double* __restrict__ src, int rows, int ld, int q, double* __restrict__ dst) {
  const long long total = static_cast<long long>(rows) * q;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = i / q, c = i % q;
    dst[i] = src[r * ld + c];
  }
}

// dense (rows x rows, row-major, zeroed beforehand) from a square CSR; one
// thread per row writes that row's entries of both value arrays
__global__ void k_csr_to_dense(int rows, const int* __restrict__ rp, const int* __restrict__ ci,
                               const double* __restrict__ a, const double* __restrict__ m, double* __restrict__ Ad,
                               double* __restrict__ Md) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const long long at = static_cast<long long>(i) * rows + ci[p];
    Ad[at] = a[p];
    Md[at] = m[p];
  }
}

int gram_chunks(int rows, int q, int w, int* chunk_rows) {
  const int tiles = ceil_div(q, kGT) * ceil_div(w, kGT);
  int chunks = ceil_div(rows, 256);
  const int cap = (4 * kNumSms + tiles - 1) / tiles;
  if (chunks > cap) chunks = cap;
  if (chunks < 1) chunks = 1;
  int cr = ceil_div(rows, chunks);
  cr = ceil_div(cr, kGramRows) * kGramRows;
  if (cr < kGramRows) cr = kGramRows;
  *chunk_rows = cr;
  return ceil_div(rows, cr) > 0 ? ceil_div(rows, cr) : 1;
}

}  // namespace

void launch_gemm_f64(int M, int N, int K, double alpha, const double* A, int lda, bool ta, const double* B, int ldb,
                     bool tb, double beta, double* C, int ldc, cudaStream_t st, int cls) {
  if (M <= 0 || N <= 0) return;
  ProfScope ps(st, cls, 8.0 * (1.0 * M * K + 1.0 * K * N + (beta != 0.0 ? 2.0 : 1.0) * M * N), 2.0 * M * N * K);
  dim3 grid(ceil_div(N, kTile), ceil_div(M, kTile));
  k_gemm<double><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, beta, C, ldc);
}

void launch_gemm_f32(int M, int N, int K, float alpha, const float* A, int lda, bool ta, const float* B, int ldb,
                     bool tb, float beta, float* C, int ldc, cudaStream_t st, int cls) {
  if (M <= 0 || N <= 0) return;
  ProfScope ps(st, cls, 4.0 * (1.0 * M * K + 1.0 * K * N + (beta != 0.0f ? 2.0 : 1.0) * M * N), 2.0 * M * N * K);
  dim3 grid(ceil_div(N, kTile), ceil_div(M, kTile));
  k_gemm<float><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, beta, C, ldc);
}

template <typename T>
void launch_dense_apply_t(int n, int w, const T* A, const T* b, T* x, cudaStream_t st, int cls) {
  if (n <= 0 || w <= 0) return;
  ProfScope ps(st, cls, sizeof(T) * (1.0 * n * n + 2.0 * n * w), 2.0 * n * n * w);
  const int segs = std::max(1, std::min(16, 256 / w));
  k_dense_apply<T><<<n, segs * w, 0, st>>>(n, w, A, b, x, segs);
}

void launch_dense_apply(int n, int w, const double* A, const double* b, double* x, cudaStream_t st, int cls) {
  launch_dense_apply_t(n, w, A, b, x, st, cls);
}
void launch_dense_apply(int n, int w, const float* A, const float* b, float* x, cudaStream_t st, int cls) {
  launch_dense_apply_t(n, w, A, b, x, st, cls);
}

size_t gram_scratch_doubles(int rows, int q, int w) {
  int cr;
  const int chunks = gram_chunks(rows, q, w, &cr);
  return static_cast<size_t>(chunks) * q * w;
}

void launch_gram_strided(int rows, const double* V, int ldv, int q, const double* W, int ldw, int w, double* scratch,
                         double* G, cudaStream_t st, bool df_arith) {
  if (q <= 0 || w <= 0) return;
  int cr;
  const int chunks = gram_chunks(rows, q, w, &cr);
  const int tiles_w = ceil_div(w, kGT);
  dim3 grid(chunks, ceil_div(q, kGT) * tiles_w);
  ProfScope ps(st, P_GRAM, 8.0 * rows * (q + w) + 16.0 * chunks * q * w, 2.0 * rows * q * w);
  if (df_arith)
    k_gram_partial<true><<<grid, 256, 0, st>>>(rows, V, ldv, q, W, ldw, w, cr, tiles_w, scratch);
  else
    k_gram_partial<false><<<grid, 256, 0, st>>>(rows, V, ldv, q, W, ldw, w, cr, tiles_w, scratch);
  launch_sum_partials(scratch, chunks, q * w, G, st);
}

void launch_gram(int rows, const double* V, int q, const double* W, int w, double* scratch, double* G,
                 cudaStream_t st, bool df_arith) {
  launch_gram_strided(rows, V, q, q, W, w, w, scratch, G, st, df_arith);
}

void launch_sum_partials(const double* part, int nparts, int len, double* out, cudaStream_t st) {
  if (len <= 0) return;
  ProfScope ps(st, P_OTHER, 8.0 * (nparts + 1.0) * len, 1.0 * nparts * len);
  if (nparts >= 64)
    k_sum_partials_wide<<<len, 256, 0, st>>>(part, nparts, len, out);
  else
    k_sum_partials<<<ceil_div(len, 256), 256, 0, st>>>(part, nparts, len, out);
}

void launch_relres(const double* sums, const double* lam, int q, double* relres, int* flags, cudaStream_t st) {
  ProfScope ps(st, P_DEFECT, 32.0 * q, 4.0 * q);
  k_relres<<<1, 256, 0, st>>>(sums, lam, q, relres, flags);
}

void launch_copy_cols(const double* src, int rows, int ld, int q, double* dst, cudaStream_t st) {
  const long long total = static_cast<long long>(rows) * q;
  if (total <= 0) return;
  ProfScope ps(st, P_OTHER, 16.0 * total, 0.0);
  long long b = (total + 255) / 256;
  if (b > 8 * kNumSms) b = 8 * kNumSms;
  k_copy_cols<<<static_cast<int>(b), 256, 0, st>>>(src, rows, ld, q, dst);
}

void launch_csr_to_dense(int rows, const int* rp, const int* ci, const double* a, const double* m, double* Ad,
                         double* Md, cudaStream_t st) {
  const double bytes = 16.0 * rows * static_cast<double>(rows);
  ProfScope ps(st, P_OTHER, bytes, 0.0, 3);
  cudaMemsetAsync(Ad, 0, sizeof(double) * rows * static_cast<size_t>(rows), st);
  cudaMemsetAsync(Md, 0, sizeof(double) * rows * static_cast<size_t>(rows), st);
  k_csr_to_dense<<<ceil_div(rows, 128), 128, 0, st>>>(rows, rp, ci, a, m, Ad, Md);
}

}  // namespace amgeig
