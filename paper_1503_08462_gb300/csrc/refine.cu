// Final float64 Rayleigh-quotient refinement of the mixed path.
//
// The mixed path iterates with a float32 V-cycle and float-float Rayleigh-Ritz
// data; the operator values it multiplies with in float-float are A and M
// rounded to 48 bits, which perturbs each eigenvalue by up to ~2^-48 |u|^T|A||u|
// / u^T A u relative -- above 1e-8 on the coefficient-jump problems, where
// |A| is large against lambda M.  The refinement recomputes, in float64 with the
// exact (float64) operator values, each vector's Rayleigh quotient
// theta_j = u_j^T A u_j / u_j^T M u_j (the eigenvalue estimate whose error is
// quadratic in the vector's error) and its relative residual
// ||A u_j - theta_j M u_j|| / (|theta_j| ||M u_j||).  The values are sorted
// ascending; the permutation is applied to the output vectors.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "prof.cuh"

namespace amgeig {
namespace {

constexpr int kThreads = 256;

// Per block and column: sums over the block's rows of u_c (A u)_c and
// u_c (M u)_c (float64 products and sums in a fixed order).  A group of G
// threads owns one row; thread t of the group holds columns t, t+G, ...
template <int CPT>
__global__ void __launch_bounds__(kThreads) k_rayleigh(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                       const double* __restrict__ a, const double* __restrict__ m,
                                                       const double* __restrict__ U, int q, int G,
                                                       double* __restrict__ partials) {
  extern __shared__ double sred[];  // [rows_per_block][2 * G * CPT]
  const int rpb = blockDim.x / G;
  const int g = threadIdx.x / G;
  const int lane = threadIdx.x % G;
  const int row = blockIdx.x * rpb + g;
  double aa[CPT], mm[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) aa[t] = mm[t] = 0.0;
  if (row < n) {
    const int p0 = rp[row], p1 = rp[row + 1];
    for (int p = p0; p < p1; ++p) {
      const int j = ci[p];
      const double av = a[p], mv = m[p];
      const double* uj = U + static_cast<long long>(j) * q;
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        const int c = lane + t * G;
        if (c < q) {
          const double u = uj[c];
          aa[t] = fma(av, u, aa[t]);
          mm[t] = fma(mv, u, mm[t]);
        }
      }
    }
  }
  const int W = G * CPT;
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    const int c = lane + t * G;
    const double ui = (row < n && c < q) ? U[static_cast<long long>(row) * q + c] : 0.0;
    sred[g * 2 * W + lane + t * G] = ui * aa[t];
    sred[g * 2 * W + W + lane + t * G] = ui * mm[t];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 2 * q; idx += blockDim.x) {
    const int which = idx / q, c = idx % q;
    double s = 0.0;
    for (int r = 0; r < rpb; ++r) s += sred[r * 2 * W + which * W + c];
    partials[static_cast<long long>(blockIdx.x) * 2 * q + idx] = s;
  }
}

// theta_j = sums[j] / sums[q + j] per column; the values sorted ascending (a
// stable insertion sort, q <= 128, one thread) into lam with perm[c] = the
// column holding the c-th smallest.
__global__ void k_rq_finish(const double* __restrict__ sums, int q, double* __restrict__ theta,
                            double* __restrict__ lam, int* __restrict__ perm) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int j = 0; j < q; ++j) {
    theta[j] = sums[j] / sums[q + j];
    perm[j] = j;
  }
  for (int i = 1; i < q; ++i) {
    const int pi = perm[i];
    const double v = theta[pi];
    int k = i - 1;
    while (k >= 0 && theta[perm[k]] > v) {
      perm[k + 1] = perm[k];
      --k;
    }
    perm[k + 1] = pi;
  }
  for (int c = 0; c < q; ++c) lam[c] = theta[perm[c]];
}

__global__ void k_gather_cols(const double* __restrict__ src, int rows, int ld, const int* __restrict__ perm, int q,
                              double* __restrict__ dst) {
  const long long total = static_cast<long long>(rows) * q;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = i / q;
    const int c = static_cast<int>(i % q);
    dst[i] = src[r * ld + perm[c]];
  }
}

}  // namespace

void launch_gather_cols(const double* src, int rows, int ld, const int* perm, int q, double* dst, cudaStream_t st) {
  const long long total = static_cast<long long>(rows) * q;
  ProfScope ps(st, P_OTHER, 16.0 * total, 0.0);
  const int blocks = static_cast<int>(std::min<long long>((total + kThreads - 1) / kThreads, 8LL * kNumSms));
  k_gather_cols<<<blocks, kThreads, 0, st>>>(src, rows, ld, perm, q, dst);
}

void launch_rayleigh_f64(const DevCsr& AM, const double* U, int q, double* partials, int* nblocks_out,
                         cudaStream_t st) {
  int G = 1;
  while (G < q && G < 32) G <<= 1;
  int cpt = 1;
  while (cpt * G < q) cpt <<= 1;
  const int rpb = kThreads / G;
  const int blocks = ceil_div(AM.rows, rpb);
  *nblocks_out = blocks;
  const double N = AM.rows, nnz = AM.nnz;
  ProfScope ps(st, P_DEFECT, 4.0 * (N + 1) + 20.0 * nnz + 8.0 * N * q, 4.0 * nnz * q + 4.0 * N * q);
  const size_t sm = sizeof(double) * rpb * 2 * G * cpt;
  switch (cpt) {
#define AMGEIG_CASE(C)                                                                                           \
  case C:                                                                                                        \
    k_rayleigh<C><<<blocks, kThreads, sm, st>>>(AM.rows, AM.rp, AM.ci, AM.v64, AM.m64, U, q, G, partials); \
    break;
    AMGEIG_CASE(1)
    AMGEIG_CASE(2)
    AMGEIG_CASE(4)
    AMGEIG_CASE(8)
#undef AMGEIG_CASE
    default:
      break;
  }
}

void launch_rq_finish(const double* sums, int q, double* theta, double* lam, int* perm, cudaStream_t st) {
  ProfScope ps(st, P_OTHER, 16.0 * q + 16.0 * q, 0.0);
  k_rq_finish<<<1, 32, 0, st>>>(sums, q, theta, lam, perm);
}

}  // namespace amgeig
