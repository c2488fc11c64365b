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

// Per block and column, over the rows the block visits (a fixed grid striding
// over the rows, so the sums are taken in a fixed order): u_c (A u)_c,
// u_c (M u)_c, (A u)_c^2, (A u)_c (M u)_c and (M u)_c^2, in float64 with the
// exact operator values.  A group of G threads owns one row at a time; thread t
// of the group holds columns t, t+G, ...
template <int CPT>
__global__ void __launch_bounds__(kThreads) k_rayleigh(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                       const double* __restrict__ a, const double* __restrict__ m,
                                                       const double* __restrict__ U, int q, int G,
                                                       double* __restrict__ partials) {
  extern __shared__ double sred[];  // [rows_per_block][5 * G * CPT]
  const int rpb = blockDim.x / G;
  const int g = threadIdx.x / G;
  const int lane = threadIdx.x % G;
  double s[5][CPT];
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int t = 0; t < CPT; ++t) s[k][t] = 0.0;
  for (int row = blockIdx.x * rpb + g; row < n; row += gridDim.x * rpb) {
    double aa[CPT], mm[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) aa[t] = mm[t] = 0.0;
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
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      const int c = lane + t * G;
      const double ui = c < q ? U[static_cast<long long>(row) * q + c] : 0.0;
      s[0][t] = fma(ui, aa[t], s[0][t]);
      s[1][t] = fma(ui, mm[t], s[1][t]);
      s[2][t] = fma(aa[t], aa[t], s[2][t]);
      s[3][t] = fma(aa[t], mm[t], s[3][t]);
      s[4][t] = fma(mm[t], mm[t], s[4][t]);
    }
  }
  const int W = G * CPT;
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int t = 0; t < CPT; ++t) sred[(g * 5 + k) * W + lane + t * G] = s[k][t];
  __syncthreads();
  for (int idx = threadIdx.x; idx < 5 * q; idx += blockDim.x) {
    const int k = idx / q, c = idx % q;
    double v = 0.0;
    for (int r = 0; r < rpb; ++r) v += sred[(r * 5 + k) * W + c];
    partials[static_cast<long long>(blockIdx.x) * 5 * q + idx] = v;
  }
}

// theta_j = u^T A u / u^T M u per column; lam = theta sorted ascending (a stable
// insertion sort, q <= 128, one thread), perm[c] = the column holding the c-th
// smallest; relres_j from ||A u - theta M u||^2 = ||Au||^2 - 2 theta (Au)^T(Mu)
// + theta^2 ||Mu||^2.  That expansion loses the digits it cancels: where the
// squared residual falls below 1e-10 of ||Au||^2 (relative residuals below
// ~1e-5), flag[0] asks for the residual to be formed explicitly instead.
__global__ void k_rq_finish(const double* __restrict__ sums, int q, double* __restrict__ theta,
                            double* __restrict__ lam, int* __restrict__ perm, double* __restrict__ relres,
                            int* __restrict__ flag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int redo = 0;
  for (int j = 0; j < q; ++j) {
    const double uau = sums[j], umu = sums[q + j], aa = sums[2 * q + j], am = sums[3 * q + j],
                 mm = sums[4 * q + j];
    const double th = uau / umu;
    theta[j] = th;
    perm[j] = j;
    const double rr = aa - 2.0 * th * am + th * th * mm;
    if (!(rr >= 1e-10 * aa)) redo = 1;
    relres[j] = sqrt(fmax(rr, 0.0)) / (fabs(th) * sqrt(mm));
    if (!isfinite(th) || !isfinite(relres[j])) redo = 2;
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
  flag[0] = redo;
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

int rayleigh_blocks(int) { return 4 * kNumSms; }

void launch_rayleigh_f64(const DevCsr& AM, const double* U, int q, double* partials, int* nblocks_out,
                         cudaStream_t st) {
  int G = 1;
  while (G < q && G < 32) G <<= 1;
  int cpt = 1;
  while (cpt * G < q) cpt <<= 1;
  const int rpb = kThreads / G;
  const int blocks = std::min(ceil_div(AM.rows, rpb), rayleigh_blocks(q));
  *nblocks_out = blocks;
  const double N = AM.rows, nnz = AM.nnz;
  ProfScope ps(st, P_DEFECT, 4.0 * (N + 1) + 20.0 * nnz + 8.0 * N * q, 4.0 * nnz * q + 10.0 * N * q);
  const size_t sm = sizeof(double) * rpb * 5 * G * cpt;
  switch (cpt) {
#define AMGEIG_CASE(C)                                                                                           \
  case C:                                                                                                        \
    k_rayleigh<C><<<blocks, kThreads, sm, st>>>(AM.rows, AM.rp, AM.ci, AM.v64, AM.m64, U, q, G, partials); \
    break;
    AMGEIG_CASE(1)
    AMGEIG_CASE(2)
    AMGEIG_CASE(4)
#undef AMGEIG_CASE
    default:
      break;
  }
}

void launch_rq_finish(const double* sums, int q, double* theta, double* lam, int* perm, double* relres, int* flag,
                      cudaStream_t st) {
  ProfScope ps(st, P_OTHER, 8.0 * 5 * q + 40.0 * q, 0.0);
  k_rq_finish<<<1, 32, 0, st>>>(sums, q, theta, lam, perm, relres, flag);
}

}  // namespace amgeig
