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

// Error-free float64 transformations for the compensated sums: Knuth's TwoSum
// and the FMA form of Dekker's TwoProduct; a running sum carries its rounding
// errors in a second word, as in Ogita, Rump and Oishi's Dot2 (2005, "Accurate
// sum and dot product"), so the result is as if accumulated in twice the
// working precision.
struct dd {
  double hi, lo;
};
// (explicitly rounded operations: no contraction into FMAs may change them)
__device__ __forceinline__ void dd_add(dd& s, double x) {
  const double t = __dadd_rn(s.hi, x);
  const double z = __dsub_rn(t, s.hi);
  s.lo = __dadd_rn(s.lo, __dadd_rn(__dsub_rn(s.hi, __dsub_rn(t, z)), __dsub_rn(x, z)));
  s.hi = t;
}
__device__ __forceinline__ void dd_fma(dd& s, double a, double b) {
  const double p = __dmul_rn(a, b);
  const double e = fma(a, b, -p);
  dd_add(s, p);
  s.lo = __dadd_rn(s.lo, e);
}

// Per block and column, over the rows the block visits (a fixed grid striding
// over the rows, so the sums are taken in a fixed order): u_c (A u)_c,
// u_c (M u)_c, (A u)_c^2, (A u)_c (M u)_c and (M u)_c^2, in float64 with the
// exact operator values.  COMP: the first two (the Rayleigh quotient's
// numerator and denominator) in compensated arithmetic, row sums and the sum
// over rows alike, written as (hi, lo) pairs: partials[block][7q] = hi0, lo0,
// hi1, lo1, s2, s3, s4 per column; otherwise partials[block][5q].  A group of
// G threads owns one row at a time; thread t of the group holds columns t,
// t+G, ...
template <int CPT, bool COMP>
__global__ void __launch_bounds__(kThreads) k_rayleigh(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                       const double* __restrict__ a, const double* __restrict__ m,
                                                       const double* __restrict__ U, int q, int G,
                                                       double* __restrict__ partials) {
  extern __shared__ double sred[];  // [rows_per_block][NS * G * CPT]
  constexpr int NS = COMP ? 7 : 5;
  const int rpb = blockDim.x / G;
  const int g = threadIdx.x / G;
  const int lane = threadIdx.x % G;
  dd s01[2][CPT];
  double s[3][CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    s01[0][t] = s01[1][t] = dd{0.0, 0.0};
    s[0][t] = s[1][t] = s[2][t] = 0.0;
  }
  for (int row = blockIdx.x * rpb + g; row < n; row += gridDim.x * rpb) {
    dd aa[CPT], mm[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) aa[t] = mm[t] = dd{0.0, 0.0};
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
          if (COMP) {
            dd_fma(aa[t], av, u);
            dd_fma(mm[t], mv, u);
          } else {
            aa[t].hi = fma(av, u, aa[t].hi);
            mm[t].hi = fma(mv, u, mm[t].hi);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      const int c = lane + t * G;
      const double ui = c < q ? U[static_cast<long long>(row) * q + c] : 0.0;
      if (COMP) {
        dd_fma(s01[0][t], ui, aa[t].hi);
        s01[0][t].lo = fma(ui, aa[t].lo, s01[0][t].lo);
        dd_fma(s01[1][t], ui, mm[t].hi);
        s01[1][t].lo = fma(ui, mm[t].lo, s01[1][t].lo);
      } else {
        s01[0][t].hi = fma(ui, aa[t].hi, s01[0][t].hi);
        s01[1][t].hi = fma(ui, mm[t].hi, s01[1][t].hi);
      }
      const double ah = aa[t].hi + aa[t].lo, mh = mm[t].hi + mm[t].lo;
      s[0][t] = fma(ah, ah, s[0][t]);
      s[1][t] = fma(ah, mh, s[1][t]);
      s[2][t] = fma(mh, mh, s[2][t]);
    }
  }
  const int W = G * CPT;
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    const int col = lane + t * G;
    double* r = sred + g * NS * W + col;
    if (COMP) {
      r[0 * W] = s01[0][t].hi;
      r[1 * W] = s01[0][t].lo;
      r[2 * W] = s01[1][t].hi;
      r[3 * W] = s01[1][t].lo;
      r[4 * W] = s[0][t];
      r[5 * W] = s[1][t];
      r[6 * W] = s[2][t];
    } else {
      r[0 * W] = s01[0][t].hi;
      r[1 * W] = s01[1][t].hi;
      r[2 * W] = s[0][t];
      r[3 * W] = s[1][t];
      r[4 * W] = s[2][t];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NS * q; idx += blockDim.x) {
    const int k = idx / q, c = idx % q;
    if (COMP && (k == 0 || k == 2)) {
      // the compensated pairs: hi words summed with TwoSum, lo words added
      dd acc{0.0, 0.0};
      for (int r = 0; r < rpb; ++r) {
        dd_add(acc, sred[(r * NS + k) * W + c]);
        acc.lo += sred[(r * NS + k + 1) * W + c];
      }
      partials[static_cast<long long>(blockIdx.x) * NS * q + k * q + c] = acc.hi;
      partials[static_cast<long long>(blockIdx.x) * NS * q + (k + 1) * q + c] = acc.lo;
    } else if (COMP && (k == 1 || k == 3)) {
      continue;  // written with its hi word
    } else {
      double v = 0.0;
      for (int r = 0; r < rpb; ++r) v += sred[(r * NS + k) * W + c];
      partials[static_cast<long long>(blockIdx.x) * NS * q + idx] = v;
    }
  }
}

// Compensated partials (7q per block) to the 5q sums the finish reads: the
// numerator and denominator summed over blocks in compensated arithmetic
// (rounded once at the end), the norms plainly; fixed order.
__global__ void k_sum_rayleigh_comp(const double* __restrict__ part, int nparts, int q, double* __restrict__ sums) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 5 * q) return;
  const int k = idx / q, c = idx % q;
  if (k < 2) {
    dd acc{0.0, 0.0};
    for (int b = 0; b < nparts; ++b) {
      dd_add(acc, part[static_cast<long long>(b) * 7 * q + (2 * k) * q + c]);
      acc.lo += part[static_cast<long long>(b) * 7 * q + (2 * k + 1) * q + c];
    }
    sums[idx] = acc.hi + acc.lo;
  } else {
    double v = 0.0;
    for (int b = 0; b < nparts; ++b) v += part[static_cast<long long>(b) * 7 * q + (k + 2) * q + c];
    sums[idx] = v;
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

void launch_rayleigh_f64(const DevCsr& AM, const double* U, int q, bool compensated, double* partials,
                         double* sums, cudaStream_t st) {
  int G = 1;
  while (G < q && G < 32) G <<= 1;
  int cpt = 1;
  while (cpt * G < q) cpt <<= 1;
  const int rpb = kThreads / G;
  const int blocks = std::min(ceil_div(AM.rows, rpb), rayleigh_blocks(q));
  const int ns = compensated ? 7 : 5;
  const double N = AM.rows, nnz = AM.nnz;
  // float64 operations: two FMAs per (nonzero, column), or the compensated
  // product-sums (about eight operations each)
  ProfScope ps(st, P_DEFECT, 4.0 * (N + 1) + 20.0 * nnz + 8.0 * N * q,
               (compensated ? 16.0 : 4.0) * nnz * q + 10.0 * N * q, 2);
  const size_t sm = sizeof(double) * rpb * ns * G * cpt;
  if (sm > 48 * 1024) {
    if (compensated) {
      ensure_dynamic_smem(reinterpret_cast<const void*>(k_rayleigh<1, true>), sm);
      ensure_dynamic_smem(reinterpret_cast<const void*>(k_rayleigh<2, true>), sm);
      ensure_dynamic_smem(reinterpret_cast<const void*>(k_rayleigh<4, true>), sm);
    }
  }
  switch (cpt) {
#define AMGEIG_CASE(C)                                                                                        \
  case C:                                                                                                     \
    if (compensated)                                                                                          \
      k_rayleigh<C, true><<<blocks, kThreads, sm, st>>>(AM.rows, AM.rp, AM.ci, AM.v64, AM.m64, U, q, G,     \
                                                        partials);                                            \
    else                                                                                                      \
      k_rayleigh<C, false><<<blocks, kThreads, sm, st>>>(AM.rows, AM.rp, AM.ci, AM.v64, AM.m64, U, q, G,    \
                                                         partials);                                           \
    break;
    AMGEIG_CASE(1)
    AMGEIG_CASE(2)
    AMGEIG_CASE(4)
#undef AMGEIG_CASE
    default:
      break;
  }
  if (compensated)
    k_sum_rayleigh_comp<<<ceil_div(5 * q, 128), 128, 0, st>>>(partials, blocks, q, sums);
  else
    launch_sum_partials(partials, blocks, 5 * q, sums, st);
}

void launch_rq_finish(const double* sums, int q, double* theta, double* lam, int* perm, double* relres, int* flag,
                      cudaStream_t st) {
  ProfScope ps(st, P_OTHER, 8.0 * 5 * q + 40.0 * q, 0.0);
  k_rq_finish<<<1, 32, 0, st>>>(sums, q, theta, lam, perm, relres, flag);
}

// ---------------------------------------------------------------- Krylov block helpers

namespace {

template <typename TV, typename TE>
__global__ void k_pack_krylov(int rows, const TV* __restrict__ V1, const TE* __restrict__ E, int lde, int q,
                              TV* __restrict__ K) {
  const long long total = static_cast<long long>(rows) * 2 * q;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = i / (2 * q);
    const int c = static_cast<int>(i % (2 * q));
    if (c < q) {
      K[i] = V1[r * q + c];
    } else {
      if constexpr (sizeof(TV) == sizeof(double) && sizeof(TE) == sizeof(double)) {
        K[i] = E[r * lde + c - q];
      } else {
        K[i] = make_float2(E[r * lde + c - q], 0.f);
      }
    }
  }
}

// U = Xp + V Y with V rows x nv and Y nv x q (float64), one thread per (row, column)
__global__ void k_recombine_wide(int rows, const double* __restrict__ Xp, const double* __restrict__ V, int nv,
                                 const double* __restrict__ Y, int q, double* __restrict__ U) {
  const long long total = static_cast<long long>(rows) * q;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = i / q;
    const int c = static_cast<int>(i % q);
    double acc = Xp[i];
    for (int d = 0; d < nv; ++d) acc = fma(V[r * nv + d], Y[d * q + c], acc);
    U[i] = acc;
  }
}

int grid_of(long long n) { return static_cast<int>(std::min<long long>((n + kThreads - 1) / kThreads, 8LL * kNumSms)); }

}  // namespace

void launch_pack_krylov_f64(int rows, const double* V1, const double* E, int lde, int q, double* K, cudaStream_t st) {
  const long long n = static_cast<long long>(rows) * 2 * q;
  ProfScope ps(st, P_OTHER, 24.0 * rows * q, 0.0);
  k_pack_krylov<double, double><<<grid_of(n), kThreads, 0, st>>>(rows, V1, E, lde, q, K);
}

void launch_pack_krylov_df(int rows, const float2* V1, const float* E, int lde, int q, float2* K, cudaStream_t st) {
  const long long n = static_cast<long long>(rows) * 2 * q;
  ProfScope ps(st, P_OTHER, 20.0 * rows * q + 4.0 * rows * lde, 0.0);
  k_pack_krylov<float2, float><<<grid_of(n), kThreads, 0, st>>>(rows, V1, E, lde, q, K);
}

void launch_recombine_wide(int rows, const double* Xp, const double* V, int nv, const double* Y, int q, double* U,
                           cudaStream_t st) {
  const long long n = static_cast<long long>(rows) * q;
  ProfScope ps(st, P_RECOMBINE, 8.0 * rows * (2.0 * q + nv) + 8.0 * nv * q, 2.0 * rows * nv * q);
  k_recombine_wide<<<grid_of(n), kThreads, 0, st>>>(rows, Xp, V, nv, Y, q, U);
}

}  // namespace amgeig
