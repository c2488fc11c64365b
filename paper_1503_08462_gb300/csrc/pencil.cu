// The small dense eigenproblems of the method, on the GPU.
//
// Algorithm 3.1 step 2 solves A_{n,k} x = lambda M_{n,k} x on V_n + span(V),
// a pencil of size d_n + q, and Algorithm 3.2 step 1 solves (A_n, M_n).  The
// paper treats these as black boxes (ARPACK, Sec. 4.1).  Here:
//
// * The coarsest level: at load A_n = L L^T gives the V-cycle's exact solve
//   A_n^-1 = L^-T L^-1 (float64); M_n = L_m L_m^T, H = L_m^-1 A_n L_m^-T,
//   H = Y Theta Y^T, Z = L_m^-T Y gives, for as many leading modes as a solve
//   needs, Z^T M_n Z = I and Z^T A_n Z = Theta: step 1 of Algorithm 3.2 (the q
//   smallest columns of Z) and the coarse modes of the pencil below.
// * Each correction's pencil is written in the basis [I_n^k Z_m, V - I_n^k Z_m B]
//   (block Gram-Schmidt of V against the first m coarse modes) with
//   K = Z_m^T I_k^n A_k V, B = Z_m^T I_k^n M_k V: it becomes
//       At = [[Theta, K - Theta B], [., V^T A V - B^T K - K^T B + B^T Theta B]],
//       Mt = [[I, 0], [0, S]],   S = V^T M V - B^T B,
//   whose eigenvectors [a; b] map back to x = I_n^k Z_m (a - B b) + V b.  The
//   q wanted pairs come from a structured Rayleigh quotient iteration checked by
//   Sylvester's inertia; when the check fails, S = L L^T reduces the pencil to
//   the standard symmetric matrix H = [[Theta, F], [F^T, T]], F = (K - Theta B)
//   L^-T, T = L^-1 (...) L^-T, solved by the dense eigensolver below.  Both are
//   the same Rayleigh-Ritz problem (same eigenvalues as the paper's pencil),
//   only better conditioned, and everything runs in float-float.
// * The symmetric eigenproblem is solved in float-float (48-bit significand):
//   Householder tridiagonalisation (one 1024-thread block), bisection with
//   Sturm counts for the wanted eigenvalues (float32), each shift refined by
//   float-float Sturm multisection, inverse iteration in float-float
//   (Gram-Schmidt inside clusters of nearly equal shifts), a Rayleigh-Ritz
//   clean-up by parallel cyclic Jacobi on each group of close shifts, and
//   back-transformation; the phases after the tridiagonalisation run one warp
//   or one block per eigenvalue, group or eigenvector.  References: Golub & Van Loan, Matrix
//   Computations, 4th ed., 8.3 (tridiagonalisation), 8.4.1 (Sturm bisection),
//   8.2.2 (inverse iteration), 8.5 (Jacobi).
#include <cooperative_groups.h>

#include <cstdio>
#include <map>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "prof.cuh"

namespace amgeig {

#ifndef AMGEIG_SY_THREADS
#define AMGEIG_SY_THREADS 1024
#endif
constexpr int kSyThreads = AMGEIG_SY_THREADS;

struct PencilWork {
  int dn = 0, qmax = 0, nmax = 0;
  void* base = nullptr;  // one device allocation holding every array below
  size_t bytes = 0;      // its size
  // Rayleigh-Ritz pencil (float-float)
  df* KB = nullptr;   // dn x 2q   Z_m^T C = [K | B]
  df* Ft = nullptr;   // dn x q    K - Theta B
  df* Tt = nullptr;   // q x q
  df* St = nullptr;   // q x q     Schur complement of the Gram matrix
  df* Lq = nullptr;   // q x q     its Cholesky factor (fallback)
  df* Xq = nullptr;   // q x q     scratch (fallback)
  double* H = nullptr;   // nmax x nmax standard form (fallback)
  double* Yh = nullptr;  // nmax x q eigenvectors [a; b]
  // float-float eigensolver
  df* W = nullptr;     // nmax x nmax
  df* tau = nullptr;   // nmax
  df* dd = nullptr;    // nmax
  df* ee = nullptr;    // nmax
  df* fac = nullptr;   // 6 x nmax x nwant_max
  df* Zt = nullptr;    // nmax x nwant_max
  df* rr = nullptr;    // 4 x nwant_max^2 (Rayleigh-Ritz clean-up)
  int* perm = nullptr; // nwant_max
  df* hv = nullptr;    // nmax x nmax reflectors (split path)
  df* shd = nullptr;   // nwant_max refined shifts (split path)
  float* bounds = nullptr;  // 4: Gershgorin bounds, ||T||, pivot floor (split path)
  int nwant_max = 0;
  // coarse decomposition
  double* Lm = nullptr;  // dn x dn
  double* Hs = nullptr;  // dn x dn
  // structured Rayleigh quotient iteration
  double* sr_mu = nullptr;  // qmax
  double* sr_X = nullptr;   // nmax x qmax
  int* sr_conv = nullptr;   // qmax
  int* sr_flag = nullptr;   // 4: accepted, reason of a rejection, inertia count, q
};

namespace {

// ------------------------------------------------------------ block helpers

// sum_i a[i sa] b[i sb] (i < len) in float-float with four interleaved
// accumulators: independent chains keep the float32 pipes busy in these
// latency-bound single-block kernels
__device__ __forceinline__ df_acc dot4(const df* a, int sa, const df* b, int sb, int len) {
  df_acc c0 = acc_zero(), c1 = acc_zero(), c2 = acc_zero(), c3 = acc_zero();
  int i = 0;
  for (; i + 4 <= len; i += 4) {
    c0.fma(a[i * sa], b[i * sb]);
    c1.fma(a[(i + 1) * sa], b[(i + 1) * sb]);
    c2.fma(a[(i + 2) * sa], b[(i + 2) * sb]);
    c3.fma(a[(i + 3) * sa], b[(i + 3) * sb]);
  }
  for (; i < len; ++i) c0.fma(a[i * sa], b[i * sb]);
  c0.merge(c1);
  c2.merge(c3);
  c0.merge(c2);
  return c0;
}

// the same with weights: sum_i a[i sa] w[i] b[i sb]
__device__ __forceinline__ df_acc dot4w(const df* a, int sa, const df* w, const df* b, int sb, int len) {
  df_acc c0 = acc_zero(), c1 = acc_zero(), c2 = acc_zero(), c3 = acc_zero();
  int i = 0;
  for (; i + 4 <= len; i += 4) {
    c0.fma(df_mul(a[i * sa], w[i]), b[i * sb]);
    c1.fma(df_mul(a[(i + 1) * sa], w[i + 1]), b[(i + 1) * sb]);
    c2.fma(df_mul(a[(i + 2) * sa], w[i + 2]), b[(i + 2) * sb]);
    c3.fma(df_mul(a[(i + 3) * sa], w[i + 3]), b[(i + 3) * sb]);
  }
  for (; i < len; ++i) c0.fma(df_mul(a[i * sa], w[i]), b[i * sb]);
  c0.merge(c1);
  c2.merge(c3);
  c0.merge(c2);
  return c0;
}

__device__ __forceinline__ int sturm_count(const float* sd, const float* se2, int n, float x, float pivmin) {
  float qv = sd[0] - x;
  int cnt = qv < 0.f;
  for (int i = 1; i < n; ++i) {
    if (fabsf(qv) < pivmin) qv = -pivmin;
    qv = sd[i] - x - __fdividef(se2[i - 1], qv);
    cnt += qv < 0.f;
  }
  return cnt;
}

// The same count in float-float; ee2 holds e_i^2.  The reciprocal of the
// previous pivot replaces the division (one Newton step on the float32 rcp).
__device__ __forceinline__ int sturm_count_df(const df* dd, const df* ee2, int n, df x, float pivmin) {
  df qv = df_sub(dd[0], x);
  int cnt = df_lt0(qv);
  for (int i = 1; i < n; ++i) {
    if (fabsf(qv.hi) < pivmin) qv = df{-pivmin, 0.f};
    qv = df_sub(df_sub(dd[i], x), df_mul(ee2[i - 1], df_recip(qv)));
    cnt += df_lt0(qv);
  }
  return cnt;
}

// ------------------------------------------------------------ float-float syev
//
// The phases of the solver are device functions with two drivers: k_syev_df
// runs all of them in one block (the allocation-free entry point), the split
// path runs the tridiagonalisation in one block (k_syev_tri) and spreads the
// per-eigenvalue phases over many: the shifts one warp each (k_syev_vals),
// inverse iteration and clean-up one block per group of close shifts
// (k_syev_vecs) and the back-transformation one warp per eigenvector
// (k_syev_back).  Each eigenvalue's phases do the same arithmetic on both.

// Householder tridiagonalisation of the symmetric W (n x n, row stride LD,
// full storage) by the whole block.  Four barriers per step: the norm of the
// next column and v^T p are formed from per-warp partial sums written in the
// preceding phase.  On return dd, ee hold the tridiagonal, tau the reflector
// scalars and column k of W below the diagonal the reflector v_k, which is
// also written to hv[k n + i] (i < n - k - 1) when hv is given.  v, p: n df of
// scratch each; red_sig, red_vp: 32 per-warp partial sums each.
__device__ void syev_tridiagonalise(int n, df* W, long long LD, df* v, df* p, df* dd, df* ee, df* tau,
                                    df_acc* red_sig, df_acc* red_vp, df* hv) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  // sigma partials of column 0 (rows 2..n-1)
  {
    df_acc a = acc_zero();
    for (int i = 2 + warp; i < n; i += nw)
      if (lane == 0) a.fma(W[i * LD], W[i * LD]);
    if (lane == 0) red_sig[warp] = a;
  }
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    df_acc sa = lane < nw ? red_sig[lane] : acc_zero();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sa.merge(shfl_xor_acc(sa, o));
    const df sigma = sa.value();
    const df x0 = W[(k + 1) * LD + k];
    if (sigma.hi == 0.f) {
      if (tid == 0) {
        tau[k] = df{0.f, 0.f};
        dd[k] = W[k * LD + k];
        ee[k] = x0;
      }
      // partials of the next column, unchanged by this step
      __syncthreads();
      df_acc a = acc_zero();
      for (int i = k + 3 + warp; i < n; i += nw)
        if (lane == 0) a.fma(W[i * LD + k + 1], W[i * LD + k + 1]);
      if (lane == 0) red_sig[warp] = a;
      __syncthreads();
      continue;
    }
    const df nrm = df_sqrt(df_add(df_mul(x0, x0), sigma));
    const df alpha = df_lt0(x0) ? nrm : df_neg(nrm);
    const df v0 = df_sub(x0, alpha);
    const df vtv = df_add(sigma, df_mul(v0, v0));
    const df t = df_div(df{2.f, 0.f}, vtv);
    for (int i = tid; i < m; i += nt) v[i] = (i == 0) ? v0 : W[(k + 1 + i) * LD + k];
    if (tid == 0) {
      tau[k] = t;
      dd[k] = W[k * LD + k];
      ee[k] = alpha;
    }
    __syncthreads();  // (1) v complete
    // p = t * W22 v, and per-warp partials of v^T p; column k keeps v for the back-transformation
    {
      df_acc pv = acc_zero();
      for (int i = warp; i < m; i += nw) {
        df_acc b0 = acc_zero(), b1 = acc_zero();
        const df* row = W + (k + 1 + i) * LD + (k + 1);
        int j = lane;
        for (; j + 32 < m; j += 64) {
          const df r0 = row[j], r1 = row[j + 32];
          const df v0j = v[j], v1j = v[j + 32];
          b0.fma(r0, v0j);
          b1.fma(r1, v1j);
        }
        if (j < m) b0.fma(row[j], v[j]);
        b0.merge(b1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b0.merge(shfl_xor_acc(b0, o));
        if (lane == 0) {
          const df pi = df_mul(t, b0.value());
          p[i] = pi;
          pv.fma(v[i], pi);
        }
      }
      if (lane == 0) red_vp[warp] = pv;
      for (int i = tid; i < m; i += nt) W[(k + 1 + i) * LD + k] = v[i];
      if (hv != nullptr)
        for (int i = tid; i < m; i += nt) hv[static_cast<long long>(k) * n + i] = v[i];
    }
    __syncthreads();  // (2) p and v^T p partials complete
    {
      df_acc c = lane < nw ? red_vp[lane] : acc_zero();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c.merge(shfl_xor_acc(c, o));
      const df kc = df_mul(df_mul_f(t, 0.5f), c.value());
      for (int i = tid; i < m; i += nt) p[i] = df_sub(p[i], df_mul(kc, v[i]));  // w
    }
    __syncthreads();  // (3) w complete
    // W22 -= v w^T + w v^T over whole rows (coalesced; no mirrored column writes):
    // entry (r, c) takes its two products in the order of (max, min), so both
    // triangles stay bitwise equal.  Lane 0 of each row also accumulates the next
    // column's norm (rows 2.. of the trailing block)
    {
      df_acc sg = acc_zero();
      for (int i = warp; i < m; i += nw) {
        const df vi = v[i], wi = p[i];
        df* rowi = W + (k + 1 + i) * LD + (k + 1);
#pragma unroll 2
        for (int j = lane; j < m; j += 32) {
          df_acc u0 = acc_zero();
          if (j <= i) {
            u0.fma(vi, p[j]);
            u0.fma(wi, v[j]);
          } else {
            u0.fma(v[j], wi);
            u0.fma(p[j], vi);
          }
          const df n0 = df_sub(rowi[j], u0.value());
          rowi[j] = n0;
          if (j == 0 && i >= 2) sg.fma(n0, n0);
        }
      }
      if (lane == 0) red_sig[warp] = sg;
    }
    __syncthreads();  // (4) trailing block and next-column partials complete
  }
  if (tid == 0) {
    if (n >= 2) {
      dd[n - 2] = W[(n - 2) * LD + (n - 2)];
      dd[n - 1] = W[(n - 1) * LD + (n - 1)];
      ee[n - 2] = W[(n - 1) * LD + (n - 2)];
      tau[n - 2] = df{0.f, 0.f};
    } else {
      dd[0] = W[0];
    }
    if (n >= 1) tau[n - 1] = df{0.f, 0.f};
  }
  __syncthreads();
}

// Gershgorin interval of the tridiagonal (float32 diagonal sd, squared
// off-diagonal se2), padded, by one thread: sf = {lower, upper, ||T|| bound,
// pivot floor of the Sturm recurrences}.
__device__ void syev_bounds(const float* sd, const float* se2, int n, float* sf) {
  float gl = 3.0e38f, gu = -3.0e38f, emax2 = 0.f;
  for (int i = 0; i < n; ++i) {
    const float r = (i > 0 ? sqrtf(se2[i - 1]) : 0.f) + (i + 1 < n ? sqrtf(se2[i]) : 0.f);
    gl = fminf(gl, sd[i] - r);
    gu = fmaxf(gu, sd[i] + r);
    if (i + 1 < n) emax2 = fmaxf(emax2, se2[i]);
  }
  const float tn = fmaxf(fabsf(gl), fabsf(gu));
  const float pad = 2.0e-6f * tn + 1.0e-30f;
  sf[0] = gl - pad;
  sf[1] = gu + pad;
  sf[2] = tn;
  sf[3] = fmaxf(1.0e-30f, 1.0e-35f * fmaxf(emax2, 1.f));
}

// float32 bisection for the (j+1)-th smallest eigenvalue, one thread.
__device__ float syev_bisect(int j, const float* sd, const float* se2, int n, float gl, float gu, float pivmin) {
  float lo = gl, hi = gu;
  for (int it = 0; it < 80; ++it) {
    const float mid = 0.5f * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(sd, se2, n, mid, pivmin) > j) hi = mid; else lo = mid;
  }
  return 0.5f * (lo + hi);
}

// The same bracket by one warp: 32-point multisection, 33x narrower per round
// (Golub & Van Loan 8.4.1), until the float32 points stop separating.
__device__ float syev_multisect(int j, const float* sd, const float* se2, int n, float gl, float gu, float pivmin) {
  const int lane = threadIdx.x & 31;
  float lo = gl, hi = gu;
  for (int round = 0; round < 40; ++round) {
    const float mid = 0.5f * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    const float x = lo + (hi - lo) * (static_cast<float>(lane + 1) * (1.f / 33.f));
    const unsigned above = __ballot_sync(0xffffffffu, sturm_count(sd, se2, n, x, pivmin) > j);
    const int l1 = above ? __ffs(above) - 1 : 32;  // first point with more than j eigenvalues below
    const float xlo = __shfl_sync(0xffffffffu, x, l1 > 0 ? l1 - 1 : 0);
    const float xhi = __shfl_sync(0xffffffffu, x, l1 < 32 ? l1 : 31);
    if (l1 > 0) lo = fmaxf(lo, xlo);
    if (l1 < 32) hi = fminf(hi, xhi);
  }
  return 0.5f * (lo + hi);
}

// Refine the float32 shift s0 of index j with float-float Sturm counts (one
// warp; ee2 holds e_i^2).  The float32 counts can be off by ~n 2^-24 ||T||,
// far more than the gaps inside a graded spectrum; with float-float shifts the
// inverse iteration separates eigenvalues down to ~1e-9 ||T|| apart on its
// own.  The bracket is first widened until its float-float counts enclose
// index j, then 32-point multisection shrinks it 33x per round.  Returns the
// midpoint of the final bracket (the same on every lane).
__device__ df syev_refine_shift(int j, float s0, const df* dd, const df* ee2, int n, float gl, float gu,
                                float tnorm, float pivmin) {
  const int lane = threadIdx.x & 31;
  float w = 1.0e-4f * tnorm + 1.0e-6f * fabsf(s0) + pivmin;
  df lo = df{s0 - w, 0.f}, hi = df{s0 + w, 0.f};
  for (int attempt = 0; attempt < 12; ++attempt) {
    int c = 0;
    if (lane < 2) c = sturm_count_df(dd, ee2, n, lane == 0 ? lo : hi, pivmin);
    const int clo = __shfl_sync(0xffffffffu, c, 0), chi = __shfl_sync(0xffffffffu, c, 1);
    if (clo <= j && chi > j) break;
    w *= 4.f;
    if (attempt == 11) {
      lo = df{gl, 0.f};
      hi = df{gu, 0.f};
    } else {
      if (clo > j) lo = df{s0 - w, 0.f};
      if (chi <= j) hi = df{s0 + w, 0.f};
    }
  }
  const float tol = 1.0e-14f * tnorm + pivmin;
  for (int round = 0; round < 12; ++round) {
    const df width = df_sub(hi, lo);
    if (!(width.hi > tol)) break;
    const df x = df_add(lo, df_mul_f(width, static_cast<float>(lane + 1) * (1.f / 33.f)));
    const unsigned above = __ballot_sync(0xffffffffu, sturm_count_df(dd, ee2, n, x, pivmin) > j);
    const int l1 = above ? __ffs(above) - 1 : 32;  // first point with more than j eigenvalues below
    const float lhi = __shfl_sync(0xffffffffu, x.hi, l1 > 0 ? l1 - 1 : 0);
    const float llo = __shfl_sync(0xffffffffu, x.lo, l1 > 0 ? l1 - 1 : 0);
    const float hhi = __shfl_sync(0xffffffffu, x.hi, l1 < 32 ? l1 : 31);
    const float hlo = __shfl_sync(0xffffffffu, x.lo, l1 < 32 ? l1 : 31);
    if (l1 > 0) lo = df{lhi, llo};
    if (l1 < 32) hi = df{hhi, hlo};
  }
  return df_mul_f(df_add(lo, hi), 0.5f);
}

// Gap between consecutive refined shifts, compared in float32 against the
// cluster and group thresholds below.
__device__ __forceinline__ float shift_gap(const df* shd, int j) {
  return j > 0 ? df_float(df_sub(shd[j], shd[j - 1])) : 3.0e38f;
}

// Clusters and clean-up groups of the ascending shifts, by one thread.  Shifts
// closer than 1e-9 ||T|| form clusters, iterated in rounds with Gram-Schmidt
// (cpos[j]: position of j in its cluster, which starts at cstart[j]); runs of
// shifts closer than 1e-4 ||T|| form the groups [gs0[j], gs1[j]) of the
// Rayleigh-Ritz clean-up.  si[0] = the largest cluster position, si[1] = 1 if
// any two shifts are closer than 1e-4 ||T||.
__device__ void syev_groups(const df* shd, int nwant, float tnorm, float pivmin, int* cstart, int* cpos, int* gs0,
                            int* gs1, int* si) {
  const float ctol = 1.0e-9f * tnorm + pivmin, rtol = 1.0e-4f * tnorm;
  int maxpos = 0, close = 0, gstart = 0;
  for (int j = 0; j < nwant; ++j) {
    const float gap = shift_gap(shd, j);
    if (gap <= ctol) {
      cstart[j] = cstart[j - 1];
      cpos[j] = cpos[j - 1] + 1;
    } else {
      cstart[j] = j;
      cpos[j] = 0;
    }
    if (gap <= rtol) {
      close = 1;
    } else if (j > 0) {
      for (int i = gstart; i < j; ++i) gs1[i] = j;
      gstart = j;
    }
    gs0[j] = gstart;
    maxpos = max(maxpos, cpos[j]);
  }
  for (int i = gstart; i < nwant; ++i) gs1[i] = nwant;
  si[0] = maxpos;
  si[1] = close;
}

// Inverse iteration in float-float for the shift sg of index j, one thread:
// T - sg I = L D L^T (pivots kept at least pv in magnitude), three solves from
// a fixed start vector, each followed by Gram-Schmidt against the finished
// members c0 .. jj-1 of its cluster and a normalisation.  Element i of the
// vector, of 1/d and of l is at [i ld + jj] of Z, dinv and lm.
__device__ void syev_inverse_iteration(int j, int jj, int c0, df sg, const df* dd, const df* ee, int n, df pv,
                                       df* dinv, df* lm, df* Z, long long ld) {
  df d = df_sub(dd[0], sg);
  if (fabsf(d.hi) < pv.hi) d = df_lt0(d) ? df_neg(pv) : pv;
  df di = df_div(df{1.f, 0.f}, d);
  dinv[jj] = di;
  for (int i = 1; i < n; ++i) {
    const df e = ee[i - 1];
    const df l = df_mul(e, di);
    lm[(i - 1) * ld + jj] = l;
    d = df_sub(df_sub(dd[i], sg), df_mul(l, e));
    if (fabsf(d.hi) < pv.hi) d = df_lt0(d) ? df_neg(pv) : pv;
    di = df_div(df{1.f, 0.f}, d);
    dinv[i * ld + jj] = di;
  }
  // start vector
  for (int i = 0; i < n; ++i) Z[i * ld + jj] = df{1.f + 0.37f * (float)((i * 7 + j * 13) % 11) / 11.f, 0.f};
  for (int it = 0; it < 3; ++it) {
    // L w = x ; z = D^-1 w ; L^T y = z
    df prev = Z[jj];
    for (int i = 1; i < n; ++i) {
      prev = df_sub(Z[i * ld + jj], df_mul(lm[(i - 1) * ld + jj], prev));
      Z[i * ld + jj] = prev;
    }
    df nxt = df_mul(Z[(n - 1) * ld + jj], dinv[(n - 1) * ld + jj]);
    Z[(n - 1) * ld + jj] = nxt;
    for (int i = n - 2; i >= 0; --i) {
      nxt = df_sub(df_mul(Z[i * ld + jj], dinv[i * ld + jj]), df_mul(lm[i * ld + jj], nxt));
      Z[i * ld + jj] = nxt;
    }
    // Gram-Schmidt against finished members of the cluster
    for (int jp = c0; jp < jj; ++jp) {
      df_acc dt = acc_zero();
      for (int i = 0; i < n; ++i) dt.fma(Z[i * ld + jp], Z[i * ld + jj]);
      const df dv = dt.value();
      for (int i = 0; i < n; ++i) Z[i * ld + jj] = df_sub(Z[i * ld + jj], df_mul(dv, Z[i * ld + jp]));
    }
    // normalise (scale first by the largest entry to stay in range)
    float amax = 0.f;
    for (int i = 0; i < n; ++i) amax = fmaxf(amax, fabsf(Z[i * ld + jj].hi));
    const float sc1 = amax > 0.f ? 1.f / amax : 1.f;
    df_acc dn = acc_zero();
    for (int i = 0; i < n; ++i) {
      const df z = df_mul_f(Z[i * ld + jj], sc1);
      Z[i * ld + jj] = z;
      dn.fma(z, z);
    }
    const df inv = df_div(df{1.f, 0.f}, df_sqrt(dn.value()));
    for (int i = 0; i < n; ++i) Z[i * ld + jj] = df_mul(Z[i * ld + jj], inv);
  }
}

// A vector alone in its group, one thread: its Rayleigh quotient with T goes
// to *eval and the vector, normalised, to Zn (element i at [i ldn]).  Z holds
// element i at [i ldz].
__device__ void syev_single(const df* Z, long long ldz, const df* dd, const df* ee, int n, df* Zn, long long ldn,
                            double* eval) {
  df_acc sq = acc_zero(), hq = acc_zero();
  for (int i = 0; i < n; ++i) {
    const df z = Z[i * ldz];
    df_acc tz = acc_zero();
    tz.fma(dd[i], z);
    if (i > 0) tz.fma(ee[i - 1], Z[(i - 1) * ldz]);
    if (i + 1 < n) tz.fma(ee[i], Z[(i + 1) * ldz]);
    sq.fma(z, z);
    hq.fma(z, tz.value());
  }
  const df sv = sq.value();
  const df inv = df_div(df{1.f, 0.f}, df_sqrt(sv));
  for (int i = 0; i < n; ++i) Zn[i * ldn] = df_mul(Z[i * ldz], inv);
  *eval = df_to_double(df_div(hq.value(), sv));
}

// Rayleigh-Ritz clean-up of one group of G >= 2 vectors by the whole block.
// The group's shifts are more than 1e-4 ||T|| from every other group's, so each
// vector's error outside its own group's span is below ~4e-11, and a
// Rayleigh-Ritz step on the span (S = Z_g^T Z_g, Hq = Z_g^T T Z_g) restores
// working accuracy: S = L L^T, C = L^-1 Hq L^-T by parallel cyclic Jacobi,
// vectors Z_g L^-T Q in ascending order.  Column c of the group is at
// Z[i ldz + c] and goes to Zn[i ldn + c], its eigenvalue to evals[c].  rrw:
// 4 G^2 df, perm: G ints, red, sf: block reduction scratch (shared).  TZ: n x G
// df scratch with Z's row stride (T Z, formed once).  TA x TB: the register
// tile of S and Hq per thread.
template <int TA, int TB>
__device__ void syev_group_rr(int G, const df* Z, long long ldz, const df* dd, const df* ee, int n, df* TZ,
                              df* rrw, int* perm, df_acc* red, float* sf, df* Zn, long long ldn, double* evals) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const long long N = n;
  df* S = rrw;
  df* Hq = rrw + G * G;
  df* Qm = rrw + 2 * G * G;
  df* Xm = rrw + 3 * G * G;
  for (int i = warp; i < n; i += nw)
    for (int c = lane; c < G; c += 32) {
      df_acc tz = acc_zero();
      tz.fma(dd[i], Z[i * ldz + c]);
      if (i > 0) tz.fma(ee[i - 1], Z[(i - 1) * ldz + c]);
      if (i + 1 < n) tz.fma(ee[i], Z[(i + 1) * ldz + c]);
      TZ[i * ldz + c] = tz.value();
    }
  __syncthreads();
  // S = Z^T Z and Hq = Z^T (T Z): the upper triangle by TA x TB tiles, one
  // compensated sum per entry over the rows in order; the lower triangle mirrors it
  {
    // tile row ta starts at tile column (ta TA) / TB, the first that reaches the diagonal
    const int na = (G + TA - 1) / TA, nbt = (G + TB - 1) / TB;
    int ntile = 0;
    for (int ta = 0; ta < na; ++ta) ntile += nbt - (ta * TA) / TB;
    for (int tix = tid; tix < ntile; tix += nt) {
      int ta = 0, rem = tix;
      while (rem >= nbt - (ta * TA) / TB) {
        rem -= nbt - (ta * TA) / TB;
        ++ta;
      }
      const int a0 = ta * TA, b0 = ((ta * TA) / TB + rem) * TB;
      df_acc sa[TA][TB], ha[TA][TB];
#pragma unroll
      for (int u = 0; u < TA; ++u)
#pragma unroll
        for (int v = 0; v < TB; ++v) sa[u][v] = ha[u][v] = acc_zero();
      for (int i = 0; i < n; ++i) {
        df za[TA], zb[TB], tb[TB];
#pragma unroll
        for (int u = 0; u < TA; ++u) za[u] = a0 + u < G ? Z[i * ldz + a0 + u] : df{0.f, 0.f};
#pragma unroll
        for (int v = 0; v < TB; ++v) {
          const bool ib = b0 + v < G;
          zb[v] = ib ? Z[i * ldz + b0 + v] : df{0.f, 0.f};
          tb[v] = ib ? TZ[i * ldz + b0 + v] : df{0.f, 0.f};
        }
#pragma unroll
        for (int u = 0; u < TA; ++u)
#pragma unroll
          for (int v = 0; v < TB; ++v) {
            sa[u][v].fma(za[u], zb[v]);
            ha[u][v].fma(za[u], tb[v]);
          }
      }
#pragma unroll
      for (int u = 0; u < TA; ++u)
#pragma unroll
        for (int v = 0; v < TB; ++v) {
          const int a = a0 + u, b = b0 + v;
          if (a <= b && b < G) {
            S[a * G + b] = S[b * G + a] = sa[u][v].value();
            Hq[a * G + b] = Hq[b * G + a] = ha[u][v].value();
          }
        }
    }
  }
  __syncthreads();
  // Cholesky S = L L^T in place (lower), right-looking
  for (int kk = 0; kk < G; ++kk) {
    if (tid == 0) S[kk * G + kk] = df_sqrt(S[kk * G + kk]);
    __syncthreads();
    const df piv = S[kk * G + kk];
    for (int i = kk + 1 + tid; i < G; i += nt) S[i * G + kk] = df_div(S[i * G + kk], piv);
    __syncthreads();
    for (int idx = tid; idx < (G - kk - 1) * (G - kk - 1); idx += nt) {
      const int i = kk + 1 + idx / (G - kk - 1), jj = kk + 1 + idx % (G - kk - 1);
      if (jj <= i) S[i * G + jj] = df_sub(S[i * G + jj], df_mul(S[i * G + kk], S[jj * G + kk]));
    }
    __syncthreads();
  }
  // C = L^-1 Hq L^-T  (two column-parallel forward substitutions; each row's
  // sum over the solved rows in four compensated chains)
  for (int pass = 0; pass < 2; ++pass) {
    df* out = pass == 0 ? Xm : Qm;
    for (int col = tid; col < G; col += nt) {
      for (int i = 0; i < G; ++i) {
        const df rhs = (pass == 0) ? Hq[i * G + col] : Xm[col * G + i];
        const df s = df_sub(rhs, dot4(S + i * G, 1, out + col, G, i).value());
        out[i * G + col] = df_div(s, S[i * G + i]);
      }
    }
    __syncthreads();
  }
  // Qm now holds C (symmetric); move it to Hq and set Qm = I
  for (int idx = tid; idx < G * G; idx += nt) {
    const int a0 = idx / G, b0 = idx % G;
    const df cab = Qm[a0 * G + b0], cba = Qm[b0 * G + a0];
    Hq[idx] = df_mul_f(df_add(cab, cba), 0.5f);
  }
  __syncthreads();
  for (int idx = tid; idx < G * G; idx += nt) Qm[idx] = df{(idx / G == idx % G) ? 1.f : 0.f, 0.f};
  __syncthreads();
  // parallel cyclic Jacobi (round-robin pairing) on C, accumulating Q
  {
    const int np = (G + 1) & ~1;  // even player count; index G is a dummy
    for (int sweep = 0; sweep < 12; ++sweep) {
      // convergence test: largest off-diagonal entry against the largest diagonal one
      float off = 0.f, dia = 0.f;
      for (int idx = tid; idx < G * G; idx += nt) {
        const int a0 = idx / G, b0 = idx % G;
        const float x = fabsf(Hq[idx].hi);
        if (a0 == b0) dia = fmaxf(dia, x); else off = fmaxf(off, x);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        off = fmaxf(off, __shfl_xor_sync(0xffffffffu, off, o));
        dia = fmaxf(dia, __shfl_xor_sync(0xffffffffu, dia, o));
      }
      if (lane == 0) {
        red[warp].s = off;
        red[warp].c = dia;
      }
      __syncthreads();
      if (tid == 0) {
        float o2 = 0.f, d2 = 0.f;
        for (int w2 = 0; w2 < nw; ++w2) {
          o2 = fmaxf(o2, red[w2].s);
          d2 = fmaxf(d2, red[w2].c);
        }
        sf[0] = o2;
        sf[1] = d2;
      }
      __syncthreads();
      const float offmax = sf[0], diamax = sf[1];
      __syncthreads();
      if (!(offmax > 1.0e-15f * fmaxf(diamax, 1.0e-30f))) break;
      for (int r = 0; r < np - 1; ++r) {
        // pair t: players (a, b) of the round-robin schedule
        for (int t = tid; t < np / 2; t += nt) {
          int a0 = (t == 0) ? 0 : 1 + (t - 1 + r) % (np - 1);
          int b0 = 1 + (np - 2 - t + r) % (np - 1);
          if (a0 > b0) {
            const int tmpi = a0;
            a0 = b0;
            b0 = tmpi;
          }
          df cs = df{1.f, 0.f}, sn = df{0.f, 0.f};
          if (b0 < G) {
            const df apq = Hq[a0 * G + b0];
            const df app = Hq[a0 * G + a0], aqq = Hq[b0 * G + b0];
            // skip entries already below the float-float resolution of the diagonal
            const float thr = 1.0e-17f * (sqrtf(fabsf(app.hi)) * sqrtf(fabsf(aqq.hi))) + 1.0e-37f;
            if (fabsf(apq.hi) > thr) {
              // theta = (aqq - app) / (2 apq); t = sign(theta) / (|theta| + sqrt(theta^2 + 1)),
              // and t = 1 / (2 theta) once theta^2 would leave the float range
              const df th = df_div(df_sub(aqq, app), df_mul_f(apq, 2.f));
              df tt;
              if (fabsf(th.hi) > 1.0e12f) {
                tt = df_div(df{0.5f, 0.f}, th);
              } else {
                const df rt = df_sqrt(df_add(df_mul(th, th), df{1.f, 0.f}));
                tt = df_div(df{1.f, 0.f}, df_add(df_abs(th), rt));
                if (df_lt0(th)) tt = df_neg(tt);
              }
              cs = df_div(df{1.f, 0.f}, df_sqrt(df_add(df_mul(tt, tt), df{1.f, 0.f})));
              sn = df_mul(tt, cs);
            }
          }
          // stash rotation in Xm row 0..np/2 (cols 0..3)
          Xm[t * 4 + 0] = cs;
          Xm[t * 4 + 1] = sn;
          reinterpret_cast<int*>(&Xm[t * 4 + 2])[0] = a0;
          reinterpret_cast<int*>(&Xm[t * 4 + 3])[0] = b0;
        }
        __syncthreads();
        // C <- J^T C J by 2 x 2 blocks (pair s, pair t), s <= t, the lower
        // triangle mirrored; the rows of each block turn first, then its columns.
        // The triangle of pair blocks is folded (row s with row P - 1 - s) so
        // that every thread gets the same share.  Q <- Q J alongside.
        {
          const int P = np / 2, half = (P + 1) / 2;
          for (int idx = tid; idx < half * (P + 1); idx += nt) {
            const int fr = idx / (P + 1), cc = idx - fr * (P + 1);
            int ps, pt;
            if (cc < P - fr) {
              ps = fr;
              pt = fr + cc;
            } else {
              ps = P - 1 - fr;
              if (ps == fr) continue;
              pt = ps + (cc - (P - fr));
            }
            const int as = reinterpret_cast<const int*>(&Xm[ps * 4 + 2])[0];
            const int bs = reinterpret_cast<const int*>(&Xm[ps * 4 + 3])[0];
            const int at = reinterpret_cast<const int*>(&Xm[pt * 4 + 2])[0];
            const int bt = reinterpret_cast<const int*>(&Xm[pt * 4 + 3])[0];
            const df css = Xm[ps * 4 + 0], sns = Xm[ps * 4 + 1];
            const df cst = Xm[pt * 4 + 0], snt = Xm[pt * 4 + 1];
            const bool rs = bs < G, rt = bt < G;
            const df zero = df{0.f, 0.f};
            df x00 = Hq[as * G + at], x01 = rt ? Hq[as * G + bt] : zero;
            df x10 = rs ? Hq[bs * G + at] : zero, x11 = (rs && rt) ? Hq[bs * G + bt] : zero;
            if (rs) {
              const df y00 = df_sub(df_mul(css, x00), df_mul(sns, x10));
              const df y10 = df_add(df_mul(sns, x00), df_mul(css, x10));
              const df y01 = df_sub(df_mul(css, x01), df_mul(sns, x11));
              const df y11 = df_add(df_mul(sns, x01), df_mul(css, x11));
              x00 = y00;
              x10 = y10;
              x01 = y01;
              x11 = y11;
            }
            if (rt) {
              const df y00 = df_sub(df_mul(cst, x00), df_mul(snt, x01));
              const df y01 = df_add(df_mul(snt, x00), df_mul(cst, x01));
              const df y10 = df_sub(df_mul(cst, x10), df_mul(snt, x11));
              const df y11 = df_add(df_mul(snt, x10), df_mul(cst, x11));
              x00 = y00;
              x01 = y01;
              x10 = y10;
              x11 = y11;
            }
            if (ps == pt) {
              // diagonal block: (as, bs) and (bs, as) take the same value
              Hq[as * G + as] = x00;
              if (rs) {
                Hq[as * G + bs] = Hq[bs * G + as] = x01;
                Hq[bs * G + bs] = x11;
              }
            } else {
              Hq[as * G + at] = Hq[at * G + as] = x00;
              if (rt) Hq[as * G + bt] = Hq[bt * G + as] = x01;
              if (rs) Hq[bs * G + at] = Hq[at * G + bs] = x10;
              if (rs && rt) Hq[bs * G + bt] = Hq[bt * G + bs] = x11;
            }
          }
          for (int t = warp; t < P; t += nw) {
            const int a0 = reinterpret_cast<const int*>(&Xm[t * 4 + 2])[0];
            const int b0 = reinterpret_cast<const int*>(&Xm[t * 4 + 3])[0];
            if (b0 >= G) continue;
            const df cs = Xm[t * 4 + 0], sn = Xm[t * 4 + 1];
            for (int row = lane; row < G; row += 32) {
              const df x = Qm[row * G + a0], y = Qm[row * G + b0];
              Qm[row * G + a0] = df_sub(df_mul(cs, x), df_mul(sn, y));
              Qm[row * G + b0] = df_add(df_mul(sn, x), df_mul(cs, y));
            }
          }
        }
        __syncthreads();
      }
    }
  }
  // order eigenvalues ascending (selection by rank; ties broken by index)
  for (int j = tid; j < G; j += nt) {
    const df lj = Hq[j * G + j];
    int rank = 0;
    for (int i = 0; i < G; ++i) {
      const df li = Hq[i * G + i];
      const df dlt = df_sub(li, lj);
      if (df_lt0(dlt) || ((dlt.hi == 0.f && dlt.lo == 0.f) && i < j)) ++rank;
    }
    perm[rank] = j;
  }
  __syncthreads();
  // Xm = L^-T Q  (back substitution per column)
  for (int col = tid; col < G; col += nt) {
    for (int i = G - 1; i >= 0; --i) {
      const df s = df_sub(Qm[i * G + col], dot4(S + (i + 1) * G + i, G, Xm + (i + 1) * G + col, G, G - 1 - i).value());
      Xm[i * G + col] = df_div(s, S[i * G + i]);
    }
  }
  __syncthreads();
  // group eigenvectors Zn[:, c] = Z_g Xm[:, perm[c]] (ascending within the group)
  for (long long idx = tid; idx < N * G; idx += nt) {
    const int i = static_cast<int>(idx / G), c = static_cast<int>(idx % G);
    const int src = perm[c];
    df_acc sa = acc_zero();
    for (int kk = 0; kk < G; ++kk) sa.fma(Z[i * ldz + kk], Xm[kk * G + src]);
    Zn[i * ldn + c] = sa.value();
  }
  for (int c = tid; c < G; c += nt) evals[c] = df_to_double(Hq[perm[c] * G + perm[c]]);
  __syncthreads();
}

// ---- one-block driver
//
// Dynamic shared memory: v, p (df, n each), sd, se2 (float, n each), shift
// (float, nwant), cstart, cpos (int, nwant), d, e, tau, e^2 (df, n each),
// shifts (df, nwant), gs0, gs1 (int, nwant), then -- when they fit -- the
// working matrix W (n x ldw df), the inverse-iteration factors (2 x n x nwant
// df) and the tridiagonal eigenvectors Zt (n x nwant df).  `flags` bit 0/1/2
// says which of W / factors / Zt live in shared memory; the others use the
// global workspace (same layout), so one code path serves every size.
constexpr int kSyW = 1, kSyF = 2, kSyZ = 4;

__global__ void __launch_bounds__(kSyThreads) k_syev_df(int n, int nwant, int ldw, int flags,
                                                        const double* __restrict__ H, double* __restrict__ evals,
                                                        double* __restrict__ evecs, df* __restrict__ Wg,
                                                        df* __restrict__ tau_g, df* __restrict__ dd_g,
                                                        df* __restrict__ ee_g, df* __restrict__ facg,
                                                        df* __restrict__ Ztg, df* __restrict__ rrw,
                                                        int* __restrict__ perm, const int* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;  // the structured fast path already produced the pairs
  extern __shared__ __align__(16) unsigned char smem_raw[];
  df* v = reinterpret_cast<df*>(smem_raw);
  df* p = v + n;
  float* sd = reinterpret_cast<float*>(p + n);
  float* se2 = sd + n;
  float* shift = se2 + n;
  int* cstart = reinterpret_cast<int*>(shift + nwant);
  int* cpos = cstart + nwant;
  size_t off = (2 * sizeof(df) * n + 2 * sizeof(float) * n + sizeof(float) * nwant + 2 * sizeof(int) * nwant +
                4 * sizeof(df) * n + sizeof(df) * nwant + 2 * sizeof(int) * nwant + 15) &
               ~static_cast<size_t>(15);
  df* W = Wg;
  if (flags & kSyW) {
    W = reinterpret_cast<df*>(smem_raw + off);
    off += sizeof(df) * static_cast<size_t>(n) * ldw;
  }
  df* fac = facg;
  if (flags & kSyF) {
    fac = reinterpret_cast<df*>(smem_raw + off);
    off += sizeof(df) * 2 * static_cast<size_t>(n) * nwant;
  }
  df* Zt = Ztg;
  if (flags & kSyZ) Zt = reinterpret_cast<df*>(smem_raw + off);
  __shared__ df_acc red[32];
  __shared__ float sf[4];
  __shared__ int si[4];

  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const long long N = n, LD = ldw;
  // the tridiagonal (d, e) and the Householder scalars live in shared memory
  df* dd = reinterpret_cast<df*>(cpos + nwant);
  df* ee = dd + n;
  df* tau = ee + n;
  df* ee2 = tau + n;     // e_i^2 in float-float (Sturm counts)
  df* shd = ee2 + n;     // float-float shifts (nwant)
  int* gs0 = reinterpret_cast<int*>(shd + nwant);  // clean-up group [gs0[j], gs1[j]) of index j
  int* gs1 = gs0 + nwant;
  __shared__ df_acc red_sig[32], red_vp[32];

  for (long long i = tid; i < N * N; i += nt) W[(i / N) * LD + (i % N)] = df_from_double(H[i]);
  __syncthreads();
  syev_tridiagonalise(n, W, LD, v, p, dd, ee, tau, red_sig, red_vp, nullptr);

  // ---- bisection (float32) for the nwant smallest eigenvalues, refined in float-float
  for (int i = tid; i < n; i += nt) {
    sd[i] = df_float(dd[i]);
    if (i + 1 < n) {
      const float e = df_float(ee[i]);
      se2[i] = e * e;
    }
  }
  __syncthreads();
  if (tid == 0) syev_bounds(sd, se2, n, sf);
  __syncthreads();
  const float gl = sf[0], gu = sf[1], tnorm = sf[2], pivmin = sf[3];
  for (int j = tid; j < nwant; j += nt) shift[j] = syev_bisect(j, sd, se2, n, gl, gu, pivmin);
  for (int i = tid; i + 1 < n; i += nt) ee2[i] = df_mul(ee[i], ee[i]);
  __syncthreads();
  for (int j = warp; j < nwant; j += nw) {
    const df s = syev_refine_shift(j, shift[j], dd, ee2, n, gl, gu, tnorm, pivmin);
    if (lane == 0) shd[j] = s;
  }
  __syncthreads();
  if (tid == 0) syev_groups(shd, nwant, tnorm, pivmin, cstart, cpos, gs0, gs1, si);
  __syncthreads();
  const int maxpos = si[0];
  const bool cleanup = si[1] != 0;

  // ---- inverse iteration in float-float: T - s I = L D L^T -----------------
  // factor arrays (element i of eigen-index j at [i * nwant + j]):
  //   fac[0 .. n*nwant) = 1/d_i, fac[n*nwant .. 2n*nwant) = l_i
  const long long NW = nwant;
  const df pv = df{fmaxf(3.6e-15f * tnorm, 1.0e-30f), 0.f};
  for (int round = 0; round <= maxpos; ++round) {
    for (int j = tid; j < nwant; j += nt) {
      if (cpos[j] != round) continue;
      syev_inverse_iteration(j, j, cstart[j], shd[j], dd, ee, n, pv, fac, fac + N * NW, Zt, NW);
    }
    __syncthreads();
  }

  df* Zn = fac;
  if (!cleanup) {
    // every gap is above 1e-4 ||T||: the vectors are accurate individually
    // (error ~ 48-bit rounding x ||T|| / gap <= 4e-11); their Rayleigh
    // quotients are the eigenvalues, already in ascending order
    for (long long idx = tid; idx < N * NW; idx += nt) Zn[idx] = Zt[idx];
    for (int j = tid; j < nwant; j += nt) {
      df_acc h = acc_zero();
      for (int i = 0; i < n; ++i) {
        df_acc tz = acc_zero();
        tz.fma(dd[i], Zt[i * NW + j]);
        if (i > 0) tz.fma(ee[i - 1], Zt[(i - 1) * NW + j]);
        if (i + 1 < n) tz.fma(ee[i], Zt[(i + 1) * NW + j]);
        h.fma(Zt[i * NW + j], tz.value());
      }
      evals[j] = df_to_double(h.value());
    }
    __syncthreads();
  } else {
    // single vectors only need their Rayleigh quotient; the groups of two or
    // more run one after another on windows of the workspace
    for (int j = tid; j < nwant; j += nt) {
      if (gs1[j] - gs0[j] != 1) continue;
      syev_single(Zt + j, NW, dd, ee, n, Zn + j, NW, evals + j);
    }
    __syncthreads();
    for (int g0 = 0; g0 < nwant;) {
      const int g1 = gs1[g0], G = g1 - g0;
      if (G >= 2)
        syev_group_rr<2, 2>(G, Zt + g0, NW, dd, ee, n, fac + N * NW + g0, rrw, perm, red, sf, Zn + g0, NW,
                            evals + g0);
      g0 = g1;
    }
  }

  // ---- back-transformation y = H_0 H_1 ... H_{n-3} z ------------------------
  // v_k (column k of W below the diagonal) is staged in shared memory once per
  // step.  Each column of Z is split over S consecutive lanes (S = 1..8 threads
  // per column, as many as the block holds): lane seg takes rows seg, seg + S, ...,
  // the partial products meet in a shuffle tree, and the same lanes apply the
  // update -- row walks stay coalesced across columns and each chain is m / S long.
  int S = 1;
  while (S < 8 && 2 * S * nwant <= nt) S <<= 1;
  for (int k = n - 3; k >= 0; --k) {
    const df t = tau[k];
    if (t.hi == 0.f) continue;
    const int m = n - k - 1;
    for (int i = tid; i < m; i += nt) v[i] = W[(k + 1 + i) * LD + k];
    __syncthreads();
    // for each column c: s_c = v^T z[k+1:, c]; z[k+1:, c] -= t s_c v
    const int total = nwant * S;
    for (int base = warp * 32; base < total; base += nt) {
      const int it = base + lane;
      const bool valid = it < total;
      const int c = valid ? it / S : 0, seg = it % S;
      df* zc = Zn + static_cast<long long>(k + 1) * NW + c;
      df_acc s0 = acc_zero(), s1 = acc_zero(), s2 = acc_zero(), s3 = acc_zero();
      if (valid) {
        int i = seg;
        for (; i + 3 * S < m; i += 4 * S) {
          s0.fma(v[i], zc[i * NW]);
          s1.fma(v[i + S], zc[(i + S) * NW]);
          s2.fma(v[i + 2 * S], zc[(i + 2 * S) * NW]);
          s3.fma(v[i + 3 * S], zc[(i + 3 * S) * NW]);
        }
        for (; i < m; i += S) s0.fma(v[i], zc[i * NW]);
      }
      s0.merge(s1);
      s2.merge(s3);
      s0.merge(s2);
      for (int o = 1; o < S; o <<= 1) s0.merge(shfl_xor_acc(s0, o));
      if (valid) {
        const df f = df_mul(t, s0.value());
        for (int i = seg; i < m; i += S) zc[i * NW] = df_sub(zc[i * NW], df_mul(f, v[i]));
      }
    }
    __syncthreads();
  }
  for (long long idx = tid; idx < N * NW; idx += nt) evecs[idx] = df_to_double(Zn[idx]);
}

// ---- split driver
//
// Global workspace: W (n x ldw df) unless it fits in shared memory, the
// reflectors hv (v_k at hv[k n ..]), dd, ee, tau (df, n each), the shifts shd
// (df, nwant) and their bounds (4 floats), the factors and working vectors of
// groups too wide for shared memory (fac: 3 n nwant df) and the tridiagonal
// eigenvectors Zg (n x nwant df).
constexpr int kSvWarps = 4;  // shifts per block of k_syev_vals
constexpr int kSvecThreads = 512;
constexpr int kSbWarps = 8;  // eigenvectors per block of k_syev_back
constexpr int kSbChunk = 8;  // reflectors staged per barrier in k_syev_back

// Tridiagonalisation, one block: W in shared memory when `inshared`, else the
// global Wg.  Writes dd, ee, tau and the reflectors hv to global memory.
__global__ void __launch_bounds__(kSyThreads) k_syev_tri(int n, int ldw, int inshared, const double* __restrict__ H,
                                                         df* __restrict__ Wg, df* __restrict__ hv,
                                                         df* __restrict__ dd_g, df* __restrict__ ee_g,
                                                         df* __restrict__ tau_g, const int* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  df* v = reinterpret_cast<df*>(smem_raw);
  df* p = v + n;
  df* dd = p + n;
  df* ee = dd + n;
  df* tau = ee + n;
  const size_t off = (5 * sizeof(df) * static_cast<size_t>(n) + 15) & ~static_cast<size_t>(15);
  df* W = inshared ? reinterpret_cast<df*>(smem_raw + off) : Wg;
  __shared__ df_acc red_sig[32], red_vp[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long N = n, LD = ldw;
  for (long long i = tid; i < N * N; i += nt) W[(i / N) * LD + (i % N)] = df_from_double(H[i]);
  __syncthreads();
  syev_tridiagonalise(n, W, LD, v, p, dd, ee, tau, red_sig, red_vp, hv);
  for (int i = tid; i < n; i += nt) {
    dd_g[i] = dd[i];
    tau_g[i] = tau[i];
    if (i + 1 < n) ee_g[i] = ee[i];
  }
}

// The same tridiagonalisation by a thread-block cluster of CS CTAs (2, 4 or 8)
// when W is too large for one block's shared memory: CTA r keeps rows
// r R .. r R + R - 1 of W (full rows, stride ldw) in its own shared memory.
// Per step k the owners of column k's entries below the diagonal write them,
// with their partial sums of squares, into every CTA's copy of v (distributed
// shared memory); after a cluster barrier every CTA forms the same reflector
// from the same partials (merged in rank order), computes p = t W22 v for its
// own rows and sends them, with its partial v^T p, to every CTA; after a
// second barrier each CTA forms w = p - (t/2)(v^T p) v and updates its own rows
// (both triangles in the (max, min) product order, so W stays bitwise
// symmetric).  v, p and the partials are double-buffered by the parity of k:
// a CTA that reaches step k + 1 writes buffers that no CTA still reads.
constexpr int kTriMaxCluster = 8;

__device__ __forceinline__ df_acc block_merge(df_acc a, df_acc* red) {
  // every thread's partial merged: warps by shuffles, then warp 0 over the warps (result in lane 0 of warp 0)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a.merge(shfl_xor_acc(a, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) red[warp] = a;
  __syncthreads();
  df_acc b = acc_zero();
  if (warp == 0) {
    b = lane < nw ? red[lane] : acc_zero();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b.merge(shfl_xor_acc(b, o));
  }
  __syncthreads();
  return b;
}

__global__ void __launch_bounds__(kSyThreads) k_syev_tri_cl(int n, int ldw, int R, const double* __restrict__ H,
                                                            df* __restrict__ hv, df* __restrict__ dd_g,
                                                            df* __restrict__ ee_g, df* __restrict__ tau_g,
                                                            const int* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;  // every CTA of the cluster returns here alike
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int CS = static_cast<int>(cl.num_blocks()), rank = static_cast<int>(cl.block_rank());
  extern __shared__ __align__(16) unsigned char smem_raw[];
  df* W = reinterpret_cast<df*>(smem_raw);  // R x ldw: rows r0 .. r1-1
  df* vb = W + static_cast<long long>(R) * ldw;  // 2 x n
  df* pb = vb + 2 * n;                            // 2 x n
  __shared__ df_acc sigp[2][kTriMaxCluster], vpp[2][kTriMaxCluster], red[32];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int r0 = rank * R, r1 = min(n, r0 + R);
  const long long LD = ldw;
  for (long long idx = tid; idx < static_cast<long long>(r1 - r0) * n; idx += nt) {
    const int i = static_cast<int>(idx / n), j = static_cast<int>(idx % n);
    W[i * LD + j] = df_from_double(H[static_cast<long long>(r0 + i) * n + j]);
  }
  __syncthreads();
  // column c's entries below the diagonal (own rows) into every CTA's v buffer, and
  // the partial sum of squares of rows c + 2 .. into every CTA's partials
  auto send_column = [&](int c) {
    const int buf = c & 1;
    df_acc a = acc_zero();
    for (int i = max(r0, c + 1) + tid; i < r1; i += nt) {
      const df x = W[(i - r0) * LD + c];
      for (int r = 0; r < CS; ++r) cl.map_shared_rank(vb + buf * n, r)[i - c - 1] = x;
      if (i >= c + 2) a.fma(x, x);
    }
    const df_acc s = block_merge(a, red);
    if (tid == 0)
      for (int r = 0; r < CS; ++r) cl.map_shared_rank(&sigp[buf][0], r)[rank] = s;
  };
  send_column(0);
  for (int k = 0; k + 2 < n; ++k) {
    const int buf = k & 1, m = n - k - 1;
    cl.sync();  // (1) column k and its partials are everywhere
    df_acc sa = sigp[buf][0];
    for (int r = 1; r < CS; ++r) sa.merge(sigp[buf][r]);
    const df sigma = sa.value();
    df* v = vb + buf * n;
    df* p = pb + buf * n;
    const df x0 = v[0];
    const bool own_k = k >= r0 && k < r1;
    if (sigma.hi == 0.f) {
      if (own_k) {
        if (tid == 0) {
          tau_g[k] = df{0.f, 0.f};
          dd_g[k] = W[(k - r0) * LD + k];
          ee_g[k] = x0;
        }
      }
      cl.sync();  // (2) the same barrier count as a reflecting step
      send_column(k + 1);
      continue;
    }
    const df nrm = df_sqrt(df_add(df_mul(x0, x0), sigma));
    const df alpha = df_lt0(x0) ? nrm : df_neg(nrm);
    const df v0 = df_sub(x0, alpha);
    const df vtv = df_add(sigma, df_mul(v0, v0));
    const df t = df_div(df{2.f, 0.f}, vtv);
    __syncthreads();  // every thread has read v[0]
    if (tid == 0) {
      v[0] = v0;
      if (own_k) {
        tau_g[k] = t;
        dd_g[k] = W[(k - r0) * LD + k];
        ee_g[k] = alpha;
      }
    }
    __syncthreads();
    if (rank == 0)
      for (int i = tid; i < m; i += nt) hv[static_cast<long long>(k) * n + i] = v[i];
    // p_i = t (W22 v)_i for the own trailing rows, one warp per row; partial v^T p
    {
      df_acc pv = acc_zero();
      for (int i = max(r0, k + 1) + warp; i < r1; i += nw) {
        const df* row = W + (i - r0) * LD + (k + 1);
        df_acc b0 = acc_zero(), b1 = acc_zero();
        int j = lane;
        for (; j + 32 < m; j += 64) {
          b0.fma(row[j], v[j]);
          b1.fma(row[j + 32], v[j + 32]);
        }
        if (j < m) b0.fma(row[j], v[j]);
        b0.merge(b1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b0.merge(shfl_xor_acc(b0, o));
        if (lane == 0) {
          const df pi = df_mul(t, b0.value());
          for (int r = 0; r < CS; ++r) cl.map_shared_rank(pb + buf * n, r)[i - k - 1] = pi;
          pv.fma(v[i - k - 1], pi);
        }
      }
      const df_acc s = block_merge(pv, red);
      if (tid == 0)
        for (int r = 0; r < CS; ++r) cl.map_shared_rank(&vpp[buf][0], r)[rank] = s;
    }
    cl.sync();  // (2) every p_i and partial v^T p are everywhere
    {
      df_acc c = vpp[buf][0];
      for (int r = 1; r < CS; ++r) c.merge(vpp[buf][r]);
      const df kc = df_mul(df_mul_f(t, 0.5f), c.value());
      for (int i = tid; i < m; i += nt) p[i] = df_sub(p[i], df_mul(kc, v[i]));  // w
    }
    __syncthreads();
    // own rows: W22 -= v w^T + w v^T, one warp per row, lanes along it (column k keeps
    // the entries of the reduced matrix)
    for (int row = max(r0, k + 1) + warp; row < r1; row += nw) {
      const int i = row - k - 1;  // trailing index of the row
      const df vi = v[i], wi = p[i];
      df* rowp = W + (row - r0) * LD + (k + 1);
#pragma unroll 2
      for (int j = lane; j < m; j += 32) {
        df_acc u0 = acc_zero();
        if (j <= i) {
          u0.fma(vi, p[j]);
          u0.fma(wi, v[j]);
        } else {
          u0.fma(v[j], wi);
          u0.fma(p[j], vi);
        }
        rowp[j] = df_sub(rowp[j], u0.value());
      }
    }
    __syncthreads();
    send_column(k + 1);
  }
  // the last 2 x 2 block
  if (tid == 0) {
    if (n >= 2) {
      if (n - 2 >= r0 && n - 2 < r1) dd_g[n - 2] = W[(n - 2 - r0) * LD + (n - 2)];
      if (n - 1 >= r0 && n - 1 < r1) {
        dd_g[n - 1] = W[(n - 1 - r0) * LD + (n - 1)];
        ee_g[n - 2] = W[(n - 1 - r0) * LD + (n - 2)];
      }
      if (rank == 0) tau_g[n - 2] = df{0.f, 0.f};
    } else if (rank == 0) {
      dd_g[0] = W[0];
    }
    if (rank == 0 && n >= 1) tau_g[n - 1] = df{0.f, 0.f};
  }
  cl.sync();  // no CTA leaves while another may still write into its shared memory
}

// The refined shifts, one warp each (kSvWarps per block): float32 multisection
// then float-float refinement.  Block 0 also writes the bounds.  Shared: dd,
// ee2 (df, n each), sd, se2 (float, n each).
__global__ void __launch_bounds__(32 * kSvWarps) k_syev_vals(int n, int nwant, const df* __restrict__ dd_g,
                                                             const df* __restrict__ ee_g, df* __restrict__ shd,
                                                             float* __restrict__ bounds,
                                                             const int* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  df* dd = reinterpret_cast<df*>(smem_raw);
  df* ee2 = dd + n;
  float* sd = reinterpret_cast<float*>(ee2 + n);
  float* se2 = sd + n;
  __shared__ float sf[4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += blockDim.x) {
    const df d = dd_g[i];
    dd[i] = d;
    sd[i] = df_float(d);
    if (i + 1 < n) {
      const df e = ee_g[i];
      const float ef = df_float(e);
      se2[i] = ef * ef;
      ee2[i] = df_mul(e, e);
    }
  }
  __syncthreads();
  if (tid == 0) syev_bounds(sd, se2, n, sf);
  __syncthreads();
  if (blockIdx.x == 0 && tid < 4) bounds[tid] = sf[tid];
  const int j = blockIdx.x * kSvWarps + warp;
  if (j >= nwant) return;  // whole warps: no block barrier below
  const float gl = sf[0], gu = sf[1], tnorm = sf[2], pivmin = sf[3];
  const float s0 = syev_multisect(j, sd, se2, n, gl, gu, pivmin);
  const df s = syev_refine_shift(j, s0, dd, ee2, n, gl, gu, tnorm, pivmin);
  if (lane == 0) shd[j] = s;
}

// Bytes of shared memory k_syev_vecs keeps for a group of G vectors: d, e
// (2n df), cluster data (2G ints), perm (G ints), and -- in shared memory when
// they fit -- the factors and vectors (3 n G df) and the clean-up matrices (4 G^2 df).
__host__ __device__ inline size_t syev_vecs_base(int n, int G) {
  return (2 * sizeof(df) * static_cast<size_t>(n) + 3 * sizeof(int) * static_cast<size_t>(G) + 15) &
         ~static_cast<size_t>(15);
}
__host__ __device__ inline size_t syev_vecs_work(int n, int G) {
  return sizeof(df) * (3 * static_cast<size_t>(n) * G + 4 * static_cast<size_t>(G) * G);
}

// Inverse iteration and clean-up, one block per group of close shifts: block b
// takes the group that starts at index b (the others exit at once).  A group's
// clusters lie inside it (1e-9 ||T|| < 1e-4 ||T||), so every block runs alone.
// Writes the tridiagonal eigenvectors Zg (n x nwant) and the eigenvalues.
__global__ void __launch_bounds__(kSvecThreads) k_syev_vecs(int n, int nwant, size_t smem_bytes,
                                                            const df* __restrict__ dd_g, const df* __restrict__ ee_g,
                                                            const df* __restrict__ shd, const float* __restrict__ bounds,
                                                            df* __restrict__ facg, df* __restrict__ rrg,
                                                            df* __restrict__ Zg, double* __restrict__ evals,
                                                            const int* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  const float tnorm = bounds[2], pivmin = bounds[3];
  const float ctol = 1.0e-9f * tnorm + pivmin, rtol = 1.0e-4f * tnorm;
  const int b = blockIdx.x;
  if (b > 0 && shift_gap(shd, b) <= rtol) return;  // not the first index of a group
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ df_acc red[32];
  __shared__ float sf[4];
  __shared__ int sg[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    int g1 = b + 1;
    while (g1 < nwant && shift_gap(shd, g1) <= rtol) ++g1;
    sg[0] = g1 - b;
  }
  __syncthreads();
  const int G = sg[0];
  df* dd = reinterpret_cast<df*>(smem_raw);
  df* ee = dd + n;
  int* cst = reinterpret_cast<int*>(ee + n);  // cluster start, local index
  int* cps = cst + G;                         // position in the cluster
  int* perm = cps + G;
  for (int i = tid; i < n; i += nt) {
    dd[i] = dd_g[i];
    if (i + 1 < n) ee[i] = ee_g[i];
  }
  if (tid == 0) {
    int maxpos = 0;
    for (int jj = 0; jj < G; ++jj) {
      if (jj == 0 || !(shift_gap(shd, b + jj) <= ctol)) {
        cst[jj] = jj;
        cps[jj] = 0;
      } else {
        cst[jj] = cst[jj - 1];
        cps[jj] = cps[jj - 1] + 1;
      }
      maxpos = max(maxpos, cps[jj]);
    }
    sg[1] = maxpos;
  }
  __syncthreads();
  const int maxpos = sg[1];
  const long long N = n, NW = nwant;
  // working storage: shared memory when the group fits, else its columns of the global workspace
  const size_t base = syev_vecs_base(n, G);
  const bool local = base + syev_vecs_work(n, G) <= smem_bytes;
  df *dinv, *lm, *Z, *rrw;
  long long ld;
  if (local) {
    dinv = reinterpret_cast<df*>(smem_raw + base);
    lm = dinv + N * G;
    Z = lm + N * G;
    rrw = Z + N * G;
    ld = G;
  } else {
    dinv = facg + b;
    lm = facg + N * NW + b;
    Z = facg + 2 * N * NW + b;
    rrw = rrg + 4LL * b * NW;  // 4 G^2 <= 4 NW (NW - b): the groups' windows do not overlap
    ld = NW;
  }
  const df pv = df{fmaxf(3.6e-15f * tnorm, 1.0e-30f), 0.f};
  for (int round = 0; round <= maxpos; ++round) {
    for (int jj = tid; jj < G; jj += nt)
      if (cps[jj] == round) syev_inverse_iteration(b + jj, jj, cst[jj], shd[b + jj], dd, ee, n, pv, dinv, lm, Z, ld);
    __syncthreads();
  }
  if (G == 1) {
    if (tid == 0) syev_single(Z, ld, dd, ee, n, Zg + b, NW, evals + b);
  } else {
    syev_group_rr<4, 2>(G, Z, ld, dd, ee, n, dinv, rrw, perm, red, sf, Zg + b, NW, evals + b);
  }
}

// Back-transformation y = H_0 H_1 ... H_{n-3} z, one warp per eigenvector
// (column c of Zg), held in shared memory; the block stages kSbChunk
// reflectors at a time (chunk = reflectors k0, k0 - 1, ...) and each warp then
// applies them to its own column without further barriers.  Writes evecs
// (n x nwant float64).
__global__ void __launch_bounds__(32 * kSbWarps) k_syev_back(int n, int nwant, int chunk, const df* __restrict__ hv,
                                                             const df* __restrict__ tau_g,
                                                             const df* __restrict__ Zg, double* __restrict__ evecs,
                                                             const int* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, wpb = blockDim.x >> 5;
  const long long NW = nwant;
  df* zs = reinterpret_cast<df*>(smem_raw);  // wpb x n
  df* vs = zs + static_cast<long long>(wpb) * n;  // chunk x n
  const int c = blockIdx.x * wpb + warp;
  const bool live = c < nwant;
  df* z = zs + static_cast<long long>(warp) * n;
  if (live)
    for (int i = lane; i < n; i += 32) z[i] = Zg[i * NW + c];
  for (int k0 = n - 3; k0 >= 0; k0 -= chunk) {
    const int nk = min(chunk, k0 + 1);
    __syncthreads();  // the previous chunk is no longer read
    for (long long idx = tid; idx < static_cast<long long>(nk) * n; idx += blockDim.x) {
      const int r = static_cast<int>(idx / n), i = static_cast<int>(idx % n);
      const int k = k0 - r, m = n - k - 1;
      vs[idx] = i < m ? hv[static_cast<long long>(k) * n + i] : df{0.f, 0.f};
    }
    __syncthreads();
    if (!live) continue;
    for (int r = 0; r < nk; ++r) {
      const int k = k0 - r;
      const df t = tau_g[k];
      if (t.hi == 0.f) continue;
      const int m = n - k - 1;
      const df* v = vs + static_cast<long long>(r) * n;
      df_acc s = acc_zero();
      for (int i = lane; i < m; i += 32) s.fma(v[i], z[k + 1 + i]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s.merge(shfl_xor_acc(s, o));
      const df f = df_mul(t, s.value());
      for (int i = lane; i < m; i += 32) z[k + 1 + i] = df_sub(z[k + 1 + i], df_mul(f, v[i]));
      __syncwarp();
    }
  }
  if (live)
    for (int i = lane; i < n; i += 32) evecs[i * NW + c] = df_to_double(z[i]);
}

// ------------------------------------------------------------ Rayleigh-Ritz pencil
//
// The pencil of Algorithm 3.1 step 2 in the basis [Phi, V - Phi B], Phi =
// I_n^k Z_m (M-orthonormal coarse modes), K = Phi^T A V, B = Phi^T M V:
//     At = [[Theta, Ft], [Ft^T, Tt]],   Mt = [[I, 0], [0, S]],
//     Ft = K - Theta B,   Tt = V^T A V - B^T K - K^T B + B^T Theta B,
//     S  = V^T M V - B^T B   (the Gram matrix of V after block Gram-Schmidt
//                             against the coarse space).
// An eigenvector [a; b] (M-normalised) gives the new vector Phi (a - B b) + V b.
//
// Fast path: a Rayleigh quotient iteration per wanted pair (one block each),
// started from the columns of V (column j is [B e_j; e_j] in this basis), with
// (At - s Mt) y = Mt x solved through the q x q Schur complement
// S(s) = Tt - s S - Ft^T (Theta - s)^-1 Ft (Gaussian elimination with partial
// pivoting), all in float-float.  k_srqi_check accepts the result only if every
// iteration converged, the vectors are mutually Mt-orthogonal to 1e-6, S is
// positive definite, and Sylvester's inertia of At - s* Mt just above the
// largest value (inertia of Theta - s* plus that of S(s*), Haynsworth) counts
// exactly q eigenvalues below, i.e. the pairs found are the q smallest.
// Otherwise the fallback forms the standard matrix H (Cholesky of S) and runs
// the dense float-float eigensolver.  Golub & Van Loan 8.2.3 (RQI), 4.4
// (inertia), 8.7 (symmetric-definite pencils).
constexpr int kPenThreads = 256;
constexpr int kSrqiThreads = 1024;  // one block per pair: the whole SM for its latency-bound steps
constexpr int kSrqiMaxQ = 64;
constexpr int kSrqiMaxIt = 8;
constexpr int kStdMaxQ = 128;  // largest border the solver accepts (q + q_extra)

__device__ __forceinline__ df to_df(double v) { return df_from_double(v); }
__device__ __forceinline__ df to_df(float2 v) { return df{v.x, v.y}; }

// Solve S y = r (S: q x (q+1) augmented, row-major, shared) by Gauss-Jordan
// elimination with partial pivoting, by the whole block: per column, warp 0
// picks the pivot among the rows not yet used and every thread then updates
// elements of the other rows (two barriers per column, no back substitution).
// Pivot rows are marked in `used` instead of swapped; their order is kept in
// prow.  The solution goes to sol.  prow, used (q ints), rinv (1) and sol (q)
// live in shared memory.
__device__ void gj_solve(df* S, int q, int* prow, int* used, df* rinv_s, df* sol) {
  const int ld = q + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < q; i += nt) used[i] = 0;
  __syncthreads();
  for (int k = 0; k < q; ++k) {
    if (tid < 32) {
      float best = -1.f;
      int bi = q;
      for (int i = tid; i < q; i += 32)
        if (!used[i]) {
          const float a = fabsf(S[i * ld + k].hi);
          if (a > best) {
            best = a;
            bi = i;
          }
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        if (b2 > best || (b2 == best && i2 < bi)) {
          best = b2;
          bi = i2;
        }
      }
      if (tid == 0) {
        prow[k] = bi;
        used[bi] = 1;
        df pv = S[bi * ld + k];
        if (fabsf(pv.hi) < 1.0e-30f) pv = df{1.0e-30f, 0.f};
        *rinv_s = df_div(df{1.f, 0.f}, pv);
      }
    }
    __syncthreads();
    const int p = prow[k];
    const df rinv = *rinv_s;
    const int cols = q - k;  // columns k+1..q
    for (int e = tid; e < q * cols; e += nt) {
      const int i = e / cols, j = k + 1 + e % cols;
      if (i == p) continue;
      const df l = df_mul(S[i * ld + k], rinv);
      S[i * ld + j] = df_sub(S[i * ld + j], df_mul(l, S[p * ld + j]));
    }
    __syncthreads();
  }
  for (int k = tid; k < q; k += nt) {
    const int p = prow[k];
    df pv = S[p * ld + k];
    if (fabsf(pv.hi) < 1.0e-30f) pv = df{1.0e-30f, 0.f};
    sol[k] = df_div(S[p * ld + q], pv);
  }
  __syncthreads();
}

// Gauss-Jordan with partial pivoting for q + nrhs <= 32 and a 1024-thread
// block: the thread (i, j) = (tid / 32, tid % 32) keeps element (i, j) of the
// augmented q x (q + nrhs) matrix in registers, so warp i holds row i.  Per column k: the
// pivot row p (chosen by a shared atomic max over |a_ik| while column k was
// updated) is scaled by 1 / a_pk inside its warp and published in shared
// memory; every other row takes its multiplier a_ik from lane k by a shuffle
// and subtracts a_ik * (scaled pivot row).  Two barriers per column, no
// integer division, no back substitution: x_k ends in the right-hand-side
// columns of row p_k.  S is read from shared memory (row stride lds); solution
// r goes to sol[r * ldsol + k].
struct GjShared {
  unsigned long long key[2];
  df prowv[33];
  int kof[32];
};

__device__ __forceinline__ unsigned long long pivot_key(float a, int i) {
  // |a| >= 0: its bits order like its value; ties go to the smaller row
  return (static_cast<unsigned long long>(__float_as_uint(a)) << 32) | static_cast<unsigned>(31 - i);
}

__device__ __forceinline__ df shfl_df(df v, int src) {
  return df{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

__device__ void gj_solve_reg(const df* S, int q, int nrhs, int lds, GjShared* g, df* sol, int ldsol) {
  const int tid = threadIdx.x;
  const int i = tid >> 5, j = tid & 31;
  const int ncol = q + nrhs;
  const bool live = i < q && j < ncol;
  df v = live ? S[i * lds + j] : df{0.f, 0.f};
  if (tid == 0) g->key[0] = 0ull;
  __syncthreads();
  if (live && j == 0) atomicMax(&g->key[0], pivot_key(fabsf(v.hi), i));
  unsigned used = 0u;
  __syncthreads();
  for (int k = 0; k < q; ++k) {
    const int p = 31 - static_cast<int>(g->key[k & 1] & 0xffffffffull);
    if (i == p) {
      df pk = shfl_df(v, k);
      if (fabsf(pk.hi) < 1.0e-30f) pk = df{1.0e-30f, 0.f};
      v = (j == k) ? df{1.f, 0.f} : df_mul(v, df_recip(pk));
      if (j < ncol) g->prowv[j] = v;
    }
    if (tid == 0) {
      g->key[(k + 1) & 1] = 0ull;
      g->kof[p] = k;
    }
    used |= 1u << p;
    __syncthreads();
    if (i < q && i != p) {
      const df l = shfl_df(v, k);
      if (j < ncol && j > k) {
        v = df_sub(v, df_mul(l, g->prowv[j]));
        if (j == k + 1 && !((used >> i) & 1u)) atomicMax(&g->key[(k + 1) & 1], pivot_key(fabsf(v.hi), i));
      }
    }
    __syncthreads();
  }
  if (live && j >= q) sol[(j - q) * ldsol + g->kof[i]] = v;
  __syncthreads();
}

// Inertia by symmetric elimination without pivoting (LDL^T) of two q x q
// matrices at once (q <= 31, 1024 threads): thread (i, j) keeps element (i, j)
// of both in registers; per step k warp k scales its row by 1 / d_k and
// publishes it, and rows i > k subtract a_ik times it.  Counts the negative
// (or zero) pivots of A into *negs and flags a non-positive pivot of B in
// *nonpd (both shared, initialised by the caller).
struct LdlShared {
  df ra[32], rb[32];
};

__device__ void ldl_inertia_reg(const df* A, const df* B, int q, LdlShared* g, int* negs, int* nonpd) {
  const int tid = threadIdx.x;
  const int i = tid >> 5, j = tid & 31;
  const bool live = i < q && j < q;
  df a = live ? A[i * q + j] : df{0.f, 0.f};
  df b = live ? B[i * q + j] : df{0.f, 0.f};
  for (int k = 0; k < q; ++k) {
    if (i == k) {
      df da = shfl_df(a, k), db = shfl_df(b, k);
      if (j == 0) {
        if (df_lt0(da) || da.hi == 0.f) ++*negs;
        if (!(db.hi > 0.f)) *nonpd = 1;
      }
      if (da.hi == 0.f) da = df{-1.0e-30f, 0.f};
      if (!(db.hi > 0.f)) db = df{1.f, 0.f};
      if (j < q) {
        g->ra[j] = df_mul(a, df_recip(da));
        g->rb[j] = df_mul(b, df_recip(db));
      }
    }
    __syncthreads();
    if (i > k && i < q) {
      const df la = shfl_df(a, k), lb = shfl_df(b, k);
      if (j > k && j < q) {
        a = df_sub(a, df_mul(la, g->ra[j]));
        b = df_sub(b, df_mul(lb, g->rb[j]));
      }
    }
    __syncthreads();
  }
}

__device__ df block_sum_df(df_acc a, df_acc* red, df* out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a.merge(shfl_xor_acc(a, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    df_acc b = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : acc_zero();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b.merge(shfl_xor_acc(b, o));
    if (threadIdx.x == 0) *out = b.value();
  }
  __syncthreads();
  const df r = *out;
  __syncthreads();
  return r;
}

// KB = Z_m^T C (m x 2q, float-float): K = KB[:, :q], B = KB[:, q:].  One block
// per column of C; the block's four thread groups split the d_n-long sums.
template <typename TC>
__global__ void __launch_bounds__(kPenThreads) k_kb(int dn, int m, int q, const float2* __restrict__ Zdf,
                                                    const TC* __restrict__ C, df* __restrict__ KB) {
  extern __shared__ __align__(16) unsigned char kraw[];
  df* col = reinterpret_cast<df*>(kraw);  // dn
  __shared__ df_acc part[4][64];
  const int c = blockIdx.x, tid = threadIdx.x;
  const int q2 = 2 * q;
  for (int l = tid; l < dn; l += blockDim.x) col[l] = to_df(C[static_cast<long long>(l) * q2 + c]);
  __syncthreads();
  const int il = tid & 63, g = tid >> 6;
  for (int i0 = 0; i0 < m; i0 += 64) {
    const int i = i0 + il;
    df_acc a = acc_zero(), a2 = acc_zero();
    if (i < m) {
      int l = g;
      for (; l + 4 < dn; l += 8) {
        a.fma(to_df(Zdf[static_cast<long long>(l) * dn + i]), col[l]);
        a2.fma(to_df(Zdf[static_cast<long long>(l + 4) * dn + i]), col[l + 4]);
      }
      if (l < dn) a.fma(to_df(Zdf[static_cast<long long>(l) * dn + i]), col[l]);
    }
    a.merge(a2);
    part[g][il] = a;
    __syncthreads();
    if (g == 0 && i < m) {
      df_acc s = part[0][il];
      s.merge(part[1][il]);
      s.merge(part[2][il]);
      s.merge(part[3][il]);
      KB[static_cast<long long>(i) * q2 + c] = s.value();
    }
    __syncthreads();
  }
}

// Ft (m x q), Tt, S (q x q), float-float; block a computes column a of Ft and
// row a of Tt and S.  G = [V^T A V | V^T M V] (q x 2q) is symmetrised.
__global__ void __launch_bounds__(kPenThreads) k_blocks(int m, int q, const df* __restrict__ KB,
                                                        const double* __restrict__ G, const double* __restrict__ th,
                                                        df* __restrict__ Ft, df* __restrict__ Tt, df* __restrict__ St) {
  __shared__ df_acc pt[8][32], ps[8][32];
  const int a = blockIdx.x, tid = threadIdx.x;
  const int q2 = 2 * q;
  for (int i = tid; i < m; i += blockDim.x) {
    const df k = KB[static_cast<long long>(i) * q2 + a], b = KB[static_cast<long long>(i) * q2 + q + a];
    Ft[static_cast<long long>(i) * q + a] = df_sub(k, df_mul(to_df(th[i]), b));
  }
  const int lane = tid & 31, g = tid >> 5;
  for (int b0 = 0; b0 < q; b0 += 32) {
    const int b = b0 + lane;
    df_acc at = acc_zero(), as = acc_zero();
    if (b < q)
      for (int i = g; i < m; i += 8) {
        const long long r = static_cast<long long>(i) * q2;
        const df ka = KB[r + a], ba = KB[r + q + a], kb = KB[r + b], bb = KB[r + q + b];
        const df fb = df_sub(kb, df_mul(to_df(th[i]), bb));  // (K - Theta B)_ib
        at.fma(ba, fb);
        at.fma(ka, bb);
        as.fma(ba, bb);
      }
    pt[g][lane] = at;
    ps[g][lane] = as;
    __syncthreads();
    if (g == 0 && b < q) {
      df_acc t = pt[0][lane], s = ps[0][lane];
      for (int h = 1; h < 8; ++h) {
        t.merge(pt[h][lane]);
        s.merge(ps[h][lane]);
      }
      const double ga = 0.5 * (G[a * static_cast<long long>(q2) + b] + G[b * static_cast<long long>(q2) + a]);
      const double gm =
          0.5 * (G[a * static_cast<long long>(q2) + q + b] + G[b * static_cast<long long>(q2) + q + a]);
      Tt[a * q + b] = df_sub(to_df(ga), t.value());
      St[a * q + b] = df_sub(to_df(gm), s.value());
    }
    __syncthreads();
  }
}

// x^T At x for x = [x1; x2] (m + q)
__device__ df pencil_rq(const df* th, const df* F, const df* T, const df* x, int m, int q, df_acc* red, df* out) {
  const int tid = threadIdx.x, nt = blockDim.x;
  df_acc a = acc_zero();
  for (int i = tid; i < m + q; i += nt) {
    if (i < m) {
      const df fx = dot4(F + i * q, 1, x + m, 1, q).value();
      // x1_i (theta_i x1_i + 2 (Ft x2)_i)
      a.fma(x[i], df_add(df_mul(th[i], x[i]), df_add(fx, fx)));
    } else {
      const int r = i - m;
      a.fma(x[i], dot4(T + r * q, 1, x + m, 1, q).value());
    }
  }
  return block_sum_df(a, red, out);
}

// x = y / ||y||_Mt (y is first scaled by a power of two near 1 / max |y_i|).  sy: q scratch.
__device__ void mt_normalise(const df* S, df* y, df* x, df* sy, int m, int q, df_acc* red, df* out) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = m + q;
  float amax = 0.f;
  for (int i = tid; i < n; i += nt) amax = fmaxf(amax, fabsf(y[i].hi));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  __shared__ float wmax[32];
  if ((tid & 31) == 0) wmax[tid >> 5] = amax;
  __syncthreads();
  float gmax = (tid & 31) < (nt >> 5) ? wmax[tid & 31] : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  // power-of-two scale keeps the scaling exact
  const float sc = gmax > 0.f ? exp2f(-floorf(log2f(gmax))) : 1.f;
  for (int i = tid; i < n; i += nt) y[i] = df{y[i].hi * sc, y[i].lo * sc};
  __syncthreads();
  for (int a = tid; a < q; a += nt) sy[a] = dot4(S + a * q, 1, y + m, 1, q).value();
  __syncthreads();
  df_acc acc = acc_zero();
  for (int i = tid; i < n; i += nt) acc.fma(y[i], i < m ? y[i] : sy[i - m]);
  const df nrm = df_sqrt(block_sum_df(acc, red, out));
  const df inv = df_recip(nrm);
  for (int i = tid; i < n; i += nt) x[i] = df_mul(y[i], inv);
  __syncthreads();
}

__global__ void __launch_bounds__(kSrqiThreads) k_srqi(int m, int q, const double* __restrict__ thg,
                                                      const df* __restrict__ KB, const df* __restrict__ Ftg,
                                                      const df* __restrict__ Ttg, const df* __restrict__ Stg,
                                                      double* __restrict__ mu, double* __restrict__ X,
                                                      int* __restrict__ conv) {
  extern __shared__ __align__(16) unsigned char sraw[];
  const int n = m + q;
  df* th = reinterpret_cast<df*>(sraw);
  df* dv = th + m;          // m: 1 / (theta_i - s)
  df* F = dv + m;           // m x q
  df* DF = F + m * q;       // m x q: (Theta - s)^-1 Ft
  df* T = DF + m * q;       // q x q
  df* S = T + q * q;        // q x q
  df* Sc = S + q * q;       // q x (q+1)
  df* x = Sc + q * (q + 1); // n
  df* y = x + n;            // n
  df* sx = y + n;           // q
  __shared__ df_acc red[32];
  __shared__ df outv;
  __shared__ int prow[kSrqiMaxQ], used[kSrqiMaxQ];
  __shared__ df ysol[kSrqiMaxQ], rinv;
  __shared__ GjShared gj;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int j = blockIdx.x;
  const int q2 = 2 * q;
  for (int i = tid; i < m; i += nt) th[i] = to_df(thg[i]);
  for (int idx = tid; idx < m * q; idx += nt) F[idx] = Ftg[idx];
  for (int idx = tid; idx < q * q; idx += nt) {
    T[idx] = Ttg[idx];
    S[idx] = Stg[idx];
  }
  // start: column j of V, i.e. [B e_j; e_j]
  for (int i = tid; i < n; i += nt)
    y[i] = i < m ? KB[static_cast<long long>(i) * q2 + q + j] : df{(i - m) == j ? 1.f : 0.f, 0.f};
  __syncthreads();
  mt_normalise(S, y, x, sx, m, q, red, &outv);
  df sg = pencil_rq(th, F, T, x, m, q, red, &outv);
  const df sg0 = sg;  // reported when the iteration fails: it places the pair for the repair
  int ok = 0;
  for (int it = 0; it < kSrqiMaxIt; ++it) {
    // S x2 for the right-hand side
    for (int a = tid; a < q; a += nt) sx[a] = dot4(S + a * q, 1, x + m, 1, q).value();
    for (int i = tid; i < m; i += nt) {
      df d = df_sub(th[i], sg);
      if (fabsf(d.hi) < 1.0e-30f) d = df{1.0e-30f, 0.f};
      dv[i] = df_recip(d);
    }
    __syncthreads();
    for (int idx = tid; idx < m * q; idx += nt) DF[idx] = df_mul(dv[idx / q], F[idx]);
    __syncthreads();
    // Schur complement S(s) (symmetric: upper triangle, mirrored below) and
    // right-hand side S x2 - Ft^T (Theta - s)^-1 x1
    for (int idx = tid; idx < q * (q + 1); idx += nt) {
      const int a = idx / (q + 1), b = idx % (q + 1);
      if (b < a) continue;
      df_acc acc = acc_zero();
      if (b < q) {
        acc.add(T[a * q + b]);
        acc.fma(df_neg(sg), S[a * q + b]);
        acc.add(df_neg(dot4(F + a, q, DF + b, q, m).value()));
      } else {
        acc.add(sx[a]);
        acc.add(df_neg(dot4(DF + a, q, x, 1, m).value()));
      }
      Sc[idx] = acc.value();
    }
    __syncthreads();
    for (int idx = tid; idx < q * q; idx += nt) {
      const int a = idx / q, b = idx % q;
      if (b < a) Sc[a * (q + 1) + b] = Sc[b * (q + 1) + a];
    }
    __syncthreads();
    if (q <= 31 && nt == 1024)
      gj_solve_reg(Sc, q, 1, q + 1, &gj, ysol, q);
    else
      gj_solve(Sc, q, prow, used, &rinv, ysol);
    // y2 = solution, y1 = (Theta - s)^-1 (x1 - Ft y2)
    for (int i = tid; i < n; i += nt) {
      if (i < m) {
        y[i] = df_mul(dv[i], df_sub(x[i], dot4(F + i * q, 1, ysol, 1, q).value()));
      } else {
        y[i] = ysol[i - m];
      }
    }
    __syncthreads();
    mt_normalise(S, y, x, sx, m, q, red, &outv);
    const df sn = pencil_rq(th, F, T, x, m, q, red, &outv);
    const df dlt = df_abs(df_sub(sn, sg));
    sg = sn;
    // RQI converges cubically: a step that moves the quotient by d (relative)
    // started from a vector with angle error ~sqrt(d), so the vector it
    // produced is accurate to ~d^(3/2): d <= 1e-10 gives working precision
    if (it >= 1 && dlt.hi <= 1.0e-10f * fabsf(sn.hi)) {
      ok = it + 1;
      break;
    }
  }
  for (int i = tid; i < n; i += nt) X[i * static_cast<long long>(q) + j] = df_to_double(x[i]);
  if (tid == 0) {
    mu[j] = df_to_double(ok ? sg : sg0);
    conv[j] = ok;  // iterations taken when converged, 0 otherwise
  }
}

// Accept the fast path (flag[0] = 1) or leave it to the dense solver (flag[0] =
// 0).  Vectors of nearly equal values come out of the iteration only accurate
// to residual / gap, and two iterations may even find the same pair; such
// clusters (chains of sorted neighbours whose Mt-overlap exceeds 1e-9, at most
// kMaxCluster vectors) are repaired by Rayleigh-Ritz on the cluster's span --
// after two steps of block inverse iteration from the starting vectors when
// the cluster holds duplicates.  The result is accepted only if every
// iteration converged, all vectors are Mt-orthogonal to 1e-6 afterwards, S is
// positive definite and the inertia count just above the largest value is q.
// On acceptance writes the ascending values to evals and the vectors [a; b]
// ((m + q) x q) to evecs, made Mt-orthonormal to second order by the first-order
// Lowdin correction X (I - E / 2), E = X^T Mt X - I.
constexpr int kMaxCluster = 4;
constexpr int kRepairRounds = 8;
constexpr float kRepairResidual = 1.0e-12f;  // relative residual of a repaired pair

struct CheckShared {
  int okf, negs, nonpd, theta_cnt, nclus;
  int perm[kSrqiMaxQ];
  int cstart[kSrqiMaxQ + 1];  // clusters: members perm[cstart[c] .. cstart[c+1])
  df muS[kSrqiMaxQ];
  df sstar, shift;
  float res;
  float omax;
  int good[kSrqiMaxQ];  // columns accepted so far (the repaired block is kept Mt-orthogonal to them)
  df Ac[kMaxCluster * kMaxCluster], Mc[kMaxCluster * kMaxCluster], Wc[kMaxCluster * kMaxCluster];
  df evc[kMaxCluster];
  GjShared gj;
  LdlShared lsh;
};

// Mt-overlaps Ov = X^T Mt X - I (upper triangle computed, mirrored); omax = max |Ov| off the diagonal
__device__ void check_overlaps(const df* X, const df* SX, df* Ov, int m, int q, CheckShared* c) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) c->omax = 0.f;
  __syncthreads();
  for (int idx = tid; idx < q * q; idx += nt) {
    const int a = idx / q, b = idx % q;
    if (b < a) continue;
    df_acc s = dot4(X + a, q, X + b, q, m);
    s.merge(dot4(X + m * q + a, q, SX + b, q, q));
    if (a == b) s.add(df{-1.f, 0.f});
    const df v = s.value();
    Ov[a * q + b] = v;
    Ov[b * q + a] = v;
    const float f = fabsf(df_float(v));
    if (a != b) atomicMax(reinterpret_cast<int*>(&c->omax), __float_as_int(f));  // f >= 0 (NaN sorts above)
  }
  __syncthreads();
}

// SX = S X2 for all columns
__device__ void check_sx(const df* S, const df* X, df* SX, int m, int q) {
  for (int idx = threadIdx.x; idx < q * q; idx += blockDim.x) {
    const int a = idx / q, j = idx % q;
    SX[idx] = dot4(S + a * q, 1, X + m * q + j, q, q).value();
  }
  __syncthreads();
}

// Yb (n x c, column stride 1, row stride kMaxCluster) -> AY = At Yb, MY = Mt Yb
__device__ void pencil_apply(const df* th, const df* F, const df* T, const df* S, const df* Yb, df* AY, df* MY,
                             int m, int q, int c) {
  const int n = m + q;
  constexpr int L = kMaxCluster;
  for (int idx = threadIdx.x; idx < n * c; idx += blockDim.x) {
    const int i = idx / c, r = idx % c;
    if (i < m) {
      const df fy = dot4(F + i * q, 1, Yb + m * L + r, L, q).value();
      AY[i * L + r] = df_add(df_mul(th[i], Yb[i * L + r]), fy);
      MY[i * L + r] = Yb[i * L + r];
    } else {
      const int a = i - m;
      df_acc t = dot4(F + a, q, Yb + r, L, m);
      t.merge(dot4(T + a * q, 1, Yb + m * L + r, L, q));
      AY[i * L + r] = t.value();
      MY[i * L + r] = dot4(S + a * q, 1, Yb + m * L + r, L, q).value();
    }
  }
  __syncthreads();
}

// c x c symmetric-definite Rayleigh-Ritz by one thread: M = L L^T, C = L^-1 A L^-T,
// cyclic Jacobi on C (one exact rotation for c = 2), W <- L^-T W; values ascending.
__device__ void small_rr(df* A, df* M, df* W, df* ev, int c) {
  constexpr int L = kMaxCluster;
  // Cholesky of M in place (lower)
  for (int k = 0; k < c; ++k) {
    df d = M[k * L + k];
    for (int t = 0; t < k; ++t) d = df_sub(d, df_mul(M[k * L + t], M[k * L + t]));
    d = df_sqrt(d.hi > 0.f ? d : df{1.0e-30f, 0.f});
    M[k * L + k] = d;
    const df id = df_recip(d);
    for (int i = k + 1; i < c; ++i) {
      df s = M[i * L + k];
      for (int t = 0; t < k; ++t) s = df_sub(s, df_mul(M[i * L + t], M[k * L + t]));
      M[i * L + k] = df_mul(s, id);
    }
  }
  // C = L^-1 A L^-T (A symmetric; rows then columns)
  for (int j = 0; j < c; ++j)
    for (int i = 0; i < c; ++i) {
      df s = A[i * L + j];
      for (int t = 0; t < i; ++t) s = df_sub(s, df_mul(M[i * L + t], A[t * L + j]));
      A[i * L + j] = df_div(s, M[i * L + i]);
    }
  for (int i = 0; i < c; ++i)
    for (int j = 0; j < c; ++j) {
      df s = A[i * L + j];
      for (int t = 0; t < j; ++t) s = df_sub(s, df_mul(M[j * L + t], A[i * L + t]));
      A[i * L + j] = df_div(s, M[j * L + j]);
    }
  for (int i = 0; i < c; ++i)
    for (int j = 0; j < c; ++j) W[i * L + j] = df{i == j ? 1.f : 0.f, 0.f};
  const int sweeps = c == 2 ? 1 : 6;
  for (int sw = 0; sw < sweeps; ++sw)
    for (int p = 0; p < c; ++p)
      for (int r = p + 1; r < c; ++r) {
        const df apr = df_mul_f(df_add(A[p * L + r], A[r * L + p]), 0.5f);
        const df dif = df_sub(A[r * L + r], A[p * L + p]);
        if (fabsf(apr.hi) <= 1.0e-30f * fabsf(dif.hi) || apr.hi == 0.f) continue;
        // t = sign(th) / (|th| + sqrt(th^2 + 1)), th = (a_rr - a_pp) / (2 a_pr);
        // t = 1 / (2 th) once th^2 would leave the float range
        const df th = df_div(dif, df_add(apr, apr));
        df t;
        if (fabsf(th.hi) > 1.0e15f) {
          t = df_recip(df_add(th, th));
        } else {
          const df rt = df_sqrt(df_add(df_mul(th, th), df{1.f, 0.f}));
          t = df_recip(df_add(df_abs(th), rt));
          if (df_lt0(th)) t = df_neg(t);
        }
        const df cs = df_recip(df_sqrt(df_add(df_mul(t, t), df{1.f, 0.f})));
        const df sn = df_mul(t, cs);
        for (int k = 0; k < c; ++k) {  // columns p, r of A
          const df akp = A[k * L + p], akr = A[k * L + r];
          A[k * L + p] = df_sub(df_mul(cs, akp), df_mul(sn, akr));
          A[k * L + r] = df_add(df_mul(sn, akp), df_mul(cs, akr));
        }
        for (int k = 0; k < c; ++k) {  // rows p, r of A
          const df apk = A[p * L + k], ark = A[r * L + k];
          A[p * L + k] = df_sub(df_mul(cs, apk), df_mul(sn, ark));
          A[r * L + k] = df_add(df_mul(sn, apk), df_mul(cs, ark));
        }
        for (int k = 0; k < c; ++k) {
          const df wkp = W[k * L + p], wkr = W[k * L + r];
          W[k * L + p] = df_sub(df_mul(cs, wkp), df_mul(sn, wkr));
          W[k * L + r] = df_add(df_mul(sn, wkp), df_mul(cs, wkr));
        }
      }
  // W <- L^-T W
  for (int j = 0; j < c; ++j)
    for (int i = c - 1; i >= 0; --i) {
      df s = W[i * L + j];
      for (int t = i + 1; t < c; ++t) s = df_sub(s, df_mul(M[t * L + i], W[t * L + j]));
      W[i * L + j] = df_div(s, M[i * L + i]);
    }
  // ascending order (selection sort of columns)
  for (int i = 0; i < c; ++i) ev[i] = A[i * L + i];
  for (int i = 0; i < c; ++i) {
    int b = i;
    for (int j = i + 1; j < c; ++j)
      if (df_lt0(df_sub(ev[j], ev[b]))) b = j;
    if (b != i) {
      const df e = ev[i];
      ev[i] = ev[b];
      ev[b] = e;
      for (int k = 0; k < c; ++k) {
        const df w = W[k * L + i];
        W[k * L + i] = W[k * L + b];
        W[k * L + b] = w;
      }
    }
  }
}

// columns of Yb (n x c, row stride kMaxCluster) scaled by powers of two to max |.| ~ 1
__device__ void block_scale(df* Yb, int n, int c) {
  constexpr int L = kMaxCluster;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int r = 0; r < c; ++r) {
      float amax = 0.f;
      for (int i = lane; i < n; i += 32) amax = fmaxf(amax, fabsf(Yb[i * L + r].hi));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      const float sc = amax > 0.f ? exp2f(-floorf(log2f(amax))) : 1.f;
      for (int i = lane; i < n; i += 32) Yb[i * L + r] = df{Yb[i * L + r].hi * sc, Yb[i * L + r].lo * sc};
    }
  }
  __syncthreads();
}

// Yb <- Yb - X_good (X_good^T Mt Yb), twice (the accepted columns of X are
// Mt-orthonormal to working accuracy).  MY, tmp: n x L scratch; coef: q x L.
__device__ void block_deflate(const df* X, const df* S, df* Yb, df* MY, df* tmp, const int* good, df* coef, int m,
                              int q, int c) {
  constexpr int L = kMaxCluster;
  const int n = m + q, tid = threadIdx.x, nt = blockDim.x;
  for (int pass = 0; pass < 2; ++pass) {
    for (int idx = tid; idx < n * c; idx += nt) {
      const int i = idx / c, r = idx % c;
      MY[i * L + r] = i < m ? Yb[i * L + r] : dot4(S + (i - m) * q, 1, Yb + m * L + r, L, q).value();
    }
    __syncthreads();
    for (int idx = tid; idx < q * c; idx += nt) {
      const int j = idx / c, r = idx % c;
      coef[j * L + r] = good[j] ? dot4(X + j, q, MY + r, L, n).value() : df{0.f, 0.f};
    }
    __syncthreads();
    for (int idx = tid; idx < n * c; idx += nt) {
      const int i = idx / c, r = idx % c;
      // skip the other columns outright: an unconverged one may hold NaN
      df_acc a0 = acc_zero(), a1 = acc_zero();
      int j = 0;
      for (; j + 2 <= q; j += 2) {
        if (good[j]) a0.fma(X[i * q + j], coef[j * L + r]);
        if (good[j + 1]) a1.fma(X[i * q + j + 1], coef[(j + 1) * L + r]);
      }
      if (j < q && good[j]) a0.fma(X[i * q + j], coef[j * L + r]);
      a0.merge(a1);
      tmp[i * L + r] = df_sub(Yb[i * L + r], a0.value());
    }
    __syncthreads();
    for (int idx = tid; idx < n * c; idx += nt) Yb[(idx / c) * L + idx % c] = tmp[(idx / c) * L + idx % c];
    __syncthreads();
  }
}

// Mt-orthonormalise the block: G = Yb^T Mt Yb = L L^T, Yb <- Yb L^-T (Cholesky-QR)
__device__ void block_cholqr(const df* th, const df* F, const df* T, const df* S, df* Yb, df* AY, df* MY,
                             CheckShared* c, int m, int q, int cs) {
  constexpr int L = kMaxCluster;
  const int n = m + q, tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < n * cs; idx += nt) {
    const int i = idx / cs, r = idx % cs;
    MY[i * L + r] = i < m ? Yb[i * L + r] : dot4(S + (i - m) * q, 1, Yb + m * L + r, L, q).value();
  }
  __syncthreads();
  for (int idx = tid; idx < cs * cs; idx += nt) {
    const int a = idx / cs, b = idx % cs;
    c->Mc[a * L + b] = dot4(Yb + a, L, MY + b, L, n).value();
  }
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < cs; ++k) {  // Cholesky in place (lower); L^-T goes to Wc
      df d = c->Mc[k * L + k];
      for (int t = 0; t < k; ++t) d = df_sub(d, df_mul(c->Mc[k * L + t], c->Mc[k * L + t]));
      d = df_sqrt(d.hi > 0.f ? d : df{1.0e-30f, 0.f});
      c->Mc[k * L + k] = d;
      const df id = df_recip(d);
      for (int i = k + 1; i < cs; ++i) {
        df t2 = c->Mc[i * L + k];
        for (int t = 0; t < k; ++t) t2 = df_sub(t2, df_mul(c->Mc[i * L + t], c->Mc[k * L + t]));
        c->Mc[i * L + k] = df_mul(t2, id);
      }
    }
    for (int j = 0; j < cs; ++j)
      for (int i = cs - 1; i >= 0; --i) {
        df t2 = df{i == j ? 1.f : 0.f, 0.f};
        for (int t = i + 1; t < cs; ++t) t2 = df_sub(t2, df_mul(c->Mc[t * L + i], c->Wc[t * L + j]));
        c->Wc[i * L + j] = df_div(t2, c->Mc[i * L + i]);
      }
  }
  __syncthreads();
  for (int idx = tid; idx < n * cs; idx += nt) {
    const int i = idx / cs, r = idx % cs;
    df_acc t2 = acc_zero();
    for (int t = 0; t <= r; ++t) t2.fma(Yb[i * L + t], c->Wc[t * L + r]);
    AY[i * L + r] = t2.value();
  }
  __syncthreads();
  for (int idx = tid; idx < n * cs; idx += nt) Yb[(idx / cs) * L + idx % cs] = AY[(idx / cs) * L + idx % cs];
  __syncthreads();
}

// Largest relative residual ||At y - mu Mt y|| / (|mu| ||Mt y||) of the Ritz pairs
// (Yb W_r, ev_r), r < cs, from AY = At Yb and MY = Mt Yb; one warp per pair.
// Result in *res (shared).
__device__ void ritz_residual(const df* AY, const df* MY, const df* W, const df* ev, int n, int cs, float* res) {
  constexpr int L = kMaxCluster;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) *res = 0.f;
  __syncthreads();
  if (w < cs) {
    float rr = 0.f, mm = 0.f;
    for (int i = lane; i < n; i += 32) {
      df_acc a = acc_zero(), b = acc_zero();
      for (int t = 0; t < cs; ++t) {
        a.fma(AY[i * L + t], W[t * L + w]);
        b.fma(MY[i * L + t], W[t * L + w]);
      }
      const df my = b.value();
      const float e = df_float(df_sub(a.value(), df_mul(ev[w], my)));
      rr = fmaf(e, e, rr);
      mm = fmaf(my.hi, my.hi, mm);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rr += __shfl_xor_sync(0xffffffffu, rr, o);
      mm += __shfl_xor_sync(0xffffffffu, mm, o);
    }
    if (lane == 0) {
      const float rel = sqrtf(rr) / (fabsf(ev[w].hi) * sqrtf(mm));
      atomicMax(reinterpret_cast<int*>(res), __float_as_int(rel == rel ? rel : 3.0e38f));
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kSrqiThreads) k_srqi_check(int m, int q, const double* __restrict__ thg,
                                                            const df* __restrict__ KB, const df* __restrict__ Ftg,
                                                            const df* __restrict__ Ttg, const df* __restrict__ Stg,
                                                            const double* __restrict__ mu,
                                                            const double* __restrict__ Xg,
                                                            const int* __restrict__ conv,
                                                            double* __restrict__ evals, double* __restrict__ evecs,
                                                            int* __restrict__ flag) {
  extern __shared__ __align__(16) unsigned char craw[];
  constexpr int L = kMaxCluster;
  const int n = m + q;
  df* X = reinterpret_cast<df*>(craw);  // n x q
  df* SX = X + n * q;                   // q x q: S X2
  df* Sc = SX + q * q;                  // q x q: S(s*)
  df* Sl = Sc + q * q;                  // q x q: S
  df* Ov = Sl + q * q;                  // q x q: X^T Mt X - I
  df* T = Ov + q * q;                   // q x q: Tt
  df* dv = T + q * q;                   // m: 1 / (theta_i - shift)
  df* th = dv + m;                      // m
  df* F = th + m;                       // m x q
  df* Sa = F + m * q;                   // q x (q + L): augmented Schur complement of the repair
  df* Yb = Sa + q * (q + L);            // n x L
  df* AY = Yb + n * L;                  // n x L
  df* MY = AY + n * L;                  // n x L
  df* ys = MY + n * L;                  // L x q
  __shared__ CheckShared c;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    c.okf = 1;
    c.negs = 0;
    c.nonpd = 0;
  }
  for (int idx = tid; idx < n * q; idx += nt) X[idx] = to_df(Xg[idx]);
  for (int idx = tid; idx < q * q; idx += nt) {
    Sl[idx] = Stg[idx];
    T[idx] = Ttg[idx];
  }
  for (int idx = tid; idx < m * q; idx += nt) F[idx] = Ftg[idx];
  for (int i = tid; i < m; i += nt) th[i] = to_df(thg[i]);
  for (int j = tid; j < q; j += nt) c.muS[j] = to_df(mu[j]);
  __syncthreads();
  check_sx(Sl, X, SX, m, q);
  check_overlaps(X, SX, Ov, m, q, &c);
  // sort by value (a NaN from a diverged iteration sorts last), then chain
  // sorted neighbours with large overlaps into clusters
  for (int j = tid; j < q; j += nt) {
    const double vj = mu[j] == mu[j] ? mu[j] : HUGE_VAL;
    int r = 0;
    for (int i = 0; i < q; ++i) {
      const double vi = mu[i] == mu[i] ? mu[i] : HUGE_VAL;
      if (vi < vj || (vi == vj && i < j)) ++r;
    }
    c.perm[r] = j;
  }
  __syncthreads();
  if (tid == 0) {
    int nc = 0, bad = 0;
    c.cstart[0] = 0;
    for (int r = 1; r <= q; ++r) {
      // an iteration that did not converge joins its sorted neighbours' cluster
      const bool join = r < q && (fabsf(df_float(Ov[c.perm[r - 1] * q + c.perm[r]])) > 1.0e-9f ||
                                  !conv[c.perm[r - 1]] || !conv[c.perm[r]]);
      if (!join) {
        const int size = r - c.cstart[nc];
        if (size > L || (size > 1 && q + size > 32) || (size == 1 && !conv[c.perm[r - 1]])) bad = 1;
        c.cstart[++nc] = r;
      }
    }
    c.nclus = nc;
    if (bad) c.okf = 0;
  }
  __syncthreads();
  if (!c.okf) {
    if (tid == 0) {
      flag[0] = 0;
      flag[1] = 1;  // a cluster larger than kMaxCluster, or an unconverged singleton
    }
    return;
  }
  bool repaired = false;
  for (int r = tid; r < q; r += nt) c.good[r] = 1;
  __syncthreads();
  if (tid == 0)
    for (int cl = 0; cl < c.nclus; ++cl)
      if (c.cstart[cl + 1] - c.cstart[cl] > 1)
        for (int r = c.cstart[cl]; r < c.cstart[cl + 1]; ++r) c.good[c.perm[r]] = 0;
  __syncthreads();
  for (int cl = 0; cl < c.nclus; ++cl) {
    const int c0 = c.cstart[cl], cs = c.cstart[cl + 1] - c0;
    if (cs < 2) continue;
    repaired = true;
    // duplicates (overlap > 0.5) or an unconverged member: restart from the
    // starting vectors [B e_j; e_j]
    bool dup = false;
    for (int r = 0; r < cs; ++r) {
      if (!conv[c.perm[c0 + r]]) dup = true;
      if (r + 1 < cs && fabsf(df_float(Ov[c.perm[c0 + r] * q + c.perm[c0 + r + 1]])) > 0.5f) dup = true;
    }
    for (int idx = tid; idx < n * cs; idx += nt) {
      const int i = idx / cs, r = idx % cs, j = c.perm[c0 + r];
      Yb[i * L + r] = dup ? (i < m ? KB[static_cast<long long>(i) * 2 * q + q + j]
                                   : df{(i - m) == j ? 1.f : 0.f, 0.f})
                          : X[i * q + j];
    }
    __syncthreads();
    if (dup) {
      // the block only has to find what the accepted vectors do not span:
      // project them out (Mt inner product) and re-normalise
      block_deflate(X, Sl, Yb, MY, AY, c.good, ys, m, q, cs);
      block_cholqr(th, F, T, Sl, Yb, AY, MY, &c, m, q, cs);
      // shift: the mean Rayleigh quotient of the block (inside the cluster)
      pencil_apply(th, F, T, Sl, Yb, AY, MY, m, q, cs);
      for (int idx = tid; idx < 2 * cs; idx += nt) {
        const int which = idx / cs, r = idx % cs;
        (which ? c.Mc : c.Ac)[r] = dot4(Yb + r, L, (which ? MY : AY) + r, L, n).value();
      }
      __syncthreads();
      if (tid == 0) {
        df sum = df{0.f, 0.f};
        for (int r = 0; r < cs; ++r) sum = df_add(sum, df_div(c.Ac[r], c.Mc[r]));
        c.shift = df_div(sum, df{static_cast<float>(cs), 0.f});
      }
      __syncthreads();
    }
    // block inverse iteration, the shift moved to the mean Ritz value after each
    // step, until the Ritz values settle (at most kRepairRounds steps)
    bool settled = false;
    for (int round = 0; dup && round < kRepairRounds; ++round) {
      // (At - s Mt) Y = Mt Yb through the Schur complement at s, all columns at
      // once; s sits 2^-30 (relative) off the mean Ritz value so that a cluster
      // of equal values cannot make the solve exactly singular
      const df sh = df_add(c.shift, df_mul_f(df_abs(c.shift), 9.313225746154785e-10f));
      for (int i = tid; i < m; i += nt) {
        df d = df_sub(th[i], sh);
        if (fabsf(d.hi) < 1.0e-30f) d = df{1.0e-30f, 0.f};
        dv[i] = df_recip(d);
      }
      __syncthreads();
      for (int idx = tid; idx < q * (q + cs); idx += nt) {
        const int a = idx / (q + cs), b = idx % (q + cs);
        df_acc acc = acc_zero();
        if (b < q) {
          acc.add(T[a * q + b]);
          acc.fma(df_neg(sh), Sl[a * q + b]);
          acc.add(df_neg(dot4w(F + a, q, dv, F + b, q, m).value()));
        } else {
          const int r = b - q;
          acc.add(dot4(Sl + a * q, 1, Yb + m * L + r, L, q).value());
          acc.add(df_neg(dot4w(F + a, q, dv, Yb + r, L, m).value()));
        }
        Sa[a * (q + L) + b] = acc.value();
      }
      __syncthreads();
      gj_solve_reg(Sa, q, cs, q + L, &c.gj, ys, q);
      for (int idx = tid; idx < n * cs; idx += nt) {
        const int i = idx / cs, r = idx % cs;
        Yb[i * L + r] = i < m ? df_mul(dv[i], df_sub(Yb[i * L + r], dot4(F + i * q, 1, ys + r * q, 1, q).value()))
                              : ys[r * q + (i - m)];
      }
      __syncthreads();
      block_scale(Yb, n, cs);
      block_deflate(X, Sl, Yb, MY, AY, c.good, ys, m, q, cs);
      block_cholqr(th, F, T, Sl, Yb, AY, MY, &c, m, q, cs);
      pencil_apply(th, F, T, Sl, Yb, AY, MY, m, q, cs);
      for (int idx = tid; idx < 2 * cs * cs; idx += nt) {
        const int which = idx / (cs * cs), e = idx % (cs * cs), a = e / cs, b = e % cs;
        const df v = dot4(Yb + a, L, (which ? MY : AY) + b, L, n).value();
        (which ? c.Mc : c.Ac)[a * L + b] = v;
      }
      __syncthreads();
      if (tid == 0) {
        small_rr(c.Ac, c.Mc, c.Wc, c.evc, cs);
        df sum = df{0.f, 0.f};
        for (int r = 0; r < cs; ++r) sum = df_add(sum, c.evc[r]);
        c.shift = df_div(sum, df{static_cast<float>(cs), 0.f});
      }
      __syncthreads();
      ritz_residual(AY, MY, c.Wc, c.evc, n, cs, &c.res);
      if (c.res <= kRepairResidual) {
        settled = true;
        break;
      }
    }
    // Rayleigh-Ritz on span(Yb); a block that settled in its last round holds
    // it already (Wc, evc and res of this Yb)
    if (!settled) {
      pencil_apply(th, F, T, Sl, Yb, AY, MY, m, q, cs);
      for (int idx = tid; idx < 2 * cs * cs; idx += nt) {
        const int which = idx / (cs * cs), e = idx % (cs * cs), a = e / cs, b = e % cs;
        const df v = dot4(Yb + a, L, (which ? MY : AY) + b, L, n).value();
        (which ? c.Mc : c.Ac)[a * L + b] = v;
      }
      __syncthreads();
      if (tid == 0) small_rr(c.Ac, c.Mc, c.Wc, c.evc, cs);
      __syncthreads();
      ritz_residual(AY, MY, c.Wc, c.evc, n, cs, &c.res);
    }
    // the repaired pairs must be eigenpairs of the pencil to working accuracy
    if (!(c.res <= kRepairResidual)) {
      if (tid == 0) {
        flag[0] = 0;
        flag[1] = 5;  // a cluster repair did not converge
        flag[2] = __float_as_int(c.res);
        flag[3] = cs;
      }
      return;
    }
    // new vectors Yb W into the cluster's columns (in the cluster's sorted order)
    for (int idx = tid; idx < n * cs; idx += nt) {
      const int i = idx / cs, r = idx % cs, j = c.perm[c0 + r];
      df_acc s2 = acc_zero();
      for (int t = 0; t < cs; ++t) s2.fma(Yb[i * L + t], c.Wc[t * L + r]);
      X[i * q + j] = s2.value();
    }
    for (int r = tid; r < cs; r += nt) {
      c.muS[c.perm[c0 + r]] = c.evc[r];
      c.good[c.perm[c0 + r]] = 1;
    }
    __syncthreads();
  }
  if (repaired) {
    check_sx(Sl, X, SX, m, q);
    check_overlaps(X, SX, Ov, m, q, &c);
  }
  if (!(c.omax <= 1.0e-6f)) {  // also rejects NaN
    if (tid == 0) {
      flag[0] = 0;
      flag[1] = 2;  // vectors not orthogonal after the cluster repairs
      int ba = 0, bb = 0;
      float bv = -1.f;
      for (int a = 0; a < q && bv == bv; ++a)
        for (int b = a + 1; b < q; ++b) {
          const float v = fabsf(df_float(Ov[a * q + b]));
          if (!(v <= bv)) {
            bv = v;
            ba = a;
            bb = b;
            if (v != v) break;  // the first NaN
          }
        }
      flag[2] = ba * 64 + bb;  // the worst pair
      flag[3] = __float_as_int(bv);
    }
    return;
  }
  // inertia just above the largest value
  if (tid == 0) {
    df mx = c.muS[0];
    for (int i = 1; i < q; ++i)
      if (df_lt0(df_sub(mx, c.muS[i]))) mx = c.muS[i];
    c.sstar = df_add(mx, df_mul_f(df_abs(mx), 1.0e-9f));
  }
  __syncthreads();
  if (tid < 32) {
    int cnt = 0;
    for (int i = tid; i < m; i += 32) cnt += df_lt0(df_sub(th[i], c.sstar));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (tid == 0) c.theta_cnt = cnt;
  }
  for (int i = tid; i < m; i += nt) {
    df d = df_sub(th[i], c.sstar);
    if (fabsf(d.hi) < 1.0e-30f) d = df{-1.0e-30f, 0.f};
    dv[i] = df_recip(d);
  }
  __syncthreads();
  for (int idx = tid; idx < q * q; idx += nt) {
    const int a = idx / q, b = idx % q;
    if (b < a) continue;
    df_acc acc = acc_zero();
    acc.add(T[idx]);
    acc.fma(df_neg(c.sstar), Sl[idx]);
    acc.add(df_neg(dot4w(F + a, q, dv, F + b, q, m).value()));
    Sc[idx] = acc.value();
  }
  __syncthreads();
  for (int idx = tid; idx < q * q; idx += nt) {
    const int a = idx / q, b = idx % q;
    if (b < a) Sc[idx] = Sc[b * q + a];
  }
  __syncthreads();
  // LDL^T of S(s*) (negative pivots) and of S (must be positive definite)
  if (q <= 31 && nt == 1024)
    ldl_inertia_reg(Sc, Sl, q, &c.lsh, &c.negs, &c.nonpd);
  else
    for (int k = 0; k < q; ++k) {
      const df pc = Sc[k * q + k], pl = Sl[k * q + k];
      if (tid == 0) {
        if (df_lt0(pc) || pc.hi == 0.f) ++c.negs;
        if (!(pl.hi > 0.f)) c.nonpd = 1;
      }
      const df ic = df_recip((pc.hi == 0.f) ? df{-1.0e-30f, 0.f} : pc);
      const df il = df_recip((pl.hi > 0.f) ? pl : df{1.f, 0.f});
      const int r = q - k - 1;
      __syncthreads();
      for (int idx = tid; idx < 2 * r * r; idx += nt) {
        const int which = idx / (r * r), e = idx % (r * r);
        const int i = k + 1 + e / r, jj = k + 1 + e % r;
        df* Mx = which ? Sl : Sc;
        const df fac = df_mul(Mx[i * q + k], which ? il : ic);
        Mx[i * q + jj] = df_sub(Mx[i * q + jj], df_mul(fac, Mx[k * q + jj]));
      }
      __syncthreads();
    }
  __syncthreads();
  if (c.nonpd || c.theta_cnt + c.negs != q) {
    if (tid == 0) {
      flag[0] = 0;
      flag[1] = c.nonpd ? 3 : 4;  // S not positive definite / not the q smallest
      flag[2] = c.theta_cnt + c.negs;
      flag[3] = q;
    }
    return;
  }
  // final order by the (possibly repaired) values
  for (int j = tid; j < q; j += nt) {
    int r = 0;
    for (int i = 0; i < q; ++i) {
      const df d = df_sub(c.muS[i], c.muS[j]);
      if (df_lt0(d) || (d.hi == 0.f && d.lo == 0.f && i < j)) ++r;
    }
    c.perm[r] = j;  // all values are finite here (the overlap test rejects NaN)
  }
  __syncthreads();
  for (int r = tid; r < q; r += nt) evals[r] = df_to_double(c.muS[c.perm[r]]);
  for (int idx = tid; idx < n * q; idx += nt) {
    const int i = idx / q, r = idx % q, b = c.perm[r];
    const df corr = dot4(X + i * q, 1, Ov + b, q, q).value();
    evecs[idx] = df_to_double(df_sub(X[i * q + b], df{0.5f * corr.hi, 0.5f * corr.lo}));
  }
  if (tid == 0) {
    flag[0] = 1;
    flag[1] = 0;
  }
}

// Fallback: H = [[Theta, Ft L^-T], [L^-1 Ft^T, L^-1 Tt L^-T]] with S = L L^T
// (float-float Cholesky; status = ENOTSPD when S is not positive definite).
__global__ void __launch_bounds__(512) k_std_form(int m, int q, const double* __restrict__ thg,
                                                  const df* __restrict__ Ft, const df* __restrict__ Tt,
                                                  const df* __restrict__ St, df* __restrict__ L, df* __restrict__ Xs,
                                                  double* __restrict__ H, int* status, const int* skip,
                                                  int* nfallback) {
  if (skip && *skip) return;
  if (threadIdx.x == 0 && nfallback) atomicAdd(nfallback, 1);
  extern __shared__ __align__(16) unsigned char fraw[];
  df* Ls = reinterpret_cast<df*>(fraw);  // q x q
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = m + q;
  const long long N = n;
  if (tid == 0) bad = 0;
  for (int idx = tid; idx < q * q; idx += nt) {
    const int r = idx / q, c = idx % q;
    Ls[idx] = c <= r ? St[idx] : df{0.f, 0.f};
  }
  __syncthreads();
  for (int k = 0; k < q; ++k) {
    if (tid == 0) {
      const df d = Ls[k * q + k];
      if (!(d.hi > 0.f)) {
        bad = 1;
        Ls[k * q + k] = df{1.f, 0.f};
      } else {
        Ls[k * q + k] = df_sqrt(d);
      }
    }
    __syncthreads();
    const df inv = df_div(df{1.f, 0.f}, Ls[k * q + k]);
    for (int i = k + 1 + tid; i < q; i += nt) Ls[i * q + k] = df_mul(Ls[i * q + k], inv);
    __syncthreads();
    const int r = q - k - 1;
    for (int idx = tid; idx < r * r; idx += nt) {
      const int i = k + 1 + idx / r, j = k + 1 + idx % r;
      if (j <= i) Ls[i * q + j] = df_sub(Ls[i * q + j], df_mul(Ls[i * q + k], Ls[j * q + k]));
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0 && status) status[0] = AMGEIG_ENOTSPD;
    return;
  }
  for (int idx = tid; idx < q * q; idx += nt) L[idx] = Ls[idx];
  // Xs = L^-1 Tt (columns in parallel; each thread reads back only what it wrote)
  for (int c = tid; c < q; c += nt)
    for (int i = 0; i < q; ++i) {
      df_acc s = acc_zero();
      s.add(Tt[i * q + c]);
      for (int k = 0; k < i; ++k) s.fma(df_neg(Ls[i * q + k]), Xs[k * q + c]);
      Xs[i * q + c] = df_div(s.value(), Ls[i * q + i]);
    }
  __syncthreads();
  // T = L^-1 Xs^T, written (symmetrised below) into H's lower-right block
  for (int c = tid; c < q; c += nt)
    for (int i = 0; i < q; ++i) {
      df_acc s = acc_zero();
      s.add(Xs[c * q + i]);
      for (int k = 0; k < i; ++k) s.fma(df_neg(Ls[i * q + k]), to_df(H[(m + k) * N + m + c]));
      H[(m + i) * N + m + c] = df_to_double(df_div(s.value(), Ls[i * q + i]));
    }
  for (long long idx = tid; idx < static_cast<long long>(m) * m; idx += nt) {
    const int r = static_cast<int>(idx / m), c = static_cast<int>(idx % m);
    H[r * N + c] = (r == c) ? thg[r] : 0.0;
  }
  // F rows: f_i = L^-1 Ft_i^T
  for (int r = tid; r < m; r += nt) {
    df f[kStdMaxQ];
    for (int i = 0; i < q; ++i) {
      df_acc s = acc_zero();
      s.add(Ft[r * q + i]);
      for (int k = 0; k < i; ++k) s.fma(df_neg(Ls[i * q + k]), f[k]);
      f[i] = df_div(s.value(), Ls[i * q + i]);
      const double v = df_to_double(f[i]);
      H[r * N + m + i] = v;
      H[(m + i) * N + r] = v;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < q * q; idx += nt) {
    const int a = idx / q, b = idx % q;
    if (b <= a) continue;
    const double v = 0.5 * (H[(m + a) * N + m + b] + H[(m + b) * N + m + a]);
    H[(m + a) * N + m + b] = v;
    H[(m + b) * N + m + a] = v;
  }
}

// Fallback back-map: b = L^-T b_std in place (rows m.. of evecs, n x q).
// b = L^-T b_std for the p wanted columns of evecs ((m + q) x p; L is the border's q x q factor)
__global__ void k_std_back(int m, int q, int p, const df* __restrict__ L, double* __restrict__ evecs,
                           const int* skip) {
  if (skip && *skip) return;
  const int c = threadIdx.x;
  if (c >= p) return;
  df b[kStdMaxQ];
  for (int i = q - 1; i >= 0; --i) {
    df_acc s = acc_zero();
    s.add(to_df(evecs[(m + i) * static_cast<long long>(p) + c]));
    for (int k = i + 1; k < q; ++k) s.fma(df_neg(L[k * q + i]), b[k]);
    b[i] = df_div(s.value(), L[i * q + i]);
  }
  for (int i = 0; i < q; ++i) evecs[(m + i) * static_cast<long long>(p) + c] = df_to_double(b[i]);
}

// Xc = Z_m (a - B b) (d_n x q) and Y = b (q x q) from evecs = [a; b].  Every
// block forms a - B b in shared memory (b staged there first), then its share
// of the rows of Xc.
// Xc = Z_m (a - B b) and Y = b for the columns [j0, j0 + qc) (chunks keep the
// staged blocks within shared memory when m and q are large)
// q: the border (columns of V), p: the pairs (columns of evecs, Xc and Y)
__global__ void __launch_bounds__(kPenThreads) k_xc(int dn, int m, int q, int p, int j0, int qc,
                                                    const float2* __restrict__ Zdf, const df* __restrict__ KB,
                                                    const double* __restrict__ evecs, double* __restrict__ Xc,
                                                    float2* __restrict__ Xc2, double* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char xraw[];
  df* bs = reinterpret_cast<df*>(xraw);  // q x qc: b[:, j0:j0+qc]
  df* tmp = bs + q * qc;                 // m x qc
  const int tid = threadIdx.x, nt = blockDim.x;
  const int q2 = 2 * q;
  for (int idx = tid; idx < q * qc; idx += nt) {
    const int r = idx / qc, jj = idx % qc;
    const double v = evecs[static_cast<long long>(m + r) * p + j0 + jj];
    bs[idx] = to_df(v);
    if (blockIdx.x == 0) Y[r * p + j0 + jj] = v;
  }
  __syncthreads();
  for (int idx = tid; idx < m * qc; idx += nt) {
    const int i = idx / qc, jj = idx % qc;
    const df* Bi = KB + static_cast<long long>(i) * q2 + q;
    // the four-accumulator dot of dot4, unrolled so that the loads of B's row
    // (L2) are in flight together
    df_acc c0 = acc_zero(), c1 = acc_zero(), c2 = acc_zero(), c3 = acc_zero();
    int t = 0;
#pragma unroll 4
    for (; t + 4 <= q; t += 4) {
      c0.fma(Bi[t], bs[t * qc + jj]);
      c1.fma(Bi[t + 1], bs[(t + 1) * qc + jj]);
      c2.fma(Bi[t + 2], bs[(t + 2) * qc + jj]);
      c3.fma(Bi[t + 3], bs[(t + 3) * qc + jj]);
    }
    for (; t < q; ++t) c0.fma(Bi[t], bs[t * qc + jj]);
    c0.merge(c1);
    c2.merge(c3);
    c0.merge(c2);
    tmp[idx] = df_sub(to_df(evecs[static_cast<long long>(i) * p + j0 + jj]), c0.value());
  }
  __syncthreads();
  const int rows = (dn + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rows, r1 = min(dn, r0 + rows);
  for (int idx = tid; idx < (r1 - r0) * qc; idx += nt) {
    const int l = r0 + idx / qc, jj = idx % qc;
    const float2* zl = Zdf + static_cast<long long>(l) * dn;
    df_acc s0 = acc_zero(), s1 = acc_zero();
    int i = 0;
#pragma unroll 8
    for (; i + 2 <= m; i += 2) {  // unrolled: the row's loads (L2) in flight together
      s0.fma(to_df(zl[i]), tmp[i * qc + jj]);
      s1.fma(to_df(zl[i + 1]), tmp[(i + 1) * qc + jj]);
    }
    if (i < m) s0.fma(to_df(zl[i]), tmp[i * qc + jj]);
    s0.merge(s1);
    const df v = s0.value();
    Xc[static_cast<long long>(l) * p + j0 + jj] = df_to_double(v);
    if (Xc2) Xc2[static_cast<long long>(l) * p + j0 + jj] = make_float2(v.hi, v.lo);
  }
}

// ------------------------------------------------------------ small FP64 kernels

// Float64 Cholesky A = L L^T (row-major, L lower, zero above) of the
// symmetric part of A, right-looking in panels of 32 columns so that the work
// spreads over many blocks (float64 runs at a fraction of the float32 rate):
// per panel the 32 x 32 diagonal block is factored by one block, the rows
// below it solve x L11^T = a one thread each, and the trailing lower triangle
// takes the rank-32 update in 32 x 32 tiles, one block each.  A pivot <= 0
// sets *status = ENOTSPD (and is replaced by 1 so the factorisation finishes).
constexpr int kCb = 32;

__global__ void k_sym_lower(int n, const double* __restrict__ A, double* __restrict__ L) {
  const long long N = n;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N * N;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / N), c = static_cast<int>(i % N);
    L[i] = (c <= r) ? 0.5 * (A[r * N + c] + A[c * N + r]) : 0.0;
  }
}

__global__ void __launch_bounds__(1024) k_chol_diag(int n, int j0, int nb, double* __restrict__ L, int* status) {
  __shared__ double T[kCb][kCb + 1];
  __shared__ int bad;
  const int tid = threadIdx.x;
  const long long N = n;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    T[i][j] = j <= i ? L[(j0 + i) * N + j0 + j] : 0.0;
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (tid == 0) {
      const double d = T[k][k];
      if (!(d > 0.0)) {
        bad = 1;
        T[k][k] = 1.0;
      } else {
        T[k][k] = sqrt(d);
      }
    }
    __syncthreads();
    if (tid > k && tid < nb) T[tid][k] /= T[k][k];
    __syncthreads();
    const int m = nb - k - 1;
    if (tid < m * m) {
      const int i = k + 1 + tid / m, j = k + 1 + tid % m;
      if (j <= i) T[i][j] -= T[i][k] * T[j][k];
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j <= i) L[(j0 + i) * N + j0 + j] = T[i][j];
  }
  if (tid == 0 && bad && status) status[0] = AMGEIG_ENOTSPD;
}

__global__ void __launch_bounds__(128) k_chol_panel(int n, int j0, int nb, double* __restrict__ L) {
  __shared__ double T[kCb][kCb + 1];
  const long long N = n;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    T[i][j] = L[(j0 + i) * N + j0 + j];
  }
  __syncthreads();
  const long long r = j0 + nb + blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (r >= n) return;
  double x[kCb];
#pragma unroll
  for (int j = 0; j < kCb; ++j) x[j] = j < nb ? L[r * N + j0 + j] : 0.0;
#pragma unroll
  for (int j = 0; j < kCb; ++j) {
    if (j < nb) {
      double s = x[j];
#pragma unroll
      for (int t = 0; t < j; ++t) s -= x[t] * T[j][t];
      x[j] = s / T[j][j];
    }
  }
#pragma unroll
  for (int j = 0; j < kCb; ++j)
    if (j < nb) L[r * N + j0 + j] = x[j];
}

// lower-triangle tile (ti, tj), tj <= ti, of the trailing block from the block index
__global__ void __launch_bounds__(256) k_chol_syrk(int n, int j0, int nb, double* __restrict__ L) {
  __shared__ double Ai[kCb][kCb + 1], Aj[kCb][kCb + 1];
  int ti = 0;
  while ((ti + 1) * (ti + 2) / 2 <= static_cast<int>(blockIdx.x)) ++ti;
  const int tj = blockIdx.x - ti * (ti + 1) / 2;
  const int base = j0 + nb, i0 = base + ti * kCb, c0 = base + tj * kCb;
  const long long N = n;
  for (int e = threadIdx.x; e < kCb * kCb; e += blockDim.x) {
    const int r = e / kCb, t = e % kCb;
    Ai[r][t] = (i0 + r < n && t < nb) ? L[(i0 + r) * N + j0 + t] : 0.0;
    Aj[r][t] = (c0 + r < n && t < nb) ? L[(c0 + r) * N + j0 + t] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x / 8, cb = (threadIdx.x % 8) * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 8
  for (int t = 0; t < kCb; ++t) {
    const double a = Ai[r][t];
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] = fma(a, Aj[cb + e][t], acc[e]);
  }
  const int i = i0 + r;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int j = c0 + cb + e;
    if (i < n && j < n && j <= i) L[i * N + j] -= acc[e];
  }
}

void launch_chol_f64(int n, const double* A, double* L, int* status, cudaStream_t st) {
  k_sym_lower<<<ceil_div(static_cast<long long>(n) * n, 256), 256, 0, st>>>(n, A, L);
  for (int j0 = 0; j0 < n; j0 += kCb) {
    const int nb = std::min(kCb, n - j0), rest = n - j0 - nb;
    k_chol_diag<<<1, 1024, 0, st>>>(n, j0, nb, L, status);
    if (rest > 0) {
      k_chol_panel<<<ceil_div(rest, 128), 128, 0, st>>>(n, j0, nb, L);
      const int T = ceil_div(rest, kCb);
      k_chol_syrk<<<T * (T + 1) / 2, 256, 0, st>>>(n, j0, nb, L);
    }
  }
}

int chol_launches(int n) {
  int c = 1;
  for (int j0 = 0; j0 < n; j0 += kCb) c += (n - j0 > kCb) ? 3 : 1;
  return c;
}

// L Y = X in place on ncols columns of the row-major n x ld block X, blocked by 32 rows: rows
// b0 .. b0+31 first take X[b0..] -= L[b0.., 0..b0) X[0..b0) (a float64 product over many blocks), then
// the 32 x 32 diagonal triangle is solved one thread per column (kernel below).
__global__ void __launch_bounds__(128) k_trsm_diag(int n, int b0, int nb, const double* __restrict__ L,
                                                   double* __restrict__ X, int ld, int ncols) {
  __shared__ double T[kCb][kCb + 1];
  const long long N = n, LDX = ld;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    T[i][j] = j <= i ? L[(b0 + i) * N + b0 + j] : 0.0;
  }
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double x[kCb];
#pragma unroll
  for (int r = 0; r < kCb; ++r) x[r] = r < nb ? X[(b0 + r) * LDX + c] : 0.0;
#pragma unroll
  for (int r = 0; r < kCb; ++r) {
    if (r < nb) {
      double s = x[r];
#pragma unroll
      for (int t = 0; t < r; ++t) s -= T[r][t] * x[t];
      x[r] = s / T[r][r];
    }
  }
#pragma unroll
  for (int r = 0; r < kCb; ++r)
    if (r < nb) X[(b0 + r) * LDX + c] = x[r];
}

void launch_trsm_lower(int n, const double* L, double* X, int ld, int ncols, cudaStream_t st) {
  for (int b0 = 0; b0 < n; b0 += kCb) {
    const int nb = std::min(kCb, n - b0);
    if (b0 > 0)
      launch_gemm_f64(nb, ncols, b0, -1.0, L + static_cast<long long>(b0) * n, n, false, X, ld, false, 1.0,
                      X + static_cast<long long>(b0) * ld, ld, st);
    k_trsm_diag<<<ceil_div(ncols, 128), 128, 0, st>>>(n, b0, nb, L, X, ld, ncols);
  }
}

__global__ void k_transpose_sym(int n, const double* __restrict__ X, double* __restrict__ Y) {
  // Y = 0.5 (X + X^T)
  const long long N = n;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N * N;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / N), c = static_cast<int>(i % N);
    Y[i] = 0.5 * (X[r * N + c] + X[c * N + r]);
  }
}

__global__ void k_identity(int n, double* __restrict__ X) {
  const long long N = n;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N * N;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    X[i] = (i / N == i % N) ? 1.0 : 0.0;
}

size_t syev_smem_base(int n, int nwant) {
  return (2 * sizeof(df) * n + 2 * sizeof(float) * n + sizeof(float) * nwant + 2 * sizeof(int) * nwant +
          4 * sizeof(df) * n + sizeof(df) * nwant + 2 * sizeof(int) * nwant + 15) &
         ~static_cast<size_t>(15);
}

constexpr size_t kSmemBudget = 225 * 1024;

}  // namespace

// ------------------------------------------------------------ host side

size_t pencil_work_bytes(int dn, int qmax) {
  PencilWork* w = pencil_work_create(dn, qmax, nullptr, true);
  const size_t b = w ? w->bytes : 0;
  pencil_work_destroy(w);
  return b;
}

PencilWork* pencil_work_create(int dn, int qmax, cudaError_t* err, bool dry) {
  auto* w = new PencilWork();
  w->dn = dn;
  w->qmax = qmax;
  w->nmax = dn + qmax;
  w->nwant_max = dn > qmax ? dn : qmax;
  const long long nm = w->nmax;
  const long long nwm = w->nwant_max;
  // two passes over the same list: sizes (256-byte aligned) into one allocation,
  // then the arrays' places in it
  size_t total = 0;
  char* at = nullptr;
  auto alloc = [&](void** p, size_t bytes) {
    const size_t b = ((bytes > 0 ? bytes : 8) + 255) / 256 * 256;
    if (at) {
      *p = at;
      at += b;
    } else {
      total += b;
    }
  };
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      w->bytes = total;
      if (dry) return w;
      cudaError_t e = dev_alloc(&w->base, total);
      if (err) *err = e;
      if (e != cudaSuccess) {
        w->base = nullptr;
        pencil_work_destroy(w);
        return nullptr;
      }
      at = static_cast<char*>(w->base);
    }
    alloc((void**)&w->KB, sizeof(df) * dn * 2 * qmax);
    alloc((void**)&w->Ft, sizeof(df) * dn * qmax);
    alloc((void**)&w->Tt, sizeof(df) * qmax * qmax);
    alloc((void**)&w->St, sizeof(df) * qmax * qmax);
    alloc((void**)&w->Lq, sizeof(df) * qmax * qmax);
    alloc((void**)&w->Xq, sizeof(df) * qmax * qmax);
    alloc((void**)&w->H, sizeof(double) * nm * nm);
    alloc((void**)&w->Yh, sizeof(double) * nm * nwm);
    alloc((void**)&w->W, sizeof(df) * nm * (nm + 1));
    alloc((void**)&w->tau, sizeof(df) * nm);
    alloc((void**)&w->dd, sizeof(df) * nm);
    alloc((void**)&w->ee, sizeof(df) * nm);
    alloc((void**)&w->fac, sizeof(df) * 6 * nm * nwm);
    alloc((void**)&w->Zt, sizeof(df) * nm * nwm);
    alloc((void**)&w->rr, sizeof(df) * 4 * (nwm * nwm > 4 * nwm ? nwm * nwm : 4 * nwm));
    alloc((void**)&w->perm, sizeof(int) * nwm);
    alloc((void**)&w->hv, sizeof(df) * nm * nm);
    alloc((void**)&w->shd, sizeof(df) * nwm);
    alloc((void**)&w->bounds, sizeof(float) * 4);
    alloc((void**)&w->Lm, sizeof(double) * dn * dn);
    alloc((void**)&w->Hs, sizeof(double) * dn * dn);
    alloc((void**)&w->sr_mu, sizeof(double) * qmax);
    alloc((void**)&w->sr_X, sizeof(double) * nm * qmax);
    alloc((void**)&w->sr_conv, sizeof(int) * qmax);
    alloc((void**)&w->sr_flag, 4 * sizeof(int));
  }
  return w;
}

void pencil_work_destroy(PencilWork* w) {
  if (!w) return;
  if (w->base) dev_release(w->base, w->bytes);  // the caller's work using it has completed
  delete w;
}

// Whether a cluster of c blocks of k_syev_tri_cl with `bytes` of shared memory each can be
// resident on this device (asked once per device and size class; the answer is kept).
bool cluster_fits(int c, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, bool> known;  // (device, c * 1024 + KiB)
  int dev = 0;
  cudaGetDevice(&dev);
  const int key = c * 1024 + static_cast<int>((bytes + 1023) / 1024);
  std::lock_guard<std::mutex> lk(mu);
  auto it = known.find({dev, key});
  if (it != known.end()) return it->second;
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_syev_tri_cl), bytes);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c);
  cfg.blockDim = dim3(kSyThreads);
  cfg.dynamicSmemBytes = bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&clusters, k_syev_tri_cl, &cfg) == cudaSuccess && clusters > 0;
  if (!ok) cudaGetLastError();
  known[{dev, key}] = ok;
  return ok;
}

void launch_syev_df(PencilWork* w, int n, int nwant, const double* H, double* evals, double* evecs,
                    cudaStream_t st, const int* skip) {
  if (n <= 0 || nwant <= 0) return;
  // tridiagonalisation: W in shared memory when it fits beside v, p, d, e, tau
  const int ldw = n | 1;  // odd row stride: column walks of W hit different banks
  const size_t tb = (5 * sizeof(df) * static_cast<size_t>(n) + 15) & ~static_cast<size_t>(15);
  const size_t wb = sizeof(df) * static_cast<size_t>(n) * ldw;
  const int inshared = tb + wb <= kSmemBudget;
  const size_t sm_tri = tb + (inshared ? wb : 0);
  const size_t sm_val = 2 * sizeof(df) * static_cast<size_t>(n) + 2 * sizeof(float) * static_cast<size_t>(n);
  // groups keep their vectors in shared memory up to the budget (the widest possible group: all nwant)
  const size_t sm_vec = std::min(kSmemBudget, syev_vecs_base(n, nwant) + syev_vecs_work(n, nwant));
  // back-transformation: kSbWarps columns and kSbChunk staged reflectors of n df, fewer when n is large
  int wpb = kSbWarps;
  while (wpb > 1 && sizeof(df) * static_cast<size_t>(wpb + 1) * n > kSmemBudget) --wpb;
  const int chunk = static_cast<int>(std::max<size_t>(
      1, std::min<size_t>(kSbChunk, (kSmemBudget - sizeof(df) * static_cast<size_t>(wpb) * n) /
                                        (sizeof(df) * static_cast<size_t>(n)))));
  const size_t sm_back = sizeof(df) * static_cast<size_t>(wpb + chunk) * n;
  ProfScope ps(st, P_PENCIL, 8.0 * n * n + 8.0 * n * nwant, 0.0, 4);
  // W too large for one block: a cluster holding its rows, the largest of 8, 4, 2 blocks that can be scheduled
  // (each block's work per step is its rows times the trailing row length: more blocks, shorter steps)
  int cs = 0, rows_per = 0;
  size_t sm_cl = 0;
  if (!inshared)
    for (int c = kTriMaxCluster; c >= 2 && cs == 0; c /= 2) {
      rows_per = (n + c - 1) / c;
      sm_cl = sizeof(df) * (static_cast<size_t>(rows_per) * ldw + 4 * static_cast<size_t>(n));
      if (sm_cl <= kSmemBudget && cluster_fits(c, sm_cl)) cs = c;
    }
  if (cs > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kSyThreads);
    cfg.dynamicSmemBytes = sm_cl;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_syev_tri_cl, n, ldw, rows_per, H, w->hv, w->dd, w->ee, w->tau, skip);
  } else {
    ensure_dynamic_smem(reinterpret_cast<const void*>(k_syev_tri), sm_tri);
    k_syev_tri<<<1, kSyThreads, sm_tri, st>>>(n, ldw, inshared, H, w->W, w->hv, w->dd, w->ee, w->tau, skip);
  }
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_syev_vals), sm_val);
  k_syev_vals<<<ceil_div(nwant, kSvWarps), 32 * kSvWarps, sm_val, st>>>(n, nwant, w->dd, w->ee, w->shd, w->bounds,
                                                                        skip);
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_syev_vecs), sm_vec);
  k_syev_vecs<<<nwant, kSvecThreads, sm_vec, st>>>(n, nwant, sm_vec, w->dd, w->ee, w->shd, w->bounds, w->fac, w->rr,
                                                   w->Zt, evals, skip);
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_syev_back), sm_back);
  k_syev_back<<<ceil_div(nwant, wpb), 32 * wpb, sm_back, st>>>(n, nwant, chunk, w->hv, w->tau, w->Zt, evecs, skip);
}

void launch_syev_df_into(int n, int nwant, const double* H, double* evals, double* evecs, df* W, df* tau, df* dd,
                         df* ee, df* fac, df* Zt, df* rr, int* perm, cudaStream_t st) {
  const int ldw = n | 1;
  size_t sm = syev_smem_base(n, nwant);
  int flags = 0;
  const size_t wb = sizeof(df) * static_cast<size_t>(n) * ldw;
  const size_t fb = sizeof(df) * 2 * static_cast<size_t>(n) * nwant;
  const size_t zb = sizeof(df) * static_cast<size_t>(n) * nwant;
  if (sm + wb <= kSmemBudget) {
    flags |= kSyW;
    sm += wb;
  }
  if (sm + fb <= kSmemBudget) {
    flags |= kSyF;
    sm += fb;
  }
  if (sm + zb <= kSmemBudget) {
    flags |= kSyZ;
    sm += zb;
  }
  ProfScope ps(st, P_PENCIL, 8.0 * n * n + 8.0 * n * nwant, 0.0);
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_syev_df), sm);
  k_syev_df<<<1, kSyThreads, sm, st>>>(n, nwant, ldw, flags, H, evals, evecs, W, tau, dd, ee, fac, Zt, rr, perm,
                                       nullptr);
}

void launch_pencil_solve(PencilWork* w, int dn, int m, int q, const double* C64, const float2* Cdf,
                         const double* G, const float2* Zdf, const double* theta, double* mu, double* Xc,
                         float2* Xcdf, double* Y, int* status, cudaStream_t st, int* nfallback, int p) {
  if (p <= 0) p = q;  // pairs wanted: the border's width unless a wider border was given
  const int n = m + q;
  auto smem_attr = [](const void* f, size_t bytes) {
    ensure_dynamic_smem(f, bytes);
  };
  const size_t kbs = sizeof(df) * dn;
  const size_t srs = sizeof(df) * (2.0 * m + 2.0 * m * q + 3.0 * q * q + 2.0 * q + 2.0 * n);
  const size_t chs = sizeof(df) * (1.0 * n * q + 5.0 * q * q + 2.0 * m + 1.0 * m * q + 1.0 * q * (q + kMaxCluster) +
                                    3.0 * n * kMaxCluster + 1.0 * kMaxCluster * q);
  const size_t fs = sizeof(df) * q * q;
  // the structured iteration finds one pair per border column: a wider border (p < q) takes the dense path
  const bool fast = p == q && q <= kSrqiMaxQ && srs <= 200 * 1024 && chs <= 220 * 1024;
  // Xc = Z_m (a - B b) runs in column chunks whose staged blocks fit in 200 KB
  const int qc = static_cast<int>(std::max<size_t>(
      1, std::min<size_t>(p, (200 * 1024) / (sizeof(df) * static_cast<size_t>(m + q)))));
  const int nxc = (p + qc - 1) / qc;
  // kernels launched here; the dense eigensolver's launcher counts its own
  ProfScope ps(st, P_PENCIL, 8.0 * (2.0 * dn * m + 2.0 * dn * q + 2.0 * m * q + 3.0 * q * q + 1.0 * n * q), 0.0,
               (fast ? 6 : 4) + nxc);
  if (Cdf) {
    smem_attr((const void*)k_kb<float2>, kbs);
    k_kb<float2><<<2 * q, kPenThreads, kbs, st>>>(dn, m, q, Zdf, Cdf, w->KB);
  } else {
    smem_attr((const void*)k_kb<double>, kbs);
    k_kb<double><<<2 * q, kPenThreads, kbs, st>>>(dn, m, q, Zdf, C64, w->KB);
  }
  k_blocks<<<q, kPenThreads, 0, st>>>(m, q, w->KB, G, theta, w->Ft, w->Tt, w->St);
  // structured Rayleigh quotient iteration, checked by inertia; the dense
  // float-float solver runs only when the check rejects it
  const int* skip = nullptr;
  if (fast) {
    smem_attr((const void*)k_srqi, srs);
    smem_attr((const void*)k_srqi_check, chs);
    k_srqi<<<q, kSrqiThreads, srs, st>>>(m, q, theta, w->KB, w->Ft, w->Tt, w->St, w->sr_mu, w->sr_X, w->sr_conv);
    k_srqi_check<<<1, kSrqiThreads, chs, st>>>(m, q, theta, w->KB, w->Ft, w->Tt, w->St, w->sr_mu, w->sr_X,
                                               w->sr_conv, mu, w->Yh, w->sr_flag);
    skip = w->sr_flag;
  }
  smem_attr((const void*)k_std_form, fs);
  k_std_form<<<1, 512, fs, st>>>(m, q, theta, w->Ft, w->Tt, w->St, w->Lq, w->Xq, w->H, status, skip, nfallback);
  launch_syev_df(w, n, p, w->H, mu, w->Yh, st, skip);
  k_std_back<<<1, kStdMaxQ, 0, st>>>(m, q, p, w->Lq, w->Yh, skip);
  // Xc = Z_m (a - B b), Y = b
  for (int j0 = 0; j0 < p; j0 += qc) {
    const int wc = std::min(qc, p - j0);
    const size_t xsc = sizeof(df) * static_cast<size_t>(m + q) * wc;
    smem_attr((const void*)k_xc, xsc);
    k_xc<<<64, kPenThreads, xsc, st>>>(dn, m, q, p, j0, wc, Zdf, w->KB, w->Yh, Xc, Xcdf, Y);
  }
}

void launch_mass_factor(PencilWork* w, int dn, const double* Mn, int* status, cudaStream_t st) {
  ProfScope ps(st, P_PENCIL, 8.0 * dn * dn * 2, dn * static_cast<double>(dn) * dn / 3.0, chol_launches(dn));
  launch_chol_f64(dn, Mn, w->Lm, status, st);
}

void launch_coarse_inverse(int dn, const double* An, double* L, double* Linv, double* Ainv, int* status,
                           cudaStream_t st) {
  // the products count their own launches
  ProfScope ps(st, P_PENCIL, 8.0 * dn * dn * 5, 2.0 * dn * dn * dn, chol_launches(dn) + 1 + ceil_div(dn, kCb));
  // A_n = L L^T; Linv = L^-1 (the identity solved in place); Ainv = Linv^T Linv = L^-T L^-1
  launch_chol_f64(dn, An, L, status, st);
  k_identity<<<ceil_div(static_cast<long long>(dn) * dn, 256), 256, 0, st>>>(dn, Linv);
  launch_trsm_lower(dn, L, Linv, dn, dn, st);
  launch_gemm_f64(dn, dn, dn, 1.0, Linv, dn, true, Linv, dn, false, 0.0, Ainv, dn, st);
}

void launch_coarse_modes(PencilWork* w, int dn, int nwant, const double* An, double* Z, double* theta,
                         cudaStream_t st) {
  // the products and the eigensolver count their own launches
  ProfScope ps(st, P_PENCIL, 8.0 * dn * dn * 6, 4.0 * dn * dn * static_cast<double>(dn), 2 + ceil_div(dn, kCb));
  // Li = L_m^-1 (the identity solved in place, in H); Hs = sym(Li A_n Li^T) by two float64
  // products (scratch: the eigensolver's W, free until the eigensolver runs, and Yh)
  double* Li = w->H;
  double* T = reinterpret_cast<double*>(w->W);
  k_identity<<<ceil_div(static_cast<long long>(dn) * dn, 256), 256, 0, st>>>(dn, Li);
  launch_trsm_lower(dn, w->Lm, Li, dn, dn, st);
  launch_gemm_f64(dn, dn, dn, 1.0, Li, dn, false, An, dn, false, 0.0, T, dn, st);
  launch_gemm_f64(dn, dn, dn, 1.0, T, dn, false, Li, dn, true, 0.0, w->Yh, dn, st);
  k_transpose_sym<<<ceil_div(static_cast<long long>(dn) * dn, 256), 256, 0, st>>>(dn, w->Yh, w->Hs);
  // the nwant lowest eigenpairs of Hs (dn x nwant into Yh); Z's first columns = L_m^-T Y = Li^T Y
  launch_syev_df(w, dn, nwant, w->Hs, theta, w->Yh, st);
  launch_gemm_f64(dn, nwant, dn, 1.0, Li, dn, true, w->Yh, nwant, false, 0.0, Z, dn, st);
}

}  // namespace amgeig
