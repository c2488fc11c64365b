// The small dense eigenproblems of the method, on the GPU.
//
// Algorithm 3.1 step 2 solves A_{n,k} x = lambda M_{n,k} x on V_n + span(V),
// a pencil of size d_n + q, and Algorithm 3.2 step 1 solves (A_n, M_n).  The
// paper treats these as black boxes (ARPACK, Sec. 4.1).  Here:
//
// * (A_n, M_n) is decomposed once per hierarchy: M_n = L L^T, H = L^-1 A_n L^-T,
//   H = Y Theta Y^T, Z = L^-T Y.  Then Z^T M_n Z = I and Z^T A_n Z = Theta, which
//   gives step 1 of Algorithm 3.2 (the q smallest columns of Z) and the exact
//   coarsest-level solve A_n^-1 = Z Theta^-1 Z^T of the V-cycle.
// * Each correction's pencil is written in the basis [I_n^k Z, V].  With
//   K = Z^T I_k^n A_k V, B = Z^T I_k^n M_k V (d_n x q), the M-part becomes
//   [[I, B], [B^T, V^T M V]]; eliminating B (block Gram-Schmidt of V against the
//   coarse space, in float64 on q x q and d_n x q data) and factoring the Schur
//   complement S = V^T M V - B^T B = L L^T reduces the pencil to the standard
//   symmetric problem
//       H = [[Theta, F], [F^T, T]],  F = (K - Theta B) L^-T,
//       T = L^-1 (V^T A V - B^T K - K^T B + B^T Theta B) L^-T,
//   whose eigenvectors y = [a; b] map back to x = [Z (a - B L^-T b); L^-T b].
//   This is the same Rayleigh-Ritz problem (its eigenvalues are those of the
//   pencil), only better conditioned.
// * The symmetric eigenproblem is solved in float-float (48-bit significand)
//   by one 1024-thread block: Householder tridiagonalisation, bisection with
//   Sturm counts for the wanted eigenvalues (float32), inverse iteration with
//   partial pivoting in float-float (Gram-Schmidt inside clusters of nearly
//   equal shifts), a Rayleigh-Ritz clean-up of the wanted vectors by parallel
//   cyclic Jacobi, and back-transformation.  References: Golub & Van Loan,
//   Matrix Computations, 4th ed., 8.3 (tridiagonalisation), 8.4.1 (Sturm
//   bisection), 8.2.2 (inverse iteration), 8.5 (Jacobi).
#include <cstdio>

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
  // pencil stage
  double* KB = nullptr;   // dn x 2q   Z^T C
  double* Y3 = nullptr;   // dn x 3q   [B | K | Theta B]
  double* P3 = nullptr;   // 2q x 3q   [B K]^T [B K Theta B]
  double* gsc = nullptr;  // gram scratch
  size_t gsc_doubles = 0;
  double* H = nullptr;    // nmax x nmax
  double* Lq = nullptr;   // q x q   Cholesky factor of the Schur complement
  double* Sq = nullptr;   // q x q   scratch
  double* Nq = nullptr;   // q x q   scratch
  double* Yh = nullptr;   // nmax x q eigenvectors of H
  double* tmp = nullptr;  // dn x q
  // float-float eigensolver
  df* W = nullptr;     // nmax x nmax
  df* tau = nullptr;   // nmax
  df* dd = nullptr;    // nmax
  df* ee = nullptr;    // nmax
  df* fac = nullptr;   // 6 x nmax x nwant_max
  df* Zt = nullptr;    // nmax x nwant_max
  df* rr = nullptr;    // 4 x nwant_max^2 (Rayleigh-Ritz clean-up)
  int* perm = nullptr; // nwant_max
  int nwant_max = 0;
  // coarse decomposition
  double* Lm = nullptr;  // dn x dn
  double* Hs = nullptr;  // dn x dn
  // structured Rayleigh quotient iteration
  double* sr_mu = nullptr;  // qmax
  double* sr_X = nullptr;   // nmax x qmax
  int* sr_conv = nullptr;   // qmax
  int* sr_flag = nullptr;   // 1
};

namespace {

// ------------------------------------------------------------ block helpers

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

// ------------------------------------------------------------ float-float syev
//
// Dynamic shared memory: v, p (df, n each), sd, se2 (float, n each), shift
// (float, nwant), cstart, cpos (int, nwant), d, e, tau (df, n each), then --
// when they fit -- the
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
                3 * sizeof(df) * n + 15) &
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
  __shared__ df_acc red_sig[32], red_vp[32];

  for (long long i = tid; i < N * N; i += nt) W[(i / N) * LD + (i % N)] = df_from_double(H[i]);
  __syncthreads();
  // sigma partials of column 0 (rows 2..n-1)
  {
    df_acc a = acc_zero();
    for (int i = 2 + warp; i < n; i += nw)
      if (lane == 0) a.fma(W[i * LD], W[i * LD]);
    if (lane == 0) red_sig[warp] = a;
  }
  __syncthreads();

  // ---- Householder tridiagonalisation (full symmetric storage) -------------
  // Four barriers per step: the norm of the next column and v^T p are formed
  // from per-warp partial sums written in the preceding phase.
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
    // W22 -= v w^T + w v^T (lower triangle computed, mirrored); lane 0 of each
    // row also accumulates the next column's norm (rows 2.. of the trailing block)
    {
      df_acc sg = acc_zero();
      for (int i = warp; i < m; i += nw) {
        const df vi = v[i], wi = p[i];
        df* rowi = W + (k + 1 + i) * LD + (k + 1);
        int j = lane;
        for (; j + 32 <= i; j += 64) {
          const df a0 = rowi[j], a1 = rowi[j + 32];
          const df pj0 = p[j], vj0 = v[j], pj1 = p[j + 32], vj1 = v[j + 32];
          df_acc u0 = acc_zero(), u1 = acc_zero();
          u0.fma(vi, pj0);
          u1.fma(vi, pj1);
          u0.fma(wi, vj0);
          u1.fma(wi, vj1);
          const df n0 = df_sub(a0, u0.value());
          const df n1 = df_sub(a1, u1.value());
          rowi[j] = n0;
          rowi[j + 32] = n1;
          W[(k + 1 + j) * LD + (k + 1 + i)] = n0;
          W[(k + 1 + j + 32) * LD + (k + 1 + i)] = n1;
          if (j == 0 && i >= 2) sg.fma(n0, n0);
        }
        if (j <= i) {
          df_acc u0 = acc_zero();
          u0.fma(vi, p[j]);
          u0.fma(wi, v[j]);
          const df n0 = df_sub(rowi[j], u0.value());
          rowi[j] = n0;
          W[(k + 1 + j) * LD + (k + 1 + i)] = n0;
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

  // ---- bisection (float32) for the nwant smallest eigenvalues -------------
  for (int i = tid; i < n; i += nt) {
    sd[i] = df_float(dd[i]);
    if (i + 1 < n) {
      const float e = df_float(ee[i]);
      se2[i] = e * e;
    }
  }
  __syncthreads();
  if (tid == 0) {
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
  __syncthreads();
  const float gl = sf[0], gu = sf[1], tnorm = sf[2], pivmin = sf[3];
  for (int j = tid; j < nwant; j += nt) {
    float lo = gl, hi = gu;
    for (int it = 0; it < 80; ++it) {
      const float mid = 0.5f * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(sd, se2, n, mid, pivmin) > j) hi = mid; else lo = mid;
    }
    shift[j] = 0.5f * (lo + hi);
  }
  __syncthreads();
  // clusters of nearly equal shifts are iterated in rounds with Gram-Schmidt
  if (tid == 0) {
    const float ctol = 1.0e-4f * tnorm;
    int maxpos = 0;
    for (int j = 0; j < nwant; ++j) {
      if (j > 0 && shift[j] - shift[j - 1] <= ctol) {
        cstart[j] = cstart[j - 1];
        cpos[j] = cpos[j - 1] + 1;
      } else {
        cstart[j] = j;
        cpos[j] = 0;
      }
      maxpos = max(maxpos, cpos[j]);
    }
    si[0] = maxpos;
  }
  __syncthreads();
  const int maxpos = si[0];

  // ---- inverse iteration in float-float: T - s I = L D L^T -----------------
  // factor arrays (element i of eigen-index j at [i * nwant + j]):
  //   fac[0 .. n*nwant) = 1/d_i, fac[n*nwant .. 2n*nwant) = l_i
  const long long NW = nwant;
  const df pv = df{fmaxf(3.6e-15f * tnorm, 1.0e-30f), 0.f};
  for (int round = 0; round <= maxpos; ++round) {
    for (int j = tid; j < nwant; j += nt) {
      if (cpos[j] != round) continue;
      const df sg = df{shift[j], 0.f};
      df* dinv = fac;
      df* lm = fac + N * NW;
      df d = df_sub(dd[0], sg);
      if (fabsf(d.hi) < pv.hi) d = df_lt0(d) ? df_neg(pv) : pv;
      df di = df_div(df{1.f, 0.f}, d);
      dinv[j] = di;
      for (int i = 1; i < n; ++i) {
        const df e = ee[i - 1];
        const df l = df_mul(e, di);
        lm[(i - 1) * NW + j] = l;
        d = df_sub(df_sub(dd[i], sg), df_mul(l, e));
        if (fabsf(d.hi) < pv.hi) d = df_lt0(d) ? df_neg(pv) : pv;
        di = df_div(df{1.f, 0.f}, d);
        dinv[i * NW + j] = di;
      }
      // start vector
      for (int i = 0; i < n; ++i) Zt[i * NW + j] = df{1.f + 0.37f * (float)((i * 7 + j * 13) % 11) / 11.f, 0.f};
      for (int it = 0; it < 3; ++it) {
        // L w = x ; z = D^-1 w ; L^T y = z
        df prev = Zt[j];
        for (int i = 1; i < n; ++i) {
          prev = df_sub(Zt[i * NW + j], df_mul(lm[(i - 1) * NW + j], prev));
          Zt[i * NW + j] = prev;
        }
        df nxt = df_mul(Zt[(n - 1) * NW + j], dinv[(n - 1) * NW + j]);
        Zt[(n - 1) * NW + j] = nxt;
        for (int i = n - 2; i >= 0; --i) {
          nxt = df_sub(df_mul(Zt[i * NW + j], dinv[i * NW + j]), df_mul(lm[i * NW + j], nxt));
          Zt[i * NW + j] = nxt;
        }
        // Gram-Schmidt against finished members of the cluster
        for (int jp = cstart[j]; jp < j; ++jp) {
          df_acc dt = acc_zero();
          for (int i = 0; i < n; ++i) dt.fma(Zt[i * NW + jp], Zt[i * NW + j]);
          const df dv = dt.value();
          for (int i = 0; i < n; ++i) Zt[i * NW + j] = df_sub(Zt[i * NW + j], df_mul(dv, Zt[i * NW + jp]));
        }
        // normalise (scale first by the largest entry to stay in range)
        float amax = 0.f;
        for (int i = 0; i < n; ++i) amax = fmaxf(amax, fabsf(Zt[i * NW + j].hi));
        const float sc1 = amax > 0.f ? 1.f / amax : 1.f;
        df_acc dn = acc_zero();
        for (int i = 0; i < n; ++i) {
          const df z = df_mul_f(Zt[i * NW + j], sc1);
          Zt[i * NW + j] = z;
          dn.fma(z, z);
        }
        const df inv = df_div(df{1.f, 0.f}, df_sqrt(dn.value()));
        for (int i = 0; i < n; ++i) Zt[i * NW + j] = df_mul(Zt[i * NW + j], inv);
      }
    }
    __syncthreads();
  }

  df* Zn = fac;
  if (maxpos == 0) {
    // no two shifts within the cluster tolerance: the vectors are accurate
    // individually (error ~ 48-bit rounding x ||T|| / gap <= 4e-11); their
    // Rayleigh quotients are the eigenvalues, already in ascending order
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
    // ---- Rayleigh-Ritz clean-up on span(Zt): S = Z^T Z, Hq = Z^T T Z ---------
    df* S = rrw;
    df* Hq = rrw + NW * NW;
    df* Qm = rrw + 2 * NW * NW;
    df* Xm = rrw + 3 * NW * NW;
    for (int idx = tid; idx < nwant * nwant; idx += nt) {
      const int a0 = idx / nwant, b0 = idx % nwant;
      if (b0 < a0) continue;
      df_acc s = acc_zero(), h = acc_zero();
      for (int i = 0; i < n; ++i) {
        const df za = Zt[i * NW + a0];
        const df zb = Zt[i * NW + b0];
        s.fma(za, zb);
        df_acc tz = acc_zero();
        tz.fma(dd[i], zb);
        if (i > 0) tz.fma(ee[i - 1], Zt[(i - 1) * NW + b0]);
        if (i + 1 < n) tz.fma(ee[i], Zt[(i + 1) * NW + b0]);
        h.fma(za, tz.value());
      }
      S[a0 * NW + b0] = S[b0 * NW + a0] = s.value();
      Hq[a0 * NW + b0] = Hq[b0 * NW + a0] = h.value();
    }
    __syncthreads();
    // Cholesky S = L L^T in place (lower), right-looking
    for (int kk = 0; kk < nwant; ++kk) {
      if (tid == 0) S[kk * NW + kk] = df_sqrt(S[kk * NW + kk]);
      __syncthreads();
      const df piv = S[kk * NW + kk];
      for (int i = kk + 1 + tid; i < nwant; i += nt) S[i * NW + kk] = df_div(S[i * NW + kk], piv);
      __syncthreads();
      for (int idx = tid; idx < (nwant - kk - 1) * (nwant - kk - 1); idx += nt) {
        const int i = kk + 1 + idx / (nwant - kk - 1), jj = kk + 1 + idx % (nwant - kk - 1);
        if (jj <= i) S[i * NW + jj] = df_sub(S[i * NW + jj], df_mul(S[i * NW + kk], S[jj * NW + kk]));
      }
      __syncthreads();
    }
    // C = L^-1 Hq L^-T  (two column-parallel forward substitutions)
    for (int pass = 0; pass < 2; ++pass) {
      for (int col = tid; col < nwant; col += nt) {
        for (int i = 0; i < nwant; ++i) {
          df s = (pass == 0) ? Hq[i * NW + col] : Xm[col * NW + i];
          for (int kk = 0; kk < i; ++kk)
            s = df_sub(s, df_mul(S[i * NW + kk], (pass == 0) ? Xm[kk * NW + col] : Qm[kk * NW + col]));
          const df r = df_div(s, S[i * NW + i]);
          if (pass == 0) Xm[i * NW + col] = r; else Qm[i * NW + col] = r;
        }
      }
      __syncthreads();
    }
    // Qm now holds C (symmetric); move it to Hq and set Qm = I
    for (int idx = tid; idx < nwant * nwant; idx += nt) {
      const int a0 = idx / nwant, b0 = idx % nwant;
      const df cab = Qm[a0 * NW + b0], cba = Qm[b0 * NW + a0];
      Hq[idx] = df_mul_f(df_add(cab, cba), 0.5f);
    }
    __syncthreads();
    for (int idx = tid; idx < nwant * nwant; idx += nt) Qm[idx] = df{(idx / nwant == idx % nwant) ? 1.f : 0.f, 0.f};
    __syncthreads();
    // parallel cyclic Jacobi (round-robin pairing) on C, accumulating Q
    {
      const int np = (nwant + 1) & ~1;  // even player count; index nwant is a dummy
      for (int sweep = 0; sweep < 12; ++sweep) {
        // convergence test: largest off-diagonal entry against the largest diagonal one
        float off = 0.f, dia = 0.f;
        for (int idx = tid; idx < nwant * nwant; idx += nt) {
          const int a0 = idx / nwant, b0 = idx % nwant;
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
            if (b0 < nwant) {
              const df apq = Hq[a0 * NW + b0];
              const df app = Hq[a0 * NW + a0], aqq = Hq[b0 * NW + b0];
              // skip entries already below the float-float resolution of the diagonal
              const float thr = 1.0e-17f * sqrtf(fabsf(app.hi) * fabsf(aqq.hi)) + 1.0e-37f;
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
          // rows: C <- J^T C
          for (int idx = tid; idx < (np / 2) * nwant; idx += nt) {
            const int t = idx / nwant, col = idx % nwant;
            const int a0 = reinterpret_cast<int*>(&Xm[t * 4 + 2])[0];
            const int b0 = reinterpret_cast<int*>(&Xm[t * 4 + 3])[0];
            if (b0 >= nwant) continue;
            const df cs = Xm[t * 4 + 0], sn = Xm[t * 4 + 1];
            const df x = Hq[a0 * NW + col], y = Hq[b0 * NW + col];
            Hq[a0 * NW + col] = df_sub(df_mul(cs, x), df_mul(sn, y));
            Hq[b0 * NW + col] = df_add(df_mul(sn, x), df_mul(cs, y));
          }
          __syncthreads();
          // columns: C <- C J, Q <- Q J
          for (int idx = tid; idx < (np / 2) * nwant; idx += nt) {
            const int t = idx / nwant, row = idx % nwant;
            const int a0 = reinterpret_cast<int*>(&Xm[t * 4 + 2])[0];
            const int b0 = reinterpret_cast<int*>(&Xm[t * 4 + 3])[0];
            if (b0 >= nwant) continue;
            const df cs = Xm[t * 4 + 0], sn = Xm[t * 4 + 1];
            df x = Hq[row * NW + a0], y = Hq[row * NW + b0];
            Hq[row * NW + a0] = df_sub(df_mul(cs, x), df_mul(sn, y));
            Hq[row * NW + b0] = df_add(df_mul(sn, x), df_mul(cs, y));
            x = Qm[row * NW + a0];
            y = Qm[row * NW + b0];
            Qm[row * NW + a0] = df_sub(df_mul(cs, x), df_mul(sn, y));
            Qm[row * NW + b0] = df_add(df_mul(sn, x), df_mul(cs, y));
          }
          __syncthreads();
        }
      }
    }
    // order eigenvalues ascending (selection by rank; ties broken by index)
    for (int j = tid; j < nwant; j += nt) {
      const df lj = Hq[j * NW + j];
      int rank = 0;
      for (int i = 0; i < nwant; ++i) {
        const df li = Hq[i * NW + i];
        const df dlt = df_sub(li, lj);
        if (df_lt0(dlt) || ((dlt.hi == 0.f && dlt.lo == 0.f) && i < j)) ++rank;
      }
      perm[rank] = j;
    }
    __syncthreads();
    // Xm = L^-T Q  (back substitution per column)
    for (int col = tid; col < nwant; col += nt) {
      for (int i = nwant - 1; i >= 0; --i) {
        df s = Qm[i * NW + col];
        for (int kk = i + 1; kk < nwant; ++kk) s = df_sub(s, df_mul(S[kk * NW + i], Xm[kk * NW + col]));
        Xm[i * NW + col] = df_div(s, S[i * NW + i]);
      }
    }
    __syncthreads();
    // tridiagonal eigenvectors Zt <- Zt Xm, written in sorted order into Qm-free
    // storage: reuse fac (no longer needed) as the new block
    for (long long idx = tid; idx < N * NW; idx += nt) {
      const int i = static_cast<int>(idx / NW), c = static_cast<int>(idx % NW);
      const int src = perm[c];
      df_acc s = acc_zero();
      for (int kk = 0; kk < nwant; ++kk) s.fma(Zt[i * NW + kk], Xm[kk * NW + src]);
      Zn[idx] = s.value();
    }
    __syncthreads();
    for (int c = tid; c < nwant; c += nt) evals[c] = df_to_double(Hq[perm[c] * NW + perm[c]]);
  }

  // ---- back-transformation y = H_0 H_1 ... H_{n-3} z ------------------------
  for (int k = n - 3; k >= 0; --k) {
    const df t = tau[k];
    if (t.hi == 0.f) continue;
    const int m = n - k - 1;
    // for each column c: s_c = v^T z[k+1:, c]; z[k+1:, c] -= t s_c v
    for (int c = warp; c < nwant; c += nw) {
      df_acc s = acc_zero();
      for (int i = lane; i < m; i += 32) s.fma(W[(k + 1 + i) * LD + k], Zn[(k + 1 + i) * NW + c]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s.merge(shfl_xor_acc(s, o));
      const df f = df_mul(t, s.value());
      for (int i = lane; i < m; i += 32)
        Zn[(k + 1 + i) * NW + c] = df_sub(Zn[(k + 1 + i) * NW + c], df_mul(f, W[(k + 1 + i) * LD + k]));
    }
    __syncthreads();
  }
  for (long long idx = tid; idx < N * NW; idx += nt) evecs[idx] = df_to_double(Zn[idx]);
}

// ------------------------------------------------------------ structured Rayleigh quotient iteration
//
// Fast path for the reduced pencil H = [[Theta, F], [F^T, T]] (Theta diagonal,
// m x m; border q): Rayleigh quotient iteration for each wanted pair in its
// own block, with (H - s I) y = x solved through the Schur complement
//   S(s) = T - s I - F^T (Theta - s I)^-1 F   (q x q, Gaussian elimination with
// partial pivoting), starting from the current iterates written in the basis
// of H (column j of V is [B e_j; L^T e_j] there).  k_srqi_check then accepts
// the result only if every iteration converged, the vectors are mutually
// orthogonal, and Sylvester's inertia of H - s* I just above the largest value
// counts exactly q eigenvalues below (inertia(Theta - s) + inertia(S(s)),
// Haynsworth), i.e. the pairs found are the q smallest; otherwise the dense
// float-float eigensolver runs.  Golub & Van Loan 8.2.3 (RQI), 4.4 (inertia).
constexpr int kSrqiThreads = 256;
constexpr int kSrqiMaxQ = 64;
constexpr int kSrqiMaxIt = 8;

// Solve S y = r in place (S: q x (q+1) augmented, row-major, shared) by GEPP;
// the solution is left in column q.
__device__ void gepp_solve(df* S, int q, int* piv_shared) {
  const int ld = q + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < q; ++k) {
    if (tid < 32) {
      float best = -1.f;
      int bi = k;
      for (int i = k + tid; i < q; i += 32) {
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
      if (tid == 0) *piv_shared = bi;
    }
    __syncthreads();
    const int pr = *piv_shared;
    if (pr != k)
      for (int j = k + tid; j <= q; j += nt) {
        const df t = S[k * ld + j];
        S[k * ld + j] = S[pr * ld + j];
        S[pr * ld + j] = t;
      }
    __syncthreads();
    df pivv = S[k * ld + k];
    if (fabsf(pivv.hi) < 1.0e-30f) pivv = df{1.0e-30f, 0.f};
    const df rinv = df_div(df{1.f, 0.f}, pivv);
    const int rows = q - k - 1, cols = q - k;  // columns k+1..q
    for (int idx = tid; idx < rows * cols; idx += nt) {
      const int i = k + 1 + idx / cols, j = k + 1 + idx % cols;
      const df l = df_mul(S[i * ld + k], rinv);
      S[i * ld + j] = df_sub(S[i * ld + j], df_mul(l, S[k * ld + j]));
    }
    __syncthreads();
  }
  // back substitution by warp 0
  if (tid < 32) {
    for (int i = q - 1; i >= 0; --i) {
      df_acc a = acc_zero();
      for (int j = i + 1 + tid; j < q; j += 32) a.fma(S[i * ld + j], S[j * ld + q]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a.merge(shfl_xor_acc(a, o));
      if (tid == 0) {
        df pivv = S[i * ld + i];
        if (fabsf(pivv.hi) < 1.0e-30f) pivv = df{1.0e-30f, 0.f};
        S[i * ld + q] = df_div(df_sub(S[i * ld + q], a.value()), pivv);
      }
      __syncwarp();
    }
  }
  __syncthreads();
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

// x^T H x with H = [[Theta, F], [F^T, T]]; hx receives H x
__device__ df rayleigh(const df* th, const df* F, const df* T, const df* x, df* hx, int m, int q, df_acc* red,
                       df* out) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < m + q; i += nt) {
    df_acc a = acc_zero();
    if (i < m) {
      a.fma(th[i], x[i]);
      for (int c = 0; c < q; ++c) a.fma(F[i * q + c], x[m + c]);
    } else {
      const int r = i - m;
      for (int k = 0; k < m; ++k) a.fma(F[k * q + r], x[k]);
      for (int c = 0; c < q; ++c) a.fma(T[r * q + c], x[m + c]);
    }
    hx[i] = a.value();
  }
  __syncthreads();
  df_acc a = acc_zero();
  for (int i = tid; i < m + q; i += nt) a.fma(x[i], hx[i]);
  return block_sum_df(a, red, out);
}

__global__ void __launch_bounds__(kSrqiThreads) k_srqi(int m, int q, const double* __restrict__ H,
                                                       const double* __restrict__ Y3,
                                                       const double* __restrict__ Lq, double* __restrict__ mu,
                                                       double* __restrict__ X, int* __restrict__ conv) {
  extern __shared__ __align__(16) unsigned char sraw[];
  const int n = m + q;
  df* th = reinterpret_cast<df*>(sraw);
  df* F = th + m;          // m x q
  df* T = F + m * q;       // q x q
  df* S = T + q * q;       // q x (q+1)
  df* x = S + q * (q + 1); // n
  df* y = x + n;           // n
  df* dinv = y + n;        // m
  __shared__ df_acc red[32];
  __shared__ df outv;
  __shared__ int piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int j = blockIdx.x;
  const long long N = n;
  for (int i = tid; i < m; i += nt) th[i] = df_from_double(H[i * N + i]);
  for (int idx = tid; idx < m * q; idx += nt) {
    const int i = idx / q, c = idx % q;
    F[idx] = df_from_double(H[i * N + m + c]);
  }
  for (int idx = tid; idx < q * q; idx += nt) {
    const int a = idx / q, b = idx % q;
    T[idx] = df_from_double(H[(m + a) * N + m + b]);
  }
  // start: column j of V in the basis of H
  for (int i = tid; i < n; i += nt) {
    double v;
    if (i < m) {
      v = Y3[i * 3LL * q + j];
    } else {
      const int a = i - m;
      v = a <= j ? Lq[j * q + a] : 0.0;
    }
    x[i] = df_from_double(v);
  }
  __syncthreads();
  {
    df_acc a = acc_zero();
    for (int i = tid; i < n; i += nt) a.fma(x[i], x[i]);
    const df nrm = df_sqrt(block_sum_df(a, red, &outv));
    const df inv = df_div(df{1.f, 0.f}, nrm);
    for (int i = tid; i < n; i += nt) x[i] = df_mul(x[i], inv);
    __syncthreads();
  }
  df sg = rayleigh(th, F, T, x, y, m, q, red, &outv);
  int ok = 0;
  for (int it = 0; it < kSrqiMaxIt; ++it) {
    // Schur complement S(s) and its right-hand side
    const float pvf = 1.0e-30f;
    for (int i = tid; i < m; i += nt) {
      df d = df_sub(th[i], sg);
      if (fabsf(d.hi) < pvf) d = df{pvf, 0.f};
      dinv[i] = df_div(df{1.f, 0.f}, d);
    }
    __syncthreads();
    for (int idx = tid; idx < q * (q + 1); idx += nt) {
      const int a = idx / (q + 1), b = idx % (q + 1);
      df_acc acc = acc_zero();
      if (b < q) {
        acc.add(T[a * q + b]);
        if (a == b) acc.add(df_neg(sg));
        for (int i = 0; i < m; ++i) acc.fma(df_neg(df_mul(F[i * q + a], dinv[i])), F[i * q + b]);
      } else {
        acc.add(x[m + a]);
        for (int i = 0; i < m; ++i) acc.fma(df_neg(df_mul(F[i * q + a], dinv[i])), x[i]);
      }
      S[idx] = acc.value();
    }
    __syncthreads();
    gepp_solve(S, q, &piv);
    for (int i = tid; i < n; i += nt) {
      if (i < m) {
        df_acc acc = acc_zero();
        acc.add(x[i]);
        for (int c = 0; c < q; ++c) acc.fma(df_neg(F[i * q + c]), S[c * (q + 1) + q]);
        y[i] = df_mul(dinv[i], acc.value());
      } else {
        y[i] = S[(i - m) * (q + 1) + q];
      }
    }
    __syncthreads();
    // normalise (scaled by the largest entry first)
    {
      float amax = 0.f;
      for (int i = tid; i < n; i += nt) amax = fmaxf(amax, fabsf(y[i].hi));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      __shared__ float wmax[32];
      if ((tid & 31) == 0) wmax[tid >> 5] = amax;
      __syncthreads();
      float gmax = 0.f;
      for (int w2 = 0; w2 < (nt >> 5); ++w2) gmax = fmaxf(gmax, wmax[w2]);
      const float sc = gmax > 0.f ? 1.f / gmax : 1.f;
      df_acc a = acc_zero();
      for (int i = tid; i < n; i += nt) {
        const df z = df_mul_f(y[i], sc);
        y[i] = z;
        a.fma(z, z);
      }
      const df nrm = df_sqrt(block_sum_df(a, red, &outv));
      const df inv = df_div(df{1.f, 0.f}, nrm);
      for (int i = tid; i < n; i += nt) x[i] = df_mul(y[i], inv);
      __syncthreads();
    }
    const df sn = rayleigh(th, F, T, x, y, m, q, red, &outv);
    const df dlt = df_abs(df_sub(sn, sg));
    sg = sn;
    if (it >= 1 && dlt.hi <= 4.0e-14f * fabsf(sn.hi)) {
      ok = 1;
      break;
    }
  }
  for (int i = tid; i < n; i += nt) X[i * static_cast<long long>(q) + j] = df_to_double(x[i]);
  if (tid == 0) {
    mu[j] = df_to_double(sg);
    conv[j] = ok;
  }
}

// Accept the fast path (flag[0] = 1) or leave it to the dense solver (flag[0] = 0).
// On acceptance writes the sorted pairs to evals / evecs (n x q).  Sg: q x q scratch.
__global__ void __launch_bounds__(256) k_srqi_check(int m, int q, const double* __restrict__ H,
                                                    const double* __restrict__ mu, const double* __restrict__ X,
                                                    const int* __restrict__ conv, double* __restrict__ Sg,
                                                    double* __restrict__ evals, double* __restrict__ evecs,
                                                    int* __restrict__ flag) {
  __shared__ int okf, negs, theta_cnt;
  __shared__ int perm[kSrqiMaxQ];
  __shared__ double sstar;
  const int n = m + q, tid = threadIdx.x, nt = blockDim.x;
  const long long N = n;
  if (tid == 0) {
    okf = 1;
    negs = 0;
    double mx = mu[0];
    for (int i = 1; i < q; ++i) mx = fmax(mx, mu[i]);
    sstar = mx + 1.0e-9 * fabs(mx) + 1.0e-300;
    int cnt = 0;
    for (int i = 0; i < m; ++i)
      if (H[i * N + i] < sstar) ++cnt;
    theta_cnt = cnt;
  }
  __syncthreads();
  for (int j = tid; j < q; j += nt)
    if (!conv[j]) okf = 0;
  // the computed vectors must be mutually orthogonal (distinct eigenvectors)
  for (int idx = tid; idx < q * q; idx += nt) {
    const int a = idx / q, b = idx % q;
    if (b <= a) continue;
    double s = 0.0;
    for (int i = 0; i < n; ++i)
      s = fma(X[i * static_cast<long long>(q) + a], X[i * static_cast<long long>(q) + b], s);
    if (fabs(s) > 1.0e-6) okf = 0;
  }
  __syncthreads();
  if (!okf) {
    if (tid == 0) flag[0] = 0;
    return;
  }
  // Sylvester inertia of H - s* I: theta_cnt + negative pivots of LDL^T(S(s*))
  for (int idx = tid; idx < q * q; idx += nt) {
    const int a = idx / q, b = idx % q;
    double acc = H[(m + a) * N + m + b] - (a == b ? sstar : 0.0);
    for (int i = 0; i < m; ++i) acc -= H[i * N + m + a] * H[i * N + m + b] / (H[i * N + i] - sstar);
    Sg[idx] = acc;
  }
  __syncthreads();
  for (int k = 0; k < q; ++k) {
    double piv = Sg[k * q + k];
    if (fabs(piv) < 1.0e-300) piv = -1.0e-300;
    if (tid == 0 && piv < 0.0) ++negs;
    const int r = q - k - 1;
    for (int idx = tid; idx < r * r; idx += nt) {
      const int i = k + 1 + idx / r, jj = k + 1 + idx % r;
      Sg[i * q + jj] -= Sg[i * q + k] * Sg[k * q + jj] / piv;
    }
    __syncthreads();
  }
  if (theta_cnt + negs != q) {
    if (tid == 0) flag[0] = 0;
    return;
  }
  for (int j = tid; j < q; j += nt) {
    int r = 0;
    for (int i = 0; i < q; ++i)
      if (mu[i] < mu[j] || (mu[i] == mu[j] && i < j)) ++r;
    perm[r] = j;
  }
  __syncthreads();
  for (int c = tid; c < q; c += nt) evals[c] = mu[perm[c]];
  for (long long idx = tid; idx < N * q; idx += nt) {
    const int i = static_cast<int>(idx / q), c = static_cast<int>(idx % q);
    evecs[idx] = X[i * static_cast<long long>(q) + perm[c]];
  }
  if (tid == 0) flag[0] = 1;
}

// ------------------------------------------------------------ small FP64 kernels

// Cholesky of a symmetric positive definite n x n row-major matrix into L
// (lower, row-major; upper part zeroed).  status[0] = ENOTSPD on failure.
__global__ void k_chol(int n, const double* __restrict__ A, double* __restrict__ L, int* status) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long N = n;
  for (long long i = tid; i < N * N; i += nt) {
    const int r = static_cast<int>(i / N), c = static_cast<int>(i % N);
    L[i] = (c <= r) ? 0.5 * (A[r * N + c] + A[c * N + r]) : 0.0;
  }
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double d = L[k * N + k];
      if (!(d > 0.0)) {
        bad = 1;
        L[k * N + k] = 1.0;
      } else {
        L[k * N + k] = sqrt(d);
      }
    }
    __syncthreads();
    const double piv = L[k * N + k];
    for (int i = k + 1 + tid; i < n; i += nt) L[i * N + k] /= piv;
    __syncthreads();
    const int m = n - k - 1;
    for (long long idx = tid; idx < static_cast<long long>(m) * m; idx += nt) {
      const int i = k + 1 + static_cast<int>(idx / m), j = k + 1 + static_cast<int>(idx % m);
      if (j <= i) L[i * N + j] -= L[i * N + k] * L[j * N + k];
    }
    __syncthreads();
  }
  if (tid == 0 && bad && status) status[0] = AMGEIG_ENOTSPD;
}

// In-place triangular solves on `ncols` columns of the row-major n x ld block X:
// trans = 0: L Y = X (forward), trans = 1: L^T Y = X (backward).  One thread per column.
__global__ void k_trsm(int n, const double* __restrict__ L, double* __restrict__ X, int ld, int ncols, int trans) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const long long N = n;
  if (!trans) {
    for (int i = 0; i < n; ++i) {
      double s = X[i * static_cast<long long>(ld) + c];
      for (int k = 0; k < i; ++k) s -= L[i * N + k] * X[k * static_cast<long long>(ld) + c];
      X[i * static_cast<long long>(ld) + c] = s / L[i * N + i];
    }
  } else {
    for (int i = n - 1; i >= 0; --i) {
      double s = X[i * static_cast<long long>(ld) + c];
      for (int k = i + 1; k < n; ++k) s -= L[k * N + i] * X[k * static_cast<long long>(ld) + c];
      X[i * static_cast<long long>(ld) + c] = s / L[i * N + i];
    }
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

__global__ void k_transpose(int rows, int cols, const double* __restrict__ X, double* __restrict__ Y) {
  const long long total = static_cast<long long>(rows) * cols;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / cols), c = static_cast<int>(i % cols);
    Y[static_cast<long long>(c) * rows + r] = X[i];
  }
}

__global__ void k_scale_cols_inv(int rows, int cols, const double* __restrict__ Z, const double* __restrict__ th,
                                 double* __restrict__ out) {
  const long long total = static_cast<long long>(rows) * cols;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    out[i] = Z[i] / th[i % cols];
}

// Y3 = [B | K | Theta B] from KB = [K | B] (dn x 2q)
__global__ void k_build_y3(int dn, int q, const double* __restrict__ KB, const double* __restrict__ th,
                           double* __restrict__ Y3) {
  const long long total = static_cast<long long>(dn) * q;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / q), c = static_cast<int>(i % q);
    const double K = KB[r * 2LL * q + c], B = KB[r * 2LL * q + q + c];
    Y3[r * 3LL * q + c] = B;
    Y3[r * 3LL * q + q + c] = K;
    Y3[r * 3LL * q + 2 * q + c] = th[r] * B;
  }
}

// Assemble H from the float64 pieces (one block):
//   S = G_M - B^T B, L = chol(S), N = G_A - B^T K - K^T B + B^T Theta B,
//   T = L^-1 N L^-T, F = (K - Theta B) L^-T, H = [[Theta, F], [F^T, T]].
__global__ void k_pencil_h(int dn, int q, const double* __restrict__ G, const double* __restrict__ P3,
                           const double* __restrict__ Y3, const double* __restrict__ th, double* __restrict__ Lq,
                           double* __restrict__ Sq, double* __restrict__ Nq, double* __restrict__ H, int* status) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = dn + q;
  const long long ld3 = 3LL * q;
  for (int idx = tid; idx < q * q; idx += nt) {
    const int a = idx / q, b = idx % q;
    const double gm = 0.5 * (G[a * 2LL * q + q + b] + G[b * 2LL * q + q + a]);
    const double ga = 0.5 * (G[a * 2LL * q + b] + G[b * 2LL * q + a]);
    const double btb = 0.5 * (P3[a * ld3 + b] + P3[b * ld3 + a]);
    const double btk_ab = P3[a * ld3 + q + b], btk_ba = P3[b * ld3 + q + a];
    const double btthb = 0.5 * (P3[a * ld3 + 2 * q + b] + P3[b * ld3 + 2 * q + a]);
    Sq[idx] = gm - btb;
    Nq[idx] = ga - btk_ab - btk_ba + btthb;
  }
  __syncthreads();
  // Cholesky of Sq into Lq
  for (int idx = tid; idx < q * q; idx += nt) {
    const int r = idx / q, c = idx % q;
    Lq[idx] = (c <= r) ? Sq[idx] : 0.0;
  }
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < q; ++k) {
    if (tid == 0) {
      const double d = Lq[k * q + k];
      if (!(d > 0.0)) {
        bad = 1;
        Lq[k * q + k] = 1.0;
      } else {
        Lq[k * q + k] = sqrt(d);
      }
    }
    __syncthreads();
    const double piv = Lq[k * q + k];
    for (int i = k + 1 + tid; i < q; i += nt) Lq[i * q + k] /= piv;
    __syncthreads();
    const int m = q - k - 1;
    for (int idx = tid; idx < m * m; idx += nt) {
      const int i = k + 1 + idx / m, j = k + 1 + idx % m;
      if (j <= i) Lq[i * q + j] -= Lq[i * q + k] * Lq[j * q + k];
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0 && status) status[0] = AMGEIG_ENOTSPD;
    return;
  }
  // X = L^-1 N  (columns), then T = L^-1 X^T  (N symmetric)
  for (int c = tid; c < q; c += nt) {
    for (int i = 0; i < q; ++i) {
      double s = Nq[i * q + c];
      for (int k = 0; k < i; ++k) s -= Lq[i * q + k] * Sq[k * q + c];
      Sq[i * q + c] = s / Lq[i * q + i];
    }
  }
  __syncthreads();
  for (int c = tid; c < q; c += nt) {
    for (int i = 0; i < q; ++i) {
      double s = Sq[c * q + i];  // X^T(i, c) = X(c, i)
      for (int k = 0; k < i; ++k) s -= Lq[i * q + k] * Nq[k * q + c];
      Nq[i * q + c] = s / Lq[i * q + i];
    }
  }
  __syncthreads();
  const long long Nn = n;
  for (long long idx = tid; idx < static_cast<long long>(dn) * dn; idx += nt) {
    const int r = static_cast<int>(idx / dn), c = static_cast<int>(idx % dn);
    H[r * Nn + c] = (r == c) ? th[r] : 0.0;
  }
  // F rows: f_i = L^-1 (K_i - theta_i B_i)^T
  for (int r = tid; r < dn; r += nt) {
    for (int i = 0; i < q; ++i) {
      double s = Y3[r * ld3 + q + i] - th[r] * Y3[r * ld3 + i];
      for (int k = 0; k < i; ++k) s -= Lq[i * q + k] * H[r * Nn + dn + k];
      const double f = s / Lq[i * q + i];
      H[r * Nn + dn + i] = f;
      H[(dn + i) * Nn + r] = f;
    }
  }
  for (int idx = tid; idx < q * q; idx += nt) {
    const int a = idx / q, b = idx % q;
    H[(dn + a) * Nn + dn + b] = 0.5 * (Nq[a * q + b] + Nq[b * q + a]);
  }
}

// Yv = L^-T b (b = Yh[dn:, :]), tmp = a (Yh[:dn, :]) -- one block
__global__ void k_pencil_back(int dn, int q, const double* __restrict__ Yh, const double* __restrict__ Lq,
                              double* __restrict__ Yv, double* __restrict__ tmp) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int c = tid; c < q; c += nt) {
    for (int i = q - 1; i >= 0; --i) {
      double s = Yh[(dn + i) * static_cast<long long>(q) + c];
      for (int k = i + 1; k < q; ++k) s -= Lq[k * q + i] * Yv[k * q + c];
      Yv[i * q + c] = s / Lq[i * q + i];
    }
  }
  for (long long idx = tid; idx < static_cast<long long>(dn) * q; idx += nt) tmp[idx] = Yh[idx];
}

size_t syev_smem_base(int n, int nwant) {
  return (2 * sizeof(df) * n + 2 * sizeof(float) * n + sizeof(float) * nwant + 2 * sizeof(int) * nwant +
          3 * sizeof(df) * n + 15) &
         ~static_cast<size_t>(15);
}

constexpr size_t kSmemBudget = 225 * 1024;

}  // namespace

// ------------------------------------------------------------ host side

PencilWork* pencil_work_create(int dn, int qmax, cudaError_t* err) {
  auto* w = new PencilWork();
  w->dn = dn;
  w->qmax = qmax;
  w->nmax = dn + qmax;
  w->nwant_max = dn > qmax ? dn : qmax;
  const long long nm = w->nmax;
  const long long nwm = w->nwant_max;
  w->gsc_doubles = gram_scratch_doubles(dn, 2 * qmax, 3 * qmax);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 8);
  };
  alloc((void**)&w->KB, sizeof(double) * dn * 2 * qmax);
  alloc((void**)&w->Y3, sizeof(double) * dn * 3 * qmax);
  alloc((void**)&w->P3, sizeof(double) * 6 * qmax * qmax);
  alloc((void**)&w->gsc, sizeof(double) * w->gsc_doubles);
  alloc((void**)&w->H, sizeof(double) * nm * nm);
  alloc((void**)&w->Lq, sizeof(double) * qmax * qmax);
  alloc((void**)&w->Sq, sizeof(double) * qmax * qmax);
  alloc((void**)&w->Nq, sizeof(double) * qmax * qmax);
  alloc((void**)&w->Yh, sizeof(double) * nm * nwm);
  alloc((void**)&w->tmp, sizeof(double) * dn * qmax);
  alloc((void**)&w->W, sizeof(df) * nm * (nm + 1));
  alloc((void**)&w->tau, sizeof(df) * nm);
  alloc((void**)&w->dd, sizeof(df) * nm);
  alloc((void**)&w->ee, sizeof(df) * nm);
  alloc((void**)&w->fac, sizeof(df) * 6 * nm * nwm);
  alloc((void**)&w->Zt, sizeof(df) * nm * nwm);
  alloc((void**)&w->rr, sizeof(df) * 4 * (nwm * nwm > 4 * nwm ? nwm * nwm : 4 * nwm));
  alloc((void**)&w->perm, sizeof(int) * nwm);
  alloc((void**)&w->Lm, sizeof(double) * dn * dn);
  alloc((void**)&w->Hs, sizeof(double) * dn * dn);
  alloc((void**)&w->sr_mu, sizeof(double) * qmax);
  alloc((void**)&w->sr_X, sizeof(double) * nm * qmax);
  alloc((void**)&w->sr_conv, sizeof(int) * qmax);
  alloc((void**)&w->sr_flag, sizeof(int));
  if (err) *err = e;
  if (e != cudaSuccess) {
    pencil_work_destroy(w);
    return nullptr;
  }
  return w;
}

void pencil_work_destroy(PencilWork* w) {
  if (!w) return;
  void* ptrs[] = {w->KB, w->Y3, w->P3, w->gsc, w->H, w->Lq, w->Sq, w->Nq, w->Yh, w->tmp, w->W,
                  w->tau, w->dd, w->ee, w->fac, w->Zt, w->rr, w->perm, w->Lm, w->Hs,
                  w->sr_mu, w->sr_X, w->sr_conv, w->sr_flag};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete w;
}

void launch_syev_df(PencilWork* w, int n, int nwant, const double* H, double* evals, double* evecs,
                    cudaStream_t st, const int* skip) {
  // place W, the factors and Zt in shared memory when they fit (in that order of benefit)
  const int ldw = n | 1;  // odd row stride: column walks of W hit different banks
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
  cudaFuncSetAttribute(k_syev_df, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
  k_syev_df<<<1, kSyThreads, sm, st>>>(n, nwant, ldw, flags, H, evals, evecs, w->W, w->tau, w->dd, w->ee, w->fac,
                                       w->Zt, w->rr, w->perm, skip);
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
  cudaFuncSetAttribute(k_syev_df, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
  k_syev_df<<<1, kSyThreads, sm, st>>>(n, nwant, ldw, flags, H, evals, evecs, W, tau, dd, ee, fac, Zt, rr, perm,
                                       nullptr);
}

void launch_pencil_solve(PencilWork* w, int dn, int m, int q, const double* C, const double* G, const double* Z,
                         const double* theta, double* mu, double* Xc, double* Y, int* status, cudaStream_t st) {
  const int n = m + q;
  // five kernels launched here; the GEMM, Gram and eigensolver launchers count their own
  ProfScope ps(st, P_PENCIL, 8.0 * (2.0 * dn * m + 2.0 * dn * q + 2.0 * q * q + 1.0 * n * n + 1.0 * m * q), 0.0, 5);
  // K | B = Z_m^T [C_A | C_M]   (Z_m: the first m columns of Z)
  launch_gemm_f64(m, 2 * q, dn, 1.0, Z, dn, true, C, 2 * q, false, 0.0, w->KB, 2 * q, st);
  k_build_y3<<<ceil_div(static_cast<long long>(m) * q, 256), 256, 0, st>>>(m, q, w->KB, theta, w->Y3);
  // P3 = [B K]^T [B K Theta B]
  launch_gram_strided(m, w->Y3, 3 * q, 2 * q, w->Y3, 3 * q, 3 * q, w->gsc, w->P3, st);
  k_pencil_h<<<1, 512, 0, st>>>(m, q, G, w->P3, w->Y3, theta, w->Lq, w->Sq, w->Nq, w->H, status);
  // structured Rayleigh quotient iteration, checked by inertia; the dense
  // float-float solver runs only when the check rejects it
  const size_t srs = sizeof(df) * (2.0 * m + 1.0 * m * q + 2.0 * q * q + q + 2.0 * n);
  const int* skip = nullptr;
  if (q <= kSrqiMaxQ && srs <= 200 * 1024) {
    if (srs > 48 * 1024) cudaFuncSetAttribute(k_srqi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)srs);
    k_srqi<<<q, kSrqiThreads, srs, st>>>(m, q, w->H, w->Y3, w->Lq, w->sr_mu, w->sr_X, w->sr_conv);
    k_srqi_check<<<1, 256, 0, st>>>(m, q, w->H, w->sr_mu, w->sr_X, w->sr_conv, w->Sq, mu, w->Yh, w->sr_flag);
    skip = w->sr_flag;
  }
  launch_syev_df(w, n, q, w->H, mu, w->Yh, st, skip);
  k_pencil_back<<<1, 256, 0, st>>>(m, q, w->Yh, w->Lq, Y, w->tmp);
  // tmp = a - B Yv ; Xc = Z_m tmp
  launch_gemm_f64(m, q, q, -1.0, w->Y3, 3 * q, false, Y, q, false, 1.0, w->tmp, q, st);
  launch_gemm_f64(dn, q, m, 1.0, Z, dn, false, w->tmp, q, false, 0.0, Xc, q, st);
}

void launch_coarse_eigh(PencilWork* w, int dn, const double* An, const double* Mn, double* Z, double* theta,
                        double* Ainv, int* status, cudaStream_t st) {
  ProfScope ps(st, P_PENCIL, 8.0 * dn * dn * 6, 0.0, 7);
  // M_n = L L^T
  k_chol<<<1, 1024, 0, st>>>(dn, Mn, w->Lm, status);
  // Hs = L^-1 A_n L^-T : X = L^-1 A_n ; Hs = L^-1 X^T
  cudaMemcpyAsync(w->Hs, An, sizeof(double) * dn * dn, cudaMemcpyDeviceToDevice, st);
  k_trsm<<<ceil_div(dn, 128), 128, 0, st>>>(dn, w->Lm, w->Hs, dn, dn, 0);
  k_transpose<<<ceil_div(static_cast<long long>(dn) * dn, 256), 256, 0, st>>>(dn, dn, w->Hs, w->H);
  k_trsm<<<ceil_div(dn, 128), 128, 0, st>>>(dn, w->Lm, w->H, dn, dn, 0);
  k_transpose_sym<<<ceil_div(static_cast<long long>(dn) * dn, 256), 256, 0, st>>>(dn, w->H, w->Hs);
  // eigenpairs of Hs (all dn)
  launch_syev_df(w, dn, dn, w->Hs, theta, Z, st);
  // Z = L^-T Y
  k_trsm<<<ceil_div(dn, 128), 128, 0, st>>>(dn, w->Lm, Z, dn, dn, 1);
  // Ainv = Z diag(1/theta) Z^T
  k_scale_cols_inv<<<ceil_div(static_cast<long long>(dn) * dn, 256), 256, 0, st>>>(dn, dn, Z, theta, w->H);
  launch_gemm_f64(dn, dn, dn, 1.0, w->H, dn, false, Z, dn, true, 0.0, Ainv, dn, st);
  // two Newton-Schulz steps bring the float-float-derived inverse to float64 accuracy
  launch_newton_schulz(dn, An, Ainv, w->Hs, w->H, st);
  launch_newton_schulz(dn, An, Ainv, w->Hs, w->H, st);
}

}  // namespace amgeig
