// Float-float ("df") sparse kernels of the mixed-precision path.
//
// In the mixed path the iterate blocks U, V, W = [AV | MV] and the transfer
// chains are stored as float-float pairs (float2: hi, lo; 48-bit significand)
// and every product accumulates with the compensated scheme of common.cuh on
// the float32 pipes.  The matrix values are split into float-float pairs once,
// at load.  This replaces float64 FMA, which issues at 1/59 of the float32 rate
// on this GPU, for the defect (Eq. Linear_Equation), the augmentation products
// A_k V, M_k V (Algorithm 3.1 step 2), the restriction / prolongation chains
// I_k^n, I_n^k and the recombination.  Rounding: ~2^-48 relative per
// operation; the cancellation in lambda M u - A u raises the floor of the
// relative residual to ~2^-48 lambda_max / lambda (float64: 2^-53 times the same).
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"
#include "prof.cuh"

namespace amgeig {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ df ld2(const float2* p, long long i) {
  const float2 v = p[i];
  return df{v.x, v.y};
}
__device__ __forceinline__ void st2(float2* p, long long i, df v) { p[i] = make_float2(v.hi, v.lo); }

// ---- bulk-copy pipeline (sm_90+ TMA engine, used here on sm_103a)
//
// One elected thread starts cp.async.bulk copies of whole contiguous row slabs
// into shared memory; each copy signals a shared-memory mbarrier with its byte
// count (complete_tx), and the block waits on the barrier's phase parity.  The
// waits are bounded: a copy that has not landed after kBulkSpins polls sets the
// status word and the block stops (no kernel spins forever).
constexpr int kBulkSpins = 1 << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (int i = 0; i < kBulkSpins; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}


struct Geo {
  int G, rows_per_block, cpt;
  // G need not divide kThreads: blocks get exactly G * rows_per_block threads, so
  // every thread owns a row slot of its own block
  int threads() const { return G * rows_per_block; }
};

// G lanes per row with CPT = ceil(width / G) <= 8 columns each: about three or
// four columns per lane gives each thread independent accumulation chains and
// cuts the redundant index / value loads of a wide row group.  G need not be a
// power of two (28 columns: 7 lanes x 4); the fewest idle column slots win,
// then CPT nearest 3.5, then the larger G.
Geo geo_for(int width) {
  int bestG = 1, bestC = width;
  long long bestKey = -1;
  for (int G = 1; G <= 32; ++G) {
    const int cpt = (width + G - 1) / G;
    if (cpt > 8) continue;
    const int waste = G * cpt - width;
    const int dist = cpt * 2 > 7 ? cpt * 2 - 7 : 7 - cpt * 2;  // |cpt - 3.5| * 2
    const long long key = static_cast<long long>(waste) * 1000 + dist * 40 + (32 - G);
    if (bestKey < 0 || key < bestKey) {
      bestKey = key;
      bestG = G;
      bestC = cpt;
    }
  }
  return Geo{bestG, kThreads / bestG, bestC};
}

// ---------------------------------------------------------------- defect
// R = lambda o (M U) - A U, rounded to float32 with row stride ldr (zero padding),
// per-block sums of r^2 and (Mu)^2 (fixed order).  The sums accumulate in
// float-float: float64 arithmetic here, once per row and column, cost more
// than the whole sparse product on this GPU.
// PW = 2 (even q, 16-byte aligned U): each lane's unit is a pair of adjacent
// columns fetched by one 16-byte load; unit u covers columns PW u .. PW u + PW - 1.
// Every column's sums run over the same nonzeros in the same order for PW = 1, 2.
template <int CPT, int PW>
__global__ void __launch_bounds__(kThreads, 4) k_defect_df(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                        const float2* __restrict__ a, const float2* __restrict__ m,
                                                        const float2* __restrict__ U, int q,
                                                        const double* __restrict__ lam, float* __restrict__ R,
                                                        int ldr, int G, double* __restrict__ partials) {
  // grid-stride over row groups; each thread keeps its columns' sums of r^2 and
  // (Mu)^2 in registers, so a block writes one row of partials
  extern __shared__ df_acc sred[];
  constexpr int K = CPT * PW;  // columns per thread
  const int rpb = blockDim.x / G;
  const int g = threadIdx.x / G;
  const int lane = threadIdx.x % G;
  df_acc rr[K], m2[K];
  df lamc[K];
#pragma unroll
  for (int t = 0; t < CPT; ++t)
#pragma unroll
    for (int e = 0; e < PW; ++e) {
      const int k = t * PW + e, c = (lane + t * G) * PW + e;
      rr[k] = m2[k] = acc_zero();
      lamc[k] = c < q ? df_from_double(lam[c]) : df{0.f, 0.f};
    }
  for (int row = blockIdx.x * rpb + g; row < n; row += gridDim.x * rpb) {
    df_acc aa[K], mm[K];
#pragma unroll
    for (int k = 0; k < K; ++k) aa[k] = mm[k] = acc_zero();
    const int p0 = rp[row], p1 = rp[row + 1];
#pragma unroll 4
    for (int p = p0; p < p1; ++p) {
      const int j = ci[p];
      const df av = ld2(a, p), mv = ld2(m, p);
      const long long base = static_cast<long long>(j) * q;
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        const int c = (lane + t * G) * PW;
        if (c < q) {
          if (PW == 2) {
            const float4 u2 = *reinterpret_cast<const float4*>(U + base + c);
            const df u0 = df{u2.x, u2.y}, u1 = df{u2.z, u2.w};
            aa[t * PW].fma(av, u0);
            mm[t * PW].fma(mv, u0);
            aa[t * PW + PW - 1].fma(av, u1);
            mm[t * PW + PW - 1].fma(mv, u1);
          } else {
            const df u = ld2(U, base + c);
            aa[t].fma(av, u);
            mm[t].fma(mv, u);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < CPT; ++t)
#pragma unroll
      for (int e = 0; e < PW; ++e) {
        const int k = t * PW + e, c = (lane + t * G) * PW + e;
        if (c < q) {
          const df mu = mm[k].value();
          const df r = df_sub(df_mul(lamc[k], mu), aa[k].value());
          const float rf = df_float(r);
          R[static_cast<long long>(row) * ldr + c] = rf;
          rr[k].fma(df{rf, 0.f}, df{rf, 0.f});
          m2[k].fma(mu, mu);
        }
      }
    for (int c = q + lane; c < ldr; c += G) R[static_cast<long long>(row) * ldr + c] = 0.f;
  }
  if (partials == nullptr) return;
  const int W = G * K;
#pragma unroll
  for (int t = 0; t < CPT; ++t)
#pragma unroll
    for (int e = 0; e < PW; ++e) {
      const int k = t * PW + e, c = (lane + t * G) * PW + e;
      sred[g * 2 * W + c] = rr[k];
      sred[g * 2 * W + W + c] = m2[k];
    }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 2 * q; idx += blockDim.x) {
    const int which = idx / q, c = idx % q;
    df_acc s = acc_zero();
    for (int r = 0; r < rpb; ++r) s.merge(sred[r * 2 * W + which * W + c]);
    partials[static_cast<long long>(blockIdx.x) * 2 * q + idx] = df_to_double(s.value());
  }
}

// ---------------------------------------------------------------- W = [A V | M V]
template <int CPT, int PW>
__global__ void __launch_bounds__(kThreads) k_dual_spmm_df(int n, const int* __restrict__ rp,
                                                           const int* __restrict__ ci, const float2* __restrict__ a,
                                                           const float2* __restrict__ m,
                                                           const float2* __restrict__ V, int q,
                                                           float2* __restrict__ W, int G) {
  constexpr int K = CPT * PW;
  const int rpb = blockDim.x / G;
  const int lane = threadIdx.x % G;
  const int row = blockIdx.x * rpb + threadIdx.x / G;
  if (row >= n) return;
  df_acc aa[K], mm[K];
#pragma unroll
  for (int k = 0; k < K; ++k) aa[k] = mm[k] = acc_zero();
  const int p0 = rp[row], p1 = rp[row + 1];
  for (int p = p0; p < p1; ++p) {
    const int j = ci[p];
    const df av = ld2(a, p), mv = ld2(m, p);
    const long long base = static_cast<long long>(j) * q;
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      const int c = (lane + t * G) * PW;
      if (c < q) {
        if (PW == 2) {
          const float4 v2 = *reinterpret_cast<const float4*>(V + base + c);
          const df v0 = df{v2.x, v2.y}, v1 = df{v2.z, v2.w};
          aa[t * PW].fma(av, v0);
          mm[t * PW].fma(mv, v0);
          aa[t * PW + PW - 1].fma(av, v1);
          mm[t * PW + PW - 1].fma(mv, v1);
        } else {
          const df v = ld2(V, base + c);
          aa[t].fma(av, v);
          mm[t].fma(mv, v);
        }
      }
    }
  }
  const long long o = static_cast<long long>(row) * 2 * q;
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    const int c = (lane + t * G) * PW;
    if (c >= q) continue;
    if (PW == 2) {
      const df a0 = aa[t * PW].value(), a1 = aa[t * PW + PW - 1].value();
      const df m0 = mm[t * PW].value(), m1 = mm[t * PW + PW - 1].value();
      *reinterpret_cast<float4*>(W + o + c) = make_float4(a0.hi, a0.lo, a1.hi, a1.lo);
      *reinterpret_cast<float4*>(W + o + q + c) = make_float4(m0.hi, m0.lo, m1.hi, m1.lo);
    } else {
      st2(W, o + c, aa[t].value());
      st2(W, o + q + c, mm[t].value());
    }
  }
}

// ---------------------------------------------------------------- Y (+)= S X
template <int CPT>
__global__ void __launch_bounds__(kThreads) k_spmm_df(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                      const float2* __restrict__ v, const float2* __restrict__ X,
                                                      int width, float2* __restrict__ Y, int G, int accumulate) {
  const int rpb = blockDim.x / G;
  const int lane = threadIdx.x % G;
  const int row = blockIdx.x * rpb + threadIdx.x / G;
  if (row >= n) return;
  df_acc acc[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) acc[t] = acc_zero();
  const int p0 = rp[row], p1 = rp[row + 1];
  for (int p = p0; p < p1; ++p) {
    const df s = ld2(v, p);
    const long long base = static_cast<long long>(ci[p]) * width;
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      const int c = lane + t * G;
      if (c < width) acc[t].fma(s, ld2(X, base + c));
    }
  }
  const long long o = static_cast<long long>(row) * width;
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    const int c = lane + t * G;
    if (c < width) {
      if (accumulate) acc[t].add(ld2(Y, o + c));
      st2(Y, o + c, acc[t].value());
    }
  }
}

// ---------------------------------------------------------------- U = Xp + V Y
template <int CPT>
__global__ void __launch_bounds__(kThreads) k_recombine_df2(int n, const float2* __restrict__ Xp,
                                                            const float2* __restrict__ V,
                                                            const double* __restrict__ Y, int q,
                                                            float2* __restrict__ U, int G) {
  extern __shared__ df dsm[];  // Y (q x q) then the block's V rows
  df* ys = dsm;
  df* vs = dsm + q * q;
  const int rpb = blockDim.x / G;
  for (int i = threadIdx.x; i < q * q; i += blockDim.x) ys[i] = df_from_double(Y[i]);
  const long long row0 = static_cast<long long>(blockIdx.x) * rpb;
  for (int i = threadIdx.x; i < rpb * q; i += blockDim.x) {
    const long long r = row0 + i / q;
    vs[i] = (r < n) ? ld2(V, r * q + i % q) : df{0.f, 0.f};
  }
  __syncthreads();
  const int g = threadIdx.x / G;
  const int lane = threadIdx.x % G;
  const long long row = row0 + g;
  if (row >= n) return;
  const long long base = row * q;
  df_acc acc[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    const int c = lane + t * G;
    acc[t] = acc_zero();
    if (c < q) acc[t].add(ld2(Xp, base + c));
  }
  const df* vr = vs + g * q;
  for (int d = 0; d < q; ++d) {
    const df v = vr[d];
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      const int c = lane + t * G;
      if (c < q) acc[t].fma(v, ys[d * q + c]);
    }
  }
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    const int c = lane + t * G;
    if (c < q) st2(U, base + c, acc[t].value());
  }
}

// Register-tiled form for wide blocks (32 < q <= 128): a block of 256 threads
// takes 32 rows; thread t computes 2 rows (t / 16 and t / 16 + 16) times the
// columns t % 16, t % 16 + 16, ... (CJ of them), so each Y value read from
// shared memory feeds two compensated products and each V value CJ: 2 CJ
// independent accumulators per thread hide the float-float dependency chains.
// Same sums in the same order (Xp, then d = 0 .. q-1) as k_recombine_df2.
constexpr int kRtRows = 32, kRtCols = 16;
template <int CJ>
__global__ void __launch_bounds__(kThreads) k_recombine_tiled(int n, const float2* __restrict__ Xp,
                                                              const float2* __restrict__ V,
                                                              const double* __restrict__ Y, int q,
                                                              float2* __restrict__ U) {
  extern __shared__ __align__(16) df tsm[];  // Y (q x q) then the block's V rows (kRtRows x q)
  df* ys = tsm;
  df* vs = tsm + q * q;
  for (int i = threadIdx.x; i < q * q; i += blockDim.x) ys[i] = df_from_double(Y[i]);
  const long long row0 = static_cast<long long>(blockIdx.x) * kRtRows;
  for (int i = threadIdx.x; i < kRtRows * q; i += blockDim.x) {
    const long long r = row0 + i / q;
    vs[i] = (r < n) ? ld2(V, r * q + i % q) : df{0.f, 0.f};
  }
  __syncthreads();
  const int cg = threadIdx.x % kRtCols, rp = threadIdx.x / kRtCols;
  const int ra = rp, rb = rp + kRtRows / 2;
  const long long rowa = row0 + ra, rowb = row0 + rb;
  df_acc acc[2][CJ];
#pragma unroll
  for (int j = 0; j < CJ; ++j) {
    const int c = cg + j * kRtCols;
    acc[0][j] = acc_zero();
    acc[1][j] = acc_zero();
    if (c < q) {
      if (rowa < n) acc[0][j].add(ld2(Xp, rowa * q + c));
      if (rowb < n) acc[1][j].add(ld2(Xp, rowb * q + c));
    }
  }
  const df* va = vs + ra * q;
  const df* vb = vs + rb * q;
  for (int d = 0; d < q; ++d) {
    const df x0 = va[d], x1 = vb[d];
    const df* yr = ys + d * q;
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      const int c = cg + j * kRtCols;
      if (c < q) {
        const df y = yr[c];
        acc[0][j].fma(x0, y);
        acc[1][j].fma(x1, y);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < CJ; ++j) {
    const int c = cg + j * kRtCols;
    if (c >= q) continue;
    if (rowa < n) st2(U, rowa * q + c, acc[0][j].value());
    if (rowb < n) st2(U, rowb * q + c, acc[1][j].value());
  }
}

// The same product with Y streamed: Y (already float-float, q x q) passes
// through shared memory in chunks of kKbChunk rows by bulk copies, two chunks
// in flight, and the block's 32 rows of V arrive by one bulk copy, so a block
// holds 32 q + 32 q values instead of q^2 + 32 q and three blocks share an SM.
// Needs even q and 16-byte aligned V, Ydf.  Same thread layout, same sums in
// the same order (Xp, then d = 0 .. q-1) as k_recombine_tiled.
constexpr int kKbChunk = 16;
template <int CJ>
__global__ void __launch_bounds__(kThreads, 3) k_recombine_kb(int n, const float2* __restrict__ Xp,
                                                              const float2* __restrict__ V,
                                                              const float2* __restrict__ Ydf, int q,
                                                              float2* __restrict__ U, int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char kraw[];
  __shared__ __align__(8) unsigned long long bar[3];  // [0], [1]: chunks of Y; [2]: the rows of V
  __shared__ int ok_s;
  float2* vs = reinterpret_cast<float2*>(kraw);  // kRtRows x q
  float2* ys = vs + kRtRows * q;                 // 2 x kKbChunk x q
  const int tid = threadIdx.x;
  const long long row0 = static_cast<long long>(blockIdx.x) * kRtRows;
  const int nr = static_cast<int>(min(static_cast<long long>(kRtRows), n - row0));
  const int nch = (q + kKbChunk - 1) / kKbChunk;
  auto issue = [&](int c) {  // thread 0: chunk c of Y into buffer c % 2
    const int d0 = c * kKbChunk, dk = min(kKbChunk, q - d0);
    const unsigned bytes = static_cast<unsigned>(sizeof(float2) * dk * q);
    mbar_expect_tx(&bar[c & 1], bytes);
    bulk_g2s(ys + (c & 1) * kKbChunk * q, Ydf + static_cast<long long>(d0) * q, bytes, &bar[c & 1]);
  };
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) mbar_init(&bar[b], 1);
    mbar_init_fence();
    ok_s = 1;
    const unsigned vb = static_cast<unsigned>(sizeof(float2) * nr * q);
    mbar_expect_tx(&bar[2], vb);
    bulk_g2s(vs, V + row0 * q, vb, &bar[2]);
    for (int c = 0; c < 2 && c < nch; ++c) issue(c);
  }
  __syncthreads();
  const int cg = tid % kRtCols, rp = tid / kRtCols;
  const int ra = rp, rb = rp + kRtRows / 2;
  const long long rowa = row0 + ra, rowb = row0 + rb;
  df_acc acc[2][CJ];
#pragma unroll
  for (int j = 0; j < CJ; ++j) {
    const int c = cg + j * kRtCols;
    acc[0][j] = acc_zero();
    acc[1][j] = acc_zero();
    if (c < q) {
      if (rowa < n) acc[0][j].add(ld2(Xp, rowa * q + c));
      if (rowb < n) acc[1][j].add(ld2(Xp, rowb * q + c));
    }
  }
  int failed = -1;  // first wait that expired: -2 the rows of V, c >= 0 chunk c
  if (tid == 0 && !mbar_wait_bounded(&bar[2], 0u)) ok_s = 0;
  __syncthreads();
  if (!ok_s) {
    failed = -2;
  } else {
    mbar_try_wait(&bar[2], 0u);
    for (int c = 0; c < nch; ++c) {
      const unsigned parity = static_cast<unsigned>((c >> 1) & 1);
      if (tid == 0 && !mbar_wait_bounded(&bar[c & 1], parity)) ok_s = 0;
      __syncthreads();
      if (!ok_s) {
        failed = c;
        break;
      }
      mbar_try_wait(&bar[c & 1], parity);
      const float2* yc = ys + (c & 1) * kKbChunk * q;
      const int d0 = c * kKbChunk, dk = min(kKbChunk, q - d0);
      for (int dd = 0; dd < dk; ++dd) {
        const int d = d0 + dd;
        const df x0 = ld2(vs, ra * q + d), x1 = ld2(vs, rb * q + d);
        const float2* yr = yc + dd * q;
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
          const int c2 = cg + j * kRtCols;
          if (c2 < q) {
            const df y = ld2(yr, c2);
            acc[0][j].fma(x0, y);
            acc[1][j].fma(x1, y);
          }
        }
      }
      __syncthreads();  // buffer c % 2 is free again
      if (tid == 0 && c + 2 < nch) issue(c + 2);
    }
  }
  if (failed != -1) {
    // a copy did not land in time: report it, give the copies still in flight another bounded wait, stop
    if (tid == 0) {
      if (status) atomicExch(status, AMGEIG_ECUDA);
      if (failed == -2) mbar_wait_bounded(&bar[2], 0u);
      const int c0 = failed == -2 ? 0 : failed;
      for (int c = c0; c < c0 + 2 && c < nch; ++c)
        mbar_wait_bounded(&bar[c & 1], static_cast<unsigned>((c >> 1) & 1));
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < CJ; ++j) {
    const int c = cg + j * kRtCols;
    if (c >= q) continue;
    if (rowa < n) st2(U, rowa * q + c, acc[0][j].value());
    if (rowb < n) st2(U, rowb * q + c, acc[1][j].value());
  }
}

// Row-per-thread form for q <= Q <= 32: each thread keeps all Q accumulators of
// its row in registers, so one V value feeds Q compensated products and the
// rows of Y (zero-padded to Q columns, shared) are read as 16-byte broadcasts.
template <int Q>
__global__ void __launch_bounds__(kThreads) k_recombine_rows(int n, const float2* __restrict__ Xp,
                                                             const float2* __restrict__ V,
                                                             const double* __restrict__ Y, int q,
                                                             float2* __restrict__ U) {
  __shared__ __align__(16) float2 ys[Q * Q];
  for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) {
    const int d = i / Q, c = i % Q;
    const df v = (d < q && c < q) ? df_from_double(Y[d * q + c]) : df{0.f, 0.f};
    ys[i] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  const long long row = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const long long base = row * q;
  df_acc acc[Q];
#pragma unroll
  for (int c = 0; c < Q; ++c) {
    acc[c] = acc_zero();
    if (c < q) acc[c].add(ld2(Xp, base + c));
  }
  for (int d = 0; d < q; ++d) {
    const df v = ld2(V, base + d);
    const float4* yr = reinterpret_cast<const float4*>(ys + d * Q);
#pragma unroll
    for (int c = 0; c < Q; c += 2) {
      const float4 y2 = yr[c / 2];
      acc[c].fma(v, df{y2.x, y2.y});
      acc[c + 1].fma(v, df{y2.z, y2.w});
    }
  }
#pragma unroll
  for (int c = 0; c < Q; ++c)
    if (c < q) st2(U, base + c, acc[c].value());
}

// U = I_n^k Xc + V Y with the composite prolongation I_n^k (CSR, float-float
// values) applied row by row: the prolongation chain and its intermediate
// blocks disappear; each thread owns one row and all Q accumulators.
// V has nv >= q columns (a Krylov block wider than the pairs: nv <= 2 Q) and Y is nv x q
template <int Q>
__global__ void __launch_bounds__(kThreads) k_recombine_pc(int n, const int* __restrict__ rp,
                                                           const int* __restrict__ ci, const float2* __restrict__ pv,
                                                           const float2* __restrict__ Xc,
                                                           const float2* __restrict__ V,
                                                           const double* __restrict__ Y, int q,
                                                           float2* __restrict__ U, int nv) {
  __shared__ __align__(16) float2 ys[2 * Q * Q];
  for (int i = threadIdx.x; i < nv * Q; i += blockDim.x) {
    const int d = i / Q, c = i % Q;
    const df v = (c < q) ? df_from_double(Y[d * q + c]) : df{0.f, 0.f};
    ys[i] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  const long long row = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const long long base = row * q;
  df_acc acc[Q];
#pragma unroll
  for (int c = 0; c < Q; ++c) acc[c] = acc_zero();
  const int p0 = rp[row], p1 = rp[row + 1];
  for (int p = p0; p < p1; ++p) {
    const df w = ld2(pv, p);
    const long long xr = static_cast<long long>(ci[p]) * q;
#pragma unroll
    for (int c = 0; c < Q; ++c)
      if (c < q) acc[c].fma(w, ld2(Xc, xr + c));
  }
  for (int d = 0; d < nv; ++d) {
    const df v = ld2(V, row * nv + d);
    const float4* yr = reinterpret_cast<const float4*>(ys + d * Q);
#pragma unroll
    for (int c = 0; c < Q; c += 2) {
      const float4 y2 = yr[c / 2];
      acc[c].fma(v, df{y2.x, y2.y});
      acc[c + 1].fma(v, df{y2.z, y2.w});
    }
  }
#pragma unroll
  for (int c = 0; c < Q; ++c)
    if (c < q) st2(U, base + c, acc[c].value());
}

// ---------------------------------------------------------------- Gram V^T W (df inputs)
// G = V^T [A V | M V] (q x 2q).  Both halves are symmetric, so only the pairs
// a <= b of each half are formed: np = q (q + 1) pairs.  A block stages a slab
// of rows of V and W in shared memory; thread t owns pairs t, t + blockDim, ...
constexpr int kGramRows = 16;
constexpr int kGramThreads = 320;
constexpr int kGramMaxPairs = 4;  // pairs per thread: q (q+1) <= 4 * 320 -> q <= 35

__device__ __forceinline__ void pair_of(int idx, int q, int* half, int* a, int* b) {
  // idx in [0, q(q+1)): half = idx / T, then the (a, b) with a <= b of the upper triangle
  const int T = q * (q + 1) / 2;
  *half = idx >= T;
  int r = idx - (*half) * T;
  int row = 0;
  while (r >= q - row) {
    r -= q - row;
    ++row;
  }
  *a = row;
  *b = row + r;
}

__global__ void __launch_bounds__(kGramThreads) k_gram_df_sym(int rows, const float2* __restrict__ V, int q,
                                                              const float2* __restrict__ W, int chunk_rows,
                                                              double* __restrict__ part) {
  extern __shared__ df gsm[];
  df* Vs = gsm;                  // kGramRows x q
  df* Ws = gsm + kGramRows * q;  // kGramRows x 2q
  const int np = q * (q + 1);
  int pa[kGramMaxPairs], pb[kGramMaxPairs];
  df_acc acc[kGramMaxPairs];
#pragma unroll
  for (int s = 0; s < kGramMaxPairs; ++s) {
    const int idx = threadIdx.x + s * blockDim.x;
    acc[s] = acc_zero();
    pa[s] = -1;
    pb[s] = 0;
    if (idx < np) {
      int half, a, b;
      pair_of(idx, q, &half, &a, &b);
      pa[s] = a;
      pb[s] = b + half * q;
    }
  }
  const int r0 = blockIdx.x * chunk_rows;
  const int r1 = min(rows, r0 + chunk_rows);
  for (int rb = r0; rb < r1; rb += kGramRows) {
    const int nr = min(kGramRows, r1 - rb);
    for (int i = threadIdx.x; i < nr * q; i += blockDim.x) Vs[i] = ld2(V, static_cast<long long>(rb) * q + i);
    for (int i = threadIdx.x; i < nr * 2 * q; i += blockDim.x)
      Ws[i] = ld2(W, static_cast<long long>(rb) * 2 * q + i);
    __syncthreads();
    for (int rr = 0; rr < nr; ++rr) {
#pragma unroll
      for (int s = 0; s < kGramMaxPairs; ++s)
        if (pa[s] >= 0) acc[s].fma(Vs[rr * q + pa[s]], Ws[rr * 2 * q + pb[s]]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < kGramMaxPairs; ++s) {
    const int idx = threadIdx.x + s * blockDim.x;
    if (idx < np) part[static_cast<long long>(blockIdx.x) * np + idx] = df_to_double(acc[s].value());
  }
}

// Register-tiled form of the same product for q <= 32: thread (g, t) owns the
// 4 x 4 output tile t of the upper triangle of one half (tiles (ta, tb) with
// ta <= tb, both halves: ntiles = T (T + 1), T = ceil(q / 4)) and accumulates
// rows g, g + rg, ... of each staged slab; 8 float-float loads feed 16
// compensated products.  The rg partial tiles are merged in a fixed order and
// written in the pair layout of k_gram_df_sym.
constexpr int kGtThreads = 256;

__global__ void __launch_bounds__(kGtThreads) k_gram_df_tiled(int rows, const float2* __restrict__ V, int q,
                                                              const float2* __restrict__ W, int chunk_rows,
                                                              int T, int rg, int slab, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char graw[];
  const int qp = 4 * T;
  float2* Vs = reinterpret_cast<float2*>(graw);  // slab x qp
  float2* Ws = Vs + slab * qp;                   // slab x 2 qp
  const int ntiles = T * (T + 1);
  const int tid = threadIdx.x;
  const int t = tid % ntiles, g = tid / ntiles;
  const bool active = g < rg;
  // tile t -> half, (ta, tb) with ta <= tb
  const int half = t >= T * (T + 1) / 2;
  int r = t - half * (T * (T + 1) / 2), ta = 0;
  while (r >= T - ta) {
    r -= T - ta;
    ++ta;
  }
  const int tb = ta + r;
  // staging roles, fixed per thread: (row offset, padded column) of V and of W
  const int vstep = blockDim.x / qp, vr0 = tid / qp, vc = tid % qp;
  const int wstep = blockDim.x / (2 * qp), wr0 = tid / (2 * qp), wc = tid % (2 * qp);
  const int whh = wc / qp, wcc = wc % qp;
  df_acc acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = acc_zero();
  const int r0 = blockIdx.x * chunk_rows;
  const int r1 = min(rows, r0 + chunk_rows);
  for (int rb = r0; rb < r1; rb += slab) {
    const int nr = min(slab, r1 - rb);
    if (vr0 < vstep)
      for (int rr = vr0; rr < nr; rr += vstep)
        Vs[rr * qp + vc] = vc < q ? V[static_cast<long long>(rb + rr) * q + vc] : make_float2(0.f, 0.f);
    if (wr0 < wstep)
      for (int rr = wr0; rr < nr; rr += wstep)
        Ws[rr * 2 * qp + wc] = wcc < q ? W[static_cast<long long>(rb + rr) * 2 * q + whh * q + wcc]
                                       : make_float2(0.f, 0.f);
    __syncthreads();
    if (active)
      for (int rr = g; rr < nr; rr += rg) {
        const float4* vp = reinterpret_cast<const float4*>(Vs + rr * qp + 4 * ta);
        const float4* wp = reinterpret_cast<const float4*>(Ws + rr * 2 * qp + half * qp + 4 * tb);
        const float4 v01 = vp[0], v23 = vp[1], w01 = wp[0], w23 = wp[1];
        const df v[4] = {df{v01.x, v01.y}, df{v01.z, v01.w}, df{v23.x, v23.y}, df{v23.z, v23.w}};
        const df w[4] = {df{w01.x, w01.y}, df{w01.z, w01.w}, df{w23.x, w23.y}, df{w23.z, w23.w}};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i * 4 + j].fma(v[i], w[j]);
      }
    __syncthreads();
  }
  // merge the rg row groups (shared memory reused; fixed order)
  df_acc* red = reinterpret_cast<df_acc*>(graw);  // rg x ntiles x 16
  if (active)
#pragma unroll
    for (int i = 0; i < 16; ++i) red[(g * ntiles + t) * 16 + i] = acc[i];
  __syncthreads();
  if (g == 0) {
    const int np = q * (q + 1);
    const int Tq = q * (q + 1) / 2;
    for (int i = 0; i < 16; ++i) {
      const int a = 4 * ta + i / 4, b = 4 * tb + i % 4;
      if (a >= q || b >= q || a > b) continue;
      df_acc s = red[t * 16 + i];
      for (int h = 1; h < rg; ++h) s.merge(red[(h * ntiles + t) * 16 + i]);
      const int idx = half * Tq + a * q - a * (a - 1) / 2 + (b - a);
      part[static_cast<long long>(blockIdx.x) * np + idx] = df_to_double(s.value());
    }
  }
}

// G (q x 2q) from the summed pairs, mirrored
__global__ void k_gram_unpack(const double* __restrict__ sums, int q, double* __restrict__ G) {
  const int np = q * (q + 1);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < np; idx += gridDim.x * blockDim.x) {
    int half, a, b;
    pair_of(idx, q, &half, &a, &b);
    const double v = sums[idx];
    G[a * 2 * q + half * q + b] = v;
    G[b * 2 * q + half * q + a] = v;
  }
}

int gram_chunks_df(int rows, int* chunk_rows) {
  int chunks = ceil_div(rows, 512);
  if (chunks > 4 * kNumSms) chunks = 4 * kNumSms;
  if (chunks < 1) chunks = 1;
  int cr = ceil_div(rows, chunks);
  cr = ceil_div(cr, kGramRows) * kGramRows;
  *chunk_rows = cr;
  return ceil_div(rows, cr) > 0 ? ceil_div(rows, cr) : 1;
}

// k_gram_df_tiled with its slabs staged by bulk copies, two slabs in flight:
// the copy of slab i + 2 starts as soon as the block has finished with slab i.
// Up to 32 columns one block holds every tile (rg row groups); wider blocks
// (up to 128 columns) give each thread one tile, tpb tiles per block and the
// tile list split over blockIdx.x; the blocks of one row chunk (blockIdx.y)
// are neighbours in launch order and stage the same slabs, mostly from L2.
// Slabs keep the global row layout (V rows of q, W rows of 2q float-float
// values), so q must be even (16-byte rows pairs) and V, W 16-byte aligned;
// the tile loads of a ragged last column tile read into the next row (or the
// 4-value pad after the slab) and feed only accumulators that are discarded.
// Same products in the same order as k_gram_df_tiled.
__global__ void __launch_bounds__(kGtThreads, 3) k_gram_df_bulk(int rows, const float2* __restrict__ V, int q,
                                                             const float2* __restrict__ W, int chunk_rows, int T,
                                                             int tpb, int rg, int slab, double* __restrict__ part,
                                                             int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char gbraw[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ int ok_s;
  const int stride = slab * 3 * q + 8;  // float2 per stage: V slab, W slab, pad
  float2* stage0 = reinterpret_cast<float2*>(gbraw);
  const int ntiles = T * (T + 1);
  const int tid = threadIdx.x;
  // rows: chunk blockIdx.y; tiles blockIdx.x * tpb .. + tpb; rg row groups of tpb threads
  const int lt = tid % tpb, g = tid / tpb;
  const int t = blockIdx.x * tpb + lt;
  const bool active = g < rg && t < ntiles;
  const int half = t >= T * (T + 1) / 2;
  int r = active ? t - half * (T * (T + 1) / 2) : 0, ta = 0;
  while (r >= T - ta) {
    r -= T - ta;
    ++ta;
  }
  const int tb = ta + r;
  df_acc acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = acc_zero();
  const int r0 = blockIdx.y * chunk_rows;
  const int r1 = min(rows, r0 + chunk_rows);
  const int nslab = r1 > r0 ? (r1 - r0 + slab - 1) / slab : 0;
  auto issue = [&](int i) {  // thread 0: slab i into stage i % 2
    const int rb = r0 + i * slab, nr = min(slab, r1 - rb);
    float2* Vs = stage0 + (i & 1) * stride;
    float2* Ws = Vs + slab * q;
    const unsigned bv = static_cast<unsigned>(sizeof(float2) * nr * q);
    mbar_expect_tx(&bar[i & 1], 3 * bv);
    bulk_g2s(Vs, V + static_cast<long long>(rb) * q, bv, &bar[i & 1]);
    bulk_g2s(Ws, W + static_cast<long long>(rb) * 2 * q, 2 * bv, &bar[i & 1]);
  };
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    ok_s = 1;
    for (int i = 0; i < 2 && i < nslab; ++i) issue(i);
  }
  __syncthreads();
  int failed = -1;
  for (int i = 0; i < nslab; ++i) {
    const unsigned parity = static_cast<unsigned>((i >> 1) & 1);
    if (tid == 0 && !mbar_wait_bounded(&bar[i & 1], parity)) ok_s = 0;
    __syncthreads();
    if (!ok_s) {
      failed = i;
      break;
    }
    mbar_try_wait(&bar[i & 1], parity);  // completed: each thread's own acquire of the copied bytes
    const int nr = min(slab, r1 - (r0 + i * slab));
    const float2* Vs = stage0 + (i & 1) * stride;
    const float2* Ws = Vs + slab * q;
    if (active)
      for (int rr = g; rr < nr; rr += rg) {
        const float4* vp = reinterpret_cast<const float4*>(Vs + rr * q + 4 * ta);
        const float4* wp = reinterpret_cast<const float4*>(Ws + rr * 2 * q + half * q + 4 * tb);
        const float4 v01 = vp[0], v23 = vp[1], w01 = wp[0], w23 = wp[1];
        const df v[4] = {df{v01.x, v01.y}, df{v01.z, v01.w}, df{v23.x, v23.y}, df{v23.z, v23.w}};
        const df w[4] = {df{w01.x, w01.y}, df{w01.z, w01.w}, df{w23.x, w23.y}, df{w23.z, w23.w}};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a * 4 + b].fma(v[a], w[b]);
      }
    __syncthreads();  // stage i % 2 is free again
    if (tid == 0 && i + 2 < nslab) issue(i + 2);
  }
  if (failed >= 0) {
    // a copy did not land in time: report it, give the copies still in flight (slabs failed and
    // failed + 1) another bounded wait, and stop
    if (tid == 0) {
      if (status) atomicExch(status, AMGEIG_ECUDA);
      for (int i = failed; i < failed + 2 && i < nslab; ++i)
        mbar_wait_bounded(&bar[i & 1], static_cast<unsigned>((i >> 1) & 1));
    }
    return;
  }
  // merge the rg row groups (shared memory reused; fixed order)
  df_acc* red = reinterpret_cast<df_acc*>(gbraw);  // rg x tpb x 16
  if (active)
#pragma unroll
    for (int i = 0; i < 16; ++i) red[(g * tpb + lt) * 16 + i] = acc[i];
  __syncthreads();
  if (g == 0 && active) {
    const int np = q * (q + 1);
    const int Tq = q * (q + 1) / 2;
    for (int i = 0; i < 16; ++i) {
      const int a = 4 * ta + i / 4, b = 4 * tb + i % 4;
      if (a >= q || b >= q || a > b) continue;
      df_acc s2 = red[lt * 16 + i];
      for (int h = 1; h < rg; ++h) s2.merge(red[(h * tpb + lt) * 16 + i]);
      const int idx = half * Tq + a * q - a * (a - 1) / 2 + (b - a);
      part[static_cast<long long>(blockIdx.y) * np + idx] = df_to_double(s2.value());
    }
  }
}

// general (non-symmetric-friendly) fallback for q > 35: 32 x 32 output tiles
constexpr int kGT = 32;
__global__ void __launch_bounds__(256) k_gram_df(int rows, const float2* __restrict__ V, int q,
                                                 const float2* __restrict__ W, int w, int chunk_rows, int tiles_w,
                                                 double* __restrict__ part) {
  __shared__ df Vs[32][kGT + 1];
  __shared__ df Ws[32][kGT + 1];
  const int chunk = blockIdx.x;
  const int ta = blockIdx.y / tiles_w, tb = blockIdx.y % tiles_w;
  const int a0 = ta * kGT, b0 = tb * kGT;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  df_acc acc[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) acc[s] = acc_zero();
  const int r0 = chunk * chunk_rows;
  const int r1 = min(rows, r0 + chunk_rows);
  for (int rb = r0; rb < r1; rb += 32) {
    for (int idx = threadIdx.x; idx < 32 * kGT; idx += blockDim.x) {
      const int rr = idx / kGT, cc = idx % kGT;
      const int r = rb + rr;
      Vs[rr][cc] = (r < r1 && a0 + cc < q) ? ld2(V, static_cast<long long>(r) * q + a0 + cc) : df{0.f, 0.f};
      Ws[rr][cc] = (r < r1 && b0 + cc < w) ? ld2(W, static_cast<long long>(r) * w + b0 + cc) : df{0.f, 0.f};
    }
    __syncthreads();
    const int nr = min(32, r1 - rb);
    for (int rr = 0; rr < nr; ++rr) {
      const df wv = Ws[rr][tx];
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[s].fma(Vs[rr][ty * 4 + s], wv);
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int a = a0 + ty * 4 + s, b = b0 + tx;
    if (a < q && b < w) part[(static_cast<long long>(chunk) * q + a) * w + b] = df_to_double(acc[s].value());
  }
}

// ---------------------------------------------------------------- conversions
__global__ void k_f64_to_df(const double* __restrict__ x, long long count, float2* __restrict__ y) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const df d = df_from_double(x[i]);
    y[i] = make_float2(d.hi, d.lo);
  }
}

__global__ void k_df_to_f64(const float2* __restrict__ x, long long count, double* __restrict__ y) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float2 v = x[i];
    y[i] = static_cast<double>(v.x) + static_cast<double>(v.y);
  }
}

// first columns of a row-major (rows x ld) float64 matrix into a rows x q df block
__global__ void k_cols_to_df(const double* __restrict__ src, int rows, int ld, int q, float2* __restrict__ dst) {
  const long long total = static_cast<long long>(rows) * q;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const df d = df_from_double(src[(i / q) * ld + i % q]);
    dst[i] = make_float2(d.hi, d.lo);
  }
}

int grid_for(long long count) {
  long long b = (count + kThreads - 1) / kThreads;
  if (b > 8LL * kNumSms) b = 8LL * kNumSms;
  return static_cast<int>(b < 1 ? 1 : b);
}

#define AMGEIG_DISPATCH(cpt, KERNEL, ...) \
  switch (cpt) {                          \
    case 1:                               \
      KERNEL<1> __VA_ARGS__;              \
      break;                              \
    case 2:                               \
      KERNEL<2> __VA_ARGS__;              \
      break;                              \
    case 3:                               \
      KERNEL<3> __VA_ARGS__;              \
      break;                              \
    case 4:                               \
      KERNEL<4> __VA_ARGS__;              \
      break;                              \
    case 5:                               \
      KERNEL<5> __VA_ARGS__;              \
      break;                              \
    case 6:                               \
      KERNEL<6> __VA_ARGS__;              \
      break;                              \
    case 7:                               \
      KERNEL<7> __VA_ARGS__;              \
      break;                              \
    case 8:                               \
      KERNEL<8> __VA_ARGS__;              \
      break;                              \
    default:                              \
      break;                              \
  }

// the same for kernels with a second template parameter PW = 1
#define AMGEIG_DISPATCH1(cpt, KERNEL, ...) \
  switch (cpt) {                          \
    case 1:                               \
      KERNEL<1, 1> __VA_ARGS__;              \
      break;                              \
    case 2:                               \
      KERNEL<2, 1> __VA_ARGS__;              \
      break;                              \
    case 3:                               \
      KERNEL<3, 1> __VA_ARGS__;              \
      break;                              \
    case 4:                               \
      KERNEL<4, 1> __VA_ARGS__;              \
      break;                              \
    case 5:                               \
      KERNEL<5, 1> __VA_ARGS__;              \
      break;                              \
    case 6:                               \
      KERNEL<6, 1> __VA_ARGS__;              \
      break;                              \
    case 7:                               \
      KERNEL<7, 1> __VA_ARGS__;              \
      break;                              \
    case 8:                               \
      KERNEL<8, 1> __VA_ARGS__;              \
      break;                              \
    default:                              \
      break;                              \
  }

}  // namespace

// Even q up to 128 with 16-byte aligned blocks: pairs of columns per 16-byte load, two pairs
// per lane, ceil(q / 4) lanes per row (pw = 2); otherwise the single-column layout of geo_for.
Geo geo_paired(int q, const void* X, const void* Y, int* pw) {
  const bool pair = q % 2 == 0 && q <= 128 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
  *pw = pair ? 2 : 1;
  if (!pair) return geo_for(q);
  const int G = (q + 3) / 4;
  return Geo{G, kThreads / G, 2};
}

void launch_defect_df(const DevCsr& AM, const float2* U, int q, const double* lam, float* R, int ldr,
                      double* partials, int* nblocks_out, cudaStream_t st) {
  int pw;
  Geo g = geo_paired(q, U, U, &pw);
  // one wave: four resident blocks per SM (the kernel's launch bound), grid-stride beyond
  int blocks = ceil_div(AM.rows, g.rows_per_block);
  if (blocks > 4 * kNumSms) blocks = 4 * kNumSms;
  if (nblocks_out) *nblocks_out = blocks;
  const size_t sm = partials ? sizeof(df_acc) * g.rows_per_block * 2 * g.G * g.cpt * pw : 0;
  const double N = AM.rows, nnz = AM.nnz;
  ProfScope ps(st, P_DEFECT, 4.0 * (N + 1) + 20.0 * nnz + 8.0 * N * q + 4.0 * N * ldr, 4.0 * nnz * q);
  if (pw == 2) {
    k_defect_df<2, 2><<<blocks, g.threads(), sm, st>>>(AM.rows, AM.rp, AM.ci, AM.d2, AM.m2, U, q, lam, R, ldr, g.G,
                                                       partials);
    return;
  }
  AMGEIG_DISPATCH1(g.cpt, k_defect_df,
                  <<<blocks, g.threads(), sm, st>>>(AM.rows, AM.rp, AM.ci, AM.d2, AM.m2, U, q, lam, R, ldr, g.G,
                                                      partials))
}

void launch_dual_spmm_df(const DevCsr& AM, const float2* V, int q, float2* W, cudaStream_t st) {
  int pw;
  Geo g = geo_paired(q, V, W, &pw);
  const int blocks = ceil_div(AM.rows, g.rows_per_block);
  const double N = AM.rows, nnz = AM.nnz;
  ProfScope ps(st, P_AUGMENT, 4.0 * (N + 1) + 20.0 * nnz + 8.0 * N * q + 16.0 * N * q, 4.0 * nnz * q);
  if (pw == 2) {
    k_dual_spmm_df<2, 2><<<blocks, g.threads(), 0, st>>>(AM.rows, AM.rp, AM.ci, AM.d2, AM.m2, V, q, W, g.G);
    return;
  }
  AMGEIG_DISPATCH1(g.cpt, k_dual_spmm_df,
                  <<<blocks, g.threads(), 0, st>>>(AM.rows, AM.rp, AM.ci, AM.d2, AM.m2, V, q, W, g.G))
}

void launch_spmm_df(const DevCsr& S, const float2* X, int width, float2* Y, bool accumulate, cudaStream_t st,
                    int cls) {
  if (S.rows == 0 || width == 0) return;
  Geo g = geo_for(width);
  const int blocks = ceil_div(S.rows, g.rows_per_block);
  ProfScope ps(st, cls,
               4.0 * (S.rows + 1) + 12.0 * S.nnz + 8.0 * S.cols * width + 8.0 * S.rows * width * (accumulate ? 2 : 1),
               2.0 * S.nnz * width);
  AMGEIG_DISPATCH(g.cpt, k_spmm_df,
                  <<<blocks, g.threads(), 0, st>>>(S.rows, S.rp, S.ci, S.d2, X, width, Y, g.G, accumulate ? 1 : 0))
}

void launch_recombine_pc_df(int rows, int nnz, const int* rp, const int* ci, const float2* pv, const float2* Xc,
                            const float2* V, const double* Y, int q, float2* U, cudaStream_t st, int nv) {
  if (rows <= 0 || q <= 0) return;
  if (nv <= 0) nv = q;
  ProfScope ps(st, P_RECOMBINE, 8.0 * rows * (q + nv) + 8.0 * nv * q + 4.0 * (rows + 1) + 12.0 * nnz,
               2.0 * rows * nv * q + 2.0 * nnz * q);
  const int blocks = ceil_div(rows, kThreads);
  if (q <= 8)
    k_recombine_pc<8><<<blocks, kThreads, 0, st>>>(rows, rp, ci, pv, Xc, V, Y, q, U, nv);
  else if (q <= 16)
    k_recombine_pc<16><<<blocks, kThreads, 0, st>>>(rows, rp, ci, pv, Xc, V, Y, q, U, nv);
  else if (q <= 20)
    k_recombine_pc<20><<<blocks, kThreads, 0, st>>>(rows, rp, ci, pv, Xc, V, Y, q, U, nv);
  else if (q <= 24)
    k_recombine_pc<24><<<blocks, kThreads, 0, st>>>(rows, rp, ci, pv, Xc, V, Y, q, U, nv);
  else if (q <= 28)
    k_recombine_pc<28><<<blocks, kThreads, 0, st>>>(rows, rp, ci, pv, Xc, V, Y, q, U, nv);
  else
    k_recombine_pc<32><<<blocks, kThreads, 0, st>>>(rows, rp, ci, pv, Xc, V, Y, q, U, nv);
}

void launch_recombine_df(int rows, const float2* Xp, const float2* V, const double* Y, int q, float2* U,
                         cudaStream_t st, float2* Ydf, int* status) {
  if (rows <= 0 || q <= 0) return;
  if (q <= 32) {
    ProfScope ps(st, P_RECOMBINE, 24.0 * rows * q + 8.0 * q * q, 2.0 * rows * q * q);
    const int blocks = ceil_div(rows, kThreads);
    if (q <= 8)
      k_recombine_rows<8><<<blocks, kThreads, 0, st>>>(rows, Xp, V, Y, q, U);
    else if (q <= 16)
      k_recombine_rows<16><<<blocks, kThreads, 0, st>>>(rows, Xp, V, Y, q, U);
    else if (q <= 24)
      k_recombine_rows<24><<<blocks, kThreads, 0, st>>>(rows, Xp, V, Y, q, U);
    else if (q <= 28)
      k_recombine_rows<28><<<blocks, kThreads, 0, st>>>(rows, Xp, V, Y, q, U);
    else
      k_recombine_rows<32><<<blocks, kThreads, 0, st>>>(rows, Xp, V, Y, q, U);
    return;
  }
  if (q <= 128 && Ydf != nullptr && q % 2 == 0 && (reinterpret_cast<uintptr_t>(V) & 15) == 0 &&
      (reinterpret_cast<uintptr_t>(Ydf) & 15) == 0) {
    // Y to float-float once, then streamed through shared memory by the blocks
    const int blocks = ceil_div(rows, kRtRows);
    ProfScope ps(st, P_RECOMBINE, 24.0 * rows * q + 8.0 * q * q, 2.0 * rows * q * q, 2);
    const long long qq = static_cast<long long>(q) * q;
    k_f64_to_df<<<ceil_div(qq, kThreads), kThreads, 0, st>>>(Y, qq, Ydf);
    const size_t sm = sizeof(float2) * (static_cast<size_t>(kRtRows) * q + 2 * static_cast<size_t>(kKbChunk) * q);
#define AMGEIG_KB(CJ)                                                                     \
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_recombine_kb<CJ>), sm);             \
  k_recombine_kb<CJ><<<blocks, kThreads, sm, st>>>(rows, Xp, V, Ydf, q, U, status)
    if (q <= 3 * kRtCols) {
      AMGEIG_KB(3);
    } else if (q <= 5 * kRtCols) {
      AMGEIG_KB(5);
    } else {
      AMGEIG_KB(8);
    }
#undef AMGEIG_KB
    return;
  }
  if (q <= 128) {
    const int blocks = ceil_div(rows, kRtRows);
    ProfScope ps(st, P_RECOMBINE, 24.0 * rows * q + 8.0 * q * q, 2.0 * rows * q * q);
    const size_t sm = sizeof(df) * (static_cast<size_t>(q) * q + static_cast<size_t>(kRtRows) * q);
#define AMGEIG_TILED(CJ)                                                                     \
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_recombine_tiled<CJ>), sm);             \
  k_recombine_tiled<CJ><<<blocks, kThreads, sm, st>>>(rows, Xp, V, Y, q, U)
    if (q <= 3 * kRtCols) {
      AMGEIG_TILED(3);
    } else if (q <= 5 * kRtCols) {
      AMGEIG_TILED(5);
    } else {
      AMGEIG_TILED(8);
    }
#undef AMGEIG_TILED
    return;
  }
  Geo g = geo_for(q);
  const int blocks = ceil_div(rows, g.rows_per_block);
  ProfScope ps(st, P_RECOMBINE, 24.0 * rows * q + 8.0 * q * q, 2.0 * rows * q * q);
  const size_t sm = sizeof(df) * (static_cast<size_t>(q) * q + static_cast<size_t>(g.rows_per_block) * q);
  switch (g.cpt) {
#define AMGEIG_CASE(C)                                                                              \
  case C:                                                                                           \
    if (sm > 48 * 1024)                                                                             \
      ensure_dynamic_smem(reinterpret_cast<const void*>(k_recombine_df2<C>), sm);            \
    k_recombine_df2<C><<<blocks, g.threads(), sm, st>>>(rows, Xp, V, Y, q, U, g.G);                      \
    break;
    AMGEIG_CASE(1)
    AMGEIG_CASE(2)
    AMGEIG_CASE(3)
    AMGEIG_CASE(4)
    AMGEIG_CASE(5)
    AMGEIG_CASE(6)
    AMGEIG_CASE(7)
    AMGEIG_CASE(8)
#undef AMGEIG_CASE
    default:
      break;
  }
}

size_t gram_df_scratch_doubles(int rows, int q, int w) {
  int cr;
  const size_t chunks = static_cast<size_t>(gram_chunks_df(rows, &cr));
  // symmetric kernel: chunks x q(q+1) partials + q(q+1) sums; tiled kernel: chunks x q x w
  return chunks * q * w + static_cast<size_t>(q) * (q + 1);
}

void launch_gram_df(int rows, const float2* V, int q, const float2* W, int w, double* scratch, double* G,
                    cudaStream_t st, int* status) {
  if (q <= 0 || w <= 0) return;
  int cr;
  const int chunks = gram_chunks_df(rows, &cr);
  // bulk-copy staging keeps the global row layout: even q and 16-byte aligned V, W
  const bool bulk = q % 2 == 0 && (reinterpret_cast<uintptr_t>(V) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(W) & 15) == 0;
  if (w == 2 * q && (q <= 32 || (bulk && q <= 128))) {
    const int T = (q + 3) / 4, ntiles = T * (T + 1);
    int tpb, rg, ny, slab;
    if (q <= 32) {
      tpb = ntiles;
      rg = kGtThreads / ntiles;
      ny = 1;
      // up to 8 rows per group, staged slab within 40 KB of shared memory
      const int rpg = std::max(1, std::min(8, 40960 / (rg * 96 * T)));
      slab = rg * rpg;
    } else {
      tpb = kGtThreads;
      rg = 1;
      ny = ceil_div(ntiles, tpb);
      slab = std::max(8, std::min(32, 24576 / (24 * q)));  // about 24 KB of rows per stage
    }
    int chunks2 = ceil_div(rows, slab);
    if (chunks2 > 3 * kNumSms) chunks2 = 3 * kNumSms;
    int cr2 = ceil_div(ceil_div(rows, chunks2), slab) * slab;
    chunks2 = ceil_div(rows, cr2);
    if (chunks2 > chunks) chunks2 = chunks;  // scratch is sized for gram_chunks_df
    cr2 = ceil_div(ceil_div(rows, chunks2), slab) * slab;
    chunks2 = ceil_div(rows, cr2);
    const int np = q * (q + 1);
    ProfScope ps(st, P_GRAM, 8.0 * rows * (q + w) + 16.0 * chunks2 * np, 1.0 * rows * np * 2.0);
    const size_t merge = sizeof(df_acc) * rg * tpb * 16;
    if (bulk) {
      const size_t stages = sizeof(float2) * 2 * (static_cast<size_t>(slab) * 3 * q + 8);
      const size_t sm = stages > merge ? stages : merge;
      ensure_dynamic_smem(reinterpret_cast<const void*>(k_gram_df_bulk), sm);
      k_gram_df_bulk<<<dim3(ny, chunks2), kGtThreads, sm, st>>>(rows, V, q, W, cr2, T, tpb, rg, slab, scratch,
                                                                status);
    } else {
      const size_t stage = sizeof(float2) * slab * 3 * 4 * T;
      const size_t sm = stage > merge ? stage : merge;
      k_gram_df_tiled<<<chunks2, kGtThreads, sm, st>>>(rows, V, q, W, cr2, T, rg, slab, scratch);
    }
    double* sums = scratch + static_cast<size_t>(chunks2) * np;
    launch_sum_partials(scratch, chunks2, np, sums, st);
    k_gram_unpack<<<ceil_div(np, 256), 256, 0, st>>>(sums, q, G);
    return;
  }
  if (w == 2 * q && q * (q + 1) <= kGramMaxPairs * kGramThreads) {
    const int np = q * (q + 1);
    ProfScope ps(st, P_GRAM, 8.0 * rows * (q + w) + 16.0 * chunks * np, 1.0 * rows * np * 2.0);
    const size_t sm = sizeof(df) * kGramRows * 3 * q;
    k_gram_df_sym<<<chunks, kGramThreads, sm, st>>>(rows, V, q, W, cr, scratch);
    double* sums = scratch + static_cast<size_t>(chunks) * np;
    launch_sum_partials(scratch, chunks, np, sums, st);
    k_gram_unpack<<<ceil_div(np, 256), 256, 0, st>>>(sums, q, G);
    return;
  }
  const int tiles_w = ceil_div(w, kGT);
  dim3 grid(chunks, ceil_div(q, kGT) * tiles_w);
  ProfScope ps(st, P_GRAM, 8.0 * rows * (q + w) + 16.0 * chunks * q * w, 2.0 * rows * q * w);
  k_gram_df<<<grid, 256, 0, st>>>(rows, V, q, W, w, cr, tiles_w, scratch);
  launch_sum_partials(scratch, chunks, q * w, G, st);
}

void launch_f64_to_df(const double* x, long long count, float2* y, cudaStream_t st) {
  ProfScope ps(st, P_OTHER, 16.0 * count, 0.0);
  k_f64_to_df<<<grid_for(count), kThreads, 0, st>>>(x, count, y);
}

void launch_df_to_f64(const float2* x, long long count, double* y, cudaStream_t st) {
  ProfScope ps(st, P_OTHER, 16.0 * count, 0.0);
  k_df_to_f64<<<grid_for(count), kThreads, 0, st>>>(x, count, y);
}

void launch_cols_to_df(const double* src, int rows, int ld, int q, float2* dst, cudaStream_t st) {
  const long long total = static_cast<long long>(rows) * q;
  ProfScope ps(st, P_OTHER, 16.0 * total, 0.0);
  k_cols_to_df<<<grid_for(total), kThreads, 0, st>>>(src, rows, ld, q, dst);
}

}  // namespace amgeig
