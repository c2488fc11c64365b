// Host-side launchers of the solve-path kernels (one declaration per kernel
// family; each launcher enqueues on `st` and returns without synchronising).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace amgeig {

// CSR matrix on the device.  vals64 / vals32 point to the same entries in
// float64 and float32 (either may be null when a path does not use it).
struct DevCsr {
  int rows = 0, cols = 0, nnz = 0;
  int* rp = nullptr;
  int* ci = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
  double* m64 = nullptr;  // second value array sharing the pattern (mass matrix)
  float2* d2 = nullptr;   // v64 as float-float pairs (hi, lo)
  float2* m2 = nullptr;   // m64 as float-float pairs
  __nv_bfloat16* vbf = nullptr;  // v64 rounded to bfloat16 (the V-cycle's operators, AMGEIG_MIXED_BF16)
  // launch shape of the float32 V-cycle kernels on this operator, per block width in float4
  // columns w4 <= 32, chosen by the autotuner: (log2 streams) << 5 | (log2 column lanes per
  // stream) << 2 | columns per lane; 0 = not tuned (the rule applies)
  unsigned char tuned[33] = {};
};

// ---- launch-shape autotuning of the float32 V-cycle kernels (spmm.cu) -------
// Times every lane layout (G lanes per row, cpt float4 columns per lane) of the
// smoothing sweep on A (kind 0: x_out = x + D^-1 (b - A x)) or of the transfer
// SpMM on S (kind 1: Y = S X) at width 4 * w4, and records the fastest in the
// operator's `tuned` table.  x / b / X and out / Y are device scratch of the
// operator's rows (or columns) x 4 w4 floats; their contents are overwritten.
struct TuneResult {
  int G = 0, cpt = 0, rule_G = 0, rule_cpt = 0, S = 1;
  float us = 0.f, rule_us = 0.f;
};
TuneResult autotune_f4(DevCsr& S, int kind, int w4, const float* dinv, const float* x, const float* b, float* out,
                       cudaStream_t st);

// ---- sparse kernels (spmm.cu) --------------------------------------------
// All blocks of vectors are row-major [rows][width].

// R = lambda o (M U) - A U   (Eq. Linear_Equation moved to the defect form),
// R written as TO; when `partials` is non-null each block also writes the
// per-column sums of R_ij^2 and (MU)_ij^2 to partials[block][2q] (fixed order).
void launch_defect_f64(const DevCsr& AM, const double* U, int q, const double* lam, double* R,
                       double* partials, int* nblocks_out, cudaStream_t st);
// float32 output with row stride ldr >= q; columns q..ldr-1 are written as zero
void launch_defect_f32out(const DevCsr& AM, const double* U, int q, const double* lam, float* R, int ldr,
                          double* partials, int* nblocks_out, cudaStream_t st);

// Y = S X (accumulate = false) or Y += S X (accumulate = true)
void launch_spmm_f64(const DevCsr& S, const double* X, int width, double* Y, bool accumulate, cudaStream_t st,
                     int cls = 2);
// bf16: read the operator's bfloat16 values (vbf) instead of the float32 ones
void launch_spmm_f32(const DevCsr& S, const float* X, int width, float* Y, bool accumulate, cudaStream_t st,
                     bool bf16 = false);

// first l1-Jacobi sweep from x = 0 fused with the residual:
//   x = D^-1 b,  r = b - A x
void launch_presmooth_residual_f64(const DevCsr& A, const double* dinv, const double* b, int width, double* x,
                                   double* r, cudaStream_t st);
void launch_presmooth_residual_f32(const DevCsr& A, const float* dinv, const float* b, int width, float* x,
                                   float* r, cudaStream_t st, bool bf16 = false);
// one l1-Jacobi sweep x_out = x + D^-1 (b - A x) (x_out != x)
void launch_jacobi_f64(const DevCsr& A, const double* dinv, const double* b, const double* x, int width,
                       double* x_out, cudaStream_t st);
void launch_jacobi_f32(const DevCsr& A, const float* dinv, const float* b, const float* x, int width,
                       float* x_out, cudaStream_t st, bool bf16 = false);
// residual r = b - A x
void launch_residual_f64(const DevCsr& A, const double* b, const double* x, int width, double* r, cudaStream_t st);
void launch_residual_f32(const DevCsr& A, const float* b, const float* x, int width, float* r, cudaStream_t st,
                         bool bf16 = false);
// last sweep on the working level fused with V = U + x_new (float64 output)
void launch_jacobi_to_v_f64(const DevCsr& A, const double* dinv, const double* b, const double* x, int width,
                            const double* U, double* V, cudaStream_t st);
// float32 variant: b and x have row stride `width` (a multiple of 4 when padded),
// U and V have row stride qv <= width
void launch_jacobi_to_v_f32(const DevCsr& A, const float* dinv, const float* b, const float* x, int width,
                            const double* U, double* V, cudaStream_t st, int qv);
// V = U + x (used when there are no post-smoothing sweeps)
void launch_add_to_v_f64(const double* U, const double* x, long long count, double* V, cudaStream_t st);
void launch_add_to_v_f32(const double* U, const float* x, long long count, double* V, cudaStream_t st);
// V = U + x with x of row stride ldx >= q (rows x q)
void launch_add_to_v_f32_strided(const double* U, const float* x, int rows, int q, int ldx, double* V, cudaStream_t st);
// padded float32 copies: dst (rows x ld) = src (rows x q), zero padding; and back
void launch_f64_to_f32_pad(const double* src, int rows, int q, int ld, float* dst, cudaStream_t st);
void launch_f32_to_f64_unpad(const float* src, int rows, int q, int ld, double* dst, cudaStream_t st);

// W = [A V | M V]  ([rows][2q])
void launch_dual_spmm(const DevCsr& AM, const double* V, int q, double* W, cudaStream_t st);

// U = Xp + V Y   (Y: q x q row-major); df_arith as for the Gram
void launch_recombine(int rows, const double* Xp, const double* V, const double* Y, int q, double* U,
                      cudaStream_t st, bool df_arith = false);
// the same with V of nv columns (a Krylov block) and Y nv x q (float64)
void launch_recombine_wide(int rows, const double* Xp, const double* V, int nv, const double* Y, int q, double* U,
                           cudaStream_t st);
// Krylov block K = [V1 | E] (rows x 2q) from V1 (rows x q) and the correction E (rows x q, row stride lde)
void launch_pack_krylov_f64(int rows, const double* V1, const double* E, int lde, int q, double* K, cudaStream_t st);
void launch_pack_krylov_df(int rows, const float2* V1, const float* E, int lde, int q, float2* K, cudaStream_t st);

// z = x + alpha y (elementwise; z may alias neither)
void launch_axpby_f64(const double* x, double alpha, const double* y, long long count, double* z, cudaStream_t st);
// y += x
void launch_axpy_f64(const double* x, long long count, double* y, cudaStream_t st);
void launch_axpy_f32(const float* x, long long count, float* y, cudaStream_t st);

// float64 -> float32 / float32 -> float64 copies
void launch_convert_f64_to_f32(const double* x, long long count, float* y, cudaStream_t st);
// l1-Jacobi inverse diagonal 1 / sum_j |a_ij| of A (float64 and float32 copies);
// *zero_row (device) is set to 1 when a row sum is not positive
void launch_l1_inv_diag(const DevCsr& A, double* d64, float* d32, int* zero_row, cudaStream_t st);
// One level of the composite prolongation I_n^k = P_k I_n^{k+1} (next: CSR with
// d_n columns, float64 values).  out_rp null: counts[i] = nonzeros of row i;
// otherwise rows i fill out_ci / out_v from out_rp[i] in column order.
void launch_composite_rows(const DevCsr& P, const int* nrp, const int* nci, const double* nv, int dn,
                           const int* out_rp, int* counts, int* out_ci, double* out_v, cudaStream_t st);
// One colour of a multicolour Gauss-Seidel sweep: the cnt rows listed in `rows`
// (no two adjacent) update x_i += (b_i - sum_j a_ij x_j) * dinv_i on w columns of
// row-major blocks with row stride ld.  `bytes` is the launch's share of the
// sweep's algorithmic traffic.
void launch_gs_colour(int cnt, const int* rows, const DevCsr& A, const double* dinv, const double* b, double* x,
                      int ld, int w, double bytes, cudaStream_t st);
void launch_gs_colour(int cnt, const int* rows, const DevCsr& A, const float* dinv, const float* b, float* x, int ld,
                      int w, double bytes, cudaStream_t st);
void launch_convert_f32_to_f64(const float* x, long long count, double* y, cudaStream_t st);

// ---- final float64 Rayleigh-quotient refinement (refine.cu) --------------
// sums[5q]: per column u^T A u, u^T M u, |Au|^2, (Au)^T Mu and |Mu|^2 (float64,
// exact operator values; `compensated`: the first two accumulated in
// compensated arithmetic, as if in twice the working precision), through
// per-block partials (scratch of rayleigh_blocks() x 7q doubles); q <= 128.
int rayleigh_blocks(int q);
void launch_rayleigh_f64(const DevCsr& AM, const double* U, int q, bool compensated, double* partials,
                         double* sums, cudaStream_t st);
// theta_j = u^T A u / u^T M u; lam = theta sorted ascending, perm[c] = column of the c-th smallest;
// relres_j from the expanded residual norm; flag[0] = 1 when the expansion cancelled too far to be
// trusted (form the residual explicitly), 2 on a NaN or Inf
void launch_rq_finish(const double* sums, int q, double* theta, double* lam, int* perm, double* relres, int* flag,
                      cudaStream_t st);
// dst (rows x q) = columns perm[0..q) of src (rows x ld)
void launch_gather_cols(const double* src, int rows, int ld, const int* perm, int q, double* dst, cudaStream_t st);

// ---- float-float kernels of the mixed path (spmm_df.cu) -------------------
// Blocks are float2 (hi, lo) pairs, row-major like the float64 blocks.
void launch_defect_df(const DevCsr& AM, const float2* U, int q, const double* lam, float* R, int ldr,
                      double* partials, int* nblocks_out, cudaStream_t st);
void launch_dual_spmm_df(const DevCsr& AM, const float2* V, int q, float2* W, cudaStream_t st);
void launch_spmm_df(const DevCsr& S, const float2* X, int width, float2* Y, bool accumulate, cudaStream_t st,
                    int cls);
// U = PC Xc + V Y with PC (CSR rows x d_n, float-float values) the composite
// prolongation I_n^k and Xc (d_n x q) float-float; q <= 32.  V has nv columns
// (0: q; a Krylov block: up to 2q) and Y is nv x q.
void launch_recombine_pc_df(int rows, int nnz, const int* rp, const int* ci, const float2* pv, const float2* Xc,
                            const float2* V, const double* Y, int q, float2* U, cudaStream_t st, int nv = 0);
// Ydf (q x q float-float, may be null): scratch for Y in float-float, which lets 32 < q <= 128 stream
// Y through shared memory; status as for launch_gram_df
void launch_recombine_df(int rows, const float2* Xp, const float2* V, const double* Y, int q, float2* U,
                         cudaStream_t st, float2* Ydf = nullptr, int* status = nullptr);
size_t gram_df_scratch_doubles(int rows, int q, int w);
// status (may be null): set to AMGEIG_ECUDA when a bulk copy into shared memory did not complete
// within the kernel's bounded wait
void launch_gram_df(int rows, const float2* V, int q, const float2* W, int w, double* scratch, double* G,
                    cudaStream_t st, int* status = nullptr);
void launch_f64_to_df(const double* x, long long count, float2* y, cudaStream_t st);
void launch_df_to_f64(const float2* x, long long count, double* y, cudaStream_t st);
void launch_cols_to_df(const double* src, int rows, int ld, int q, float2* dst, cudaStream_t st);
// last float32 sweep on the working level fused with V = U + x (U, V float-float,
// row stride qv; b and x row stride width)
void launch_jacobi_to_vdf_f32(const DevCsr& A, const float* dinv, const float* b, const float* x, int width,
                              const float2* U, float2* V, cudaStream_t st, int qv, const float* xadd = nullptr,
                              bool bf16 = false);
// float32 -> bfloat16 (round to nearest even)
void launch_f32_to_bf16(const float* x, long long count, __nv_bfloat16* y, cudaStream_t st);
// V = U + x (U, V float-float rows x q; x float32 with row stride ldx)
void launch_add_to_vdf(const float2* U, const float* x, int rows, int q, int ldx, float2* V, cudaStream_t st);

// ---- dense kernels (dense.cu) ---------------------------------------------

// C = alpha op(A) op(B) + beta C, all row-major; op = transpose when t* != 0.
// A is M x K (or K x M when ta), B is K x N (or N x K when tb).
// cls: the profiler class the launch is accounted to (prof.cuh; 8 = other)
// x = A b, A dense n x n row-major, b and x n x w row-major (w <= 256)
void launch_dense_apply(int n, int w, const double* A, const double* b, double* x, cudaStream_t st, int cls);
void launch_dense_apply(int n, int w, const float* A, const float* b, float* x, cudaStream_t st, int cls);
void launch_gemm_f64(int M, int N, int K, double alpha, const double* A, int lda, bool ta, const double* B,
                     int ldb, bool tb, double beta, double* C, int ldc, cudaStream_t st, int cls = 8);
void launch_gemm_f32(int M, int N, int K, float alpha, const float* A, int lda, bool ta, const float* B, int ldb,
                     bool tb, float beta, float* C, int ldc, cudaStream_t st, int cls = 8);

// Gram G = V^T W  (V: rows x q, W: rows x w) -> G: q x w, via per-chunk partials
// in `scratch` (size gram_scratch_doubles(rows, q, w)) and a fixed-order sum.
size_t gram_scratch_doubles(int rows, int q, int w);
// df_arith: products and sums in float-float on the float32 pipes (48-bit
// significand, compensated accumulation) instead of float64 FMA.
void launch_gram(int rows, const double* V, int q, const double* W, int w, double* scratch, double* G,
                 cudaStream_t st, bool df_arith = false);
// same with explicit row strides ldv >= q and ldw >= w
void launch_gram_strided(int rows, const double* V, int ldv, int q, const double* W, int ldw, int w, double* scratch,
                         double* G, cudaStream_t st, bool df_arith = false);


// Sum `nparts` partial rows of length `len` in fixed order: out[j] = sum_b part[b*len + j]
void launch_sum_partials(const double* part, int nparts, int len, double* out, cudaStream_t st);

// relres_j = sqrt(rr_j) / (|lambda_j| sqrt(mm_j)) from the summed defect norms;
// writes relres[q] and flags[0] = 1 if any value is NaN/Inf.
void launch_relres(const double* sums, const double* lam, int q, double* relres, int* flags, cudaStream_t st);

// Dense copies (rows x rows, row-major) of a square CSR's two value arrays
void launch_csr_to_dense(int rows, const int* rp, const int* ci, const double* a, const double* m, double* Ad,
                         double* Md, cudaStream_t st);

// Copy the first q columns of a row-major (rows x ld) matrix into a rows x q block
void launch_copy_cols(const double* src, int rows, int ld, int q, double* dst, cudaStream_t st);

// ---- small dense eigen-machinery (pencil.cu) ------------------------------

struct PencilWork;  // opaque device workspace, sized by pencil_work_create

// Workspace for pencils of coarse size dn with up to qmax border vectors.
// dry: size the workspace (PencilWork::bytes) without allocating it
PencilWork* pencil_work_create(int dn, int qmax, cudaError_t* err, bool dry = false);
// device bytes pencil_work_create(dn, qmax) allocates
size_t pencil_work_bytes(int dn, int qmax);
void pencil_work_destroy(PencilWork* w);

// One Rayleigh-Ritz step on V_n + span(V) (Algorithm 3.1 step 2) in the
// coarse eigenbasis: inputs C = [I_k^n A V | I_k^n M V] (dn x 2q, float64 in
// C64 or float-float in Cdf, the other null), G = [V^T A V | V^T M V] (q x 2q),
// the coarse eigenbasis Z (dn x dn, M_n-orthonormal, as float-float pairs Zdf)
// and Theta (dn).  The coarse part of the trial space is spanned by the first
// m <= dn columns of Z (m = dn: all of V_n).  Outputs the q smallest Ritz
// values mu (q), the coarse coefficients Xc (dn x q; also as float-float pairs
// in Xcdf when non-null) and the V-coefficients Y (q x q) so that the new
// vectors are I_n^k Xc + V Y.  status[0] receives AMGEIG_ENOTSPD when the Gram
// Schur complement is not positive definite.  nfallback (device, may be null)
// is incremented when the dense eigensolver had to run.
// p > 0 and p < q: a border of q columns (C: dn x 2q, G: q x 2q) of which the p smallest pairs are wanted
// (mu: p, Xc: dn x p, Y: q x p); the structured iteration is then not used.
void launch_pencil_solve(PencilWork* w, int dn, int m, int q, const double* C64, const float2* Cdf,
                         const double* G, const float2* Zdf, const double* theta, double* mu, double* Xc,
                         float2* Xcdf, double* Y, int* status, cudaStream_t st, int* nfallback = nullptr,
                         int p = 0);

// The float64 Cholesky factor M_n = L_m L_m^T into the workspace (the first step
// of launch_coarse_modes, and the check that M_n is positive definite: status =
// ENOTSPD otherwise).
void launch_mass_factor(PencilWork* w, int dn, const double* Mn, int* status, cudaStream_t st);
// The coarsest level's exact solve: Ainv = A_n^-1 (dn x dn, row-major) from the
// float64 Cholesky factor A_n = L L^T as L^-T L^-1; L and Linv are dn x dn
// scratch; status = ENOTSPD when A_n is not positive definite.  Independent of
// the workspace, so it can run beside launch_mass_factor / launch_coarse_modes.
void launch_coarse_inverse(int dn, const double* An, double* L, double* Linv, double* Ainv, int* status,
                           cudaStream_t st);
// The nwant lowest eigenpairs of the coarsest pencil (A_n, M_n) (needs the
// M_n factor of launch_mass_factor in the same workspace): the first nwant
// columns of Z (dn x dn row-major, stride dn) with Z^T M_n Z = I and
// Z^T A_n Z = diag(theta), theta ascending.
void launch_coarse_modes(PencilWork* w, int dn, int nwant, const double* An, double* Z, double* theta,
                         cudaStream_t st);

// Symmetric eigensolver in float-float: the `nwant` smallest eigenpairs of the
// symmetric n x n row-major float64 matrix H.  evals (nwant), evecs (n x nwant
// row-major).  Exposed for the kernel-level tests.
// skip (device, may be null): when *skip != 0 at run time the kernel returns at once
void launch_syev_df(PencilWork* w, int n, int nwant, const double* H, double* evals, double* evecs,
                    cudaStream_t st, const int* skip = nullptr);

// The same eigensolver on caller-provided workspace (device pointers sized as in
// pencil_work_create for nmax >= n + 1 and nwant_max >= nwant); enqueues only.
struct df;
void launch_syev_df_into(int n, int nwant, const double* H, double* evals, double* evecs, df* W, df* tau, df* dd,
                         df* ee, df* fac, df* Zt, df* rr, int* perm, cudaStream_t st);

// Hierarchy load on the device (the blob copied in one piece): *out += the word sum (mod 2^64) of
// `bytes` (a multiple of 8) at blob; *bad |= 1 unless (rp, ci) is a valid CSR structure of a
// rows x cols matrix with nnz entries; R = P^T (rows x cols P in, cols x rows R out, rows of R in
// ascending column order), scratch: cols ints.
void launch_blob_checksum(const void* blob, size_t bytes, unsigned long long* out, cudaStream_t st);
void launch_csr_check(const int* rp, const int* ci, long long rows, long long cols, long long nnz, int* bad,
                      cudaStream_t st);
// out[0] = 0, out[i + 1] = cnt[0] + .. + cnt[i] (int32; the exact total in *total when given);
// tmp: 1024 int64 of scratch (also for the transpose)
void launch_exclusive_scan(const int* cnt, long long n, int* out, long long* tmp, long long* total,
                           cudaStream_t st);
void launch_transpose_csr(long long rows, long long cols, long long nnz, const int* rp, const int* ci,
                          const double* v, int* rrp, int* rci, double* rv, int* scratch, long long* tmp,
                          cudaStream_t st);

}  // namespace amgeig
