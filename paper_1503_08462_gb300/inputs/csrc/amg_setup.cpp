// Host-side classical AMG setup (Sec. 2 of the paper): strength of connection,
// Ruge-Stueben C/F splitting, direct interpolation and Galerkin coarse operators
// for the stiffness matrix A and the mass matrix M.
//
// This is input preparation, not the eigensolver: the hierarchy it produces is
// serialised once and read by both the CUDA solve path and the CPU oracle.
//
//   strength       S_i = { j != i : -a_ij >= theta * max_{l != i, a_il < 0} |a_il| }
//                  (Sec. 2.1, strong dependent set; theta = 0.25 in Sec. 4.1)
//   C/F splitting  classical Ruge-Stueben first pass driven by the measure
//                  |S_i^T| (Sec. 2.1) plus the classical second pass that makes
//                  every strong F-F pair share a C point.  Tie order: points with
//                  equal measure are taken most-recently-updated first.
//   interpolation  direct interpolation, P_i = S_i cap C (Eqs. Interpolation_Def
//                  and Interpolation_Dir).  P_i holds only negative couplings,
//                  so the positive off-diagonal sum is lumped onto the diagonal.
//                  An F point without a strong C neighbour is made a C point.
//   coarse ops     A_{k+1} = P^T A_k P, M_{k+1} = P^T M_k P (Eq. Coarse_Matrices),
//                  computed on the symbolic product pattern so that A_{k+1} and
//                  M_{k+1} keep one shared pattern (explicit zeros are kept).
//
// Plain C ABI so that Python can drive it through ctypes; portable C++17 only.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <vector>

namespace {

struct Csr {
  int64_t rows = 0, cols = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> a, m;  // m is empty for P
};

struct Hierarchy {
  std::vector<Csr> levels;     // A_k, M_k (shared pattern)
  std::vector<Csr> prolong;    // P_k : N_k x N_{k+1}
};

// Strength matrix S (pattern only) and its transpose.
void strength(const Csr& A, double theta, std::vector<int32_t>& srp, std::vector<int32_t>& sci) {
  const int64_t n = A.rows;
  srp.assign(n + 1, 0);
  sci.clear();
  sci.reserve(A.ci.size());
  for (int64_t i = 0; i < n; ++i) {
    double maxneg = 0.0;
    for (int32_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      if (A.ci[p] != i && A.a[p] < 0.0) maxneg = std::max(maxneg, -A.a[p]);
    }
    if (maxneg > 0.0) {
      const double thr = theta * maxneg;
      for (int32_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
        if (A.ci[p] != i && -A.a[p] >= thr) sci.push_back(A.ci[p]);
      }
    }
    srp[i + 1] = static_cast<int32_t>(sci.size());
  }
}

void transpose_pattern(int64_t n_rows, int64_t n_cols, const std::vector<int32_t>& rp,
                       const std::vector<int32_t>& ci, std::vector<int32_t>& trp,
                       std::vector<int32_t>& tci) {
  trp.assign(n_cols + 1, 0);
  for (int32_t c : ci) trp[c + 1]++;
  for (int64_t j = 0; j < n_cols; ++j) trp[j + 1] += trp[j];
  tci.resize(ci.size());
  std::vector<int32_t> pos(trp.begin(), trp.end() - 1);
  for (int64_t i = 0; i < n_rows; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) tci[pos[ci[p]]++] = static_cast<int32_t>(i);
}

enum : int8_t { U_PT = 0, C_PT = 1, F_PT = 2 };

// Bucket priority structure over integer measures; O(1) updates.
struct Buckets {
  std::vector<int32_t> head, next, prev;
  std::vector<int32_t> lam;
  int32_t top = -1;
  Buckets(int64_t n, int32_t maxlam) : head(maxlam + 1, -1), next(n, -1), prev(n, -1), lam(n, 0) {}
  void insert(int32_t i) {
    int32_t b = lam[i];
    next[i] = head[b];
    prev[i] = -1;
    if (head[b] >= 0) prev[head[b]] = i;
    head[b] = i;
    if (b > top) top = b;
  }
  void remove(int32_t i) {
    int32_t b = lam[i];
    if (prev[i] >= 0) next[prev[i]] = next[i]; else head[b] = next[i];
    if (next[i] >= 0) prev[next[i]] = prev[i];
    next[i] = prev[i] = -1;
  }
  int32_t pop_max() {
    while (top >= 0 && head[top] < 0) --top;
    if (top < 0) return -1;
    int32_t i = head[top];
    remove(i);
    return i;
  }
};

void rs_split(const Csr& A, double theta, std::vector<int8_t>& state) {
  const int64_t n = A.rows;
  std::vector<int32_t> srp, sci, strp, stci;
  strength(A, theta, srp, sci);
  transpose_pattern(n, n, srp, sci, strp, stci);
  state.assign(n, U_PT);
  int32_t maxdeg = 0;
  for (int64_t i = 0; i < n; ++i) maxdeg = std::max(maxdeg, strp[i + 1] - strp[i]);
  // measure can grow up to |S_i^T| + (number of F in S_i^T) <= 2 |S_i^T|
  Buckets bk(n, 2 * maxdeg + 2);
  for (int64_t i = n - 1; i >= 0; --i) {
    bk.lam[i] = strp[i + 1] - strp[i];
    bk.insert(static_cast<int32_t>(i));
  }
  // first pass
  for (;;) {
    int32_t i = bk.pop_max();
    if (i < 0) break;
    if (bk.lam[i] == 0) {
      // nothing undecided depends on i any more: it becomes F (promoted later
      // if it has no strong C neighbour)
      state[i] = F_PT;
      continue;
    }
    state[i] = C_PT;
    for (int32_t p = strp[i]; p < strp[i + 1]; ++p) {
      int32_t j = stci[p];
      if (state[j] != U_PT) continue;
      state[j] = F_PT;
      bk.remove(j);
      for (int32_t r = srp[j]; r < srp[j + 1]; ++r) {
        int32_t k = sci[r];
        if (state[k] == U_PT) {
          bk.remove(k);
          bk.lam[k]++;
          bk.insert(k);
        }
      }
    }
    for (int32_t p = srp[i]; p < srp[i + 1]; ++p) {
      int32_t j = sci[p];
      if (state[j] == U_PT && bk.lam[j] > 0) {
        bk.remove(j);
        bk.lam[j]--;
        bk.insert(j);
      }
    }
  }
  // second pass: every strong F-F connection must share a strong C point
  std::vector<int32_t> mark(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    if (state[i] != F_PT) continue;
    const int32_t tag = static_cast<int32_t>(i);
    for (int32_t p = srp[i]; p < srp[i + 1]; ++p)
      if (state[sci[p]] == C_PT) mark[sci[p]] = tag;
    int32_t tentative = -1;
    for (int32_t p = srp[i]; p < srp[i + 1]; ++p) {
      int32_t j = sci[p];
      if (state[j] != F_PT) continue;
      bool shared = false;
      for (int32_t r = srp[j]; r < srp[j + 1]; ++r) {
        if (mark[sci[r]] == tag) { shared = true; break; }
      }
      if (shared) continue;
      if (tentative >= 0) {
        // second violation: make i itself a C point instead
        state[i] = C_PT;
        tentative = -1;
        break;
      }
      tentative = j;
      mark[j] = tag;  // j is now treated as one of i's C points
    }
    if (tentative >= 0) state[tentative] = C_PT;
  }
  // any F point without a strong C neighbour becomes C
  for (int64_t i = 0; i < n; ++i) {
    if (state[i] != F_PT) continue;
    bool has_c = false;
    for (int32_t p = srp[i]; p < srp[i + 1]; ++p)
      if (state[sci[p]] == C_PT) { has_c = true; break; }
    if (!has_c) state[i] = C_PT;
  }
}

Csr direct_interpolation(const Csr& A, double theta, const std::vector<int8_t>& state) {
  const int64_t n = A.rows;
  std::vector<int32_t> srp, sci;
  strength(A, theta, srp, sci);
  std::vector<int32_t> cidx(n, -1);
  int32_t nc = 0;
  for (int64_t i = 0; i < n; ++i)
    if (state[i] == C_PT) cidx[i] = nc++;
  Csr P;
  P.rows = n;
  P.cols = nc;
  P.rp.assign(n + 1, 0);
  std::vector<char> strong(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (state[i] == C_PT) {
      P.ci.push_back(cidx[i]);
      P.a.push_back(1.0);
    } else {
      for (int32_t p = srp[i]; p < srp[i + 1]; ++p) strong[sci[p]] = 1;
      double diag = 0.0, neg_all = 0.0, pos_all = 0.0, neg_p = 0.0;
      for (int32_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
        const int32_t j = A.ci[p];
        const double v = A.a[p];
        if (j == i) { diag += v; continue; }
        if (v < 0.0) neg_all += v; else pos_all += v;
        if (v < 0.0 && strong[j] && state[j] == C_PT) neg_p += v;
      }
      const double alpha = neg_all / neg_p;
      const double dd = diag + pos_all;  // positive couplings lumped onto the diagonal
      for (int32_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
        const int32_t j = A.ci[p];
        if (j != i && strong[j] && state[j] == C_PT && A.a[p] < 0.0) {
          P.ci.push_back(cidx[j]);
          P.a.push_back(-alpha * A.a[p] / dd);
        }
      }
      for (int32_t p = srp[i]; p < srp[i + 1]; ++p) strong[sci[p]] = 0;
    }
    P.rp[i + 1] = static_cast<int32_t>(P.ci.size());
  }
  return P;
}

// C = X * Y on the symbolic pattern (no numerical dropping).  X may carry two
// value arrays (a and m) sharing its pattern; Y has one (a).
void spgemm(const Csr& X, bool two, const Csr& Y, Csr& C) {
  C.rows = X.rows;
  C.cols = Y.cols;
  C.rp.assign(X.rows + 1, 0);
  C.ci.clear();
  C.a.clear();
  C.m.clear();
  std::vector<int32_t> marker(Y.cols, -1);
  std::vector<double> acc_a(Y.cols, 0.0), acc_m(two ? Y.cols : 0, 0.0);
  std::vector<int32_t> cols;
  for (int64_t i = 0; i < X.rows; ++i) {
    cols.clear();
    for (int32_t p = X.rp[i]; p < X.rp[i + 1]; ++p) {
      const int32_t k = X.ci[p];
      const double xa = X.a[p];
      const double xm = two ? X.m[p] : 0.0;
      for (int32_t r = Y.rp[k]; r < Y.rp[k + 1]; ++r) {
        const int32_t j = Y.ci[r];
        if (marker[j] != i) {
          marker[j] = static_cast<int32_t>(i);
          cols.push_back(j);
          acc_a[j] = 0.0;
          if (two) acc_m[j] = 0.0;
        }
        acc_a[j] += xa * Y.a[r];
        if (two) acc_m[j] += xm * Y.a[r];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t j : cols) {
      C.ci.push_back(j);
      C.a.push_back(acc_a[j]);
      if (two) C.m.push_back(acc_m[j]);
    }
    C.rp[i + 1] = static_cast<int32_t>(C.ci.size());
  }
}

Csr transpose_values(const Csr& P) {
  Csr R;
  R.rows = P.cols;
  R.cols = P.rows;
  R.rp.assign(P.cols + 1, 0);
  for (int32_t c : P.ci) R.rp[c + 1]++;
  for (int64_t j = 0; j < P.cols; ++j) R.rp[j + 1] += R.rp[j];
  R.ci.resize(P.ci.size());
  R.a.resize(P.ci.size());
  std::vector<int32_t> pos(R.rp.begin(), R.rp.end() - 1);
  for (int64_t i = 0; i < P.rows; ++i)
    for (int32_t p = P.rp[i]; p < P.rp[i + 1]; ++p) {
      const int32_t q = pos[P.ci[p]]++;
      R.ci[q] = static_cast<int32_t>(i);
      R.a[q] = P.a[p];
    }
  return R;
}

// Galerkin product R (A, M) P with R = P^T; the two results share one pattern.
Csr galerkin(const Csr& A, const Csr& P) {
  Csr AP, RAP;
  spgemm(A, true, P, AP);
  Csr R = transpose_values(P);
  // R has one value array; multiply it against AP's two value arrays by
  // computing R*AP_a and R*AP_m on the same pattern.
  Csr APa = AP, APm = AP;
  APa.m.clear();
  APm.a = AP.m;
  APm.m.clear();
  Csr Ca, Cm;
  spgemm(R, false, APa, Ca);
  spgemm(R, false, APm, Cm);
  RAP.rows = Ca.rows;
  RAP.cols = Ca.cols;
  RAP.rp = Ca.rp;
  RAP.ci = Ca.ci;
  RAP.a = Ca.a;
  RAP.m = Cm.a;
  return RAP;
}

}  // namespace

extern "C" {

// Build the hierarchy.  Returns 0 on success, <0 on invalid input.
int amgsetup_build(int64_t n, const int32_t* rp, const int32_t* ci, const double* a,
                   const double* m, double theta, int64_t coarse_cap, int32_t max_levels,
                   void** out) {
  if (!out || n <= 0 || !rp || !ci || !a || !m || theta <= 0.0 || theta >= 1.0 || coarse_cap < 1 ||
      max_levels < 1)
    return -1;
  *out = nullptr;
  auto h = std::make_unique<Hierarchy>();
  Csr A;
  A.rows = A.cols = n;
  A.rp.assign(rp, rp + n + 1);
  const int64_t nnz = A.rp[n];
  if (A.rp[0] != 0 || nnz < 0) return -1;
  for (int64_t i = 0; i < n; ++i)
    if (A.rp[i + 1] < A.rp[i]) return -1;
  A.ci.assign(ci, ci + nnz);
  for (int32_t c : A.ci)
    if (c < 0 || c >= n) return -1;
  A.a.assign(a, a + nnz);
  A.m.assign(m, m + nnz);
  h->levels.push_back(std::move(A));
  while (static_cast<int32_t>(h->levels.size()) < max_levels && h->levels.back().rows > coarse_cap) {
    const Csr& Af = h->levels.back();
    std::vector<int8_t> state;
    rs_split(Af, theta, state);
    Csr P = direct_interpolation(Af, theta, state);
    if (P.cols == 0 || P.cols >= Af.rows) break;  // coarsening stalled
    Csr Ac = galerkin(Af, P);
    h->prolong.push_back(std::move(P));
    h->levels.push_back(std::move(Ac));
  }
  *out = h.release();
  return 0;
}

// The C/F splitting alone (the first step of each level's setup), for a setup
// whose other steps run elsewhere: state[i] = 1 for a C point, 2 for an F point.
// Returns 0, or -1 on invalid input.
int amgsetup_cf_split(int64_t n, const int32_t* rp, const int32_t* ci, const double* a, double theta,
                      int8_t* state) {
  if (n <= 0 || !rp || !ci || !a || !state || theta <= 0.0 || theta >= 1.0) return -1;
  Csr A;
  A.rows = A.cols = n;
  A.rp.assign(rp, rp + n + 1);
  const int64_t nnz = A.rp[n];
  A.ci.assign(ci, ci + nnz);
  A.a.assign(a, a + nnz);
  std::vector<int8_t> st;
  rs_split(A, theta, st);
  std::memcpy(state, st.data(), static_cast<size_t>(n));
  return 0;
}

int32_t amgsetup_num_levels(void* hp) { return static_cast<int32_t>(static_cast<Hierarchy*>(hp)->levels.size()); }

// Sizes of level l: rows, nnz of (A,M), nnz of P_l (0 for the coarsest level).
int amgsetup_level_sizes(void* hp, int32_t l, int64_t* rows, int64_t* nnz, int64_t* nnz_p) {
  auto* h = static_cast<Hierarchy*>(hp);
  if (l < 0 || l >= static_cast<int32_t>(h->levels.size())) return -1;
  *rows = h->levels[l].rows;
  *nnz = static_cast<int64_t>(h->levels[l].ci.size());
  *nnz_p = l < static_cast<int32_t>(h->prolong.size()) ? static_cast<int64_t>(h->prolong[l].ci.size()) : 0;
  return 0;
}

int amgsetup_get_level(void* hp, int32_t l, int32_t* rp, int32_t* ci, double* a, double* m) {
  auto* h = static_cast<Hierarchy*>(hp);
  if (l < 0 || l >= static_cast<int32_t>(h->levels.size())) return -1;
  const Csr& L = h->levels[l];
  std::memcpy(rp, L.rp.data(), L.rp.size() * sizeof(int32_t));
  std::memcpy(ci, L.ci.data(), L.ci.size() * sizeof(int32_t));
  std::memcpy(a, L.a.data(), L.a.size() * sizeof(double));
  std::memcpy(m, L.m.data(), L.m.size() * sizeof(double));
  return 0;
}

int amgsetup_get_prolongation(void* hp, int32_t l, int32_t* rp, int32_t* ci, double* p) {
  auto* h = static_cast<Hierarchy*>(hp);
  if (l < 0 || l >= static_cast<int32_t>(h->prolong.size())) return -1;
  const Csr& P = h->prolong[l];
  std::memcpy(rp, P.rp.data(), P.rp.size() * sizeof(int32_t));
  std::memcpy(ci, P.ci.data(), P.ci.size() * sizeof(int32_t));
  std::memcpy(p, P.a.data(), P.a.size() * sizeof(double));
  return 0;
}

void amgsetup_free(void* hp) { delete static_cast<Hierarchy*>(hp); }

}  // extern "C"
