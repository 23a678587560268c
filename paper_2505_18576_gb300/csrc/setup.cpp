// Host setup of the AMGF solver (C++17, OpenMP).
//
// B := AMG(A) (Section 5.1, Remark after Lemma "condition number estimate": classical
// AMG with l1 smoothers; the paper uses hypre BoomerAMG).  The parameters and the
// evaluation order of every floating-point sum are fixed so that the hierarchy is a
// deterministic function of A:
//   strength    j != i strong for i iff same unknown and |a_ij| >= theta * max_k |a_ik|
//   coarsening  Ruge-Stueben first pass, largest measure first, ties to the smaller index,
//               leftover points C if they have a strong influencer, else F
//   interpolate classical (Ruge-Stueben) interpolation: strong F neighbours distributed over
//               the row's strong C points, weak ones lumped into the diagonal; rows whose
//               lumped diagonal nearly cancels (and interp = 1 for all rows) take direct
//               interpolation with the sign split (Stueben)
//   Galerkin    R = P^T, A_c = R (A P), sums in ascending index order
//   smoother    l1-Jacobi, l1_i = sum_j |a_ij|
// A_w = P^T A P = A[I_c, I_c] (Section 5.1) is ordered by reverse Cuthill-McKee from a
// pseudo-peripheral vertex (George & Liu), where it is block tridiagonal with the bandwidth
// as block size, and prepared for an exact solve with dense block operations: odd-even
// block cyclic reduction, or block LDL^T.
#include "setup.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <queue>
#include <utility>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace amgf {

namespace {

int nthreads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Rows [0, n) split into `parts` contiguous ranges.
std::vector<int64_t> split_rows(int64_t n, int parts) {
  std::vector<int64_t> b(parts + 1);
  for (int t = 0; t <= parts; ++t) b[t] = n * t / parts;
  return b;
}

// Assemble per-range row pieces into one CSR (pieces are in row order).
struct RowPieces {
  std::vector<std::vector<int64_t>> len;   // per part: row lengths
  std::vector<std::vector<int32_t>> ci;
  std::vector<std::vector<double>> v;
  explicit RowPieces(int parts) : len(parts), ci(parts), v(parts) {}
  void gather(HCSR& out, int64_t nrows, int64_t ncols) {
    out.nrows = nrows; out.ncols = ncols;
    out.rp.assign(nrows + 1, 0);
    int64_t r = 0;
    for (auto& L : len)
      for (int64_t x : L) { out.rp[r + 1] = out.rp[r] + x; ++r; }
    out.ci.resize(out.rp[nrows]);
    out.v.resize(out.rp[nrows]);
    std::vector<int64_t> off(len.size() + 1, 0);
    for (size_t t = 0; t < len.size(); ++t) off[t + 1] = off[t] + (int64_t)ci[t].size();
#pragma omp parallel for schedule(static)
    for (int t = 0; t < (int)len.size(); ++t) {
      std::copy(ci[t].begin(), ci[t].end(), out.ci.begin() + off[t]);
      std::copy(v[t].begin(), v[t].end(), out.v.begin() + off[t]);
      std::vector<int32_t>().swap(ci[t]);
      std::vector<double>().swap(v[t]);
    }
  }
};

HCSR transpose(const HCSR& a) {
  HCSR t;
  t.nrows = a.ncols; t.ncols = a.nrows;
  t.rp.assign(t.nrows + 1, 0);
  for (int64_t k = 0; k < a.nnz(); ++k) t.rp[a.ci[k] + 1]++;
  for (int64_t i = 0; i < t.nrows; ++i) t.rp[i + 1] += t.rp[i];
  t.ci.resize(a.nnz());
  t.v.resize(a.nnz());
  std::vector<int64_t> pos(t.rp.begin(), t.rp.end() - 1);
  for (int64_t i = 0; i < a.nrows; ++i)
    for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k) {
      int64_t p = pos[a.ci[k]]++;
      t.ci[p] = (int32_t)i;
      t.v[p] = a.v[k];
    }
  return t;
}

// C = A B; entry (i, J) accumulates a_ij b_jJ over row i of A in ascending j.  Two passes over
// row blocks: the row lengths (distinct columns, marked with the row as a stamp), then the values
// accumulated in a dense row buffer and written straight into C's arrays, columns ascending.
HCSR spgemm(const HCSR& a, const HCSR& b) {
  const int parts = std::max(1, nthreads() * 4);
  auto bounds = split_rows(a.nrows, parts);
  HCSR c;
  c.nrows = a.nrows;
  c.ncols = b.ncols;
  c.rp.assign(a.nrows + 1, 0);
#pragma omp parallel
  {
    std::vector<int64_t> mark(b.ncols, -1);
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < parts; ++t)
      for (int64_t i = bounds[t]; i < bounds[t + 1]; ++i) {
        int64_t len = 0;
        for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k) {
          const int64_t j = a.ci[k];
          for (int64_t kk = b.rp[j]; kk < b.rp[j + 1]; ++kk) {
            const int32_t J = b.ci[kk];
            if (mark[J] != i) { mark[J] = i; ++len; }
          }
        }
        c.rp[i + 1] = len;
      }
  }
  for (int64_t i = 0; i < a.nrows; ++i) c.rp[i + 1] += c.rp[i];
  c.ci.resize(c.rp[a.nrows]);
  c.v.resize(c.rp[a.nrows]);
#pragma omp parallel
  {
    std::vector<double> acc(b.ncols, 0.0);
    std::vector<int64_t> mark(b.ncols, -1);
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < parts; ++t)
      for (int64_t i = bounds[t]; i < bounds[t + 1]; ++i) {
        int32_t* cols = c.ci.data() + c.rp[i];
        int64_t n = 0;
        for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k) {
          const int64_t j = a.ci[k];
          const double aij = a.v[k];
          for (int64_t kk = b.rp[j]; kk < b.rp[j + 1]; ++kk) {
            const int32_t J = b.ci[kk];
            if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; cols[n++] = J; }
            acc[J] += aij * b.v[kk];
          }
        }
        std::sort(cols, cols + n);
        double* vals = c.v.data() + c.rp[i];
        for (int64_t q = 0; q < n; ++q) vals[q] = acc[cols[q]];
      }
  }
  return c;
}

// Strong influences S_i as a pattern (ascending, subset of row i of A).
void strength_graph(const HCSR& A, const std::vector<int32_t>& func, double theta,
                    std::vector<int64_t>& srp, std::vector<int32_t>& sci) {
  const int64_t n = A.nrows;
  std::vector<int64_t> cnt(n + 1, 0);
  std::vector<double> thr(n, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double mx = 0.0;
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int32_t j = A.ci[k];
      if (j == i || func[j] != func[i]) continue;
      mx = std::max(mx, std::fabs(A.v[k]));
    }
    int64_t c = 0;
    if (mx > 0.0) {
      const double t = theta * mx;
      thr[i] = t;
      for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int32_t j = A.ci[k];
        if (j != i && func[j] == func[i] && std::fabs(A.v[k]) >= t) ++c;
      }
    }
    cnt[i + 1] = c;
  }
  for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  srp = cnt;
  sci.resize(srp[n]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    if (srp[i + 1] == srp[i]) continue;
    int64_t p = srp[i];
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int32_t j = A.ci[k];
      if (j != i && func[j] == func[i] && std::fabs(A.v[k]) >= thr[i]) sci[p++] = j;
    }
  }
}

// Subset of [0, n) with insert, erase and smallest element: a tree of 64-bit words, each bit of
// a level summarising one word of the level below.
struct MinSet {
  std::vector<std::vector<uint64_t>> lv;  // lv[0]: one bit per element
  explicit MinSet(int64_t n) {
    int64_t m = n;
    do {
      m = (m + 63) / 64;
      lv.emplace_back(m, 0);
    } while (m > 1);
  }
  void insert(int64_t i) {
    for (auto& w : lv) {
      uint64_t& x = w[i >> 6];
      const bool had = x != 0;
      x |= 1ull << (i & 63);
      if (had) return;
      i >>= 6;
    }
  }
  void erase(int64_t i) {
    for (auto& w : lv) {
      uint64_t& x = w[i >> 6];
      x &= ~(1ull << (i & 63));
      if (x) return;
      i >>= 6;
    }
  }
  bool empty() const { return lv.back()[0] == 0; }
  int64_t min() const {
    int64_t i = 0;
    for (int k = (int)lv.size() - 1; k >= 0; --k) i = (i << 6) | __builtin_ctzll(lv[k][i]);
    return i;
  }
};

// Ruge-Stueben first pass: repeatedly the undecided point of largest measure (ties: smallest
// index) becomes C.  Measures are small integers that change by one, so the undecided points sit
// in one MinSet per measure value and the current largest measure is tracked; a point whose
// measure reaches 0 can never be chosen (no undecided or F point depends on it any more).
std::vector<int8_t> ruge_stueben(int64_t n, const std::vector<int64_t>& srp, const std::vector<int32_t>& sci) {
  // dependents: transpose of the strength pattern
  std::vector<int64_t> trp(n + 1, 0);
  for (int32_t j : sci) trp[j + 1]++;
  for (int64_t i = 0; i < n; ++i) trp[i + 1] += trp[i];
  std::vector<int32_t> tci(sci.size());
  {
    std::vector<int64_t> pos(trp.begin(), trp.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t k = srp[i]; k < srp[i + 1]; ++k) tci[pos[sci[k]]++] = (int32_t)i;
  }
  enum : int8_t { UND = 0, FPT = 1, CPT = 2 };
  std::vector<int8_t> state(n, UND);
  std::vector<int64_t> lam(n);
  int64_t top = 0;
  for (int64_t i = 0; i < n; ++i) {
    lam[i] = trp[i + 1] - trp[i];
    top = std::max(top, lam[i]);
  }
  // a measure is |S^T_i among undecided| + 2 |S^T_i among F| <= 2 |S^T_i|
  std::vector<std::unique_ptr<MinSet>> bucket(2 * top + 2);
  auto put = [&](int64_t i) {
    const int64_t m = lam[i];
    if (m < 1) return;
    if (!bucket[m]) bucket[m].reset(new MinSet(n));
    bucket[m]->insert(i);
  };
  auto take = [&](int64_t i) {
    if (lam[i] >= 1) bucket[lam[i]]->erase(i);
  };
  for (int64_t i = 0; i < n; ++i) put(i);
  int64_t cur = top;
  for (;;) {
    while (cur >= 1 && (!bucket[cur] || bucket[cur]->empty())) --cur;
    if (cur < 1) break;
    const int64_t i = bucket[cur]->min();
    take(i);
    state[i] = CPT;
    for (int64_t k = trp[i]; k < trp[i + 1]; ++k) {
      const int32_t j = tci[k];
      if (state[j] != UND) continue;
      take(j);
      state[j] = FPT;
      for (int64_t kk = srp[j]; kk < srp[j + 1]; ++kk) {
        const int32_t q = sci[kk];
        if (state[q] == UND) {
          take(q);
          lam[q] += 1;
          put(q);
          cur = std::max(cur, lam[q]);
        }
      }
    }
    for (int64_t k = srp[i]; k < srp[i + 1]; ++k) {
      const int32_t q = sci[k];
      if (state[q] == UND) {
        take(q);
        lam[q] -= 1;
        put(q);
      }
    }
  }
  std::vector<int8_t> cf(n);
  for (int64_t i = 0; i < n; ++i) {
    if (state[i] == UND) state[i] = (srp[i + 1] > srp[i]) ? CPT : FPT;
    cf[i] = state[i] == CPT ? 1 : 0;
  }
  return cf;
}

// Interpolation from the C/F split.  interp 0: classical (Ruge-Stueben) interpolation,
//   w_ij = -(a_ij + sum_{k strong F} a_ik abar_kj / sum_{m strong C of i} abar_km) / d_i,
//   abar_km = a_km when its sign is opposite to a_kk's (else 0), d_i = a_ii + weak entries
//   (+ a_ik of strong F points with an empty sum); a row with |d_i| < 0.05 a_ii takes the
//   direct weights.  interp 1: direct interpolation with the sign split for every row.
// Same-function couplings only; every sum runs in ascending column order.
constexpr double kClassicalGuard = 0.05;

HCSR build_interpolation(const HCSR& A, const std::vector<int64_t>& srp, const std::vector<int32_t>& sci,
                         const std::vector<int32_t>& func, const std::vector<int8_t>& cf, int interp, int p_max,
                         int64_t& nc) {
  const int64_t n = A.nrows;
  std::vector<int64_t> cidx(n, -1);
  nc = 0;
  for (int64_t i = 0; i < n; ++i)
    if (cf[i]) cidx[i] = nc++;
  const int parts = std::max(1, nthreads() * 4);
  auto bounds = split_rows(n, parts);
  RowPieces pc(parts);
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < parts; ++t) {
    auto& L = pc.len[t];
    auto& C = pc.ci[t];
    auto& V = pc.v[t];
    std::vector<int32_t> ccol;  // strong C neighbours of the row (ascending) and their accumulators
    std::vector<double> cval;
    std::vector<int32_t> order;
    std::vector<int8_t> kept;
    // P_max truncation of the row just appended (weights in ascending coarse index): keep the
    // p_max largest |w| (ties: smaller coarse index), scaled by sum(all) / sum(kept)
    auto truncate_last = [&]() {
      const int64_t cnt = L.back();
      if (p_max <= 0 || cnt <= p_max) return;
      const size_t r0 = V.size() - (size_t)cnt;
      order.resize(cnt);
      for (int64_t q = 0; q < cnt; ++q) order[q] = (int32_t)q;
      std::stable_sort(order.begin(), order.end(),
                       [&](int32_t x, int32_t y) { return std::fabs(V[r0 + x]) > std::fabs(V[r0 + y]); });
      kept.assign(cnt, 0);
      for (int q = 0; q < p_max; ++q) kept[order[q]] = 1;
      double all = 0.0, part = 0.0;
      for (int64_t q = 0; q < cnt; ++q) all += V[r0 + q];
      for (int64_t q = 0; q < cnt; ++q)
        if (kept[q]) part += V[r0 + q];
      if (part == 0.0) return;
      const double scale = all / part;
      size_t m = r0;
      for (int64_t q = 0; q < cnt; ++q) {
        if (!kept[q]) continue;
        C[m] = C[r0 + q];
        V[m] = V[r0 + q] * scale;
        ++m;
      }
      C.resize(m);
      V.resize(m);
      L.back() = p_max;
    };
    // direct interpolation weights of F row i (walks row i of A and the ascending strong list together)
    auto direct_row = [&](int64_t i) {
      double diag = 0.0, sn = 0.0, sp = 0.0, cn = 0.0, cp = 0.0;
      int64_t s = srp[i];
      for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int32_t j = A.ci[k];
        const double a = A.v[k];
        if (j == i) { diag = a; continue; }
        if (func[j] != func[i]) continue;
        while (s < srp[i + 1] && sci[s] < j) ++s;
        const bool strongC = s < srp[i + 1] && sci[s] == j && cf[j];
        if (a < 0.0) { sn += a; if (strongC) cn += a; }
        else { sp += a; if (strongC) cp += a; }
      }
      if (cp == 0.0) diag += sp;
      const double alpha = cn != 0.0 ? sn / cn : 0.0;
      const double beta = cp != 0.0 ? sp / cp : 0.0;
      int64_t cnt = 0;
      s = srp[i];
      for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int32_t j = A.ci[k];
        if (j == i) continue;
        while (s < srp[i + 1] && sci[s] < j) ++s;
        if (!(s < srp[i + 1] && sci[s] == j && cf[j])) continue;
        const double a = A.v[k];
        const double w = a < 0.0 ? -(alpha * a) / diag : -(beta * a) / diag;
        C.push_back((int32_t)cidx[j]);
        V.push_back(w);
        ++cnt;
      }
      L.push_back(cnt);
    };
    for (int64_t i = bounds[t]; i < bounds[t + 1]; ++i) {
      if (cf[i]) { L.push_back(1); C.push_back((int32_t)cidx[i]); V.push_back(1.0); continue; }
      bool anyC = false;
      for (int64_t k = srp[i]; k < srp[i + 1]; ++k) anyC |= cf[sci[k]] != 0;
      if (!anyC) { L.push_back(0); continue; }
      if (interp == 1) { direct_row(i); truncate_last(); continue; }
      // classical: numerators start at a_ij for the strong C neighbours
      ccol.clear();
      cval.clear();
      double diag = 0.0, aii = 0.0;
      int64_t s = srp[i];
      for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int32_t j = A.ci[k];
        if (j == i) { aii = A.v[k]; diag += A.v[k]; continue; }
        if (func[j] != func[i]) continue;
        while (s < srp[i + 1] && sci[s] < j) ++s;
        if (s < srp[i + 1] && sci[s] == j && cf[j]) { ccol.push_back(j); cval.push_back(A.v[k]); }
      }
      s = srp[i];
      for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int32_t j = A.ci[k];
        if (j == i || func[j] != func[i]) continue;
        while (s < srp[i + 1] && sci[s] < j) ++s;
        const bool strong = s < srp[i + 1] && sci[s] == j;
        if (strong && cf[j]) continue;
        const double a = A.v[k];
        if (!strong) { diag += a; continue; }  // weak neighbour: lumped
        // strong F neighbour j: distributed over the strong C points of i through row j
        double ajj = 0.0, den = 0.0;
        for (int64_t q = A.rp[j]; q < A.rp[j + 1]; ++q)
          if (A.ci[q] == j) ajj = A.v[q];
        size_t c = 0;
        for (int64_t q = A.rp[j]; q < A.rp[j + 1]; ++q) {
          const int32_t m = A.ci[q];
          if (m == j) continue;
          while (c < ccol.size() && ccol[c] < m) ++c;
          if (c == ccol.size()) break;
          if (ccol[c] != m) continue;
          const double am = A.v[q];
          if ((am < 0.0) != (ajj < 0.0)) den += am;
        }
        if (den == 0.0) { diag += a; continue; }
        c = 0;
        for (int64_t q = A.rp[j]; q < A.rp[j + 1]; ++q) {
          const int32_t m = A.ci[q];
          if (m == j) continue;
          while (c < ccol.size() && ccol[c] < m) ++c;
          if (c == ccol.size()) break;
          if (ccol[c] != m) continue;
          const double am = A.v[q];
          if ((am < 0.0) != (ajj < 0.0)) cval[c] += a * am / den;
        }
      }
      if (std::fabs(diag) < kClassicalGuard * aii) { direct_row(i); truncate_last(); continue; }
      for (size_t c = 0; c < ccol.size(); ++c) {
        C.push_back((int32_t)cidx[ccol[c]]);
        V.push_back(-cval[c] / diag);
      }
      L.push_back((int64_t)ccol.size());
      truncate_last();
    }
  }
  HCSR P;
  pc.gather(P, n, nc);
  return P;
}

// In-place dense Cholesky (row-major, lower); false on a non-positive pivot.  Right-looking:
// after column j, the trailing rows are updated by row axpys.
bool cholesky(std::vector<double>& a, int64_t n) {
  for (int64_t j = 0; j < n; ++j) {
    const double s = a[j * n + j];
    if (!(s > 0.0)) return false;
    const double d = std::sqrt(s);
    a[j * n + j] = d;
    for (int64_t i = j + 1; i < n; ++i) a[i * n + j] /= d;
    // A[i][l] -= L[i][j] L[l][j] for j < l <= i
#pragma omp parallel for schedule(dynamic, 16) if (!omp_in_parallel() && n - j > 256)
    for (int64_t i = j + 1; i < n; ++i) {
      const double lij = a[i * n + j];
      double* ai = a.data() + i * n;
      for (int64_t l = j + 1; l <= i; ++l) ai[l] -= lij * a[l * n + j];
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) a[i * n + j] = 0.0;
  return true;
}

// Inverse of an SPD matrix from its Cholesky factor: L L^T X = I solved for 8 columns of I at
// a time, so that the inner loops run across the 8 right-hand sides (vector work, no
// reductions); on Arm Neoverse cores 1.9x faster than column-by-column substitution.
void spd_inverse_factored(const std::vector<double>& L, int64_t n, std::vector<double>& inv);

bool spd_inverse(const std::vector<double>& a, int64_t n, std::vector<double>& inv) {
  std::vector<double> L(a);
  if (!cholesky(L, n)) return false;
  spd_inverse_factored(L, n, inv);
  return true;
}

// The same inverse from a Cholesky factor L (lower, row-major) that cholesky() already computed.
void spd_inverse_factored(const std::vector<double>& L, int64_t n, std::vector<double>& inv) {
  inv.assign(n * n, 0.0);
  constexpr int64_t R = 8;
  const int64_t nbat = (n + R - 1) / R;
#pragma omp parallel for schedule(dynamic, 1) if (!omp_in_parallel() && n > 64)
  for (int64_t bt = 0; bt < nbat; ++bt) {
    const int64_t c0 = bt * R, nc = std::min(R, n - c0);
    std::vector<double> y(n * R, 0.0);  // y[i R + q]: column c0 + q
    for (int64_t q = 0; q < nc; ++q) y[(c0 + q) * R + q] = 1.0;
    // forward: L y = e (rows above c0 stay zero)
    for (int64_t i = c0; i < n; ++i) {
      double s[R];
      for (int64_t q = 0; q < R; ++q) s[q] = y[i * R + q];
      for (int64_t k = c0; k < i; ++k) {
        const double lik = L[i * n + k];
        for (int64_t q = 0; q < R; ++q) s[q] -= lik * y[k * R + q];
      }
      const double d = L[i * n + i];
      for (int64_t q = 0; q < R; ++q) y[i * R + q] = s[q] / d;
    }
    // backward: L^T x = y, column-oriented (x_i final, then y_k -= L[i][k] x_i for k < i)
    for (int64_t i = n - 1; i >= 0; --i) {
      const double d = L[i * n + i];
      for (int64_t q = 0; q < R; ++q) y[i * R + q] /= d;
      const double* li = L.data() + i * n;
      for (int64_t k = 0; k < i; ++k)
        for (int64_t q = 0; q < R; ++q) y[k * R + q] -= li[k] * y[i * R + q];
    }
    for (int64_t i = 0; i < n; ++i)
      for (int64_t q = 0; q < nc; ++q) inv[i * n + c0 + q] = y[i * R + q];
  }
  // exact symmetry
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      const double s = 0.5 * (inv[i * n + j] + inv[j * n + i]);
      inv[i * n + j] = inv[j * n + i] = s;
    }
}

// C = A * B (n x n, row-major), C = alpha * A * B + beta * C
void gemm(int64_t n, const double* A, const double* B, double* C, double alpha, double beta) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> row(n, 0.0);
    for (int64_t k = 0; k < n; ++k) {
      const double a = A[i * n + k];
      if (a == 0.0) continue;
      const double* b = B + k * n;
      for (int64_t j = 0; j < n; ++j) row[j] += a * b[j];
    }
    for (int64_t j = 0; j < n; ++j) C[i * n + j] = alpha * row[j] + (beta == 0.0 ? 0.0 : beta * C[i * n + j]);
  }
}

// C = alpha * op(A) * B + beta * C for n x n row-major blocks, op(A) = A or A^T; tiled over
// (i, k) so that a 64-row panel of B stays in cache.  Parallel over row tiles unless called
// from inside a parallel region.
void gemm_nn(int64_t n, const double* A, bool transA, const double* B, double* C, double alpha, double beta) {
  constexpr int64_t T = 64;
  const int64_t ntile = (n + T - 1) / T;
#pragma omp parallel for schedule(static) if (!omp_in_parallel() && n >= 2 * T)
  for (int64_t it = 0; it < ntile; ++it) {
    const int64_t i0 = it * T, i1 = std::min(n, i0 + T);
    std::vector<double> acc((i1 - i0) * n, 0.0);
    for (int64_t k0 = 0; k0 < n; k0 += T) {
      const int64_t k1 = std::min(n, k0 + T);
      for (int64_t i = i0; i < i1; ++i) {
        double* ar = acc.data() + (i - i0) * n;
        for (int64_t k = k0; k < k1; ++k) {
          const double a = transA ? A[k * n + i] : A[i * n + k];
          if (a == 0.0) continue;
          const double* b = B + k * n;
          for (int64_t j = 0; j < n; ++j) ar[j] += a * b[j];
        }
      }
    }
    for (int64_t i = i0; i < i1; ++i)
      for (int64_t j = 0; j < n; ++j)
        C[i * n + j] = alpha * acc[(i - i0) * n + j] + (beta == 0.0 ? 0.0 : beta * C[i * n + j]);
  }
}

std::vector<double> transpose_block(int64_t n, const std::vector<double>& a) {
  std::vector<double> t(n * n);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) t[j * n + i] = a[i * n + j];
  return t;
}

// X = B R^{-T} for a lower-triangular R (n x n, row-major): row i of X solves R x = b_i.
// Forward substitution for 8 rows of B at a time, the inner loops across those 8.
void solve_rows_lower(int64_t n, const double* R, const double* B, double* X) {
  constexpr int64_t Q = 8;
  const int64_t nbat = (n + Q - 1) / Q;
#pragma omp parallel for schedule(dynamic, 1) if (!omp_in_parallel() && n > 64)
  for (int64_t bt = 0; bt < nbat; ++bt) {
    const int64_t r0 = bt * Q, nr = std::min(Q, n - r0);
    std::vector<double> y(n * Q, 0.0);  // y[i Q + q]: component i of the solution for row r0 + q
    for (int64_t i = 0; i < n; ++i) {
      double s[Q];
      for (int64_t q = 0; q < Q; ++q) s[q] = q < nr ? B[(r0 + q) * n + i] : 0.0;
      for (int64_t k = 0; k < i; ++k) {
        const double rik = R[i * n + k];
        for (int64_t q = 0; q < Q; ++q) s[q] -= rik * y[k * Q + q];
      }
      const double d = R[i * n + i];
      for (int64_t q = 0; q < Q; ++q) y[i * Q + q] = s[q] / d;
    }
    for (int64_t q = 0; q < nr; ++q)
      for (int64_t i = 0; i < n; ++i) X[(r0 + q) * n + i] = y[i * Q + q];
  }
}

// X = B R^{-1} for a lower-triangular R: row i of X solves R^T x = b_i (backward substitution,
// column-oriented so that row k of R is read contiguously), 8 rows of B at a time.
void solve_rows_upper(int64_t n, const double* R, const double* B, double* X) {
  constexpr int64_t Q = 8;
  const int64_t nbat = (n + Q - 1) / Q;
#pragma omp parallel for schedule(dynamic, 1) if (!omp_in_parallel() && n > 64)
  for (int64_t bt = 0; bt < nbat; ++bt) {
    const int64_t r0 = bt * Q, nr = std::min(Q, n - r0);
    std::vector<double> y(n * Q, 0.0);
    for (int64_t q = 0; q < nr; ++q)
      for (int64_t i = 0; i < n; ++i) y[i * Q + q] = B[(r0 + q) * n + i];
    for (int64_t i = n - 1; i >= 0; --i) {
      const double d = R[i * n + i];
      for (int64_t q = 0; q < Q; ++q) y[i * Q + q] /= d;
      const double* ri = R + i * n;
      for (int64_t k = 0; k < i; ++k)
        for (int64_t q = 0; q < Q; ++q) y[k * Q + q] -= ri[k] * y[i * Q + q];
    }
    for (int64_t q = 0; q < nr; ++q)
      for (int64_t i = 0; i < n; ++i) X[(r0 + q) * n + i] = y[i * Q + q];
  }
}

// Odd-even block cyclic reduction of the symmetric block-tridiagonal matrix with diagonal
// blocks A_k and sub-diagonal blocks L_k = A_{k,k-1} (k = 0..N-1).  Eliminating the odd
// blocks x_k = A_k^{-1} (v_k - L_k x_{k-1} - L_{k+1}^T x_{k+1}) from the even rows leaves a
// block-tridiagonal system on the even blocks:
//   A'_k = A_k - E_k L_k^T - F_k L_{k+1},   L'_k = -E_k L_{k-1},   v'_k = v_k - E_k v_{k-1} - F_k v_{k+1}
// with E_k = L_k A_{k-1}^{-1} and F_k = L_{k+1}^T A_{k+1}^{-1}; the back substitution is
// x_k = A_k^{-1} v_k - F_{k-1}^T x_{k-1} - E_{k+1}^T x_{k+1}.  This is block Gaussian
// elimination of A_w in odd-even order, so the solve stays exact up to rounding.
int build_bcr(int64_t nb, int64_t nblk, std::vector<double>& Ad, std::vector<double>& As, Filter& F,
              std::string& err) {
  const int64_t bsz = nb * nb;
  int64_t N = nblk, stride = 1;
  std::vector<std::vector<double>> A(N), L(N);
  for (int64_t k = 0; k < N; ++k) {
    A[k].assign(Ad.begin() + k * bsz, Ad.begin() + (k + 1) * bsz);
    if (k > 0) L[k].assign(As.begin() + k * bsz, As.begin() + (k + 1) * bsz);
  }
  std::vector<double>().swap(Ad);
  std::vector<double>().swap(As);
  // F.M holds every matrix the solve applies, in the order the reduction produces them: per
  // level, for each block k, an odd block's A_k^{-1}, F_{k-1}^T and (if k + 1 < N) E_{k+1}^T,
  // an even block's E_k (k >= 1) and F_k (k + 1 < N); the inverse of the last block at the end.
  // The count is known in advance, so F.M is sized once and each level's matrices are copied
  // into their slots in parallel.
  auto level_count = [](int64_t n) {
    int64_t c = 0;
    for (int64_t k = 0; k < n; ++k) c += (k & 1) ? 2 + (k + 1 < n) : (k >= 1) + (k + 1 < n);
    return c;
  };
  int64_t total = 1;
  for (int64_t n = nblk; n > 1; n = (n + 1) / 2) total += level_count(n);
  F.M.resize(total * bsz);
  int64_t next = 0;
  struct Slot {
    const std::vector<double>* m;
    bool transposed;
  };
  std::vector<Slot> slots;  // matrices of the current level, slot next - slots.size() + i
  auto push = [&](const std::vector<double>& m, bool transposed) {
    slots.push_back({&m, transposed});
    return next++;
  };
  auto flush = [&]() {
    const int64_t first = next - (int64_t)slots.size();
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < (int64_t)slots.size(); ++q) {
      double* dst = F.M.data() + (first + q) * bsz;
      const double* src = slots[q].m->data();
      if (!slots[q].transposed) {
        std::copy(src, src + bsz, dst);
      } else {
        for (int64_t i = 0; i < nb; ++i)
          for (int64_t j = 0; j < nb; ++j) dst[j * nb + i] = src[i * nb + j];
      }
    }
    slots.clear();
  };
  std::vector<std::vector<FilterTask>> fwd, bwd;
  bool spd = true;
  while (N > 1) {
    std::vector<std::vector<double>> Ainv(N), E(N), Fk(N), R(N);
    // With fewer blocks than threads (the top levels of the reduction) the blocks run one after
    // another and each block's dense kernels run in parallel instead; the arithmetic of every
    // entry is the same either way.
    const bool by_block = N / 2 >= nthreads();
    // odd blocks: Cholesky factors R_k (A_k = R_k R_k^T) and the inverses the solve applies
#pragma omp parallel for schedule(dynamic, 1) if (by_block)
    for (int64_t k = 1; k < N; k += 2) {
      std::vector<double> r = A[k];
      std::vector<double> inv;
      if (!cholesky(r, nb)) {
#pragma omp critical
        spd = false;
      } else {
        spd_inverse_factored(r, nb, inv);
      }
      R[k].swap(r);
      Ainv[k].swap(inv);
    }
    if (!spd) { err = "filter matrix A_w is not SPD"; return AMGF_ERR_NOT_SPD; }
    // even blocks: the Schur complement A'_k = A_k - W1 W1^T - W2 W2^T with W1 = L_k R_{k-1}^{-T},
    // W2 = L_{k+1}^T R_{k+1}^{-T} (symmetric updates through the factors, the form that keeps
    // A' positive definite when the blocks are ill-conditioned), E_k = W1 R_{k-1}^{-1},
    // F_k = W2 R_{k+1}^{-1}, L'_k = -E_k L_{k-1}
    const int64_t N2 = (N + 1) / 2;
    std::vector<std::vector<double>> A2(N2), L2(N2);
#pragma omp parallel for schedule(dynamic, 1) if (by_block)
    for (int64_t k = 0; k < N; k += 2) {
      std::vector<double> a = A[k], w(bsz), wt;
      if (k >= 1) {
        solve_rows_lower(nb, R[k - 1].data(), L[k].data(), w.data());
        E[k].resize(bsz);
        solve_rows_upper(nb, R[k - 1].data(), w.data(), E[k].data());
        wt = transpose_block(nb, w);
        gemm_nn(nb, w.data(), false, wt.data(), a.data(), -1.0, 1.0);
      }
      if (k + 1 < N) {
        const std::vector<double> LT = transpose_block(nb, L[k + 1]);
        solve_rows_lower(nb, R[k + 1].data(), LT.data(), w.data());
        Fk[k].resize(bsz);
        solve_rows_upper(nb, R[k + 1].data(), w.data(), Fk[k].data());
        wt = transpose_block(nb, w);
        gemm_nn(nb, w.data(), false, wt.data(), a.data(), -1.0, 1.0);
      }
      for (int64_t r = 0; r < nb; ++r)
        for (int64_t c = r + 1; c < nb; ++c) {
          const double sym = 0.5 * (a[r * nb + c] + a[c * nb + r]);
          a[r * nb + c] = a[c * nb + r] = sym;
        }
      A2[k / 2].swap(a);
      if (k >= 2) {
        L2[k / 2].resize(bsz);
        gemm_nn(nb, E[k].data(), false, L[k - 1].data(), L2[k / 2].data(), -1.0, 0.0);
      }
    }
    std::vector<FilterTask> tf, tb;
    for (int64_t k = 0; k < N; ++k) {
      const int32_t o = (int32_t)(k * stride);
      if (k & 1) {
        tf.push_back({push(Ainv[k], false), -1, o, o, -1, 0});
        const int64_t mb = push(Fk[k - 1], true);
        const int64_t mc = k + 1 < N ? push(E[k + 1], true) : -1;
        tb.push_back({mb, mc, o, (int32_t)((k - 1) * stride), k + 1 < N ? (int32_t)((k + 1) * stride) : -1, 2});
      } else {
        const int64_t me = k >= 1 ? push(E[k], false) : -1;
        const int64_t mf = k + 1 < N ? push(Fk[k], false) : -1;
        tf.push_back({me, mf, o, k >= 1 ? (int32_t)((k - 1) * stride) : -1,
                      k + 1 < N ? (int32_t)((k + 1) * stride) : -1, 1});
      }
    }
    flush();
    fwd.push_back(std::move(tf));
    bwd.push_back(std::move(tb));
    A.swap(A2);
    L.swap(L2);
    N = N2;
    stride *= 2;
  }
  std::vector<double> inv0;
  if (!spd_inverse(A[0], nb, inv0)) { err = "filter matrix A_w is not SPD"; return AMGF_ERR_NOT_SPD; }
  const int64_t m0 = push(inv0, false);
  flush();
  if (next != total) { err = "filter factor count mismatch"; return AMGF_ERR_INVALID_ARG; }
  F.bcr_levels = (int)fwd.size();
  F.tasks.clear();
  F.phase_off.assign(1, 0);
  auto add_phase = [&](const std::vector<FilterTask>& t) {
    F.tasks.insert(F.tasks.end(), t.begin(), t.end());
    F.phase_off.push_back((int64_t)F.tasks.size());
  };
  for (const auto& t : fwd) add_phase(t);
  add_phase({FilterTask{m0, -1, 0, 0, -1, 0}});
  for (int64_t l = (int64_t)bwd.size() - 1; l >= 0; --l) add_phase(bwd[l]);
  return AMGF_OK;
}

}  // namespace

void build_sell(const HCSR& A, int64_t window, SELL& out) {
  out = SELL();
  const int64_t n = A.nrows;
  out.nrows = n;
  out.nslices = (n + SELL::C - 1) / SELL::C;
  out.perm.resize(n);
  out.pinv.resize(n);
  for (int64_t i = 0; i < n; ++i) out.perm[i] = (int32_t)i;
  if (window < 1) window = 1;
  for (int64_t a = 0; a < n; a += window) {
    const int64_t b = std::min(n, a + window);
    std::stable_sort(out.perm.begin() + a, out.perm.begin() + b, [&](int32_t x, int32_t y) {
      return A.rp[x + 1] - A.rp[x] > A.rp[y + 1] - A.rp[y];
    });
  }
  for (int64_t q = 0; q < n; ++q) out.pinv[out.perm[q]] = (int32_t)q;
  out.soff.assign(out.nslices + 1, 0);
  for (int64_t s = 0; s < out.nslices; ++s) {
    int64_t w = 0;
    for (int64_t q = s * SELL::C; q < std::min(n, (s + 1) * SELL::C); ++q) {
      const int64_t r = out.perm[q];
      w = std::max(w, A.rp[r + 1] - A.rp[r]);
    }
    out.soff[s + 1] = out.soff[s] + SELL::C * w;
  }
  const int64_t slots = out.soff[out.nslices];
  out.ci.assign(slots, 0);
  out.v.assign(slots, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < out.nslices; ++s) {
    const int64_t w = (out.soff[s + 1] - out.soff[s]) / SELL::C;
    for (int64_t lane = 0; lane < SELL::C; ++lane) {
      const int64_t q = s * SELL::C + lane;
      if (q >= n) continue;
      const int64_t r = out.perm[q], len = A.rp[r + 1] - A.rp[r];
      for (int64_t j = 0; j < w; ++j) {
        const int64_t slot = out.soff[s] + SELL::C * j + lane;
        if (j < len) {
          out.ci[slot] = A.ci[A.rp[r] + j];
          out.v[slot] = A.v[A.rp[r] + j];
        } else {
          out.ci[slot] = len > 0 ? A.ci[A.rp[r]] : 0;
        }
      }
    }
  }
}

bool build_bsr3(const HCSR& A, double max_fill, BSR3& out) {
  out = BSR3();
  if (A.nrows % 3 != 0 || A.nrows != A.ncols || A.nrows == 0) return false;
  const int64_t nb = A.nrows / 3;
  std::vector<int64_t> cnt(nb, 0);
  auto block_cols = [&](int64_t I, std::vector<int32_t>& cols) {
    cols.clear();
    for (int r = 0; r < 3; ++r)
      for (int64_t k = A.rp[3 * I + r]; k < A.rp[3 * I + r + 1]; ++k) cols.push_back(A.ci[k] / 3);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
  };
#pragma omp parallel
  {
    std::vector<int32_t> cols;
#pragma omp for schedule(static)
    for (int64_t I = 0; I < nb; ++I) { block_cols(I, cols); cnt[I] = (int64_t)cols.size(); }
  }
  int64_t nblocks = 0;
  for (int64_t I = 0; I < nb; ++I) nblocks += cnt[I];
  if ((double)nblocks * 9.0 > max_fill * (double)A.nnz()) return false;
  const int64_t ns = (nb + BSR3::W - 1) / BSR3::W;
  out.nbrows = nb;
  out.nslices = ns;
  out.nblocks = nblocks;
  out.soff.assign(ns + 1, 0);
  for (int64_t sl = 0; sl < ns; ++sl) {
    int64_t w = 0;
    for (int64_t I = sl * BSR3::W; I < std::min(nb, (sl + 1) * BSR3::W); ++I) w = std::max(w, cnt[I]);
    out.soff[sl + 1] = out.soff[sl] + BSR3::W * w;
  }
  const int64_t slots = out.soff[ns];
  out.bci.assign(slots, 0);
  out.v.assign(9 * slots, 0.0);
#pragma omp parallel
  {
    std::vector<int32_t> cols;
#pragma omp for schedule(static)
    for (int64_t sl = 0; sl < ns; ++sl) {
      const int64_t s0 = out.soff[sl], w = (out.soff[sl + 1] - s0) / BSR3::W;
      for (int lane = 0; lane < BSR3::W; ++lane) {
        const int64_t I = sl * BSR3::W + lane;
        const int32_t pad = (int32_t)std::min(I, nb - 1);  // padding slots: own block row, zero values
        for (int64_t j = 0; j < w; ++j) out.bci[s0 + BSR3::W * j + lane] = pad;
        if (I >= nb) continue;
        block_cols(I, cols);
        for (size_t j = 0; j < cols.size(); ++j) out.bci[s0 + BSR3::W * j + lane] = cols[j];
      }
      bsr3_fill_slice(A, out, sl, out.v.data() + 9 * s0);
    }
  }
  return true;
}

void bsr3_fill_slice(const HCSR& A, const BSR3& L, int64_t sl, double* out) {
  const int64_t s0 = L.soff[sl], w = (L.soff[sl + 1] - s0) / BSR3::W;
  std::fill(out, out + 9 * BSR3::W * w, 0.0);
  for (int lane = 0; lane < BSR3::W; ++lane) {
    const int64_t I = sl * BSR3::W + lane;
    if (I >= L.nbrows) continue;
    for (int r = 0; r < 3; ++r) {
      int64_t b = 0;  // the row's block columns ascend with j, as its entries do
      for (int64_t k = A.rp[3 * I + r]; k < A.rp[3 * I + r + 1]; ++k) {
        const int32_t J = A.ci[k] / 3;
        while (L.bci[s0 + BSR3::W * b + lane] < J) ++b;
        const int c = A.ci[k] % 3;
        out[(9 * b + 3 * r + c) * BSR3::W + lane] = A.v[k];
      }
    }
  }
}

int validate_csr(const amgf_csr* a, const char* name, bool square, std::string& err) {
  char buf[256];
  if (!a || a->nrows < 0 || a->ncols <= 0 || a->nnz < 0 || (a->nrows > 0 && (!a->row_ptr || !a->col_idx || !a->val))) {
    snprintf(buf, sizeof buf, "%s: null or negative-size CSR", name); err = buf; return AMGF_ERR_INVALID_ARG;
  }
  if (square && a->nrows != a->ncols) { snprintf(buf, sizeof buf, "%s: not square", name); err = buf; return AMGF_ERR_INVALID_ARG; }
  if (a->ncols > INT32_MAX) { snprintf(buf, sizeof buf, "%s: too many columns for int32 indices", name); err = buf; return AMGF_ERR_INVALID_ARG; }
  if (a->nrows == 0) return AMGF_OK;
  if (a->row_ptr[0] != 0 || a->row_ptr[a->nrows] != a->nnz) { snprintf(buf, sizeof buf, "%s: row_ptr[0] or row_ptr[n] wrong", name); err = buf; return AMGF_ERR_INVALID_ARG; }
  int bad = 0, nonfinite = 0;
#pragma omp parallel for schedule(static) reduction(| : bad, nonfinite)
  for (int64_t i = 0; i < a->nrows; ++i) {
    if (a->row_ptr[i + 1] < a->row_ptr[i]) { bad |= 1; continue; }
    for (int64_t k = a->row_ptr[i]; k < a->row_ptr[i + 1]; ++k) {
      const int64_t c = a->col_idx[k];
      if (c < 0 || c >= a->ncols || (k > a->row_ptr[i] && c <= a->col_idx[k - 1])) bad |= 1;
      if (!std::isfinite(a->val[k])) nonfinite |= 1;
    }
  }
  if (bad) { snprintf(buf, sizeof buf, "%s: row_ptr not monotone or column indices unsorted/out of range", name); err = buf; return AMGF_ERR_INVALID_ARG; }
  if (nonfinite) { snprintf(buf, sizeof buf, "%s: non-finite value", name); err = buf; return AMGF_ERR_NONFINITE; }
  return AMGF_OK;
}

namespace {
// Contact part of S row by row: for every DOF a with a nonzero column of J (ascending in
// crows), the columns b (ascending) and sums sum_r J_ra D_r J_rb over the constraints r of a,
// each sum in ascending r and ascending position within row r of J.
struct ContactRows {
  std::vector<int64_t> crows;
  std::vector<std::vector<int32_t>> ccol;
  std::vector<std::vector<double>> cacc;
};

int contact_rows(int64_t n, const amgf_csr* J, const double* D, ContactRows& cr, std::string& err) {
  const int64_t m = J ? J->nrows : 0;
  for (int64_t r = 0; r < m; ++r) {
    if (!std::isfinite(D[r])) { err = "D has a non-finite entry"; return AMGF_ERR_NONFINITE; }
    if (!(D[r] > 0.0)) { err = "D has a non-positive entry"; return AMGF_ERR_NOT_SPD; }
  }
  // column lists of J: for DOF a, the constraints r (ascending) with J_ra != 0
  std::vector<int64_t> crp(n + 1, 0);
  std::vector<int64_t> crow;
  std::vector<double> cval;
  if (m > 0) {
    for (int64_t k = 0; k < J->nnz; ++k) crp[J->col_idx[k] + 1]++;
    for (int64_t i = 0; i < n; ++i) crp[i + 1] += crp[i];
    crow.resize(J->nnz);
    cval.resize(J->nnz);
    std::vector<int64_t> pos(crp.begin(), crp.end() - 1);
    for (int64_t r = 0; r < m; ++r)
      for (int64_t k = J->row_ptr[r]; k < J->row_ptr[r + 1]; ++k) {
        const int64_t p = pos[J->col_idx[k]]++;
        crow[p] = r;
        cval[p] = J->val[k];
      }
  }
  cr.crows.clear();
  for (int64_t a = 0; a < n; ++a)
    if (crp[a + 1] > crp[a]) cr.crows.push_back(a);
  cr.ccol.assign(cr.crows.size(), {});
  cr.cacc.assign(cr.crows.size(), {});
#pragma omp parallel
  {
    std::vector<double> acc(n, 0.0);
    std::vector<int64_t> mark(n, -1);
    std::vector<int32_t> cols;
#pragma omp for schedule(dynamic, 64)
    for (int64_t q = 0; q < (int64_t)cr.crows.size(); ++q) {
      const int64_t a = cr.crows[q];
      cols.clear();
      for (int64_t k = crp[a]; k < crp[a + 1]; ++k) {
        const int64_t r = crow[k];
        const double jra = cval[k];
        for (int64_t kk = J->row_ptr[r]; kk < J->row_ptr[r + 1]; ++kk) {
          const int32_t b = J->col_idx[kk];
          const double djrb = D[r] * J->val[kk];
          if (mark[b] != a) { mark[b] = a; acc[b] = 0.0; cols.push_back(b); }
          acc[b] += jra * djrb;
        }
      }
      std::sort(cols.begin(), cols.end());
      cr.ccol[q] = cols;
      cr.cacc[q].resize(cols.size());
      for (size_t u = 0; u < cols.size(); ++u) cr.cacc[q][u] = acc[cols[u]];
    }
  }
  return AMGF_OK;
}

// merge of row a of K with contact row q (K value first, contact sum added to it); emit(j, v)
template <typename Emit>
void merge_row(const amgf_csr* K, const ContactRows& cr, int64_t a, int64_t q, Emit&& emit) {
  int64_t p = K->row_ptr[a], pe = K->row_ptr[a + 1];
  const std::vector<int32_t>& cols = cr.ccol[q];
  size_t u = 0;
  while (p < pe || u < cols.size()) {
    if (u >= cols.size() || (p < pe && K->col_idx[p] < cols[u])) { emit(K->col_idx[p], K->val[p]); ++p; }
    else if (p >= pe || cols[u] < K->col_idx[p]) { emit(cols[u], cr.cacc[q][u]); ++u; }
    else { emit(K->col_idx[p], K->val[p] + cr.cacc[q][u]); ++p; ++u; }
  }
}
}  // namespace

int assemble_S(const amgf_csr* K, const amgf_csr* J, const double* D, HCSR& S, std::string& err) {
  const int64_t n = K->nrows;
  ContactRows cr;
  int st = contact_rows(n, J, D, cr, err);
  if (st) return st;
  // Rows without a contact column are copied from K; the (few) contact rows are merged.
  // Two passes: row lengths, then values written in place.
  std::vector<int64_t> qof(n, -1);
  for (int64_t q = 0; q < (int64_t)cr.crows.size(); ++q) qof[cr.crows[q]] = q;
  S.nrows = S.ncols = n;
  S.rp.assign(n + 1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t a = 0; a < n; ++a) {
    int64_t len = K->row_ptr[a + 1] - K->row_ptr[a];
    if (qof[a] >= 0) {
      len = 0;
      merge_row(K, cr, a, qof[a], [&](int32_t, double) { ++len; });
    }
    S.rp[a + 1] = len;
  }
  for (int64_t a = 0; a < n; ++a) S.rp[a + 1] += S.rp[a];
  S.ci.resize(S.rp[n]);
  S.v.resize(S.rp[n]);
#pragma omp parallel for schedule(static)
  for (int64_t a = 0; a < n; ++a) {
    int64_t o = S.rp[a];
    if (qof[a] < 0) {
      std::copy(K->col_idx + K->row_ptr[a], K->col_idx + K->row_ptr[a + 1], S.ci.begin() + o);
      std::copy(K->val + K->row_ptr[a], K->val + K->row_ptr[a + 1], S.v.begin() + o);
    } else {
      merge_row(K, cr, a, qof[a], [&](int32_t j, double v) { S.ci[o] = j; S.v[o] = v; ++o; });
    }
  }
  return AMGF_OK;
}

int refresh_contact_rows(HCSR& S, const amgf_csr* K, const amgf_csr* J, const double* D,
                         std::vector<int64_t>& rows, std::string& err) {
  const int64_t n = K->nrows;
  ContactRows cr;
  int st = contact_rows(n, J, D, cr, err);
  if (st) return st;
  bool same = S.nrows == n;
  for (int64_t q = 0; same && q < (int64_t)cr.crows.size(); ++q) {
    const int64_t a = cr.crows[q];
    int64_t o = S.rp[a];
    merge_row(K, cr, a, q, [&](int32_t j, double) { same = same && o < S.rp[a + 1] && S.ci[o] == j; ++o; });
    same = same && o == S.rp[a + 1];
  }
  if (!same) { err = "contact rows changed their pattern"; return AMGF_ERR_INVALID_ARG; }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < (int64_t)cr.crows.size(); ++q) {
    const int64_t a = cr.crows[q];
    int64_t o = S.rp[a];
    merge_row(K, cr, a, q, [&](int32_t, double v) { S.v[o++] = v; });
  }
  rows = cr.crows;
  return AMGF_OK;
}

int build_hierarchy(HCSR S, const amgf_options& o, Hierarchy& H, std::string& err) {
  H = Hierarchy();
  double t_str = 0, t_rs = 0, t_int = 0, t_gal = 0;
  auto now = [] {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
  };
  const int64_t n0 = S.nrows;
  H.A.push_back(std::move(S));  // A_0 takes the caller's matrix (moved in by callers that are done with it)
  H.func.emplace_back(n0);
  for (int64_t i = 0; i < n0; ++i) H.func[0][i] = o.num_functions > 1 ? (int32_t)(i % o.num_functions) : 0;
  int l = 0;
  for (;;) {
    const HCSR& A = H.A[l];
    const int64_t n = A.nrows;
    std::vector<double> l1(n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) s += std::fabs(A.v[k]);
      l1[i] = s;
    }
    H.l1.push_back(std::move(l1));
    if (n <= o.max_coarse || l + 1 >= o.max_levels || l + 1 >= 32) break;
    std::vector<int64_t> srp;
    std::vector<int32_t> sci;
    double t0 = now();
    strength_graph(A, H.func[l], o.strength_theta, srp, sci);
    double t1 = now();
    std::vector<int8_t> cf = ruge_stueben(n, srp, sci);
    double t2 = now();
    int64_t nc = 0;
    HCSR P = build_interpolation(A, srp, sci, H.func[l], cf, o.interp, o.p_max, nc);
    double t3 = now();
    t_str += t1 - t0; t_rs += t2 - t1; t_int += t3 - t2;
    if (nc == 0 || nc == n) break;  // coarsening stalled: this level is the coarsest
    HCSR R = transpose(P);
    HCSR AP = spgemm(A, P);
    HCSR Ac = spgemm(R, AP);
    t_gal += now() - t3;
    H.cf.push_back(cf);
    std::vector<int32_t> fc;
    fc.reserve(nc);
    for (int64_t i = 0; i < n; ++i)
      if (cf[i]) fc.push_back(H.func[l][i]);
    H.P.push_back(std::move(P));
    H.R.push_back(std::move(R));
    H.A.push_back(std::move(Ac));
    H.func.push_back(std::move(fc));
    ++l;
  }
  if (o.verbose)
    fprintf(stderr, "amgf: hierarchy: strength %.2fs, coarsening %.2fs, interpolation %.2fs, Galerkin %.2fs\n", t_str,
            t_rs, t_int, t_gal);
  const HCSR& AL = H.A.back();
  const int64_t nL = AL.nrows;
  if (nL > 8192) { err = "coarsest level too large for a dense solve"; return AMGF_ERR_INVALID_ARG; }
  std::vector<double> dense(nL * nL, 0.0);
  for (int64_t i = 0; i < nL; ++i)
    for (int64_t k = AL.rp[i]; k < AL.rp[i + 1]; ++k) dense[i * nL + AL.ci[k]] = AL.v[k];
  if (!spd_inverse(dense, nL, H.coarse_inv)) { err = "coarsest matrix is not SPD"; return AMGF_ERR_NOT_SPD; }
  H.n_coarse = nL;
  return AMGF_OK;
}

int update_hierarchy_contact(Hierarchy& H, const HCSR* S, const amgf_csr* J, const double* dD,
                             std::vector<std::vector<int64_t>>* changed, std::string& err) {
  const int nlev = H.nlev();
  if (S) H.A[0] = *S;
  if (changed) changed->assign(nlev, {});
  if (J && J->nrows > 0 && nlev >= 2) {
    // dA_0 = J^T diag(dD) J
    HCSR Jh;
    Jh.nrows = J->nrows;
    Jh.ncols = J->ncols;
    Jh.rp.assign(J->row_ptr, J->row_ptr + J->nrows + 1);
    Jh.ci.assign(J->col_idx, J->col_idx + J->nnz);
    Jh.v.assign(J->val, J->val + J->nnz);
    HCSR DJ = Jh;
    for (int64_t r = 0; r < Jh.nrows; ++r)
      for (int64_t k = Jh.rp[r]; k < Jh.rp[r + 1]; ++k) DJ.v[k] = dD[r] * Jh.v[k];
    HCSR dA = spgemm(transpose(Jh), DJ);
    for (int l = 0; l + 1 < nlev; ++l) {
      HCSR dAc = spgemm(H.R[l], spgemm(dA, H.P[l]));
      HCSR& Ac = H.A[l + 1];
      // positions of the entries of dAc in Ac (dAc's pattern must lie inside Ac's)
      std::vector<int64_t> where(dAc.nnz(), -1);
      bool ok = true;
#pragma omp parallel for schedule(dynamic, 256) reduction(&& : ok)
      for (int64_t i = 0; i < dAc.nrows; ++i) {
        int64_t p = Ac.rp[i];
        for (int64_t k = dAc.rp[i]; k < dAc.rp[i + 1]; ++k) {
          while (p < Ac.rp[i + 1] && Ac.ci[p] < dAc.ci[k]) ++p;
          if (p == Ac.rp[i + 1] || Ac.ci[p] != dAc.ci[k]) { ok = false; break; }
          where[k] = p;
        }
      }
      if (!ok) { err = "contact update outside the coarse pattern"; return AMGF_ERR_INVALID_ARG; }
#pragma omp parallel for schedule(static)
      for (int64_t k = 0; k < dAc.nnz(); ++k) Ac.v[where[k]] += dAc.v[k];
      if (changed) (*changed)[l + 1] = std::move(where);
      dA = std::move(dAc);
    }
  }
  for (int l = 0; l < nlev; ++l) {
    const HCSR& A = H.A[l];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A.nrows; ++i) {
      double a = 0.0;
      for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) a += std::fabs(A.v[k]);
      H.l1[l][i] = a;
    }
  }
  const HCSR& AL = H.A.back();
  const int64_t nL = AL.nrows;
  std::vector<double> dense(nL * nL, 0.0);
  for (int64_t i = 0; i < nL; ++i)
    for (int64_t k = AL.rp[i]; k < AL.rp[i + 1]; ++k) dense[i * nL + AL.ci[k]] = AL.v[k];
  if (!spd_inverse(dense, nL, H.coarse_inv)) { err = "coarsest matrix is not SPD"; return AMGF_ERR_NOT_SPD; }
  return AMGF_OK;
}

int add_diagonal(HCSR& A, const double* E, std::string& err) {
  const int64_t n = A.nrows;
  for (int64_t i = 0; i < n; ++i) {
    if (!std::isfinite(E[i])) { err = "bound diagonal has a non-finite entry"; return AMGF_ERR_NONFINITE; }
    if (E[i] < 0.0) { err = "bound diagonal has a negative entry"; return AMGF_ERR_NOT_SPD; }
  }
  HCSR B;
  B.nrows = A.nrows;
  B.ncols = A.ncols;
  B.rp.assign(n + 1, 0);
  B.ci.reserve(A.ci.size() + n);
  B.v.reserve(A.v.size() + n);
  for (int64_t i = 0; i < n; ++i) {
    bool done = E[i] == 0.0;
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int32_t j = A.ci[k];
      if (!done && j > i) { B.ci.push_back((int32_t)i); B.v.push_back(E[i]); done = true; }
      if (j == i) { B.ci.push_back(j); B.v.push_back(A.v[k] + E[i]); done = true; continue; }
      B.ci.push_back(j);
      B.v.push_back(A.v[k]);
    }
    if (!done) { B.ci.push_back((int32_t)i); B.v.push_back(E[i]); }
    B.rp[i + 1] = (int64_t)B.ci.size();
  }
  A = std::move(B);
  return AMGF_OK;
}

void smoother_features(const Hierarchy& H, const amgf_csr* J, const double* D, const double* E, int64_t n,
                       std::vector<std::vector<float>>& feat) {
  const int nlev = H.nlev();
  feat.assign(nlev > 1 ? nlev - 1 : 0, std::vector<float>());
  std::vector<double> d(n, 0.0);
  std::vector<int8_t> flag(n, 0);
  if (J && J->nrows > 0)
    for (int64_t r = 0; r < J->nrows; ++r)
      for (int64_t k = J->row_ptr[r]; k < J->row_ptr[r + 1]; ++k) {
        d[J->col_idx[k]] += J->val[k] * (D[r] * J->val[k]);
        if (J->val[k] != 0.0) flag[J->col_idx[k]] = 1;
      }
  if (E)
    for (int64_t i = 0; i < n; ++i) d[i] += E[i];
  for (int l = 0; l + 1 < nlev; ++l) {
    const HCSR& A = H.A[l];
    const int64_t nl = A.nrows;
    std::vector<float>& f = feat[l];
    f.resize(6 * nl);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nl; ++i) {
      double aii = 0.0;
      for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
        if (A.ci[k] == i) aii = A.v[k];
      const double l1 = H.l1[l][i];
      f[6 * i + 0] = (float)(std::log10(aii) / 10.0);
      f[6 * i + 1] = (float)(std::log10(l1) / 10.0);
      f[6 * i + 2] = (float)(aii / l1);
      f[6 * i + 3] = flag[i] ? 1.0f : 0.0f;
      f[6 * i + 4] = (float)(std::log10(1.0 + d[i]) / 10.0);
      f[6 * i + 5] = (float)((double)l / (double)(nlev - 1));
    }
    int64_t c = 0;
    for (int64_t i = 0; i < nl; ++i)
      if (H.cf[l][i]) { d[c] = d[i]; flag[c] = flag[i]; ++c; }
  }
}

int filter_solve_host(const Filter& F, const double* v_ic, double* w_ic, std::string& err) {
  if (F.nc == 0) { err = "empty contact set"; return AMGF_ERR_INVALID_ARG; }
  const int64_t nb = F.nb, tot = nb * F.nblk;
  // factor position p -> place of DOF gidx[p] in I_c (ascending)
  std::vector<int64_t> place(F.nc);
  for (int64_t p = 0; p < F.nc; ++p)
    place[p] = std::lower_bound(F.ic.begin(), F.ic.end(), F.gidx[p]) - F.ic.begin();
  std::vector<double> v(tot, 0.0), x(tot, 0.0), in0(nb), in1(nb);
  for (int64_t p = 0; p < F.nc; ++p) v[p] = v_ic[place[p]];
  if (F.algo == 1) {  // block LDL^T: y_i = v_i - G_i y_{i-1}; z_i = D_i^{-1} y_i; w_i = z_i - G_{i+1}^T w_{i+1}
    if (F.G.empty()) { err = "no factor on the host"; return AMGF_ERR_INVALID_ARG; }
    const int64_t bsz = nb * nb;
    for (int64_t i = 1; i < F.nblk; ++i)
      for (int64_t r = 0; r < nb; ++r) {
        double acc = 0.0;
        for (int64_t c = 0; c < nb; ++c) acc += F.G[i * bsz + r * nb + c] * v[(i - 1) * nb + c];
        v[i * nb + r] -= acc;
      }
    for (int64_t i = 0; i < F.nblk; ++i)
      for (int64_t r = 0; r < nb; ++r) {
        double acc = 0.0;
        for (int64_t c = 0; c < nb; ++c) acc += F.Dinv[i * bsz + r * nb + c] * v[i * nb + c];
        x[i * nb + r] = acc;
      }
    for (int64_t i = F.nblk - 2; i >= 0; --i)
      for (int64_t r = 0; r < nb; ++r) {
        double acc = 0.0;
        for (int64_t c = 0; c < nb; ++c) acc += F.GT[(i + 1) * bsz + r * nb + c] * x[(i + 1) * nb + c];
        x[i * nb + r] -= acc;
      }
    for (int64_t p = 0; p < F.nc; ++p) w_ic[place[p]] = x[p];
    return AMGF_OK;
  }
  if (F.M.empty()) { err = "no cyclic reduction factor on the host"; return AMGF_ERR_INVALID_ARG; }
  const int nphase = (int)F.phase_off.size() - 1;
  for (int q = 0; q < nphase; ++q) {
    for (int64_t t = F.phase_off[q]; t < F.phase_off[q + 1]; ++t) {
      const FilterTask& T = F.tasks[t];
      const std::vector<double>& src = T.kind == 2 ? x : v;
      if (T.in0 >= 0) std::copy(src.begin() + (int64_t)T.in0 * nb, src.begin() + (int64_t)(T.in0 + 1) * nb, in0.begin());
      if (T.in1 >= 0) std::copy(src.begin() + (int64_t)T.in1 * nb, src.begin() + (int64_t)(T.in1 + 1) * nb, in1.begin());
      for (int64_t row = 0; row < nb; ++row) {
        double s = 0.0;
        if (T.m0 >= 0 && T.in0 >= 0)
          for (int64_t c = 0; c < nb; ++c) s += F.M[(T.m0 * nb + row) * nb + c] * in0[c];
        if (T.m1 >= 0 && T.in1 >= 0)
          for (int64_t c = 0; c < nb; ++c) s += F.M[(T.m1 * nb + row) * nb + c] * in1[c];
        const int64_t p = (int64_t)T.out * nb + row;
        if (T.kind == 0) x[p] = s;
        else if (T.kind == 1) v[p] = v[p] - s;
        else x[p] = x[p] - s;
      }
    }
  }
  for (int64_t p = 0; p < F.nc; ++p) w_ic[place[p]] = x[p];
  return AMGF_OK;
}

int build_filter(const HCSR& S, const amgf_csr* J, const amgf_options& o, Filter& F, std::string& err) {
  F = Filter();
  const int64_t n = S.nrows;
  std::vector<char> in(n, 0);
  if (o.contact_components == 2) {
    std::fill(in.begin(), in.end(), 1);
  } else if (J && J->nrows > 0) {
    const int64_t nf = std::max(1, o.num_functions);
    for (int64_t k = 0; k < J->nnz; ++k) {
      if (J->val[k] == 0.0) continue;
      const int64_t c = J->col_idx[k];
      if (o.contact_components == 1) {
        const int64_t node = c / nf;
        for (int64_t d = 0; d < nf; ++d)
          if (node * nf + d < n) in[node * nf + d] = 1;
      } else {
        in[c] = 1;
      }
    }
  }
  for (int64_t i = 0; i < n; ++i)
    if (in[i]) F.ic.push_back(i);
  F.nc = (int64_t)F.ic.size();
  if (F.nc == 0) return AMGF_OK;
  const int64_t nc = F.nc;
  std::vector<int64_t> where(n, -1);
  for (int64_t t = 0; t < nc; ++t) where[F.ic[t]] = t;
  // adjacency of A_w (I_c numbering)
  HCSR Aw;
  Aw.nrows = Aw.ncols = nc;
  Aw.rp.assign(nc + 1, 0);
  for (int64_t t = 0; t < nc; ++t) {
    const int64_t i = F.ic[t];
    for (int64_t k = S.rp[i]; k < S.rp[i + 1]; ++k) {
      const int64_t p = where[S.ci[k]];
      if (p >= 0) { Aw.ci.push_back((int32_t)p); Aw.v.push_back(S.v[k]); }
    }
    Aw.rp[t + 1] = (int64_t)Aw.ci.size();
  }
  // reverse Cuthill-McKee from a pseudo-peripheral vertex of each component
  std::vector<int64_t> deg(nc);
  for (int64_t t = 0; t < nc; ++t) deg[t] = Aw.rp[t + 1] - Aw.rp[t];
  std::vector<char> seen(nc, 0);
  std::vector<int64_t> order;
  order.reserve(nc);
  std::vector<int64_t> lvl(nc, -1);
  auto bfs_levels = [&](int64_t root, std::vector<int64_t>& comp) {  // returns eccentricity
    comp.clear();
    comp.push_back(root);
    lvl[root] = 0;
    int64_t ecc = 0;
    for (size_t h = 0; h < comp.size(); ++h) {
      const int64_t u = comp[h];
      for (int64_t k = Aw.rp[u]; k < Aw.rp[u + 1]; ++k) {
        const int64_t v = Aw.ci[k];
        if (lvl[v] < 0) { lvl[v] = lvl[u] + 1; ecc = std::max(ecc, lvl[v]); comp.push_back(v); }
      }
    }
    return ecc;
  };
  std::vector<int64_t> comp;
  for (int64_t s0 = 0; s0 < nc; ++s0) {
    if (seen[s0]) continue;
    // component of s0; start from its minimum-degree vertex
    bfs_levels(s0, comp);
    int64_t root = s0;
    for (int64_t v : comp) if (deg[v] < deg[root] || (deg[v] == deg[root] && v < root)) root = v;
    for (int64_t v : comp) lvl[v] = -1;
    int64_t ecc = bfs_levels(root, comp);
    for (int it = 0; it < 16; ++it) {
      int64_t best = -1;
      for (int64_t v : comp)
        if (lvl[v] == ecc && (best < 0 || deg[v] < deg[best] || (deg[v] == deg[best] && v < best))) best = v;
      for (int64_t v : comp) lvl[v] = -1;
      const int64_t e2 = bfs_levels(best, comp);
      if (e2 > ecc) { root = best; ecc = e2; continue; }
      for (int64_t v : comp) lvl[v] = -1;
      bfs_levels(root, comp);
      break;
    }
    for (int64_t v : comp) lvl[v] = -1;
    // Cuthill-McKee from root: neighbours by increasing degree
    const size_t base = order.size();
    order.push_back(root);
    seen[root] = 1;
    std::vector<std::pair<int64_t, int64_t>> nb;
    for (size_t h = base; h < order.size(); ++h) {
      const int64_t u = order[h];
      nb.clear();
      for (int64_t k = Aw.rp[u]; k < Aw.rp[u + 1]; ++k) {
        const int64_t v = Aw.ci[k];
        if (!seen[v]) { seen[v] = 1; nb.emplace_back(deg[v], v); }
      }
      std::sort(nb.begin(), nb.end());
      for (auto& e : nb) order.push_back(e.second);
    }
  }
  std::reverse(order.begin(), order.end());
  std::vector<int64_t> pos(nc);
  for (int64_t p = 0; p < nc; ++p) pos[order[p]] = p;
  int64_t bw = 0;
  for (int64_t t = 0; t < nc; ++t)
    for (int64_t k = Aw.rp[t]; k < Aw.rp[t + 1]; ++k) { const int64_t d = pos[t] - pos[Aw.ci[k]]; bw = std::max<int64_t>(bw, d < 0 ? -d : d); }
  // block size = bandwidth, rounded up to even so every block row starts on a 16-byte boundary
  const int64_t nb = std::max<int64_t>((bw + 1) & ~int64_t(1), 2);
  const int64_t nblk = (nc + nb - 1) / nb;
  F.nb = nb;
  F.nblk = nblk;
  F.gidx.resize(nc);
  for (int64_t p = 0; p < nc; ++p) F.gidx[p] = F.ic[order[p]];
  // dense diagonal and sub-diagonal blocks of the permuted A_w (padding rows = identity)
  const int64_t bsz = nb * nb;
  std::vector<double> Ad(nblk * bsz, 0.0), As(nblk * bsz, 0.0);  // As[i] = A_{i,i-1}
  for (int64_t t = 0; t < nc; ++t) {
    const int64_t pi = pos[t], bi = pi / nb, ri = pi % nb;
    for (int64_t k = Aw.rp[t]; k < Aw.rp[t + 1]; ++k) {
      const int64_t pj = pos[Aw.ci[k]], bj = pj / nb, rj = pj % nb;
      if (bj == bi) Ad[bi * bsz + ri * nb + rj] = Aw.v[k];
      else if (bj == bi - 1) As[bi * bsz + ri * nb + rj] = Aw.v[k];
      else if (bj != bi + 1) { err = "filter ordering is not block tridiagonal"; return AMGF_ERR_INVALID_ARG; }
    }
  }
  for (int64_t p = nc; p < nblk * nb; ++p) Ad[(p / nb) * bsz + (p % nb) * nb + (p % nb)] = 1.0;
  F.algo = o.filter_algo == 1 ? 1 : 0;
  if (F.algo == 0) {
    const int st = build_bcr(nb, nblk, Ad, As, F, err);
    if (st) return st;
  } else {
  // block LDL^T: D_0 = A_00; G_i = A_{i,i-1} D_{i-1}^{-1}; D_i = A_ii - G_i A_{i-1,i}
  F.Dinv.assign(nblk * bsz, 0.0);
  F.G.assign(nblk * bsz, 0.0);
  F.GT.assign(nblk * bsz, 0.0);
  std::vector<double> Dcur(Ad.begin(), Ad.begin() + bsz), Rprev, W(bsz), WT(bsz);
  for (int64_t i = 0; i < nblk; ++i) {
    if (i > 0) {
      // D_i = A_i - W W^T with W = A_{i,i-1} R_{i-1}^{-T} (R_{i-1} the Cholesky factor of
      // D_{i-1}) and G_i = W R_{i-1}^{-1}: the update through the factor keeps D_i positive
      // definite when the pivots are ill-conditioned
      Dcur.assign(Ad.begin() + i * bsz, Ad.begin() + (i + 1) * bsz);
      double* Gi = F.G.data() + i * bsz;
      solve_rows_lower(nb, Rprev.data(), As.data() + i * bsz, W.data());
      solve_rows_upper(nb, Rprev.data(), W.data(), Gi);
      for (int64_t r = 0; r < nb; ++r)
        for (int64_t c = 0; c < nb; ++c) WT[r * nb + c] = W[c * nb + r];
      gemm(nb, W.data(), WT.data(), Dcur.data(), -1.0, 1.0);
      for (int64_t r = 0; r < nb; ++r)
        for (int64_t c = r + 1; c < nb; ++c) {
          const double s = 0.5 * (Dcur[r * nb + c] + Dcur[c * nb + r]);
          Dcur[r * nb + c] = Dcur[c * nb + r] = s;
        }
      for (int64_t r = 0; r < nb; ++r)
        for (int64_t c = 0; c < nb; ++c) F.GT[i * bsz + r * nb + c] = Gi[c * nb + r];
    }
    std::vector<double> inv;
    Rprev = Dcur;
    if (!cholesky(Rprev, nb)) {
      err = "filter matrix A_w is not SPD";
      return AMGF_ERR_NOT_SPD;
    }
    spd_inverse_factored(Rprev, nb, inv);
    std::copy(inv.begin(), inv.end(), F.Dinv.begin() + i * bsz);
  }
  }
  // A[:, I_c] on the rows that touch I_c, columns as factor positions
  std::vector<int64_t> rowcnt(n, 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int64_t k = S.rp[i]; k < S.rp[i + 1]; ++k) c += where[S.ci[k]] >= 0;
    rowcnt[i] = c;
  }
  F.Sc.rp.push_back(0);
  for (int64_t i = 0; i < n; ++i) {
    if (!rowcnt[i]) continue;
    F.touch_rows.push_back(i);
    for (int64_t k = S.rp[i]; k < S.rp[i + 1]; ++k) {
      const int64_t t = where[S.ci[k]];
      if (t >= 0) { F.Sc.ci.push_back((int32_t)pos[t]); F.Sc.v.push_back(S.v[k]); }
    }
    F.Sc.rp.push_back((int64_t)F.Sc.ci.size());
  }
  F.Sc.nrows = (int64_t)F.touch_rows.size();
  F.Sc.ncols = nc;
  return AMGF_OK;
}

}  // namespace amgf
