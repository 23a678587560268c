// Host-side setup of the AMGF solver: assembly of A = K + J^T D J, classical AMG
// hierarchy, contact set I_c and the block-tridiagonal factor of A_w = P^T A P.
// Internal to the library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/amgf.h"

namespace amgf {

// Allocator whose value-less resize leaves the new elements uninitialised: the large CSR
// arrays of the setup are sized first and then written in parallel, so the pages are first
// touched by the threads that write them instead of by one serial zero-fill.
template <class T>
struct NoInitAlloc : std::allocator<T> {
  using value_type = T;
  template <class U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() noexcept = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};

struct HCSR {
  int64_t nrows = 0, ncols = 0;
  std::vector<int64_t> rp;   // nrows + 1
  std::vector<int32_t, NoInitAlloc<int32_t>> ci;  // resize() leaves entries unset: write them all
  std::vector<double, NoInitAlloc<double>> v;
  int64_t nnz() const { return rp.empty() ? 0 : rp.back(); }
};

struct Hierarchy {
  std::vector<HCSR> A;                    // A[0] = S, A[l+1] = R_l A_l P_l
  std::vector<HCSR> P, R;                 // P[l]: n_l x n_{l+1}, R[l] = P[l]^T
  std::vector<std::vector<double>> l1;    // l1_i = sum_j |a_ij|
  std::vector<std::vector<int32_t>> func; // unknown (displacement component) of each row
  std::vector<std::vector<int8_t>> cf;    // C (1) / F (0) split of every coarsened level
  std::vector<double> coarse_inv;         // dense inverse of the coarsest A (row-major)
  int64_t n_coarse = 0;
  int nlev() const { return (int)A.size(); }
};

// One output block of a block cyclic reduction phase (all block indices are positions in
// the original block order; matrices are offsets in units of nb*nb doubles, -1 = absent):
//   kind 0: x[out] = M[m0] v[in0]                       (eliminated block: u = A^{-1} v)
//   kind 1: v[out] = v[out] - M[m0] v[in0] - M[m1] v[in1]   (kept block: reduced right side)
//   kind 2: x[out] = x[out] - M[m0] x[in0] - M[m1] x[in1]   (back substitution)
struct FilterTask {
  int64_t m0, m1;
  int32_t out, in0, in1, kind;
};

struct Filter {
  int64_t nc = 0;                 // |I_c|
  std::vector<int64_t> ic;        // I_c, ascending DOF indices
  std::vector<int64_t> gidx;      // factor position p -> DOF index (p < nc)
  int64_t nb = 0, nblk = 0;       // block size, number of diagonal blocks (nblk*nb >= nc)
  int algo = 0;                   // 0: block cyclic reduction, 1: sequential block LDL^T sweeps
  // algo 1: block LDL^T
  std::vector<double> Dinv;       // nblk blocks nb x nb: inverse of the block pivots D_i
  std::vector<double> G;          // nblk blocks: G_i = A_{i,i-1} D_{i-1}^{-1} (G_0 = 0)
  std::vector<double> GT;         // transposes of G_i
  // algo 0: odd-even block cyclic reduction; matrices nb x nb row-major in M, one task list
  // per phase: phases 0..L-1 reduce level 0..L-1, phase L solves the last block, phases
  // L+1..2L substitute back through levels L-1..0
  std::vector<double, NoInitAlloc<double>> M;  // sized once, every entry written
  std::vector<FilterTask> tasks;
  std::vector<int64_t> phase_off; // tasks of phase q: [phase_off[q], phase_off[q+1])
  int bcr_levels = 0;             // L
  // A[:, I_c] restricted to rows that touch I_c; columns are factor positions p
  std::vector<int64_t> touch_rows;
  HCSR Sc;
};

// Fine-level operator in 3x3 node blocks, in slices of W = 32 consecutive block rows (one
// GPU lane per block row): slice s has width w_s = the longest block row of the slice and
// owns slots soff[s] .. soff[s] + 32 w_s; block j of block row I = 32 s + lane sits in slot
// soff[s] + 32 j + lane, its column in bci[slot] and its value k (row k/3, column k%3) at
// v[9 soff[s] + (9 j + k) 32 + lane].  A warp's load of one value of block j of its 32 rows
// is one contiguous segment.  Padding slots (j beyond the row's length, rows past the end)
// hold zero values and the row's own block column.
struct BSR3 {
  static constexpr int64_t W = 32;
  int64_t nbrows = 0, nslices = 0;
  int64_t nblocks = 0;            // stored blocks, padding excluded
  std::vector<int64_t> soff;      // nslices + 1, multiples of W
  std::vector<int32_t> bci;
  std::vector<double> v;
};

// Converts A to BSR3 when n % 3 == 0 and the explicit zero fill inside the blocks stays
// below `max_fill` (9 x blocks / nnz); returns false otherwise.
bool build_bsr3(const HCSR& A, double max_fill, BSR3& out);

// Values of slice sl of A in the layout L (soff, bci, nbrows of an earlier build_bsr3 of a
// matrix with A's pattern): 9 * 32 * w_sl doubles in the order of BSR3::v from out on.
void bsr3_fill_slice(const HCSR& A, const BSR3& L, int64_t sl, double* out);

// Sliced ELL with one GPU lane per row (SELL-32-sigma): rows are sorted by length, longest first,
// within windows of `window` consecutive rows (ties keep their order), and cut into slices of
// 32 sorted rows.  Slice s has width w_s (its longest row) and owns 32 w_s slots from soff[s]:
// entry j of sorted row 32 s + lane sits in slot soff[s] + 32 j + lane, entries in the row's
// CSR order.  Slots past a row's end hold 0.0 and the row's first column (so a padded row reads
// only entries of x it uses anyway; column 0 for an empty row); the slots of the rows missing
// from the last slice hold 0.0 and column 0.  perm maps a sorted row to its row of A, pinv the
// other way.
struct SELL {
  static constexpr int64_t C = 32;
  int64_t nrows = 0, nslices = 0;
  std::vector<int64_t> soff;     // nslices + 1, multiples of C
  std::vector<int32_t> perm, pinv;
  std::vector<int32_t> ci;
  std::vector<double> v;
};
void build_sell(const HCSR& A, int64_t window, SELL& out);

// Slot of A's CSR entry k (row r: rp[r] <= k < rp[r + 1]) in a SELL built from A.
inline int64_t sell_slot(const HCSR& A, const SELL& S, int64_t r, int64_t k) {
  const int64_t q = S.pinv[r];
  return S.soff[q / SELL::C] + SELL::C * (k - A.rp[r]) + q % SELL::C;
}

// Input validation; returns an amgf_status.
int validate_csr(const amgf_csr* a, const char* name, bool square, std::string& err);

// A = K + J^T D J.  Entry (a, b) of J^T D J sums J_ra (D_r J_rb) over ascending r and is
// added to K_ab after it.
int assemble_S(const amgf_csr* K, const amgf_csr* J, const double* D, HCSR& S, std::string& err);

// The rows of an assembled S = K + J^T D_old J that J touches, rewritten for a new D with
// the arithmetic of assemble_S (same bits as a fresh assembly); rows = those DOFs, ascending.
// AMGF_ERR_INVALID_ARG if S's pattern is not the one assemble_S gives.
int refresh_contact_rows(HCSR& S, const amgf_csr* K, const amgf_csr* J, const double* D,
                         std::vector<int64_t>& rows, std::string& err);

// New contact term for a hierarchy built earlier (interpolation reused): A_0 = *S (when S is
// given; else A_0 already holds the new operator) and A_{l+1} += R_l dA_l P_l with
// dA_0 = J^T diag(dD) J, dD = D_new - D_old, so that every A_l is again the Galerkin operator
// of the new A for the old P; l1 sums and the coarsest inverse are recomputed.  changed
// (optional) receives, per level l >= 1, the positions in A_l.v that the update touched.
// AMGF_ERR_INVALID_ARG if an update falls outside a coarse pattern.
int update_hierarchy_contact(Hierarchy& H, const HCSR* S, const amgf_csr* J, const double* dD,
                             std::vector<std::vector<int64_t>>* changed, std::string& err);

// A += diag(E) (E finite, >= 0, length A.nrows): entries are added to stored diagonal
// entries, and a diagonal entry is inserted (in column order) where a row has none and
// E_i != 0.  The bound-constrained variant K + J^T D J + diag(D_lo + D_hi).
int add_diagonal(HCSR& A, const double* E, std::string& err);

// B := AMG(A): strength, Ruge-Stueben first pass, direct interpolation, Galerkin, l1 sums,
// dense inverse of the coarsest level.
int build_hierarchy(HCSR S, const amgf_options& o, Hierarchy& H, std::string& err);

// Features of the learned smoother for every smoothed level (6 per row, row-major):
//   log10(a_ii)/10, log10(l1_i)/10, a_ii/l1_i, contact flag, log10(1 + d_i)/10, l/(nlev-1),
// with d = diag(J^T D J) (+ E, the bound-constraint diagonal, when given) and the flag
// (nonzero column of J) on the fine level, carried to a
// coarse row from the fine C point it comes from.
void smoother_features(const Hierarchy& H, const amgf_csr* J, const double* D, const double* E, int64_t n,
                       std::vector<std::vector<float>>& feat);

// I_c, A_w = A[I_c, I_c], reverse Cuthill-McKee order, and the exact solver of the
// block-tridiagonal A_w: block cyclic reduction (o.filter_algo 0) or block LDL^T (1).
int build_filter(const HCSR& S, const amgf_csr* J, const amgf_options& o, Filter& F, std::string& err);
// w = A_w^{-1} v on the host with the cyclic reduction factor (the task semantics of the
// device solve, phase by phase); v, w of length nc in ascending-DOF order of I_c.
int filter_solve_host(const Filter& F, const double* v_ic, double* w_ic, std::string& err);


}  // namespace amgf
