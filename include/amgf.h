/*
 * amgf.h -- C ABI of the GB300 AMGF-PCG library.
 *
 * Solves the condensed interior-point Newton system
 *     A u = b,   A = K + J^T D J                       (Section 3, eq. linsystem1)
 * by preconditioned conjugate gradients with the AMGF preconditioner
 *     I - M A = (I - B A)(I - P A_w^{-1} P^T A)(I - B A),  A_w = P^T A P
 * (Section 5.1, Definition "AMGF"), where B is one classical AMG V-cycle built
 * from A (Remark after Lemma "condition number estimate": B := AMG(A) with l1
 * smoothers) and P is the natural embedding of the contact DOFs
 * I_c = nonzero columns of J (Section 4 and Section 5.1).
 *
 * The hierarchy setup (coarsening, Galerkin products, I_c and the factorisation
 * of A_w) runs on the host.  Every step of amgf_apply and amgf_pcg_solve runs
 * in this library's sm_103a CUDA kernels; there is no CPU fallback: without a
 * CUDA device every call that touches the device returns AMGF_ERR_CUDA.
 *
 * Conventions for every entry point:
 *   - Return value: an amgf_status code; 0 = success.  No call throws or aborts
 *     across the ABI.  amgf_last_error() gives a message for the calling thread.
 *   - Host arrays are read during the call only; the caller keeps ownership.
 *   - Device pointers (suffix _dev) are caller-owned, 8-byte aligned, of the
 *     stated length, on the device that was current at amgf_setup.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work is
 *     ordered after prior work on `stream`, and later work on `stream` sees its
 *     results; the library runs it on its own stream joined by events.
 *   - A handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef AMGF_H
#define AMGF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AMGF_OK = 0,
  AMGF_ERR_INVALID_ARG = 1,  /* null pointer, bad size, unsorted or out-of-range CSR index */
  AMGF_ERR_NONFINITE = 2,    /* NaN/Inf in D, b or in a PCG scalar */
  AMGF_ERR_NOT_SPD = 3,      /* D_r <= 0, non-positive pivot in the coarse or filter factor */
  AMGF_ERR_BREAKDOWN = 4,    /* p^T A p <= 0 or r^T z <= 0 during PCG */
  AMGF_ERR_NOT_CONVERGED = 5,/* maxit reached; x holds the last iterate */
  AMGF_ERR_CUDA = 6,         /* CUDA runtime error or no device; also a device-side wait of the
                                staged sweeps that gave up after 4 s (the kernel sets a flag and
                                returns instead of hanging; amgf_pcg_solve and amgf_time_kernel
                                read the flag, which stays set for the handle) */
  AMGF_ERR_OOM = 7           /* device or host allocation failed */
} amgf_status;

/* Host CSR matrix: row_ptr[nrows+1] (int64, row_ptr[0] = 0), col_idx[nnz] (int32,
 * strictly ascending within a row, 0 <= col < ncols), val[nnz] (float64). */
typedef struct {
  int64_t nrows, ncols, nnz;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
} amgf_csr;

typedef struct {
  double strength_theta;  /* AMG strength threshold (0.52) */
  double rtol;            /* PCG stop: sqrt(r^T z / r0^T z0) < rtol (1e-8); Section 4 uses this norm */
  int max_levels;         /* AMG levels including the coarsest (25) */
  int max_coarse;         /* stop coarsening at n_l <= max_coarse (1200); coarsest solved exactly */
  int num_functions;      /* unknowns per node for the unknown approach (3); DOF i has function i % 3 */
  int nu;                 /* l1-Jacobi sweeps before and after the coarse correction, or the
                             degree of the Chebyshev smoother (1) */
  int filter;             /* 1: AMGF (default); 0: plain AMG V-cycle, M = B */
  int contact_components; /* 0: I_c = nonzero columns of J; 1: all num_functions DOFs of those nodes;
                             2: all DOFs (P = I, test) */
  int maxit;              /* PCG iteration cap (5000, Section 6.1) */
  int use_graph;          /* 1: capture the PCG loop in one CUDA graph with a device-side while node */
  int verbose;            /* 1: print setup summary to stderr */
  int precision;          /* 0: FP64 throughout (default).  1: V-cycle in FP32 (FP32 matrices and
                             vectors, int32 indices, FP32 accumulation) inside an FP64 flexible PCG;
                             the outer residual, the dot products, the J^T D J term and the filter
                             solve stay FP64.  2: as 1 with the fine-level K values in BF16.
                             3: as 2 with every V-cycle matrix (coarse A_l, P_l, R_l) in BF16
                             (FP32 accumulation throughout).
                             Needs >= 2 levels and 3 unknowns per node, else FP64 is used. */
  int filter_algo;        /* exact solver of the block-tridiagonal A_w (Section 5.1 filter step; the
                             paper uses a sparse direct solver): 0 = odd-even block cyclic reduction,
                             one launch per reduction level (default); 1 = sequential block LDL^T
                             forward/backward sweeps on one thread-block cluster */
  int interp;             /* AMG interpolation: 0 = classical Ruge-Stueben interpolation (strong F
                             neighbours distributed over the strong C points, weak ones lumped;
                             rows whose lumped diagonal nearly vanishes use direct weights), the
                             default; 1 = direct interpolation with Stueben's sign split */
  int p_max;              /* interpolation truncation (4; 0 = none): every F row of P_l with more
                             weights keeps its p_max weights of largest magnitude (ties: smaller
                             coarse index), scaled by (sum of all) / (sum of kept) so that the
                             row sum is unchanged; rows whose kept weights sum to zero stay whole.
                             Lowers the operator complexity of the coarse levels. */
  int update_in_place;    /* 1 (default): amgf_update_D_fine writes the new values into the
                             device image (same arrays, same solve graph); 0: it rebuilds and
                             uploads the whole image, as amgf_update_D does */
  int smoother;           /* 0 (default): l1-Jacobi, nu sweeps x += W (b - A x), W = 1/l1;
                             1: Chebyshev polynomial of degree nu in W A for the interval
                             [cheby_lower, 1] (the l1 sums bound the spectrum of W A by 1), by the
                             three-term recurrence of Chebyshev acceleration; the same polynomial
                             before and after the coarse correction keeps B symmetric.  One
                             residual pass plus one vector update per degree.  Learned weights
                             (amgf_set_mlp) apply to smoother 0 only. */
  double cheby_lower;     /* lower end of the Chebyshev interval, in (0, 1) (0.3) */
  int stage_rows;         /* BF16 V-cycle matrices (precision 3): rows per tile of the staged sweeps of
                             the coarse levels whose rows hold at most 160 entries on average; a
                             producer warp copies each tile's row pointers, indices, values and
                             vectors into shared memory with bulk asynchronous copies while the
                             other warps sweep the tiles before it (32; rounded up to whole passes
                             of the CTA's row groups; 0: plain loads, csr_kernel, everywhere).
                             Same results either way.  At most 4096. */
  int stage_depth;        /* tiles in flight per CTA of the staged sweeps, 2..8 (2) */
  int sell_window;        /* FP64 V-cycle: the long-row coarse levels with enough rows to give each
                             GPU lane its own row are swept from a sliced-ELL copy (one lane per
                             row, slices of 32 rows sorted by length within windows of this many
                             rows; 256).  0: CSR with lane groups everywhere.  The per-row sums
                             then run in CSR order in one FMA chain instead of in lane-interleaved
                             partial sums, so the two forms differ by rounding. */
} amgf_options;

typedef struct {
  int iters;              /* PCG iterations (A p products) */
  int converged;          /* 1 if the stop test was met */
  int status;             /* amgf_status of the solve */
  int nlevels;
  double rel_res_precond; /* final sqrt(r^T z / r0^T z0) */
  double rz0;             /* r0^T z0 */
  double t_solve_s;       /* device time of the solve (CUDA events) */
  int64_t kernel_launches;/* this library's kernels executed by the solve */
  int mlp_fallback;       /* 1: the learned weights missed the stop test and the solve was redone
                             with theta = 1 (the plain l1-Jacobi smoother) */
  double rel_res_l2;      /* true relative residual ||b - A x||_2 / ||b||_2 of the returned x, from
                             one FP64 A x after the solve (not part of t_solve_s); 0 when b = 0.
                             With barrier entries up to D_max it stalls near u D_max |x| / |b|
                             while the preconditioned norm of the stop test keeps falling. */
  double t_setup_s;       /* host setup and upload time of the handle (amgf_info.t_setup_s) */
} amgf_stats;

typedef struct {
  int64_t n, m, nc;          /* DOFs, constraints, |I_c| */
  int nlevels;
  int64_t level_rows[32];
  int64_t level_nnz[32];     /* nnz(A_l) */
  int64_t interp_nnz[32];    /* nnz(P_l), l < nlevels-1 */
  int64_t filter_block;      /* block size of the block-tridiagonal A_w factor */
  int64_t filter_nblocks;
  double op_complexity;      /* sum nnz(A_l) / nnz(A_0) */
  double t_setup_s;          /* setup wall time (host setup and device upload) */
  double t_assemble_s;       /* of which: assembling A */
  double t_hierarchy_s;      /*           the AMG hierarchy */
  double t_filter_s;         /*           I_c, ordering and the A_w factor */
  int64_t staged_levels;     /* bit l set: the sweeps of level l run staged (amgf_options.stage_rows) */
  int64_t sell_levels;       /* bit l set: level l's FP64 sweeps run from the sliced-ELL copy
                                (amgf_options.sell_window) */
} amgf_info;

typedef struct amgf_ctx* amgf_handle;

/* Fill *o with the defaults listed above. */
int amgf_options_default(amgf_options* o);

/* Build the solver for A = K + J^T D J (Section 3, eq. linsystem1).
 * K: n x n SPD stiffness (host CSR).  J: m x n contact Jacobian (host CSR), may
 * have m = 0 (then I_c is empty).  D: host array of m positive finite values.
 * o: options (NULL = defaults).  On success *out owns all device memory. */
int amgf_setup(const amgf_csr* K, const amgf_csr* J, const double* D,
               const amgf_options* o, amgf_handle* out);

/* Host-only variant of amgf_setup: runs the whole host setup (A, the AMG hierarchy, I_c
 * and the A_w factor) without touching any CUDA device.  The handle only serves
 * amgf_get_info, amgf_export_matrix, amgf_export_contact_set, amgf_update_D and
 * amgf_destroy; every device call on it returns AMGF_ERR_INVALID_ARG. */
int amgf_setup_host(const amgf_csr* K, const amgf_csr* J, const double* D,
                    const amgf_options* o, amgf_handle* out);

/* New interior-point iterate: same K and J, new barrier diagonal D (host, length m).
 * Across IP iterations only D changes (Section 4); B := AMG(A) is rebuilt for the new A. */
int amgf_update_D(amgf_handle h, const double* D);

/* New IP iterate reusing the coarsening and interpolation of the last full setup (not in the
 * paper, which rebuilds B := AMG(A) for every A): A = K + J^T D J, the filter A_w and the
 * fine-level smoother weights are recomputed for the new D (host, length m), and every coarse
 * operator is brought up to date by the Galerkin product of the change of the contact term,
 * A_{l+1} += R_l dA_l P_l with dA_0 = J^T diag(D_new - D_old) J, so A_l = R ... A P ... for
 * the old P_l.  B therefore stays the V-cycle of a Galerkin hierarchy of the current A (and
 * M stays SPD, lambda_max(B A) <= 1); only its interpolation is from an earlier A, so PCG may
 * need more iterations.  Skips strength, coarsening, interpolation and the full Galerkin
 * products (most of the setup time).  With options.update_in_place (default) only values move
 * on the device: the contact rows of A (their 32-row slices of the fine-level image), the
 * touched coarse entries, l1 weights, the coarsest inverse, the filter matrices and the
 * learned smoother's inputs, written into the existing arrays (the solve graph stays valid);
 * the results equal those of a full re-upload bit for bit.  Falls back to the full re-upload
 * when a bound diagonal is present or the filter's layout changes, and to amgf_update_D when
 * the hierarchy has one level or an update would leave a coarse pattern.  Errors as
 * amgf_update_D. */
int amgf_update_D_fine(amgf_handle h, const double* D);

/* Bound-constrained variant (Section 3, remark on bound constraints): with the additional
 * bounds d_lo <= u - u_* <= d_hi the condensed matrix becomes K + J~^T D~ J~ with
 * J~ = [J; I; -I] and D~ = diag(D, D_lo, D_hi), i.e. A = K + J^T D J + diag(D_lo + D_hi).
 * d_lower, d_upper: host arrays of n finite values >= 0 (either may be NULL = 0), copied.
 * The diagonal term is added after J^T D J; the filter space stays the nonzero columns of
 * J (the bound rows touch every DOF and are not filtered; they only add to A's diagonal,
 * which AMG takes as part of A), and in mixed precision the term stays FP64 with the
 * contact term.  host_only != 0 behaves as amgf_setup_host.  Errors as amgf_setup, plus
 * AMGF_ERR_NONFINITE / AMGF_ERR_NOT_SPD for a non-finite / negative bound entry.  The paper
 * gives no solver for this variant beyond the matrix; this entry applies AMGF to it. */
int amgf_setup_bounds(const amgf_csr* K, const amgf_csr* J, const double* D, const double* d_lower,
                      const double* d_upper, const amgf_options* o, int host_only, amgf_handle* out);

/* New IP iterate of the bound-constrained variant: D (length m) and the bound barrier
 * diagonals (length n, NULL = 0; both NULL removes the bound term); same K and J. */
int amgf_update_bounds(amgf_handle h, const double* D, const double* d_lower, const double* d_upper);

/* z_dev = M r_dev, one AMGF application (Definition "AMGF"): y1 = B r; r1 = r - A y1;
 * y2 = y1 + P A_w^{-1} P^T r1; r2 = r1 - A P (A_w^{-1} P^T r1); z = y2 + B r2.
 * With filter = 0: z = B r.  Both vectors have length n.  r_dev and z_dev must not alias. */
int amgf_apply(amgf_handle h, const double* r_dev, double* z_dev, void* stream);

/* amgf_apply with copies of its intermediate vectors (tests; Definition "AMGF" in the product
 * form of Section 5.1): y1 = B r, r1 = r - A y1, w = A_w^{-1} P^T r1 (length nc, ascending-DOF
 * order of I_c) and r2 = r1 - A P w, each written to the caller's device buffer when its pointer
 * is not NULL; z_dev receives z = y1 + P w + B r2 exactly as amgf_apply computes it.  The copies
 * let a test check each step on the library's own vectors, e.g. that P^T r2 = P^T r1 - A_w w
 * vanishes to rounding whatever kappa(A_w) is.  w and r2 need options.filter = 1 and a nonempty
 * I_c (AMGF_ERR_INVALID_ARG otherwise); with filter = 0 (M = B) only y1 = z is written. */
int amgf_apply_stages(amgf_handle h, const double* r_dev, double* z_dev, double* y1_dev, double* r1_dev,
                      double* w_dev, double* r2_dev, void* stream);

/* x_dev = B r_dev, one V-cycle from a zero start (the B of Section 5.1). */
int amgf_vcycle(amgf_handle h, const double* r_dev, double* x_dev, void* stream);

/* y_dev = A x_dev with A = K + J^T D J. */
int amgf_matvec(amgf_handle h, const double* x_dev, double* y_dev, void* stream);

/* w_dev = A_w^{-1} v_dev with A_w = A[I_c, I_c] (Section 5.1); v, w of length nc in
 * ascending-DOF order of I_c.  An exact solve up to rounding: A_w is put in reverse
 * Cuthill-McKee order, where it is block tridiagonal, and solved by odd-even block cyclic
 * reduction (filter_algo 0) or block LDL^T sweeps (filter_algo 1). */
int amgf_filter_solve(amgf_handle h, const double* v_dev, double* w_dev, void* stream);

/* The same solve on the host with the filter's factor (either filter_algo), for handles of
 * amgf_setup_host (a device handle keeps the factor on the device only: AMGF_ERR_INVALID_ARG).
 * v, w: host arrays of length nc in ascending-DOF order of I_c.  The device solve runs the same
 * tasks phase by phase, so this checks the factorisation without a GPU. */
int amgf_filter_solve_host(amgf_handle h, const double* v, double* w);

/* Same result as amgf_filter_solve, for callers that cannot allocate device memory while
 * they run (another allocator owns the device, or a cudaMalloc and the synchronisation it
 * may imply are not allowed in their loop).  The paper has no counterpart: this is a
 * property of the library, not of the method.  Its four work vectors live in one array of
 * 524288 doubles (4 MiB) compiled into the library, which every GPU that loads the library
 * holds until the process exits; a filter needing more than 4 x 131072 doubles (block
 * size x number of blocks, see amgf_info) is rejected with AMGF_ERR_INVALID_ARG.  The call
 * allocates nothing.  Its first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call before any
 * stream capture.  All calls share the array: two calls whose work overlaps on the GPU
 * (different streams, or different handles on one device) race and give wrong results;
 * keep them ordered.  Nothing in the array needs clearing between calls. */
int amgf_filter_solve_noalloc(amgf_handle h, const double* v_dev, double* w_dev, void* stream);

/* PCG on A x = b (x_dev holds x0 on entry, the solution on exit), preconditioned by
 * M, stopped when sqrt(r^T z / r0^T z0) < rtol (Section 4) or after maxit
 * iterations.  Synchronises `stream` to fill *st (may be NULL).
 * Returns AMGF_ERR_NOT_CONVERGED when maxit is reached. */
int amgf_pcg_solve(amgf_handle h, const double* b_dev, double* x_dev, amgf_stats* st, void* stream);

/* Same as amgf_pcg_solve with host arrays (length n): copies b and x0 to the device,
 * solves, copies x back.  Blocking. */
int amgf_pcg_solve_host(amgf_handle h, const double* b_host, double* x_host, amgf_stats* st);

/* Learned smoother (not in the paper).  Every smoothed level's l1-Jacobi step is scaled
 * per row, W_i = theta_i / l1_i, with theta_i = 0.3 + 0.9 sigmoid(MLP(f_i)), an MLP
 * 6 -> 32 -> 32 -> 1 (ReLU) evaluated in FP32 on the GPU from the row's features f_i =
 * (log10(a_ii)/10, log10(l1_i)/10, a_ii/l1_i, contact flag, log10(1 + d_i)/10, l/(nlev-1)),
 * d = diag(J^T D J) on the fine level (a coarse row inherits flag and d from its fine C point).
 * theta in [0.3, 1.2] < 2 keeps the smoother convergent and B, M SPD.
 * weights: host array of 1313 floats laid out W1[32][6], b1[32], W2[32][32], b2[32],
 * w3[32], b3; NULL restores theta = 1.  The weights stay active across amgf_update_D.
 * With active weights, a PCG solve that misses its stop test is redone with theta = 1
 * (amgf_stats.mlp_fallback = 1). */
int amgf_set_mlp(amgf_handle h, const float* weights, int64_t nw);

/* `iters` Adam steps (lr, beta 0.9/0.999) on the MLP weights for this handle's hierarchy:
 * loss = mean over smoothed levels of ||(I - A_l W_l) r_l||^2 / ||r_l||^2 with r_l uniform in
 * (-1, 1) from SplitMix64 counters derived from `seed` and the step number.  params, adam_m,
 * adam_v (1313 floats each) and *adam_step are read and updated (host memory); loss (host,
 * length iters, may be NULL) receives the loss before each step.  Forward, backward and
 * update run in this library's kernels.  Needs an FP64 handle (precision 0) with >= 2 levels.
 * The active smoother weights (amgf_set_mlp) are left unchanged. */
int amgf_mlp_train(amgf_handle h, float* params, float* adam_m, float* adam_v, int64_t* adam_step,
                   int iters, float lr, uint64_t seed, float* loss);

/* The training objective of amgf_mlp_train and its gradient for given weights and given
 * vectors r_l (tests: the same kernels as one training step, without the Adam update).
 * params: 1313 floats (layout of amgf_set_mlp); r_all: host array holding r_0, r_1, ...,
 * r_{L-2} back to back (level_rows[l] doubles each, every level but the coarsest);
 * *loss = mean_l ||(I - A_l W_l) r_l||^2 / ||r_l||^2 (may be NULL); grad: 1313 floats,
 * d loss / d params.  Needs an FP64 handle with >= 2 levels.  The active smoother weights are
 * left unchanged. */
int amgf_mlp_grad(amgf_handle h, const float* params, const double* r_all, float* grad, double* loss);

/* Hierarchy and sizes. */
int amgf_get_info(amgf_handle h, amgf_info* info);

/* Host copy of a hierarchy matrix (tests).  which: 0 = A_l, 1 = P_l, 2 = R_l.
 * With row_ptr == NULL only *nrows, *ncols, *nnz are written. */
int amgf_export_matrix(amgf_handle h, int which, int level, int64_t* nrows, int64_t* ncols, int64_t* nnz,
                       int64_t* row_ptr, int32_t* col_idx, double* val);

/* Host copy of I_c (length nc, ascending DOF indices). */
int amgf_export_contact_set(amgf_handle h, int64_t* ic);

/* One launch of a PCG iteration, as recorded by amgf_profile_iteration. */
typedef struct {
  char op[64];    /* what the launch computes, e.g. "x + W (b - A x)" (the post-smoother) */
  int level;      /* hierarchy level of its operator (-1: filter phases, PCG scalars) */
  double ms;      /* CUDA-event time from the previous launch's end to this one's */
  double bytes;   /* algorithmic bytes: stored values + indices at their precision, one read of
                     every input vector (a gathered vector counted once), one write of every output */
  double flops;   /* 2 per stored nonzero or dense-matrix entry applied (0 for vector kernels) */
} amgf_launch_rec;

/* Runs one PCG iteration (A p, the x/r update, one AMGF application, the p update and the stop
 * test) on `stream` outside the captured graph, with a CUDA event after every kernel, and
 * returns each launch's time, algorithmic bytes and flops in launch order (*count = number of
 * launches; at most `cap` records are written).  Achieved bandwidth of a launch = bytes / ms.
 * Meant for profiling after an amgf_pcg_solve on the same handle: it restarts PCG from the
 * handle's current iterate (untimed) and runs one iteration of it; the next amgf_pcg_solve starts
 * afresh.  Not part of the paper. */
int amgf_profile_iteration(amgf_handle h, void* stream, amgf_launch_rec* recs, int cap, int* count);

/* Time `reps` back-to-back launches of one kernel of the solve phase on `stream`
 * with CUDA events, after `warmup` untimed launches.  which: 0 = fine-level
 * A x (SpMV of level 0), 1 = fine-level FP64 post-smoother, 2 = fine-level post-smoother
 * of the FP32 V-cycle (mixed-precision handles only), 3 = level-1 post-smoother in the
 * V-cycle's precision (hierarchies of >= 3 levels).  *ms = average per launch;
 * *bytes = algorithmic bytes one launch moves (values + indices + vectors). */
int amgf_time_kernel(amgf_handle h, int which, int warmup, int reps, void* stream,
                     double* ms, double* bytes);

/* Free all device and host memory of the handle. */
int amgf_destroy(amgf_handle h);

/* Message of the last error on the calling thread ("" if none). */
const char* amgf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AMGF_H */
