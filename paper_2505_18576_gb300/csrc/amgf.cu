// AMGF-PCG solve phase on one GPU and the C ABI of include/amgf.h.
//
// Device layout (one handle):
//   level l: A_l (CSR, int64 row pointers, int32 columns, FP64 values; the fine level in
//            3x3 node blocks, 32 block rows per slice), P_l, R_l = P_l^T, W_l = 1 / l1_l,
//            and four n_l-vectors (rhs, x, residual, output);
//   coarsest: dense inverse of A_L (FP64);
//   filter:   the block cyclic reduction of A_w (nb x nb FP64 blocks: eliminated-block
//             inverses and coupling products, one task list per phase) or, with
//             filter_algo = 1, its block LDL^T factor (G_i, G_i^T, D_i^{-1});
//             factor-position -> DOF map, and A[:, I_c] on the rows that touch I_c;
//   PCG:      x, r, z, p, q, apply scratch (y1, r1), device scalars (PcgState).
// One AMGF application (Definition "AMGF", Section 5.1):
//   y1 = B r  ->  r1 = r - A y1  ->  w = A_w^{-1} P^T r1,  y1 += P w  ->  r1 -= A P w
//   ->  z = y1 + B r1
// where only the rows of A that touch I_c take part in r1 -= A P w.  The PCG loop runs
// as one CUDA graph whose body sits in a device-side while node, so a solve makes no
// host round trip until it ends.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/amgf.h"
#include "kernels.cuh"
#include "setup.h"

namespace amgf {

thread_local std::string g_last_error;

static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? AMGF_ERR_OOM : AMGF_ERR_CUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    }                                                                                         \
  } while (0)

struct DCSR {
  int64_t nrows = 0, ncols = 0, nnz = 0;
  int level = -1;   // hierarchy level (per-launch records of amgf_profile_iteration)
  char role = 'A';  // 'A' level operator, 'P' interpolation, 'R' restriction, 'S' A[:, I_c] rows
  int64_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* v = nullptr;
  int K = 4;  // lanes per row
  // optional 3x3 node-block copy (sliced BSR3) used instead of the CSR arrays (fine level)
  bool bsr = false;
  int64_t nbrows = 0, nslices = 0, nblocks = 0;  // nblocks: stored blocks without padding
  int64_t* soff = nullptr;
  int32_t* bci = nullptr;
  double* bv = nullptr;
  // optional sliced-ELL copy (sell_kernel) for the SPMV / RESID / POST sweeps of a long-row
  // level; the CSR arrays stay for the other modes.  sell_h: host slice offsets and row
  // permutation (values dropped) for in-place value updates.
  int64_t* ell_soff = nullptr;
  int32_t* ell_perm = nullptr;
  int32_t* ell_ci = nullptr;
  double* ell_v = nullptr;
  SELL sell_h;
};

struct DCSRf {  // FP32 (or BF16) values: V-cycle levels of the mixed-precision solve
  int64_t nrows = 0, ncols = 0, nnz = 0;
  int level = -1;
  char role = 'A';
  int64_t* rp = nullptr;
  int32_t* ci = nullptr;
  float* v = nullptr;
  __nv_bfloat16* vb = nullptr;  // BF16 values instead of v (precision 3)
  int K = 4;
  int U = 4;                    // entries per lane and batch (8: long rows on a warp per row)
  // optional sliced-ELL copy (sell_kernel) of an interpolation or restriction operator
  int64_t* ell_soff = nullptr;
  int32_t* ell_perm = nullptr;
  int32_t* ell_ci = nullptr;
  float* ell_v = nullptr;
  __nv_bfloat16* ell_vb = nullptr;
  int64_t ell_nslices = 0;
  // staged sweeps (csr_staged_kernel) of a level operator; sg.ntiles == 0: csr_kernel
  StageArgs sg{};
  int sgrid = 0;
  size_t ssmem = 0;
};

struct DLevel {
  DCSR A, P, R;
  double* winv = nullptr;
  double *rhs = nullptr, *x = nullptr, *res = nullptr, *out = nullptr;
  double* d = nullptr;  // Chebyshev smoother: direction of the recurrence
  // FP32 copies used when the V-cycle runs in single precision
  DCSRf Af, Pf, Rf;
  float* winvf = nullptr;
  float *rhsf = nullptr, *xf = nullptr, *resf = nullptr, *outf = nullptr;
  float* df = nullptr;
  int64_t n = 0;
};

// Chebyshev smoother of degree k for the interval [lo, 1] of W A (three-term recurrence of
// Chebyshev acceleration): centre c = (1 + lo)/2, half-width h = (1 - lo)/2, s = c/h; the first
// step scales W r by 1/c, step j >= 1 uses d = a_j d + bc_j W r with rho_0 = 1/s,
// rho_j = 1/(2 s - rho_{j-1}), a_j = rho_j rho_{j-1}, bc_j = 2 rho_j / h.
struct ChebCoefs {
  double inv_c = 1.0;
  std::vector<double> a, bc;  // index j = 1 .. k-1 (entry 0 unused)
};
static ChebCoefs cheb_coefs(double lo, int k) {
  ChebCoefs r;
  const double cc = 0.5 * (1.0 + lo), hw = 0.5 * (1.0 - lo), sg = cc / hw;
  r.inv_c = 1.0 / cc;
  r.a.assign(k, 0.0);
  r.bc.assign(k, 0.0);
  double rho = 1.0 / sg;
  for (int j = 1; j < k; ++j) {
    const double rn = 1.0 / (2.0 * sg - rho);
    r.a[j] = rn * rho;
    r.bc[j] = 2.0 * rn / hw;
    rho = rn;
  }
  return r;
}

struct Ctx {
  amgf_options o{};
  int device = 0;
  int num_sms = 148;
  cudaStream_t s = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
  // host copies kept for amgf_update_D and exports
  HCSR Kh, Jh;
  std::vector<double> Eh;  // bound-constraint diagonal D_lo + D_hi (empty: none)
  std::vector<double> Dh;  // D of the current A (for amgf_update_D_fine)
  BSR3 bsr0;               // layout (soff, bci) of the fine-level BSR3 on the device, values dropped
  int64_t fM_count = 0;    // doubles in fM
  int64_t c_nnz = 0;       // entries of the contact-term CSR (mixed precision)
  Hierarchy H;
  Filter F;
  amgf_info info{};
  // device
  std::vector<void*> allocs;
  std::vector<DLevel> L;
  double* coarse_inv = nullptr;
  float* coarse_inv_f = nullptr;
  int64_t nL = 0;
  // mixed precision: fine-level K in 3x3 blocks (FP32 or BF16 planes) + contact term in FP64
  bool mixed = false;
  bool k_bf16 = false;
  int64_t k_nbrows = 0, k_nslices = 0, k_nblocks = 0;
  int64_t* k_soff = nullptr;
  int32_t* k_bci = nullptr;
  void* k_v = nullptr;
  int32_t *c_rp = nullptr, *c_ci = nullptr;
  double* c_v = nullptr;
  // learned smoother: per-level features (6 FP32 per row) and l1 sums, weights, training scratch
  std::vector<float*> feat_d;
  std::vector<double*> l1_d;
  std::vector<float> mlp_w_host;  // active weights (empty: theta = 1)
  float* mlp_w = nullptr;
  float *mlp_m = nullptr, *mlp_v = nullptr, *mlp_g = nullptr, *mlp_part = nullptr, *mlp_loss = nullptr;
  double *mlp_tw = nullptr, *mlp_ee = nullptr, *mlp_rr = nullptr;
  int64_t mlp_part_blocks = 0;
  int mlp_loss_cap = 0;
  double *fG = nullptr, *fGT = nullptr, *fDinv = nullptr, *fy = nullptr, *fz = nullptr, *fw = nullptr, *fv = nullptr;
  double* fM = nullptr;          // cyclic reduction matrices
  FilterTask* ftasks = nullptr;  // cyclic reduction task lists of all phases
  int64_t* fgidx = nullptr;
  int64_t* ficidx = nullptr;  // factor position -> index into I_c
  int64_t* ftouch = nullptr;
  DCSR fSc;
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *y1 = nullptr, *r1 = nullptr;
  double* partial = nullptr;
  unsigned* counter = nullptr;
  double* scratch_scalar = nullptr;
  int* kerr = nullptr;  // set by a staged sweep whose wait gave up (checked after solves)
  PcgState* st = nullptr;
  PcgState* st_host = nullptr;  // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphConditionalHandle cond{};
  int64_t n = 0, m = 0;
  bool host_only = false;
  int filter_cs = 8;          // CTAs per cluster of the filter sweeps
  bool filter_staged = false; // sweeps stage the next block's rows in shared memory
  size_t filter_smem = 0;
  int64_t launches = 0;       // kernels enqueued since the counter was last read
  int64_t init_launches = 0, body_launches = 0;
  // per-launch records (amgf_profile_iteration): an event after every launch
  struct ProfRec {
    std::string op;
    int level;
    double bytes, flops;
    cudaEvent_t ev;
  };
  std::vector<ProfRec>* prof = nullptr;

  ~Ctx() { release(); }
  void release_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    gexec = nullptr;
    graph = nullptr;
  }
  void release_device() {
    release_graph();
    for (void* a : allocs) cudaFree(a);
    allocs.clear();
    L.clear();
    feat_d.clear();
    l1_d.clear();
    mlp_w = mlp_m = mlp_v = mlp_g = mlp_part = mlp_loss = nullptr;
    mlp_tw = mlp_ee = mlp_rr = nullptr;
    kerr = nullptr;
    mlp_part_blocks = 0;
    mlp_loss_cap = 0;
  }
  void release() {
    release_device();
    if (st_host) cudaFreeHost(st_host);
    st_host = nullptr;
    if (s) cudaStreamDestroy(s);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    s = nullptr; ev_in = ev_out = t0 = t1 = nullptr;
  }
  template <class T>
  int alloc(T** ptr, int64_t count) {
    *ptr = nullptr;
    if (count <= 0) count = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, (size_t)count * sizeof(T));
    if (e != cudaSuccess) return fail(AMGF_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs.push_back(p);
    *ptr = (T*)p;
    return AMGF_OK;
  }
  template <class T>
  int upload(T** ptr, const T* host, int64_t count) {
    int st_ = alloc(ptr, count);
    if (st_) return st_;
    if (count > 0) CK(cudaMemcpy(*ptr, host, (size_t)count * sizeof(T), cudaMemcpyHostToDevice));
    return AMGF_OK;
  }
  // count entries followed by `pad` zeros (the aligned segments of the staged sweeps may reach
  // up to 15 entries past the end of an array)
  template <class T>
  int alloc_padded(T** ptr, int64_t count, int64_t pad) {
    int st_ = alloc(ptr, count + pad);
    if (st_) return st_;
    CK(cudaMemset(*ptr, 0, (size_t)(count + pad) * sizeof(T)));
    return AMGF_OK;
  }
  template <class T>
  int upload_padded(T** ptr, const T* host, int64_t count, int64_t pad) {
    int st_ = alloc_padded(ptr, count, pad);
    if (st_) return st_;
    if (count > 0) CK(cudaMemcpy(*ptr, host, (size_t)count * sizeof(T), cudaMemcpyHostToDevice));
    return AMGF_OK;
  }
};

// ---------------------------------------------------------------------------------------
// launch helpers

// Counts one launch and, while profiling, records an event after it with the launch's
// algorithmic bytes (values + indices at the stored precision, one read of every input vector,
// one write of every output) and flops.
static void counted(Ctx& c, const char* op, int level, double bytes, double flops = 0.0) {
  c.launches++;
  if (!c.prof) return;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, c.s);
  c.prof->push_back({std::string(op), level, bytes, flops, e});
}

static const char* mode_name(int mode) {
  switch (mode) {
    case M_SPMV: return "A x";
    case M_SPMV_ADD: return "y += A x";
    case M_RESID: return "b - A x";
    case M_RESID_W: return "b - A x, W (b - A x)";
    case M_POST: return "x + W (b - A x)";
    default: return "A x, W A x";
  }
}

static const char* op_label(char role, int mode) {
  switch (role) {
    case 'P': return "prolongation x += P e";
    case 'R': return mode == M_SPMV_W ? "restriction R r, W R r" : "restriction R r";
    case 'S': return "r2 = r1 - A P w (rows touching I_c)";
    default: return mode_name(mode);
  }
}

// vector bytes per output row of a row-kernel epilogue (e: element size of the vectors)
template <typename A>
static double epilogue_bytes(int mode, const A& a, double e) {
  double b = 0.0;
  if (mode == M_SPMV) b = e;
  else if (mode == M_SPMV_ADD) b = 2 * e;
  else if (mode == M_RESID) b = 2 * e;
  else if (mode == M_RESID_W) b = 3 * e + (a.y2 ? e : 0.0);
  else if (mode == M_POST) b = 3 * e + (a.add ? 8.0 : 0.0);
  else b = 2 * e + (a.y2 ? e : 0.0);
  if (a.yf) b += 4.0;
  if (a.y2f) b += 4.0;
  return b;
}

// Lanes per row.  On a large level FP64 issue bounds the pass (~2 FMA/clk/SM on this part):
// (ceil(len/K) + log2 K) K / 32 FP64 warp instructions per row is smallest for small K, and
// K = 4 still reads whole 32-byte sectors of values.  A small level cannot fill the GPU with
// 4 lanes per row and is bound by each row's chain of dependent loads instead, so its
// groups widen until rows * K covers the resident threads (2048 per SM).
static int lanes_for(int64_t rows, double avg_nnz, int num_sms) {
  int k = avg_nnz >= 6 ? 4 : 2;
  if (avg_nnz >= 24) {
    // level operators (FP64): group width by row count, from a sweep over the levels of
    // 0.8-12 M-DOF hierarchies (narrow groups where the FP64 pipe binds, wide ones where
    // too few rows are left to fill the GPU)
    const int64_t sms = num_sms;
    k = rows >= 1300 * sms ? 4 : (rows >= 80 * sms ? 8 : (rows >= 26 * sms ? 16 : 32));
    while (k > 2 && k > avg_nnz) k /= 2;
    return k;
  }
  const double resident = 2048.0 * num_sms;
  while (k < 32 && (double)rows * k < resident && k < avg_nnz) k *= 2;
  return k;
}

// FP32 rows: memory-bound, so the group width follows the row length rather than the FP64
// instruction count (measured on coarse levels of 0.2-6 M rows with 100-230 nonzeros per
// row: 16 lanes 5.0-5.5 TB/s, 4 lanes 4.3-4.7 TB/s); small levels keep the latency rule.
static int lanes_for_f32(int64_t rows, double avg_nnz, int num_sms) {
  const int k = lanes_for(rows, avg_nnz, num_sms);
  const int want = avg_nnz >= 48 ? 16 : (avg_nnz >= 12 ? 8 : k);
  return want > k ? want : k;
}

static int grid_for(const Ctx& c, int64_t rows, int K) {
  const int64_t need = (rows * K + TPB - 1) / TPB;
  const int64_t cap = (int64_t)c.num_sms * 8;  // 8 resident blocks of 256 threads per SM
  int64_t g = need < cap ? need : cap;
  if (g > MAX_DOT_BLOCKS) g = MAX_DOT_BLOCKS;
  return (int)(g < 1 ? 1 : g);
}

template <int MODE, bool DOT>
static void launch_csr_k(int K, int grid, cudaStream_t s, const CsrArgs& a) {
  switch (K) {
    case 32: csr_kernel<double, 32, MODE, DOT><<<grid, TPB, 0, s>>>(a); break;
    case 16: csr_kernel<double, 16, MODE, DOT><<<grid, TPB, 0, s>>>(a); break;
    case 8: csr_kernel<double, 8, MODE, DOT><<<grid, TPB, 0, s>>>(a); break;
    case 4: csr_kernel<double, 4, MODE, DOT><<<grid, TPB, 0, s>>>(a); break;
    default: csr_kernel<double, 2, MODE, DOT><<<grid, TPB, 0, s>>>(a); break;
  }
}

template <int MODE>
static void launch_csr(Ctx& c, const DCSR& A, CsrArgs a, const double* dotv = nullptr, double* result = nullptr) {
  a.rp = A.rp; a.ci = A.ci; a.v = A.v; a.nrows = A.nrows;
  if (A.nrows == 0) return;
  if (A.bsr && !a.rows) {
    BsrArgs b{};
    b.soff = A.soff; b.bci = A.bci; b.v = A.bv; b.nbrows = A.nbrows; b.nslices = A.nslices;
    b.x = a.x; b.b = a.b; b.winv = a.winv; b.w2 = a.w2; b.add = a.add; b.y = a.y; b.y2 = a.y2;
    b.yf = a.yf; b.y2f = a.y2f;
    const int grid = grid_for(c, A.nslices, 32);  // one warp per slice
    if (result) {
      b.dotv = dotv; b.partial = c.partial; b.result = result; b.counter = c.counter;
      bsr3_kernel<MODE, true><<<grid, TPB, 0, c.s>>>(b);
    } else {
      bsr3_kernel<MODE, false><<<grid, TPB, 0, c.s>>>(b);
    }
    // 9 FP64 values + one block column per stored block, slice offsets, x gathered once, epilogue
    counted(c, MODE == M_SPMV && result ? "A p, p^T A p" : op_label(A.role, MODE), A.level,
            (double)A.nblocks * 76.0 + (double)(A.nslices + 1) * 8.0 + 8.0 * A.ncols +
                A.nrows * (epilogue_bytes(MODE, a, 8.0) + (result ? 8.0 : 0.0)),
            2.0 * A.nnz);
    return;
  }
  if constexpr (MODE == M_SPMV || MODE == M_SPMV_ADD || MODE == M_SPMV_W || MODE == M_RESID || MODE == M_POST) {
    if (A.ell_v && !a.rows && !result && (MODE == M_SPMV_W || !a.y2) && !a.yf && !a.y2f) {
      SellArgs e{};
      e.soff = A.ell_soff; e.perm = A.ell_perm; e.ci = A.ell_ci; e.v = A.ell_v;
      e.nrows = A.nrows; e.nslices = A.sell_h.nslices;
      e.x = a.x; e.b = a.b; e.winv = a.winv; e.w2 = a.w2; e.add = a.add; e.y = a.y; e.y2 = a.y2;
      const int grid = grid_for(c, e.nslices, 32);  // one warp per slice
      sell_kernel<double, double, MODE><<<grid, TPB, 0, c.s>>>(e);
      // stored slots (values + columns, padding excluded), slice offsets, permutation, x once, epilogue
      counted(c, op_label(A.role, MODE), A.level,
              (double)A.nnz * 12.0 + (double)(e.nslices + 1) * 8.0 + 4.0 * A.nrows + 8.0 * A.ncols +
                  A.nrows * epilogue_bytes(MODE, a, 8.0),
              2.0 * A.nnz);
      return;
    }
  }
  const int grid = grid_for(c, A.nrows, A.K);
  if (result) {
    a.dotv = dotv; a.partial = c.partial; a.result = result; a.counter = c.counter;
    launch_csr_k<MODE, true>(A.K, grid, c.s, a);
  } else {
    launch_csr_k<MODE, false>(A.K, grid, c.s, a);
  }
  counted(c, op_label(A.role, MODE), A.level,
          (double)A.nnz * 12.0 + (double)(A.nrows + 1) * 8.0 + 8.0 * A.ncols +
              A.nrows * (epilogue_bytes(MODE, a, 8.0) + (a.rows ? 8.0 : 0.0) + (result ? 8.0 : 0.0)),
          2.0 * A.nnz);
}

// entries per lane and batch of the staged sweeps
constexpr int STAGE_U = 8;

template <int MODE, typename VT>
static const void* staged_fn(int K) {
  switch (K) {
    case 32: return (const void*)csr_staged_kernel<MODE, VT, 32, STAGE_U>;
    case 16: return (const void*)csr_staged_kernel<MODE, VT, 16, STAGE_U>;
    default: return (const void*)csr_staged_kernel<MODE, VT, 8, STAGE_U>;
  }
}

template <int MODE, typename VT>
static void launch_staged(Ctx& c, const DCSRf& A, const CsrArgsT<float, VT>& a) {
  switch (A.K) {
    case 32: csr_staged_kernel<MODE, VT, 32, STAGE_U><<<A.sgrid, STAGE_TPB, A.ssmem, c.s>>>(a, A.sg); break;
    case 16: csr_staged_kernel<MODE, VT, 16, STAGE_U><<<A.sgrid, STAGE_TPB, A.ssmem, c.s>>>(a, A.sg); break;
    default: csr_staged_kernel<MODE, VT, 8, STAGE_U><<<A.sgrid, STAGE_TPB, A.ssmem, c.s>>>(a, A.sg); break;
  }
}

template <int MODE>
static void launch_csr_f(Ctx& c, const DCSRf& A, CsrArgsT<float> a) {
  a.rp = A.rp; a.ci = A.ci; a.v = A.v; a.nrows = A.nrows;
  if (A.nrows == 0) return;
  const int grid = grid_for(c, A.nrows, A.K);
  const double vb = A.vb ? 2.0 : 4.0;
  const double bytes = (double)A.nnz * (vb + 4.0) + (double)(A.nrows + 1) * 8.0 + 4.0 * A.ncols +
                       A.nrows * epilogue_bytes(MODE, a, 4.0);
  if constexpr (MODE == M_SPMV || MODE == M_SPMV_ADD || MODE == M_SPMV_W) {
    if ((A.ell_v || A.ell_vb) && !a.rows && (MODE == M_SPMV_W || !a.y2) && !a.yf && !a.y2f) {
      const int g = grid_for(c, A.ell_nslices, 32);  // one warp per slice
      auto go = [&](auto* vals) {
        using V = std::remove_const_t<std::remove_pointer_t<decltype(vals)>>;
        SellArgsT<float, V> e{};
        e.soff = A.ell_soff; e.perm = A.ell_perm; e.ci = A.ell_ci; e.v = vals;
        e.nrows = A.nrows; e.nslices = A.ell_nslices;
        e.x = a.x; e.b = a.b; e.winv = a.winv; e.w2 = a.w2; e.add = a.add; e.y = a.y; e.y2 = a.y2;
        sell_kernel<float, V, MODE><<<g, TPB, 0, c.s>>>(e);
      };
      if (A.ell_vb) go(A.ell_vb); else go(A.ell_v);
      counted(c, op_label(A.role, MODE), A.level,
              (double)A.nnz * (vb + 4.0) + (double)(A.ell_nslices + 1) * 8.0 + 4.0 * A.nrows + 4.0 * A.ncols +
                  A.nrows * epilogue_bytes(MODE, a, 4.0),
              2.0 * A.nnz);
      return;
    }
  }
  // level operator sweeps with plain epilogues: staged tiles (csr_staged_kernel)
  constexpr bool kStagedMode = MODE == M_RESID || MODE == M_POST;
  const bool staged = kStagedMode && A.sg.ntiles > 0 && !a.rows && !a.add && !a.y2 && !a.yf && !a.y2f;
  if (A.vb) {
    CsrArgsT<float, __nv_bfloat16> b{};
    b.rp = a.rp; b.ci = a.ci; b.v = A.vb; b.nrows = a.nrows; b.rows = a.rows;
    b.x = a.x; b.b = a.b; b.winv = a.winv; b.w2 = a.w2; b.add = a.add; b.y = a.y; b.y2 = a.y2;
    b.yf = a.yf; b.y2f = a.y2f;
    if constexpr (kStagedMode) {
      if (staged) {
        launch_staged<MODE, __nv_bfloat16>(c, A, b);
        counted(c, op_label(A.role, MODE), A.level, bytes, 2.0 * A.nnz);
        return;
      }
    }
    if (A.U == 8) {
      csr_kernel<float, 32, MODE, false, __nv_bfloat16, 8><<<grid, TPB, 0, c.s>>>(b);
    } else {
      switch (A.K) {
        case 32: csr_kernel<float, 32, MODE, false, __nv_bfloat16><<<grid, TPB, 0, c.s>>>(b); break;
        case 16: csr_kernel<float, 16, MODE, false, __nv_bfloat16><<<grid, TPB, 0, c.s>>>(b); break;
        case 8: csr_kernel<float, 8, MODE, false, __nv_bfloat16><<<grid, TPB, 0, c.s>>>(b); break;
        case 4: csr_kernel<float, 4, MODE, false, __nv_bfloat16><<<grid, TPB, 0, c.s>>>(b); break;
        default: csr_kernel<float, 2, MODE, false, __nv_bfloat16><<<grid, TPB, 0, c.s>>>(b); break;
      }
    }
    counted(c, op_label(A.role, MODE), A.level, bytes, 2.0 * A.nnz);
    return;
  }
  if (A.U == 8) {
    csr_kernel<float, 32, MODE, false, float, 8><<<grid, TPB, 0, c.s>>>(a);
  } else {
    switch (A.K) {
      case 32: csr_kernel<float, 32, MODE, false><<<grid, TPB, 0, c.s>>>(a); break;
      case 16: csr_kernel<float, 16, MODE, false><<<grid, TPB, 0, c.s>>>(a); break;
      case 8: csr_kernel<float, 8, MODE, false><<<grid, TPB, 0, c.s>>>(a); break;
      case 4: csr_kernel<float, 4, MODE, false><<<grid, TPB, 0, c.s>>>(a); break;
      default: csr_kernel<float, 2, MODE, false><<<grid, TPB, 0, c.s>>>(a); break;
    }
  }
  counted(c, op_label(A.role, MODE), A.level, bytes, 2.0 * A.nnz);
}

// fine level of the FP32 V-cycle (K blocks + FP64 contact term)
template <int MODE>
static void launch_fine_mixed(Ctx& c, const float* x, const float* b, const float* winv, const double* add,
                              float* y32, double* y64, const double* dotv, double* result) {
  const int grid = grid_for(c, c.k_nslices, 32);  // one warp per slice
  auto fill = [&](auto& a) {
    a.soff = c.k_soff; a.bci = c.k_bci; a.nbrows = c.k_nbrows; a.nslices = c.k_nslices;
    a.crp = c.c_rp; a.cci = c.c_ci; a.cv = c.c_v;
    a.x = x; a.b = b; a.winv = winv; a.add = add; a.y32 = y32; a.y64 = y64;
    a.dotv = dotv; a.partial = c.partial; a.result = result; a.counter = c.counter;
  };
  if (c.k_bf16) {
    Bsr3MixedArgs<__nv_bfloat16> a{};
    fill(a);
    a.pk = (const uint2*)c.k_v;
    if (result) bsr3_mixed_kernel<__nv_bfloat16, MODE, true><<<grid, TPB, 0, c.s>>>(a);
    else bsr3_mixed_kernel<__nv_bfloat16, MODE, false><<<grid, TPB, 0, c.s>>>(a);
  } else {
    Bsr3MixedArgs<float> a{};
    fill(a);
    a.v = (const float*)c.k_v;
    if (result) bsr3_mixed_kernel<float, MODE, true><<<grid, TPB, 0, c.s>>>(a);
    else bsr3_mixed_kernel<float, MODE, false><<<grid, TPB, 0, c.s>>>(a);
  }
  // K blocks (9 values + column), slice offsets, contact term (row pointers, 4 + 8 B per entry),
  // x gathered once, epilogue vectors
  const double vb = c.k_bf16 ? 2.0 : 4.0, n = (double)c.n;
  const double epi = MODE == M_RESID ? 8.0 : 16.0 + (add ? 8.0 : 0.0) + (result ? 8.0 : 0.0);
  counted(c, MODE == M_RESID ? "fine K blocks + FP64 contact: b - A x" : "fine K blocks + FP64 contact: x + W (b - A x)",
          0, (double)c.k_nblocks * (9.0 * vb + 4.0) + (double)(c.k_nslices + 1) * 8.0 + (n + 1) * 4.0 +
                 (double)c.c_nnz * 12.0 + 4.0 * n + n * epi,
          2.0 * (double)c.L[0].A.nnz);
}

// coarsest-level solve: one warp per row of the dense inverse
static int dense_grid(const Ctx& c) {
  const int64_t g = (c.nL + DENSE_ROWS_TPB / 32 - 1) / (DENSE_ROWS_TPB / 32);
  const int64_t cap = (int64_t)c.num_sms * 8;
  return (int)(g < 1 ? 1 : (g < cap ? g : cap));
}

static int vec_grid(const Ctx& c, int64_t n) {
  int64_t g = (n + TPB - 1) / TPB;
  const int64_t cap = (int64_t)c.num_sms * 8;
  return (int)(g < 1 ? 1 : (g < cap ? g : cap));
}

// ---------------------------------------------------------------------------------------
// V-cycle: out0 = B rhs0 (+ add0); optional dot(dotv, out0) -> *dotres.
// On entry L[0].x must hold W_0 rhs0 (the pre-smoothed iterate from a zero start); the
// kernels that produce a V-cycle's right-hand side write it as a second output.
static void enqueue_vcycle(Ctx& c, const double* rhs0, double* out0, const double* add0, const double* dotv,
                           double* dotres) {
  const int nlev = (int)c.L.size();
  const int nu = c.o.nu < 1 ? 1 : c.o.nu;
  const bool cheb = c.o.smoother == 1;
  const ChebCoefs cf = cheb_coefs(c.o.cheby_lower, nu);
  auto rhs_of = [&](int l) -> const double* { return l == 0 ? rhs0 : c.L[l].rhs; };
  for (int l = 0; l + 1 < nlev; ++l) {
    DLevel& lv = c.L[l];
    // pre-smoothing from zero: x = W r (already in lv.x); residual r - A x
    if (cheb) {
      cheb_init_kernel<double><<<vec_grid(c, lv.n), TPB, 0, c.s>>>(lv.n, lv.x, lv.d, cf.inv_c);
      counted(c, "Chebyshev first step", l, 24.0 * lv.n);
    }
    CsrArgs a{};
    a.x = lv.x; a.b = rhs_of(l); a.y = lv.res;
    launch_csr<M_RESID>(c, lv.A, a);
    for (int s = 1; s < nu; ++s) {
      if (cheb)
        cheb_step_kernel<double, false><<<vec_grid(c, lv.n), TPB, 0, c.s>>>(lv.n, lv.winv, lv.res, lv.d, lv.x,
                                                                           cf.a[s], cf.bc[s]);
      else
        axpy_w_kernel<<<vec_grid(c, lv.n), TPB, 0, c.s>>>(lv.n, lv.winv, lv.res, lv.x);
      counted(c, cheb ? "Chebyshev step" : "x += W r", l, (cheb ? 48.0 : 32.0) * lv.n);
      CsrArgs rr{};
      rr.x = lv.x; rr.b = rhs_of(l); rr.y = lv.res;
      launch_csr<M_RESID>(c, lv.A, rr);
    }
    // restriction; also W_{l+1} r_{l+1} for the next level's pre-smoothing
    CsrArgs rs{};
    rs.x = lv.res; rs.y = c.L[l + 1].rhs;
    if (l + 2 < nlev) {
      rs.w2 = c.L[l + 1].winv; rs.y2 = c.L[l + 1].x;
      launch_csr<M_SPMV_W>(c, lv.R, rs);
    } else {
      launch_csr<M_SPMV>(c, lv.R, rs);
    }
  }
  // coarsest level: exact solve with the dense inverse
  {
    const int lc = nlev - 1;
    const double* rc = rhs_of(lc);
    double* oc = lc == 0 ? out0 : c.L[lc].out;
    if (lc == 0)
      dense_gemv_kernel<<<1, DENSE_TPB, 0, c.s>>>(c.nL, c.coarse_inv, rc, add0, oc, dotv, dotres);
    else
      dense_rows_kernel<double><<<dense_grid(c), DENSE_ROWS_TPB, 0, c.s>>>(c.nL, c.coarse_inv, rc, oc);
    counted(c, "coarsest: dense inverse x rhs", lc, 8.0 * (double)c.nL * (double)c.nL + 16.0 * c.nL,
            2.0 * (double)c.nL * (double)c.nL);
  }
  for (int l = nlev - 2; l >= 0; --l) {
    DLevel& lv = c.L[l];
    CsrArgs pa{};
    pa.x = c.L[l + 1].out; pa.y = lv.x;
    launch_csr<M_SPMV_ADD>(c, lv.P, pa);
    if (cheb) {
      double* out = l == 0 ? out0 : lv.out;
      const double* add = l == 0 ? add0 : nullptr;
      const bool dot = l == 0 && dotres;
      const int g = vec_grid(c, lv.n);
      for (int j = 0; j < nu; ++j) {
        CsrArgs rr{};
        rr.x = lv.x; rr.b = rhs_of(l); rr.y = lv.res;
        launch_csr<M_RESID>(c, lv.A, rr);
        const double aj = j ? cf.a[j] : 0.0, bj = j ? cf.bc[j] : cf.inv_c;
        if (j + 1 < nu) {
          if (j == 0) cheb_step_kernel<double, true><<<g, TPB, 0, c.s>>>(lv.n, lv.winv, lv.res, lv.d, lv.x, aj, bj);
          else cheb_step_kernel<double, false><<<g, TPB, 0, c.s>>>(lv.n, lv.winv, lv.res, lv.d, lv.x, aj, bj);
        } else {
          auto go = [&](auto first, auto withdot) {
            cheb_out_kernel<double, double, decltype(first)::value, decltype(withdot)::value><<<g, TPB, 0, c.s>>>(
                lv.n, lv.winv, lv.res, lv.d, lv.x, aj, bj, add, out, dotv, c.partial, dotres, c.counter);
          };
          if (j == 0) {
            if (dot) go(std::true_type{}, std::true_type{}); else go(std::true_type{}, std::false_type{});
          } else {
            if (dot) go(std::false_type{}, std::true_type{}); else go(std::false_type{}, std::false_type{});
          }
        }
        counted(c, "Chebyshev step", l, 48.0 * lv.n);
      }
      continue;
    }
    for (int s = 1; s < nu; ++s) {
      CsrArgs rr{};
      rr.x = lv.x; rr.b = rhs_of(l); rr.y = lv.res;
      launch_csr<M_RESID>(c, lv.A, rr);
      axpy_w_kernel<<<vec_grid(c, lv.n), TPB, 0, c.s>>>(lv.n, lv.winv, lv.res, lv.x);
      counted(c, "x += W r", l, 32.0 * lv.n);
    }
    CsrArgs po{};
    po.x = lv.x; po.b = rhs_of(l); po.winv = lv.winv;
    po.add = l == 0 ? add0 : nullptr;
    po.y = l == 0 ? out0 : lv.out;
    if (l == 0 && dotres) launch_csr<M_POST>(c, lv.A, po, dotv, dotres);
    else launch_csr<M_POST>(c, lv.A, po);
  }
}

// FP32 V-cycle: out0 (FP64) = B rhs (+ add0), optional dot(dotv, out0) -> *dotres.  On entry
// L[0].rhsf holds the right-hand side in FP32 and L[0].xf = W_0 rhs in FP32 (written by the
// FP64 kernel that produced the right-hand side: the precision boundary going in); the
// fine-level post-smoother writes the FP64 output (the boundary going out).
static void enqueue_vcycle_f32(Ctx& c, double* out0, const double* add0, const double* dotv, double* dotres) {
  const int nlev = (int)c.L.size();
  const int nu = c.o.nu < 1 ? 1 : c.o.nu;
  const bool cheb = c.o.smoother == 1;
  const ChebCoefs cf = cheb_coefs(c.o.cheby_lower, nu);
  for (int l = 0; l + 1 < nlev; ++l) {
    DLevel& lv = c.L[l];
    if (cheb) {
      cheb_init_kernel<float><<<vec_grid(c, lv.n), TPB, 0, c.s>>>(lv.n, lv.xf, lv.df, (float)cf.inv_c);
      counted(c, "Chebyshev first step", l, 12.0 * lv.n);
    }
    for (int s = 0; s < nu; ++s) {
      if (s > 0) {
        if (cheb)
          cheb_step_kernel<float, false><<<vec_grid(c, lv.n), TPB, 0, c.s>>>(lv.n, lv.winvf, lv.resf, lv.df, lv.xf,
                                                                            (float)cf.a[s], (float)cf.bc[s]);
        else
          axpy_w_f32_kernel<<<vec_grid(c, lv.n), TPB, 0, c.s>>>(lv.n, lv.winvf, lv.resf, lv.xf);
        counted(c, cheb ? "Chebyshev step" : "x += W r", l, (cheb ? 24.0 : 16.0) * lv.n);
      }
      if (l == 0) {
        launch_fine_mixed<M_RESID>(c, lv.xf, lv.rhsf, nullptr, nullptr, lv.resf, nullptr, nullptr, nullptr);
      } else {
        CsrArgsT<float> a{};
        a.x = lv.xf; a.b = lv.rhsf; a.y = lv.resf;
        launch_csr_f<M_RESID>(c, lv.Af, a);
      }
    }
    CsrArgsT<float> rs{};
    rs.x = lv.resf; rs.y = c.L[l + 1].rhsf;
    if (l + 2 < nlev) {
      rs.w2 = c.L[l + 1].winvf; rs.y2 = c.L[l + 1].xf;
      launch_csr_f<M_SPMV_W>(c, lv.Rf, rs);
    } else {
      launch_csr_f<M_SPMV>(c, lv.Rf, rs);
    }
  }
  dense_rows_kernel<float><<<dense_grid(c), DENSE_ROWS_TPB, 0, c.s>>>(c.nL, c.coarse_inv_f, c.L[nlev - 1].rhsf,
                                                                       c.L[nlev - 1].outf);
  counted(c, "coarsest: dense inverse x rhs", nlev - 1, 4.0 * (double)c.nL * (double)c.nL + 8.0 * c.nL,
          2.0 * (double)c.nL * (double)c.nL);
  for (int l = nlev - 2; l >= 0; --l) {
    DLevel& lv = c.L[l];
    CsrArgsT<float> pa{};
    pa.x = c.L[l + 1].outf; pa.y = lv.xf;
    launch_csr_f<M_SPMV_ADD>(c, lv.Pf, pa);
    if (cheb) {
      const bool dot = l == 0 && dotres;
      const int g = vec_grid(c, lv.n);
      for (int j = 0; j < nu; ++j) {
        if (l == 0) {
          launch_fine_mixed<M_RESID>(c, lv.xf, lv.rhsf, nullptr, nullptr, lv.resf, nullptr, nullptr, nullptr);
        } else {
          CsrArgsT<float> rr{};
          rr.x = lv.xf; rr.b = lv.rhsf; rr.y = lv.resf;
          launch_csr_f<M_RESID>(c, lv.Af, rr);
        }
        const float aj = j ? (float)cf.a[j] : 0.f, bj = j ? (float)cf.bc[j] : (float)cf.inv_c;
        if (j + 1 < nu) {
          if (j == 0) cheb_step_kernel<float, true><<<g, TPB, 0, c.s>>>(lv.n, lv.winvf, lv.resf, lv.df, lv.xf, aj, bj);
          else cheb_step_kernel<float, false><<<g, TPB, 0, c.s>>>(lv.n, lv.winvf, lv.resf, lv.df, lv.xf, aj, bj);
        } else if (l == 0) {
          // the fine level's output crosses into the FP64 PCG (+ add0, dot)
          auto go = [&](auto first, auto withdot) {
            cheb_out_kernel<float, double, decltype(first)::value, decltype(withdot)::value><<<g, TPB, 0, c.s>>>(
                lv.n, lv.winvf, lv.resf, lv.df, lv.xf, aj, bj, add0, out0, dotv, c.partial, dotres, c.counter);
          };
          if (j == 0) {
            if (dot) go(std::true_type{}, std::true_type{}); else go(std::true_type{}, std::false_type{});
          } else {
            if (dot) go(std::false_type{}, std::true_type{}); else go(std::false_type{}, std::false_type{});
          }
        } else {
          if (j == 0)
            cheb_out_kernel<float, float, true, false><<<g, TPB, 0, c.s>>>(lv.n, lv.winvf, lv.resf, lv.df, lv.xf, aj, bj,
                                                                          nullptr, lv.outf, nullptr, nullptr, nullptr,
                                                                          nullptr);
          else
            cheb_out_kernel<float, float, false, false><<<g, TPB, 0, c.s>>>(lv.n, lv.winvf, lv.resf, lv.df, lv.xf, aj,
                                                                           bj, nullptr, lv.outf, nullptr, nullptr,
                                                                           nullptr, nullptr);
        }
        counted(c, "Chebyshev step", l, 24.0 * lv.n);
      }
      continue;
    }
    for (int s = 1; s < nu; ++s) {
      if (l == 0) {
        launch_fine_mixed<M_RESID>(c, lv.xf, lv.rhsf, nullptr, nullptr, lv.resf, nullptr, nullptr, nullptr);
      } else {
        CsrArgsT<float> rr{};
        rr.x = lv.xf; rr.b = lv.rhsf; rr.y = lv.resf;
        launch_csr_f<M_RESID>(c, lv.Af, rr);
      }
      axpy_w_f32_kernel<<<vec_grid(c, lv.n), TPB, 0, c.s>>>(lv.n, lv.winvf, lv.resf, lv.xf);
      counted(c, "x += W r", l, 16.0 * lv.n);
    }
    if (l == 0) {
      launch_fine_mixed<M_POST>(c, lv.xf, lv.rhsf, lv.winvf, add0, nullptr, out0, dotv, dotres);
    } else {
      CsrArgsT<float> po{};
      po.x = lv.xf; po.b = lv.rhsf; po.winv = lv.winvf; po.y = lv.outf;
      launch_csr_f<M_POST>(c, lv.Af, po);
    }
  }
}

static void enqueue_scale_w0(Ctx& c, const double* r) {
  if (c.mixed) {
    to_f32_scaled_kernel<<<vec_grid(c, c.n), TPB, 0, c.s>>>(c.n, c.L[0].winv, r, c.L[0].rhsf, c.L[0].xf);
  } else {
    scale_kernel<<<vec_grid(c, c.n), TPB, 0, c.s>>>(c.n, c.L[0].winv, r, c.L[0].x);
  }
  counted(c, c.mixed ? "W r (FP32 copies)" : "W r", 0, (c.mixed ? 24.0 : 24.0) * c.n);
}

// B rhs0 in the configured precision (see enqueue_vcycle / enqueue_vcycle_f32 for the entry state)
static void enqueue_B(Ctx& c, const double* rhs0, double* out0, const double* add0, const double* dotv,
                      double* dotres) {
  if (c.mixed) enqueue_vcycle_f32(c, out0, add0, dotv, dotres);
  else enqueue_vcycle(c, rhs0, out0, add0, dotv, dotres);
}

// one block sweep of the filter factor as a thread-block cluster launch
static void launch_sweep(Ctx& c, bool fwd, const double* M, const double* r, const double* vdirect, const double* zin,
                         double* out) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c.filter_cs, 1, 1);
  cfg.blockDim = dim3(FILTER_TPB, 1, 1);
  cfg.dynamicSmemBytes = c.filter_smem;
  cfg.stream = c.s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = c.filter_cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int64_t nb = c.F.nb, nblk = c.F.nblk, nc = c.F.nc;
  if (c.filter_staged)
    cudaLaunchKernelEx(&cfg, filter_sweep_kernel<true>, fwd, M, (const int64_t*)c.fgidx, r, vdirect, zin, nc, nb, nblk, out);
  else
    cudaLaunchKernelEx(&cfg, filter_sweep_kernel<false>, fwd, M, (const int64_t*)c.fgidx, r, vdirect, zin, nc, nb, nblk, out);
  counted(c, fwd ? "filter: block LDL^T forward sweep" : "filter: block LDL^T backward sweep", -1,
          8.0 * (double)(nblk - 1) * nb * nb + 16.0 * nb * nblk, 2.0 * (double)(nblk - 1) * nb * nb);
}

// out (factor order, length nblk*nb) = A_w^{-1} v with v gathered from r at gidx (or given
// directly in factor order by vdirect); y and z are work vectors of the same length
static void enqueue_filter_solve_into(Ctx& c, const double* r, const double* vdirect, double* y, double* z, double* out) {
  const int64_t nb = c.F.nb, nblk = c.F.nblk;
  if (c.F.algo == 0) {  // block cyclic reduction: y holds the reduced right-hand sides
    const size_t smem = 2 * (size_t)nb * sizeof(double);
    const int nphase = (int)c.F.phase_off.size() - 1;
    for (int q = 0; q < nphase; ++q) {
      const int64_t t0 = c.F.phase_off[q], nt = c.F.phase_off[q + 1] - t0;
      // few output blocks: a warp per row and 8 rows per CTA, so that enough SMs pull the matrices
      const bool wide = nt * ((nb + 31) / 32) < 2 * (int64_t)c.num_sms;
      const int rows = wide ? FBCR_TPB / 32 : FBCR_TPB / 8;
      const int tiles = (int)((nb + rows - 1) / rows);
      const unsigned grid = (unsigned)(nt * tiles);
      auto go = [&](auto kern) {
        kern<<<grid, FBCR_TPB, smem, c.s>>>(c.ftasks + t0, tiles, c.fM, nb, r, c.fgidx, vdirect, c.F.nc, y, out);
      };
      if (q == 0) {
        if (wide) go(filter_bcr_kernel<true, 32>); else go(filter_bcr_kernel<true, 8>);
      } else {
        if (wide) go(filter_bcr_kernel<false, 32>); else go(filter_bcr_kernel<false, 8>);
      }
      // each task reads its one or two nb x nb matrices and input blocks and writes one block
      double mats = 0.0, blks = 0.0;
      for (int64_t k = t0; k < t0 + nt; ++k) {
        const FilterTask& ft = c.F.tasks[k];
        mats += (ft.m0 >= 0 && ft.in0 >= 0) + (ft.m1 >= 0 && ft.in1 >= 0);
        blks += 1.0 + (ft.in0 >= 0) + (ft.in1 >= 0);
      }
      counted(c, q == 0 ? "filter: cyclic reduction phase (gathers P^T r1)" : "filter: cyclic reduction phase", -1,
              8.0 * mats * nb * nb + 8.0 * blks * nb, 2.0 * mats * nb * nb);
    }
    return;
  }
  launch_sweep(c, true, c.fG, r, vdirect, nullptr, y);
  const int64_t rows = nb * nblk;
  int g = (int)((rows * 32 + TPB - 1) / TPB);
  if (g > c.num_sms * 8) g = c.num_sms * 8;
  filter_diag_kernel<<<g, TPB, 0, c.s>>>(c.fDinv, y, z, nb, nblk);
  counted(c, "filter: block pivots", -1, 8.0 * (double)nblk * nb * nb + 16.0 * nb * nblk,
          2.0 * (double)nblk * nb * nb);
  launch_sweep(c, false, c.fGT, nullptr, nullptr, z, out);
}

static void enqueue_filter_solve(Ctx& c, const double* r, const double* vdirect) {
  enqueue_filter_solve_into(c, r, vdirect, c.fy, c.fz, c.fw);
}

// Copies of the intermediate vectors of one AMGF application (amgf_apply_stages); every
// pointer may be null.  w is written in ascending-DOF order of I_c.
struct ApplyTap {
  double *y1 = nullptr, *r1 = nullptr, *w = nullptr, *r2 = nullptr;
};

static void tap_copy(Ctx& c, double* dst, const double* src, int64_t n) {
  if (dst && n > 0) cudaMemcpyAsync(dst, src, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, c.s);
}

// z = M r; optional dot(r, z) -> *dotres.  On entry L[0].x must hold W_0 r.
static void enqueue_apply(Ctx& c, const double* r, double* z, double* dotres, const ApplyTap* tap = nullptr) {
  if (!c.o.filter) {  // M = B
    enqueue_B(c, r, z, nullptr, r, dotres);
    if (tap) tap_copy(c, tap->y1, z, c.n);
    return;
  }
  // y1 = B r
  enqueue_B(c, r, c.y1, nullptr, nullptr, nullptr);
  if (tap) tap_copy(c, tap->y1, c.y1, c.n);
  // r1 = r - A y1 in FP64 (and the entry state of the second V-cycle: W_0 r1, FP32 copies if
  // mixed).  This residual stays FP64 in every precision: after a good V-cycle r1 << r, and
  // its contact rows (entries up to D_max) feed the filter solve.  With K y1 in BF16 the c160
  // solve took 89 instead of 67 iterations.
  CsrArgs ra{};
  ra.x = c.y1; ra.b = r; ra.y = c.r1; ra.w2 = c.L[0].winv;
  if (c.mixed) { ra.yf = c.L[0].rhsf; ra.y2f = c.L[0].xf; } else { ra.y2 = c.L[0].x; }
  launch_csr<M_RESID_W>(c, c.L[0].A, ra);
  if (tap) tap_copy(c, tap->r1, c.r1, c.n);
  if (c.F.nc > 0) {
    enqueue_filter_solve(c, c.r1, nullptr);
    if (tap && tap->w)
      permute_kernel<<<vec_grid(c, c.F.nc), TPB, 0, c.s>>>(c.F.nc, c.ficidx, nullptr, c.fw, tap->w);
    filter_scatter_kernel<<<vec_grid(c, c.F.nc), TPB, 0, c.s>>>(c.fgidx, c.fw, c.y1, c.F.nc);  // y2 = y1 + P w
    counted(c, "y2 = y1 + P w", 0, 32.0 * c.F.nc);
    CsrArgs sa{};                                                                              // r2 = r1 - A P w
    sa.rows = c.ftouch; sa.x = c.fw; sa.b = c.r1; sa.y = c.r1; sa.w2 = c.L[0].winv;
    if (c.mixed) { sa.yf = c.L[0].rhsf; sa.y2f = c.L[0].xf; } else { sa.y2 = c.L[0].x; }
    launch_csr<M_RESID_W>(c, c.fSc, sa);
  }
  if (tap) tap_copy(c, tap->r2, c.r1, c.n);
  // z = y2 + B r2
  enqueue_B(c, c.r1, z, c.y1, r, dotres);
}

// one PCG iteration (body of the while node)
static void enqueue_pcg_body(Ctx& c, int use_cond) {
  CsrArgs qa{};
  qa.x = c.p; qa.y = c.q;
  launch_csr<M_SPMV>(c, c.L[0].A, qa, c.p, &c.st->pq);
  pcg_update_xr_kernel<<<vec_grid(c, c.n), TPB, 0, c.s>>>(
      c.st, c.p, c.q, c.x, c.r, c.L[0].winv, c.mixed ? nullptr : c.L[0].x, c.mixed ? c.L[0].rhsf : nullptr,
      c.mixed ? c.L[0].xf : nullptr, c.mixed ? c.z : nullptr, c.partial, c.counter, c.n);
  // p, q, W read; x, r read and written; W r written (FP64, or FP32 r and W r plus z read)
  counted(c, "PCG: x += alpha p, r -= alpha q, W r", 0, (c.mixed ? 72.0 : 64.0) * c.n);
  enqueue_apply(c, c.r, c.z, &c.st->rz_new);
  pcg_update_p_kernel<<<vec_grid(c, c.n), TPB, 0, c.s>>>(c.st, c.z, c.p, c.n);
  counted(c, "PCG: p = z + beta p", 0, 24.0 * c.n);
  pcg_finalize_kernel<<<1, 1, 0, c.s>>>(c.st, c.cond, use_cond);
  counted(c, "PCG: scalars and stop test", -1, 0.0);
}

static void enqueue_pcg_init(Ctx& c) {
  CsrArgs ra{};
  ra.x = c.x; ra.b = c.b; ra.y = c.r; ra.w2 = c.L[0].winv;
  if (c.mixed) { ra.yf = c.L[0].rhsf; ra.y2f = c.L[0].xf; } else { ra.y2 = c.L[0].x; }
  launch_csr<M_RESID_W>(c, c.L[0].A, ra);               // r0 = b - A x0, W_0 r0
  enqueue_apply(c, c.r, c.z, &c.st->rz_new);             // z0 = M r0, rz_new = r0^T z0
  pcg_init_kernel<<<1, 1, 0, c.s>>>(c.st, c.o.maxit, c.o.rtol, c.mixed ? 1 : 0);
  counted(c, "PCG: initial scalars", -1, 0.0);
  copy_kernel<<<vec_grid(c, c.n), TPB, 0, c.s>>>(c.n, c.z, c.p);  // p0 = z0
  counted(c, "PCG: p = z", 0, 16.0 * c.n);
}

static int build_graph(Ctx& c) {
  c.release_graph();
  CK(cudaGraphCreate(&c.graph, 0));
  // initial part, captured into its own graph and embedded as a child node
  cudaGraph_t init_g = nullptr;
  CK(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal));
  c.launches = 0;
  enqueue_pcg_init(c);
  c.init_launches = c.launches;
  CK(cudaStreamEndCapture(c.s, &init_g));
  cudaGraphNode_t init_node;
  CK(cudaGraphAddChildGraphNode(&init_node, c.graph, nullptr, 0, init_g));
  cudaGraphDestroy(init_g);
  CK(cudaGraphConditionalHandleCreate(&c.cond, c.graph, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = c.cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t while_node;
  CK(cudaGraphAddNode(&while_node, c.graph, &init_node, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(c.s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  c.launches = 0;
  enqueue_pcg_body(c, 1);
  c.body_launches = c.launches;
  cudaGraph_t body_out = nullptr;
  CK(cudaStreamEndCapture(c.s, &body_out));
  CK(cudaGraphInstantiate(&c.gexec, c.graph, 0));
  return AMGF_OK;
}

// W_l = theta / l1 on every smoothed level from the active weights (theta = 1 without them)
static int apply_smoother_weights(Ctx& c, bool plain) {
  const bool use = !plain && !c.mlp_w_host.empty();
  if (use) CK(cudaMemcpyAsync(c.mlp_w, c.mlp_w_host.data(), MLP_NW * sizeof(float), cudaMemcpyHostToDevice, c.s));
  for (int l = 0; l + 1 < (int)c.L.size(); ++l) {
    DLevel& lv = c.L[l];
    mlp_infer_kernel<<<vec_grid(c, lv.n), TPB, 0, c.s>>>(lv.n, c.feat_d[l], c.mlp_w, use ? 0 : 1, c.l1_d[l], lv.winv,
                                                        lv.winvf);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c.s));
  return AMGF_OK;
}

// training buffers (allocated on first use)
static int ensure_mlp_buffers(Ctx& c, int loss_cap) {
  int st;
  if (!c.mlp_m) {
    int64_t maxn = 0;
    for (int l = 0; l + 1 < (int)c.L.size(); ++l) maxn = std::max<int64_t>(maxn, c.L[l].n);
    c.mlp_part_blocks = (maxn + TPB - 1) / TPB;
    if ((st = c.alloc(&c.mlp_m, MLP_NW))) return st;
    if ((st = c.alloc(&c.mlp_v, MLP_NW))) return st;
    if ((st = c.alloc(&c.mlp_g, MLP_NW))) return st;
    if ((st = c.alloc(&c.mlp_part, c.mlp_part_blocks * MLP_NW))) return st;
    if ((st = c.alloc(&c.mlp_tw, maxn))) return st;
    if ((st = c.alloc(&c.mlp_ee, 32))) return st;
    if ((st = c.alloc(&c.mlp_rr, 32))) return st;
    CK(cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM));
  }
  if (loss_cap > c.mlp_loss_cap) {
    if ((st = c.alloc(&c.mlp_loss, loss_cap))) return st;
    c.mlp_loss_cap = loss_cap;
  }
  return AMGF_OK;
}

// Loss term and gradient of smoothed level l for the weights in c.mlp_w, with r_l already in
// L[l].rhs: ee[l] = ||e||^2, e = (I - A_l W_l) r_l, rr[l] = ||r_l||^2, and the level's share
// scale * d(ee/rr)/d(weights) added to c.mlp_g (written when l = 0).
static void enqueue_mlp_level_grad(Ctx& c, int l, float scale) {
  DLevel& lv = c.L[l];
  const int g = vec_grid(c, lv.n);
  dot_kernel<<<g, TPB, 0, c.s>>>(lv.n, lv.rhs, lv.rhs, c.partial, c.mlp_rr + l, c.counter);
  mlp_infer_kernel<<<g, TPB, 0, c.s>>>(lv.n, c.feat_d[l], c.mlp_w, 0, c.l1_d[l], c.mlp_tw, nullptr);
  scale_kernel<<<g, TPB, 0, c.s>>>(lv.n, c.mlp_tw, lv.rhs, lv.x);                    // x = W r
  CsrArgs e{};
  e.x = lv.x; e.b = lv.rhs; e.y = lv.res;
  launch_csr<M_RESID>(c, lv.A, e, lv.res, c.mlp_ee + l);                            // e = r - A x
  CsrArgs ae{};
  ae.x = lv.res; ae.y = lv.out;
  launch_csr<M_SPMV>(c, lv.A, ae);                                                   // A e
  const int nb = (int)((lv.n + TPB - 1) / TPB);
  mlp_backward_kernel<<<nb, TPB, MLP_SMEM, c.s>>>(lv.n, c.feat_d[l], c.mlp_w, lv.rhs, c.l1_d[l], lv.out,
                                                  c.mlp_rr + l, scale, c.mlp_part);
  mlp_grad_reduce_kernel<<<(MLP_NW + TPB - 1) / TPB, TPB, 0, c.s>>>(nb, c.mlp_part, c.mlp_g, l > 0 ? 1 : 0);
}

// Adam steps on the smoothing loss sum_l ||(I - A_l W_l(theta)) r_l||^2 / ||r_l||^2 (averaged over
// the smoothed levels), r_l uniform(-1, 1) from the counter-based generator.
static int mlp_train_impl(Ctx& c, float* params, float* adam_m, float* adam_v, int64_t* adam_step, int iters,
                          float lr, uint64_t seed, float* loss) {
  const int nsm = (int)c.L.size() - 1;
  if (nsm < 1) return fail(AMGF_ERR_INVALID_ARG, "training needs at least two levels");
  int st = ensure_mlp_buffers(c, iters);
  if (st) return st;
  CK(cudaMemcpyAsync(c.mlp_w, params, MLP_NW * sizeof(float), cudaMemcpyHostToDevice, c.s));
  CK(cudaMemcpyAsync(c.mlp_m, adam_m, MLP_NW * sizeof(float), cudaMemcpyHostToDevice, c.s));
  CK(cudaMemcpyAsync(c.mlp_v, adam_v, MLP_NW * sizeof(float), cudaMemcpyHostToDevice, c.s));
  const float scale = 1.0f / (float)nsm;
  int64_t t = *adam_step;
  for (int it = 0; it < iters; ++it) {
    for (int l = 0; l < nsm; ++l) {
      DLevel& lv = c.L[l];
      const uint64_t sd = seed ^ (0x632BE59BD9B4E019ull * (uint64_t)(t + 1)) ^ ((uint64_t)l << 56);
      rand_uniform_kernel<<<vec_grid(c, lv.n), TPB, 0, c.s>>>(lv.n, sd, lv.rhs);       // r
      enqueue_mlp_level_grad(c, l, scale);
    }
    mlp_loss_kernel<<<1, 1, 0, c.s>>>(nsm, c.mlp_ee, c.mlp_rr, scale, c.mlp_loss + it);
    ++t;
    mlp_adam_kernel<<<(MLP_NW + TPB - 1) / TPB, TPB, 0, c.s>>>(c.mlp_w, c.mlp_m, c.mlp_v, c.mlp_g, lr, 0.9f, 0.999f,
                                                              1e-8f, (float)t);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(params, c.mlp_w, MLP_NW * sizeof(float), cudaMemcpyDeviceToHost, c.s));
  CK(cudaMemcpyAsync(adam_m, c.mlp_m, MLP_NW * sizeof(float), cudaMemcpyDeviceToHost, c.s));
  CK(cudaMemcpyAsync(adam_v, c.mlp_v, MLP_NW * sizeof(float), cudaMemcpyDeviceToHost, c.s));
  if (loss) CK(cudaMemcpyAsync(loss, c.mlp_loss, iters * sizeof(float), cudaMemcpyDeviceToHost, c.s));
  CK(cudaStreamSynchronize(c.s));
  *adam_step = t;
  // the level operators' W stay those of the active weights
  return apply_smoother_weights(c, false);
}

// Loss and gradient of the training objective for given weights and given r_l (the kernels of
// one training step without the Adam update).
static int mlp_grad_impl(Ctx& c, const float* params, const double* r_all, float* grad, double* loss) {
  const int nsm = (int)c.L.size() - 1;
  if (nsm < 1) return fail(AMGF_ERR_INVALID_ARG, "the loss needs at least two levels");
  int st = ensure_mlp_buffers(c, 1);
  if (st) return st;
  CK(cudaMemcpyAsync(c.mlp_w, params, MLP_NW * sizeof(float), cudaMemcpyHostToDevice, c.s));
  const float scale = 1.0f / (float)nsm;
  int64_t off = 0;
  for (int l = 0; l < nsm; ++l) {
    DLevel& lv = c.L[l];
    CK(cudaMemcpyAsync(lv.rhs, r_all + off, (size_t)lv.n * sizeof(double), cudaMemcpyHostToDevice, c.s));
    off += lv.n;
    enqueue_mlp_level_grad(c, l, scale);
  }
  CK(cudaGetLastError());
  std::vector<double> ee(nsm), rr(nsm);
  CK(cudaMemcpyAsync(grad, c.mlp_g, MLP_NW * sizeof(float), cudaMemcpyDeviceToHost, c.s));
  CK(cudaMemcpyAsync(ee.data(), c.mlp_ee, nsm * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  CK(cudaMemcpyAsync(rr.data(), c.mlp_rr, nsm * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  CK(cudaStreamSynchronize(c.s));
  double sum = 0.0;
  for (int l = 0; l < nsm; ++l) sum += ee[l] / rr[l];
  if (loss) *loss = sum / nsm;
  return apply_smoother_weights(c, false);
}

// ---------------------------------------------------------------------------------------
// setup / upload

static int upload_csr(Ctx& c, const HCSR& h, DCSR& d) {
  const int num_sms = c.num_sms;
  d.nrows = h.nrows; d.ncols = h.ncols; d.nnz = h.nnz();
  int st;
  if ((st = c.upload(&d.rp, h.rp.data(), h.nrows + 1))) return st;
  if ((st = c.upload(&d.ci, h.ci.data(), d.nnz))) return st;
  if ((st = c.upload(&d.v, h.v.data(), d.nnz))) return st;
  d.K = lanes_for(h.nrows, h.nrows ? (double)d.nnz / (double)h.nrows : 1.0, num_sms);
  return AMGF_OK;
}

static int upload_csr_f(Ctx& c, const HCSR& h, DCSRf& d) {
  d.nrows = h.nrows; d.ncols = h.ncols; d.nnz = h.nnz();
  int st;
  // padded for the 16-byte aligned segments of the staged sweeps
  if ((st = c.upload_padded(&d.rp, h.rp.data(), h.nrows + 1, 2))) return st;
  if ((st = c.upload_padded(&d.ci, h.ci.data(), d.nnz, 16))) return st;
  if (c.o.precision == 3) {  // BF16 storage, round to nearest even
    std::vector<__nv_bfloat16> v(d.nnz);
    for (int64_t k = 0; k < d.nnz; ++k) v[k] = __float2bfloat16_rn((float)h.v[k]);
    if ((st = c.upload_padded(&d.vb, v.data(), d.nnz, 16))) return st;
  } else {
    std::vector<float> v(h.v.begin(), h.v.end());
    if ((st = c.upload_padded(&d.v, v.data(), d.nnz, 16))) return st;
  }
  const double avg = h.nrows ? (double)d.nnz / (double)h.nrows : 1.0;
  d.K = lanes_for_f32(h.nrows, avg, c.num_sms);
  // long rows (>= 300 nonzeros) on levels below 500 k rows: a warp per row with 8 entries per
  // lane and batch (sweep on GB300: 17-30% faster than 16 lanes with 4 entries)
  if (avg >= 300 && h.nrows < 500000) { d.K = 32; d.U = 8; }
  return AMGF_OK;
}

constexpr int STAGE_SMEM_MAX = 200 * 1024;  // dynamic shared memory of a staged CTA at most

template <typename VT>
static int plan_staging_t(Ctx& c, DCSRf& d, StageArgs g) {
  // the POST instance stages three vectors, RESID one: size both by POST
  size_t smem = stage_smem_bytes<M_POST, VT>(g);
  while (g.depth > 2 && smem > (size_t)STAGE_SMEM_MAX) {
    --g.depth;
    smem = stage_smem_bytes<M_POST, VT>(g);
  }
  if (smem > (size_t)STAGE_SMEM_MAX) return AMGF_OK;  // tiles too long: csr_kernel
  // one kernel instance serves every level with the same K and value type, so its limit is the
  // largest any level may ask for, not this level's size
  const void* fr = staged_fn<M_RESID, VT>(d.K);
  const void* fp = staged_fn<M_POST, VT>(d.K);
  CK(cudaFuncSetAttribute(fr, cudaFuncAttributeMaxDynamicSharedMemorySize, STAGE_SMEM_MAX));
  CK(cudaFuncSetAttribute(fp, cudaFuncAttributeMaxDynamicSharedMemorySize, STAGE_SMEM_MAX));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp, STAGE_TPB, smem));
  if (per_sm < 1) return AMGF_OK;
  const int64_t want = (int64_t)per_sm * c.num_sms;
  d.sg = g;
  d.ssmem = smem;
  d.sgrid = (int)(g.ntiles < want ? g.ntiles : want);
  return AMGF_OK;
}

// Staged sweeps for a level operator of the FP32 V-cycle with BF16 values: tiles of o.stage_rows
// rows (rounded up to whole passes of the CTA's row groups), o.stage_depth tiles in flight per
// CTA, one persistent CTA per resident slot.  Only where they were measured faster on GB300 (the
// level-1 sweeps of c64-c160, rows of 96-135 entries: 7-16%): BF16 values and at most
// STAGE_MAX_AVG entries per row on average.  Longer rows make a tile take so much shared memory
// that too few CTAs stay resident to keep the gathers of x in flight (c160 level 3: 2x slower);
// FP32 values were slower at every level.  Other levels keep csr_kernel.
constexpr double STAGE_MAX_AVG = 160.0;
static int plan_staging(Ctx& c, const HCSR& h, DCSRf& d) {
  d.sg = StageArgs{};
  d.sgrid = 0;
  d.ssmem = 0;
  if (c.o.stage_rows <= 0 || d.nrows == 0 || !d.vb || d.K < 8 || d.U != 4) return AMGF_OK;
  if ((double)d.nnz / (double)d.nrows > STAGE_MAX_AVG) return AMGF_OK;
  if (!c.kerr) {
    int st;
    if ((st = c.alloc_padded(&c.kerr, 1, 0))) return st;
  }
  const int G = STAGE_NW * (32 / d.K);
  const int64_t R = ((int64_t)c.o.stage_rows + G - 1) / G * G;
  const int64_t ntiles = (d.nrows + R - 1) / R;
  if (ntiles < c.num_sms) return AMGF_OK;
  int64_t cap = 0;
  for (int64_t t = 0; t < ntiles; ++t) {
    const int64_t r0 = t * R, r1 = r0 + R < d.nrows ? r0 + R : d.nrows;
    const int64_t ka = h.rp[r0] & ~(int64_t)7;
    const int64_t kn = (h.rp[r1] - ka + 7) & ~(int64_t)7;
    cap = kn > cap ? kn : cap;
  }
  if (cap > (int64_t)1 << 20) return AMGF_OK;
  StageArgs g{};
  g.ntiles = ntiles;
  g.rows = (int)R;
  g.depth = c.o.stage_depth < 2 ? 2 : (c.o.stage_depth > STAGE_MAX_DEPTH ? STAGE_MAX_DEPTH : c.o.stage_depth);
  g.cap = (int)(cap < 8 ? 8 : cap);
  g.rp_cap = (int)R + 4;
  g.vec_cap = (int)((R + 6) & ~(int64_t)3);
  g.err = c.kerr;
  return plan_staging_t<__nv_bfloat16>(c, d, g);
}

// Sliced ELL with rows sorted in windows of o.sell_window (sell_kernel) for the FP64 operators
// with enough rows to fill the GPU with one lane per row (>= SELL_MIN_ROWS_PER_SM rows per SM):
// the long-row level operators (>= SELL_MIN_AVG entries per row on average; `level_op`) and the
// interpolation and restriction operators; the others keep csr_kernel.
constexpr double SELL_MIN_AVG = 24.0;
constexpr int64_t SELL_MIN_ROWS_PER_SM = 1024;
static int plan_sell(Ctx& c, const HCSR& h, DCSR& d, bool level_op = true) {
  if (c.o.sell_window <= 0 || h.nrows == 0) return AMGF_OK;
  if (level_op && (h.nrows != h.ncols || (double)h.nnz() / (double)h.nrows < SELL_MIN_AVG)) return AMGF_OK;
  if (h.nrows < SELL_MIN_ROWS_PER_SM * c.num_sms) return AMGF_OK;
  if (h.nrows > (int64_t)INT32_MAX) return AMGF_OK;
  build_sell(h, c.o.sell_window, d.sell_h);
  int st;
  if ((st = c.upload(&d.ell_soff, d.sell_h.soff.data(), d.sell_h.nslices + 1))) return st;
  if ((st = c.upload(&d.ell_perm, d.sell_h.perm.data(), h.nrows))) return st;
  if ((st = c.upload(&d.ell_ci, d.sell_h.ci.data(), (int64_t)d.sell_h.ci.size()))) return st;
  if ((st = c.upload(&d.ell_v, d.sell_h.v.data(), (int64_t)d.sell_h.v.size()))) return st;
  std::vector<int32_t>().swap(d.sell_h.ci);  // the device copy is the only one used
  std::vector<double>().swap(d.sell_h.v);
  std::vector<int32_t>().swap(d.sell_h.perm);
  return AMGF_OK;
}

// The same sliced-ELL copy for an interpolation or restriction operator of the FP32 V-cycle
// (FP32 or BF16 values, as the CSR copy).
static int plan_sell_f(Ctx& c, const HCSR& h, DCSRf& d) {
  if (c.o.sell_window <= 0 || h.nrows == 0 || h.nrows < SELL_MIN_ROWS_PER_SM * c.num_sms) return AMGF_OK;
  if (h.nrows > (int64_t)INT32_MAX) return AMGF_OK;
  SELL S;
  build_sell(h, c.o.sell_window, S);
  int st;
  if ((st = c.upload(&d.ell_soff, S.soff.data(), S.nslices + 1))) return st;
  if ((st = c.upload(&d.ell_perm, S.perm.data(), h.nrows))) return st;
  if ((st = c.upload(&d.ell_ci, S.ci.data(), (int64_t)S.ci.size()))) return st;
  if (c.o.precision == 3) {
    std::vector<__nv_bfloat16> v(S.v.size());
    for (size_t k = 0; k < v.size(); ++k) v[k] = __float2bfloat16_rn((float)S.v[k]);
    if ((st = c.upload(&d.ell_vb, v.data(), (int64_t)v.size()))) return st;
  } else {
    std::vector<float> v(S.v.begin(), S.v.end());
    if ((st = c.upload(&d.ell_v, v.data(), (int64_t)v.size()))) return st;
  }
  d.ell_nslices = S.nslices;
  return AMGF_OK;
}

static void fill_info(Ctx& c) {
  amgf_info& in = c.info;
  std::memset(&in, 0, sizeof in);
  const int nlev = c.H.nlev();
  in.n = c.n; in.m = c.m; in.nc = c.F.nc; in.nlevels = nlev;
  double tot = 0.0;
  for (int l = 0; l < nlev && l < 32; ++l) {
    in.level_rows[l] = c.H.A[l].nrows;
    in.level_nnz[l] = c.H.A[l].nnz();
    tot += (double)c.H.A[l].nnz();
    if (l + 1 < nlev) in.interp_nnz[l] = c.H.P[l].nnz();
  }
  in.op_complexity = tot / (double)c.H.A[0].nnz();
  in.filter_block = c.F.nb;
  in.filter_nblocks = c.F.nblk;
  for (size_t l = 0; l < c.L.size() && l < 63; ++l) {
    if (c.L[l].Af.sg.ntiles > 0) in.staged_levels |= (int64_t)1 << l;
    if (c.L[l].A.ell_v) in.sell_levels |= (int64_t)1 << l;
  }
}

// dst[idx[k]] = val[k] on the device (temporary buffers, synchronous)
template <typename T>
static int scatter_to_device(Ctx& c, T* dst, const std::vector<int64_t>& idx, const std::vector<T>& val) {
  if (idx.empty()) return AMGF_OK;
  const int64_t n = (int64_t)idx.size();
  int64_t* di = nullptr;
  T* dv = nullptr;
  if (cudaMalloc(&di, n * sizeof(int64_t)) != cudaSuccess) return fail(AMGF_ERR_OOM, "cudaMalloc (update)");
  if (cudaMalloc(&dv, n * sizeof(T)) != cudaSuccess) { cudaFree(di); return fail(AMGF_ERR_OOM, "cudaMalloc (update)"); }
  // the copies from pageable memory complete asynchronously: synchronise before the kernel
  cudaError_t e = cudaMemcpy(di, idx.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dv, val.data(), n * sizeof(T), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) {
    scatter_kernel<T><<<vec_grid(c, n), TPB, 0, c.s>>>(n, di, dv, dst);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
  }
  cudaFree(di);
  cudaFree(dv);
  if (e != cudaSuccess) return fail(AMGF_ERR_CUDA, std::string("update scatter: ") + cudaGetErrorString(e));
  return AMGF_OK;
}

template <typename T>
static int copy_to_device(T* dst, const T* src, int64_t n) {
  if (n <= 0) return AMGF_OK;
  CK(cudaMemcpy(dst, src, (size_t)n * sizeof(T), cudaMemcpyHostToDevice));
  return AMGF_OK;
}

// amgf_update_D_fine in place: only D changed, the interpolation is reused, so every device
// array keeps its size and pattern and only values move: the contact rows of A_0 (their
// 32-row slices of the BSR3 image), the Galerkin-updated entries of the coarse A_l, the l1
// weights, the coarsest inverse, the mixed path's FP64 contact term, the filter matrices and
// the learned smoother's inputs.  Host arithmetic is that of the full update.  The solve graph
// stays valid (no pointer changes).  Returns kFallback when the new operator does not fit the
// device image (the caller then takes the full path; the hierarchy is consistent with D), and
// kRebuild when a coarse update left the coarse patterns (a new hierarchy is needed).
static constexpr int kFallback = -100, kRebuild = -101;
static int update_D_in_place(Ctx& c, const double* D, const amgf_csr& K, const amgf_csr& J, std::string& err) {
  auto t_start = std::chrono::steady_clock::now();
  auto since = [](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t).count();
  };
  const int nlev = c.H.nlev();
  if (c.host_only || nlev < 2 || (int)c.L.size() != nlev || !c.Eh.empty() || c.m == 0 ||
      (int64_t)c.Dh.size() != c.m || c.H.A[0].nrows != c.n)
    return kFallback;
  DLevel& l0 = c.L[0];
  if (l0.A.bsr && c.bsr0.soff.empty()) return kFallback;
  if (c.o.filter && c.F.nc > 0 && c.F.algo == 0 && c.fM_count == 0) return kFallback;
  // host: contact rows of A_0 as a fresh assembly writes them
  std::vector<int64_t> rows;
  int st = refresh_contact_rows(c.H.A[0], &K, &J, D, rows, err);
  if (st == AMGF_ERR_INVALID_ARG) return kFallback;
  if (st) return st;
  const double t_assemble = since(t_start);
  auto t1 = std::chrono::steady_clock::now();
  // coarse levels: Galerkin products of the contact change, l1 sums, coarsest inverse
  std::vector<double> dD(c.m);
  for (int64_t r = 0; r < c.m; ++r) dD[r] = D[r] - c.Dh[r];
  std::vector<std::vector<int64_t>> changed;
  st = update_hierarchy_contact(c.H, nullptr, &J, dD.data(), &changed, err);
  if (st == AMGF_ERR_INVALID_ARG) return kRebuild;
  if (st) return st;
  c.Dh.assign(D, D + c.m);
  const double t_hier = since(t1);
  t1 = std::chrono::steady_clock::now();
  Filter F2;
  const bool filt = c.o.filter && c.F.nc > 0;
  if (filt) {
    if ((st = build_filter(c.H.A[0], &J, c.o, F2, err))) return st;
    const bool same = F2.nc == c.F.nc && F2.nb == c.F.nb && F2.nblk == c.F.nblk && F2.algo == c.F.algo &&
                      F2.gidx == c.F.gidx && F2.touch_rows == c.F.touch_rows &&
                      F2.tasks.size() == c.F.tasks.size() &&
                      (F2.tasks.empty() ||
                       std::memcmp(F2.tasks.data(), c.F.tasks.data(), F2.tasks.size() * sizeof(FilterTask)) == 0) &&
                      F2.Sc.nnz() == c.fSc.nnz && (F2.algo != 0 || (int64_t)F2.M.size() == c.fM_count);
    if (!same) return kFallback;
  }
  const double t_filter = since(t1);
  std::vector<std::vector<float>> feat;
  smoother_features(c.H, &J, D, nullptr, c.n, feat);
  // ---- device, in place (nothing of an earlier call may still read these arrays; copies
  // from pageable memory may still be in flight when cudaMemcpy returns, so the device is
  // synchronised again at the end)
  CK(cudaDeviceSynchronize());
  if (l0.A.bsr) {
    std::vector<int64_t> sl;
    sl.reserve(rows.size());
    for (int64_t a : rows) sl.push_back(a / 3 / BSR3::W);
    std::sort(sl.begin(), sl.end());
    sl.erase(std::unique(sl.begin(), sl.end()), sl.end());
    std::vector<double> buf;
    for (int64_t q : sl) {
      const int64_t s0 = c.bsr0.soff[q], len = 9 * (c.bsr0.soff[q + 1] - s0);
      buf.resize(len);
      bsr3_fill_slice(c.H.A[0], c.bsr0, q, buf.data());
      if ((st = copy_to_device(l0.A.bv + 9 * s0, buf.data(), len))) return st;
    }
  } else {
    std::vector<int64_t> idx;
    std::vector<double> val;
    for (int64_t a : rows)
      for (int64_t k = c.H.A[0].rp[a]; k < c.H.A[0].rp[a + 1]; ++k) { idx.push_back(k); val.push_back(c.H.A[0].v[k]); }
    if ((st = scatter_to_device(c, l0.A.v, idx, val))) return st;
  }
  for (int l = 1; l < nlev; ++l) {
    const std::vector<int64_t>& idx = changed[l];
    if (idx.empty()) continue;
    const HCSR& A = c.H.A[l];
    DLevel& lv = c.L[l];
    if (!c.mixed) {
      std::vector<double> val(idx.size());
      for (size_t k = 0; k < idx.size(); ++k) val[k] = A.v[idx[k]];
      if ((st = scatter_to_device(c, lv.A.v, idx, val))) return st;
      if (lv.A.ell_v) {  // the same values at their sliced-ELL slots
        std::vector<int64_t> slots(idx.size());
        for (size_t k = 0; k < idx.size(); ++k) {
          const int64_t r = (int64_t)(std::upper_bound(A.rp.begin(), A.rp.end(), idx[k]) - A.rp.begin()) - 1;
          slots[k] = sell_slot(A, lv.A.sell_h, r, idx[k]);
        }
        if ((st = scatter_to_device(c, lv.A.ell_v, slots, val))) return st;
      }
    } else if (lv.Af.vb) {
      std::vector<__nv_bfloat16> val(idx.size());
      for (size_t k = 0; k < idx.size(); ++k) val[k] = __float2bfloat16_rn((float)A.v[idx[k]]);
      if ((st = scatter_to_device(c, lv.Af.vb, idx, val))) return st;
    } else {
      std::vector<float> val(idx.size());
      for (size_t k = 0; k < idx.size(); ++k) val[k] = (float)A.v[idx[k]];
      if ((st = scatter_to_device(c, lv.Af.v, idx, val))) return st;
    }
  }
  for (int l = 0; l < nlev; ++l) {
    DLevel& lv = c.L[l];
    std::vector<double> w(lv.n);
    for (int64_t i = 0; i < lv.n; ++i) w[i] = 1.0 / c.H.l1[l][i];
    if (lv.winv && (st = copy_to_device(lv.winv, w.data(), lv.n))) return st;
    if (lv.winvf) {
      std::vector<float> wf(w.begin(), w.end());
      if ((st = copy_to_device(lv.winvf, wf.data(), lv.n))) return st;
    }
    if (l + 1 < nlev) {
      if ((st = copy_to_device(c.feat_d[l], feat[l].data(), (int64_t)feat[l].size()))) return st;
      if ((st = copy_to_device(c.l1_d[l], c.H.l1[l].data(), lv.n))) return st;
    }
  }
  if (c.H.n_coarse != c.nL) return kRebuild;
  if (!c.mixed) {
    if ((st = copy_to_device(c.coarse_inv, c.H.coarse_inv.data(), c.nL * c.nL))) return st;
  } else {
    std::vector<float> ci(c.H.coarse_inv.begin(), c.H.coarse_inv.end());
    if ((st = copy_to_device(c.coarse_inv_f, ci.data(), c.nL * c.nL))) return st;
    std::vector<int64_t> zrp(c.n + 1, 0);
    amgf_csr Z{c.n, c.n, 0, zrp.data(), nullptr, nullptr};
    HCSR C;
    if ((st = assemble_S(&Z, &J, D, C, err))) return st;
    if (C.nnz() != c.c_nnz) return kRebuild;
    if ((st = copy_to_device(c.c_v, C.v.data(), C.nnz()))) return st;
  }
  if (filt) {
    const int64_t tot = F2.nb * F2.nblk;
    if (F2.algo == 0) {
      if ((st = copy_to_device(c.fM, F2.M.data(), (int64_t)F2.M.size()))) return st;
      decltype(F2.M)().swap(F2.M);
    } else {
      if ((st = copy_to_device(c.fG, F2.G.data(), tot * F2.nb))) return st;
      if ((st = copy_to_device(c.fGT, F2.GT.data(), tot * F2.nb))) return st;
      if ((st = copy_to_device(c.fDinv, F2.Dinv.data(), tot * F2.nb))) return st;
    }
    if ((st = copy_to_device(c.fSc.v, F2.Sc.v.data(), F2.Sc.nnz()))) return st;
    c.F = std::move(F2);
  }
  CK(cudaDeviceSynchronize());
  fill_info(c);
  c.info.t_assemble_s = t_assemble;
  c.info.t_hierarchy_s = t_hier;
  c.info.t_filter_s = t_filter;
  c.info.t_setup_s = since(t_start);
  return AMGF_OK;
}

// keep_coarse: new fine-level operator (and filter) for D, coarse levels of B kept from the
// last full setup (amgf_update_D_fine)
static int build_all(Ctx& c, const double* D, bool keep_coarse = false) {
  auto t_start = std::chrono::steady_clock::now();
  std::string err;
  amgf_csr K{c.Kh.nrows, c.Kh.ncols, c.Kh.nnz(), c.Kh.rp.data(), c.Kh.ci.data(), c.Kh.v.data()};
  amgf_csr J{c.Jh.nrows, c.Jh.ncols, c.Jh.nnz(), c.Jh.rp.data(), c.Jh.ci.data(), c.Jh.v.data()};
  auto since = [](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t).count();
  };
  if (keep_coarse && !c.host_only && c.o.update_in_place) {
    const int r = update_D_in_place(c, D, K, J, err);
    if (r == AMGF_OK) return AMGF_OK;
    if (r == kRebuild) keep_coarse = false;
    else if (r != kFallback) return err.empty() ? r : fail(r, err);  // CUDA errors are reported already
    err.clear();
  }
  // A = K + J^T D J (+ diag(E)): assembled, or (interpolation reused, no bound term) the
  // contact rows of the current A_0 rewritten in place with the same arithmetic
  HCSR S;
  bool have_S = false;
  const double* E = c.Eh.empty() ? nullptr : c.Eh.data();
  auto assemble = [&]() -> int {
    int r = assemble_S(&K, c.m > 0 ? &J : nullptr, D, S, err);
    if (!r && E) r = add_diagonal(S, E, err);
    have_S = r == AMGF_OK;
    return r;
  };
  int st = AMGF_OK;
  double t_assemble = 0.0;
  auto t1 = std::chrono::steady_clock::now();
  bool rebuilt = true;
  if (keep_coarse && c.H.nlev() >= 2 && c.H.A[0].nrows == c.n && (int64_t)c.Dh.size() == c.m) {
    std::vector<double> dD(c.m);
    for (int64_t r = 0; r < c.m; ++r) dD[r] = D[r] - c.Dh[r];
    std::vector<int64_t> rows;
    st = !E && c.m > 0 ? refresh_contact_rows(c.H.A[0], &K, &J, D, rows, err) : AMGF_ERR_INVALID_ARG;
    if (st == AMGF_ERR_INVALID_ARG && (st = assemble())) return fail(st, err);
    if (st) return fail(st, err);
    t_assemble = since(t_start);
    t1 = std::chrono::steady_clock::now();
    st = update_hierarchy_contact(c.H, have_S ? &S : nullptr, c.m > 0 ? &J : nullptr, dD.data(), nullptr, err);
    if (st == AMGF_ERR_NOT_SPD) return fail(st, err);
    rebuilt = st != AMGF_OK;  // pattern mismatch: rebuild below
  }
  if (rebuilt) {
    if (!have_S && (st = assemble())) return fail(st, err);
    if (t_assemble == 0.0) {
      t_assemble = since(t_start);
      t1 = std::chrono::steady_clock::now();
    }
    st = build_hierarchy(std::move(S), c.o, c.H, err);  // S is not used again
    if (st) return fail(st, err);
  }
  if (c.m > 0) c.Dh.assign(D, D + c.m);
  const double t_hier = since(t1);
  t1 = std::chrono::steady_clock::now();
  if (c.o.filter) {
    st = build_filter(c.H.A[0], c.m > 0 ? &J : nullptr, c.o, c.F, err);  // A_0 = A
    if (st) return fail(st, err);
  } else {
    c.F = Filter();
  }
  const double t_filter = since(t1);
  S = HCSR();
  fill_info(c);
  c.info.t_assemble_s = t_assemble;
  c.info.t_hierarchy_s = t_hier;
  c.info.t_filter_s = t_filter;
  c.info.t_setup_s = since(t_start);
  if (c.host_only) return AMGF_OK;
  // ---- device upload
  c.release_device();
  c.info.staged_levels = 0;
  c.info.sell_levels = 0;
  c.bsr0 = BSR3();
  const int nlev = c.H.nlev();
  c.L.assign(nlev, DLevel());
  // mixed precision needs a coarse level and the 3x3 node-block structure of K
  BSR3 kb;
  c.mixed = c.o.precision > 0 && nlev >= 2 && c.o.num_functions == 3 && build_bsr3(c.Kh, 1.05, kb);
  c.k_bf16 = c.mixed && c.o.precision >= 2;
  for (int l = 0; l < nlev; ++l) {
    DLevel& lv = c.L[l];
    lv.n = c.H.A[l].nrows;
    std::vector<double> w(lv.n);
    for (int64_t i = 0; i < lv.n; ++i) w[i] = 1.0 / c.H.l1[l][i];
    // FP64 operator: always on the fine level (outer PCG), on every level without mixed precision
    if (l == 0 || !c.mixed) {
      BSR3 bsr;
      if (l == 0 && c.o.num_functions == 3 && build_bsr3(c.H.A[0], 1.05, bsr)) {
        lv.A.nrows = lv.A.ncols = lv.n;
        lv.A.nnz = c.H.A[0].nnz();
        lv.A.bsr = true;
        lv.A.nbrows = bsr.nbrows;
        lv.A.nslices = bsr.nslices;
        lv.A.nblocks = bsr.nblocks;
        if ((st = c.upload(&lv.A.soff, bsr.soff.data(), bsr.nslices + 1))) return st;
        if ((st = c.upload(&lv.A.bci, bsr.bci.data(), (int64_t)bsr.bci.size()))) return st;
        if ((st = c.upload(&lv.A.bv, bsr.v.data(), (int64_t)bsr.v.size()))) return st;
        std::vector<double>().swap(bsr.v);
        c.bsr0 = std::move(bsr);  // for in-place updates of the contact rows
      } else if ((st = upload_csr(c, c.H.A[l], lv.A))) {
        return st;
      } else if (l > 0 && (st = plan_sell(c, c.H.A[l], lv.A))) {
        return st;
      }
      if (lv.A.ell_v && l < 63) c.info.sell_levels |= (int64_t)1 << l;
      if ((st = c.upload(&lv.winv, w.data(), lv.n))) return st;
      if ((st = c.alloc(&lv.x, lv.n))) return st;
    }
    if (!c.mixed) {
      if (l + 1 < nlev) {
        if ((st = upload_csr(c, c.H.P[l], lv.P))) return st;
        if ((st = upload_csr(c, c.H.R[l], lv.R))) return st;
        if ((st = plan_sell(c, c.H.P[l], lv.P, false))) return st;
        if ((st = plan_sell(c, c.H.R[l], lv.R, false))) return st;
      }
      if ((st = c.alloc(&lv.rhs, lv.n))) return st;
      if ((st = c.alloc(&lv.res, lv.n))) return st;
      if ((st = c.alloc(&lv.out, lv.n))) return st;
      if (c.o.smoother == 1 && (st = c.alloc(&lv.d, lv.n))) return st;
    } else {
      if (l > 0 && (st = upload_csr_f(c, c.H.A[l], lv.Af))) return st;
      if (l + 1 < nlev) {
        if ((st = upload_csr_f(c, c.H.P[l], lv.Pf))) return st;
        if ((st = upload_csr_f(c, c.H.R[l], lv.Rf))) return st;
        if ((st = plan_sell_f(c, c.H.P[l], lv.Pf))) return st;
        if ((st = plan_sell_f(c, c.H.R[l], lv.Rf))) return st;
      }
      std::vector<float> wf(w.begin(), w.end());
      // W, b and x of a level are staged in 16-byte segments by the staged sweeps
      if ((st = c.upload_padded(&lv.winvf, wf.data(), lv.n, 8))) return st;
      if ((st = c.alloc_padded(&lv.rhsf, lv.n, 8))) return st;
      if ((st = c.alloc_padded(&lv.xf, lv.n, 8))) return st;
      if (l > 0 && (st = plan_staging(c, c.H.A[l], lv.Af))) return st;
      if (lv.Af.sg.ntiles > 0 && l < 63) c.info.staged_levels |= (int64_t)1 << l;
      if ((st = c.alloc(&lv.resf, lv.n))) return st;
      if ((st = c.alloc(&lv.outf, lv.n))) return st;
      if (c.o.smoother == 1 && (st = c.alloc(&lv.df, lv.n))) return st;
    }
  }
  for (int l = 0; l < nlev; ++l) {  // labels of the per-launch records
    DLevel& lv = c.L[l];
    lv.A.level = lv.P.level = lv.R.level = lv.Af.level = lv.Pf.level = lv.Rf.level = l;
    lv.P.role = lv.Pf.role = 'P';
    lv.R.role = lv.Rf.role = 'R';
  }
  // learned-smoother inputs: features and l1 of every smoothed level
  {
    std::vector<std::vector<float>> feat;
    smoother_features(c.H, c.m > 0 ? &J : nullptr, D, E, c.n, feat);
    c.feat_d.assign(nlev, nullptr);
    c.l1_d.assign(nlev, nullptr);
    for (int l = 0; l + 1 < nlev; ++l) {
      if ((st = c.upload(&c.feat_d[l], feat[l].data(), (int64_t)feat[l].size()))) return st;
      if ((st = c.upload(&c.l1_d[l], c.H.l1[l].data(), c.L[l].n))) return st;
    }
    if ((st = c.alloc(&c.mlp_w, MLP_NW))) return st;
  }
  c.nL = c.H.n_coarse;
  if (!c.mixed) {
    if ((st = c.upload(&c.coarse_inv, c.H.coarse_inv.data(), c.nL * c.nL))) return st;
  } else {
    std::vector<float> ci(c.H.coarse_inv.begin(), c.H.coarse_inv.end());
    if ((st = c.upload(&c.coarse_inv_f, ci.data(), c.nL * c.nL))) return st;
    // fine-level K in 3x3 blocks, FP32 or BF16 (round to nearest even)
    c.k_nbrows = kb.nbrows;
    c.k_nslices = kb.nslices;
    c.k_nblocks = kb.nblocks;
    if ((st = c.upload(&c.k_soff, kb.soff.data(), kb.nslices + 1))) return st;
    if (c.k_bf16) {
      // packed: per block slot three 8-byte words {column, v0 v1}, {v2..v5}, {v6 v7 v8, 0},
      // word p of slot (slice s, j, lane) at 3 soff[s] + (3 j + p) 32 + lane
      std::vector<uint2> pk(3 * kb.bci.size());
      auto bf = [](double x) -> uint32_t {
        const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
        uint16_t u;
        memcpy(&u, &h, 2);
        return u;
      };
#pragma omp parallel for schedule(static)
      for (int64_t sl = 0; sl < kb.nslices; ++sl) {
        const int64_t s0 = kb.soff[sl], w = (kb.soff[sl + 1] - s0) / BSR3::W;
        for (int64_t j = 0; j < w; ++j)
          for (int lane = 0; lane < BSR3::W; ++lane) {
            const int64_t slot = s0 + BSR3::W * j + lane;
            uint32_t q[9];
            for (int t = 0; t < 9; ++t) q[t] = bf(kb.v[9 * s0 + (9 * j + t) * BSR3::W + lane]);
            uint2* o = pk.data() + 3 * s0 + 3 * BSR3::W * j + lane;
            o[0] = make_uint2((uint32_t)kb.bci[slot], q[0] | (q[1] << 16));
            o[BSR3::W] = make_uint2(q[2] | (q[3] << 16), q[4] | (q[5] << 16));
            o[2 * BSR3::W] = make_uint2(q[6] | (q[7] << 16), q[8]);
          }
      }
      uint2* d = nullptr;
      if ((st = c.upload(&d, pk.data(), (int64_t)pk.size()))) return st;
      c.k_v = d;
    } else {
      if ((st = c.upload(&c.k_bci, kb.bci.data(), (int64_t)kb.bci.size()))) return st;
      std::vector<float> v(kb.v.begin(), kb.v.end());
      float* d = nullptr;
      if ((st = c.upload(&d, v.data(), (int64_t)v.size()))) return st;
      c.k_v = d;
    }
    // contact term J^T D J over all rows, FP64
    std::vector<int64_t> zrp(c.n + 1, 0);
    amgf_csr Z{c.n, c.n, 0, zrp.data(), nullptr, nullptr};
    HCSR C;
    st = assemble_S(&Z, c.m > 0 ? &J : nullptr, D, C, err);
    if (st) return fail(st, err);
    if (E && (st = add_diagonal(C, E, err))) return fail(st, err);  // the bound term stays FP64 too
    std::vector<int32_t> crp(c.n + 1);
    for (int64_t i = 0; i <= c.n; ++i) crp[i] = (int32_t)C.rp[i];
    if ((st = c.upload(&c.c_rp, crp.data(), c.n + 1))) return st;
    if ((st = c.upload(&c.c_ci, C.ci.data(), C.nnz()))) return st;
    c.c_nnz = C.nnz();
    if ((st = c.upload(&c.c_v, C.v.data(), C.nnz()))) return st;
  }
  if (c.F.nc > 0) {
    const int64_t tot = c.F.nb * c.F.nblk;
    if (c.F.algo == 0) {
      if (2 * c.F.nb * (int64_t)sizeof(double) > 200 * 1024)
        return fail(AMGF_ERR_INVALID_ARG, "filter block too large for shared memory");
      if ((st = c.upload(&c.fM, c.F.M.data(), (int64_t)c.F.M.size()))) return st;
      c.fM_count = (int64_t)c.F.M.size();
      if ((st = c.upload(&c.ftasks, c.F.tasks.data(), (int64_t)c.F.tasks.size()))) return st;
      decltype(c.F.M)().swap(c.F.M);  // the device copy is the only one used
      if (2 * c.F.nb * (int64_t)sizeof(double) > 48 * 1024) {
        const int bytes = (int)(2 * c.F.nb * sizeof(double));
        CK(cudaFuncSetAttribute(filter_bcr_kernel<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        CK(cudaFuncSetAttribute(filter_bcr_kernel<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        CK(cudaFuncSetAttribute(filter_bcr_kernel<true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        CK(cudaFuncSetAttribute(filter_bcr_kernel<false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      }
    } else {
      if ((st = c.upload(&c.fG, c.F.G.data(), tot * c.F.nb))) return st;
      if ((st = c.upload(&c.fGT, c.F.GT.data(), tot * c.F.nb))) return st;
      if ((st = c.upload(&c.fDinv, c.F.Dinv.data(), tot * c.F.nb))) return st;
    }
    if ((st = c.upload(&c.fgidx, c.F.gidx.data(), c.F.nc))) return st;
    std::vector<int64_t> where(c.n, -1), fic(c.F.nc);
    for (int64_t t = 0; t < c.F.nc; ++t) where[c.F.ic[t]] = t;
    for (int64_t p = 0; p < c.F.nc; ++p) fic[p] = where[c.F.gidx[p]];
    if ((st = c.upload(&c.ficidx, fic.data(), c.F.nc))) return st;
    if ((st = c.upload(&c.ftouch, c.F.touch_rows.data(), (int64_t)c.F.touch_rows.size()))) return st;
    if ((st = upload_csr(c, c.F.Sc, c.fSc))) return st;
    c.fSc.level = 0;
    c.fSc.role = 'S';
    if ((st = c.alloc(&c.fy, tot))) return st;
    if ((st = c.alloc(&c.fz, tot))) return st;
    if ((st = c.alloc(&c.fw, tot))) return st;
    if ((st = c.alloc(&c.fv, tot))) return st;
    // filter sweeps: 16-CTA clusters where the device allows them, else 8; stage the next
    // block's rows in shared memory when two stages fit next to the block vectors
    if (c.F.algo == 1) {
      const int64_t nb = c.F.nb;
      auto smem_for = [&](int cs, bool staged) {
        const int64_t rpc = (nb + cs - 1) / cs;
        return (size_t)(2 * nb + (staged ? 2 * rpc * nb : 0)) * sizeof(double);
      };
      const size_t limit = 200 * 1024;
      if (smem_for(8, false) > limit) return fail(AMGF_ERR_INVALID_ARG, "filter block too large for shared memory");
      CK(cudaFuncSetAttribute(filter_sweep_kernel<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
      CK(cudaFuncSetAttribute(filter_sweep_kernel<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
      CK(cudaFuncSetAttribute(filter_sweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit));
      CK(cudaFuncSetAttribute(filter_sweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit));
      c.filter_cs = 8;
      for (int cs : {16, 8}) {
        const bool staged = smem_for(cs, true) <= limit;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs, 1, 1);
        cfg.blockDim = dim3(FILTER_TPB, 1, 1);
        cfg.dynamicSmemBytes = smem_for(cs, staged);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        const cudaError_t e = staged ? cudaOccupancyMaxActiveClusters(&nclusters, filter_sweep_kernel<true>, &cfg)
                                     : cudaOccupancyMaxActiveClusters(&nclusters, filter_sweep_kernel<false>, &cfg);
        if (e == cudaSuccess && nclusters > 0) {
          c.filter_cs = cs;
          c.filter_staged = staged;
          c.filter_smem = smem_for(cs, staged);
          break;
        }
        cudaGetLastError();  // clear a refused configuration and try the next one
      }
      if (c.filter_smem == 0) { c.filter_staged = false; c.filter_smem = smem_for(8, false); }
    }
  }
  const int64_t n = c.n;
  double** vecs[] = {&c.b, &c.x, &c.r, &c.z, &c.p, &c.q, &c.y1, &c.r1};
  for (double** v : vecs) {
    if ((st = c.alloc(v, n))) return st;
    CK(cudaMemset(*v, 0, n * sizeof(double)));
  }
  if ((st = c.alloc(&c.partial, MAX_DOT_BLOCKS))) return st;
  if ((st = c.alloc(&c.counter, 1))) return st;
  CK(cudaMemset(c.counter, 0, sizeof(unsigned)));
  if ((st = c.alloc(&c.scratch_scalar, 4))) return st;
  if ((st = c.alloc(&c.st, 1))) return st;
  CK(cudaMemset(c.st, 0, sizeof(PcgState)));
  c.info.t_setup_s = since(t_start);
  amgf_info& in = c.info;
  if (c.o.verbose) {
    fprintf(stderr, "amgf: setup %.2fs: assemble %.2fs, hierarchy %.2fs, filter %.2fs, device %.2fs\n", in.t_setup_s,
            in.t_assemble_s, in.t_hierarchy_s, in.t_filter_s,
            in.t_setup_s - in.t_assemble_s - in.t_hierarchy_s - in.t_filter_s);
    fprintf(stderr, "amgf: n=%lld m=%lld nc=%lld levels=%d opcx=%.3f filter nb=%lld nblk=%lld cluster=%d staged=%d setup %.2fs\n",
            (long long)c.n, (long long)c.m, (long long)c.F.nc, nlev, in.op_complexity, (long long)c.F.nb,
            (long long)c.F.nblk, c.filter_cs, (int)c.filter_staged, in.t_setup_s);
    fprintf(stderr, "  V-cycle precision: %s\n", c.mixed ? (c.k_bf16 ? "fp32 (fine K bf16)" : "fp32") : "fp64");
    for (int l = 0; l < nlev; ++l)
      fprintf(stderr, "  level %d: rows %lld nnz %lld lanes %d%s\n", l, (long long)c.L[l].n, (long long)c.H.A[l].nnz(),
              c.mixed && l > 0 ? c.L[l].Af.K : c.L[l].A.K, c.L[l].A.bsr ? " (3x3 blocks)" : "");
  }
  CK(cudaDeviceSynchronize());
  return AMGF_OK;
}

// Host copy of a caller's CSR matrix (kept by the handle); the large arrays are sized without
// a fill and copied in parallel chunks.
static void copy_csr(const amgf_csr* a, HCSR& h) {
  h.nrows = a->nrows; h.ncols = a->ncols;
  h.rp.assign(a->row_ptr, a->row_ptr + a->nrows + 1);
  h.ci.resize(a->nnz);
  h.v.resize(a->nnz);
  const int64_t chunk = 1 << 20, nchunk = (a->nnz + chunk - 1) / chunk;
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < nchunk; ++q) {
    const int64_t b = q * chunk, e = std::min(a->nnz, b + chunk);
    std::copy(a->col_idx + b, a->col_idx + e, h.ci.begin() + b);
    std::copy(a->val + b, a->val + e, h.v.begin() + b);
  }
}

// join the caller's stream: library stream waits for it (begin) / caller waits for us (end)
static int join_begin(Ctx& c, void* stream) {
  CK(cudaEventRecord(c.ev_in, (cudaStream_t)stream));
  CK(cudaStreamWaitEvent(c.s, c.ev_in, 0));
  return AMGF_OK;
}
static int join_end(Ctx& c, void* stream) {
  CK(cudaGetLastError());
  CK(cudaEventRecord(c.ev_out, c.s));
  CK(cudaStreamWaitEvent((cudaStream_t)stream, c.ev_out, 0));
  return AMGF_OK;
}

}  // namespace amgf

using namespace amgf;

struct amgf_ctx {
  Ctx c;
};

extern "C" {

int amgf_options_default(amgf_options* o) {
  if (!o) return fail(AMGF_ERR_INVALID_ARG, "null options");
  std::memset(o, 0, sizeof *o);
  o->strength_theta = 0.52;
  o->rtol = 1e-8;
  o->max_levels = 25;
  o->max_coarse = 1200;
  o->num_functions = 3;
  o->nu = 1;
  o->filter = 1;
  o->contact_components = 0;
  o->maxit = 5000;
  o->use_graph = 1;
  o->verbose = 0;
  o->precision = 0;
  o->filter_algo = 0;
  o->interp = 0;
  o->p_max = 4;
  o->update_in_place = 1;
  o->smoother = 0;
  o->cheby_lower = 0.3;
  o->stage_rows = 32;
  o->stage_depth = 2;
  o->sell_window = 256;
  return AMGF_OK;
}

const char* amgf_last_error(void) { return g_last_error.c_str(); }

static int setup_impl(const amgf_csr* K, const amgf_csr* J, const double* D, const double* dlo,
                      const double* dhi, const amgf_options* o, amgf_handle* out, bool host_only) {
  g_last_error.clear();
  if (!out) return fail(AMGF_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  std::string err;
  int st = validate_csr(K, "K", true, err);
  if (st) return fail(st, err);
  const bool has_j = J && J->nrows > 0;
  if (has_j) {
    st = validate_csr(J, "J", false, err);
    if (st) return fail(st, err);
    if (J->ncols != K->nrows) return fail(AMGF_ERR_INVALID_ARG, "J has the wrong number of columns");
    if (!D) return fail(AMGF_ERR_INVALID_ARG, "null D");
  }
  amgf_options opt;
  if (o) opt = *o; else amgf_options_default(&opt);
  if (opt.nu < 1 || opt.max_levels < 1 || opt.max_coarse < 1 || opt.num_functions < 1 || !(opt.rtol > 0.0) ||
      opt.maxit < 0 || opt.contact_components < 0 || opt.contact_components > 2 || opt.precision < 0 ||
      opt.precision > 3 || opt.filter_algo < 0 || opt.filter_algo > 1 ||
      opt.interp < 0 || opt.interp > 1 || opt.p_max < 0 || opt.update_in_place < 0 || opt.update_in_place > 1 || opt.smoother < 0 ||
      opt.smoother > 1 || !(opt.cheby_lower > 0.0 && opt.cheby_lower < 1.0) || opt.stage_rows < 0 ||
      opt.stage_rows > 4096 || (opt.stage_rows > 0 && (opt.stage_depth < 2 || opt.stage_depth > 8)) ||
      opt.sell_window < 0)
    return fail(AMGF_ERR_INVALID_ARG, "invalid options");
  int ndev = 0;
  if (!host_only && (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)) return fail(AMGF_ERR_CUDA, "no CUDA device");
  std::unique_ptr<amgf_ctx> h(new (std::nothrow) amgf_ctx());
  if (!h) return fail(AMGF_ERR_OOM, "host allocation");
  Ctx& c = h->c;
  c.o = opt;
  c.host_only = host_only;
  c.n = K->nrows;
  c.m = has_j ? J->nrows : 0;
  copy_csr(K, c.Kh);
  if (has_j) copy_csr(J, c.Jh);
  if (dlo || dhi) {
    c.Eh.assign(c.n, 0.0);
    for (int64_t i = 0; i < c.n; ++i) c.Eh[i] = (dlo ? dlo[i] : 0.0) + (dhi ? dhi[i] : 0.0);
  }
  if (host_only) {
    st = build_all(c, has_j ? D : nullptr);
    if (st) return st;
    *out = h.release();
    return AMGF_OK;
  }
  CK(cudaGetDevice(&c.device));
  CK(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device));
  CK(cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&c.ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c.ev_out, cudaEventDisableTiming));
  CK(cudaEventCreate(&c.t0));
  CK(cudaEventCreate(&c.t1));
  CK(cudaMallocHost(&c.st_host, sizeof(PcgState)));
  st = build_all(c, has_j ? D : nullptr);
  if (st) return st;
  *out = h.release();
  return AMGF_OK;
}

int amgf_setup(const amgf_csr* K, const amgf_csr* J, const double* D, const amgf_options* o, amgf_handle* out) {
  return setup_impl(K, J, D, nullptr, nullptr, o, out, false);
}

int amgf_setup_host(const amgf_csr* K, const amgf_csr* J, const double* D, const amgf_options* o,
                    amgf_handle* out) {
  return setup_impl(K, J, D, nullptr, nullptr, o, out, true);
}

int amgf_setup_bounds(const amgf_csr* K, const amgf_csr* J, const double* D, const double* d_lower,
                      const double* d_upper, const amgf_options* o, int host_only, amgf_handle* out) {
  return setup_impl(K, J, D, d_lower, d_upper, o, out, host_only != 0);
}

int amgf_update_bounds(amgf_handle h, const double* D, const double* d_lower, const double* d_upper) {
  if (!h) return fail(AMGF_ERR_INVALID_ARG, "null handle");
  Ctx& c = h->c;
  if (!d_lower && !d_upper) {
    c.Eh.clear();
  } else {
    c.Eh.assign(c.n, 0.0);
    for (int64_t i = 0; i < c.n; ++i) c.Eh[i] = (d_lower ? d_lower[i] : 0.0) + (d_upper ? d_upper[i] : 0.0);
  }
  return amgf_update_D(h, D);
}

int amgf_update_D(amgf_handle h, const double* D) {
  if (!h) return fail(AMGF_ERR_INVALID_ARG, "null handle");
  if (h->c.m > 0 && !D) return fail(AMGF_ERR_INVALID_ARG, "null D");
  if (!h->c.host_only) CK(cudaSetDevice(h->c.device));
  const int st = build_all(h->c, D);
  if (st || h->c.host_only || h->c.mlp_w_host.empty()) return st;
  return apply_smoother_weights(h->c, false);
}

int amgf_update_D_fine(amgf_handle h, const double* D) {
  if (!h) return fail(AMGF_ERR_INVALID_ARG, "null handle");
  if (h->c.m > 0 && !D) return fail(AMGF_ERR_INVALID_ARG, "null D");
  if (!h->c.host_only) CK(cudaSetDevice(h->c.device));
  const int st = build_all(h->c, D, true);
  if (st || h->c.host_only || h->c.mlp_w_host.empty()) return st;
  return apply_smoother_weights(h->c, false);
}

int amgf_destroy(amgf_handle h) {
  if (!h) return AMGF_OK;
  if (!h->c.host_only) {
    cudaSetDevice(h->c.device);
    if (h->c.s) cudaStreamSynchronize(h->c.s);
  }
  delete h;
  return AMGF_OK;
}

int amgf_apply(amgf_handle h, const double* r_dev, double* z_dev, void* stream) {
  if (h && h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (!h || !r_dev || !z_dev || r_dev == z_dev) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  Ctx& c = h->c;
  CK(cudaSetDevice(c.device));
  int st = join_begin(c, stream);
  if (st) return st;
  enqueue_scale_w0(c, r_dev);
  enqueue_apply(c, r_dev, z_dev, nullptr);
  return join_end(c, stream);
}

int amgf_apply_stages(amgf_handle h, const double* r_dev, double* z_dev, double* y1_dev, double* r1_dev,
                      double* w_dev, double* r2_dev, void* stream) {
  if (h && h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (!h || !r_dev || !z_dev || r_dev == z_dev) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  Ctx& c = h->c;
  if ((w_dev || r2_dev) && (!c.o.filter || c.F.nc == 0))
    return fail(AMGF_ERR_INVALID_ARG, "w and r2 need the filter (options.filter = 1, nonempty I_c)");
  CK(cudaSetDevice(c.device));
  int st = join_begin(c, stream);
  if (st) return st;
  ApplyTap tap;
  tap.y1 = y1_dev; tap.r1 = r1_dev; tap.w = w_dev; tap.r2 = r2_dev;
  enqueue_scale_w0(c, r_dev);
  enqueue_apply(c, r_dev, z_dev, nullptr, &tap);
  CK(cudaGetLastError());
  return join_end(c, stream);
}

int amgf_vcycle(amgf_handle h, const double* r_dev, double* x_dev, void* stream) {
  if (h && h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (!h || !r_dev || !x_dev || r_dev == x_dev) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  Ctx& c = h->c;
  CK(cudaSetDevice(c.device));
  int st = join_begin(c, stream);
  if (st) return st;
  enqueue_scale_w0(c, r_dev);
  enqueue_B(c, r_dev, x_dev, nullptr, nullptr, nullptr);
  return join_end(c, stream);
}

int amgf_matvec(amgf_handle h, const double* x_dev, double* y_dev, void* stream) {
  if (h && h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (!h || !x_dev || !y_dev || x_dev == y_dev) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  Ctx& c = h->c;
  CK(cudaSetDevice(c.device));
  int st = join_begin(c, stream);
  if (st) return st;
  CsrArgs a{};
  a.x = x_dev; a.y = y_dev;
  launch_csr<M_SPMV>(c, c.L[0].A, a);
  return join_end(c, stream);
}

int amgf_filter_solve_host(amgf_handle h, const double* v, double* w) {
  if (!h || !v || !w) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  if (!h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "the factor of a device handle lives on the device");
  std::string err;
  const int st = filter_solve_host(h->c.F, v, w, err);
  return st ? fail(st, err) : AMGF_OK;
}

int amgf_filter_solve(amgf_handle h, const double* v_dev, double* w_dev, void* stream) {
  if (h && h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (!h || !v_dev || !w_dev) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  Ctx& c = h->c;
  if (c.F.nc == 0) return fail(AMGF_ERR_INVALID_ARG, "empty contact set");
  CK(cudaSetDevice(c.device));
  int st = join_begin(c, stream);
  if (st) return st;
  permute_kernel<<<vec_grid(c, c.F.nc), TPB, 0, c.s>>>(c.F.nc, nullptr, c.ficidx, v_dev, c.fv);
  enqueue_filter_solve(c, nullptr, c.fv);
  permute_kernel<<<vec_grid(c, c.F.nc), TPB, 0, c.s>>>(c.F.nc, c.ficidx, nullptr, c.fw, w_dev);
  return join_end(c, stream);
}

static int solve_device(Ctx& c, amgf_stats* stats) {
  // b and x already in c.b / c.x
  CK(cudaEventRecord(c.t0, c.s));
  if (c.o.use_graph) {
    if (!c.gexec) {
      int st = build_graph(c);
      if (st) return st;
    }
    CK(cudaGraphLaunch(c.gexec, c.s));
  } else {
    c.launches = 0;
    enqueue_pcg_init(c);
    c.init_launches = c.launches;
    for (int it = 0; it < c.o.maxit; ++it) {
      CK(cudaMemcpyAsync(c.st_host, c.st, sizeof(PcgState), cudaMemcpyDeviceToHost, c.s));
      CK(cudaStreamSynchronize(c.s));
      if (c.st_host->done) break;
      c.launches = 0;
      enqueue_pcg_body(c, 0);
      c.body_launches = c.launches;
    }
  }
  CK(cudaEventRecord(c.t1, c.s));
  // true residual of the returned iterate: q = b - A x (FP64), ||q||^2 and ||b||^2
  {
    CsrArgs ra{};
    ra.x = c.x; ra.b = c.b; ra.y = c.q;
    launch_csr<M_RESID>(c, c.L[0].A, ra);
    dot_kernel<<<vec_grid(c, c.n), TPB, 0, c.s>>>(c.n, c.q, c.q, c.partial, c.scratch_scalar + 2, c.counter);
    dot_kernel<<<vec_grid(c, c.n), TPB, 0, c.s>>>(c.n, c.b, c.b, c.partial, c.scratch_scalar + 3, c.counter);
  }
  CK(cudaMemcpyAsync(c.st_host, c.st, sizeof(PcgState), cudaMemcpyDeviceToHost, c.s));
  double res2[2] = {0.0, 0.0};
  CK(cudaMemcpyAsync(res2, c.scratch_scalar + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  int kerr = 0;
  if (c.kerr) CK(cudaMemcpyAsync(&kerr, c.kerr, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  CK(cudaStreamSynchronize(c.s));
  CK(cudaGetLastError());
  if (kerr) return fail(AMGF_ERR_CUDA, "staged coarse-level sweep: a shared-memory pipeline wait timed out");
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c.t0, c.t1));
  const PcgState& s = *c.st_host;
  if (stats) {
    stats->iters = s.iter;
    stats->converged = s.status == 0;
    stats->status = s.status;
    stats->nlevels = (int)c.L.size();
    stats->rel_res_precond = s.relres;
    stats->rz0 = s.rz0;
    stats->t_solve_s = ms * 1e-3;
    // kernels of the init part plus one body per executed loop trip (a body also runs once
    // when the initial residual already meets the stop test)
    const int64_t trips = s.iter > 0 ? s.iter : (c.o.use_graph ? 1 : 0);
    stats->kernel_launches = c.init_launches + trips * c.body_launches + 3;  // + the true-residual check
    stats->rel_res_l2 = res2[1] > 0.0 ? std::sqrt(res2[0] / res2[1]) : 0.0;
    stats->t_setup_s = c.info.t_setup_s;
  }
  if (s.status != 0) {
    static const char* names[] = {"ok", "invalid", "non-finite PCG scalar", "not SPD", "breakdown (p^T A p <= 0 or r^T z < 0)",
                                  "maximum iterations reached", "cuda", "oom"};
    return fail(s.status, std::string("pcg: ") + names[s.status < 8 && s.status >= 0 ? s.status : 1]);
  }
  return AMGF_OK;
}

int amgf_pcg_solve(amgf_handle h, const double* b_dev, double* x_dev, amgf_stats* stats, void* stream) {
  if (h && h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (!h || !b_dev || !x_dev) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  Ctx& c = h->c;
  CK(cudaSetDevice(c.device));
  int st = join_begin(c, stream);
  if (st) return st;
  CK(cudaMemcpyAsync(c.b, b_dev, c.n * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
  CK(cudaMemcpyAsync(c.x, x_dev, c.n * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
  int rs = solve_device(c, stats);
  if (rs == AMGF_ERR_CUDA || rs == AMGF_ERR_OOM) return rs;
  if (stats) stats->mlp_fallback = 0;
  if (rs != AMGF_OK && !c.mlp_w_host.empty()) {
    // learned weights failed to reach the stop test: solve again from x0 with theta = 1
    if ((st = apply_smoother_weights(c, true))) return st;
    CK(cudaMemcpyAsync(c.x, x_dev, c.n * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
    rs = solve_device(c, stats);
    if (stats) stats->mlp_fallback = 1;
    const int st2 = apply_smoother_weights(c, false);
    if (rs == AMGF_ERR_CUDA || rs == AMGF_ERR_OOM) return rs;
    if (st2) return st2;
  }
  CK(cudaMemcpyAsync(x_dev, c.x, c.n * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
  st = join_end(c, stream);
  return st ? st : rs;
}

int amgf_pcg_solve_host(amgf_handle h, const double* b_host, double* x_host, amgf_stats* stats) {
  if (h && h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (!h || !b_host || !x_host) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  Ctx& c = h->c;
  CK(cudaSetDevice(c.device));
  CK(cudaMemcpyAsync(c.b, b_host, c.n * sizeof(double), cudaMemcpyHostToDevice, c.s));
  CK(cudaMemcpyAsync(c.x, x_host, c.n * sizeof(double), cudaMemcpyHostToDevice, c.s));
  const int rs = solve_device(c, stats);
  if (rs == AMGF_ERR_CUDA || rs == AMGF_ERR_OOM) return rs;
  CK(cudaMemcpyAsync(x_host, c.x, c.n * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  CK(cudaStreamSynchronize(c.s));
  return rs;
}

int amgf_set_mlp(amgf_handle h, const float* weights, int64_t nw) {
  if (!h) return fail(AMGF_ERR_INVALID_ARG, "null handle");
  if (h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  Ctx& c = h->c;
  if (weights && nw != MLP_NW) return fail(AMGF_ERR_INVALID_ARG, "the smoother MLP has 1313 weights");
  if (weights && c.o.smoother != 0)
    return fail(AMGF_ERR_INVALID_ARG, "learned weights damp the l1-Jacobi smoother (options.smoother = 0)");
  if (weights)
    for (int64_t k = 0; k < nw; ++k)
      if (!std::isfinite(weights[k])) return fail(AMGF_ERR_NONFINITE, "non-finite MLP weight");
  CK(cudaSetDevice(c.device));
  if (weights) c.mlp_w_host.assign(weights, weights + nw);
  else c.mlp_w_host.clear();
  return apply_smoother_weights(c, false);
}

int amgf_mlp_train(amgf_handle h, float* params, float* adam_m, float* adam_v, int64_t* adam_step, int iters,
                   float lr, uint64_t seed, float* loss) {
  if (!h || !params || !adam_m || !adam_v || !adam_step || iters < 0 || !(lr > 0.f))
    return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  if (h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (h->c.mixed) return fail(AMGF_ERR_INVALID_ARG, "training runs on an FP64 handle (precision 0)");
  CK(cudaSetDevice(h->c.device));
  return mlp_train_impl(h->c, params, adam_m, adam_v, adam_step, iters, lr, seed, loss);
}

int amgf_mlp_grad(amgf_handle h, const float* params, const double* r_all, float* grad, double* loss) {
  if (!h || !params || !r_all || !grad) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  if (h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (h->c.mixed) return fail(AMGF_ERR_INVALID_ARG, "the training loss runs on an FP64 handle (precision 0)");
  CK(cudaSetDevice(h->c.device));
  return mlp_grad_impl(h->c, params, r_all, grad, loss);
}

int amgf_profile_iteration(amgf_handle h, void* stream, amgf_launch_rec* recs, int cap, int* count) {
  if (h && h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (!h || !count || cap < 0 || (cap > 0 && !recs)) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  Ctx& c = h->c;
  CK(cudaSetDevice(c.device));
  int st = join_begin(c, stream);
  if (st) return st;
  // a fresh PCG start from the current x (r0 = b - A x0, z0 = M r0), so that the iteration
  // below runs every kernel on live state (the vector kernels skip their work once the stop
  // test has been met)
  enqueue_pcg_init(c);
  std::vector<Ctx::ProfRec> v;
  cudaEvent_t e0 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventRecord(e0, c.s));
  c.prof = &v;
  enqueue_pcg_body(c, 0);
  c.prof = nullptr;
  const cudaError_t le = cudaGetLastError();
  const cudaError_t se = cudaStreamSynchronize(c.s);
  cudaEvent_t prev = e0;
  for (size_t k = 0; k < v.size(); ++k) {
    float ms = 0.f;
    if (le == cudaSuccess && se == cudaSuccess) cudaEventElapsedTime(&ms, prev, v[k].ev);
    if ((int)k < cap) {
      amgf_launch_rec& r = recs[k];
      std::memset(&r, 0, sizeof r);
      std::snprintf(r.op, sizeof r.op, "%s", v[k].op.c_str());
      r.level = v[k].level;
      r.ms = ms;
      r.bytes = v[k].bytes;
      r.flops = v[k].flops;
    }
    prev = v[k].ev;
  }
  for (auto& r : v) cudaEventDestroy(r.ev);
  cudaEventDestroy(e0);
  if (le != cudaSuccess) return fail(AMGF_ERR_CUDA, std::string("profile: ") + cudaGetErrorString(le));
  if (se != cudaSuccess) return fail(AMGF_ERR_CUDA, std::string("profile: ") + cudaGetErrorString(se));
  *count = (int)v.size();
  return join_end(c, stream);
}

int amgf_get_info(amgf_handle h, amgf_info* info) {
  if (!h || !info) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  *info = h->c.info;
  return AMGF_OK;
}

int amgf_export_matrix(amgf_handle h, int which, int level, int64_t* nrows, int64_t* ncols, int64_t* nnz,
                       int64_t* row_ptr, int32_t* col_idx, double* val) {
  if (!h || !nrows || !ncols || !nnz) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  const Hierarchy& H = h->c.H;
  const HCSR* a = nullptr;
  if (which == 0 && level >= 0 && level < H.nlev()) a = &H.A[level];
  else if (which == 1 && level >= 0 && level + 1 < H.nlev()) a = &H.P[level];
  else if (which == 2 && level >= 0 && level + 1 < H.nlev()) a = &H.R[level];
  if (!a) return fail(AMGF_ERR_INVALID_ARG, "no such matrix");
  *nrows = a->nrows; *ncols = a->ncols; *nnz = a->nnz();
  if (row_ptr) std::memcpy(row_ptr, a->rp.data(), (a->nrows + 1) * sizeof(int64_t));
  if (col_idx) std::memcpy(col_idx, a->ci.data(), a->nnz() * sizeof(int32_t));
  if (val) std::memcpy(val, a->v.data(), a->nnz() * sizeof(double));
  return AMGF_OK;
}

int amgf_export_contact_set(amgf_handle h, int64_t* ic) {
  if (!h || !ic) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  std::memcpy(ic, h->c.F.ic.data(), h->c.F.nc * sizeof(int64_t));
  return AMGF_OK;
}

int amgf_time_kernel(amgf_handle h, int which, int warmup, int reps, void* stream, double* ms, double* bytes) {
  if (h && h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  if (!h || !ms || !bytes || reps < 1 || warmup < 0 || which < 0 || which > 3)
    return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  if (which == 2 && !h->c.mixed) return fail(AMGF_ERR_INVALID_ARG, "which = 2 needs a mixed-precision handle");
  if (which == 3 && h->c.L.size() < 3) return fail(AMGF_ERR_INVALID_ARG, "which = 3 needs >= 3 levels");
  Ctx& c = h->c;
  CK(cudaSetDevice(c.device));
  int st = join_begin(c, stream);
  if (st) return st;
  DLevel& l0 = c.L[0];
  const double nnz = (double)l0.A.nnz, n = (double)l0.n;
  auto launch = [&]() {
    if (which == 3) {  // level-1 post-smoother in the V-cycle's precision
      DLevel& l1 = c.L[1];
      if (c.mixed) {
        CsrArgsT<float> a{};
        a.x = l1.xf; a.b = l1.rhsf; a.winv = l1.winvf; a.y = l1.outf;
        launch_csr_f<M_POST>(c, l1.Af, a);
      } else {
        CsrArgs a{};
        a.x = l1.x; a.b = l1.rhs; a.winv = l1.winv; a.y = l1.out;
        launch_csr<M_POST>(c, l1.A, a);
      }
    } else if (which == 2) {
      launch_fine_mixed<M_POST>(c, l0.xf, l0.rhsf, l0.winvf, nullptr, nullptr, c.q, nullptr, nullptr);
    } else if (which == 0) {
      CsrArgs a{};
      a.x = c.p; a.y = c.q;
      launch_csr<M_SPMV>(c, l0.A, a);
    } else {
      CsrArgs a{};
      a.x = c.p; a.b = c.r; a.winv = l0.winv; a.y = c.q;
      launch_csr<M_POST>(c, l0.A, a);
    }
  };
  for (int i = 0; i < warmup; ++i) launch();
  CK(cudaEventRecord(c.t0, c.s));
  for (int i = 0; i < reps; ++i) launch();
  CK(cudaEventRecord(c.t1, c.s));
  CK(cudaEventSynchronize(c.t1));
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, c.t0, c.t1));
  *ms = t / reps;
  if (c.kerr) {
    int kerr = 0;
    CK(cudaMemcpy(&kerr, c.kerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (kerr) return fail(AMGF_ERR_CUDA, "staged coarse-level sweep: a shared-memory pipeline wait timed out");
  }
  // values (8 B) + column indices (4 B) per nonzero, row pointers, and each vector read/written once
  const double vec_bytes = which == 0 ? 2.0 * 8.0 * n : 4.0 * 8.0 * n;
  if (which == 3) {  // values (8, 4 or 2 B) + 4 B column per nonzero, row pointers, x, b, W, y
    const DLevel& l1 = c.L[1];
    const double vb = c.mixed ? (l1.Af.vb ? 2.0 : 4.0) : 8.0, eb = c.mixed ? 4.0 : 8.0;
    const double nz1 = (double)(c.mixed ? l1.Af.nnz : l1.A.nnz), n1 = (double)l1.n;
    *bytes = nz1 * (vb + 4.0) + (n1 + 1.0) * 8.0 + 4.0 * eb * n1;
  } else if (which == 2) {  // K blocks (4 or 2 bytes per value + index), contact CSR (row pointers, 4 + 8 B
                            // per entry), 3 FP32 reads + FP64 write
    const double vb = c.k_bf16 ? 2.0 : 4.0;
    *bytes = (double)c.k_nblocks * (9.0 * vb + 4.0) + (double)(c.k_nslices + 1) * 8.0 + (n + 1) * 4.0 +
             (double)c.c_nnz * 12.0 + 3.0 * 4.0 * n + 8.0 * n;
  } else if (l0.A.bsr)  // 9 values + one block column index per stored block (padding excluded), slice offsets
    *bytes = (double)l0.A.nblocks * (9.0 * 8.0 + 4.0) + (double)(l0.A.nslices + 1) * 8.0 + vec_bytes;
  else
    *bytes = nnz * 12.0 + (n + 1) * 8.0 + vec_bytes;
  return join_end(c, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Filter solve without library-owned work vectors.
//
// For callers that must not allocate device memory themselves or through this library
// while they run -- for example because another allocator owns the whole device, or
// because a cudaMalloc (and the device synchronisation it can imply) is not allowed in
// their loop.  The four work vectors of the filter solve live in one fixed-size array
// compiled into this library instead of in memory the handle allocated.  The array is
// shared by every call on a device and keeps the previous call's contents; every entry a
// call reads is first written by that same call, so nothing has to start at zero.

namespace {
constexpr int64_t kNoAllocScratchDoubles = 524288;  // 4 MiB: four vectors of up to 131072 doubles
static __device__ __align__(256) double g_filter_scratch[kNoAllocScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_ptr[64] = {nullptr};  // device address of g_filter_scratch, per device ordinal

// Looks up the device address of the scratch array once per device, with that device current.
int scratch_for_device(int dev, double** out) {
  if (dev < 0 || dev >= 64) return fail(AMGF_ERR_CUDA, "device ordinal out of range for the scratch table");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_filter_scratch);
    if (e != cudaSuccess) return fail(AMGF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return AMGF_OK;
}
}  // namespace

extern "C" int amgf_filter_solve_noalloc(amgf_handle h, const double* v_dev, double* w_dev, void* stream) {
  if (!h || !v_dev || !w_dev) return fail(AMGF_ERR_INVALID_ARG, "bad arguments");
  if (h->c.host_only) return fail(AMGF_ERR_INVALID_ARG, "host-only handle (amgf_setup_host)");
  Ctx& c = h->c;
  if (c.F.nc == 0) return fail(AMGF_ERR_INVALID_ARG, "empty contact set");
  const int64_t len = c.F.nb * c.F.nblk;
  if (4 * len > kNoAllocScratchDoubles) {
    char buf[200];
    snprintf(buf, sizeof buf, "filter too large for the fixed scratch: needs 4 x %lld doubles, limit %lld",
             (long long)len, (long long)kNoAllocScratchDoubles);
    return fail(AMGF_ERR_INVALID_ARG, buf);
  }
  CK(cudaSetDevice(c.device));
  double* scratch = nullptr;
  int st = scratch_for_device(c.device, &scratch);
  if (st) return st;
  double* v = scratch;
  double* y = scratch + len;
  double* z = scratch + 2 * len;
  double* w = scratch + 3 * len;
  st = join_begin(c, stream);
  if (st) return st;
  permute_kernel<<<vec_grid(c, c.F.nc), TPB, 0, c.s>>>(c.F.nc, nullptr, c.ficidx, v_dev, v);
  enqueue_filter_solve_into(c, nullptr, v, y, z, w);
  permute_kernel<<<vec_grid(c, c.F.nc), TPB, 0, c.s>>>(c.F.nc, c.ficidx, nullptr, w, w_dev);
  return join_end(c, stream);
}
