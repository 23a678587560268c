// CUDA kernels of the AMGF solve phase (sm_103a).
//
// Everything here is bandwidth- or latency-bound sparse/vector work:
//   - csr_kernel<K, MODE, DOT>: one group of K lanes per row (K = 2..32), coalesced
//     loads of the row's values and column indices, shuffle reduction.  The epilogue
//     fuses what the V-cycle and PCG need around each A x:
//       SPMV      y = A x
//       SPMV_ADD  y += A x                         (prolongation x_l += P_l e_{l+1})
//       RESID     y = b - A x                      (r1 = r - A y1, residual sweeps)
//       PRE       x = W b ; y = b - A W b          (l1-Jacobi from zero + residual)
//       POST      y = x + W (b - A x) [+ add]      (l1-Jacobi sweep; z = y2 + B r2)
//     with W = diag(1 / l1), and optionally a deterministic dot product of the output
//     with another vector (p^T A p, r^T z) finished by the last block to arrive.
//   - csr_staged_kernel<MODE, VT, K, U>: the same sweeps (RESID, POST) for the BF16 coarse
//     levels of the mixed V-cycle, with each tile of rows streamed into shared memory by a
//     producer warp (cp.async.bulk + mbarrier) ahead of the consumer warps' gathers.
//   - dense_gemv / dense_rows: coarsest-level solve with the host-computed inverse.
//   - filter_bcr: one phase of the odd-even block cyclic reduction solve of the
//     block-tridiagonal A_w (Section 5.1 filter step): all block GEMVs of a reduction
//     level at once over the whole GPU.
//   - filter_sweep / filter_diag: the alternative sequential block LDL^T sweeps, run by
//     one thread-block cluster that keeps the running block vector in distributed
//     shared memory; filter_diag applies the block pivots in parallel.
//   - PCG scalar/vector kernels with device-resident scalars.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "setup.h"

namespace amgf {

constexpr int TPB = 256;          // threads per block of the row kernels
constexpr int MAX_DOT_BLOCKS = 4096;

// Epilogues around s = (A x)_i:
//   SPMV    y = s                      SPMV_W  y = s, y2 = w2 * s (restriction: coarse rhs and W_c rhs)
//   SPMV_ADD y += s                    RESID   y = b - s
//   RESID_W y = b - s, y2 = w2 * y     POST    y = x + w (b - s) [+ add]
enum : int { M_SPMV = 0, M_SPMV_ADD = 1, M_RESID = 2, M_RESID_W = 3, M_POST = 4, M_SPMV_W = 5 };

template <typename T, typename VT = T>
struct CsrArgsT {
  const int64_t* __restrict__ rp;
  const int32_t* __restrict__ ci;
  const VT* __restrict__ v;  // stored values (VT = T, or BF16 for an FP32 V-cycle)
  int64_t nrows;
  const int64_t* __restrict__ rows;  // optional row indirection (output row = rows[i])
  const T* x;           // gathered vector
  const T* b;           // right-hand side (RESID, POST)
  const T* winv;        // 1 / l1 of the rows (POST)
  const T* w2;          // scaling of the second output (RESID_W, SPMV_W)
  const T* add;         // POST: optional vector added to the output
  T* y;                 // output
  T* y2;                // RESID_W, SPMV_W: second output w2 * y (may be null)
  float* yf;            // optional FP32 copy of y (precision boundary into an FP32 V-cycle)
  float* y2f;           // optional FP32 copy of w2 * y
  const T* dotv;        // DOT: partner vector of the output
  double* partial;      // DOT: one partial per block
  double* result;       // DOT: final scalar
  unsigned* counter;    // DOT: arrival counter (zero between launches)
};
using CsrArgs = CsrArgsT<double>;

struct PcgState {
  double rz;       // r_k^T z_k
  double rz0;      // r_0^T z_0
  double rz_new;   // written by the preconditioner's last kernel
  double pq;       // p^T A p
  double relres;   // sqrt(rz / rz0)
  double rtol;
  double rz_cross; // r_{k+1}^T z_k (flexible PCG)
  int iter;
  int maxit;
  int done;
  int status;
  int flexible;    // 1: beta = (r+^T z+ - r+^T z) / r^T z  (Polak-Ribiere; inexact preconditioner)
};

__device__ __forceinline__ double warp_sum(double s) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// Deterministic grid reduction: block partial -> partial[blockIdx.x]; the last block to
// arrive sums the partials in index order and writes *result.
__device__ __forceinline__ void grid_dot_finish(double local, double* partial, double* result, unsigned* counter) {
  __shared__ double red[TPB / 32];
  __shared__ bool last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  local = warp_sum(local);
  if (lane == 0) red[warp] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(partial + i);
  s = warp_sum(s);
  __syncthreads();
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *result = t;
    *counter = 0u;
  }
}

__device__ __forceinline__ double load_val(const double* p) { return __ldg(p); }
__device__ __forceinline__ float load_val(const float* p) { return __ldg(p); }
__device__ __forceinline__ float load_val(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T, int K, int MODE, bool DOT, typename VT = T, int U = 4>
__global__ void __launch_bounds__(TPB) csr_kernel(CsrArgsT<T, VT> a) {
  static_assert(K >= 1 && K <= 32 && (K & (K - 1)) == 0, "K must be a power of two <= 32");
  const int lane_w = threadIdx.x & 31;
  const int sub = lane_w & (K - 1);
  const int64_t gid = ((int64_t)blockIdx.x * TPB + threadIdx.x) / K;
  const int64_t warp_first = gid - (lane_w / K);
  const int64_t stride = (int64_t)gridDim.x * (TPB / K);
  double dacc = 0.0;
  for (int64_t base = warp_first; base < a.nrows; base += stride) {
    const int64_t i = base + lane_w / K;
    const bool valid = i < a.nrows;
    T s = T(0);
    if (valid) {
      const int64_t k1 = a.rp[i + 1];
      // batches of U entries per lane: all index/value loads of a batch are issued before
      // the dependent gathers, so each batch costs two memory round trips
      for (int64_t kb = a.rp[i] + sub; kb < k1; kb += U * K) {
        int32_t jj[U];
        T vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t k = kb + (int64_t)u * K;
          const bool ok = k < k1;
          jj[u] = ok ? __ldg(a.ci + k) : -1;
          vv[u] = ok ? (T)load_val(a.v + k) : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (jj[u] >= 0) s += vv[u] * __ldg(a.x + jj[u]);
      }
    }
#pragma unroll
    for (int off = K / 2; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off, K);
    if (valid && sub == 0) {
      const int64_t o = a.rows ? a.rows[i] : i;
      T out;
      if (MODE == M_SPMV || MODE == M_SPMV_W) out = s;
      else if (MODE == M_SPMV_ADD) out = a.y[o] + s;
      else if (MODE == M_RESID || MODE == M_RESID_W) out = a.b[o] - s;
      else { out = a.x[o] + a.winv[o] * (a.b[o] - s); if (a.add) out += a.add[o]; }
      a.y[o] = out;
      if (MODE == M_RESID_W || MODE == M_SPMV_W) {
        const T w = a.w2[o] * out;
        if (a.y2) a.y2[o] = w;
        if (a.y2f) a.y2f[o] = (float)w;
      }
      if (a.yf) a.yf[o] = (float)out;
      if (DOT) dacc += (double)a.dotv[o] * (double)out;
    }
  }
  if (DOT) grid_dot_finish(dacc, a.partial, a.result, a.counter);
}

// ---------------- FP64 level operators in sliced ELL, one lane per row ----------------
//
// On this GPU a FP64 warp instruction costs a pipe slot whether 1 or 32 lanes are active, so
// the FP64 sweeps of the long-row coarse levels lose slots in csr_kernel to rows of different
// length sharing a warp, partial batches and the shuffle reduction.  Here each lane owns one
// row of a slice of 32 rows sorted by length (SELL, see setup.h), walks it with one FMA per
// entry in CSR order (4 entries' loads in flight at a time), and runs the epilogue itself;
// every warp load of values or columns is one contiguous 256- or 128-byte segment.  The same
// form serves the short-row interpolation and restriction operators of the large levels, where
// it replaces csr_kernel's chain of dependent loads (row pointers, then entries, then x).
template <typename T, typename VT>
struct SellArgsT {
  const int64_t* __restrict__ soff;
  const int32_t* __restrict__ perm;  // sorted row -> row of A
  const int32_t* __restrict__ ci;
  const VT* __restrict__ v;          // stored values (FP64, FP32 or BF16)
  int64_t nrows, nslices;
  const T* x;
  const T* b;
  const T* winv;
  const T* w2;
  const T* add;
  T* y;
  T* y2;
};
using SellArgs = SellArgsT<double, double>;

__device__ __forceinline__ double sell_val(const double* p) { return __ldg(p); }
__device__ __forceinline__ float sell_val(const float* p) { return __ldg(p); }
__device__ __forceinline__ float sell_val(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

// MODE: M_SPMV (y = A x), M_SPMV_ADD (y += A x, prolongation), M_SPMV_W (y = A x, y2 = w2 y,
// restriction), M_RESID (y = b - A x) or M_POST (y = x + W (b - A x) [+ add]).  T: vectors and
// arithmetic (FP64, or FP32 in the mixed V-cycle); VT: stored values.
template <typename T, typename VT, int MODE>
__global__ void __launch_bounds__(TPB) sell_kernel(SellArgsT<T, VT> a) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * TPB + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * TPB) >> 5;
  for (int64_t s = w0; s < a.nslices; s += nw) {
    const int64_t s0 = __ldg(a.soff + s), w = (__ldg(a.soff + s + 1) - s0) >> 5;
    const int32_t* cp = a.ci + s0 + lane;
    const VT* vp = a.v + s0 + lane;
    T acc = T(0);
    int64_t j = 0;
    for (; j + 4 <= w; j += 4) {
      const int32_t c0 = __ldg(cp), c1 = __ldg(cp + 32), c2 = __ldg(cp + 64), c3 = __ldg(cp + 96);
      const T v0 = sell_val(vp), v1 = sell_val(vp + 32), v2 = sell_val(vp + 64), v3 = sell_val(vp + 96);
      const T x0 = __ldg(a.x + c0), x1 = __ldg(a.x + c1), x2 = __ldg(a.x + c2), x3 = __ldg(a.x + c3);
      acc = fma(v0, x0, acc);
      acc = fma(v1, x1, acc);
      acc = fma(v2, x2, acc);
      acc = fma(v3, x3, acc);
      cp += 128;
      vp += 128;
    }
    for (; j < w; ++j) {
      acc = fma((T)sell_val(vp), __ldg(a.x + __ldg(cp)), acc);
      cp += 32;
      vp += 32;
    }
    const int64_t q = s * 32 + lane;
    if (q < a.nrows) {
      const int64_t o = __ldg(a.perm + q);
      T out;
      if (MODE == M_SPMV || MODE == M_SPMV_W) out = acc;
      else if (MODE == M_SPMV_ADD) out = a.y[o] + acc;
      else if (MODE == M_RESID) out = a.b[o] - acc;
      else { out = a.x[o] + a.winv[o] * (a.b[o] - acc); if (a.add) out += a.add[o]; }
      a.y[o] = out;
      if (MODE == M_SPMV_W && a.y2) a.y2[o] = a.w2[o] * out;
    }
  }
}

// ---------------- staged CSR sweeps of the FP32 V-cycle's coarse levels ----------------
//
// The coarse-level sweeps of the mixed-precision V-cycle (r = b - A x and the l1-Jacobi
// post-smoother x + W (b - A x)) stream each row's column indices and values once and gather
// x at those columns.  In csr_kernel every warp alternates between the two kinds of load, so
// only part of the resident warps keep DRAM requests in flight.  Here one producer warp per
// CTA streams whole tiles of consecutive rows (their row pointers, column indices, values and
// the epilogue's b, x, W segments) into shared memory with bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier), STAGE_DEPTH tiles ahead, while eight
// consumer warps read the staged tile and issue only the gathers of x.  A lane sums the same
// entries in the same order as csr_kernel with the same K, so both give identical results.
//
// Bulk copies start on 16-byte boundaries: each staged segment starts at the aligned index
// at or below the first one the tile needs and is padded to whole 16-byte chunks; the device
// arrays carry that padding (row pointers +2 entries, indices and values +16, vectors +8).

constexpr int STAGE_NW = 8;                       // consumer warps per CTA
constexpr int STAGE_TPB = (STAGE_NW + 1) * 32;    // + one producer warp
constexpr int STAGE_MAX_DEPTH = 8;
constexpr uint64_t STAGE_WAIT_NS = 4000000000ull; // a wait that has not completed in 4 s gives up

struct StageArgs {
  int64_t ntiles;
  int rows;       // rows per tile
  int depth;      // tiles in flight per CTA (<= STAGE_MAX_DEPTH)
  int cap;        // staged index/value entries per tile (multiple of 8)
  int rp_cap;     // staged row pointers per tile (even)
  int vec_cap;    // staged entries of each epilogue vector per tile (multiple of 4)
  int* err;       // set to 1 when a wait gave up (the host reports AMGF_ERR_CUDA)
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait for the phase of parity `parity` to complete; false when it has not after
// STAGE_WAIT_NS (or 2^26 polls), so no wait can hang the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1; it < (1u << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0u && global_ns() - t0 > STAGE_WAIT_NS) break;
  }
  return false;
}
// bulk asynchronous copy global -> this CTA's shared memory, completion counted on `bar`
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Byte layout of one stage: row pointers, column indices, values, then the epilogue vectors
// (b for RESID; b, x, W for POST).  Every part is a multiple of 16 bytes.
template <int MODE, typename VT>
struct StageLayout {
  static constexpr int nvec = MODE == M_POST ? 3 : 1;
  __host__ __device__ static size_t bytes(int rp_cap, int cap, int vec_cap) {
    return (size_t)rp_cap * 8 + (size_t)cap * (4 + sizeof(VT)) + (size_t)nvec * vec_cap * 4;
  }
};
template <int MODE, typename VT>
inline size_t stage_smem_bytes(const StageArgs& g) {
  return 2 * STAGE_MAX_DEPTH * sizeof(uint64_t) + (size_t)g.depth * StageLayout<MODE, VT>::bytes(g.rp_cap, g.cap, g.vec_cap);
}

// MODE: M_RESID (y = b - A x) or M_POST (y = x + W (b - A x)); FP32 vectors, VT values.
template <int MODE, typename VT, int K, int U>
__global__ void __launch_bounds__(STAGE_TPB) csr_staged_kernel(CsrArgsT<float, VT> a, StageArgs g) {
  static_assert(MODE == M_RESID || MODE == M_POST, "staged modes");
  static_assert(K >= 2 && K <= 32 && (K & (K - 1)) == 0, "K must be a power of two <= 32");
  extern __shared__ __align__(16) unsigned char stage_smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(stage_smem);
  uint64_t* empty = full + STAGE_MAX_DEPTH;
  unsigned char* stages = stage_smem + 2 * STAGE_MAX_DEPTH * sizeof(uint64_t);
  const size_t sbytes = StageLayout<MODE, VT>::bytes(g.rp_cap, g.cap, g.vec_cap);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int depth = g.depth;
  if (threadIdx.x == 0) {
    for (int s = 0; s < depth; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, STAGE_NW);
    }
    mbar_init_fence();
  }
  __syncthreads();

  auto stage_ptrs = [&](int s, int64_t*& rps, int32_t*& cis, VT*& vs, float*& bs, float*& xs, float*& ws) {
    unsigned char* p = stages + (size_t)s * sbytes;
    rps = reinterpret_cast<int64_t*>(p);
    p += (size_t)g.rp_cap * 8;
    cis = reinterpret_cast<int32_t*>(p);
    p += (size_t)g.cap * 4;
    vs = reinterpret_cast<VT*>(p);
    p += (size_t)g.cap * sizeof(VT);
    bs = reinterpret_cast<float*>(p);
    xs = bs + g.vec_cap;
    ws = xs + g.vec_cap;
  };

  if (warp == STAGE_NW) {
    // producer: one lane issues the copies of this CTA's tiles, `depth` ahead of the consumers
    if (lane != 0) return;
    int64_t issued = 0;
    // the next tile's nonzero range is loaded one tile ahead, so its latency overlaps the wait
    // for a free stage
    auto tile_rows = [&](int64_t t, int64_t& r0, int64_t& r1) {
      r0 = t * g.rows;
      r1 = r0 + g.rows < a.nrows ? r0 + g.rows : a.nrows;
    };
    int64_t k0n = 0, k1n = 0;
    if ((int64_t)blockIdx.x < g.ntiles) {
      int64_t r0, r1;
      tile_rows(blockIdx.x, r0, r1);
      k0n = __ldg(a.rp + r0);
      k1n = __ldg(a.rp + r1);
    }
    for (int64_t j = 0;; ++j) {
      const int64_t t = blockIdx.x + j * gridDim.x;
      if (t >= g.ntiles) break;
      const int64_t k0 = k0n, k1 = k1n;
      if (t + gridDim.x < g.ntiles) {
        int64_t r0n, r1n;
        tile_rows(t + gridDim.x, r0n, r1n);
        k0n = __ldg(a.rp + r0n);
        k1n = __ldg(a.rp + r1n);
      }
      const int s = (int)(j % depth);
      const int64_t q = j / depth;
      if (q > 0 && !mbar_wait_bounded(empty + s, (uint32_t)((q - 1) & 1))) {
        atomicExch(g.err, 1);
        break;
      }
      int64_t r0, r1;
      tile_rows(t, r0, r1);
      const int64_t ka = k0 & ~(int64_t)7;
      const int64_t kn = (k1 - ka + 7) & ~(int64_t)7;
      const int64_t ra = r0 & ~(int64_t)1;
      const int64_t rn = (r1 + 1 - ra + 1) & ~(int64_t)1;
      const int64_t va = r0 & ~(int64_t)3;
      const int64_t vn = (r1 - va + 3) & ~(int64_t)3;
      const int nvec = StageLayout<MODE, VT>::nvec;
      const uint32_t bytes = (uint32_t)(rn * 8 + kn * (4 + (int64_t)sizeof(VT)) + nvec * vn * 4);
      int64_t* rps; int32_t* cis; VT* vs; float *bs, *xs, *ws;
      stage_ptrs(s, rps, cis, vs, bs, xs, ws);
      mbar_arrive_expect_tx(full + s, bytes);
      bulk_to_smem(rps, a.rp + ra, (uint32_t)(rn * 8), full + s);
      if (kn > 0) {
        bulk_to_smem(cis, a.ci + ka, (uint32_t)(kn * 4), full + s);
        bulk_to_smem(vs, a.v + ka, (uint32_t)(kn * sizeof(VT)), full + s);
      }
      bulk_to_smem(bs, a.b + va, (uint32_t)(vn * 4), full + s);
      if (MODE == M_POST) {
        bulk_to_smem(xs, a.x + va, (uint32_t)(vn * 4), full + s);
        bulk_to_smem(ws, a.winv + va, (uint32_t)(vn * 4), full + s);
      }
      ++issued;
    }
    // no copy may still be landing in this CTA's shared memory when it exits: wait for the
    // last phase issued into every stage
    for (int s = 0; s < depth; ++s) {
      const int64_t n_s = issued > s ? (issued - 1 - s) / depth + 1 : 0;  // issues into stage s
      if (n_s > 0 && !mbar_wait_bounded(full + s, (uint32_t)((n_s - 1) & 1))) atomicExch(g.err, 1);
    }
    return;
  }

  // consumers: K lanes per row, rows of a tile spread over the eight warps
  const int sub = lane & (K - 1);
  constexpr int G = STAGE_NW * (32 / K);  // row groups per CTA
  for (int64_t j = 0;; ++j) {
    const int64_t t = blockIdx.x + j * gridDim.x;
    if (t >= g.ntiles) break;
    const int s = (int)(j % depth);
    if (!mbar_wait_bounded(full + s, (uint32_t)((j / depth) & 1))) {
      if (lane == 0) atomicExch(g.err, 1);
      break;
    }
    int64_t* rps; int32_t* cis; VT* vs; float *bs, *xs, *ws;
    stage_ptrs(s, rps, cis, vs, bs, xs, ws);
    const int64_t r0 = t * g.rows;
    const int nr = (int)(r0 + g.rows < a.nrows ? g.rows : a.nrows - r0);
    const int roff = (int)(r0 & 1), voff = (int)(r0 & 3);
    const int64_t ka = rps[roff] & ~(int64_t)7;
    for (int base = warp * (32 / K); base < nr; base += G) {
      const int rr = base + lane / K;
      const bool valid = rr < nr;
      float sum = 0.f;
      if (valid) {
        const int ke = (int)(rps[roff + rr + 1] - ka);
        for (int kb = (int)(rps[roff + rr] - ka) + sub; kb < ke; kb += U * K) {
          int32_t jj[U];
          float vv[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int k = kb + u * K;
            const bool ok = k < ke;
            jj[u] = ok ? cis[k] : -1;
            vv[u] = ok ? to_float(vs[k]) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (jj[u] >= 0) sum += vv[u] * __ldg(a.x + jj[u]);
        }
      }
#pragma unroll
      for (int off = K / 2; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off, K);
      if (valid && sub == 0) {
        const int vi = voff + rr;
        float out;
        if (MODE == M_RESID) out = bs[vi] - sum;
        else out = xs[vi] + ws[vi] * (bs[vi] - sum);
        a.y[r0 + rr] = out;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + s);
  }
}

// Fine-level operator in 3x3 node blocks (BSR3, slices of 32 block rows; see setup.h):
// one warp per slice, one lane per block row I, which owns rows 3I..3I+2.  Every load of
// block values or block columns is one contiguous segment per warp, the slice's blocks are
// walked in lockstep (no divergence, no shuffles), and each nonzero costs exactly one FP64
// FMA.  Same epilogues as csr_kernel (SPMV, RESID, RESID_W, POST, optional dot).
struct BsrArgs {
  const int64_t* __restrict__ soff;
  const int32_t* __restrict__ bci;
  const double* __restrict__ v;
  int64_t nbrows, nslices;
  const double* x;
  const double* b;
  const double* winv;
  const double* w2;
  const double* add;
  double* y;
  double* y2;
  float* yf;
  float* y2f;
  const double* dotv;
  double* partial;
  double* result;
  unsigned* counter;
};

template <int MODE, bool DOT>
__global__ void __launch_bounds__(TPB) bsr3_kernel(BsrArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * TPB + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * TPB) >> 5;
  double dacc = 0.0;
  for (int64_t sl = warp0; sl < a.nslices; sl += nwarp) {
    const int64_t s0 = a.soff[sl];
    const int64_t w = (a.soff[sl + 1] - s0) >> 5;
    const int32_t* ci = a.bci + s0 + lane;
    const double* vb = a.v + 9 * s0 + lane;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    auto block = [&](const double* m, int64_t J) {
      const double x0 = __ldg(a.x + 3 * J), x1 = __ldg(a.x + 3 * J + 1), x2 = __ldg(a.x + 3 * J + 2);
      a0 = fma(m[0], x0, a0); a0 = fma(m[1], x1, a0); a0 = fma(m[2], x2, a0);
      a1 = fma(m[3], x0, a1); a1 = fma(m[4], x1, a1); a1 = fma(m[5], x2, a1);
      a2 = fma(m[6], x0, a2); a2 = fma(m[7], x1, a2); a2 = fma(m[8], x2, a2);
    };
    int64_t j = 0;
    // A p with its dot product: two blocks' values loaded together; the other epilogues one block
    // at a time, unrolled by 4.  Each form was the faster one for its epilogue on GB300 at c160
    // (A p 1875 -> 1740 us, post-smoother 1935 -> 1783 us, r1 = r - A y1 1942 -> 1762 us against
    // the earlier single loop unrolled by 2); the FMAs run in the same order in every form.
    if (DOT) {
      for (; j + 1 < w; j += 2) {
        const int64_t J0 = __ldg(ci + 32 * j), J1 = __ldg(ci + 32 * j + 32);
        const double* p = vb + 288 * j;
        double m[18];
#pragma unroll
        for (int q = 0; q < 18; ++q) m[q] = __ldg(p + 32 * q);
        block(m, J0);
        block(m + 9, J1);
      }
    }
#pragma unroll 4
    for (; j < w; ++j) {
      const int64_t J = __ldg(ci + 32 * j);
      const double* p = vb + 288 * j;
      double m[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) m[q] = __ldg(p + 32 * q);
      block(m, J);
    }
    const int64_t I = sl * 32 + lane;
    if (I < a.nbrows) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {  // rows 3I + c
        const double s = c == 0 ? a0 : (c == 1 ? a1 : a2);
        const int64_t o = 3 * I + c;
        double out;
        if (MODE == M_SPMV || MODE == M_SPMV_W) out = s;
        else if (MODE == M_SPMV_ADD) out = a.y[o] + s;
        else if (MODE == M_RESID || MODE == M_RESID_W) out = a.b[o] - s;
        else { out = a.x[o] + a.winv[o] * (a.b[o] - s); if (a.add) out += a.add[o]; }
        a.y[o] = out;
        if (MODE == M_RESID_W || MODE == M_SPMV_W) {
          const double wv = a.w2[o] * out;
          if (a.y2) a.y2[o] = wv;
          if (a.y2f) a.y2f[o] = (float)wv;
        }
        if (a.yf) a.yf[o] = (float)out;
        if (DOT) dacc += a.dotv[o] * out;
      }
    }
  }
  if (DOT) grid_dot_finish(dacc, a.partial, a.result, a.counter);
}

// Fine level of the FP32 V-cycle: K in 3x3 node blocks with FP32 or BF16 values (same sliced
// layout as bsr3_kernel), FP32 vectors and accumulation, plus the contact term
// J^T D J (entries up to D_max) in FP64 from a CSR over all rows (mostly empty), so that
//   s_i = (K x)_i [FP32] + (J^T D J x)_i [FP64].
//   RESID: y32 = b - s                        (pre-smoothing residual, FP32)
//   POST : y64 = x + w (b - s) [+ add64]      (post-smoothing, written in FP64: the
//          V-cycle's output crosses back into the FP64 PCG here)
template <typename VT>
struct Bsr3MixedArgs {
  const int64_t* __restrict__ soff;
  const int32_t* __restrict__ bci;  // FP32 values: block columns, values by plane
  const VT* __restrict__ v;
  const uint2* __restrict__ pk;     // BF16 values: column and 9 values packed in 3 words per slot
  int64_t nbrows, nslices;
  const int32_t* __restrict__ crp;  // contact term rows (length n + 1)
  const int32_t* __restrict__ cci;
  const double* __restrict__ cv;
  const float* x;
  const float* b;
  const float* winv;
  const double* add;
  float* y32;
  double* y64;
  const double* dotv;
  double* partial;
  double* result;
  unsigned* counter;
};

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename VT, int MODE, bool DOT>
__global__ void __launch_bounds__(TPB) bsr3_mixed_kernel(Bsr3MixedArgs<VT> a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * TPB + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * TPB) >> 5;
  double dacc = 0.0;
  for (int64_t sl = warp0; sl < a.nslices; sl += nwarp) {
    const int64_t s0 = a.soff[sl];
    const int64_t w = (a.soff[sl + 1] - s0) >> 5;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    if constexpr (std::is_same<VT, __nv_bfloat16>::value) {
      // three coalesced 8-byte loads per slot (256 bytes per warp and load) instead of ten
      // 2- and 4-byte ones; a BF16 value widens to FP32 exactly by a 16-bit shift
      const uint2* pb = a.pk + 3 * s0 + lane;
#pragma unroll 4
      for (int64_t j = 0; j < w; ++j) {
        const uint2 w0 = __ldg(pb + 96 * j), w1 = __ldg(pb + 96 * j + 32), w2 = __ldg(pb + 96 * j + 64);
        const int64_t J = (int32_t)w0.x;
        const float x0 = __ldg(a.x + 3 * J), x1 = __ldg(a.x + 3 * J + 1), x2 = __ldg(a.x + 3 * J + 2);
        auto lo = [](uint32_t u) { return __uint_as_float(u << 16); };
        auto hi = [](uint32_t u) { return __uint_as_float(u & 0xffff0000u); };
        a0 = fmaf(lo(w0.y), x0, a0); a0 = fmaf(hi(w0.y), x1, a0); a0 = fmaf(lo(w1.x), x2, a0);
        a1 = fmaf(hi(w1.x), x0, a1); a1 = fmaf(lo(w1.y), x1, a1); a1 = fmaf(hi(w1.y), x2, a1);
        a2 = fmaf(lo(w2.x), x0, a2); a2 = fmaf(hi(w2.x), x1, a2); a2 = fmaf(lo(w2.y), x2, a2);
      }
    } else {
      const int32_t* ci = a.bci + s0 + lane;
      const VT* vb = a.v + 9 * s0 + lane;
#pragma unroll 2
      for (int64_t j = 0; j < w; ++j) {
        const int64_t J = __ldg(ci + 32 * j);
        const VT* p = vb + 288 * j;
        float m[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) m[q] = to_f32(p[32 * q]);
        const float x0 = __ldg(a.x + 3 * J), x1 = __ldg(a.x + 3 * J + 1), x2 = __ldg(a.x + 3 * J + 2);
        a0 = fmaf(m[0], x0, a0); a0 = fmaf(m[1], x1, a0); a0 = fmaf(m[2], x2, a0);
        a1 = fmaf(m[3], x0, a1); a1 = fmaf(m[4], x1, a1); a1 = fmaf(m[5], x2, a1);
        a2 = fmaf(m[6], x0, a2); a2 = fmaf(m[7], x1, a2); a2 = fmaf(m[8], x2, a2);
      }
    }
    const int64_t I = sl * 32 + lane;
    if (I < a.nbrows) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int64_t o = 3 * I + c;
        double s = (double)(c == 0 ? a0 : (c == 1 ? a1 : a2));
        for (int32_t k = a.crp[o]; k < a.crp[o + 1]; ++k) s += a.cv[k] * (double)a.x[a.cci[k]];
        if (MODE == M_RESID) {
          a.y32[o] = (float)((double)a.b[o] - s);
        } else {
          double out = (double)a.x[o] + (double)a.winv[o] * ((double)a.b[o] - s);
          if (a.add) out += a.add[o];
          a.y64[o] = out;
          if (DOT) dacc += a.dotv[o] * out;
        }
      }
    }
  }
  if (DOT) grid_dot_finish(dacc, a.partial, a.result, a.counter);
}

// Coarsest-level solve out = A_L^{-1} r with the host-computed dense inverse. A V-cycle
// with a single level needs the add and dot outputs: one CTA of DENSE_TPB threads, a warp
// per row (dense_gemv_kernel). Every other coarsest solve spreads its rows over the grid
// (dense_rows_kernel, FP64 or FP32).
constexpr int DENSE_TPB = 1024;

// Chebyshev smoother (three-term recurrence of Chebyshev acceleration for W A, W = 1/l1):
// each step follows a RESID pass res = b - A x and applies d = a d + bc W res, x += d (the
// first step of a sweep from a nonzero x: d = bc W res).  A sweep from zero starts from the
// producer's x = W b: cheb_init scales it to d = x = W b / c.  The last step of a
// post-smoothing writes out = x + d [+ add] to the level's output instead of updating x, with
// an optional dot product of the output.
template <typename T>
__global__ void cheb_init_kernel(int64_t n, T* x, T* d, T s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = x[i] * s;
    x[i] = v;
    d[i] = v;
  }
}

template <typename T, bool FIRST>
__global__ void cheb_step_kernel(int64_t n, const T* __restrict__ winv, const T* __restrict__ res, T* d, T* x, T a,
                                 T bc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = FIRST ? bc * (winv[i] * res[i]) : a * d[i] + bc * (winv[i] * res[i]);
    d[i] = v;
    x[i] += v;
  }
}

template <typename T, typename TO, bool FIRST, bool DOT>
__global__ void __launch_bounds__(TPB) cheb_out_kernel(int64_t n, const T* __restrict__ winv, const T* __restrict__ res,
                                                       const T* __restrict__ d, const T* __restrict__ x, T a, T bc,
                                                       const double* add, TO* out, const double* dotv,
                                                       double* partial, double* result, unsigned* counter) {
  double dacc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = FIRST ? bc * (winv[i] * res[i]) : a * d[i] + bc * (winv[i] * res[i]);
    double o = (double)(x[i] + v);
    if (add) o += add[i];
    out[i] = (TO)o;
    if (DOT) dacc += dotv[i] * o;
  }
  if (DOT) grid_dot_finish(dacc, partial, result, counter);
}

// out[idx[k]] = val[k] (values of an updated operator written into its device image)
template <typename T>
__global__ void scatter_kernel(int64_t n, const int64_t* __restrict__ idx, const T* __restrict__ val, T* out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[idx[k]] = val[k];
}

// x_i += W_i * res_i in FP32 (extra sweeps when nu > 1)
__global__ void axpy_w_f32_kernel(int64_t n, const float* __restrict__ winv, const float* __restrict__ res, float* x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += winv[i] * res[i];
}

// r32 = (float) r, x32 = (float)(W0 r): entry of an FP32 V-cycle from an FP64 vector
__global__ void to_f32_scaled_kernel(int64_t n, const double* __restrict__ w, const double* __restrict__ r,
                                     float* r32, float* x32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    r32[i] = (float)r[i];
    x32[i] = (float)(w[i] * r[i]);
  }
}

// y = W r elementwise (entry of a V-cycle whose rhs was not produced by a fused kernel)
__global__ void scale_kernel(int64_t n, const double* __restrict__ w, const double* __restrict__ r, double* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = w[i] * r[i];
}

// x_i += W_i * res_i (extra pre-smoothing sweeps when nu > 1)
__global__ void axpy_w_kernel(int64_t n, const double* __restrict__ winv, const double* __restrict__ res, double* x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += winv[i] * res[i];
}

// out = Ainv * r with the rows spread over the grid: a warp per row, grid-stride, the
// row's loads coalesced across the warp and summed by the same lane split and butterfly as
// dense_gemv_kernel (so both give the same bits). For coarsest levels of a few thousand
// rows, whose inverse (n^2 values) is too large for one CTA to stream quickly.
constexpr int DENSE_ROWS_TPB = 256;
template <typename T>
__global__ void __launch_bounds__(DENSE_ROWS_TPB) dense_rows_kernel(int64_t n, const T* __restrict__ Ainv,
                                                                    const T* __restrict__ r, T* out) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * DENSE_ROWS_TPB + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * DENSE_ROWS_TPB) >> 5;
  for (int64_t i = w0; i < n; i += nw) {
    const T* row = Ainv + i * n;
    T s = 0;
    for (int64_t k = lane; k < n; k += 32) s += row[k] * r[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[i] = s;
  }
}

// out = Ainv * r (+ add), Ainv dense n x n row-major; optional dot(dotv, out). One block.
__global__ void __launch_bounds__(DENSE_TPB) dense_gemv_kernel(int64_t n, const double* __restrict__ Ainv,
                                                               const double* __restrict__ r, const double* add,
                                                               double* out, const double* dotv, double* result) {
  __shared__ double red[DENSE_TPB / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double dacc = 0.0;
  for (int64_t i = warp; i < n; i += nw) {
    const double* row = Ainv + i * n;
    double s = 0.0;
    for (int64_t k = lane; k < n; k += 32) s += row[k] * r[k];
    s = warp_sum(s);
    if (add) s += add[i];
    if (lane == 0) { out[i] = s; if (dotv) dacc += dotv[i] * s; }
  }
  if (result) {
    dacc = warp_sum(dacc);
    if (lane == 0) red[warp] = dacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[w];
      *result = t;
    }
  }
}

// ---------------- filter: A_w^{-1} of the block-tridiagonal A_w ----------------

constexpr int FILTER_TPB = 512;

// 16-byte asynchronous global->shared copies (no spin waits: cp.async.wait_group is a
// hardware wait on this thread's own copies)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Copy the rows this warp will use (rr = r0 + warp, r0 + warp + nw, ...) of one nb x nb block
// (row-major, nb even) to this CTA's staging buffer, whose row q holds block row r0 + q.
__device__ __forceinline__ void stage_warp_rows(double* dst, const double* blk, int64_t r0, int64_t r1, int64_t nb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t chunks = nb / 2;  // 16-byte chunks per row
  for (int64_t rr = r0 + warp; rr < r1; rr += nw) {
    const double* src = blk + rr * nb;
    double* d = dst + (rr - r0) * nb;
    for (int64_t q = lane; q < chunks; q += 32) cp_async16(d + 2 * q, src + 2 * q);
  }
}

// One dependent step of a block sweep: rows [r0, r1) of  out = vin - M xprev, where M's rows
// come from shared memory (staged) or global memory; results go to every CTA of the cluster
// (distributed shared memory, buffer `cur`) and to global memory.
template <bool STAGED>
__device__ __forceinline__ void sweep_rows(cooperative_groups::cluster_group& cluster, int cs, double* xbuf,
                                           int cur, const double* xprev, bool has_prev, const double* Mrows,
                                           const double* Mglob, int64_t r0, int64_t r1, int64_t nb,
                                           int64_t pbase, int64_t nc, const double* r, const int64_t* gidx,
                                           const double* vdirect, const double* zin, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int64_t rr = r0 + warp; rr < r1; rr += nw) {
    const int64_t p = pbase + rr;
    double s = 0.0;
    if (has_prev) {
      const double* row = STAGED ? (Mrows + (rr - r0) * nb) : (Mglob + rr * nb);
#pragma unroll 4
      for (int64_t k = lane; k < nb; k += 32) s += row[k] * xprev[k];
    }
    s = warp_sum(s);
    double vin;
    if (zin) vin = zin[p];
    else vin = p < nc ? (vdirect ? vdirect[p] : r[gidx[p]]) : 0.0;
    const double val = vin - s;
    for (int t = lane; t < cs; t += 32) {
      double* dst = cluster.map_shared_rank(xbuf, t);
      dst[cur * nb + rr] = val;
    }
    if (lane == 0) out[p] = val;
  }
}

// Block-tridiagonal LDL^T sweeps of A_w (Section 5.1 filter solve), one thread-block cluster
// of cs CTAs (cluster size set at launch).  Each dependent block step is a GEMV split by
// rows over the cluster; the running block vector is exchanged through distributed shared
// memory.  With STAGED the next step's matrix rows are copied to shared memory with
// cp.async while the current step computes and waits at the cluster barrier.
//   forward  (fwd = true):  y_0 = v_0,            y_i = v_i - G_i y_{i-1}
//   backward (fwd = false): w_{N-1} = z_{N-1},    w_i = z_i - G_{i+1}^T w_{i+1}
// v_p = r[gidx[p]] (or vdirect[p]) for p < nc, 0 on padding rows.
template <bool STAGED>
__global__ void __launch_bounds__(FILTER_TPB)
filter_sweep_kernel(bool fwd, const double* __restrict__ M, const int64_t* __restrict__ gidx,
                    const double* __restrict__ r, const double* __restrict__ vdirect, const double* __restrict__ zin,
                    int64_t nc, int64_t nb, int64_t nblk, double* out) {
  namespace cgp = cooperative_groups;
  cgp::cluster_group cluster = cgp::this_cluster();
  extern __shared__ __align__(16) double fsm[];
  double* xbuf = fsm;                 // [2][nb]
  double* gbuf = fsm + 2 * nb;        // [2][rpc][nb] when STAGED
  const int cs = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int64_t rpc = (nb + cs - 1) / cs;
  const int64_t r0 = rank * rpc < nb ? rank * rpc : nb;
  const int64_t r1 = r0 + rpc < nb ? r0 + rpc : nb;
  // matrix used by step t (t >= 1): forward G_t, backward G_{i+1}^T with i = nblk-1-t
  auto mat_of = [&](int64_t t) -> const double* {
    const int64_t blk = fwd ? t : (nblk - t);
    return M + blk * nb * nb;
  };
  cluster.sync();  // every CTA of the cluster has started before peers write its shared memory
  for (int64_t t = 0; t < nblk; ++t) {
    const int cur = (int)(t & 1);
    if (STAGED) {
      // each warp stages the rows it will use one step ahead; a warp only reads rows it copied,
      // so landing its own copies (wait_group) and a warp barrier are enough
      if (t + 1 < nblk) stage_warp_rows(gbuf + ((t + 1) & 1) * rpc * nb, mat_of(t + 1), r0, r1, nb);
      cp_async_commit();
      cp_async_wait1();  // the copy for step t (committed one iteration earlier) has landed
      __syncwarp();
    }
    const int64_t i = fwd ? t : nblk - 1 - t;
    sweep_rows<STAGED>(cluster, cs, xbuf, cur, xbuf + (cur ^ 1) * nb, t > 0, gbuf + cur * rpc * nb,
                       t > 0 ? mat_of(t) : M, r0, r1, nb, i * nb, fwd ? nc : 0, r, gidx, vdirect,
                       fwd ? nullptr : zin, out);
    cluster.sync();
  }
}

// One phase of the block cyclic reduction solve of A_w (tasks built on the host, see
// FilterTask).  CTA = (task, tile of FBCR_ROWS output rows); the task's input blocks are
// staged in shared memory, eight lanes reduce one row of each nb x nb GEMV (row-major,
// coalesced) with two independent FMA chains.  GATHER: the phase reads the right-hand
// side v straight from r[gidx[p]] (or vdirect[p]) in factor order, 0 on padding rows.
constexpr int FBCR_TPB = 256;

// LPR lanes reduce one row (8: 32 rows per CTA, for phases with many output blocks; 32: 8 rows
// per CTA, four times the CTAs, for the few-block phases near the top of the reduction, which
// are bound by how many loads are in flight rather than by the FP64 pipe).
template <bool GATHER, int LPR>
__global__ void __launch_bounds__(FBCR_TPB)
filter_bcr_kernel(const FilterTask* __restrict__ tasks, int tiles, const double* __restrict__ M, int64_t nb,
                  const double* __restrict__ r, const int64_t* __restrict__ gidx, const double* __restrict__ vdirect,
                  int64_t nc, double* v, double* x) {
  static_assert(LPR == 8 || LPR == 16 || LPR == 32, "lanes per row");
  constexpr int ROWS = FBCR_TPB / LPR;
  extern __shared__ __align__(16) double fin[];  // [2][nb]: input blocks in0, in1
  const FilterTask t = tasks[blockIdx.x / tiles];
  const int64_t tile = blockIdx.x % tiles;
  auto vin = [&](int64_t p) -> double {
    if (GATHER) return p < nc ? (vdirect ? vdirect[p] : r[gidx[p]]) : 0.0;
    return v[p];
  };
  auto stage = [&](int32_t blk, double* dst) {
    if (blk < 0) return;
    const int64_t base = (int64_t)blk * nb;
    for (int64_t q = threadIdx.x; q < nb; q += FBCR_TPB) dst[q] = t.kind == 2 ? x[base + q] : vin(base + q);
  };
  stage(t.in0, fin);
  stage(t.in1, fin + nb);
  __syncthreads();
  const int sub = threadIdx.x & (LPR - 1);
  const int64_t row = tile * ROWS + threadIdx.x / LPR;
  double sa = 0.0, sb = 0.0;
  auto term = [&](int64_t mat, int32_t blk, const double* xv) {
    if (mat < 0 || blk < 0) return;
    const double* mr = M + mat * nb * nb + row * nb;
    int64_t c = sub;
    for (; c + LPR < nb; c += 2 * LPR) {
      sa = fma(__ldg(mr + c), xv[c], sa);
      sb = fma(__ldg(mr + c + LPR), xv[c + LPR], sb);
    }
    if (c < nb) sa = fma(__ldg(mr + c), xv[c], sa);
  };
  if (row < nb) {
    term(t.m0, t.in0, fin);
    term(t.m1, t.in1, fin + nb);
  }
  double s = sa + sb;
#pragma unroll
  for (int off = LPR / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off, LPR);
  if (row < nb && sub == 0) {
    const int64_t p = (int64_t)t.out * nb + row;
    if (t.kind == 0) x[p] = s;
    else if (t.kind == 1) v[p] = vin(p) - s;
    else x[p] = x[p] - s;
  }
}

// z_i = Dinv_i y_i for all blocks in parallel (one warp per row).
__global__ void __launch_bounds__(TPB) filter_diag_kernel(const double* __restrict__ Dinv, const double* __restrict__ y,
                                                          double* z, int64_t nb, int64_t nblk) {
  const int lane = threadIdx.x & 31;
  const int64_t nrow = nb * nblk;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t ws = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = w0; p < nrow; p += ws) {
    const int64_t blk = p / nb, rr = p % nb;
    const double* row = Dinv + blk * nb * nb + rr * nb;
    const double* yb = y + blk * nb;
    double s = 0.0;
#pragma unroll 4
    for (int64_t k = lane; k < nb; k += 32) s += row[k] * yb[k];
    s = warp_sum(s);
    if (lane == 0) z[p] = s;
  }
}

// y[gidx[p]] += w[p] for p < nc   (y2 = y1 + P w)
__global__ void filter_scatter_kernel(const int64_t* __restrict__ gidx, const double* __restrict__ w, double* y, int64_t nc) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nc; p += (int64_t)gridDim.x * blockDim.x)
    y[gidx[p]] += w[p];
}

// out[map[p]] = in[p] (map != null) or out[p] = in[map2[p]] -- permutations for the standalone filter solve
__global__ void permute_kernel(int64_t n, const int64_t* __restrict__ scatter_to, const int64_t* __restrict__ gather_from,
                               const double* __restrict__ in, double* out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    if (scatter_to) out[scatter_to[p]] = in[p];
    else out[p] = in[gather_from[p]];
  }
}

// ---------------- learned smoother (per-row l1-Jacobi damping) ----------------
// theta_i = 0.3 + 0.9 sigmoid(MLP(f_i)), MLP 6 -> 32 -> 32 -> 1 with ReLU, weights (1313, FP32):
//   W1[32][6] | b1[32] | W2[32][32] | b2[32] | w3[32] | b3.   W_i = theta_i / l1_i.
// theta in [0.3, 1.2] < 2 keeps the l1 smoother convergent and the V-cycle SPD.
constexpr int MLP_NW = 1313;
constexpr int MLP_H = 32;

struct MlpAct {
  float h1[MLP_H], h2[MLP_H];
  float o;
};

__device__ __forceinline__ void mlp_forward(const float* w, const float* f, MlpAct& a) {
  const float* W1 = w;
  const float* b1 = w + 192;
  const float* W2 = w + 224;
  const float* b2 = w + 1248;
  const float* w3 = w + 1280;
#pragma unroll 4
  for (int j = 0; j < MLP_H; ++j) {
    float s = b1[j];
#pragma unroll
    for (int k = 0; k < 6; ++k) s += W1[6 * j + k] * f[k];
    a.h1[j] = s > 0.f ? s : 0.f;
  }
#pragma unroll 2
  for (int j = 0; j < MLP_H; ++j) {
    float s = b2[j];
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) s += W2[MLP_H * j + k] * a.h1[k];
    a.h2[j] = s > 0.f ? s : 0.f;
  }
  float o = w[1312];
#pragma unroll
  for (int k = 0; k < MLP_H; ++k) o += w3[k] * a.h2[k];
  a.o = o;
}

__device__ __forceinline__ float mlp_sigmoid(float o) { return 1.f / (1.f + __expf(-o)); }

// W = theta / l1 for every row (plain = 1: theta = 1, the plain l1-Jacobi weights)
__global__ void __launch_bounds__(TPB) mlp_infer_kernel(int64_t n, const float* __restrict__ feat,
                                                        const float* __restrict__ wglob, int plain,
                                                        const double* __restrict__ l1, double* winv, float* winvf) {
  __shared__ float w[MLP_NW];
  for (int p = threadIdx.x; p < MLP_NW; p += blockDim.x) w[p] = plain ? 0.f : wglob[p];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double theta = 1.0;
    if (!plain) {
      float f[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) f[k] = feat[6 * i + k];
      MlpAct a;
      mlp_forward(w, f, a);
      theta = 0.3 + 0.9 * (double)mlp_sigmoid(a.o);
    }
    const double wi = theta / l1[i];
    if (winv) winv[i] = wi;
    if (winvf) winvf[i] = (float)wi;
  }
}

// uniform(-1, 1) training vectors from SplitMix64 (Steele, Lea, Flood) of seed + (i+1) * golden gamma
__global__ void rand_uniform_kernel(int64_t n, uint64_t seed, double* r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    r[i] = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
  }
}

// deterministic dot product: *result = sum a_i b_i
__global__ void __launch_bounds__(TPB) dot_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                                  double* partial, double* result, unsigned* counter) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  grid_dot_finish(s, partial, result, counter);
}

// Backward pass of the smoothing loss L = ||e||^2 / ||r||^2, e = (I - A W_theta) r, through the
// MLP.  dL/dtheta_i = -2 (r_i / l1_i) (A e)_i / ||r||^2 (A symmetric).  One row per thread; the
// block's 256 rows give one partial gradient (sums over rows in a fixed order), written to
// partial[blockIdx.x][MLP_NW].  Dynamic shared memory: MLP_SMEM bytes.
constexpr int MLP_LD = MLP_H + 1;
constexpr size_t MLP_SMEM = sizeof(float) * (MLP_NW + 4 * TPB * MLP_LD + 6 * TPB + TPB);

__global__ void __launch_bounds__(TPB) mlp_backward_kernel(int64_t n, const float* __restrict__ feat,
                                                           const float* __restrict__ wglob,
                                                           const double* __restrict__ r, const double* __restrict__ l1,
                                                           const double* __restrict__ Ae, const double* rr, float scale,
                                                           float* partial) {
  extern __shared__ float msm[];
  float* w = msm;
  float* H1 = w + MLP_NW;
  float* H2 = H1 + TPB * MLP_LD;
  float* D1 = H2 + TPB * MLP_LD;
  float* D2 = D1 + TPB * MLP_LD;
  float* F = D2 + TPB * MLP_LD;
  float* DO = F + 6 * TPB;
  for (int p = threadIdx.x; p < MLP_NW; p += blockDim.x) w[p] = wglob[p];
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * TPB + t;
  float f[6] = {0, 0, 0, 0, 0, 0};
  MlpAct a;
  for (int j = 0; j < MLP_H; ++j) { a.h1[j] = 0.f; a.h2[j] = 0.f; }
  float dout = 0.f;
  if (i < n) {
#pragma unroll
    for (int k = 0; k < 6; ++k) f[k] = feat[6 * i + k];
    mlp_forward(w, f, a);
    const float sg = mlp_sigmoid(a.o);
    const double dth = -2.0 * (r[i] / l1[i]) * Ae[i] / *rr;
    dout = scale * (float)dth * 0.9f * sg * (1.f - sg);
  }
  const float* W2 = w + 224;
  const float* w3 = w + 1280;
  float d2[MLP_H];
  for (int j = 0; j < MLP_H; ++j) d2[j] = (a.h2[j] > 0.f) ? dout * w3[j] : 0.f;
  for (int k = 0; k < MLP_H; ++k) {
    float s = 0.f;
    for (int j = 0; j < MLP_H; ++j) s += W2[MLP_H * j + k] * d2[j];
    D1[t * MLP_LD + k] = (a.h1[k] > 0.f) ? s : 0.f;
    H1[t * MLP_LD + k] = a.h1[k];
    H2[t * MLP_LD + k] = a.h2[k];
    D2[t * MLP_LD + k] = d2[k];
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) F[6 * t + k] = f[k];
  DO[t] = dout;
  __syncthreads();
  for (int p = t; p < MLP_NW; p += TPB) {
    float s = 0.f;
    if (p < 192) {                 // W1[j][k] += d1_j f_k
      const int j = p / 6, k = p % 6;
      for (int q = 0; q < TPB; ++q) s += D1[q * MLP_LD + j] * F[6 * q + k];
    } else if (p < 224) {          // b1
      const int j = p - 192;
      for (int q = 0; q < TPB; ++q) s += D1[q * MLP_LD + j];
    } else if (p < 1248) {         // W2[j][k] += d2_j h1_k
      const int j = (p - 224) / MLP_H, k = (p - 224) % MLP_H;
      for (int q = 0; q < TPB; ++q) s += D2[q * MLP_LD + j] * H1[q * MLP_LD + k];
    } else if (p < 1280) {         // b2
      const int j = p - 1248;
      for (int q = 0; q < TPB; ++q) s += D2[q * MLP_LD + j];
    } else if (p < 1312) {         // w3[k] += dout h2_k
      const int k = p - 1280;
      for (int q = 0; q < TPB; ++q) s += DO[q] * H2[q * MLP_LD + k];
    } else {                       // b3
      for (int q = 0; q < TPB; ++q) s += DO[q];
    }
    partial[(int64_t)blockIdx.x * MLP_NW + p] = s;
  }
}

// grad[p] (+)= sum over parts of partial[part][p], parts in index order
__global__ void mlp_grad_reduce_kernel(int64_t nparts, const float* __restrict__ partial, float* grad, int accumulate) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NW) return;
  float s = 0.f;
  for (int64_t b = 0; b < nparts; ++b) s += partial[b * MLP_NW + p];
  grad[p] = accumulate ? grad[p] + s : s;
}

// Adam (Kingma & Ba) on the MLP parameters
__global__ void mlp_adam_kernel(float* w, float* m, float* v, const float* __restrict__ g, float lr, float beta1,
                                float beta2, float eps, float t) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NW) return;
  const float gi = g[p];
  const float mi = beta1 * m[p] + (1.f - beta1) * gi;
  const float vi = beta2 * v[p] + (1.f - beta2) * gi * gi;
  m[p] = mi;
  v[p] = vi;
  const float mh = mi / (1.f - powf(beta1, t));
  const float vh = vi / (1.f - powf(beta2, t));
  w[p] -= lr * mh / (sqrtf(vh) + eps);
}

// loss[it] = scale * sum_l ee[l] / rr[l]
__global__ void mlp_loss_kernel(int nl, const double* ee, const double* rr, float scale, float* loss) {
  double s = 0.0;
  for (int l = 0; l < nl; ++l) s += ee[l] / rr[l];
  *loss = (float)(scale * s);
}

// ---------------- PCG ----------------

// x += alpha p ; r -= alpha q with alpha = rz / pq (breakdown if pq <= 0).  Also writes the
// entry of the next V-cycle: wr = W0 r (FP64 V-cycle) or r32 = r, wr32 = W0 r (FP32 V-cycle),
// and with a flexible PCG the dot r_{k+1}^T z_k into st->rz_cross.
__global__ void __launch_bounds__(TPB) pcg_update_xr_kernel(PcgState* st, const double* __restrict__ p,
                                                            const double* __restrict__ q, double* x, double* r,
                                                            const double* __restrict__ w0, double* wr, float* r32,
                                                            float* wr32, const double* __restrict__ zold,
                                                            double* partial, unsigned* counter, int64_t n) {
  if (st->done) return;
  const double pq = st->pq;
  if (!(pq > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) { st->status = isfinite(pq) ? 4 : 2; st->done = 1; }
    return;
  }
  const double alpha = st->rz / pq;
  double dacc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    const double wri = w0[i] * ri;
    if (wr) wr[i] = wri;
    if (r32) { r32[i] = (float)ri; wr32[i] = (float)wri; }
    if (zold) dacc += ri * zold[i];
  }
  if (zold) grid_dot_finish(dacc, partial, &st->rz_cross, counter);
}

// p = z + beta p with beta = rz_new / rz
__global__ void pcg_update_p_kernel(const PcgState* st, const double* __restrict__ z, double* p, int64_t n) {
  if (st->done) return;
  const double beta = st->flexible ? (st->rz_new - st->rz_cross) / st->rz : st->rz_new / st->rz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// One thread: advance the iteration count and evaluate the stop test sqrt(rz/rz0) < rtol.
__global__ void pcg_finalize_kernel(PcgState* st, cudaGraphConditionalHandle cond, int use_cond) {
  if (!st->done) {
    const double rzn = st->rz_new;
    st->iter += 1;
    if (!isfinite(rzn)) { st->status = 2; st->done = 1; }
    else if (rzn < 0.0) { st->status = 4; st->done = 1; }
    else {
      st->relres = sqrt(rzn / st->rz0);
      st->rz = rzn;
      if (st->relres < st->rtol) { st->status = 0; st->done = 1; }
      else if (st->iter >= st->maxit) { st->status = 5; st->done = 1; }
    }
  }
  if (use_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

// After r0 = b - A x0 and z0 = M r0 (rz_new = r0^T z0): initialise the scalars.
__global__ void pcg_init_kernel(PcgState* st, int maxit, double rtol, int flexible) {
  const double rz = st->rz_new;
  st->flexible = flexible;
  st->rz_cross = 0.0;
  st->rz = rz;
  st->rz0 = rz;
  st->iter = 0;
  st->maxit = maxit;
  st->rtol = rtol;
  st->relres = 1.0;
  st->pq = 0.0;
  st->done = 0;
  st->status = 5;
  if (!isfinite(rz)) { st->status = 2; st->done = 1; }
  else if (rz < 0.0) { st->status = 4; st->done = 1; }
  else if (rz == 0.0) { st->status = 0; st->done = 1; st->relres = 0.0; }
  else if (maxit <= 0) { st->done = 1; }
}

__global__ void copy_kernel(int64_t n, const double* __restrict__ a, double* b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = a[i];
}

}  // namespace amgf
