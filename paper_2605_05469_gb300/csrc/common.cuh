// Shared device helpers for the PIC library: PTX wrappers for mbarriers and
// bulk (TMA-engine) copies, bounded waits, and FP64 block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pic.h"

namespace pic {

// Device-side error word bits (the context's error word, read by the host).
enum : int {
  DEV_ERR_TIMEOUT = 1,  // a bounded mbarrier wait expired
  DEV_ERR_NONFINITE = 2,
  DEV_ERR_BOUNDS = 4,   // a guarded index fell outside its buffer
};

// Periodic node grid: N^3 nodes x_i = i h on [0, L)^3.
struct Grid {
  int N;
  double L, h, inv_h;
};

// Solver scalars shared between the kernels of one solve. Written only by the
// last block of a reduction kernel, read by all blocks of later kernels.
struct Scalars {
  double rr;        // current (r, r) or (r, z)
  double rr_prev;
  double pq;        // (p, A p)
  double alpha, beta;
  double bb;        // (b, b)
  double tol2;      // (tol * ||b||)^2 in the units of rr
  double rmax2;     // MIXED: (r, r) at the last FP64 residual recomputation
  double delta2;    // MIXED: reliable-update trigger factor squared
  double rz;        // FCG: (r, z)
  double rz_old;    // unused
  double true_rr;   // MIXED: last recomputed FP64 (r, r)
  double sum0, sum1;  // mean projections
  double scale;     // CNN: RMS of r
  int iter, maxit;
  int done;         // 0 running, 1 converged, 2 maxit, 3 breakdown
  int need_update;  // MIXED: a reliable update is pending
  int updates;      // MIXED: number of reliable updates so far
  int fallbacks;    // CNN: Jacobi fallbacks
  int final_check;  // MIXED: the pending update was triggered by convergence
  int xsel;         // MIXED: which of the two FP64 solution buffers is current
  int x32_reset;    // MIXED: the FP32 correction was folded; read it as zero
  int fcg;          // flexible CG: alpha = (r, z) / (p, A p)
  int fallback_now; // FCG: this iteration's z is replaced by the Jacobi direction
  int refine_max;   // MIXED: FP64 residual recomputations allowed (0 = no cap)
  int redo;         // FCG: a reliable update replaced r after the fused update;
                    // z and the direction's dots are recomputed from it
};

// One particle, 64 bytes, so that a particle moved by the sort fills exactly
// two 32-byte sectors and the kernels read it with four 16-byte loads:
//   fx, fy, fz  position inside its cell in units of 2^-64 h (exact fixed
//               point: cell changes and the periodic wrap are integer adds);
//   vx, vy, vz  velocity as double-float pairs (hi + lo, ~48-bit significand;
//               the push runs on the FP32 pipes);
//   id          the index the particle was sampled with;
//   key         its cell ix + N (iy + N iz);
//   cell        ix | iy << 10 | iz << 20 (N <= 1024);
//   rank        its rank among the particles of its cell, for the next sort
//               (key and rank are written together by whoever moves the
//               particle to a new cell: the initial sampling, the push, the
//               state loaded from the caller).
struct __align__(64) PRec {
  uint64_t fx, fy, fz;
  float2 vx, vy, vz;
  uint32_t id, key, cell, rank;
};
static_assert(sizeof(PRec) == 64, "particle record");

__host__ __device__ __forceinline__ uint32_t pack_cell(int ix, int iy, int iz) {
  return (uint32_t)ix | ((uint32_t)iy << 10) | ((uint32_t)iz << 20);
}
__host__ __device__ __forceinline__ int cell_x(uint32_t c) { return (int)(c & 1023u); }
__host__ __device__ __forceinline__ int cell_y(uint32_t c) { return (int)((c >> 10) & 1023u); }
__host__ __device__ __forceinline__ int cell_z(uint32_t c) { return (int)(c >> 20); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Wall-time budget of every bounded device-side wait.
constexpr uint64_t kWaitBudgetNs = 2000000000ull;

// Wait for the phase with the given parity to complete. Gives up after
// budget_ns of wall time (about two seconds by default), records
// DEV_ERR_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  uint64_t budget_ns = kWaitBudgetNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 0 && global_timer_ns() - t0 > budget_ns) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      return false;
    }
  }
}

// Async-proxy fence: generic-proxy accesses of shared memory before it are
// ordered before later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy global -> shared (TMA engine), completion counted on `bar` in bytes.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of `v` over the block, valid in every thread. blockDim.x a multiple of
// 32 and <= 1024. `red` is shared scratch of >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];  // fixed order: deterministic
  return s;
}

// Last-block reduction of K values per block. Every block calls it with its
// per-thread contributions v[0..K). Returns true in the last block to finish,
// where out[0..K) then holds the totals summed over blocks in block order
// (deterministic). The counter is reset for the next launch.
template <int K>
__device__ __forceinline__ bool grid_reduce_last(const double (&v)[K], double* partials, unsigned* counter,
                                                 double (&out)[K]) {
  __shared__ double red[32];
  __shared__ bool am_last;
  double bs[K];
#pragma unroll
  for (int q = 0; q < K; ++q) bs[q] = block_sum(v[q], red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) partials[(size_t)blockIdx.x * K + q] = bs[q];
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] += __ldcg(&partials[(size_t)b * K + q]);
  }
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = block_sum(acc[q], red);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

// Compensated FP32 running sum (Knuth's TwoSum, branch-free): keeps per-thread
// partial dot products accurate to a few FP32 ulps of the sum without FP64
// instructions, which run at 1/58 of the FP32 rate on this GPU. Widened to
// FP64 once per thread before the FP64 block and grid reduction.
struct CompSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

}  // namespace pic
