// Conjugate-gradient kernels on the periodic 7-point operator (Sec. 3.2).
//
// All solves run on the scaled system (h^2 A) x = h^2 b, whose operator
// 6 I - (sum of neighbours) has integer coefficients. With the constant
// Jacobi diagonal 6/h^2 folded into the scalars, Jacobi-PCG and CG produce
// the same iterates, so the preconditioner costs nothing per cell.
//
// One iteration is two kernels, each a single pass over the grid with its
// reduction finished on the device by the last block (alpha and beta never
// leave the GPU):
//   pap   : p = r + beta p_in (on the whole streamed slab incl. halo),
//           writes p, optionally q = A p, reduces (p, A p) -> alpha;
//   update: x += alpha p, r -= alpha q (FP64, q stored) or
//           r -= alpha A p (FP32, stencil recomputed), reduces (r, r) -> beta,
//           convergence and iteration count.
#pragma once
#include "stream.cuh"

namespace pic {

constexpr int kMaxStages = 8;

// Layout of one stage: vector 0 (type A) then optional vector 1 (type B),
// each rows*N elements; stage size rounded up to 128 bytes.
template <typename A, typename B, int NV>
struct StageLayout {
  size_t e, bytes;
  __host__ __device__ StageLayout(int rows, int N) {
    e = (size_t)rows * N;
    size_t b = e * sizeof(A) + (NV == 2 ? e * sizeof(B) : 0);
    bytes = (b + 127) & ~(size_t)127;
  }
  __device__ A* v0(unsigned char* base, int st) const { return reinterpret_cast<A*>(base + st * bytes); }
  __device__ B* v1(unsigned char* base, int st) const {
    return reinterpret_cast<B*>(base + st * bytes + e * sizeof(A));
  }
};

// Streams the slab's planes through the stage ring and calls
//   conv(st)            once per arriving stage (all threads, then a barrier),
//   body(t, sp, sc, sn) once per output plane t with the stage indices of
//                       planes z-1, z, z+1.
// Returns false if a bounded wait expired (the caller skips its epilogue
// writes but still takes part in its final reduction).
template <typename A, typename B, int NV, typename Conv, typename Body>
__device__ __forceinline__ bool stream_slab(const Slab& s, unsigned char* smem, uint64_t* bars, const A* src0,
                                            const B* src1, int* err, Conv conv, Body body) {
  const StageLayout<A, B, NV> lay(s.rows, s.N);
  const int nload = s.ZC + 2;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int st = 0; st < s.S; ++st) mbar_init(&bars[st], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t tx = plane_bytes<A>(s) + (NV == 2 ? plane_bytes<B>(s) : 0u);
  auto issue = [&](int l) {
    const int st = l % s.S;
    const int z = load_plane(s, l);
    mbar_arrive_expect_tx(&bars[st], tx);
    issue_plane(lay.v0(smem, st), src0, s, z, &bars[st]);
    if (NV == 2) issue_plane(lay.v1(smem, st), src1, s, z, &bars[st]);
  };
  if (threadIdx.x == 0) {
    const int pre = nload < s.S ? nload : s.S;
    for (int l = 0; l < pre; ++l) issue(l);
  }
  auto acquire = [&](int l) {
    const int st = l % s.S;
    if (!mbar_wait_bounded(&bars[st], (uint32_t)((l / s.S) & 1), err)) abort_flag = 1;
    conv(st);
  };
  acquire(0);
  acquire(1);
  bool ok = true;
  for (int t = 0; t < s.ZC; ++t) {
    acquire(t + 2);
    __syncthreads();
    if (abort_flag) { ok = false; break; }
    body(t, t % s.S, (t + 1) % s.S, (t + 2) % s.S);
    __syncthreads();
    if (threadIdx.x == 0 && t + s.S < nload) {
      fence_proxy_async_smem();
      issue(t + s.S);
    }
  }
  return ok;
}

// ---------------------------------------------------------------------------
// pap: p = r + beta p_in over the streamed slab; q = (h^2 A) p; (p, q) -> alpha
// ---------------------------------------------------------------------------
template <typename T, bool STORE_Q>
__global__ void __launch_bounds__(256) k_cg_pap(const T* __restrict__ r, const T* __restrict__ pin,
                                                T* __restrict__ pout, T* __restrict__ q, Scalars* sc,
                                                double* partials, unsigned* counter, int* err, StreamGeo g) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  if (sc->done) return;
  const Slab s = make_slab(g);
  const T beta = (T)sc->beta;
  const StageLayout<T, T, 2> lay(s.rows, s.N);
  double dot = 0.0;
  auto conv = [&](int st) {
    T* R = lay.v0(smem, st);
    T* P = lay.v1(smem, st);
    for (size_t i = threadIdx.x; i < lay.e; i += blockDim.x) P[i] = R[i] + beta * P[i];
  };
  auto body = [&](int t, int sp, int scur, int sn) {
    if (!s.active) return;
    V4<T> c;
    const V4<T> ap = stencil4(lay.v1(smem, sp), lay.v1(smem, scur), lay.v1(smem, sn), s, c);
    const size_t off = cell_offset(s, t);
    st4(pout + off, c);
    if (STORE_Q) st4(q + off, ap);
    T d = c.v[0] * ap.v[0];
#pragma unroll
    for (int i = 1; i < 4; ++i) d += c.v[i] * ap.v[i];
    dot += (double)d;
  };
  stream_slab<T, T, 2>(s, smem, bars, r, pin, err, conv, body);
  double v[1] = {dot}, tot[1];
  if (grid_reduce_last<1>(v, partials, counter, tot) && threadIdx.x == 0) {
    const double pq = tot[0];
    sc->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
      sc->done = 3;
    } else {
      sc->alpha = sc->rr / pq;
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 update: x += alpha p; r -= alpha q; (r, r) -> beta, convergence
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cg_update64(double* __restrict__ x, double* __restrict__ r,
                                                     const double* __restrict__ p, const double* __restrict__ q,
                                                     size_t n4, Scalars* sc, double* partials, unsigned* counter) {
  if (sc->done) return;
  const double alpha = sc->alpha;
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    V4<double> xv = ldg4(x + 4 * i), rv = ldg4(r + 4 * i);
    const V4<double> pv = ldg4(p + 4 * i), qv = ldg4(q + 4 * i);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      xv.v[k] = fma(alpha, pv.v[k], xv.v[k]);
      rv.v[k] = fma(-alpha, qv.v[k], rv.v[k]);
      acc = fma(rv.v[k], rv.v[k], acc);
    }
    st4(x + 4 * i, xv);
    st4(r + 4 * i, rv);
  }
  double v[1] = {acc}, tot[1];
  if (grid_reduce_last<1>(v, partials, counter, tot) && threadIdx.x == 0) {
    const double rr = tot[0];
    sc->rr_prev = sc->rr;
    sc->beta = rr / sc->rr;
    sc->rr = rr;
    sc->iter += 1;
    if (!isfinite(rr)) sc->done = 3;
    else if (rr <= sc->tol2) sc->done = 1;
    else if (sc->iter >= sc->maxit) sc->done = 2;
  }
}

// ---------------------------------------------------------------------------
// FP32 update: x += alpha p; r -= alpha (h^2 A) p; (r, r) -> beta; triggers a
// reliable update when (r, r) fell by delta^2 since the last one, or reached
// the tolerance.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cg_update32(float* __restrict__ x, float* __restrict__ r,
                                                     const float* __restrict__ p, Scalars* sc, double* partials,
                                                     unsigned* counter, int* err, StreamGeo g) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  if (sc->done) return;
  const Slab s = make_slab(g);
  const float alpha = (float)sc->alpha;
  const bool x_zero = sc->x32_reset != 0;
  const StageLayout<float, float, 1> lay(s.rows, s.N);
  double acc = 0.0;
  auto conv = [&](int) {};
  auto body = [&](int t, int sp, int scur, int sn) {
    if (!s.active) return;
    V4<float> c;
    const V4<float> ap = stencil4(lay.v0(smem, sp), lay.v0(smem, scur), lay.v0(smem, sn), s, c);
    const size_t off = cell_offset(s, t);
    V4<float> xv = x_zero ? V4<float>{{0.f, 0.f, 0.f, 0.f}} : ldg4(x + off);
    V4<float> rv = ldg4(r + off);
    float d = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      xv.v[i] = fmaf(alpha, c.v[i], xv.v[i]);
      rv.v[i] = fmaf(-alpha, ap.v[i], rv.v[i]);
      d = fmaf(rv.v[i], rv.v[i], d);
    }
    st4(x + off, xv);
    st4(r + off, rv);
    acc += (double)d;
  };
  stream_slab<float, float, 1>(s, smem, bars, p, (const float*)nullptr, err, conv, body);
  double v[1] = {acc}, tot[1];
  if (grid_reduce_last<1>(v, partials, counter, tot) && threadIdx.x == 0) {
    const double rr = tot[0];
    sc->x32_reset = 0;
    sc->rr_prev = sc->rr;
    sc->beta = rr / sc->rr;
    sc->rr = rr;
    sc->iter += 1;
    if (!isfinite(rr)) {
      sc->done = 3;
    } else {
      if (rr <= sc->tol2) {
        sc->need_update = 1;
        sc->final_check = 1;
      } else if (rr <= sc->delta2 * sc->rmax2) {
        sc->need_update = 1;
      }
      if (!sc->need_update && sc->iter >= sc->maxit) sc->done = 2;
    }
  }
}

// ---------------------------------------------------------------------------
// Initial FP64 residual of the judge: r = h^2 b - (h^2 A) x, (r, r).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_residual64(const double* __restrict__ x, const double* __restrict__ b,
                                                    double* __restrict__ r, Scalars* sc, double* partials,
                                                    unsigned* counter, int* err, StreamGeo g) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  if (sc->done) return;
  const Slab s = make_slab(g);
  const StageLayout<double, double, 1> lay(s.rows, s.N);
  double acc = 0.0;
  auto conv = [&](int) {};
  auto body = [&](int t, int sp, int scur, int sn) {
    if (!s.active) return;
    V4<double> c;
    const V4<double> ax = stencil4(lay.v0(smem, sp), lay.v0(smem, scur), lay.v0(smem, sn), s, c);
    const size_t off = cell_offset(s, t);
    const V4<double> bv = ldg4(b + off);
    V4<double> rv;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      rv.v[i] = bv.v[i] - ax.v[i];
      acc = fma(rv.v[i], rv.v[i], acc);
    }
    st4(r + off, rv);
  };
  stream_slab<double, double, 1>(s, smem, bars, x, (const double*)nullptr, err, conv, body);
  double v[1] = {acc}, tot[1];
  if (grid_reduce_last<1>(v, partials, counter, tot) && threadIdx.x == 0) {
    const double rr = tot[0];
    sc->rr = rr;
    sc->rr_prev = rr;
    sc->true_rr = rr;
    sc->beta = 0.0;
    sc->iter = 0;
    if (!isfinite(rr)) sc->done = 3;
    else if (rr <= sc->tol2) sc->done = 1;
  }
}

// ---------------------------------------------------------------------------
// Mixed-precision reliable update (van der Vorst & Ye 2000; Clark et al.
// 2010): fold the FP32 correction into the FP64 solution and recompute the
// true residual in FP64:
//   xs = x64[sel] + x32 (on the streamed slab, in FP64),
//   r64 = h^2 b - (h^2 A) xs,  x64[sel^1] = xs,  r32 = (float) r64.
// x64 is ping-ponged and x32 is not rewritten here, because neighbouring
// blocks are still reading both as halo; the next FP32 update treats x32 as
// zero (x32_reset) instead. mode 0: set-up (always runs); 1: runs only if an
// update is pending; 2: forced final fold.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_reliable(double* __restrict__ x64a, double* __restrict__ x64b,
                                                  const float* __restrict__ x32, const double* __restrict__ b,
                                                  float* __restrict__ r32, Scalars* sc, double* partials,
                                                  unsigned* counter, int* err, StreamGeo g, int mode) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  if (mode == 0 && sc->done) return;
  if (mode == 1 && (sc->done || !sc->need_update)) return;
  const Slab s = make_slab(g);
  const int sel = sc->xsel;
  const double* xin = sel ? x64b : x64a;
  double* xout = sel ? x64a : x64b;
  // x32 holds a stale correction that has already been folded: read it as zero
  const bool x32_zero = sc->x32_reset != 0;
  const StageLayout<double, float, 2> lay(s.rows, s.N);
  double acc64 = 0.0, acc32 = 0.0;
  auto conv = [&](int st) {
    if (x32_zero) return;
    double* X = lay.v0(smem, st);
    const float* Y = lay.v1(smem, st);
    for (size_t i = threadIdx.x; i < lay.e; i += blockDim.x) X[i] += (double)Y[i];
  };
  auto body = [&](int t, int sp, int scur, int sn) {
    if (!s.active) return;
    V4<double> c;
    const V4<double> ax = stencil4(lay.v0(smem, sp), lay.v0(smem, scur), lay.v0(smem, sn), s, c);
    const size_t off = cell_offset(s, t);
    const V4<double> bv = ldg4(b + off);
    V4<float> rf;
    float d = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double rv = bv.v[i] - ax.v[i];
      acc64 = fma(rv, rv, acc64);
      rf.v[i] = (float)rv;
      d = fmaf(rf.v[i], rf.v[i], d);
    }
    st4(xout + off, c);
    st4(r32 + off, rf);
    acc32 += (double)d;
  };
  stream_slab<double, float, 2>(s, smem, bars, xin, x32, err, conv, body);
  double v[2] = {acc64, acc32}, tot[2];
  if (grid_reduce_last<2>(v, partials, counter, tot) && threadIdx.x == 0) {
    const double rr64 = tot[0], rr = tot[1];
    sc->xsel = sel ^ 1;
    sc->x32_reset = 1;
    sc->true_rr = rr64;
    if (mode == 0) {
      sc->rr = rr;
      sc->rr_prev = rr;
      sc->beta = 0.0;
      sc->rmax2 = rr;
      sc->iter = 0;
    } else {
      sc->updates += 1;
      // continue the recursion from the recomputed residual
      sc->beta = rr / sc->rr_prev;
      sc->rr = rr;
      sc->rmax2 = rr;
    }
    sc->need_update = 0;
    sc->final_check = 0;
    if (!isfinite(rr64)) sc->done = 3;
    else if (rr64 <= sc->tol2) sc->done = 1;
    else if (mode == 1 && sc->iter >= sc->maxit) sc->done = 2;
  }
}

// ---------------------------------------------------------------------------
// Streaming helpers: sums, projection, copy-out.
// ---------------------------------------------------------------------------
// sc->sum0 = sum(a), sc->sum1 = sum(b) (b may be null).
__global__ void __launch_bounds__(256) k_sum2(const double* __restrict__ a, const double* __restrict__ b, size_t n4,
                                              Scalars* sc, double* partials, unsigned* counter) {
  double s0 = 0.0, s1 = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const V4<double> av = ldg4(a + 4 * i);
    s0 += (av.v[0] + av.v[1]) + (av.v[2] + av.v[3]);
    if (b) {
      const V4<double> bv = ldg4(b + 4 * i);
      s1 += (bv.v[0] + bv.v[1]) + (bv.v[2] + bv.v[3]);
    }
  }
  double v[2] = {s0, s1}, tot[2];
  if (grid_reduce_last<2>(v, partials, counter, tot) && threadIdx.x == 0) {
    sc->sum0 = tot[0];
    sc->sum1 = tot[1];
  }
}

// b = h^2 (rho - mean(rho)); x = phi - mean(phi); (b, b) -> bb, tol2.
__global__ void __launch_bounds__(256) k_project(const double* __restrict__ rho, const double* __restrict__ phi,
                                                 double* __restrict__ b, double* __restrict__ x, size_t n4,
                                                 double inv_n, double h2, double tol, Scalars* sc, double* partials,
                                                 unsigned* counter) {
  const double m0 = sc->sum0 * inv_n, m1 = sc->sum1 * inv_n;
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    V4<double> rv = ldg4(rho + 4 * i), pv = ldg4(phi + 4 * i);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      rv.v[k] = h2 * (rv.v[k] - m0);
      pv.v[k] -= m1;
      acc = fma(rv.v[k], rv.v[k], acc);
    }
    st4(b + 4 * i, rv);
    st4(x + 4 * i, pv);
  }
  double v[1] = {acc}, tot[1];
  if (grid_reduce_last<1>(v, partials, counter, tot) && threadIdx.x == 0) {
    sc->bb = tot[0];
    sc->tol2 = tol * tol * tot[0];
    sc->done = !isfinite(tot[0]) ? 3 : (tot[0] == 0.0 ? 1 : 0);  // zero rhs: phi = 0
    sc->need_update = 0;
    sc->final_check = 0;
    sc->updates = 0;
    sc->fallbacks = 0;
  }
}

// phi = x - mean(x) (sc->sum0 = sum(x)); phi = 0 when the right-hand side is zero.
__global__ void __launch_bounds__(256) k_finish(const double* __restrict__ x, double* __restrict__ phi, size_t n4,
                                                double inv_n, const Scalars* sc) {
  const bool zero = !(sc->bb > 0.0);
  const double m = sc->sum0 * inv_n;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    V4<double> v = ldg4(x + 4 * i);
#pragma unroll
    for (int k = 0; k < 4; ++k) v.v[k] = zero ? 0.0 : v.v[k] - m;
    st4(phi + 4 * i, v);
  }
}

// y = A x = (h^2 A) x / h^2 in FP64.
__global__ void __launch_bounds__(256) k_apply64(const double* __restrict__ x, double* __restrict__ y, double inv_h2,
                                                 int* err, StreamGeo g) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  const Slab s = make_slab(g);
  const StageLayout<double, double, 1> lay(s.rows, s.N);
  auto conv = [&](int) {};
  auto body = [&](int t, int sp, int scur, int sn) {
    if (!s.active) return;
    V4<double> c;
    V4<double> ax = stencil4(lay.v0(smem, sp), lay.v0(smem, scur), lay.v0(smem, sn), s, c);
#pragma unroll
    for (int i = 0; i < 4; ++i) ax.v[i] *= inv_h2;
    st4(y + cell_offset(s, t), ax);
  };
  stream_slab<double, double, 1>(s, smem, bars, x, (const double*)nullptr, err, conv, body);
}

}  // namespace pic
