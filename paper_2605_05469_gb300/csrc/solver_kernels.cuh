// Conjugate-gradient kernels on the periodic 7-point operator (Sec. 3.2).
//
// All solves run on the scaled system (h^2 A) x = h^2 b, whose operator
// 6 I - (sum of neighbours) has integer coefficients. With the constant
// Jacobi diagonal 6/h^2 folded into the scalars, Jacobi-PCG and CG produce
// the same iterates, so the preconditioner costs nothing per cell.
//
// One iteration is two kernels (plus, for flexible CG, the preconditioner and
// a dot-product kernel), each a single pass over the grid with its reduction
// finished on the device by the last block (alpha and beta never leave the
// GPU):
//   pap   : p = r + beta p_in (on the whole streamed slab incl. halo),
//           writes p and q = A p, reduces (p, A p) -> alpha;
//   update: x += alpha p, r -= alpha q (q stored by pap; FP64, or the FP32
//           streaming update of the mixed-precision solvers), reduces
//           (r, r) -> beta, convergence and iteration count.
#pragma once
#include "stream.cuh"

namespace pic {

// ---------------------------------------------------------------------------
// pap: p = r + beta p_in over the streamed slab; q = (h^2 A) p; (p, q) -> alpha
// ---------------------------------------------------------------------------
template <typename T, bool STORE_Q, bool TALL = false>
__global__ void __launch_bounds__(TALL ? kStreamTall : kStreamSmall) k_cg_pap(const T* __restrict__ r, const T* __restrict__ pin,
                                                T* __restrict__ pout, T* __restrict__ q, Scalars* sc,
                                                double* partials, unsigned* counter, int* err, StreamGeo g) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  if (sc->done) return;
  const T beta = (T)sc->beta;
  const StageLayout<T, T, 2> lay(g.rows, g.N);
  double dot = 0.0;  // FP64 path
  CompSum dot32;     // FP32 path
  auto ingest = [&](int st, size_t e, const Slab&, int) {
    const V4<T> rv = ld4(lay.v0(smem, st) + e);
    V4<T> pv = ld4(lay.v1(smem, st) + e);
#pragma unroll
    for (int i = 0; i < 4; ++i) pv.v[i] = rv.v[i] + beta * pv.v[i];
    return pv;
  };
  auto start = [&](const Slab&) {};
  auto body = [&](const Slab& s, int t, const T* pb, const V4<T>& zm, const V4<T>& c, const V4<T>& zp) {
    const V4<T> ap = stencil_q(pb, s, zm, c, zp);
    const size_t off = cell_offset(s, t);
    st4(pout + off, c);
    if (STORE_Q) st4(q + off, ap);
    T d = c.v[0] * ap.v[0];
#pragma unroll
    for (int i = 1; i < 4; ++i) d += c.v[i] * ap.v[i];
    if (sizeof(T) == 8) dot += (double)d;
    else dot32.add((float)d);
  };
  stream_slab<T, T, T, 2>(g, smem, bars, r, pin, err, start, ingest, body);
  double v[1] = {sizeof(T) == 8 ? dot : dot32.value()}, tot[1];
  if (grid_reduce_last<1>(v, partials, counter, tot) && threadIdx.x == 0) {
    const double pq = tot[0];
    sc->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
      sc->done = 3;
    } else {
      sc->alpha = (sc->fcg ? sc->rz : sc->rr) / pq;
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
// FP32 update of the mixed-precision solvers (Jacobi-CG and flexible CG),
// where q = (h^2 A) p was stored by the direction kernel: x += alpha p,
// r -= alpha q as a plain stream (no stencil, no halo), (r, r) -> beta, and a
// reliable update is triggered when (r, r) fell by delta^2 since the last one
// or reached the tolerance.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fcg_update32(float* __restrict__ x, float* __restrict__ r,
                                                      const float* __restrict__ p, const float* __restrict__ q,
                                                      size_t n4, Scalars* sc, double* partials, unsigned* counter) {
  if (sc->done) return;
  const float alpha = (float)sc->alpha;
  const bool x_zero = sc->x32_reset != 0;
  CompSum acc;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const V4<float> pv = ldg4(p + 4 * i), qv = ldg4(q + 4 * i);
    V4<float> xv = x_zero ? V4<float>{{0.f, 0.f, 0.f, 0.f}} : ld4(x + 4 * i);
    V4<float> rv = ld4(r + 4 * i);
    float d = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      xv.v[k] = fmaf(alpha, pv.v[k], xv.v[k]);
      rv.v[k] = fmaf(-alpha, qv.v[k], rv.v[k]);
      d = fmaf(rv.v[k], rv.v[k], d);
    }
    st4(x + 4 * i, xv);
    st4(r + 4 * i, rv);
    acc.add(d);
  }
  double v[1] = {acc.value()}, tot[1];
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
// Initial FP64 residual of the FP64 reference solve: r = h^2 b - (h^2 A) x, (r, r).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kStreamSmall) k_residual64(const double* __restrict__ x, const double* __restrict__ b,
                                                    double* __restrict__ r, Scalars* sc, double* partials,
                                                    unsigned* counter, int* err, StreamGeo g) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  if (sc->done) return;
  const StageLayout<double, double, 1> lay(g.rows, g.N);
  double acc = 0.0;
  V4<double> cb;
  auto start = [&](const Slab& s) { cb = ldg4(b + cell_offset(s, 0)); };
  auto ingest = [&](int st, size_t e, const Slab&, int) { return ld4(lay.v0(smem, st) + e); };
  auto body = [&](const Slab& s, int t, const double* pb, const V4<double>& zm, const V4<double>& c,
                  const V4<double>& zp) {
    V4<double> nb = cb;
    if (t + 1 < s.ZC) nb = ldg4(b + cell_offset(s, t + 1));
    const V4<double> ax = stencil_q(pb, s, zm, c, zp);
    const size_t off = cell_offset(s, t);
    const V4<double> bv = cb;
    cb = nb;
    V4<double> rv;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      rv.v[i] = bv.v[i] - ax.v[i];
      acc = fma(rv.v[i], rv.v[i], acc);
    }
    st4(r + off, rv);
  };
  stream_slab<double, double, double, 1>(g, smem, bars, x, (const double*)nullptr, err, start, ingest, body);
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
__global__ void __launch_bounds__(kStreamSmall) k_reliable(double* __restrict__ x64a, double* __restrict__ x64b,
                                                  const float* __restrict__ x32, const double* __restrict__ b,
                                                  float* __restrict__ r32, Scalars* sc, double* partials,
                                                  unsigned* counter, int* err, StreamGeo g, int mode) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  if (mode == 0 && sc->done) return;
  if (mode == 1 && (sc->done || !sc->need_update)) return;
  const int sel = sc->xsel;
  const double* xin = sel ? x64b : x64a;
  double* xout = sel ? x64a : x64b;
  // x32 holds a stale correction that has already been folded: read it as zero
  const bool x32_zero = sc->x32_reset != 0;
  const StageLayout<double, float, 2> lay(g.rows, g.N);
  double acc64 = 0.0;
  CompSum acc32;
  V4<double> cb;
  auto start = [&](const Slab& s) { cb = ldg4(b + cell_offset(s, 0)); };
  auto ingest = [&](int st, size_t e, const Slab&, int) {
    V4<double> xv = ld4(lay.v0(smem, st) + e);
    if (!x32_zero) {
      const V4<float> yv = ld4(lay.v1(smem, st) + e);
#pragma unroll
      for (int i = 0; i < 4; ++i) xv.v[i] += (double)yv.v[i];
    }
    return xv;
  };
  auto body = [&](const Slab& s, int t, const double* pb, const V4<double>& zm, const V4<double>& c,
                  const V4<double>& zp) {
    V4<double> nb = cb;
    if (t + 1 < s.ZC) nb = ldg4(b + cell_offset(s, t + 1));
    const V4<double> ax = stencil_q(pb, s, zm, c, zp);
    const size_t off = cell_offset(s, t);
    const V4<double> bv = cb;
    cb = nb;
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
    acc32.add(d);
  };
  stream_slab<double, double, float, 2>(g, smem, bars, xin, x32, err, start, ingest, body);
  double v[2] = {acc64, acc32.value()}, tot[2];
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
      if (mode == 1) sc->updates += 1;  // the forced final fold (mode 2) is not a reliable update
      // continue the recursion from the recomputed residual
      sc->beta = rr / sc->rr_prev;
      sc->rr = rr;
      sc->rmax2 = rr;
      if (mode == 1) sc->redo = 1;
    }
    sc->need_update = 0;
    sc->final_check = 0;
    if (!isfinite(rr64)) sc->done = 3;
    else if (rr64 <= sc->tol2) sc->done = 1;
    else if (mode == 1 && sc->iter >= sc->maxit) sc->done = 2;
    else if (mode == 1 && sc->refine_max > 0 && sc->updates >= sc->refine_max) sc->done = 2;
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
    sc->redo = 0;
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

// ---------------------------------------------------------------------------
// Flexible CG, FCG(1) (Notay 2000), with a nonlinear preconditioner z = P(r):
// the new direction is z made A-conjugate to the previous p,
// beta = -(z, A p_prev) / (p_prev, A p_prev), with A p_prev = q stored by the
// pap kernel and (p_prev, A p_prev) = sc->pq. Reduces (r, z), (z, q), (r, q).
// Descent guard: when (r, z) <= 0 or is not finite the iteration uses the
// Jacobi direction z = r / 6 (scaled operator diagonal), whose dots follow
// from (r, r) and (r, q). init: first direction, beta = 0.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fcg_dot(const float* __restrict__ r, const float* __restrict__ z,
                                                 const float* __restrict__ q, size_t n4, Scalars* sc,
                                                 double* partials, unsigned* counter, int init, int only_redo) {
  if (sc->done) return;
  if (only_redo && !sc->redo) return;
  CompSum arz, azq, arq;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const V4<float> rv = ldg4(r + 4 * i), zv = ldg4(z + 4 * i);
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
    if (init) {
#pragma unroll
      for (int k = 0; k < 4; ++k) d0 = fmaf(rv.v[k], zv.v[k], d0);
    } else {
      const V4<float> qv = ldg4(q + 4 * i);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        d0 = fmaf(rv.v[k], zv.v[k], d0);
        d1 = fmaf(zv.v[k], qv.v[k], d1);
        d2 = fmaf(rv.v[k], qv.v[k], d2);
      }
    }
    arz.add(d0);
    azq.add(d1);
    arq.add(d2);
  }
  double v[3] = {arz.value(), azq.value(), arq.value()}, tot[3];
  if (grid_reduce_last<3>(v, partials, counter, tot) && threadIdx.x == 0) {
    double rz = tot[0], zq = tot[1];
    sc->fallback_now = 0;
    if (!(rz > 0.0) || !isfinite(rz) || !isfinite(zq)) {
      sc->fallback_now = 1;
      sc->fallbacks += 1;
      rz = sc->rr / 6.0;
      zq = tot[2] / 6.0;
    }
    sc->beta = init ? 0.0 : -zq / sc->pq;
    sc->rz = rz;
    sc->redo = 0;
    if (!isfinite(sc->beta)) sc->done = 3;
  }
}

__global__ void __launch_bounds__(256) k_fcg_fallback(const float* __restrict__ r, float* __restrict__ z,
                                                      size_t n4, const Scalars* sc) {
  if (sc->done || !sc->fallback_now) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    V4<float> v = ldg4(r + 4 * i);
#pragma unroll
    for (int k = 0; k < 4; ++k) v.v[k] *= (1.0f / 6.0f);
    st4(z + 4 * i, v);
  }
}

// a *= s (elementwise, FP64).
__global__ void __launch_bounds__(256) k_scale64(double* __restrict__ a, size_t n4, double sc) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    V4<double> v = ldg4(a + 4 * i);
#pragma unroll
    for (int k = 0; k < 4; ++k) v.v[k] *= sc;
    st4(a + 4 * i, v);
  }
}

// y = A x = (h^2 A) x / h^2 in FP64.
__global__ void __launch_bounds__(kStreamSmall) k_apply64(const double* __restrict__ x, double* __restrict__ y, double inv_h2,
                                                 int* err, StreamGeo g) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  const StageLayout<double, double, 1> lay(g.rows, g.N);
  auto start = [&](const Slab&) {};
  auto ingest = [&](int st, size_t e, const Slab&, int) { return ld4(lay.v0(smem, st) + e); };
  auto body = [&](const Slab& s, int t, const double* pb, const V4<double>& zm, const V4<double>& c,
                  const V4<double>& zp) {
    V4<double> ax = stencil_q(pb, s, zm, c, zp);
#pragma unroll
    for (int i = 0; i < 4; ++i) ax.v[i] *= inv_h2;
    st4(y + cell_offset(s, t), ax);
  };
  stream_slab<double, double, double, 1>(g, smem, bars, x, (const double*)nullptr, err, start, ingest, body);
}

// Self-test of the bounded device wait (mbar_wait_bounded): one warp waits on
// an mbarrier of one expected arrival; with `producer` lane 1 arrives, else
// nothing does and the wait gives up after budget_ns, recording
// DEV_ERR_TIMEOUT. No copy is ever issued, so nothing is in flight when the
// warp leaves.
__global__ void k_selftest_wait(uint64_t budget_ns, int producer, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (producer && threadIdx.x == 1)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  mbar_wait_bounded(&bar, 0, err, budget_ns);
}

}  // namespace pic
