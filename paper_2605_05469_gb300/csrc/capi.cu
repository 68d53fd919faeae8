// C ABI of the PIC library: context, buffers and the drivers that enqueue the
// kernels of each call on the context's stream. See include/pic.h.
#include <math.h>
#include <string.h>

#include <new>

#include "cnn.h"
#include "mg.h"
#include "fft.h"
#include "pif.h"
#include "ssor.h"
#include "ctx.h"
#include "particle_kernels.cuh"
#include "slab_geo.h"
#include "solver_kernels.cuh"

using namespace pic;

namespace {

void free_particles(pic_ctx* c) {
  for (int b = 0; b < 2; ++b) {
    dfree(c->prec[b]);
  }
  dfree(c->counts);
  dfree(c->offsets);
  dfree(c->chunks);
  dfree(c->E);
  dfree(c->dep);
  dfree(c->pif_E);
  dfree(c->stage);
  c->np = 0;
}

// Particles per chunk of a host transfer (6 FP64 blocks: 805 MB per staging
// buffer, two buffers).
constexpr uint64_t kStageParticles = 1ull << 24;

int ensure_stage(pic_ctx* c) {
  int e;
  if (!c->stage && (e = dalloc(&c->stage, 2 * 6 * kStageParticles))) return e;
  if (!c->io_flag && (e = dalloc(&c->io_flag, 1))) return e;
  if (!c->io_stream) CK(cudaStreamCreateWithFlags(&c->io_stream, cudaStreamNonBlocking));
  for (int i = 0; i < 5; ++i)
    if (!c->io_ev[i]) CK(cudaEventCreateWithFlags(&c->io_ev[i], cudaEventDisableTiming));
  return PIC_OK;
}

double* stage_buf(pic_ctx* c, int b) { return c->stage + (size_t)b * 6 * kStageParticles; }

void free_solver(pic_ctx* c) {
  SolverWs& w = c->ws;
  dfree(w.x); dfree(w.r); dfree(w.p[0]); dfree(w.p[1]); dfree(w.q);
  dfree(w.xm[0]); dfree(w.xm[1]);
  dfree(w.x32); dfree(w.r32); dfree(w.r32b); dfree(w.p32[0]); dfree(w.p32[1]);
  dfree(w.z32[0]); dfree(w.z32[1]); dfree(w.q32);
  dfree(w.b);
  dfree(c->partials);
  c->partials_len = 0;
}

PRec* pptrs(pic_ctx* c, int b) { return c->prec[b]; }

// Slab geometry of a plane-streaming kernel on the context grid.
template <typename TP, typename A, typename B, int NV, typename K>
int geo_for(pic_ctx* c, K kernel, StreamGeo* out, size_t* smem, bool tall = false) {
  return slab_geometry<TP, A, B, NV>(c, c->N, kernel, out, smem, tall);
}

int streaming_blocks(pic_ctx* c) {
  size_t n4 = c->n / 4;
  size_t b = (n4 + 255) / 256;
  size_t cap = (size_t)c->sms * 4;
  return (int)(b < cap ? b : cap);
}

int ensure_partials(pic_ctx* c, size_t need) {
  if (c->partials_len >= need) return PIC_OK;
  dfree(c->partials);
  int e = dalloc(&c->partials, need);
  if (e) return e;
  c->partials_len = need;
  return PIC_OK;
}

int check_dev_err(pic_ctx* c) {
  // caller has synchronised; the faults stay recorded for the context's life
  if (*c->err_host & DEV_ERR_TIMEOUT) return PIC_ETIMEOUT;
  if (*c->err_host & DEV_ERR_NONFINITE) return PIC_EBREAKDOWN;  // a push met a non-finite field
  return PIC_OK;
}

int sync_status(pic_ctx* c) {
  CK(cudaMemcpyAsync(c->err_host, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return check_dev_err(c);
}


bool dev_ptr_ok(const void* p) { return p != nullptr && ((uintptr_t)p % 16) == 0; }

// --------------------------------------------------------------------------
// FP64 Jacobi-PCG (the reference solve)
// --------------------------------------------------------------------------
int solve_common_setup(pic_ctx* c, const double* rho, const double* phi, double tol, int maxit, double delta,
                       double* xout, int refine_max = 0) {
  Scalars init;
  memset(&init, 0, sizeof(init));
  init.maxit = maxit;
  init.delta2 = delta * delta;
  init.refine_max = refine_max;
  init.xsel = 0;
  c->sc_host[0] = init;
  CK(cudaMemcpyAsync(c->sc, &c->sc_host[0], sizeof(Scalars), cudaMemcpyHostToDevice, c->stream));
  const int sb = streaming_blocks(c);
  const size_t n4 = c->n / 4;
  launch(c, k_sum2, sb, 256, 0, rho, phi, n4, c->sc, c->partials, c->counter);
  launch(c, k_project, sb, 256, 0, rho, phi, c->ws.b, xout, n4, 1.0 / (double)c->n, c->h * c->h, tol, c->sc,
                                      c->partials, c->counter);
  CK(cudaGetLastError());
  return PIC_OK;
}

// Run batches of `m` iterations (each batch a fixed launch sequence) until the
// device reports done. The status of batch b-1 is read while batch b runs.
template <typename LaunchBatch>
int run_batches(pic_ctx* c, int m, int maxit, LaunchBatch launch_batch) {
  int b = 0;
  long launched = 0;
  for (;;) {
    launch_batch();
    CK(cudaGetLastError());
    launched += m;
    CK(cudaMemcpyAsync(&c->sc_host[b & 1], c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaEventRecord(c->batch_ev[b & 1], c->stream));
    if (b > 0) {
      CK(cudaEventSynchronize(c->batch_ev[(b - 1) & 1]));
      if (c->sc_host[(b - 1) & 1].done) break;
    }
    if (launched > (long)maxit + 2L * m) break;
    ++b;
  }
  return PIC_OK;
}

int solve_fp64(pic_ctx* c, const double* rho, double* phi, double tol, int maxit, int m, pic_solve_info* info) {
  SolverWs& w = c->ws;
  int e;
  if (!w.x) {
    if ((e = dalloc(&w.x, c->n)) || (e = dalloc(&w.r, c->n)) || (e = dalloc(&w.p[0], c->n)) ||
        (e = dalloc(&w.p[1], c->n)) || (e = dalloc(&w.q, c->n)))
      return e;
  }
  if (!w.b && (e = dalloc(&w.b, c->n))) return e;
  size_t smem_pap, smem_res;
  StreamGeo gp, gr;
  if ((e = geo_for<double, double, double, 2>(c, k_cg_pap<double, true>, &gp, &smem_pap))) return e;
  if ((e = geo_for<double, double, double, 1>(c, k_residual64, &gr, &smem_res))) return e;
  if ((e = ensure_partials(c, (size_t)3 * (gp.blocks > gr.blocks ? gp.blocks : gr.blocks) + 3 * 4096))) return e;

  CK(cudaEventRecord(c->ev0, c->stream));
  if ((e = solve_common_setup(c, rho, phi, tol, maxit, 0.0, w.x))) return e;
  CK(cudaMemsetAsync(w.p[0], 0, c->n * sizeof(double), c->stream));
  const int tp = round32(gp.threads), tr = round32(gr.threads);
  launch(c, k_residual64, gr.blocks, tr, smem_res, w.x, w.b, w.r, c->sc, c->partials, c->counter, c->err, gr);
  const int sb = streaming_blocks(c);
  const size_t n4 = c->n / 4;
  int cur = 0;
  auto batch = [&]() {
    for (int i = 0; i < m; ++i) {
      const bool sample = c->prof_on && i == 0;
      int slot = sample ? c->ker[PIC_KER_PAP].begin(c->stream) : -1;
      launch(c, k_cg_pap<double, true>, gp.blocks, tp, smem_pap, w.r, w.p[cur], w.p[cur ^ 1], w.q, c->sc,
             c->partials, c->counter, c->err, gp);
      if (sample) c->ker[PIC_KER_PAP].end(slot, c->stream);
      slot = sample ? c->ker[PIC_KER_UPDATE].begin(c->stream) : -1;
      launch(c, k_cg_update64, sb, 256, 0, w.x, w.r, w.p[cur ^ 1], w.q, n4, c->sc, c->partials, c->counter);
      if (sample) c->ker[PIC_KER_UPDATE].end(slot, c->stream);
      cur ^= 1;
    }
  };
  if ((e = run_batches(c, m, maxit, batch))) return e;
  launch(c, k_sum2, sb, 256, 0, w.x, nullptr, n4, c->sc, c->partials, c->counter);
  launch(c, k_finish, sb, 256, 0, w.x, phi, n4, 1.0 / (double)c->n, c->sc);
  CK(cudaGetLastError());
  CK(cudaEventRecord(c->ev1, c->stream));
  CK(cudaMemcpyAsync(&c->sc_host[0], c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
  if ((e = sync_status(c))) return e;
  if (c->prof_on) {
    for (int kk = 0; kk < PIC_NKER; ++kk) {
      c->ker[kk].flush();
      c->ker_prec[kk] = PIC_PREC_FP64;
    }
  }
  const Scalars& s = c->sc_host[0];
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    info->iters = s.iter;
    info->reliable_updates = 0;
    info->fallbacks = 0;
    info->converged = s.done == 1;
    info->rel_res = s.bb > 0.0 ? sqrt(s.rr / s.bb) : 0.0;
    info->bnorm = sqrt(s.bb) / (c->h * c->h);
    info->t_ms = ms;
  }
  if (s.done == 1) return PIC_OK;
  if (s.done == 3) return PIC_EBREAKDOWN;
  return PIC_ENOCONV;
}

// --------------------------------------------------------------------------
// Mixed precision: FP32 CG with FP64 reductions and reliable updates
// --------------------------------------------------------------------------
int solve_mixed(pic_ctx* c, const double* rho, double* phi, double tol, int maxit, int m, double delta, int refine_max,
                pic_solve_info* info) {
  SolverWs& w = c->ws;
  int e;
  if (!w.xm[0]) {
    if ((e = dalloc(&w.xm[0], c->n)) || (e = dalloc(&w.xm[1], c->n)) || (e = dalloc(&w.x32, c->n)) ||
        (e = dalloc(&w.r32, c->n)) || (e = dalloc(&w.p32[0], c->n)) || (e = dalloc(&w.p32[1], c->n)))
      return e;
  }
  if (!w.b && (e = dalloc(&w.b, c->n))) return e;
  // the direction kernel stores q = A p, so the update streams x, r, p, q
  // (no stencil): more bytes than recomputing A p, but at streaming speed
  if (!w.q32 && (e = dalloc(&w.q32, c->n))) return e;
  size_t smem_pap, smem_rel;
  StreamGeo gp, gr;
  const bool tall = c->N >= 512;
  auto* kpap = tall ? k_cg_pap<float, true, true> : k_cg_pap<float, true, false>;
  if ((e = geo_for<float, float, float, 2>(c, kpap, &gp, &smem_pap, tall))) return e;
  if ((e = geo_for<double, double, float, 2>(c, k_reliable, &gr, &smem_rel))) return e;
  const int sb = streaming_blocks(c);
  const size_t n4 = c->n / 4;
  int mb = gp.blocks;
  if (sb > mb) mb = sb;
  if (gr.blocks > mb) mb = gr.blocks;
  if ((e = ensure_partials(c, (size_t)3 * mb + 3 * 4096))) return e;

  CK(cudaEventRecord(c->ev0, c->stream));
  if ((e = solve_common_setup(c, rho, phi, tol, maxit, delta, w.xm[0], refine_max))) return e;
  CK(cudaMemsetAsync(w.x32, 0, c->n * sizeof(float), c->stream));
  CK(cudaMemsetAsync(w.p32[0], 0, c->n * sizeof(float), c->stream));
  const int tp = round32(gp.threads), tr = round32(gr.threads);
  launch(c, k_reliable, gr.blocks, tr, smem_rel, w.xm[0], w.xm[1], w.x32, w.b, w.r32, c->sc, c->partials,
                                                    c->counter, c->err, gr, 0);
  int cur = 0;
  auto batch = [&]() {
    for (int i = 0; i < m; ++i) {
      const bool sample = c->prof_on && i == 0;
      int slot = sample ? c->ker[PIC_KER_PAP].begin(c->stream) : -1;
      launch(c, kpap, gp.blocks, tp, smem_pap, w.r32, w.p32[cur], w.p32[cur ^ 1], w.q32,
             c->sc, c->partials, c->counter, c->err, gp);
      if (sample) c->ker[PIC_KER_PAP].end(slot, c->stream);
      slot = sample ? c->ker[PIC_KER_UPDATE].begin(c->stream) : -1;
      launch(c, k_fcg_update32, sb, 256, 0, w.x32, w.r32, (const float*)w.p32[cur ^ 1], (const float*)w.q32, n4,
             c->sc, c->partials, c->counter);
      if (sample) c->ker[PIC_KER_UPDATE].end(slot, c->stream);
      launch(c, k_reliable, gr.blocks, tr, smem_rel, w.xm[0], w.xm[1], w.x32, w.b, w.r32, c->sc, c->partials,
                                                        c->counter, c->err, gr, 1);
      cur ^= 1;
    }
  };
  if ((e = run_batches(c, m, maxit, batch))) return e;
  CK(cudaMemcpyAsync(&c->sc_host[0], c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
  if ((e = sync_status(c))) return e;
  if (c->sc_host[0].done != 1 && c->sc_host[0].done != 3) {
    // fold the last FP32 correction and measure the true residual
    launch(c, k_reliable, gr.blocks, tr, smem_rel, w.xm[0], w.xm[1], w.x32, w.b, w.r32, c->sc, c->partials,
                                                      c->counter, c->err, gr, 2);
    CK(cudaMemcpyAsync(&c->sc_host[0], c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
    if ((e = sync_status(c))) return e;
  }
  const int sel = c->sc_host[0].xsel;
  launch(c, k_sum2, sb, 256, 0, w.xm[sel], nullptr, n4, c->sc, c->partials, c->counter);
  launch(c, k_finish, sb, 256, 0, w.xm[sel], phi, n4, 1.0 / (double)c->n, c->sc);
  CK(cudaGetLastError());
  CK(cudaEventRecord(c->ev1, c->stream));
  CK(cudaMemcpyAsync(&c->sc_host[0], c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
  if ((e = sync_status(c))) return e;
  if (c->prof_on) {
    for (int kk = 0; kk < PIC_NKER; ++kk) {
      c->ker[kk].flush();
      c->ker_prec[kk] = PIC_PREC_MIXED;
    }
  }
  const Scalars& s = c->sc_host[0];
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    info->iters = s.iter;
    info->reliable_updates = s.updates;
    info->fallbacks = s.fallbacks;
    info->converged = s.done == 1;
    info->rel_res = s.bb > 0.0 ? sqrt(s.true_rr / s.bb) : 0.0;
    info->bnorm = sqrt(s.bb) / (c->h * c->h);
    info->t_ms = ms;
  }
  if (s.done == 1) return PIC_OK;
  if (s.done == 3) return PIC_EBREAKDOWN;
  return PIC_ENOCONV;
}

// --------------------------------------------------------------------------
// Flexible CG, FCG(1) (Notay 2000), with the learned preconditioner, FP32
// vectors with FP64 reductions and reliable updates (as the mixed path). One
// iteration: pap (p = z + beta p, q = A p, alpha = (r,z)/(p,q)), update,
// reliable update if due, network z = s N(r/s), dots (r,z), (z,q), (r,q) with
// the descent guard and beta = -(z,q)/(p,q), Jacobi fallback if it fired.
// --------------------------------------------------------------------------
int solve_fcg(pic_ctx* c, const double* rho, double* phi, double tol, int maxit, int m, double delta, int refine_max,
              int pc,
              pic_solve_info* info) {
  SolverWs& w = c->ws;
  int e;
  const bool uses_net = pc == PIC_PC_CNN || pc == PIC_PC_MG_CNN;
  if (uses_net && !cnn_ready(c)) return PIC_ESTATE;
  if (pc == PIC_PC_CNN && c->N % 16 != 0) return PIC_EINVAL;
  // z = M r for the chosen preconditioner (enqueued on the context stream)
  auto precond = [&](const float* r, float* z, bool sample) -> int {
    if (pc == PIC_PC_CNN) return cnn_apply(c, r, z, &c->sc->rr, c->n);
    if (pc == PIC_PC_SSOR) return ssor_apply(c, r, z, &c->sc->done);
    return mg_apply(c, r, z, pc == PIC_PC_MG_CNN, &c->sc->done, sample);
  };
  if (!w.xm[0]) {
    if ((e = dalloc(&w.xm[0], c->n)) || (e = dalloc(&w.xm[1], c->n)) || (e = dalloc(&w.x32, c->n)) ||
        (e = dalloc(&w.r32, c->n)) || (e = dalloc(&w.p32[0], c->n)) || (e = dalloc(&w.p32[1], c->n)))
      return e;
  }
  if (!w.z32[0] && ((e = dalloc(&w.z32[0], c->n)) || (e = dalloc(&w.z32[1], c->n)) || (e = dalloc(&w.q32, c->n))))
    return e;
  if (!w.b && (e = dalloc(&w.b, c->n))) return e;
  size_t smem_pap, smem_rel;
  StreamGeo gp, gr;
  const bool tall = c->N >= 512;
  auto* kpap = tall ? k_cg_pap<float, true, true> : k_cg_pap<float, true, false>;
  if ((e = geo_for<float, float, float, 2>(c, kpap, &gp, &smem_pap, tall))) return e;
  if ((e = geo_for<double, double, float, 2>(c, k_reliable, &gr, &smem_rel))) return e;
  int mb = gp.blocks;
  if (streaming_blocks(c) > mb) mb = streaming_blocks(c);
  if (gr.blocks > mb) mb = gr.blocks;
  if ((e = ensure_partials(c, (size_t)4 * mb + 3 * 4096))) return e;

  CK(cudaEventRecord(c->ev0, c->stream));
  if ((e = solve_common_setup(c, rho, phi, tol, maxit, delta, w.xm[0], refine_max))) return e;
  c->sc_host[1] = c->sc_host[0];
  c->sc_host[1].fcg = 1;
  CK(cudaMemcpyAsync(&c->sc->fcg, &c->sc_host[1].fcg, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(w.x32, 0, c->n * sizeof(float), c->stream));
  CK(cudaMemsetAsync(w.p32[0], 0, c->n * sizeof(float), c->stream));
  const int tp = round32(gp.threads), tr = round32(gr.threads);
  const int sb = streaming_blocks(c);
  const size_t n4 = c->n / 4;
  launch(c, k_reliable, gr.blocks, tr, smem_rel, w.xm[0], w.xm[1], (const float*)w.x32, (const double*)w.b, w.r32,
         c->sc, c->partials, c->counter, c->err, gr, 0);
  int zc = 0;
  if ((e = precond(w.r32, w.z32[zc], false))) return e;
  launch(c, k_fcg_dot, sb, 256, 0, (const float*)w.r32, (const float*)w.z32[zc], (const float*)w.q32, n4, c->sc,
         c->partials, c->counter, 1, 0);
  launch(c, k_fcg_fallback, sb, 256, 0, (const float*)w.r32, w.z32[zc], n4, (const Scalars*)c->sc);
  int cur = 0;
  int inner_err = PIC_OK;
  // Tensor-core preconditioner: the update, the preconditioner and the
  // direction's dots are one kernel; the residual ping-pongs between r32 and
  // r32b (rc = current). A reliable update (rare) replaces r, and then z and
  // the dots are recomputed from it by the redo kernels, which return at once
  // otherwise.
  const bool fused = pc == PIC_PC_CNN && cnn_fused_ok(c);
  if (fused && !w.r32b && (e = dalloc(&w.r32b, c->n))) return e;
  float* rbuf[2] = {w.r32, w.r32b};
  int rc = 0;
  auto batch_fused = [&]() {
    for (int i = 0; i < m; ++i) {
      const bool sample = c->prof_on && i == 0;
      int slot = sample ? c->ker[PIC_KER_PAP].begin(c->stream) : -1;
      launch(c, kpap, gp.blocks, tp, smem_pap, (const float*)w.z32[zc], (const float*)w.p32[cur],
             w.p32[cur ^ 1], w.q32, c->sc, c->partials, c->counter, c->err, gp);
      if (sample) c->ker[PIC_KER_PAP].end(slot, c->stream);
      slot = sample ? c->ker[PIC_KER_PRECOND].begin(c->stream) : -1;
      int ce = cnn_apply_fused(c, rbuf[rc], rbuf[rc ^ 1], w.z32[zc ^ 1], w.q32, w.p32[cur ^ 1], w.x32);
      if (sample) c->ker[PIC_KER_PRECOND].end(slot, c->stream);
      rc ^= 1;
      zc ^= 1;
      launch(c, k_reliable, gr.blocks, tr, smem_rel, w.xm[0], w.xm[1], (const float*)w.x32, (const double*)w.b,
             rbuf[rc], c->sc, c->partials, c->counter, c->err, gr, 1);
      if (!ce) ce = cnn_apply_redo(c, rbuf[rc], w.z32[zc]);
      if (ce && !inner_err) inner_err = ce;
      launch(c, k_fcg_dot, sb, 256, 0, (const float*)rbuf[rc], (const float*)w.z32[zc], (const float*)w.q32, n4,
             c->sc, c->partials, c->counter, 0, 1);
      launch(c, k_fcg_fallback, sb, 256, 0, (const float*)rbuf[rc], w.z32[zc], n4, (const Scalars*)c->sc);
      cur ^= 1;
    }
  };
  auto batch = [&]() {
    for (int i = 0; i < m; ++i) {
      const bool sample = c->prof_on && i == 0;
      int slot = sample ? c->ker[PIC_KER_PAP].begin(c->stream) : -1;
      launch(c, kpap, gp.blocks, tp, smem_pap, (const float*)w.z32[zc], (const float*)w.p32[cur],
             w.p32[cur ^ 1], w.q32, c->sc, c->partials, c->counter, c->err, gp);
      if (sample) c->ker[PIC_KER_PAP].end(slot, c->stream);
      slot = sample ? c->ker[PIC_KER_UPDATE].begin(c->stream) : -1;
      launch(c, k_fcg_update32, sb, 256, 0, w.x32, w.r32, (const float*)w.p32[cur ^ 1], (const float*)w.q32, n4,
             c->sc, c->partials, c->counter);
      if (sample) c->ker[PIC_KER_UPDATE].end(slot, c->stream);
      launch(c, k_reliable, gr.blocks, tr, smem_rel, w.xm[0], w.xm[1], (const float*)w.x32, (const double*)w.b,
             w.r32, c->sc, c->partials, c->counter, c->err, gr, 1);
      zc ^= 1;
      slot = sample ? c->ker[PIC_KER_PRECOND].begin(c->stream) : -1;
      const int ce = precond(w.r32, w.z32[zc], sample);
      if (sample) c->ker[PIC_KER_PRECOND].end(slot, c->stream);
      if (ce && !inner_err) inner_err = ce;
      slot = sample ? c->ker[PIC_KER_DOT].begin(c->stream) : -1;
      launch(c, k_fcg_dot, sb, 256, 0, (const float*)w.r32, (const float*)w.z32[zc], (const float*)w.q32, n4, c->sc,
             c->partials, c->counter, 0, 0);
      if (sample) c->ker[PIC_KER_DOT].end(slot, c->stream);
      launch(c, k_fcg_fallback, sb, 256, 0, (const float*)w.r32, w.z32[zc], n4, (const Scalars*)c->sc);
      cur ^= 1;
    }
  };
  if (fused) {
    if ((e = run_batches(c, m, maxit, batch_fused))) return e;
  } else {
    if ((e = run_batches(c, m, maxit, batch))) return e;
  }
  if (inner_err) return inner_err;
  CK(cudaMemcpyAsync(&c->sc_host[0], c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
  if ((e = sync_status(c))) return e;
  if (c->sc_host[0].done != 1 && c->sc_host[0].done != 3) {
    launch(c, k_reliable, gr.blocks, tr, smem_rel, w.xm[0], w.xm[1], (const float*)w.x32, (const double*)w.b,
           rbuf[rc], c->sc, c->partials, c->counter, c->err, gr, 2);
    CK(cudaMemcpyAsync(&c->sc_host[0], c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
    if ((e = sync_status(c))) return e;
  }
  const int sel = c->sc_host[0].xsel;
  launch(c, k_sum2, sb, 256, 0, (const double*)w.xm[sel], (const double*)nullptr, n4, c->sc, c->partials,
         c->counter);
  launch(c, k_finish, sb, 256, 0, (const double*)w.xm[sel], phi, n4, 1.0 / (double)c->n, (const Scalars*)c->sc);
  CK(cudaGetLastError());
  CK(cudaEventRecord(c->ev1, c->stream));
  CK(cudaMemcpyAsync(&c->sc_host[0], c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
  if ((e = sync_status(c))) return e;
  if (c->prof_on) {
    for (int kk = 0; kk < PIC_NKER; ++kk) {
      c->ker[kk].flush();
      c->ker_prec[kk] = PIC_PREC_MIXED;
    }
  }
  const Scalars& s = c->sc_host[0];
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    info->iters = s.iter;
    info->reliable_updates = s.updates;
    info->fallbacks = s.fallbacks;
    info->converged = s.done == 1;
    info->rel_res = s.bb > 0.0 ? sqrt(s.true_rr / s.bb) : 0.0;
    info->bnorm = sqrt(s.bb) / (c->h * c->h);
    info->t_ms = ms;
  }
  if (s.done == 1) return PIC_OK;
  if (s.done == 3) return PIC_EBREAKDOWN;
  return PIC_ENOCONV;
}

// E_x, E_y, E_z and the double-float copy of phi (4 n double-float values).
int ensure_E(pic_ctx* c) {
  if (c->E) return PIC_OK;
  return dalloc(&c->E, 4 * c->n);
}

// A double-float constant (hi, lo) for the particle kernels.
float2 df_const(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

// The push with the node field -grad phi by central differences (phi), or a
// given node field (Efield: 3 n FP64, E_x, E_y, E_z; phi == nullptr).
int launch_push(pic_ctx* c, const double* phi, const double* Efield, double kick, double dt, int drift) {
  int e;
  if ((e = ensure_E(c))) return e;
  const int sb = streaming_blocks(c);
  if (phi) {
    float2* phid = c->E + 3 * c->n;
    launch(c, k_phi_df, sb, 256, 0, phi, phid, c->n);
    const unsigned per_plane = (unsigned)c->N * (unsigned)c->N;
    launch(c, k_gradient, dim3((per_plane + 255) / 256, c->N), 256, 0, (const float2*)phid,
           reinterpret_cast<float4*>(c->E), c->E + 2 * c->n, c->N, df_const(0.5 * c->grid.inv_h));
  } else {
    launch(c, k_field_df, sb, 256, 0, Efield, reinterpret_cast<float4*>(c->E), c->E + 2 * c->n, c->n);
  }
  if (drift) CK(cudaMemsetAsync(c->counts, 0, c->n * sizeof(uint32_t), c->stream));
  const unsigned blocks = (unsigned)((c->np + 255) / 256);
  const int slot = c->prof_on ? c->ker[PIC_KER_PUSH].begin(c->stream) : -1;
  launch(c, k_gather_push<false>, blocks, 256, 0, pptrs(c, c->cur), c->np, (const float4*)c->E,
         (const float2*)(c->E + 2 * c->n), c->grid, df_const(-kick),
         df_const(dt * c->grid.inv_h), drift, c->counts, (const double*)nullptr, c->err);
  if (c->prof_on) c->ker[PIC_KER_PUSH].end(slot, c->stream);
  CK(cudaGetLastError());
  return PIC_OK;
}

}  // namespace

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

const char* pic_strerror(int code) {
  switch (code) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument";
    case PIC_ENOMEM: return "out of device or pinned memory";
    case PIC_ECUDA: return "CUDA runtime error";
    case PIC_ENOCONV: return "solver did not converge within maxit";
    case PIC_EBREAKDOWN: return "solver breakdown (p.Ap <= 0 or non-finite value)";
    case PIC_ETIMEOUT: return "bounded device wait expired";
    case PIC_ESTATE: return "call out of order";
    default: return "unknown error";
  }
}

const char* pic_cuda_error(void) {
  return g_last_cuda_error == cudaSuccess ? "no CUDA error" : cudaGetErrorName(g_last_cuda_error);
}

int pic_create(pic_ctx** out, void* cuda_stream) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  pic_ctx* c = new (std::nothrow) pic_ctx();
  if (!c) return PIC_ENOMEM;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return PIC_ECUDA;
  }
  bool ok = cudaMalloc(&c->sc, sizeof(Scalars)) == cudaSuccess &&
            cudaMallocHost(&c->sc_host, 2 * sizeof(Scalars)) == cudaSuccess &&
            cudaMalloc(&c->counter, sizeof(unsigned)) == cudaSuccess &&
            cudaMalloc(&c->err, sizeof(int)) == cudaSuccess &&
            cudaMallocHost(&c->err_host, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&c->out3, 4 * sizeof(double)) == cudaSuccess &&
            cudaMallocHost(&c->out3_host, 4 * sizeof(double)) == cudaSuccess &&
            cudaEventCreate(&c->ev0) == cudaSuccess && cudaEventCreate(&c->ev1) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->batch_ev[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->batch_ev[1], cudaEventDisableTiming) == cudaSuccess &&
            cudaMemset(c->counter, 0, sizeof(unsigned)) == cudaSuccess &&
            cudaMemset(c->err, 0, sizeof(int)) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pic_destroy(c);
    return PIC_ENOMEM;
  }
  *c->err_host = 0;
  *out = c;
  return PIC_OK;
}

void pic_destroy(pic_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_particles(c);
  free_solver(c);
  dfree(c->sc);
  dfree(c->counter);
  dfree(c->err);
  dfree(c->io_flag);
  dfree(c->out3);
  if (c->sc_host) cudaFreeHost(c->sc_host);
  if (c->err_host) cudaFreeHost(c->err_host);
  if (c->out3_host) cudaFreeHost(c->out3_host);
  if (c->io_stream) cudaStreamSynchronize(c->io_stream);
  for (int i = 0; i < 5; ++i)
    if (c->io_ev[i]) cudaEventDestroy(c->io_ev[i]);
  if (c->io_stream) cudaStreamDestroy(c->io_stream);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  for (int i = 0; i < 2; ++i)
    if (c->batch_ev[i]) cudaEventDestroy(c->batch_ev[i]);
  if (c->phase) {
    for (int i = 0; i < PIC_NPHASE; ++i) c->phase[i].destroy();
    delete[] c->phase;
  }
  if (c->ker) {
    for (int i = 0; i < PIC_NKER; ++i) c->ker[i].destroy();
    delete[] c->ker;
  }
  cnn_state_free(c->cnn);
  mg_state_free(c->mg);
  fft_state_free(c->fft);
  pif_state_free(c->pif);
  delete c;
}

int pic_init(pic_ctx* c, const pic_params* p, uint64_t seed) {
  if (!c || !p) return PIC_EINVAL;
  if (p->N < 8 || p->N > 1024 || p->N % 8 != 0 || p->ppc < 0) return PIC_EINVAL;
  if (!(p->k > 0.0) || !isfinite(p->k) || !isfinite(p->alpha) || fabs(p->alpha) >= 1.0) return PIC_EINVAL;
  if (p->init_mode != 0 && p->init_mode != 1) return PIC_EINVAL;
  if (p->init_mode == 1 && !(3.0 * fabs(p->alpha) < 1.0)) return PIC_EINVAL;  // the sum density stays positive
  const double vth = p->vth == 0.0 ? 1.0 : p->vth;
  if (!(vth > 0.0) || !isfinite(vth)) return PIC_EINVAL;
  const uint64_t n = (uint64_t)p->N * p->N * p->N;
  const uint64_t np = (uint64_t)p->ppc * n;
  if (np >= (1ull << 32)) return PIC_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  free_particles(c);
  free_solver(c);
  c->N = p->N;
  c->n = (size_t)n;
  c->k = p->k;
  c->alpha = p->alpha;
  c->L = 2.0 * M_PI / p->k;
  c->h = c->L / p->N;
  c->ppc = p->ppc;
  c->grid.N = p->N;
  c->grid.L = c->L;
  c->grid.h = c->h;
  c->grid.inv_h = (double)p->N / c->L;
  c->has_grid = true;
  c->keys_valid = c->sorted = c->half_step = false;
  c->cur = 0;
  int e;
  if ((e = ensure_partials(c, 3 * 4096 + 3 * (size_t)c->sms * 8))) return e;
  if (np == 0) return PIC_OK;
  for (int b = 0; b < 2; ++b)
    if ((e = dalloc(&c->prec[b], np))) return e;
  const size_t nchunks = (n + kScanChunk - 1) / kScanChunk;
  if ((e = dalloc(&c->counts, n)) ||
      (e = dalloc(&c->offsets, n + 1)) || (e = dalloc(&c->chunks, nchunks)))
    return e;
  c->np = np;
  CK(cudaMemsetAsync(c->counts, 0, n * sizeof(uint32_t), c->stream));
  const unsigned blocks = (unsigned)((np + 255) / 256);
  launch(c, k_init_particles, blocks, 256, 0, pptrs(c, 0), np, seed, p->alpha, p->k, vth, p->init_mode, c->grid,
         c->counts);
  CK(cudaGetLastError());
  c->keys_valid = true;
  return PIC_OK;
}

int64_t pic_num_particles(const pic_ctx* c) { return c ? (int64_t)c->np : 0; }

// Counting sort of the particle records by cell key (a no-op when they are
// sorted): the keys and in-cell ranks in the records (written by the last
// push or state load, else counted here), an exclusive scan of the per-cell
// counts, and the scatter of the records into the other buffer.
static int sort_particles(pic_ctx* c) {
  if (c->sorted) return PIC_OK;
  const unsigned pblocks = (unsigned)((c->np + 255) / 256);
  if (!c->keys_valid) {
    CK(cudaMemsetAsync(c->counts, 0, c->n * sizeof(uint32_t), c->stream));
    launch(c, k_count_keys, pblocks, 256, 0, pptrs(c, c->cur), c->np, c->grid, c->counts);
  }
  const int nchunks = (int)((c->n + kScanChunk - 1) / kScanChunk);
  launch(c, k_scan_chunks, nchunks, 256, 0, c->counts, c->n, c->chunks);
  launch(c, k_scan_chunk_sums, 1, 1024, 0, c->chunks, nchunks);
  launch(c, k_scan_apply, nchunks, 256, 0, c->counts, c->n, c->chunks, c->offsets);
  const unsigned sblocks = (unsigned)(((c->np + 31) / 32 * 32 + 255) / 256);
  const int slot = c->prof_on ? c->ker[PIC_KER_SCATTER].begin(c->stream) : -1;
  launch(c, k_scatter, sblocks, 256, 0, pptrs(c, c->cur), pptrs(c, c->cur ^ 1), c->np,
         (const uint32_t*)c->offsets);
  if (c->prof_on) c->ker[PIC_KER_SCATTER].end(slot, c->stream);
  CK(cudaGetLastError());
  c->cur ^= 1;
  c->sorted = true;
  c->keys_valid = false;
  return PIC_OK;
}

int pic_deposit(pic_ctx* c, double* rho) {
  if (!c || !dev_ptr_ok(rho)) return PIC_EINVAL;
  if (!c->has_grid || c->np == 0) return PIC_ESTATE;
  PhaseScope ps(c, PIC_PHASE_DEPOSIT);
  int e;
  if ((e = sort_particles(c))) return e;
  if (!c->dep && (e = dalloc(&c->dep, 8 * c->n))) return e;
  const double qscale = -(double)c->n / (double)c->np;  // q_p / h^3 = -N^3 / Np
  const unsigned cblocks = (unsigned)((c->n + 255) / 256);
  const int slot = c->prof_on ? c->ker[PIC_KER_DEPOSIT].begin(c->stream) : -1;
  launch(c, k_deposit_cells, cblocks, 256, 0, (const PRec*)c->prec[c->cur], (const uint32_t*)c->offsets, c->dep,
         c->n);
  const unsigned per_plane = (unsigned)c->N * (unsigned)c->N;
  launch(c, k_deposit_nodes, dim3((per_plane + 255) / 256, c->N), 256, 0, (const float2*)c->dep, rho, c->N,
         qscale);
  if (c->prof_on) c->ker[PIC_KER_DEPOSIT].end(slot, c->stream);
  CK(cudaGetLastError());
  return PIC_OK;
}

int poisson_solve_ex(pic_ctx* c, const double* rho, double* phi, double tol, int maxit, const pic_solve_opts* o,
                     pic_solve_info* info) {
  if (!c || !dev_ptr_ok(rho) || !dev_ptr_ok(phi)) return PIC_EINVAL;
  if (!c->has_grid) return PIC_ESTATE;
  if (!(tol >= 0.0) || maxit < 0) return PIC_EINVAL;
  pic_solve_opts opts = {PIC_PREC_FP64, PIC_PC_JACOBI, 0.0, 0, 0};
  if (o) opts = *o;
  if (opts.precond < PIC_PC_JACOBI || opts.precond > PIC_PC_SSOR) return PIC_EINVAL;
  // status-check cadence: the multigrid solve converges in about ten
  // iterations, so its batches are single iterations (each iteration
  // launched past convergence still costs the launches of its kernels)
  const bool mgpc = opts.precond == PIC_PC_MG || opts.precond == PIC_PC_MG_CNN;
  int m = opts.check_every > 0 ? opts.check_every : (mgpc ? 1 : (c->N <= 64 ? 32 : 8));
  if (opts.precond != PIC_PC_JACOBI && opts.precision != PIC_PREC_MIXED) return PIC_EINVAL;
  PhaseScope ps(c, PIC_PHASE_SOLVE);
  if (opts.precision == PIC_PREC_FP64) return solve_fp64(c, rho, phi, tol, maxit, m, info);
  if (opts.precision == PIC_PREC_MIXED) {
    // reliable-update trigger: a recomputation of the FP64 residual each time
    // (r, r) falls by delta^2; measured on GB300 (256^3, 512^3 Landau
    // deposits), 0.1 is best for Jacobi-CG (smaller values cost iterations),
    // 0.03 for flexible CG with the learned preconditioner (fewer FP64
    // recomputations at the same iteration count) and 0.001 with the V-cycle
    // (its residual falls ~10x an iteration; at 512^3 0.001 kept 11
    // iterations with 3 recomputations instead of 4 at 0.003). Below 1e-4 the
    // FP32 recursion runs out of precision before its first recomputation
    // (measured: p.Ap <= 0 after ~20 V-cycle iterations at 1e-6), so smaller
    // values are rejected.
    const double delta = opts.reliable_delta > 0.0 ? opts.reliable_delta
                                                   : (opts.precond == PIC_PC_JACOBI ? 0.1 : (mgpc ? 0.001 : 0.03));
    if (!(delta < 1.0) || delta < 1e-4) return PIC_EINVAL;
    if (opts.refine_max < 0) return PIC_EINVAL;
    if (opts.precond != PIC_PC_JACOBI)
      return solve_fcg(c, rho, phi, tol, maxit, m, delta, opts.refine_max, opts.precond, info);
    return solve_mixed(c, rho, phi, tol, maxit, m, delta, opts.refine_max, info);
  }
  return PIC_EINVAL;
}

int poisson_solve(pic_ctx* c, const double* rho, double* phi, double tol, int maxit) {
  return poisson_solve_ex(c, rho, phi, tol, maxit, nullptr, nullptr);
}

int pic_gather_push(pic_ctx* c, const double* phi, double dt) {
  if (!c || !dev_ptr_ok(phi) || !isfinite(dt)) return PIC_EINVAL;
  if (!c->has_grid || c->np == 0) return PIC_ESTATE;
  const double kick = c->half_step ? dt : 0.5 * dt;
  PhaseScope ps(c, PIC_PHASE_PUSH);
  int e;
  if ((e = launch_push(c, phi, nullptr, kick, dt, 1))) return e;
  c->half_step = true;
  c->keys_valid = true;
  c->sorted = false;
  return PIC_OK;
}

int pic_gather_push_field(pic_ctx* c, const double* E, double dt) {
  if (!c || !dev_ptr_ok(E) || !isfinite(dt)) return PIC_EINVAL;
  if (!c->has_grid || c->np == 0) return PIC_ESTATE;
  const double kick = c->half_step ? dt : 0.5 * dt;
  PhaseScope ps(c, PIC_PHASE_PUSH);
  int e;
  if ((e = launch_push(c, nullptr, E, kick, dt, 1))) return e;
  c->half_step = true;
  c->keys_valid = true;
  c->sorted = false;
  return PIC_OK;
}

int pic_sync_velocity(pic_ctx* c, const double* phi, double dt) {
  if (!c || !dev_ptr_ok(phi) || !isfinite(dt)) return PIC_EINVAL;
  if (!c->has_grid || c->np == 0) return PIC_ESTATE;
  if (!c->half_step) return PIC_OK;
  int e;
  if ((e = launch_push(c, phi, nullptr, 0.5 * dt, dt, 0))) return e;
  c->half_step = false;
  return PIC_OK;
}

int pic_sync_velocity_field(pic_ctx* c, const double* E, double dt) {
  if (!c || !dev_ptr_ok(E) || !isfinite(dt)) return PIC_EINVAL;
  if (!c->has_grid || c->np == 0) return PIC_ESTATE;
  if (!c->half_step) return PIC_OK;
  int e;
  if ((e = launch_push(c, nullptr, E, 0.5 * dt, dt, 0))) return e;
  c->half_step = false;
  return PIC_OK;
}

int pic_field_energy_E(pic_ctx* c, const double* E, double out_w[3]) {
  if (!c || !dev_ptr_ok(E) || !out_w) return PIC_EINVAL;
  if (!c->has_grid) return PIC_ESTATE;
  const int sb = streaming_blocks(c);
  {
    PhaseScope ps(c, PIC_PHASE_ENERGY);
    launch(c, k_field_energy_E, sb, 256, 0, E, c->n, c->grid.h * c->grid.h * c->grid.h, c->out3, c->partials,
           c->counter);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->out3_host, c->out3, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  int e;
  if ((e = sync_status(c))) return e;
  for (int d = 0; d < 3; ++d) out_w[d] = c->out3_host[d];
  return PIC_OK;
}

int pic_field_energy(pic_ctx* c, const double* phi, double out_w[3]) {
  if (!c || !dev_ptr_ok(phi) || !out_w) return PIC_EINVAL;
  if (!c->has_grid) return PIC_ESTATE;
  const int sb = streaming_blocks(c);
  {
  PhaseScope ps(c, PIC_PHASE_ENERGY);
  launch(c, k_field_energy, sb, 256, 0, phi, c->grid, c->out3, c->partials, c->counter);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->out3_host, c->out3, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  int e;
  if ((e = sync_status(c))) return e;
  for (int d = 0; d < 3; ++d) out_w[d] = c->out3_host[d];
  return PIC_OK;
}

int pic_pif_field(pic_ctx* c, double tol, double* E) {
  if (!c || !dev_ptr_ok(E) || !(tol > 0.0)) return PIC_EINVAL;
  if (!c->has_grid || c->np == 0) return PIC_ESTATE;
  int e;
  if (!c->pif_E && (e = dalloc(&c->pif_E, 3 * c->np))) return e;
  if ((e = sort_particles(c))) return e;  // cell order: neighbouring threads share window points
  if ((e = pif_field(c, tol, c->pif_E))) return e;
  const unsigned blocks = (unsigned)((c->np + 255) / 256);
  launch(c, k_unsort_field, blocks, 256, 0, (const PRec*)pptrs(c, c->cur), c->np, (const double*)c->pif_E, E);
  CK(cudaGetLastError());
  return PIC_OK;
}

int pic_pif_push(pic_ctx* c, double tol, double dt) {
  if (!c || !(tol > 0.0) || !isfinite(dt)) return PIC_EINVAL;
  if (!c->has_grid || c->np == 0) return PIC_ESTATE;
  const double kick = c->half_step ? dt : 0.5 * dt;
  PhaseScope ps(c, PIC_PHASE_PUSH);
  int e;
  if (!c->pif_E && (e = dalloc(&c->pif_E, 3 * c->np))) return e;
  if ((e = sort_particles(c))) return e;  // cell order: neighbouring threads share window points
  if ((e = pif_field(c, tol, c->pif_E))) return e;
  CK(cudaMemsetAsync(c->counts, 0, c->n * sizeof(uint32_t), c->stream));
  const unsigned blocks = (unsigned)((c->np + 255) / 256);
  const int slot = c->prof_on ? c->ker[PIC_KER_PUSH].begin(c->stream) : -1;
  launch(c, k_gather_push<true>, blocks, 256, 0, pptrs(c, c->cur), c->np, (const float4*)nullptr,
         (const float2*)nullptr, c->grid, df_const(-kick), df_const(dt * c->grid.inv_h), 1,
         c->counts, (const double*)c->pif_E, c->err);
  if (c->prof_on) c->ker[PIC_KER_PUSH].end(slot, c->stream);
  CK(cudaGetLastError());
  c->half_step = true;
  c->keys_valid = true;
  c->sorted = false;
  return PIC_OK;
}

int pic_get_particles(pic_ctx* c, double* out, int on_device, int* half_step) {
  if (!c || !out) return PIC_EINVAL;
  if (c->np == 0) return PIC_ESTATE;
  if (half_step) *half_step = c->half_step ? 1 : 0;
  const unsigned blocks = (unsigned)((c->np + 255) / 256);
  if (on_device) {
    launch(c, k_unsort, blocks, 256, 0, (const PRec*)pptrs(c, c->cur), c->np, c->grid, out);
    CK(cudaGetLastError());
    return PIC_OK;
  }
  // host: the records in the original order in the sort's scratch buffer
  // (free between calls), then converted and copied in chunks
  int e;
  if ((e = ensure_stage(c))) return e;
  // the inverse permutation of the sort (4 B a particle, in the sort's
  // scratch buffer, free between calls); each chunk then gathers its
  // particles from the sorted records (no pass that moves every record)
  uint32_t* inv = reinterpret_cast<uint32_t*>(pptrs(c, c->cur ^ 1));
  launch(c, k_inverse_ids, blocks, 256, 0, (const PRec*)pptrs(c, c->cur), c->np, inv);
  // chunk i: converted into buffer i % 2 on the context stream, copied out on
  // the copy stream while chunk i + 1 is converted into the other buffer
  int i = 0;
  for (uint64_t base = 0; base < c->np; base += kStageParticles, ++i) {
    const uint64_t cnt = c->np - base < kStageParticles ? c->np - base : kStageParticles;
    const int b = i & 1;
    double* st = stage_buf(c, b);
    if (i >= 2) CK(cudaStreamWaitEvent(c->stream, c->io_ev[b], 0));  // chunk i - 2 has left this buffer
    launch(c, k_records_to_soa, (unsigned)((cnt + 255) / 256), 256, 0, (const PRec*)pptrs(c, c->cur), base, cnt,
           c->grid, st, cnt, (const uint32_t*)inv);
    CK(cudaEventRecord(c->io_ev[2 + b], c->stream));
    CK(cudaStreamWaitEvent(c->io_stream, c->io_ev[2 + b], 0));
    for (int q = 0; q < 6; ++q)
      CK(cudaMemcpyAsync(out + q * c->np + base, st + q * cnt, cnt * sizeof(double), cudaMemcpyDeviceToHost,
                         c->io_stream));
    CK(cudaEventRecord(c->io_ev[b], c->io_stream));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->io_stream));
  CK(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

int pic_selftest_bounded_wait(pic_ctx* c, uint64_t budget_ns, int producer) {
  if (!c || budget_ns == 0 || budget_ns > kWaitBudgetNs || (producer != 0 && producer != 1)) return PIC_EINVAL;
  launch(c, k_selftest_wait, 1, 32, 0, budget_ns, producer, c->err);
  CK(cudaGetLastError());
  return sync_status(c);
}

int pic_set_particles(pic_ctx* c, const double* in, int on_device, int half_step) {
  if (!c || !in || (half_step != 0 && half_step != 1)) return PIC_EINVAL;
  if (on_device && ((uintptr_t)in % 8) != 0) return PIC_EINVAL;
  if (c->np == 0) return PIC_ESTATE;
  int e;
  if ((e = ensure_stage(c))) return e;
  CK(cudaMemsetAsync(c->io_flag, 0, sizeof(int), c->stream));
  // the conversion also counts the cells for the next sort
  CK(cudaMemsetAsync(c->counts, 0, c->n * sizeof(uint32_t), c->stream));
  PRec* P = pptrs(c, c->cur);
  if (on_device) {
    launch(c, k_set_particles, (unsigned)((c->np + 255) / 256), 256, 0, in, c->np, c->np, (uint64_t)0, P, c->grid,
           c->io_flag, c->counts);
  } else {
    // chunk i: copied into buffer i % 2 on the copy stream while chunk i - 1
    // is converted from the other buffer on the context stream
    CK(cudaEventRecord(c->io_ev[4], c->stream));
    CK(cudaStreamWaitEvent(c->io_stream, c->io_ev[4], 0));
    int i = 0;
    for (uint64_t base = 0; base < c->np; base += kStageParticles, ++i) {
      const uint64_t cnt = c->np - base < kStageParticles ? c->np - base : kStageParticles;
      const int b = i & 1;
      double* st = stage_buf(c, b);
      if (i >= 2) CK(cudaStreamWaitEvent(c->io_stream, c->io_ev[2 + b], 0));  // chunk i - 2 converted
      for (int q = 0; q < 6; ++q)
        CK(cudaMemcpyAsync(st + q * cnt, in + q * c->np + base, cnt * sizeof(double), cudaMemcpyHostToDevice,
                           c->io_stream));
      CK(cudaEventRecord(c->io_ev[b], c->io_stream));
      CK(cudaStreamWaitEvent(c->stream, c->io_ev[b], 0));
      launch(c, k_set_particles, (unsigned)((cnt + 255) / 256), 256, 0, (const double*)st, cnt, cnt, base, P,
             c->grid, c->io_flag, c->counts);
      CK(cudaEventRecord(c->io_ev[2 + b], c->stream));
    }
  }
  CK(cudaGetLastError());
  int flag = 0;
  CK(cudaMemcpyAsync(c->err_host, c->io_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  flag = *c->err_host;
  // the records are in the caller's order, their keys and ranks counted:
  // the next deposit sorts them
  c->keys_valid = true;
  c->sorted = false;
  c->half_step = half_step != 0;
  return (flag & DEV_ERR_NONFINITE) ? PIC_EINVAL : PIC_OK;
}

int pic_residual(pic_ctx* c, const double* rho, const double* phi, double* r) {
  if (!c || !dev_ptr_ok(rho) || !dev_ptr_ok(phi) || !dev_ptr_ok(r)) return PIC_EINVAL;
  if (!c->has_grid) return PIC_ESTATE;
  SolverWs& w = c->ws;
  int e;
  if (!w.x && (e = dalloc(&w.x, c->n))) return e;
  if (!w.b && (e = dalloc(&w.b, c->n))) return e;
  size_t smem;
  StreamGeo g;
  if ((e = geo_for<double, double, double, 1>(c, k_residual64, &g, &smem))) return e;
  if ((e = ensure_partials(c, (size_t)3 * g.blocks + 3 * 4096))) return e;
  Scalars init;
  memset(&init, 0, sizeof(init));
  init.maxit = 1;
  c->sc_host[0] = init;
  CK(cudaMemcpyAsync(c->sc, &c->sc_host[0], sizeof(Scalars), cudaMemcpyHostToDevice, c->stream));
  const int sb = streaming_blocks(c);
  const size_t n4 = c->n / 4;
  // b = h^2 (rho - mean rho), x = phi - mean phi, r = b - (h^2 A) x, then r /= h^2
  launch(c, k_sum2, sb, 256, 0, rho, phi, n4, c->sc, c->partials, c->counter);
  launch(c, k_project, sb, 256, 0, rho, phi, w.b, w.x, n4, 1.0 / (double)c->n, c->h * c->h, 1.0, c->sc,
         c->partials, c->counter);
  // the residual kernel skips work once a solve is marked done; clear it
  CK(cudaMemsetAsync(&c->sc->done, 0, sizeof(int), c->stream));
  launch(c, k_residual64, g.blocks, round32(g.threads), smem, (const double*)w.x, (const double*)w.b, r, c->sc,
         c->partials, c->counter, c->err, g);
  launch(c, k_scale64, sb, 256, 0, r, n4, 1.0 / (c->h * c->h));
  CK(cudaGetLastError());
  return PIC_OK;
}

int pic_apply_laplacian(pic_ctx* c, const double* x, double* y) {
  if (!c || !dev_ptr_ok(x) || !dev_ptr_ok(y)) return PIC_EINVAL;
  if (!c->has_grid) return PIC_ESTATE;
  size_t smem;
  StreamGeo g;
  int e;
  if ((e = geo_for<double, double, double, 1>(c, k_apply64, &g, &smem))) return e;
  launch(c, k_apply64, g.blocks, round32(g.threads), smem, x, y, 1.0 / (c->h * c->h), c->err, g);
  CK(cudaGetLastError());
  return PIC_OK;
}

int pic_profile_enable(pic_ctx* c, int on) {
  if (!c) return PIC_EINVAL;
  if (on && !c->phase) {
    c->phase = new (std::nothrow) EventPool[PIC_NPHASE];
    c->ker = new (std::nothrow) EventPool[PIC_NKER];
    if (!c->phase || !c->ker) return PIC_ENOMEM;
    for (int i = 0; i < PIC_NPHASE; ++i)
      if (!c->phase[i].init()) return PIC_ECUDA;
    for (int i = 0; i < PIC_NKER; ++i)
      if (!c->ker[i].init()) return PIC_ECUDA;
  }
  c->prof_on = on != 0;
  return PIC_OK;
}

int pic_profile_read(pic_ctx* c, pic_profile_stats* out, int reset) {
  if (!c || !out) return PIC_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  memset(out, 0, sizeof(*out));
  out->launches = c->launches;
  if (c->phase) {
    for (int i = 0; i < PIC_NPHASE; ++i) {
      c->phase[i].flush();
      out->phase_calls[i] = c->phase[i].count;
      out->phase_ms[i] = c->phase[i].ms;
      if (reset) c->phase[i].reset();
    }
    for (int i = 0; i < PIC_NKER; ++i) {
      c->ker[i].flush();
      out->ker_samples[i] = c->ker[i].count;
      out->ker_ms[i] = c->ker[i].ms;
      out->ker_precision[i] = c->ker_prec[i];
      if (reset) c->ker[i].reset();
    }
  }
  if (reset) c->launches = 0;
  return PIC_OK;
}

}  // extern "C"
