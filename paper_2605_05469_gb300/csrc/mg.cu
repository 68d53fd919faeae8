// Multigrid V-cycle preconditioner: level hierarchy, buffers and the launch
// sequence (kernels in mg_kernels.cuh).
#include <new>

#include "cnn.h"
#include "ctx.h"
#include "mg.h"
#include "mg_kernels.cuh"
#include "slab_geo.h"

namespace pic {

// The plane-streamed kernels of a level (its size a multiple of 4).
enum MgKer { kPre, kResid, kResidProlong, kSmoothProlong, kSmooth, kNumMgKer };

struct MgLevel {
  int N = 0;
  float *x = nullptr, *r = nullptr, *t = nullptr, *res = nullptr;
  bool streamed = false;          // N % 4 == 0: plane-streamed kernels
  bool tall = false;              // N >= 512: one 1024-thread block per SM
  bool zmarch = false;            // N % 128 == 0: z-marching pre-smoothing, residual, smoothing
  StreamGeo geo[kNumMgKer]{};
  size_t smem[kNumMgKer]{};
};

struct MgState {
  int N0 = 0;
  int nbig = 0;              // levels above kSmallN (level 0 = the context grid)
  MgLevel lev[12];           // lev[nbig] is the first small level (its r and x only)
  mg::SmallLevels small{};
  size_t small_smem = 0;
};

void mg_state_free(MgState* s) {
  if (!s) return;
  for (auto& L : s->lev) {
    dfree(L.x); dfree(L.r); dfree(L.t); dfree(L.res);
  }
  delete s;
}

namespace {

// Shared memory of a small V-cycle block (the CG kernels' budget: three
// blocks an SM; measured, four blocks with fewer stages were slower, the
// kernels spilling at the 64-register limit that four blocks impose).
constexpr size_t kMgSmemBudget = 72 * 1024;
// damped-Jacobi sweeps before and after the coarse-grid correction (even, >= 2)
constexpr int kMgNu = 2;

// Whether kernel k of level L runs in the tall-block form: the kernels with
// the prolongation keep the small block (their coarse-value registers would
// spill at the tall block's 64-register limit; measured no faster at 512^3).
bool tall_form(const MgLevel& L, MgKer k) {
  const bool prolong = k == kResidProlong || k == kSmoothProlong;
  return L.tall && !prolong;
}

// The plane-streamed kernel k in its small- or tall-block form.
const void* mg_kernel(MgKer k, bool tall) {
  switch (k) {
    case kPre: return tall ? (const void*)mg::k_mg_pre<true> : (const void*)mg::k_mg_pre<false>;
    case kResid:
      return tall ? (const void*)mg::k_mg_stencil<mg::kResid, false, true>
                  : (const void*)mg::k_mg_stencil<mg::kResid, false, false>;
    case kResidProlong:
      return tall ? (const void*)mg::k_mg_stencil<mg::kResid, true, true>
                  : (const void*)mg::k_mg_stencil<mg::kResid, true, false>;
    case kSmoothProlong:
      return tall ? (const void*)mg::k_mg_stencil<mg::kSmooth, true, true>
                  : (const void*)mg::k_mg_stencil<mg::kSmooth, true, false>;
    default:
      return tall ? (const void*)mg::k_mg_stencil<mg::kSmooth, false, true>
                  : (const void*)mg::k_mg_stencil<mg::kSmooth, false, false>;
  }
}

int grid_for(const pic_ctx* c, size_t n) {
  size_t b = (n + 255) / 256;
  const size_t cap = (size_t)c->sms * 8;
  return (int)(b < cap ? b : cap);
}

// The hierarchy of the oracle's V-cycle: halve while the level is even and
// above the coarsest size; levels at or below kSmallN run in one CTA.
int ensure_state(pic_ctx* c) {
  if (c->mg && c->mg->N0 == c->N) return PIC_OK;
  if (c->mg) {
    mg_state_free(c->mg);
    c->mg = nullptr;
  }
  MgState* s = new (std::nothrow) MgState();
  if (!s) return PIC_ENOMEM;
  s->N0 = c->N;
  int sizes[24], nl = 0;
  for (int N = c->N;; N /= 2) {
    sizes[nl++] = N;
    if (N <= mg::kCoarsestN || N % 2) break;
  }
  int b = 0;
  while (b < nl && sizes[b] > mg::kSmallN) ++b;
  s->nbig = b;
  int e = PIC_OK;
  for (int l = 0; l <= b && l < nl && !e; ++l) {
    MgLevel& L = s->lev[l];
    L.N = sizes[l];
    const size_t n = (size_t)L.N * L.N * L.N;
    if (l > 0) {
      if ((e = dalloc(&L.x, n)) || (e = dalloc(&L.r, n))) break;
    }
    if (l < b) {
      if ((e = dalloc(&L.t, n)) || (e = dalloc(&L.res, n))) break;
    }
  }
  // slab geometry of every streamed level; each kernel's shared-memory limit
  // ends at the largest size any level launches it with
  size_t smax[2][kNumMgKer] = {};
  for (int l = 0; l < b && !e; ++l) {
    MgLevel& L = s->lev[l];
    L.streamed = L.N % 4 == 0;
    if (!L.streamed) continue;
    L.zmarch = L.N % 128 == 0;
    // the tall block re-reads fewer halo rows on large grids (as for the CG
    // direction kernel); coarse levels are latency-bound: more blocks with
    // fewer planes each
    L.tall = L.N >= 512;
    const int min_planes = L.N >= 256 ? 4 : (L.N >= 128 ? 2 : 1);
    for (int k = 0; k < kNumMgKer && !e; ++k) {
      const bool t = tall_form(L, (MgKer)k);
      // pre-smoothing streams r alone, the others x and r
      if (k == kPre)
        e = slab_geometry<float, float, float, 1>(c, L.N, mg_kernel((MgKer)k, t), &L.geo[k], &L.smem[k], t,
                                                  min_planes, kMgSmemBudget);
      else
        e = slab_geometry<float, float, float, 2>(c, L.N, mg_kernel((MgKer)k, t), &L.geo[k], &L.smem[k], t,
                                                  min_planes, kMgSmemBudget);
      size_t& m = smax[t][k];
      if (L.smem[k] > m) m = L.smem[k];
    }
  }
  for (int t = 0; t < 2; ++t)
    for (int k = 0; k < kNumMgKer && !e; ++k) {
      if (smax[t][k] && cudaFuncSetAttribute(mg_kernel((MgKer)k, t != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smax[t][k]) != cudaSuccess)
        e = PIC_ECUDA;
    }
  // the small levels (first one = lev[b])
  mg::SmallLevels& S = s->small;
  S.n = nl - b;
  int off = 0;
  for (int q = 0; q < S.n; ++q) {
    S.N[q] = sizes[b + q];
    S.off[q] = off;
    off += S.N[q] * S.N[q] * S.N[q];
  }
  S.total = off;
  s->small_smem = (size_t)3 * off * sizeof(float);
  if (!e && b == 0) {
    // the context grid itself is small: the CTA kernel does the whole cycle
    s->lev[0].N = sizes[0];
  }
  if (e) {
    mg_state_free(s);
    return e;
  }
  c->mg = s;
  return PIC_OK;
}

}  // namespace

int mg_apply(pic_ctx* c, const float* r, float* z, bool learned, const int* done, bool sample) {
  int e;
  if ((e = ensure_state(c))) return e;
  MgState* s = c->mg;
  static bool configured = false;
  if (!configured) {
    CK(cudaFuncSetAttribute((const void*)mg::k_mg_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(3 * (16 * 16 * 16 + 8 * 8 * 8 + 4 * 4 * 4) * sizeof(float))));
    configured = true;
  }
  const int B = s->nbig;
  // the learned smoother works on the finest of the full-grid levels
  if (learned && B == 0) return PIC_EINVAL;
  auto xl = [&](int l) { return l == 0 ? z : s->lev[l].x; };
  auto rl = [&](int l) { return l == 0 ? r : (const float*)s->lev[l].r; };
  // plane-streamed kernel k of level L; the finest level's launches are
  // timed into event pool `pool` when sampling
  sample = sample && c->prof_on;
  // the z-marching form (levels whose size is a multiple of 128) of the
  // pre-smoothing, residual and plain smoothing kernels
  auto zmarch = [&](const MgLevel& L, int pool, auto kernel, const float* field, const float* aux, float* out,
                    const float* ec_in = nullptr, float* xout = nullptr) {
    const bool t = sample && &L == &s->lev[0];
    const int slot = t ? c->ker[pool].begin(c->stream) : -1;
    const unsigned tiles = (unsigned)(L.N / 128) * (unsigned)(L.N / 8);
    // the longest chunk (a power of two dividing N) that still gives about
    // four blocks an SM
    int zc = mg::kZChunkMax;
    while (zc > 4 && (long)tiles * (L.N / zc) < 4L * c->sms) zc /= 2;
    launch(c, kernel, dim3(tiles, L.N / zc), dim3(32, 8), 0, field, aux, out, L.N, zc, done, ec_in, xout);
    if (t) c->ker[pool].end(slot, c->stream);
  };
  auto slab = [&](const MgLevel& L, MgKer k, int pool, auto kernel, auto... args) {
    const StreamGeo& g = L.geo[k];
    const bool t = sample && &L == &s->lev[0];
    const int slot = t ? c->ker[pool].begin(c->stream) : -1;
    launch(c, kernel, g.blocks, round32(g.threads), L.smem[k], args..., c->err, g, done);
    if (t) c->ker[pool].end(slot, c->stream);
  };
  const float* nul = nullptr;
  float* nulw = nullptr;
  // damped-Jacobi sweeps before and after the coarse correction (even); the
  // first two are fused (from zero before, with the prolongation after) and
  // every further pair ping-pongs x -> t -> x
  const int nu = kMgNu;
  auto sweep_pair = [&](MgLevel& L) {
    const int l = (int)(&L - s->lev);
    if (L.zmarch) {
      zmarch(L, PIC_KER_MG_SMOOTH, mg::k_mg_zmarch<mg::kZSmooth, false>, (const float*)xl(l), rl(l), L.t);
      zmarch(L, PIC_KER_MG_SMOOTH, mg::k_mg_zmarch<mg::kZSmooth, false>, (const float*)L.t, rl(l), xl(l));
    } else if (L.streamed) {
      auto k = tall_form(L, kSmooth) ? mg::k_mg_stencil<mg::kSmooth, false, true> : mg::k_mg_stencil<mg::kSmooth, false, false>;
      slab(L, kSmooth, PIC_KER_MG_SMOOTH, k, (const float*)xl(l), rl(l), L.t, nulw, nul);
      slab(L, kSmooth, PIC_KER_MG_SMOOTH, k, (const float*)L.t, rl(l), xl(l), nulw, nul);
    } else {
      const int g = grid_for(c, (size_t)L.N * L.N * L.N);
      launch(c, mg::k_mg_jacobi, g, 256, 0, (const float*)xl(l), rl(l), L.t, L.N, done);
      launch(c, mg::k_mg_jacobi, g, 256, 0, (const float*)L.t, rl(l), xl(l), L.N, done);
    }
  };
  // down: pre-smooth, residual, restrict
  for (int l = 0; l < B; ++l) {
    MgLevel& L = s->lev[l];
    const size_t n = (size_t)L.N * L.N * L.N;
    const int g = grid_for(c, n);
    if (l == 0 && learned) {
      if ((e = cnn_apply(c, rl(0), xl(0), nullptr, n))) return e;
    } else if (L.zmarch) {
      zmarch(L, PIC_KER_MG_PRE, mg::k_mg_zmarch<mg::kZPre, false>, rl(l), nul, xl(l));
      for (int k = 2; k < nu; k += 2) sweep_pair(L);
    } else if (L.streamed) {
      slab(L, kPre, PIC_KER_MG_PRE, tall_form(L, kPre) ? mg::k_mg_pre<true> : mg::k_mg_pre<false>, rl(l), xl(l));
      for (int k = 2; k < nu; k += 2) sweep_pair(L);
    } else {
      launch(c, mg::k_mg_jacobi, g, 256, 0, nul, rl(l), L.t, L.N, done);
      launch(c, mg::k_mg_jacobi, g, 256, 0, (const float*)L.t, rl(l), xl(l), L.N, done);
      for (int k = 2; k < nu; k += 2) sweep_pair(L);
    }
    if (L.streamed) {
      if (L.zmarch)
        zmarch(L, PIC_KER_MG_RESID, mg::k_mg_zmarch<mg::kZResid, false>, (const float*)xl(l), rl(l), L.res);
      else
        slab(L, kResid, PIC_KER_MG_RESID, tall_form(L, kResid) ? mg::k_mg_stencil<mg::kResid, false, true> : mg::k_mg_stencil<mg::kResid, false, false>, (const float*)xl(l), rl(l), L.res, nulw, nul);
      const int Nc = L.N / 2;
      const unsigned per_plane = (unsigned)(Nc / 2) * (unsigned)Nc;
      const unsigned bx = (per_plane + 255) / 256;
      const bool t = sample && l == 0;
      const int slot = t ? c->ker[PIC_KER_MG_RESTRICT].begin(c->stream) : -1;
      launch(c, mg::k_mg_restrict2, dim3(bx, Nc), 256, 0, (const float*)L.res, s->lev[l + 1].r, L.N, done);
      if (t) c->ker[PIC_KER_MG_RESTRICT].end(slot, c->stream);
    } else {
      launch(c, mg::k_mg_residual, g, 256, 0, (const float*)xl(l), rl(l), L.res, L.N, done);
      launch(c, mg::k_mg_restrict, grid_for(c, n / 8), 256, 0, (const float*)L.res, s->lev[l + 1].r, L.N, done);
    }
  }
  // the small levels in one CTA
  launch(c, mg::k_mg_small, 1, mg::kSmallThreads, s->small_smem, rl(B), xl(B), s->small, nu, done);
  // up: prolong-add, post-smooth
  for (int l = B - 1; l >= 0; --l) {
    MgLevel& L = s->lev[l];
    const size_t n = (size_t)L.N * L.N * L.N;
    const int g = grid_for(c, n);
    const float* ec = xl(l + 1);
    if (l == 0 && learned) {
      // x' = x + P e_c (into t), res = r - A^ x', x = x' + K res
      if (L.zmarch) {
        zmarch(L, PIC_KER_MG_PROLONG_SMOOTH, mg::k_mg_zmarch<mg::kZResid, true>, (const float*)xl(0), rl(0), L.res,
               ec, L.t);
      } else if (L.streamed) {
        slab(L, kResidProlong, PIC_KER_MG_PROLONG_SMOOTH, tall_form(L, kResidProlong) ? mg::k_mg_stencil<mg::kResid, true, true> : mg::k_mg_stencil<mg::kResid, true, false>, (const float*)xl(0), rl(0), L.res, L.t, ec);
      } else {
        launch(c, mg::k_mg_prolong_add, g, 256, 0, xl(0), ec, L.N / 2, done);
        launch(c, mg::k_mg_copy, grid_for(c, n), 256, 0, (const float*)xl(0), L.t, n, done);
        launch(c, mg::k_mg_residual, g, 256, 0, (const float*)xl(0), rl(0), L.res, L.N, done);
      }
      if ((e = cnn_apply(c, L.res, xl(0), nullptr, n))) return e;
      launch(c, mg::k_mg_add, grid_for(c, n / 4), 256, 0, xl(0), (const float*)L.t, n / 4, done);
    } else if (L.zmarch) {
      zmarch(L, PIC_KER_MG_PROLONG_SMOOTH, mg::k_mg_zmarch<mg::kZSmooth, true>, (const float*)xl(l), rl(l), L.t, ec);
      zmarch(L, PIC_KER_MG_SMOOTH, mg::k_mg_zmarch<mg::kZSmooth, false>, (const float*)L.t, rl(l), xl(l));
      for (int k = 2; k < nu; k += 2) sweep_pair(L);
    } else if (L.streamed) {
      slab(L, kSmoothProlong, PIC_KER_MG_PROLONG_SMOOTH, tall_form(L, kSmoothProlong) ? mg::k_mg_stencil<mg::kSmooth, true, true> : mg::k_mg_stencil<mg::kSmooth, true, false>, (const float*)xl(l), rl(l), L.t, nulw, ec);
      slab(L, kSmooth, PIC_KER_MG_SMOOTH, tall_form(L, kSmooth) ? mg::k_mg_stencil<mg::kSmooth, false, true> : mg::k_mg_stencil<mg::kSmooth, false, false>, (const float*)L.t, rl(l), xl(l), nulw, nul);
      for (int k = 2; k < nu; k += 2) sweep_pair(L);
    } else {
      launch(c, mg::k_mg_prolong_add, g, 256, 0, xl(l), ec, L.N / 2, done);
      launch(c, mg::k_mg_jacobi, g, 256, 0, (const float*)xl(l), rl(l), L.t, L.N, done);
      launch(c, mg::k_mg_jacobi, g, 256, 0, (const float*)L.t, rl(l), xl(l), L.N, done);
      for (int k = 2; k < nu; k += 2) sweep_pair(L);
    }
  }
  CK(cudaGetLastError());
  return PIC_OK;
}

}  // namespace pic

extern "C" int pic_mg_apply(pic_ctx* c, const float* r, float* z, int learned) {
  if (!c || !r || !z) return PIC_EINVAL;
  if (!c->has_grid) return PIC_ESTATE;
  if (learned && !pic::cnn_ready(c)) return PIC_ESTATE;
  return pic::mg_apply(c, r, z, learned != 0, nullptr);
}
