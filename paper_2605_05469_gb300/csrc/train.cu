// pic_cnn_train: training of the learned preconditioner behind the C ABI.
//
// Data are (residual, error) pairs. For the preconditioner they come from the
// method's own FP64 Jacobi-PCG solves (Sec. 3.2) of CIC deposits of seeded
// Landau initial conditions (Sec. 2.1): the converged phi* (tol 1e-12) and
// the iterates phi_k after k = 1, 2, 4, ..., 128 iterations from zero give
// r_k = b - A phi_k and e_k = phi* - phi_k. For the multigrid smoother they
// are white-noise errors e (Philox4x32-10 normals) and r = A e, whose energy
// sits in the high frequencies a smoother must remove. Every step draws a
// set, a snapshot and B crop origins from a counter-based Philox stream
// keyed by the seed (counter = the Adam step, so a resumed training continues
// the stream), then runs the library's crop, forward, loss, backward and Adam
// kernels. Every validate_every steps the weights are scored by the flexible
// CG iterations of a held-out deposit solve, and the best scored training
// state (weights, Adam moments, step) over `restarts` independent trainings
// (other initial weights and crop streams, the same data) is the one the
// context keeps.
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <deque>
#include <vector>

#include "cnn.h"
#include "ctx.h"

using namespace pic;

namespace {

constexpr int kWeightsN = PIC_CNN_WEIGHTS;
constexpr int kSnapIters[8] = {1, 2, 4, 8, 16, 32, 64, 128};

// Philox4x32-10 (Salmon et al., SC'11) on the host: ten rounds of the
// multiply-xor round function with the Weyl key schedule.
struct U4 {
  uint32_t x, y, z, w;
};

U4 philox(U4 c, uint64_t key) {
  uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  for (int i = 0; i < 10; ++i) {
    if (i > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)M0 * c.x, p1 = (uint64_t)M1 * c.z;
    c = {(uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0};
  }
  return c;
}

double unit53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

// A standard normal from counter i of the stream (Box-Muller, Box & Muller 1958).
double normal_host(uint64_t key, uint32_t i, uint32_t stream) {
  const U4 r = philox({i, stream, 0x5EEDu, 0u}, key);
  const double u1 = unit53(r.x, r.y), u2 = unit53(r.z, r.w);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

// White-noise field on the device: e_i ~ N(0, 1) from Philox counters (i, 0).
__device__ __forceinline__ uint4 philox_dev(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  for (int i = 0; i < 10; ++i) {
    if (i > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__global__ void k_noise_field(double* e, size_t n, uint64_t key) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox_dev(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, 0u),
                             make_uint2((uint32_t)key, (uint32_t)(key >> 32)));
  const double u1 = ((double)(r.x >> 5) * 67108864.0 + (double)(r.y >> 6) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((double)(r.z >> 5) * 67108864.0 + (double)(r.w >> 6) + 0.5) * (1.0 / 9007199254740992.0);
  e[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

// Initial weights: the Jacobi direction plus small seeded noise. Channel 0 of
// layer 1 carries r / sqrt(6) through its centre tap and layer 2 passes
// channel 0 on, so N = G^T G = 1/6 (layers 3 and 4 are the adjoints, set by
// the library); He-scaled normals times 0.02 everywhere else.
void initial_weights(uint64_t seed, float* w) {
  memset(w, 0, sizeof(float) * kWeightsN);
  const double s1 = 0.02 * sqrt(2.0 / 27.0), s2 = 0.02 * sqrt(2.0 / (27.0 * 16.0));
  for (int i = 0; i < 16 * 27; ++i) w[i] = (float)(s1 * normal_host(seed, (uint32_t)i, 1u));
  for (int i = 0; i < 16 * 16 * 27; ++i) w[432 + i] = (float)(s2 * normal_host(seed, (uint32_t)i, 2u));
  w[0 * 27 + 13] += (float)(1.0 / sqrt(6.0));
  w[432 + 13] += 1.0f;
}

struct DevBuf {
  void* p = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;  // owns its allocation: never copied or relocated
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  template <typename T>
  T* get() const {
    return static_cast<T*>(p);
  }
  int alloc(size_t bytes) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return PIC_ENOMEM;
    }
    return PIC_OK;
  }
};

struct CtxGuard {
  pic_ctx* c = nullptr;
  ~CtxGuard() {
    if (c) pic_destroy(c);
  }
};

// One training set: the target solution a, and snapshots (r_k, b_k) with
// e_k = a - b_k.
struct Set {
  double* a = nullptr;
  std::vector<double*> r, b;
};

int make_context(cudaStream_t st, int N, int ppc, uint64_t seed, double alpha, double k, CtxGuard* g) {
  int e;
  if ((e = pic_create(&g->c, st))) return e;
  pic_params p{N, ppc, alpha, k, 1.0, 0};
  return pic_init(g->c, &p, seed);
}

// A device FP64 field of n values owned by `pool` (a deque: its elements stay
// where they are while it grows).
int dfield(std::deque<DevBuf>& pool, size_t n, double** out) {
  pool.emplace_back();
  int e = pool.back().alloc(n * sizeof(double));
  *out = pool.back().get<double>();
  return e;
}

// Flexible-CG iterations of the held-out solve with the weights in `src`
// (the training state buffer), the cost that selects the kept state.
int validate(pic_ctx* v, const double* rho, double* phi, size_t n, const float* state, int pc, int* iters) {
  int e;
  if ((e = cnn_state_set(v, state, 0))) return e;
  CK(cudaMemsetAsync(phi, 0, n * sizeof(double), v->stream));
  pic_solve_opts o{PIC_PREC_MIXED, pc, 0.0, 0, 0};
  pic_solve_info info;
  e = poisson_solve_ex(v, rho, phi, 1e-10, 2000, &o, &info);
  if (e != PIC_OK && e != PIC_ENOCONV) return e;
  *iters = info.converged ? info.iters : 2001;
  return PIC_OK;
}

}  // namespace

extern "C" int pic_cnn_train(pic_ctx* c, const pic_train_opts* o, pic_train_info* info) {
  if (!c || !o) return PIC_EINVAL;
  const pic_train_opts& O = *o;
  if (O.target != PIC_TRAIN_PRECONDITIONER && O.target != PIC_TRAIN_SMOOTHER) return PIC_EINVAL;
  if (O.grid < 32 || O.grid > 256 || O.grid % 16 != 0 || O.crop < 16 || O.crop % 16 != 0 || O.crop > O.grid ||
      O.sets < 1 || O.sets > 64 || O.steps < 0 || O.batch < 1 || O.batch > 64 || !(O.lr > 0.0) ||
      O.validate_every < 0 || (O.resume != 0 && O.resume != 1))
    return PIC_EINVAL;
  if (O.validate_every > 0 && (O.val_grid < 32 || O.val_grid > 512 || O.val_grid % 32 != 0)) return PIC_EINVAL;
  if (O.restarts < 1 || O.restarts > 16 || (O.restarts > 1 && (O.resume || O.validate_every == 0)))
    return PIC_EINVAL;
  if (O.resume && !cnn_ready(c)) return PIC_ESTATE;
  const timespec t_start = [] {
    timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return t;
  }();
  const double alpha = c->has_grid ? c->alpha : 0.05, kw = c->has_grid ? c->k : 0.5;
  const int N = O.grid;
  const size_t n = (size_t)N * N * N;
  const double h = 2.0 * M_PI / kw / N;
  int e;

  // the training context (the crop kernels read fields of its grid)
  CtxGuard tg;
  if ((e = make_context(c->stream, N, 0, 0, alpha, kw, &tg))) return e;
  pic_ctx* t = tg.c;
  DevBuf state, best;  // training state (w, m, v) and the best scored one
  if ((e = state.alloc(3 * kWeightsN * sizeof(float))) || (e = best.alloc(3 * kWeightsN * sizeof(float)))) return e;
  int adam_t0 = 0;  // Adam step count the training starts from
  DevBuf start;     // resume: the caller's training state
  if (O.resume) {
    if ((e = start.alloc(3 * kWeightsN * sizeof(float))) || (e = cnn_state_get(c, start.get<float>(), &adam_t0)))
      return e;
  }

  // training data
  std::deque<DevBuf> pool;
  std::vector<Set> sets(O.sets);
  double* zero = nullptr;
  if ((e = dfield(pool, n, &zero))) return e;
  CK(cudaMemsetAsync(zero, 0, n * sizeof(double), c->stream));
  for (int si = 0; si < O.sets; ++si) {
    Set& S = sets[si];
    if ((e = dfield(pool, n, &S.a))) return e;
    if (O.target == PIC_TRAIN_SMOOTHER) {
      double* r;
      if ((e = dfield(pool, n, &r))) return e;
      k_noise_field<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(S.a, n, O.seed + (uint64_t)si);
      CK(cudaGetLastError());
      if ((e = pic_apply_laplacian(t, S.a, r))) return e;
      S.r.push_back(r);
      S.b.push_back(zero);
      continue;
    }
    CtxGuard dg;
    if ((e = make_context(c->stream, N, 8, O.seed + (uint64_t)si, alpha, kw, &dg))) return e;
    double* rho;
    if ((e = dfield(pool, n, &rho))) return e;
    if ((e = pic_deposit(dg.c, rho))) return e;
    CK(cudaMemsetAsync(S.a, 0, n * sizeof(double), c->stream));
    pic_solve_opts fp64{PIC_PREC_FP64, PIC_PC_JACOBI, 0.0, 0, 0};
    if ((e = poisson_solve_ex(dg.c, rho, S.a, 1e-12, 50 * N + 1000, &fp64, nullptr))) return e;
    for (int k : kSnapIters) {
      double *x, *r;
      if ((e = dfield(pool, n, &x)) || (e = dfield(pool, n, &r))) return e;
      CK(cudaMemsetAsync(x, 0, n * sizeof(double), c->stream));
      e = poisson_solve_ex(dg.c, rho, x, 1e-300, k, &fp64, nullptr);
      if (e != PIC_OK && e != PIC_ENOCONV) return e;
      if ((e = pic_residual(dg.c, rho, x, r))) return e;
      S.r.push_back(r);
      S.b.push_back(x);
    }
  }

  // validation: a held-out deposit on another grid and seed
  CtxGuard vg;
  DevBuf vrho, vphi;
  const int pc = O.target == PIC_TRAIN_SMOOTHER ? PIC_PC_MG_CNN : PIC_PC_CNN;
  if (O.validate_every > 0) {
    const size_t vn = (size_t)O.val_grid * O.val_grid * O.val_grid;
    if ((e = make_context(c->stream, O.val_grid, 8, O.val_seed, alpha, kw, &vg))) return e;
    if ((e = vrho.alloc(vn * sizeof(double))) || (e = vphi.alloc(vn * sizeof(double)))) return e;
    if ((e = pic_deposit(vg.c, vrho.get<double>()))) return e;
  }

  // the loop
  const int B = O.batch, D = O.crop;
  const size_t m = (size_t)B * D * D * D;
  DevBuf xb, tb, yb, gb;
  if ((e = xb.alloc(m * 4)) || (e = tb.alloc(m * 4)) || (e = yb.alloc(m * 4)) || (e = gb.alloc(m * 4))) return e;
  std::vector<int> origins(3 * B);
  std::vector<double> losses;
  int best_iters = 0x7fffffff, best_step = -1, best_t = adam_t0, best_restart = 0;
  int restart = 0;
  std::vector<double> best_losses;
  auto score = [&](int step) -> int {
    int it = 0, ee, tt;
    if ((ee = cnn_state_get(t, state.get<float>(), &tt))) return ee;
    if ((ee = validate(vg.c, vrho.get<double>(), vphi.get<double>(),
                       (size_t)O.val_grid * O.val_grid * O.val_grid, state.get<float>(), pc, &it)))
      return ee;
    if (it < best_iters) {
      best_iters = it;
      best_step = step;
      best_t = tt;
      best_restart = restart;
      best_losses = losses;
      CK(cudaMemcpyAsync(best.get<float>(), state.get<float>(), 3 * kWeightsN * sizeof(float),
                         cudaMemcpyDeviceToDevice, c->stream));
    }
    return PIC_OK;
  };
  for (restart = 0; restart < O.restarts; ++restart) {
    // each restart: its own initial weights and crop stream (restart 0 is the plain training)
    const uint64_t key = (O.seed + 0x9E3779B97F4A7C15ull * (uint64_t)restart) ^ 0xC7A1B5EEDull;
    if (O.resume) {
      if ((e = cnn_state_set(t, start.get<float>(), adam_t0))) return e;
    } else {
      std::vector<float> w0(kWeightsN);
      initial_weights(O.seed + 7919ull * (uint64_t)restart, w0.data());
      if ((e = pic_cnn_set_weights(t, w0.data()))) return e;
    }
    const int adam_t = adam_t0;
    losses.clear();
    for (int step = 0; step < O.steps; ++step) {
      const uint32_t ctr = (uint32_t)(adam_t + step);
      const U4 pick = philox({ctr, 0u, 0u, 0u}, key);
      const Set& S = sets[pick.x % (uint32_t)O.sets];
      const size_t sn = pick.y % (uint32_t)S.r.size();
      for (int b = 0; b < B; ++b) {
        const U4 r = philox({ctr, 1u + (uint32_t)b, 0u, 0u}, key);
        origins[3 * b] = (int)(r.x % (uint32_t)N);
        origins[3 * b + 1] = (int)(r.y % (uint32_t)N);
        origins[3 * b + 2] = (int)(r.z % (uint32_t)N);
      }
      double loss = 0.0;
      if ((e = pic_cnn_make_batch(t, S.r[sn], S.a, S.b[sn], origins.data(), B, D, xb.get<float>(), tb.get<float>(),
                                  h * h)) ||
          (e = pic_cnn_forward(t, xb.get<float>(), yb.get<float>(), B, D)) ||
          (e = pic_cnn_loss(t, yb.get<float>(), tb.get<float>(), B, D, gb.get<float>(), &loss)) ||
          (e = pic_cnn_backward(t, gb.get<float>(), B, D)) || (e = pic_cnn_adam(t, O.lr)))
        return e;
      losses.push_back(loss);
      if (O.validate_every > 0 && (step + 1) % O.validate_every == 0 && step + 1 < O.steps && (e = score(step + 1)))
        return e;
    }
    if (O.validate_every > 0 && (e = score(O.steps))) return e;
  }  // restarts
  int final_t = 0;
  if (O.validate_every > 0) {
    losses = best_losses;
    if ((e = cnn_state_set(c, best.get<float>(), best_t))) return e;
    final_t = best_t;
  } else {
    if ((e = cnn_state_get(t, state.get<float>(), &final_t)) || (e = cnn_state_set(c, state.get<float>(), final_t)))
      return e;
  }
  CK(cudaStreamSynchronize(c->stream));
  if (info) {
    memset(info, 0, sizeof(*info));
    info->steps = O.steps;
    info->adam_steps = final_t;
    const size_t k1 = losses.size() < 10 ? losses.size() : 10, k2 = losses.size() < 50 ? losses.size() : 50;
    for (size_t i = 0; i < k1; ++i) info->loss_first += losses[i] / (double)k1;
    for (size_t i = losses.size() - k2; i < losses.size(); ++i) info->loss_last += losses[i] / (double)k2;
    info->best_step = O.validate_every > 0 ? best_step : O.steps;
    info->best_iters = O.validate_every > 0 ? best_iters : -1;
    info->best_restart = best_restart;
    timespec t_end;
    clock_gettime(CLOCK_MONOTONIC, &t_end);
    info->seconds = (double)(t_end.tv_sec - t_start.tv_sec) + 1e-9 * (double)(t_end.tv_nsec - t_start.tv_nsec);
  }
  return PIC_OK;
}
