// Particle-in-Fourier field (Sec. 3.4, Appendix A). The charge goes straight
// to the Fourier modes K_N (N = the context grid, modes -N/2..N/2-1) by a
// type-1 NUFFT, Poisson's equation is solved mode by mode and the field is
// evaluated at the particles by a type-2 NUFFT; both NUFFTs follow the
// factorisation of Appendix A: spreading with a compact window onto an
// oversampled grid (sigma = 2, M = 2N points a side), a uniform FFT (cuFFT,
// FP64), and division by the window's Fourier transform at the kept modes;
// type 2 runs the same steps in reverse.
//   window: exponential of semicircle phi(z) = exp(beta (sqrt(1 - z^2) - 1)),
//           |z| <= 1, over w grid points (Barnett, Magland & af Klinteberg,
//           SIAM J. Sci. Comput. 2019), beta = 2.30 w; w from the tolerance;
//   field:  E_hat(k) = -i k rho_hat(k) / (|k|^2 L^3) over the symmetric modes
//           |m_d| <= N/2 - 1 (k != 0), rho_hat(k) = sum_j q_j exp(-i k.x_j),
//           q_j = -L^3 / Np (the electrons; the background is the k = 0 mode).
// The modes of the three field components are formed directly on the
// half spectrum of the real oversampled grid (Hermitian by construction), so
// the inverse transforms are complex-to-real. FP64 arithmetic for tolerances
// below 1e-5; at 1e-5 and above (the paper's runs use 1e-4) the window sums,
// the spread grid and the transforms are FP32, whose rounding (about 1e-6 of
// the field's maximum, measured against the direct sums) stays well inside
// the tolerance, with the particle positions taken to FP32 as an integer grid
// index plus an exact fraction so the window arguments keep full precision.
#include <cufft.h>
#include <math.h>

#include <new>
#include <vector>

#include "ctx.h"
#include "pif.h"

namespace pic {

struct PifState {
  int N = 0, M = 0, w = 0;
  double beta = 0.0;
  cufftHandle fwd = 0, inv = 0;
  bool have_fwd = false, have_inv = false;
  double* G = nullptr;                 // M^3 spread charge, then the field's x component
  double* Gyz[2] = {nullptr, nullptr}; // M^3 each: the field's y and z components
  cufftDoubleComplex* Gh = nullptr;    // M x M x (M/2 + 1)
  cufftDoubleComplex* F = nullptr;     // M x M x (M/2 + 1)
  double* phihat = nullptr;            // window transform at the signed modes -N/2 .. N/2 - 1
  // FP32 form (tolerances >= 1e-5)
  bool f32 = false;
  cufftHandle fwd32 = 0, inv32 = 0;
  bool have_fwd32 = false, have_inv32 = false;
  float* G32 = nullptr;                 // M^3: spread charge, then E_x
  float* Gyz32[2] = {nullptr, nullptr}; // M^3 each: E_y, E_z
  cufftComplex* Gh32 = nullptr;         // M x M x (M/2 + 1)
  cufftComplex* F32 = nullptr;
};

void pif_state_free(PifState* s) {
  if (!s) return;
  if (s->have_fwd) cufftDestroy(s->fwd);
  if (s->have_inv) cufftDestroy(s->inv);
  cudaFree(s->G);
  cudaFree(s->Gyz[0]);
  cudaFree(s->Gyz[1]);
  cudaFree(s->Gh);
  cudaFree(s->F);
  cudaFree(s->phihat);
  if (s->have_fwd32) cufftDestroy(s->fwd32);
  if (s->have_inv32) cufftDestroy(s->inv32);
  cudaFree(s->G32);
  cudaFree(s->Gyz32[0]);
  cudaFree(s->Gyz32[1]);
  cudaFree(s->Gh32);
  cudaFree(s->F32);
  delete s;
}

namespace {

constexpr int kPifMinW = 4, kPifMaxW = 16;

__host__ __device__ inline double es_window(double z, double beta) {
  return fabs(z) <= 1.0 ? exp(beta * (sqrt(1.0 - z * z) - 1.0)) : 0.0;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton's method on the
// Legendre polynomial from Chebyshev initial guesses; Golub & Welsch give the
// same rule).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  // P_n(t) and P_n'(t) = n (t P_n - P_{n-1}) / (t^2 - 1) by the three-term recurrence
  auto legendre = [n](double t, double& pn, double& dpn) {
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    pn = p1;
    dpn = n * (t * p1 - p0) / (t * t - 1.0);
  };
  for (int i = 0; i < n; ++i) {
    double t = cos(pi * (i + 0.75) / (n + 0.5));
    double pn, dpn;
    for (int it = 0; it < 100; ++it) {
      legendre(t, pn, dpn);
      const double dt = pn / dpn;
      t -= dt;
      if (fabs(dt) <= 1e-15 * fabs(t) + 1e-300) break;
    }
    legendre(t, pn, dpn);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dpn * dpn);
  }
}

// Continuous Fourier transform of the window in grid units,
// phi_hat(k) = int phi(2 x / w) exp(-i k x) dx over |x| <= w/2 (even: a cosine
// transform), by Gauss-Legendre quadrature.
double window_ft(double k, int w, double beta, const std::vector<double>& gx, const std::vector<double>& gw) {
  double s = 0.0;
  for (size_t i = 0; i < gx.size(); ++i) {
    const double x = 0.5 * w * gx[i];
    s += gw[i] * es_window(gx[i], beta) * cos(k * x);
  }
  return 0.5 * w * s;
}

// Position of particle p in oversampled grid units (M = 2N): u_d = 2 (i_d + f_d 2^-64).
__device__ __forceinline__ void grid_units(const PRec* P, uint64_t p, double u[3]) {
  const uint4* rec = reinterpret_cast<const uint4*>(P + p);
  const uint4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r3 = __ldg(rec + 3);
  const uint64_t f[3] = {((uint64_t)r0.y << 32) | r0.x, ((uint64_t)r0.w << 32) | r0.z, ((uint64_t)r1.y << 32) | r1.x};
  const int c[3] = {cell_x(r3.z), cell_y(r3.z), cell_z(r3.z)};
#pragma unroll
  for (int d = 0; d < 3; ++d) u[d] = 2.0 * ((double)c[d] + (double)(f[d] >> 11) * (1.0 / 9007199254740992.0));
}

// First grid index of the window along one axis (unwrapped: may be negative)
// and its W weights.
template <int W>
__device__ __forceinline__ int axis_weights(double u, double beta, double* wt) {
  const int g0 = (int)ceil(u - 0.5 * W);
#pragma unroll
  for (int a = 0; a < W; ++a) wt[a] = es_window(2.0 * (u - (double)(g0 + a)) / W, beta);
  return g0;
}

// Index g in [-M, 2M) reduced to [0, M).
__device__ __forceinline__ int wrap_m(int g, int M) { return g < 0 ? g + M : (g >= M ? g - M : g); }

// Type-1 spreading: G[g] += q phi_x phi_y phi_z over the W^3 window of each
// particle (FP64 atomics; the particles are in cell order, so the threads of
// a warp update neighbouring points).
template <int W>
__global__ void __launch_bounds__(128) k_pif_spread(const PRec* __restrict__ P, uint64_t np, int M, double beta,
                                                    double q, double* G) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double u[3];
  grid_units(P, p, u);
  double wx[W], wy[W];
  const int gx = axis_weights<W>(u[0], beta, wx), gy = axis_weights<W>(u[1], beta, wy);
  const int gz = (int)ceil(u[2] - 0.5 * W);
  const size_t Ms = M;
  int xs[W];
#pragma unroll
  for (int a = 0; a < W; ++a) xs[a] = wrap_m(gx + a, M);
  for (int c = 0; c < W; ++c) {
    const int z = wrap_m(gz + c, M);
    const double qz = q * es_window(2.0 * (u[2] - (double)(gz + c)) / W, beta);
#pragma unroll
    for (int b = 0; b < W; ++b) {
      const double qzy = qz * wy[b];
      double* row = G + ((size_t)z * Ms + wrap_m(gy + b, M)) * Ms;
#pragma unroll
      for (int a = 0; a < W; ++a) atomicAdd(row + xs[a], qzy * wx[a]);
    }
  }
}

// F = -i k_d G_hat / (|k|^2 L^3 phi_hat^2) on the half spectrum, zero outside
// the symmetric nonzero modes (component d = 0, 1, 2).
__global__ void __launch_bounds__(256) k_pif_modes(const cufftDoubleComplex* __restrict__ Gh,
                                                   cufftDoubleComplex* __restrict__ F, int N, int M,
                                                   const double* __restrict__ phihat, double two_pi_over_L,
                                                   double inv_L3, int d) {
  const int Mh = M / 2 + 1;
  const size_t total = (size_t)M * M * Mh;
  const int lim = N / 2 - 1;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(t % Mh), iy = (int)((t / Mh) % M), iz = (int)(t / ((size_t)Mh * M));
    const int sx = ix, sy = iy <= M / 2 ? iy : iy - M, sz = iz <= M / 2 ? iz : iz - M;
    cufftDoubleComplex out = make_cuDoubleComplex(0.0, 0.0);
    if (sx <= lim && sy >= -lim && sy <= lim && sz >= -lim && sz <= lim && (sx | sy | sz) != 0) {
      const double kx = two_pi_over_L * sx, ky = two_pi_over_L * sy, kz = two_pi_over_L * sz;
      const double k2 = kx * kx + ky * ky + kz * kz;
      const double ph = phihat[sx + N / 2] * phihat[sy + N / 2] * phihat[sz + N / 2];
      const double kd = d == 0 ? kx : (d == 1 ? ky : kz);
      const double f = kd * inv_L3 / (k2 * ph * ph);
      const cufftDoubleComplex g = Gh[t];
      // -i f (a + i b) = f b - i f a
      out = make_cuDoubleComplex(f * g.y, -f * g.x);
    }
    F[t] = out;
  }
}

// Type-2 interpolation of the three field components at once (the window
// weights and the particle's record are shared): Ep[d np + p] = sum over the
// window of f_d[g] phi_x phi_y phi_z.
template <int W>
__global__ void __launch_bounds__(128) k_pif_gather3(const PRec* __restrict__ P, uint64_t np, int M, double beta,
                                                     const double* __restrict__ f0, const double* __restrict__ f1,
                                                     const double* __restrict__ f2, double* __restrict__ Ep) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double u[3];
  grid_units(P, p, u);
  double wx[W], wy[W];
  const int gx = axis_weights<W>(u[0], beta, wx), gy = axis_weights<W>(u[1], beta, wy);
  const int gz = (int)ceil(u[2] - 0.5 * W);
  const size_t Ms = M;
  int xs[W];
#pragma unroll
  for (int a = 0; a < W; ++a) xs[a] = wrap_m(gx + a, M);
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  for (int c = 0; c < W; ++c) {
    const int z = wrap_m(gz + c, M);
    const double wz = es_window(2.0 * (u[2] - (double)(gz + c)) / W, beta);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int b = 0; b < W; ++b) {
      const size_t row = ((size_t)z * Ms + wrap_m(gy + b, M)) * Ms;
      double t0 = 0.0, t1 = 0.0, t2 = 0.0;
#pragma unroll
      for (int a = 0; a < W; ++a) {
        t0 = fma(__ldg(f0 + row + xs[a]), wx[a], t0);
        t1 = fma(__ldg(f1 + row + xs[a]), wx[a], t1);
        t2 = fma(__ldg(f2 + row + xs[a]), wx[a], t2);
      }
      s0 = fma(t0, wy[b], s0);
      s1 = fma(t1, wy[b], s1);
      s2 = fma(t2, wy[b], s2);
    }
    acc0 = fma(s0, wz, acc0);
    acc1 = fma(s1, wz, acc1);
    acc2 = fma(s2, wz, acc2);
  }
  Ep[p] = acc0;
  Ep[np + p] = acc1;
  Ep[2 * np + p] = acc2;
}

// ---- FP32 form --------------------------------------------------------------
// Position of particle p in oversampled grid units as an integer plus an exact
// fraction: u_d = 2 (i_d + f_d 2^-64) = s_d + t_d, t_d in [0, 1) (24 bits).
__device__ __forceinline__ void grid_units32(const PRec* P, uint64_t p, int s[3], float t[3]) {
  const uint4* rec = reinterpret_cast<const uint4*>(P + p);
  const uint4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r3 = __ldg(rec + 3);
  const uint64_t f[3] = {((uint64_t)r0.y << 32) | r0.x, ((uint64_t)r0.w << 32) | r0.z, ((uint64_t)r1.y << 32) | r1.x};
  const int c[3] = {cell_x(r3.z), cell_y(r3.z), cell_z(r3.z)};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    s[d] = 2 * c[d] + (int)(f[d] >> 63);
    t[d] = __uint2float_rn((uint32_t)((f[d] << 1) >> 40)) * 0x1p-24f;
  }
}

__device__ __forceinline__ float es_window32(float z, float beta) {
  return fabsf(z) <= 1.0f ? expf(beta * (sqrtf(1.0f - z * z) - 1.0f)) : 0.0f;
}

// First window index (unwrapped) and the W weights along one axis; the
// distances (s - g0 - a) + t are exact small integers plus the fraction.
template <int W>
__device__ __forceinline__ int axis_weights32(int s, float t, float beta, float* wt) {
  const int g0 = s + (int)ceilf(t - 0.5f * (float)W);
#pragma unroll
  for (int a = 0; a < W; ++a) wt[a] = es_window32(2.0f * ((float)(s - g0 - a) + t) / (float)W, beta);
  return g0;
}

// Type-1 spreading of 128 particles a block. The particles are in cell order,
// so a block's windows usually cover a small box of the oversampled grid: the
// block finds that box, accumulates its windows there in shared memory and
// adds the box to the grid with one global atomic per point (far fewer than
// one per particle and window point, which the L2 atomics bound). A box
// larger than the tile (a block that spans the end of a row of cells) takes
// the direct path.
constexpr int kSpreadTile = 4096;  // floats of shared memory per block (16 KB)

template <int W>
__global__ void __launch_bounds__(128) k_pif_spread32(const PRec* __restrict__ P, uint64_t np, int M, float beta,
                                                      float q, float* G) {
  __shared__ float tile[kSpreadTile];
  __shared__ int lo[3], hi[3];
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = p < np;
  if (threadIdx.x < 3) {
    lo[threadIdx.x] = 0x7fffffff;
    hi[threadIdx.x] = -0x7fffffff;
  }
  float wx[W], wy[W], wz[W];
  int g[3] = {0, 0, 0};
  if (valid) {
    int s[3];
    float t[3];
    grid_units32(P, p, s, t);
    g[0] = axis_weights32<W>(s[0], t[0], beta, wx);
    g[1] = axis_weights32<W>(s[1], t[1], beta, wy);
    g[2] = axis_weights32<W>(s[2], t[2], beta, wz);
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      atomicMin(&lo[d], g[d]);
      atomicMax(&hi[d], g[d]);
    }
  }
  __syncthreads();
  const int bx = hi[0] - lo[0] + W, by = hi[1] - lo[1] + W, bz = hi[2] - lo[2] + W;
  const bool tiled = lo[0] <= hi[0] && (long)bx * by * bz <= kSpreadTile;  // uniform over the block
  const size_t Ms = M;
  if (!tiled) {
    if (!valid) return;
    int xs[W];
#pragma unroll
    for (int a = 0; a < W; ++a) xs[a] = wrap_m(g[0] + a, M);
    for (int c = 0; c < W; ++c) {
      const int z = wrap_m(g[2] + c, M);
      const float qz = q * wz[c];
#pragma unroll
      for (int b = 0; b < W; ++b) {
        const float qzy = qz * wy[b];
        float* row = G + ((size_t)z * Ms + wrap_m(g[1] + b, M)) * Ms;
#pragma unroll
        for (int a = 0; a < W; ++a) atomicAdd(row + xs[a], qzy * wx[a]);
      }
    }
    return;
  }
  const int vol = bx * by * bz;
  for (int i = threadIdx.x; i < vol; i += blockDim.x) tile[i] = 0.f;
  __syncthreads();
  if (valid) {
    const int ox = g[0] - lo[0], oy = g[1] - lo[1], oz = g[2] - lo[2];
    for (int c = 0; c < W; ++c) {
      const float qz = q * wz[c];
#pragma unroll
      for (int b = 0; b < W; ++b) {
        const float qzy = qz * wy[b];
        float* row = tile + ((oz + c) * by + (oy + b)) * bx + ox;
#pragma unroll
        for (int a = 0; a < W; ++a) atomicAdd(row + a, qzy * wx[a]);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < vol; i += blockDim.x) {
    const float v = tile[i];
    if (v != 0.f) {
      const int x = i % bx, y = (i / bx) % by, z = i / (bx * by);
      atomicAdd(G + ((size_t)wrap_m(lo[2] + z, M) * Ms + wrap_m(lo[1] + y, M)) * Ms + wrap_m(lo[0] + x, M), v);
    }
  }
}

__global__ void __launch_bounds__(256) k_pif_modes32(const cufftComplex* __restrict__ Gh, cufftComplex* __restrict__ F,
                                                     int N, int M, const double* __restrict__ phihat,
                                                     double two_pi_over_L, double inv_L3, int d) {
  const int Mh = M / 2 + 1;
  const size_t total = (size_t)M * M * Mh;
  const int lim = N / 2 - 1;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(t % Mh), iy = (int)((t / Mh) % M), iz = (int)(t / ((size_t)Mh * M));
    const int sx = ix, sy = iy <= M / 2 ? iy : iy - M, sz = iz <= M / 2 ? iz : iz - M;
    cufftComplex out = make_cuComplex(0.f, 0.f);
    if (sx <= lim && sy >= -lim && sy <= lim && sz >= -lim && sz <= lim && (sx | sy | sz) != 0) {
      const double kx = two_pi_over_L * sx, ky = two_pi_over_L * sy, kz = two_pi_over_L * sz;
      const double k2 = kx * kx + ky * ky + kz * kz;
      const double ph = phihat[sx + N / 2] * phihat[sy + N / 2] * phihat[sz + N / 2];
      const double kd = d == 0 ? kx : (d == 1 ? ky : kz);
      const float f = (float)(kd * inv_L3 / (k2 * ph * ph));
      const cufftComplex g = Gh[t];
      out = make_cuComplex(f * g.y, -f * g.x);  // -i f (a + i b) = f b - i f a
    }
    F[t] = out;
  }
}

template <int W>
__global__ void __launch_bounds__(128) k_pif_gather3_32(const PRec* __restrict__ P, uint64_t np, int M, float beta,
                                                        const float* __restrict__ f0, const float* __restrict__ f1,
                                                        const float* __restrict__ f2, double* __restrict__ Ep) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  int s[3];
  float t[3];
  grid_units32(P, p, s, t);
  float wx[W], wy[W], wz[W];
  const int gx = axis_weights32<W>(s[0], t[0], beta, wx), gy = axis_weights32<W>(s[1], t[1], beta, wy);
  const int gz = axis_weights32<W>(s[2], t[2], beta, wz);
  const size_t Ms = M;
  int xs[W];
#pragma unroll
  for (int a = 0; a < W; ++a) xs[a] = wrap_m(gx + a, M);
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  for (int c = 0; c < W; ++c) {
    const int z = wrap_m(gz + c, M);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int b = 0; b < W; ++b) {
      const size_t row = ((size_t)z * Ms + wrap_m(gy + b, M)) * Ms;
      float t0 = 0.f, t1 = 0.f, t2 = 0.f;
#pragma unroll
      for (int a = 0; a < W; ++a) {
        t0 = fmaf(__ldg(f0 + row + xs[a]), wx[a], t0);
        t1 = fmaf(__ldg(f1 + row + xs[a]), wx[a], t1);
        t2 = fmaf(__ldg(f2 + row + xs[a]), wx[a], t2);
      }
      s0 = fmaf(t0, wy[b], s0);
      s1 = fmaf(t1, wy[b], s1);
      s2 = fmaf(t2, wy[b], s2);
    }
    acc0 = fmaf(s0, wz[c], acc0);
    acc1 = fmaf(s1, wz[c], acc1);
    acc2 = fmaf(s2, wz[c], acc2);
  }
  Ep[p] = (double)acc0;
  Ep[np + p] = (double)acc1;
  Ep[2 * np + p] = (double)acc2;
}

// Launch kernel template K<W> for the runtime width w (kPifMinW..kPifMaxW).
#define PIF_DISPATCH_W(w, KER, ...)                              \
  switch (w) {                                                   \
    case 4: launch(c, KER<4>, __VA_ARGS__); break;               \
    case 5: launch(c, KER<5>, __VA_ARGS__); break;               \
    case 6: launch(c, KER<6>, __VA_ARGS__); break;               \
    case 7: launch(c, KER<7>, __VA_ARGS__); break;               \
    case 8: launch(c, KER<8>, __VA_ARGS__); break;               \
    case 9: launch(c, KER<9>, __VA_ARGS__); break;               \
    case 10: launch(c, KER<10>, __VA_ARGS__); break;             \
    case 11: launch(c, KER<11>, __VA_ARGS__); break;             \
    case 12: launch(c, KER<12>, __VA_ARGS__); break;             \
    case 13: launch(c, KER<13>, __VA_ARGS__); break;             \
    case 14: launch(c, KER<14>, __VA_ARGS__); break;             \
    case 15: launch(c, KER<15>, __VA_ARGS__); break;             \
    default: launch(c, KER<16>, __VA_ARGS__); break;             \
  }

// The window width for a relative tolerance (about one digit per point with
// sigma = 2), 4 <= w <= kPifMaxW.
int width_for(double tol) {
  int w = (int)ceil(-log10(tol > 0.0 ? tol : 1e-16)) + 1;
  if (w < kPifMinW) w = kPifMinW;
  if (w > kPifMaxW) w = kPifMaxW;
  return w;
}

// The FP32 form for tolerances >= 1e-5 (window widths 4 to 6).
constexpr double kPifF32Tol = 1e-5;

int ensure_pif(pic_ctx* c, int w, bool f32) {
  if (c->pif && c->pif->N == c->N && c->pif->w == w && c->pif->f32 == f32) return PIC_OK;
  pif_state_free(c->pif);
  c->pif = nullptr;
  PifState* s = new (std::nothrow) PifState();
  if (!s) return PIC_ENOMEM;
  s->N = c->N;
  s->M = 2 * c->N;
  s->w = w;
  s->beta = 2.30 * w;
  s->f32 = f32;
  const size_t M = s->M, nr = M * M * M, nc = M * M * (M / 2 + 1);
  int e = PIC_OK;
  if (f32) {
    if (cudaMalloc(reinterpret_cast<void**>(&s->G32), nr * sizeof(float)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&s->Gyz32[0]), nr * sizeof(float)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&s->Gyz32[1]), nr * sizeof(float)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&s->Gh32), nc * sizeof(cufftComplex)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&s->F32), nc * sizeof(cufftComplex)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&s->phihat), (size_t)s->N * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      e = PIC_ENOMEM;
    }
  } else if (cudaMalloc(reinterpret_cast<void**>(&s->G), nr * sizeof(double)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&s->Gyz[0]), nr * sizeof(double)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&s->Gyz[1]), nr * sizeof(double)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&s->Gh), nc * sizeof(cufftDoubleComplex)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&s->F), nc * sizeof(cufftDoubleComplex)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&s->phihat), (size_t)s->N * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    e = PIC_ENOMEM;
  }
  if (!e) {
    std::vector<double> gx, gw, ph(s->N);
    gauss_legendre(200, gx, gw);
    const double pi = 3.14159265358979323846;
    for (int m = -s->N / 2; m < s->N / 2; ++m) ph[m + s->N / 2] = window_ft(2.0 * pi * m / s->M, w, s->beta, gx, gw);
    if (cudaMemcpy(s->phihat, ph.data(), ph.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      e = PIC_ECUDA;
  }
  if (f32) {
    if (!e && cufftPlan3d(&s->fwd32, s->M, s->M, s->M, CUFFT_R2C) == CUFFT_SUCCESS) s->have_fwd32 = true;
    else if (!e) e = PIC_ECUDA;
    if (!e && cufftPlan3d(&s->inv32, s->M, s->M, s->M, CUFFT_C2R) == CUFFT_SUCCESS) s->have_inv32 = true;
    else if (!e) e = PIC_ECUDA;
  } else {
    if (!e && cufftPlan3d(&s->fwd, s->M, s->M, s->M, CUFFT_D2Z) == CUFFT_SUCCESS) s->have_fwd = true;
    else if (!e) e = PIC_ECUDA;
    if (!e && cufftPlan3d(&s->inv, s->M, s->M, s->M, CUFFT_Z2D) == CUFFT_SUCCESS) s->have_inv = true;
    else if (!e) e = PIC_ECUDA;
  }
  if (e) {
    pif_state_free(s);
    return e;
  }
  c->pif = s;
  return PIC_OK;
}

}  // namespace

int pif_field(pic_ctx* c, double tol, double* Ep) {
  if (c->np == 0) return PIC_ESTATE;
  const int w = width_for(tol);
  // the window must fit in one period of the oversampled grid (w <= M = 2N),
  // which also keeps every window index within [-M, 2M) for wrap_m
  if (w > 2 * c->N) return PIC_EINVAL;
  int e;
  const bool f32 = tol >= kPifF32Tol;
  if ((e = ensure_pif(c, w, f32))) return e;
  PifState* s = c->pif;
  const size_t M = s->M, nr = M * M * M, nc = M * M * (M / 2 + 1);
  const double L = c->grid.L;
  const PRec* P = c->prec[c->cur];
  const unsigned pb = (unsigned)((c->np + 127) / 128);
  const double pi = 3.14159265358979323846;
  if (f32) {
    if (cufftSetStream(s->fwd32, c->stream) != CUFFT_SUCCESS || cufftSetStream(s->inv32, c->stream) != CUFFT_SUCCESS)
      return PIC_ECUDA;
    CK(cudaMemsetAsync(s->G32, 0, nr * sizeof(float), c->stream));
    int slot32 = c->prof_on ? c->ker[PIC_KER_PIF_SPREAD].begin(c->stream) : -1;
    PIF_DISPATCH_W(s->w, k_pif_spread32, pb, 128, 0, P, c->np, s->M, (float)s->beta,
                   (float)(-L * L * L / (double)c->np), s->G32);
    if (c->prof_on) c->ker[PIC_KER_PIF_SPREAD].end(slot32, c->stream);
    if (cufftExecR2C(s->fwd32, s->G32, s->Gh32) != CUFFT_SUCCESS) return PIC_ECUDA;
    size_t b32 = (nc + 255) / 256;
    const size_t cap32 = (size_t)c->sms * 16;
    const unsigned grid32 = (unsigned)(b32 < cap32 ? b32 : cap32);
    float* comp32[3] = {s->G32, s->Gyz32[0], s->Gyz32[1]};
    for (int d = 0; d < 3; ++d) {
      launch(c, k_pif_modes32, grid32, 256, 0, (const cufftComplex*)s->Gh32, s->F32, s->N, s->M,
             (const double*)s->phihat, 2.0 * pi / L, 1.0 / (L * L * L), d);
      if (cufftExecC2R(s->inv32, s->F32, comp32[d]) != CUFFT_SUCCESS) return PIC_ECUDA;
    }
    slot32 = c->prof_on ? c->ker[PIC_KER_PIF_GATHER].begin(c->stream) : -1;
    PIF_DISPATCH_W(s->w, k_pif_gather3_32, pb, 128, 0, P, c->np, s->M, (float)s->beta, (const float*)comp32[0],
                   (const float*)comp32[1], (const float*)comp32[2], Ep);
    if (c->prof_on) c->ker[PIC_KER_PIF_GATHER].end(slot32, c->stream);
    CK(cudaGetLastError());
    return PIC_OK;
  }
  if (cufftSetStream(s->fwd, c->stream) != CUFFT_SUCCESS || cufftSetStream(s->inv, c->stream) != CUFFT_SUCCESS)
    return PIC_ECUDA;
  CK(cudaMemsetAsync(s->G, 0, nr * sizeof(double), c->stream));
  int slot = c->prof_on ? c->ker[PIC_KER_PIF_SPREAD].begin(c->stream) : -1;
  PIF_DISPATCH_W(s->w, k_pif_spread, pb, 128, 0, P, c->np, s->M, s->beta, -L * L * L / (double)c->np, s->G);
  if (c->prof_on) c->ker[PIC_KER_PIF_SPREAD].end(slot, c->stream);
  if (cufftExecD2Z(s->fwd, s->G, s->Gh) != CUFFT_SUCCESS) return PIC_ECUDA;
  size_t b = (nc + 255) / 256;
  const size_t cap = (size_t)c->sms * 16;
  const unsigned grid = (unsigned)(b < cap ? b : cap);
  // G is free again after the forward transform: it takes the x component
  double* comp[3] = {s->G, s->Gyz[0], s->Gyz[1]};
  for (int d = 0; d < 3; ++d) {
    launch(c, k_pif_modes, grid, 256, 0, (const cufftDoubleComplex*)s->Gh, s->F, s->N, s->M,
           (const double*)s->phihat, 2.0 * pi / L, 1.0 / (L * L * L), d);
    // the complex-to-real transform overwrites F, which the next component rebuilds
    if (cufftExecZ2D(s->inv, s->F, comp[d]) != CUFFT_SUCCESS) return PIC_ECUDA;
  }
  slot = c->prof_on ? c->ker[PIC_KER_PIF_GATHER].begin(c->stream) : -1;
  PIF_DISPATCH_W(s->w, k_pif_gather3, pb, 128, 0, P, c->np, s->M, s->beta, (const double*)comp[0],
                 (const double*)comp[1], (const double*)comp[2], Ep);
  if (c->prof_on) c->ker[PIC_KER_PIF_GATHER].end(slot, c->stream);
  CK(cudaGetLastError());
  return PIC_OK;
}

}  // namespace pic
