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
// the inverse transforms are complex-to-real. FP64 throughout.
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
  double* G = nullptr;                 // M^3 spread charge, then each field component
  cufftDoubleComplex* Gh = nullptr;    // M x M x (M/2 + 1)
  cufftDoubleComplex* F = nullptr;     // M x M x (M/2 + 1)
  double* phihat = nullptr;            // window transform at the signed modes -N/2 .. N/2 - 1
};

void pif_state_free(PifState* s) {
  if (!s) return;
  if (s->have_fwd) cufftDestroy(s->fwd);
  if (s->have_inv) cufftDestroy(s->inv);
  cudaFree(s->G);
  cudaFree(s->Gh);
  cudaFree(s->F);
  cudaFree(s->phihat);
  delete s;
}

namespace {

constexpr int kPifMaxW = 16;

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
  const int c[3] = {(int)(r3.z & 0xFFFFu), (int)(r3.z >> 16), (int)(r3.w & 0xFFFFu)};
#pragma unroll
  for (int d = 0; d < 3; ++d) u[d] = 2.0 * ((double)c[d] + (double)(f[d] >> 11) * (1.0 / 9007199254740992.0));
}

// The window's w weights along one axis and the first grid index (mod M).
__device__ __forceinline__ int axis_weights(double u, int w, double beta, int M, double* wt) {
  const int g0 = (int)ceil(u - 0.5 * w);
  for (int a = 0; a < w; ++a) wt[a] = es_window(2.0 * (u - (double)(g0 + a)) / w, beta);
  int g = g0 % M;
  return g < 0 ? g + M : g;
}

// Type-1 spreading: G[g] += q phi_x phi_y phi_z over the w^3 window of each particle.
__global__ void __launch_bounds__(128) k_pif_spread(const PRec* __restrict__ P, uint64_t np, int M, int w,
                                                    double beta, double q, double* G) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double u[3];
  grid_units(P, p, u);
  double wx[kPifMaxW], wy[kPifMaxW], wz[kPifMaxW];
  const int gx = axis_weights(u[0], w, beta, M, wx), gy = axis_weights(u[1], w, beta, M, wy),
            gz = axis_weights(u[2], w, beta, M, wz);
  const size_t Ms = M;
  for (int c = 0; c < w; ++c) {
    const int z = gz + c < M ? gz + c : gz + c - M;
    const double qz = q * wz[c];
    for (int b = 0; b < w; ++b) {
      const int y = gy + b < M ? gy + b : gy + b - M;
      const double qzy = qz * wy[b];
      double* row = G + ((size_t)z * Ms + y) * Ms;
      for (int a = 0; a < w; ++a) {
        const int x = gx + a < M ? gx + a : gx + a - M;
        atomicAdd(row + x, qzy * wx[a]);
      }
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

// Type-2 interpolation of one field component: Ep[p] = sum over the window of f[g] phi.
__global__ void __launch_bounds__(128) k_pif_gather(const PRec* __restrict__ P, uint64_t np, int M, int w, double beta,
                                                    const double* __restrict__ f, double* __restrict__ Ep) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double u[3];
  grid_units(P, p, u);
  double wx[kPifMaxW], wy[kPifMaxW], wz[kPifMaxW];
  const int gx = axis_weights(u[0], w, beta, M, wx), gy = axis_weights(u[1], w, beta, M, wy),
            gz = axis_weights(u[2], w, beta, M, wz);
  const size_t Ms = M;
  double acc = 0.0;
  for (int c = 0; c < w; ++c) {
    const int z = gz + c < M ? gz + c : gz + c - M;
    double sz = 0.0;
    for (int b = 0; b < w; ++b) {
      const int y = gy + b < M ? gy + b : gy + b - M;
      const double* row = f + ((size_t)z * Ms + y) * Ms;
      double sy = 0.0;
      for (int a = 0; a < w; ++a) {
        const int x = gx + a < M ? gx + a : gx + a - M;
        sy = fma(__ldg(row + x), wx[a], sy);
      }
      sz = fma(sy, wy[b], sz);
    }
    acc = fma(sz, wz[c], acc);
  }
  Ep[p] = acc;
}

// The window width for a relative tolerance (about one digit per point with
// sigma = 2), 4 <= w <= kPifMaxW.
int width_for(double tol) {
  int w = (int)ceil(-log10(tol > 0.0 ? tol : 1e-16)) + 1;
  if (w < 4) w = 4;
  if (w > kPifMaxW) w = kPifMaxW;
  return w;
}

int ensure_pif(pic_ctx* c, int w) {
  if (c->pif && c->pif->N == c->N && c->pif->w == w) return PIC_OK;
  pif_state_free(c->pif);
  c->pif = nullptr;
  PifState* s = new (std::nothrow) PifState();
  if (!s) return PIC_ENOMEM;
  s->N = c->N;
  s->M = 2 * c->N;
  s->w = w;
  s->beta = 2.30 * w;
  const size_t M = s->M, nr = M * M * M, nc = M * M * (M / 2 + 1);
  int e = PIC_OK;
  if (cudaMalloc(reinterpret_cast<void**>(&s->G), nr * sizeof(double)) != cudaSuccess ||
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
  if (!e && cufftPlan3d(&s->fwd, s->M, s->M, s->M, CUFFT_D2Z) == CUFFT_SUCCESS) s->have_fwd = true;
  else if (!e) e = PIC_ECUDA;
  if (!e && cufftPlan3d(&s->inv, s->M, s->M, s->M, CUFFT_Z2D) == CUFFT_SUCCESS) s->have_inv = true;
  else if (!e) e = PIC_ECUDA;
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
  int e;
  if ((e = ensure_pif(c, width_for(tol)))) return e;
  PifState* s = c->pif;
  if (cufftSetStream(s->fwd, c->stream) != CUFFT_SUCCESS || cufftSetStream(s->inv, c->stream) != CUFFT_SUCCESS)
    return PIC_ECUDA;
  const size_t M = s->M, nr = M * M * M, nc = M * M * (M / 2 + 1);
  const double L = c->grid.L;
  const PRec* P = c->prec[c->cur];
  const unsigned pb = (unsigned)((c->np + 127) / 128);
  CK(cudaMemsetAsync(s->G, 0, nr * sizeof(double), c->stream));
  launch(c, k_pif_spread, pb, 128, 0, P, c->np, s->M, s->w, s->beta, -L * L * L / (double)c->np, s->G);
  if (cufftExecD2Z(s->fwd, s->G, s->Gh) != CUFFT_SUCCESS) return PIC_ECUDA;
  size_t b = (nc + 255) / 256;
  const size_t cap = (size_t)c->sms * 16;
  const unsigned grid = (unsigned)(b < cap ? b : cap);
  const double pi = 3.14159265358979323846;
  for (int d = 0; d < 3; ++d) {
    launch(c, k_pif_modes, grid, 256, 0, (const cufftDoubleComplex*)s->Gh, s->F, s->N, s->M,
           (const double*)s->phihat, 2.0 * pi / L, 1.0 / (L * L * L), d);
    // the complex-to-real transform overwrites F; G is free again after the forward transform
    if (cufftExecZ2D(s->inv, s->F, s->G) != CUFFT_SUCCESS) return PIC_ECUDA;
    launch(c, k_pif_gather, pb, 128, 0, P, c->np, s->M, s->w, s->beta, (const double*)s->G,
           Ep + (size_t)d * c->np);
  }
  CK(cudaGetLastError());
  return PIC_OK;
}

}  // namespace pic
