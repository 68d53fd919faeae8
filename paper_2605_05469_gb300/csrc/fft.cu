// FFT pseudo-spectral periodic Poisson solve (Sec. 3.1), the solver the paper
// sets beside PCG: phi = F^-1(rho_hat / k^2), E = F^-1(-i k rho_hat / k^2),
// k = 2 pi m / L. The 3-D real-to-complex transforms are cuFFT's (FP64, a
// library FFT like a library GEMM); the spectral multiplications are the
// kernels below. The k = 0 mode is zero (mean-zero phi, neutralising
// background); the Nyquist mode m_d = N/2 of the derivative along d is zero
// (a real field has no consistent derivative there).
#include <cufft.h>

#include <new>

#include "ctx.h"
#include "fft.h"

namespace pic {

struct FftState {
  int N = 0;
  cufftHandle fwd = 0, inv = 0;
  bool have_fwd = false, have_inv = false;
  cufftDoubleComplex *F = nullptr, *W = nullptr;  // N x N x (N/2 + 1) each
};

void fft_state_free(FftState* s) {
  if (!s) return;
  if (s->have_fwd) cufftDestroy(s->fwd);
  if (s->have_inv) cufftDestroy(s->inv);
  if (s->F) cudaFree(s->F);
  if (s->W) cudaFree(s->W);
  delete s;
}

namespace {

// Mode number m of index i along a transformed axis of length N (FFT order).
__device__ __forceinline__ int mode_of(int i, int N) { return i <= N / 2 ? i : i - N; }

// F <- F / (k^2 N^3) (the inverse transforms are unnormalised), 0 at k = 0.
__global__ void __launch_bounds__(256) k_spec_phi(cufftDoubleComplex* F, int N, double two_pi_over_L) {
  const int Nh = N / 2 + 1;
  const size_t total = (size_t)N * N * Nh;
  const double scale = 1.0 / ((double)N * N * N);
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(q % Nh);
    const int iy = (int)((q / Nh) % N), iz = (int)(q / ((size_t)Nh * N));
    const double kx = two_pi_over_L * ix, ky = two_pi_over_L * mode_of(iy, N), kz = two_pi_over_L * mode_of(iz, N);
    const double k2 = kx * kx + ky * ky + kz * kz;
    const double f = k2 > 0.0 ? scale / k2 : 0.0;
    cufftDoubleComplex v = F[q];
    v.x *= f;
    v.y *= f;
    F[q] = v;
  }
}

// W <- -i k_d F along axis d (0 = x, 1 = y, 2 = z), the Nyquist mode zero.
__global__ void __launch_bounds__(256) k_spec_grad(const cufftDoubleComplex* __restrict__ F,
                                                   cufftDoubleComplex* __restrict__ W, int N, double two_pi_over_L,
                                                   int d) {
  const int Nh = N / 2 + 1;
  const size_t total = (size_t)N * N * Nh;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(q % Nh);
    const int iy = (int)((q / Nh) % N), iz = (int)(q / ((size_t)Nh * N));
    const int i = d == 0 ? ix : (d == 1 ? iy : iz);
    const double k = (i == N / 2) ? 0.0 : two_pi_over_L * (d == 0 ? i : mode_of(i, N));
    const cufftDoubleComplex v = F[q];
    // -i k (a + i b) = k b - i k a
    W[q] = make_cuDoubleComplex(k * v.y, -k * v.x);
  }
}

int ensure_fft(pic_ctx* c) {
  if (c->fft && c->fft->N == c->N) return PIC_OK;
  fft_state_free(c->fft);
  c->fft = nullptr;
  FftState* s = new (std::nothrow) FftState();
  if (!s) return PIC_ENOMEM;
  s->N = c->N;
  const size_t nc = (size_t)c->N * c->N * (c->N / 2 + 1);
  int e = PIC_OK;
  if (cudaMalloc(reinterpret_cast<void**>(&s->F), nc * sizeof(cufftDoubleComplex)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&s->W), nc * sizeof(cufftDoubleComplex)) != cudaSuccess) {
    cudaGetLastError();
    e = PIC_ENOMEM;
  }
  if (!e && cufftPlan3d(&s->fwd, c->N, c->N, c->N, CUFFT_D2Z) == CUFFT_SUCCESS) s->have_fwd = true;
  else if (!e) e = PIC_ECUDA;
  if (!e && cufftPlan3d(&s->inv, c->N, c->N, c->N, CUFFT_Z2D) == CUFFT_SUCCESS) s->have_inv = true;
  else if (!e) e = PIC_ECUDA;
  if (e) {
    fft_state_free(s);
    return e;
  }
  c->fft = s;
  return PIC_OK;
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" int pic_fft_solve(pic_ctx* c, const double* rho, double* phi, double* E) {
  if (!c || !rho || !phi) return PIC_EINVAL;
  if (!c->has_grid) return PIC_ESTATE;
  int e;
  if ((e = ensure_fft(c))) return e;
  PhaseScope ps(c, PIC_PHASE_SOLVE);
  FftState* s = c->fft;
  if (cufftSetStream(s->fwd, c->stream) != CUFFT_SUCCESS || cufftSetStream(s->inv, c->stream) != CUFFT_SUCCESS)
    return PIC_ECUDA;
  const int N = c->N;
  const double tk = 2.0 * 3.14159265358979323846 / c->grid.L;
  const size_t nc = (size_t)N * N * (N / 2 + 1);
  size_t b = (nc + 255) / 256;
  const size_t cap = (size_t)c->sms * 16;
  const unsigned grid = (unsigned)(b < cap ? b : cap);
  if (cufftExecD2Z(s->fwd, const_cast<double*>(rho), s->F) != CUFFT_SUCCESS) return PIC_ECUDA;
  launch(c, k_spec_phi, grid, 256, 0, s->F, N, tk);
  if (E) {
    for (int d = 0; d < 3; ++d) {
      launch(c, k_spec_grad, grid, 256, 0, (const cufftDoubleComplex*)s->F, s->W, N, tk, d);
      // the complex-to-real transform overwrites its input (W)
      if (cufftExecZ2D(s->inv, s->W, E + (size_t)d * c->n) != CUFFT_SUCCESS) return PIC_ECUDA;
    }
  }
  if (cufftExecZ2D(s->inv, s->F, phi) != CUFFT_SUCCESS) return PIC_ECUDA;
  CK(cudaGetLastError());
  return PIC_OK;
}
