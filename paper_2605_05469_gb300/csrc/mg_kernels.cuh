// Geometric multigrid V-cycle, the preconditioner of flexible CG beyond the
// paper's Jacobi-PCG (the paper names multigrid as the follow-on, Sec. 6).
//
// All levels work in the solver's scaled units: on level l (N_l^3 nodes,
// spacing h_l = 2^l h) the system is A^ x = r^ with A^ = 6 I - (sum of the
// 6 periodic neighbours), the same integer stencil on every level, and
// r^ = h_l^2 r. Hence
//   damped Jacobi   x <- x + (omega/6)(r^ - A^ x),     omega = 6/7;
//   coarse r.h.s.   r^_c = 4 R (r^ - A^ x)            (h_c^2 = 4 h^2);
//   correction      x <- x + P e_c                    (no factor);
// R full weighting (coarse node I <- fine 2I and its 26 neighbours, weights
// prod_d w(o_d), w(0) = 1/2, w(+-1) = 1/4), P trilinear interpolation
// (R = P^T / 8). FP32 throughout.
#pragma once
#include "common.cuh"

namespace pic {
namespace mg {

constexpr float kOmega = 6.0f / 7.0f;
constexpr int kSmallN = 16;          // levels at or below this size run in one CTA
constexpr int kCoarsestN = 4;        // coarsest level (or the first odd one)
constexpr int kCoarseSweeps = 40;    // damped Jacobi sweeps there
constexpr int kSmallThreads = 1024;

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// A^ x at node (i, j, k) of an N^3 periodic grid, x-fastest layout.
__device__ __forceinline__ float apply_hat(const float* __restrict__ x, int N, int i, int j, int k) {
  const size_t Ns = N;
  const size_t row = ((size_t)k * Ns + j) * Ns;
  const float c = x[row + i];
  const float xm = x[row + wrapi(i - 1, N)], xp = x[row + wrapi(i + 1, N)];
  const float ym = x[((size_t)k * Ns + wrapi(j - 1, N)) * Ns + i], yp = x[((size_t)k * Ns + wrapi(j + 1, N)) * Ns + i];
  const float zm = x[((size_t)wrapi(k - 1, N) * Ns + j) * Ns + i], zp = x[((size_t)wrapi(k + 1, N) * Ns + j) * Ns + i];
  return 6.0f * c - (((xm + xp) + (ym + yp)) + (zm + zp));
}

// out = x + (omega/6)(r - A^ x); x == nullptr reads x as zero.
// Every kernel returns at once when the solve it serves has finished (done
// != nullptr and *done set), so batches launched past convergence cost no work.
__global__ void __launch_bounds__(256) k_mg_jacobi(const float* __restrict__ x, const float* __restrict__ r,
                                                   float* __restrict__ out, int N, const int* done) {
  if (done && *done) return;
  const size_t n = (size_t)N * N * N;
  const float w = kOmega / 6.0f;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const float rv = __ldg(r + c);
    if (!x) {
      out[c] = w * rv;
      continue;
    }
    const int i = (int)(c % N), j = (int)((c / N) % N), k = (int)(c / ((size_t)N * N));
    out[c] = x[c] + w * (rv - apply_hat(x, N, i, j, k));
  }
}

// res = r - A^ x.
__global__ void __launch_bounds__(256) k_mg_residual(const float* __restrict__ x, const float* __restrict__ r,
                                                     float* __restrict__ res, int N, const int* done) {
  if (done && *done) return;
  const size_t n = (size_t)N * N * N;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % N), j = (int)((c / N) % N), k = (int)(c / ((size_t)N * N));
    res[c] = __ldg(r + c) - apply_hat(x, N, i, j, k);
  }
}

// rc = 4 R res (coarse grid Nf/2).
__global__ void __launch_bounds__(256) k_mg_restrict(const float* __restrict__ res, float* __restrict__ rc, int Nf,
                                                     const int* done) {
  if (done && *done) return;
  const int Nc = Nf / 2;
  const size_t nc = (size_t)Nc * Nc * Nc, Ns = Nf;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(c % Nc), J = (int)((c / Nc) % Nc), K = (int)(c / ((size_t)Nc * Nc));
    float acc = 0.f;
#pragma unroll
    for (int oz = -1; oz <= 1; ++oz) {
      const size_t zb = (size_t)wrapi(2 * K + oz, Nf) * Ns;
      const float wz = oz ? 0.25f : 0.5f;
      float sy = 0.f;
#pragma unroll
      for (int oy = -1; oy <= 1; ++oy) {
        const float* rowp = res + (zb + (size_t)wrapi(2 * J + oy, Nf)) * Ns;
        const float wy = oy ? 0.25f : 0.5f;
        const float sx = 0.25f * __ldg(rowp + wrapi(2 * I - 1, Nf)) + 0.5f * __ldg(rowp + 2 * I) +
                         0.25f * __ldg(rowp + wrapi(2 * I + 1, Nf));
        sy = fmaf(wy, sx, sy);
      }
      acc = fmaf(wz, sy, acc);
    }
    rc[c] = 4.0f * acc;
  }
}

// x += P ec (fine grid 2 Nc).
__global__ void __launch_bounds__(256) k_mg_prolong_add(float* __restrict__ x, const float* __restrict__ ec, int Nc,
                                                        const int* done) {
  if (done && *done) return;
  const int Nf = 2 * Nc;
  const size_t n = (size_t)Nf * Nf * Nf, Ns = Nc;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % Nf), j = (int)((c / Nf) % Nf), k = (int)(c / ((size_t)Nf * Nf));
    const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
    const int I1 = (i & 1) ? wrapi(I0 + 1, Nc) : I0, J1 = (j & 1) ? wrapi(J0 + 1, Nc) : J0,
              K1 = (k & 1) ? wrapi(K0 + 1, Nc) : K0;
    // mean of the 1, 2, 4 or 8 distinct coarse nodes around the fine node
    const float wx = (i & 1) ? 0.5f : 1.f, wy = (j & 1) ? 0.5f : 1.f, wz = (k & 1) ? 0.5f : 1.f;
    auto e = [&](int I, int J, int K) { return __ldg(ec + ((size_t)K * Ns + J) * Ns + I); };
    float v = e(I0, J0, K0);
    if (i & 1) v += e(I1, J0, K0);
    if (j & 1) {
      v += e(I0, J1, K0);
      if (i & 1) v += e(I1, J1, K0);
    }
    if (k & 1) {
      v += e(I0, J0, K1);
      if (i & 1) v += e(I1, J0, K1);
      if (j & 1) {
        v += e(I0, J1, K1);
        if (i & 1) v += e(I1, J1, K1);
      }
    }
    x[c] += wx * wy * wz * v;
  }
}

// x += y.
__global__ void __launch_bounds__(256) k_mg_add(float* __restrict__ x, const float* __restrict__ y, size_t n4,
                                                const int* done) {
  if (done && *done) return;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n4; c += (size_t)gridDim.x * blockDim.x) {
    float4 a = reinterpret_cast<float4*>(x)[c];
    const float4 b = __ldg(reinterpret_cast<const float4*>(y) + c);
    a.x += b.x;
    a.y += b.y;
    a.z += b.z;
    a.w += b.w;
    reinterpret_cast<float4*>(x)[c] = a;
  }
}

// ---------------------------------------------------------------------------
// The cycle below kSmallN^3 in one CTA: every level's x, r and a scratch
// array in shared memory, one barrier per pass.
// ---------------------------------------------------------------------------
struct SmallLevels {
  int n;          // number of levels (the first is the input grid)
  int N[8];       // nodes per dimension
  int off[8];     // element offset of each level's arrays in each region
  int total;      // elements per region
};

__device__ __forceinline__ void sm_jacobi(const float* x, const float* r, float* out, int N, bool x_zero) {
  const int n = N * N * N;
  const float w = kOmega / 6.0f;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    if (x_zero) {
      out[c] = w * r[c];
    } else {
      const int i = c % N, j = (c / N) % N, k = c / (N * N);
      out[c] = x[c] + w * (r[c] - apply_hat(x, N, i, j, k));
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void sm_copy(const float* a, float* b, int n) {
  for (int c = threadIdx.x; c < n; c += blockDim.x) b[c] = a[c];
  __syncthreads();
}

__global__ void __launch_bounds__(kSmallThreads) k_mg_small(const float* __restrict__ r_in, float* __restrict__ x_out,
                                                            SmallLevels S, int nu, const int* done) {
  if (done && *done) return;
  extern __shared__ float sm[];
  float* X = sm;                 // solutions
  float* R = sm + S.total;       // right-hand sides
  float* T = sm + 2 * S.total;   // scratch (Jacobi ping-pong, residuals)
  const int n0 = S.N[0] * S.N[0] * S.N[0];
  for (int c = threadIdx.x; c < n0; c += blockDim.x) R[c] = r_in[c];
  __syncthreads();
  // down: pre-smooth, residual, restrict
  for (int l = 0; l + 1 < S.n; ++l) {
    const int N = S.N[l], n = N * N * N;
    float *x = X + S.off[l], *r = R + S.off[l], *t = T + S.off[l];
    for (int s = 0; s < nu; ++s) {
      sm_jacobi(s ? x : nullptr, r, t, N, s == 0);
      sm_copy(t, x, n);
    }
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int i = c % N, j = (c / N) % N, k = c / (N * N);
      t[c] = r[c] - apply_hat(x, N, i, j, k);
    }
    __syncthreads();
    const int Nc = S.N[l + 1], nc = Nc * Nc * Nc;
    float* rc = R + S.off[l + 1];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const int I = c % Nc, J = (c / Nc) % Nc, K = c / (Nc * Nc);
      float acc = 0.f;
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            const float w = (ox ? 0.25f : 0.5f) * (oy ? 0.25f : 0.5f) * (oz ? 0.25f : 0.5f);
            acc += w * t[(wrapi(2 * K + oz, N) * N + wrapi(2 * J + oy, N)) * N + wrapi(2 * I + ox, N)];
          }
      rc[c] = 4.0f * acc;
    }
    __syncthreads();
  }
  // coarsest: damped Jacobi sweeps from zero
  {
    const int l = S.n - 1, N = S.N[l], n = N * N * N;
    float *x = X + S.off[l], *r = R + S.off[l], *t = T + S.off[l];
    for (int s = 0; s < kCoarseSweeps; ++s) {
      sm_jacobi(s ? x : nullptr, r, t, N, s == 0);
      sm_copy(t, x, n);
    }
  }
  // up: prolong-add, post-smooth
  for (int l = S.n - 2; l >= 0; --l) {
    const int N = S.N[l], n = N * N * N, Nc = S.N[l + 1];
    float *x = X + S.off[l], *r = R + S.off[l], *t = T + S.off[l];
    const float* ec = X + S.off[l + 1];
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int i = c % N, j = (c / N) % N, k = c / (N * N);
      const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
      const int I1 = (i & 1) ? wrapi(I0 + 1, Nc) : I0, J1 = (j & 1) ? wrapi(J0 + 1, Nc) : J0,
                K1 = (k & 1) ? wrapi(K0 + 1, Nc) : K0;
      const float w = ((i & 1) ? 0.5f : 1.f) * ((j & 1) ? 0.5f : 1.f) * ((k & 1) ? 0.5f : 1.f);
      auto e = [&](int I, int J, int K) { return ec[(K * Nc + J) * Nc + I]; };
      float v = e(I0, J0, K0);
      if (i & 1) v += e(I1, J0, K0);
      if (j & 1) {
        v += e(I0, J1, K0);
        if (i & 1) v += e(I1, J1, K0);
      }
      if (k & 1) {
        v += e(I0, J0, K1);
        if (i & 1) v += e(I1, J0, K1);
        if (j & 1) {
          v += e(I0, J1, K1);
          if (i & 1) v += e(I1, J1, K1);
        }
      }
      x[c] += w * v;
    }
    __syncthreads();
    for (int s = 0; s < nu; ++s) {
      sm_jacobi(x, r, t, N, false);
      sm_copy(t, x, n);
    }
  }
  for (int c = threadIdx.x; c < n0; c += blockDim.x) x_out[c] = X[c];
}

}  // namespace mg
}  // namespace pic
