// Particle kernels of the PIC loop (Fig. 1): initial sampling (Sec. 2.1),
// sort by cell, CIC scatter (Eq. 2), E = -grad phi, CIC gather and leapfrog
// push (Eqs. 3-4), field energy (Fig. 2).
//
// Particles are 64-byte FP64 records (PRec). Each step they are counting-sorted
// by cell: the push kernel computes every particle's new cell key and takes
// its rank inside the cell with one integer atomic; a scan turns the cell
// counts into offsets and a scatter moves the particles. The deposit then
// runs one thread per cell over that cell's contiguous particles, sums the 8
// corner weights in registers and issues 8 FP64 reductions per cell instead of
// 8 per particle.
#pragma once
#include "common.cuh"

namespace pic {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    if (i > 0) {
      k.x += W0;
      k.y += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// 53-bit uniform in (0, 1) from two words: ((a >> 5) 2^26 + (b >> 6) + 0.5) 2^-53.
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

// Inverse of F(x) = (x + (alpha/k) sin kx)/L by 12 Newton steps from u L.
__device__ __forceinline__ double inverse_cdf(double u, double L, double alpha, double k) {
  double x = u * L;
  const double ak = alpha / k;
#pragma unroll 1
  for (int it = 0; it < 12; ++it) {
    double sn, cs;
    sincos(k * x, &sn, &cs);
    const double f = (x + ak * sn) / L - u;
    const double fp = (1.0 + alpha * cs) / L;
    x = x - f / fp;
  }
  return x;
}

__device__ __forceinline__ int cell_of(double x, const Grid& g) {
  int i = (int)floor(x * g.inv_h);
  i = i < 0 ? 0 : i;
  return i > g.N - 1 ? g.N - 1 : i;
}

__device__ __forceinline__ uint32_t key_of(double x, double y, double z, const Grid& g) {
  return (uint32_t)cell_of(x, g) + (uint32_t)g.N * ((uint32_t)cell_of(y, g) + (uint32_t)g.N * (uint32_t)cell_of(z, g));
}

__device__ __forceinline__ void rec_pos(const PRec* P, uint64_t p, double& x, double& y, double& z) {
  const double2* r = reinterpret_cast<const double2*>(P + p);
  const double2 a = __ldg(r), b = __ldg(r + 1);
  x = a.x;
  y = a.y;
  z = b.x;
}

// S0: sample particle p of the Landau initial condition, and count its cell.
__global__ void k_init_particles(PRec* P, uint64_t np, uint64_t seed, double alpha, double k, Grid g,
                                 uint32_t* keys, uint32_t* ranks, uint32_t* counts) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  double u[8];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), (uint32_t)j, 0u), key);
    u[2 * j] = u53(r.x, r.y);
    u[2 * j + 1] = u53(r.z, r.w);
  }
  const double x = inverse_cdf(u[0], g.L, alpha, k);
  const double y = inverse_cdf(u[1], g.L, alpha, k);
  const double z = inverse_cdf(u[2], g.L, alpha, k);
  const double two_pi = 6.283185307179586476925286766559;
  // Box-Muller (Box & Muller 1958)
  const double r1 = sqrt(-2.0 * log(u[4])), r2 = sqrt(-2.0 * log(u[6]));
  double s1, c1, s2, c2;
  sincos(two_pi * u[5], &s1, &c1);
  sincos(two_pi * u[7], &s2, &c2);
  double2* rec = reinterpret_cast<double2*>(P + p);
  rec[0] = make_double2(x, y);
  rec[1] = make_double2(z, r1 * c1);
  rec[2] = make_double2(r1 * s1, r2 * c2);
  const uint32_t kk = key_of(x, y, z, g);
  reinterpret_cast<uint4*>(rec)[3] = make_uint4((uint32_t)p, kk, 0u, 0u);
  keys[p] = kk;
  ranks[p] = atomicAdd(&counts[kk], 1u);
}

// Cell keys and in-cell ranks of the current particles (after an external load).
__global__ void k_count_keys(PRec* P, uint64_t np, Grid g, uint32_t* keys, uint32_t* ranks,
                             uint32_t* counts) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double x, y, z;
  rec_pos(P, p, x, y, z);
  const uint32_t kk = key_of(x, y, z, g);
  P[p].key = kk;
  keys[p] = kk;
  ranks[p] = atomicAdd(&counts[kk], 1u);
}

// ---------------------------------------------------------------------------
// Exclusive scan of the cell counts, three phases: chunk sums, scan of the
// chunk sums (one block), chunk-local scans plus chunk offsets.
// ---------------------------------------------------------------------------
constexpr int kScanChunk = 4096;  // 256 threads x 16

__global__ void __launch_bounds__(256) k_scan_chunks(const uint32_t* __restrict__ counts, size_t n,
                                                     uint32_t* __restrict__ chunk_sums) {
  __shared__ uint32_t red[8];
  const size_t base = (size_t)blockIdx.x * kScanChunk;
  uint32_t s = 0;
  for (int i = threadIdx.x; i < kScanChunk; i += 256) {
    const size_t j = base + i;
    if (j < n) s += counts[j];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    chunk_sums[blockIdx.x] = t;
  }
}

// In-place exclusive scan of chunk_sums[0..nc) by one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_chunk_sums(uint32_t* chunk_sums, int nc) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nc; base += 1024) {
    const int i = base + threadIdx.x;
    const uint32_t v = (i < nc) ? chunk_sums[i] : 0u;
    uint32_t incl = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
      uint32_t t = warp_tot[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += u;
      }
      warp_tot[lane] = t;  // inclusive scan of warp totals
    }
    __syncthreads();
    const uint32_t before = (w > 0 ? warp_tot[w - 1] : 0u) + carry;
    if (i < nc) chunk_sums[i] = before + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = before + incl;
    __syncthreads();
  }
}

// offsets[j] = exclusive prefix of counts; offsets[n] = total.
__global__ void __launch_bounds__(256) k_scan_apply(const uint32_t* __restrict__ counts, size_t n,
                                                    const uint32_t* __restrict__ chunk_offsets,
                                                    uint32_t* __restrict__ offsets) {
  __shared__ uint32_t warp_tot[8];
  const size_t base = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * 16;
  uint32_t v[16];
  uint32_t tsum = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v[i] = (base + i < n) ? counts[base + i] : 0u;
    tsum += v[i];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t incl = tsum;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  uint32_t wbefore = 0;
  for (int q = 0; q < w; ++q) wbefore += warp_tot[q];
  uint32_t run = chunk_offsets[blockIdx.x] + wbefore + incl - tsum;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (base + i < n) offsets[base + i] = run;
    run += v[i];
  }
  if (base + 16 >= n && base < n) offsets[n] = run;  // the thread holding the last count
}

// Move particle p to offsets[key] + rank (the other buffer). Each thread
// moves 2 consecutive particles, 64 bytes each as four 16-byte vectors, so
// every destination is written in whole sectors (np % 2 == 0).
__global__ void __launch_bounds__(256) k_scatter(const PRec* __restrict__ src, PRec* __restrict__ dst, uint64_t np,
                                                 const uint32_t* __restrict__ keys,
                                                 const uint32_t* __restrict__ ranks,
                                                 const uint32_t* __restrict__ offsets) {
  const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * q >= np) return;
  const uint2 k2 = __ldg(reinterpret_cast<const uint2*>(keys) + q);
  const uint2 r2 = __ldg(reinterpret_cast<const uint2*>(ranks) + q);
  const uint64_t d0 = (uint64_t)__ldg(offsets + k2.x) + r2.x;
  const uint64_t d1 = (uint64_t)__ldg(offsets + k2.y) + r2.y;
  const uint4* s0 = reinterpret_cast<const uint4*>(src + 2 * q);
  const uint4* s1 = reinterpret_cast<const uint4*>(src + 2 * q + 1);
  uint4 a[4], b[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[i] = __ldg(s0 + i);
    b[i] = __ldg(s1 + i);
  }
  uint4* t0 = reinterpret_cast<uint4*>(dst + d0);
  uint4* t1 = reinterpret_cast<uint4*>(dst + d1);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    t0[i] = a[i];
    t1[i] = b[i];
  }
}

__global__ void k_fill(double* a, size_t n, double v) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) a[i] = v;
}

// ---------------------------------------------------------------------------
// S2: CIC scatter from cell-sorted particles, one thread per cell.
// rho (pre-filled with the +1 background) += (q_p / h^3) sum_p W.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_deposit_cells(const PRec* __restrict__ P,
                                                       const uint32_t* __restrict__ offsets, double* rho, Grid g,
                                                       double qscale) {
  const int N = g.N;
  const size_t n = (size_t)N * N * N;
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const uint32_t b = offsets[c], e = offsets[c + 1];
  if (b == e) return;
  const int ix = (int)(c % N), iy = (int)((c / N) % N), iz = (int)(c / ((size_t)N * N));
  const double cx = (double)ix, cy = (double)iy, cz = (double)iz;
  // the 8 corner weights summed over the cell's particles follow from the
  // moments of the offsets f in [0, 1)^3: sum_p prod_d (f_d or 1 - f_d)
  // expands into the count and sums of f_x, f_y, f_z, f_x f_y, f_x f_z,
  // f_y f_z, f_x f_y f_z (14 FP64 operations per particle instead of 18)
  double mx = 0, my = 0, mz = 0, mxy = 0, mxz = 0, myz = 0, mxyz = 0;
  for (uint32_t p = b; p < e; ++p) {
    double px, py, pz;
    rec_pos(P, p, px, py, pz);
    const double fx = fma(px, g.inv_h, -cx);
    const double fy = fma(py, g.inv_h, -cy);
    const double fz = fma(pz, g.inv_h, -cz);
    const double fxy = fx * fy;
    mx += fx;
    my += fy;
    mz += fz;
    mxy += fxy;
    mxz = fma(fx, fz, mxz);
    myz = fma(fy, fz, myz);
    mxyz = fma(fxy, fz, mxyz);
  }
  const double cnt = (double)(e - b);
  double s[8];
  s[7] = mxyz;                                  // f_x f_y f_z
  s[3] = mxy - mxyz;                            // f_x f_y (1 - f_z)
  s[5] = mxz - mxyz;                            // f_x (1 - f_y) f_z
  s[6] = myz - mxyz;                            // (1 - f_x) f_y f_z
  s[1] = mx - mxy - mxz + mxyz;                 // f_x (1 - f_y)(1 - f_z)
  s[2] = my - mxy - myz + mxyz;                 // (1 - f_x) f_y (1 - f_z)
  s[4] = mz - mxz - myz + mxyz;                 // (1 - f_x)(1 - f_y) f_z
  s[0] = cnt - mx - my - mz + mxy + mxz + myz - mxyz;  // (1 - f_x)(1 - f_y)(1 - f_z)
  const int jx = ix + 1 == N ? 0 : ix + 1, jy = iy + 1 == N ? 0 : iy + 1, jz = iz + 1 == N ? 0 : iz + 1;
  const size_t Ns = N;
  const size_t z0 = (size_t)iz * Ns * Ns, z1 = (size_t)jz * Ns * Ns, y0 = (size_t)iy * Ns, y1 = (size_t)jy * Ns;
  atomicAdd(rho + z0 + y0 + ix, qscale * s[0]);
  atomicAdd(rho + z0 + y0 + jx, qscale * s[1]);
  atomicAdd(rho + z0 + y1 + ix, qscale * s[2]);
  atomicAdd(rho + z0 + y1 + jx, qscale * s[3]);
  atomicAdd(rho + z1 + y0 + ix, qscale * s[4]);
  atomicAdd(rho + z1 + y0 + jx, qscale * s[5]);
  atomicAdd(rho + z1 + y1 + ix, qscale * s[6]);
  atomicAdd(rho + z1 + y1 + jx, qscale * s[7]);
}

// ---------------------------------------------------------------------------
// S5: E = -grad phi, central differences, periodic. Ex = (phi[i-1] - phi[i+1]) / 2h.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gradient(const double* __restrict__ phi, double* __restrict__ Ex,
                                                  double* __restrict__ Ey, double* __restrict__ Ez, Grid g) {
  const int N = g.N;
  const size_t Ns = N, n = Ns * Ns * Ns;
  const double s = 0.5 * g.inv_h;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
    const int ix = (int)(c % Ns), iy = (int)((c / Ns) % Ns), iz = (int)(c / (Ns * Ns));
    const size_t row = c - ix, pl = c - (size_t)iy * Ns;
    const double xm = __ldg(phi + row + (ix == 0 ? N - 1 : ix - 1));
    const double xp = __ldg(phi + row + (ix == N - 1 ? 0 : ix + 1));
    const double ym = __ldg(phi + pl + (size_t)(iy == 0 ? N - 1 : iy - 1) * Ns);
    const double yp = __ldg(phi + pl + (size_t)(iy == N - 1 ? 0 : iy + 1) * Ns);
    const size_t col = c - (size_t)iz * Ns * Ns;
    const double zm = __ldg(phi + col + (size_t)(iz == 0 ? N - 1 : iz - 1) * Ns * Ns);
    const double zp = __ldg(phi + col + (size_t)(iz == N - 1 ? 0 : iz + 1) * Ns * Ns);
    Ex[c] = (xm - xp) * s;
    Ey[c] = (ym - yp) * s;
    Ez[c] = (zm - zp) * s;
  }
}

// S7: W_d = h^3 sum E_d^2 with E from central differences of phi.
__global__ void __launch_bounds__(256) k_field_energy(const double* __restrict__ phi, Grid g, double* out3,
                                                      double* partials, unsigned* counter) {
  const int N = g.N;
  const size_t Ns = N, n = Ns * Ns * Ns;
  double a[3] = {0.0, 0.0, 0.0};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
    const int ix = (int)(c % Ns), iy = (int)((c / Ns) % Ns), iz = (int)(c / (Ns * Ns));
    const size_t row = c - ix, pl = c - (size_t)iy * Ns, col = c - (size_t)iz * Ns * Ns;
    const double dx = __ldg(phi + row + (ix == 0 ? N - 1 : ix - 1)) - __ldg(phi + row + (ix == N - 1 ? 0 : ix + 1));
    const double dy = __ldg(phi + pl + (size_t)(iy == 0 ? N - 1 : iy - 1) * Ns) -
                      __ldg(phi + pl + (size_t)(iy == N - 1 ? 0 : iy + 1) * Ns);
    const double dz = __ldg(phi + col + (size_t)(iz == 0 ? N - 1 : iz - 1) * Ns * Ns) -
                      __ldg(phi + col + (size_t)(iz == N - 1 ? 0 : iz + 1) * Ns * Ns);
    a[0] = fma(dx, dx, a[0]);
    a[1] = fma(dy, dy, a[1]);
    a[2] = fma(dz, dz, a[2]);
  }
  double tot[3];
  if (grid_reduce_last<3>(a, partials, counter, tot) && threadIdx.x == 0) {
    // E = d / (2h): W = h^3 sum d^2 / (4 h^2) = h sum d^2 / 4
    const double f = 0.25 * g.h;
    out3[0] = f * tot[0];
    out3[1] = f * tot[1];
    out3[2] = f * tot[2];
  }
}

// ---------------------------------------------------------------------------
// S6: CIC gather of E and leapfrog push; then the new cell key and in-cell
// rank (counts must be zero on entry) for the next sort. drift == 0 gives the
// closing half-kick only (no key update).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gather_push(PRec* P, uint64_t np, const double* __restrict__ Ex,
                                                     const double* __restrict__ Ey, const double* __restrict__ Ez,
                                                     Grid g, double kick_qm, double dt, int drift, uint32_t* keys,
                                                     uint32_t* ranks, uint32_t* counts) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double2* rec = reinterpret_cast<double2*>(P + p);
  const double2 r0 = rec[0], r1 = rec[1], r2 = rec[2];
  const uint4 r3 = reinterpret_cast<const uint4*>(rec)[3];
  double x = r0.x, y = r0.y, z = r1.x;
  const int N = g.N;
  // the cell of the current position, kept in the record since its key was
  // computed (integer decode instead of three FP64 floors)
  const uint32_t key = r3.y;
  const int ix = (int)(key % (uint32_t)N), iy = (int)((key / (uint32_t)N) % (uint32_t)N),
            iz = (int)(key / ((uint32_t)N * (uint32_t)N));
  const double fx = fma(x, g.inv_h, -(double)ix), fy = fma(y, g.inv_h, -(double)iy),
               fz = fma(z, g.inv_h, -(double)iz);
  const double gx = 1.0 - fx, gy = 1.0 - fy, gz = 1.0 - fz;
  const double w00 = gy * gz, w10 = fy * gz, w01 = gy * fz, w11 = fy * fz;
  const double w[8] = {gx * w00, fx * w00, gx * w10, fx * w10, gx * w01, fx * w01, gx * w11, fx * w11};
  const int jx = ix + 1 == N ? 0 : ix + 1, jy = iy + 1 == N ? 0 : iy + 1, jz = iz + 1 == N ? 0 : iz + 1;
  const size_t Ns = N;
  const size_t z0 = (size_t)iz * Ns * Ns, z1 = (size_t)jz * Ns * Ns, y0 = (size_t)iy * Ns, y1 = (size_t)jy * Ns;
  const size_t idx[8] = {z0 + y0 + ix, z0 + y0 + jx, z0 + y1 + ix, z0 + y1 + jx,
                         z1 + y0 + ix, z1 + y0 + jx, z1 + y1 + ix, z1 + y1 + jx};
  double ex = 0.0, ey = 0.0, ez = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    ex = fma(w[c], __ldg(Ex + idx[c]), ex);
    ey = fma(w[c], __ldg(Ey + idx[c]), ey);
    ez = fma(w[c], __ldg(Ez + idx[c]), ez);
  }
  double vx = fma(kick_qm, ex, r1.y);
  double vy = fma(kick_qm, ey, r2.x);
  double vz = fma(kick_qm, ez, r2.y);
  rec[2] = make_double2(vy, vz);
  if (!drift) {
    rec[1] = make_double2(z, vx);
    return;
  }
  const double L = g.L;
  x = fma(dt, vx, x);
  y = fma(dt, vy, y);
  z = fma(dt, vz, z);
  // periodic wrap into [0, L); a value that rounds to L becomes 0. Only the
  // few particles that left the box take the full sequence; for the others
  // it is the identity (same result, fewer FP64 operations).
  if (x < 0.0 || x >= L) {
    x = x >= L ? x - L : x; x = x < 0.0 ? x + L : x; x = x >= L ? 0.0 : x;
  }
  if (y < 0.0 || y >= L) {
    y = y >= L ? y - L : y; y = y < 0.0 ? y + L : y; y = y >= L ? 0.0 : y;
  }
  if (z < 0.0 || z >= L) {
    z = z >= L ? z - L : z; z = z < 0.0 ? z + L : z; z = z >= L ? 0.0 : z;
  }
  rec[0] = make_double2(x, y);
  rec[1] = make_double2(z, vx);
  const uint32_t kk = key_of(x, y, z, g);
  reinterpret_cast<uint4*>(rec)[3] = make_uint4(r3.x, kk, 0u, 0u);
  keys[p] = kk;
  ranks[p] = atomicAdd(&counts[kk], 1u);
}

// Copy particles back to the original order: out[q * np + id[p]] = field q of p.
__global__ void k_unsort(const PRec* P, uint64_t np, double* out) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const PRec r = P[p];
  const uint64_t d = r.id;
  out[d] = r.x;
  out[np + d] = r.y;
  out[2 * np + d] = r.z;
  out[3 * np + d] = r.vx;
  out[4 * np + d] = r.vy;
  out[5 * np + d] = r.vz;
}

}  // namespace pic
