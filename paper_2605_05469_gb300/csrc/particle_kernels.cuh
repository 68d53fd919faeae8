// Particle kernels of the PIC loop (Fig. 1): initial sampling (Sec. 2.1),
// sort by cell, CIC scatter (Eq. 2), E = -grad phi, CIC gather and leapfrog
// push (Eqs. 3-4), field energy (Fig. 2).
//
// Particles are 64-byte records (PRec): the position as the cell and a 64-bit
// fixed-point offset inside it, the velocity as double-float pairs. All
// per-particle arithmetic runs in double-float on the FP32 pipes (GB300's
// FP64 rate is 1/58 of its FP32 rate); the grid-side quantities keep FP64
// (phi, rho) and the conversions happen once per node. Each step the particles
// are counting-sorted by cell: the push computes every particle's new cell and
// its rank inside the cell (one integer atomic per group of equal cells in a
// warp); a scan turns the cell counts into offsets and a scatter moves the
// records. The deposit then runs one thread per cell over the cell's
// contiguous particles and writes the cell's 8 corner charges, and one thread
// per node adds the 8 charges that reach it (no atomics).
#pragma once
#include "common.cuh"
#include "dfloat.cuh"

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

__device__ __forceinline__ uint32_t cell_key(int ix, int iy, int iz, int N) {
  return (uint32_t)ix + (uint32_t)N * ((uint32_t)iy + (uint32_t)N * (uint32_t)iz);
}

// A position coordinate x in [0, L] as its cell and 64-bit offset (FP64 in,
// for the initial condition and loads only). A value that rounds to the top of
// the box wraps to 0.
__device__ __forceinline__ void to_cell_offset(double x, const Grid& g, int& i, uint64_t& f) {
  const double u = x * g.inv_h;
  i = cell_of(x, g);
  double r = u - (double)i;
  if (!(r < 1.0)) {  // x == L after rounding (or the clamp at N - 1)
    i = 0;
    r = 0.0;
  }
  if (r < 0.0) r = 0.0;
  f = __double2ull_rn(r * 18446744073709551616.0);  // r 2^64 < 2^64
}

// The coordinate (i + f 2^-64) h in FP64 (outputs only).
__device__ __forceinline__ double from_cell_offset(int i, uint64_t f, const Grid& g) {
  return ((double)i + (double)(f >> 11) * (1.0 / 9007199254740992.0)) * g.h;
}

// The offset f 2^-64 in [0, 1) as a double-float: its top 24 bits and the next
// 24 (each exactly an FP32 value), normalised; the 16 lowest bits are dropped
// (2^-48 of a cell).
__device__ __forceinline__ df frac_df(uint64_t f) {
  const float hi = __uint2float_rn((uint32_t)(f >> 40)) * 0x1p-24f;
  const float lo = __uint2float_rn((uint32_t)(f >> 16) & 0xFFFFFFu) * 0x1p-48f;
  return fast_two_sum(hi, lo);  // hi == 0 or hi >= 2^-24 > lo
}

// 1 - f 2^-64 as a double-float (2^64 - f in the same fixed point; f == 0 is 1).
__device__ __forceinline__ df one_minus_frac_df(uint64_t f) {
  if (f == 0) return {1.0f, 0.0f};
  return frac_df(0ull - f);
}

// |x| 2^64 truncated to an integer, for |x| < 1, with two 32-bit
// conversions (a 64-bit float-to-integer conversion would run on GB300's
// FP64 pipe): a = |x| 2^32 < 2^32 splits exactly into its integer part and
// its fraction, and the fraction times 2^32 is the low word.
__device__ __forceinline__ uint64_t abs_times_2p64(float x) {
  const float a = __fmul_rn(fabsf(x), 0x1p32f);
  const float h = truncf(a);
  const float l = __fmul_rn(__fsub_rn(a, h), 0x1p32f);
  return ((uint64_t)__float2uint_rz(h) << 32) | __float2uint_rz(l);
}

// Moves one coordinate by d cells (double-float): the offset takes the
// fraction of d in exact 64-bit arithmetic, the carries and the integer part
// of d move the cell index, which wraps periodically. Needs |d| < 2^20.
// The leading word splits as n + r with n = trunc(d.hi): r = d.hi - n is then
// exact (its bits are a subset of d.hi's), which d.hi - floor(d.hi) is not
// for negative d.hi (-0.3 + 1 needs one more bit than 0.7 has).
__device__ __forceinline__ void move_coord(uint64_t& f, int& i, df d, int N) {
  const float n = fminf(fmaxf(truncf(d.hi), -1048576.0f), 1048576.0f);  // keeps the index arithmetic in range
  const float r = __fsub_rn(d.hi, n);  // exact, |r| < 1, sign of d.hi
  const uint64_t A = abs_times_2p64(r), B = abs_times_2p64(d.lo);
  const bool ra = r >= 0.0f, ba = d.lo >= 0.0f;
  const uint64_t f1 = ra ? f + A : f - A;
  int carry = ra ? (f1 < f ? 1 : 0) : (f1 > f ? -1 : 0);
  const uint64_t f2 = ba ? f1 + B : f1 - B;
  carry += ba ? (f2 < f1 ? 1 : 0) : (f2 > f1 ? -1 : 0);
  f = f2;
  int t = i + (int)n + carry;
  if (t < 0 || t >= N) {
    t %= N;
    if (t < 0) t += N;
  }
  i = t;
}

// A double-float constant passed from the host as (hi, lo).
__device__ __forceinline__ df dfc(float2 v) { return {v.x, v.y}; }

// S0: sample particle p of the Landau initial condition (FP64), store it as a
// record, and count its cell.
// Trials of the rejection sampling of the sum-form density (mode 1).
constexpr int kSumFormTrials = 32;

// mode 0: the paper's product density prod_d (1 + alpha cos k x_d), exact
// per-dimension inverse CDF (Philox calls 0 and 1). mode 1: the sum density
// 1 + alpha sum_d cos k x_d by rejection from the uniform density: trial t
// takes calls 4 + 2t (u_x, u_y) and 5 + 2t (u_z, u_accept) and accepts x = u L
// when u_accept (1 + 3 alpha) <= 1 + alpha sum_d cos k x_d; the first accepted
// trial is kept, the last proposal if none is (probability below
// (3 alpha / (1 + 3 alpha))^32). Velocities: vth times Box-Muller normals
// (calls 2 and 3).
__global__ void k_init_particles(PRec* P, uint64_t np, uint64_t seed, double alpha, double k, double vth, int mode,
                                 Grid g, uint32_t* counts) {
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
  double x, y, z;
  if (mode == 1) {
    const double top = 1.0 + 3.0 * alpha;
    for (int t = 0; t < kSumFormTrials; ++t) {
      const uint4 a = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), (uint32_t)(4 + 2 * t), 0u), key);
      const uint4 b = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), (uint32_t)(5 + 2 * t), 0u), key);
      x = u53(a.x, a.y) * g.L;
      y = u53(a.z, a.w) * g.L;
      z = u53(b.x, b.y) * g.L;
      const double dens = 1.0 + alpha * (cos(k * x) + cos(k * y) + cos(k * z));
      if (u53(b.z, b.w) * top <= dens) break;
    }
  } else {
    x = inverse_cdf(u[0], g.L, alpha, k);
    y = inverse_cdf(u[1], g.L, alpha, k);
    z = inverse_cdf(u[2], g.L, alpha, k);
  }
  const double two_pi = 6.283185307179586476925286766559;
  // Box-Muller (Box & Muller 1958)
  const double r1 = vth * sqrt(-2.0 * log(u[4])), r2 = vth * sqrt(-2.0 * log(u[6]));
  double s1, c1, s2, c2;
  sincos(two_pi * u[5], &s1, &c1);
  sincos(two_pi * u[7], &s2, &c2);
  PRec rec;
  int ix, iy, iz;
  to_cell_offset(x, g, ix, rec.fx);
  to_cell_offset(y, g, iy, rec.fy);
  to_cell_offset(z, g, iz, rec.fz);
  rec.vx = df_pack(df_of_double(r1 * c1));
  rec.vy = df_pack(df_of_double(r1 * s1));
  rec.vz = df_pack(df_of_double(r2 * c2));
  rec.id = (uint32_t)p;
  rec.key = cell_key(ix, iy, iz, g.N);
  rec.cell = pack_cell(ix, iy, iz);
  rec.rank = atomicAdd(&counts[rec.key], 1u);
  P[p] = rec;
}

// Cell keys and in-cell ranks of the current particles.
__global__ void k_count_keys(PRec* P, uint64_t np, Grid g, uint32_t* counts) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const uint32_t c = P[p].cell;
  const uint32_t kk = cell_key(cell_x(c), cell_y(c), cell_z(c), g.N);
  P[p].key = kk;
  P[p].rank = atomicAdd(&counts[kk], 1u);
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

// Move particle p to offsets[key] + rank (the other buffer), key and rank
// read from the record itself. Each warp moves 32 consecutive particles; lane
// l first reads the last 16-byte word (id, key, cell, rank) of particle l and
// starts its destination lookup, then holds 16-byte word (l & 3) of particles
// 8k + (l >> 2), k = 0..3, so every load and every store instruction of the
// warp covers 8 whole 64-byte records (whole sectors at both ends; the early
// word read touches sectors the record loads read again from L1).
__global__ void __launch_bounds__(256) k_scatter(const PRec* __restrict__ src, PRec* __restrict__ dst, uint64_t np,
                                                 const uint32_t* __restrict__ offsets) {
  const uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
  if (base >= np) return;  // uniform over the warp
  const int lane = threadIdx.x & 31;
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  const uint64_t p = base + lane;
  uint64_t d = 0;
  if (p < np) {
    const uint4 w3 = __ldg(s4 + p * 4 + 3);
    d = (uint64_t)__ldg(offsets + w3.y) + w3.w;
  }
  const int word = lane & 3;
  uint4 v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint64_t q = base + 8 * k + (lane >> 2);
    if (q < np) v[k] = __ldg(s4 + q * 4 + word);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int ql = 8 * k + (lane >> 2);
    const uint64_t dq = __shfl_sync(0xffffffffu, d, ql);
    if (base + ql < np) d4[dq * 4 + word] = v[k];
  }
}

// ---------------------------------------------------------------------------
// S2: CIC scatter from cell-sorted particles (Eq. 2), in two passes.
// Cells: one thread per cell sums, over the cell's particles, the corner
// weights prod_d (f_d or 1 - f_d) of its 8 corners from the moments of the
// offsets f in [0, 1)^3 (count, f_x, f_y, f_z, f_x f_y, f_x f_z, f_y f_z,
// f_x f_y f_z), in double-float, and writes them to dep[corner][cell].
// Nodes: one thread per node adds the 8 corner sums that reach it and writes
// rho = 1 + (q_p / h^3) sum (the +1 background) in FP64.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_deposit_cells(const PRec* __restrict__ P,
                                                       const uint32_t* __restrict__ offsets, float2* __restrict__ dep,
                                                       size_t n) {
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const uint32_t b = offsets[c], e = offsets[c + 1];
  DfAcc mx, my, mz, mxy, mxz, myz, mxyz;
  for (uint32_t p = b; p < e; ++p) {
    const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2*>(P + p));
    const unsigned long long fz = __ldg(reinterpret_cast<const unsigned long long*>(P + p) + 2);
    const df fx = frac_df(a.x), fy = frac_df(a.y), fzd = frac_df(fz);
    const df fxy = df_mul(fx, fy);
    mx.add(fx);
    my.add(fy);
    mz.add(fzd);
    mxy.add(fxy);
    mxz.add_mul(fx, fzd);
    myz.add_mul(fy, fzd);
    mxyz.add_mul(fxy, fzd);
  }
  const df Mx = mx.value(), My = my.value(), Mz = mz.value(), Mxy = mxy.value(), Mxz = mxz.value(),
           Myz = myz.value(), Mxyz = mxyz.value();
  const df cnt = {(float)(e - b), 0.0f};  // exact below 2^24 particles per cell
  df s[8];
  s[7] = Mxyz;                                            // f_x f_y f_z
  s[3] = df_sub(Mxy, Mxyz);                               // f_x f_y (1 - f_z)
  s[5] = df_sub(Mxz, Mxyz);                               // f_x (1 - f_y) f_z
  s[6] = df_sub(Myz, Mxyz);                               // (1 - f_x) f_y f_z
  s[1] = df_sub(Mx, df_add(df_add(Mxy, Mxz), df_neg(Mxyz)));  // f_x (1 - f_y)(1 - f_z)
  s[2] = df_sub(My, df_add(df_add(Mxy, Myz), df_neg(Mxyz)));  // (1 - f_x) f_y (1 - f_z)
  s[4] = df_sub(Mz, df_add(df_add(Mxz, Myz), df_neg(Mxyz)));  // (1 - f_x)(1 - f_y) f_z
  // (1 - f_x)(1 - f_y)(1 - f_z) = cnt - mx - my - mz + mxy + mxz + myz - mxyz
  s[0] = df_add(df_sub(cnt, df_add(df_add(Mx, My), Mz)), df_sub(df_add(df_add(Mxy, Mxz), Myz), Mxyz));
#pragma unroll
  for (int k = 0; k < 8; ++k) dep[(size_t)k * n + c] = df_pack(s[k]);
}

// Node (i, j, k) is corner (a, b, c) of cell (i - a, j - b, k - c).
__global__ void __launch_bounds__(256) k_deposit_nodes(const float2* __restrict__ dep, double* __restrict__ rho,
                                                       int N, double qscale) {
  const size_t Ns = N, n = Ns * Ns * Ns;
  const int k = blockIdx.y;
  const unsigned per_plane = (unsigned)N * (unsigned)N;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < per_plane; t += gridDim.x * blockDim.x) {
    const int j = (int)(t / (unsigned)N), i = (int)(t - (unsigned)j * (unsigned)N);
    const int im = i == 0 ? N - 1 : i - 1, jm = j == 0 ? N - 1 : j - 1, km = k == 0 ? N - 1 : k - 1;
    const int xs[2] = {i, im}, ys[2] = {j, jm}, zs[2] = {k, km};
    DfAcc acc;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int a = q & 1, b = (q >> 1) & 1, c = q >> 2;
      const size_t cell = ((size_t)zs[c] * Ns + ys[b]) * Ns + xs[a];
      acc.add(df_from(__ldg(dep + (size_t)q * n + cell)));
    }
    rho[(size_t)k * per_plane + t] = fma(qscale, double_of_df(acc.value()), 1.0);
  }
}

// ---------------------------------------------------------------------------
// S5: E = -grad phi, central differences, periodic (Eq. 2):
// Ex = (phi[i-1] - phi[i+1]) / 2h. phi is converted to double-float once per
// node (FP64 operations), the differences run in double-float.
// ---------------------------------------------------------------------------
// (also converts a given 3 n node field)
// A given FP64 node field (E_x, E_y, E_z blocks of n) into the push's layout.
__global__ void __launch_bounds__(256) k_field_df(const double* __restrict__ E, float4* __restrict__ Exy,
                                                  float2* __restrict__ Ez, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
    const df ex = df_of_double(__ldg(E + c)), ey = df_of_double(__ldg(E + n + c));
    Exy[c] = make_float4(ex.hi, ey.hi, ex.lo, ey.lo);
    Ez[c] = df_pack(df_of_double(__ldg(E + 2 * n + c)));
  }
}

__global__ void __launch_bounds__(256) k_phi_df(const double* __restrict__ phi, float2* __restrict__ out, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride)
    out[c] = df_pack(df_of_double(__ldg(phi + c)));
}

// E = -grad phi by central differences (Eq. 2) in double-float, into the
// push's node field: E_x, E_y interleaved {x.hi, y.hi, x.lo, y.lo}, E_z alone.
__global__ void __launch_bounds__(256) k_gradient(const float2* __restrict__ phi, float4* __restrict__ Exy,
                                                  float2* __restrict__ Ez, int N, float2 half_inv_h) {
  const size_t Ns = N;
  const int k = blockIdx.y;
  const unsigned per_plane = (unsigned)N * (unsigned)N;
  const df s = dfc(half_inv_h);
  const int km = k == 0 ? N - 1 : k - 1, kp = k == N - 1 ? 0 : k + 1;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < per_plane; t += gridDim.x * blockDim.x) {
    const int j = (int)(t / (unsigned)N), i = (int)(t - (unsigned)j * (unsigned)N);
    const int im = i == 0 ? N - 1 : i - 1, ip = i == N - 1 ? 0 : i + 1;
    const int jm = j == 0 ? N - 1 : j - 1, jp = j == N - 1 ? 0 : j + 1;
    const size_t pl = (size_t)k * per_plane, row = pl + (size_t)j * Ns;
    const df xm = df_from(__ldg(phi + row + im)), xp = df_from(__ldg(phi + row + ip));
    const df ym = df_from(__ldg(phi + pl + (size_t)jm * Ns + i)), yp = df_from(__ldg(phi + pl + (size_t)jp * Ns + i));
    const df zm = df_from(__ldg(phi + (size_t)km * per_plane + (size_t)j * Ns + i));
    const df zp = df_from(__ldg(phi + (size_t)kp * per_plane + (size_t)j * Ns + i));
    const size_t c = row + i;
    const df ex = df_mul(df_sub(xm, xp), s), ey = df_mul(df_sub(ym, yp), s);
    Exy[c] = make_float4(ex.hi, ey.hi, ex.lo, ey.lo);
    Ez[c] = df_pack(df_mul(df_sub(zm, zp), s));
  }
}

// S7 for a given node field (the spectral solve's): W_d = h^3 sum E_d^2.
__global__ void __launch_bounds__(256) k_field_energy_E(const double* __restrict__ E, size_t n, double h3,
                                                        double* out3, double* partials, unsigned* counter) {
  double a[3] = {0.0, 0.0, 0.0};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double v = __ldg(E + (size_t)d * n + c);
      a[d] = fma(v, v, a[d]);
    }
  }
  double tot[3];
  if (grid_reduce_last<3>(a, partials, counter, tot) && threadIdx.x == 0) {
    out3[0] = h3 * tot[0];
    out3[1] = h3 * tot[1];
    out3[2] = h3 * tot[2];
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
// S6: CIC gather of E and leapfrog push (Eqs. 3-4), in double-float; then the
// new cell key and in-cell rank for the next sort, written into the record's
// last word (counts must be zero on entry). drift == 0 gives the closing
// half-kick only (no key update).
//   kick_qm = -kick (q/m = -1), dth = dt / h, both double-float (hi, lo).
// The node field is E_x and E_y interleaved as one float4 a node
// {x.hi, y.hi, x.lo, y.lo} and E_z as a float2: the x and y components run
// as pairs on the packed FP32 instructions (df2), z alone, with the same
// per-lane rounding as three scalar computations. Each thread reads and
// writes its own 64-byte record (four 16-byte words). The ranks come from one
// atomic per run of equal keys in a warp (the particles are in cell order, so
// a warp covers a few cells). Four blocks an SM (64 registers, no spills).
// ---------------------------------------------------------------------------
constexpr int kPushThreads = 256;

// GIVEN: the field at the particles is given (Ep: 3 np FP64, E_x, E_y, E_z in
// the current particle order; the particle-in-Fourier scheme) instead of
// gathered from the node field.
template <bool GIVEN>
__global__ void __launch_bounds__(kPushThreads, 4) k_gather_push(PRec* P, uint64_t np, const float4* __restrict__ Exy,
                                                              const float2* __restrict__ Ez, Grid g, float2 kick_qm,
                                                              float2 dth, int drift,
                                                              uint32_t* counts, const double* __restrict__ Ep,
                                                              int* err) {
  const uint64_t base = (uint64_t)blockIdx.x * kPushThreads;
  const uint64_t p = base + threadIdx.x;
  const bool valid = p < np;
  uint32_t kk = 0xFFFFFFFFu;
  uint32_t rid = 0, rcell = 0;  // the record's id and (new) packed cell
  if (valid) {
    uint4* rec = reinterpret_cast<uint4*>(P + p);
    const uint4 r0 = rec[0], r1 = rec[1], r3 = rec[3];
    const float4 r2 = *reinterpret_cast<const float4*>(rec + 2);
    uint64_t fx = ((uint64_t)r0.y << 32) | r0.x, fy = ((uint64_t)r0.w << 32) | r0.z;
    uint64_t fz = ((uint64_t)r1.y << 32) | r1.x;
    df2 vxy = {make_float2(__uint_as_float(r1.z), r2.x), make_float2(__uint_as_float(r1.w), r2.y)};
    df vz = {r2.z, r2.w};
    int ix = cell_x(r3.z), iy = cell_y(r3.z), iz = cell_z(r3.z);
    rid = r3.x;
    const int N = g.N;
    df2 exy;
    df ez;
    if (GIVEN) {
      exy = df2_pair(df_of_double(__ldg(Ep + p)), df_of_double(__ldg(Ep + np + p)));
      ez = df_of_double(__ldg(Ep + 2 * np + p));
    } else {
      // CIC weights prod_d (f_d or 1 - f_d) of the 8 corners, in pairs
      const df ax = frac_df(fx), ay = frac_df(fy), az = frac_df(fz);
      const df bx = one_minus_frac_df(fx), by = one_minus_frac_df(fy), bz = one_minus_frac_df(fz);
      const df2 yb = df2_pair(by, ay), xb = df2_pair(bx, ax);
      const df2 wz0 = df2_mul(yb, df2_bcast(bz)), wz1 = df2_mul(yb, df2_bcast(az));  // (w00, w10), (w01, w11)
      const df2 w2[4] = {df2_mul(xb, df2_bcast(df2_x(wz0))), df2_mul(xb, df2_bcast(df2_y(wz0))),
                         df2_mul(xb, df2_bcast(df2_x(wz1))), df2_mul(xb, df2_bcast(df2_y(wz1)))};
      const int jx = ix + 1 == N ? 0 : ix + 1, jy = iy + 1 == N ? 0 : iy + 1, jz = iz + 1 == N ? 0 : iz + 1;
      const size_t Ns = N;
      const size_t z0 = (size_t)iz * Ns * Ns, z1 = (size_t)jz * Ns * Ns, y0 = (size_t)iy * Ns, y1 = (size_t)jy * Ns;
      const size_t idx[8] = {z0 + y0 + ix, z0 + y0 + jx, z0 + y1 + ix, z0 + y1 + jx,
                             z1 + y0 + ix, z1 + y0 + jx, z1 + y1 + ix, z1 + y1 + jx};
      DfAcc2 axy;
      DfAcc az_;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const df w = (c & 1) ? df2_y(w2[c >> 1]) : df2_x(w2[c >> 1]);
        const float4 e = __ldg(Exy + idx[c]);
        axy.add_mul(df2_bcast(w), {make_float2(e.x, e.y), make_float2(e.z, e.w)});
        az_.add_mul(w, df_from(__ldg(Ez + idx[c])));
      }
      exy = axy.value();
      ez = az_.value();
    }
    const df kq = dfc(kick_qm);
    const df2 uxy = df2_add(vxy, df2_mul(df2_bcast(kq), exy));
    const df uz = df_add(vz, df_mul(kq, ez));
    // a non-finite field at the particle: record the fault and leave the
    // particle as it is (its key and rank are still written below)
    const bool fin = isfinite(uxy.hi.x) && isfinite(uxy.hi.y) && isfinite(uz.hi) && isfinite(uxy.lo.x) &&
                     isfinite(uxy.lo.y) && isfinite(uz.lo);
    if (fin) {
      vxy = uxy;
      vz = uz;
    } else {
      atomicOr(err, DEV_ERR_NONFINITE);
    }
    *reinterpret_cast<float4*>(rec + 2) = make_float4(vxy.hi.y, vxy.lo.y, vz.hi, vz.lo);
    if (drift && fin) {
      const df s = dfc(dth);
      const df2 dxy = df2_mul(vxy, df2_bcast(s));
      move_coord(fx, ix, df2_x(dxy), N);
      move_coord(fy, iy, df2_y(dxy), N);
      move_coord(fz, iz, df_mul(vz, s), N);
      rec[0] = make_uint4((uint32_t)fx, (uint32_t)(fx >> 32), (uint32_t)fy, (uint32_t)(fy >> 32));
    }
    if (drift) {
      kk = cell_key(ix, iy, iz, N);
      rcell = pack_cell(ix, iy, iz);
    }
    rec[1] = make_uint4((uint32_t)fz, (uint32_t)(fz >> 32), __float_as_uint(vxy.hi.x), __float_as_uint(vxy.lo.x));
  }
  if (!drift) return;  // uniform over the launch: every lane reaches the warp collectives below
  // runs of equal keys: the first lane of a run takes the run's ranks with one atomic
  const int lane = threadIdx.x & 31;
  const uint32_t prev = __shfl_up_sync(0xffffffffu, kk, 1);
  const bool start = lane == 0 || prev != kk;
  const unsigned starts = __ballot_sync(0xffffffffu, start);
  const unsigned upto = 0xffffffffu >> (31 - lane);  // lanes 0..lane
  const int run0 = 31 - __clz(starts & upto);
  const unsigned after = starts & ~upto;
  const int run1 = after ? __ffs(after) - 1 : 32;
  uint32_t b = 0;
  if (start && valid) b = atomicAdd(&counts[kk], (uint32_t)(run1 - run0));
  b = __shfl_sync(0xffffffffu, b, run0);
  // the record's last word: id, the new key and cell, and the rank
  if (valid) reinterpret_cast<uint4*>(P + p)[3] = make_uint4(rid, kk, rcell, b + (uint32_t)(lane - run0));
}

// A per-particle field (3 np, current order) back to the original order.
__global__ void k_unsort_field(const PRec* P, uint64_t np, const double* Ep, double* out) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const uint64_t d = P[p].id;
#pragma unroll
  for (int q = 0; q < 3; ++q) out[q * np + d] = Ep[q * np + p];
}

// Copy particles back to the original order, in FP64: out[q * np + id[p]] =
// field q of p (x, y, z, vx, vy, vz).
__global__ void k_unsort(const PRec* P, uint64_t np, Grid g, double* out) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const PRec r = P[p];
  const uint64_t d = r.id;
  out[d] = from_cell_offset(cell_x(r.cell), r.fx, g);
  out[np + d] = from_cell_offset(cell_y(r.cell), r.fy, g);
  out[2 * np + d] = from_cell_offset(cell_z(r.cell), r.fz, g);
  out[3 * np + d] = double_of_df(df_from(r.vx));
  out[4 * np + d] = double_of_df(df_from(r.vy));
  out[5 * np + d] = double_of_df(df_from(r.vz));
}

// Particles from caller data (FP64 structure of arrays, blocks of `ld`
// values: x, y, z, vx, vy, vz): particle base + i takes element i of each
// block, for i < count. Positions are wrapped into [0, L); a non-finite value
// sets DEV_ERR_NONFINITE in *flag and the particle is stored at the origin at
// rest.
__global__ void k_set_particles(const double* __restrict__ in, uint64_t ld, uint64_t count, uint64_t base, PRec* P,
                                Grid g, int* flag, uint32_t* counts) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double v[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) v[q] = in[q * ld + i];
  bool ok = true;
#pragma unroll
  for (int q = 0; q < 6; ++q) ok = ok && isfinite(v[q]);
  if (!ok) {
    atomicOr(flag, DEV_ERR_NONFINITE);
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = 0.0;
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    double x = v[q];
    if (!(x >= 0.0 && x < g.L)) {  // outside the box (rare): its periodic image
      x = fmod(x, g.L);            // exact; |x| < L
      if (x < 0.0) x += g.L;       // may round to L, which to_cell_offset wraps to 0
    }
    v[q] = x;
  }
  PRec rec;
  int ix, iy, iz;
  to_cell_offset(v[0], g, ix, rec.fx);
  to_cell_offset(v[1], g, iy, rec.fy);
  to_cell_offset(v[2], g, iz, rec.fz);
  rec.vx = df_pack(df_of_double(v[3]));
  rec.vy = df_pack(df_of_double(v[4]));
  rec.vz = df_pack(df_of_double(v[5]));
  rec.id = (uint32_t)(base + i);
  rec.key = cell_key(ix, iy, iz, g.N);
  rec.cell = pack_cell(ix, iy, iz);
  // the next sort's in-cell rank (counts zeroed by the caller)
  rec.rank = atomicAdd(&counts[rec.key], 1u);
  P[base + i] = rec;
}


// inv[id] = p: the current (cell-sorted) position of every particle, by the
// index it was sampled with (reads only the records' id words).
__global__ void __launch_bounds__(256) k_inverse_ids(const PRec* __restrict__ P, uint64_t np,
                                                     uint32_t* __restrict__ inv) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  inv[P[p].id] = (uint32_t)p;
}

// Particles base .. base + count - 1 of the original order to FP64 structure
// of arrays (blocks of `ld` values: x, y, z, vx, vy, vz): from an array in the
// original order, or (inv given) gathered from the sorted records through
// the inverse permutation.
__global__ void k_records_to_soa(const PRec* __restrict__ P, uint64_t base, uint64_t count, Grid g, double* out,
                                 uint64_t ld, const uint32_t* __restrict__ inv) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const PRec r = P[inv ? (uint64_t)inv[base + i] : base + i];
  out[i] = from_cell_offset(cell_x(r.cell), r.fx, g);
  out[ld + i] = from_cell_offset(cell_y(r.cell), r.fy, g);
  out[2 * ld + i] = from_cell_offset(cell_z(r.cell), r.fz, g);
  out[3 * ld + i] = double_of_df(df_from(r.vx));
  out[4 * ld + i] = double_of_df(df_from(r.vy));
  out[5 * ld + i] = double_of_df(df_from(r.vz));
}

}  // namespace pic
