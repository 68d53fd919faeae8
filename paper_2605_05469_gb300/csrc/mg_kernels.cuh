// Geometric multigrid V-cycle, the preconditioner of flexible CG beyond the
// paper's Jacobi-PCG (its conclusion, Sec. 5, sets PCG beside the multigrid
// solvers of a cited comparison; better preconditioning is its named future
// work, Secs. 4.3 and 5).
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
//
// Levels whose size is a multiple of 4 stream their planes through the
// shared-memory slabs of the CG kernels (one HBM pass per kernel, 4 cells a
// thread) with the passes fused where the arithmetic allows:
//   pre-smoothing   both sweeps from x = 0 in one pass, x = w (2 r - w A^ r);
//   post-smoothing  the prolongation folded into the first sweep, the fine
//                   x' = x + P e_c formed as each plane arrives;
//   residual        (with the prolongation, for the learned smoother);
//   restriction     two coarse nodes a thread from float4 rows.
// Other sizes take the per-cell kernels below them.
#pragma once
#include "common.cuh"
#include "stream.cuh"

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

// ---------------------------------------------------------------------------
// Plane-streamed kernels (N % 4 == 0)
// ---------------------------------------------------------------------------

// v += (P e_c) on the 4 fine cells x0..x0+3 (x0 % 4 == 0) of fine row j,
// plane z (fine grid N, coarse Nc = N / 2 even): fine x = 2I is coarse I, fine
// x = 2I+1 the mean of I and I+1, likewise in y and z, so the cells need
// coarse x-nodes I0, I0+1, I0+2 (I0 = x0 / 2) summed over the 1, 2 or 4
// coarse (row, plane) pairs around (j / 2, z / 2).
__device__ __forceinline__ void add_prolonged(V4<float>& v, const float* __restrict__ ec, int Nc, int x0, int j,
                                              int z) {
  const int I0 = x0 >> 1;
  const int I2 = (I0 + 2 == Nc) ? 0 : I0 + 2;
  const int J0 = j >> 1, K0 = z >> 1;
  const int J1 = (J0 + 1 == Nc) ? 0 : J0 + 1;
  const int K1 = (K0 + 1 == Nc) ? 0 : K0 + 1;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  auto acc = [&](int J, int K) {
    const float* row = ec + ((size_t)K * Nc + J) * Nc;
    const float2 a = __ldg(reinterpret_cast<const float2*>(row + I0));
    s0 += a.x;
    s1 += a.y;
    s2 += __ldg(row + I2);
  };
  acc(J0, K0);
  if (j & 1) acc(J1, K0);
  if (z & 1) {
    acc(J0, K1);
    if (j & 1) acc(J1, K1);
  }
  const float wyz = ((j & 1) ? 0.5f : 1.f) * ((z & 1) ? 0.5f : 1.f);
  v.v[0] += wyz * s0;
  v.v[1] += wyz * (0.5f * (s0 + s1));
  v.v[2] += wyz * s1;
  v.v[3] += wyz * (0.5f * (s1 + s2));
}

// Global row of stage offset e (stage rows are the slab's rows plus one halo
// row each side, or the whole plane when TY == N) and the x of its first cell.
__device__ __forceinline__ void stage_row_x(const Slab& s, size_t e, int& j, int& x0) {
  const int N = s.N;
  const unsigned sr = (unsigned)e / (unsigned)N;
  x0 = (int)((unsigned)e - sr * (unsigned)N);
  j = (s.TY == N) ? (int)sr : wrapi(s.j0 - 1 + (int)sr, N);
}

// Pre-smoothing, nu1 = 2 damped sweeps from x = 0 in one pass:
// x1 = w r, x2 = x1 + w (r - A^ x1) = w (2 r - w A^ r), w = omega / 6.
template <bool TALL>
__global__ void __launch_bounds__(TALL ? kStreamTall : kStreamSmall) k_mg_pre(const float* __restrict__ r,
                                                                            float* __restrict__ x, int* err,
                                                                            StreamGeo g, const int* done) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  if (done && *done) return;
  const StageLayout<float, float, 1> lay(g.rows, g.N);
  const float w = kOmega / 6.0f;
  auto start = [&](const Slab&) {};
  auto ingest = [&](int st, size_t e, const Slab&, int) { return ld4(lay.v0(smem, st) + e); };
  auto body = [&](const Slab& s, int t, const float* pb, const V4<float>& zm, const V4<float>& c,
                  const V4<float>& zp) {
    const V4<float> ar = stencil_q(pb, s, zm, c, zp);
    V4<float> o;
#pragma unroll
    for (int i = 0; i < 4; ++i) o.v[i] = w * (2.0f * c.v[i] - w * ar.v[i]);
    st4(x + cell_offset(s, t), o);
  };
  stream_slab<float, float, float, 1>(g, smem, bars, r, (const float*)nullptr, err, start, ingest, body);
}

enum : int { kResid = 0, kSmooth = 1 };

// With x' = x (PROLONG false) or x' = x + P e_c (PROLONG true):
//   kResid : out = r - A^ x'        (and xout = x' when PROLONG)
//   kSmooth: out = x' + w (r - A^ x')
// out and xout must not alias x (other blocks read x's halo rows).
// x streams through the slab stages together with r (r's own cells are
// kept in a two-deep register queue at ingest: the body of plane t runs one
// arriving plane later).
template <int MODE, bool PROLONG, bool TALL>
__global__ void __launch_bounds__(TALL ? kStreamTall : kStreamSmall) k_mg_stencil(
    const float* __restrict__ x, const float* __restrict__ r, float* __restrict__ out, float* __restrict__ xout,
    const float* __restrict__ ec, int* err, StreamGeo g, const int* done) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  if (done && *done) return;
  const StageLayout<float, float, 2> lay(g.rows, g.N);
  const float w = kOmega / 6.0f;
  const int Nc = g.N >> 1;
  V4<float> r_prev, r_cur;
  auto start = [&](const Slab&) {};
  auto ingest = [&](int st, size_t e, const Slab& s, int z) {
    V4<float> v = ld4(lay.v0(smem, st) + e);
    if (PROLONG) {
      int j, x0;
      stage_row_x(s, e, j, x0);
      add_prolonged(v, ec, Nc, x0, j, z);
    }
    if (e == (size_t)s.srow * s.N + s.x0) {
      r_prev = r_cur;
      r_cur = ld4(lay.v1(smem, st) + e);
    }
    return v;
  };
  auto body = [&](const Slab& s, int t, const float* pb, const V4<float>& zm, const V4<float>& c,
                  const V4<float>& zp) {
    const V4<float> ax = stencil_q(pb, s, zm, c, zp);
    const size_t off = cell_offset(s, t);
    V4<float> o;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      o.v[i] = MODE == kResid ? r_prev.v[i] - ax.v[i] : c.v[i] + w * (r_prev.v[i] - ax.v[i]);
    st4(out + off, o);
    if (PROLONG && MODE == kResid) st4(xout + off, c);
  };
  stream_slab<float, float, float, 2>(g, smem, bars, x, r, err, start, ingest, body);
}

// ---------------------------------------------------------------------------
// z-marching kernels (N % 128 == 0): a block is 32 x 8 threads over a tile of
// 128 x-cells by 8 rows; each thread owns 4 x-cells of one row and marches up
// a chunk of ZC planes, keeping the field at planes z-1, z, z+1 in registers
// (the next plane's load is issued a plane ahead). x-neighbours come from the
// adjacent lanes (each warp is one row of the tile; lanes 0 and 31 load the
// cell beyond the tile), y-neighbours are loads of the adjacent rows (L1 hits
// within the tile). No shared memory and no barriers.
//   kZPre   : field r:  out = w (2 r - w A^ r)      (both pre-sweeps from 0)
//   kZResid : field x:  out = aux - A^ x             (aux = r)
//   kZSmooth: field x:  out = x + w (aux - A^ x)
// ---------------------------------------------------------------------------
//   with PROLONG the field is x' = x + P e_c (formed for every value loaded:
//   own column, adjacent rows, the cells beyond the tile), and kZResid also
//   writes x' to xout.
enum : int { kZPre = 0, kZResid = 1, kZSmooth = 2 };
constexpr int kZChunkMax = 16;  // planes a block marches (fewer on small grids, for more blocks)

// (P e_c) at one fine node (i, j, z): the mean of the 1, 2, 4 or 8 coarse
// nodes around it (coarse grid Nc = N / 2).
__device__ __forceinline__ float prolonged_at(const float* __restrict__ ec, int Nc, int i, int j, int z) {
  const int I0 = i >> 1, J0 = j >> 1, K0 = z >> 1;
  const int I1 = (i & 1) ? (I0 + 1 == Nc ? 0 : I0 + 1) : I0;
  const int J1 = (j & 1) ? (J0 + 1 == Nc ? 0 : J0 + 1) : J0;
  const int K1 = (z & 1) ? (K0 + 1 == Nc ? 0 : K0 + 1) : K0;
  auto e = [&](int I, int J, int K) { return __ldg(ec + ((size_t)K * Nc + J) * Nc + I); };
  const float s = ((e(I0, J0, K0) + e(I1, J0, K0)) + (e(I0, J1, K0) + e(I1, J1, K0))) +
                  ((e(I0, J0, K1) + e(I1, J0, K1)) + (e(I0, J1, K1) + e(I1, J1, K1)));
  return 0.125f * s;
}

template <int MODE, bool PROLONG = false>
__global__ void __launch_bounds__(256) k_mg_zmarch(const float* __restrict__ field, const float* __restrict__ aux,
                                                   float* __restrict__ out, int N, int zc, const int* done,
                                                   const float* __restrict__ ec, float* __restrict__ xout) {
  if (done && *done) return;
  const int tiles_x = N >> 7;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int lane = threadIdx.x;
  const int i0 = (tx << 7) + 4 * lane;
  const int j = ty * 8 + threadIdx.y;
  const int jm = j == 0 ? N - 1 : j - 1, jp = j == N - 1 ? 0 : j + 1;
  const int z0 = blockIdx.y * zc;
  const size_t NN = (size_t)N * N;
  const int il = i0 == 0 ? N - 1 : i0 - 1, ir = i0 + 4 == N ? 0 : i0 + 4;
  const float w = kOmega / 6.0f;
  const int Nc = N >> 1;
  auto at = [&](int z, int jj) { return (size_t)z * NN + (size_t)jj * N; };
  auto ld = [&](const float* p, size_t off) { return __ldg(reinterpret_cast<const float4*>(p + off)); };
  // the field's float4 at (z, row jj) (x' when PROLONG)
  auto fld = [&](int z, int jj) {
    float4 v = ld(field, at(z, jj) + i0);
    if (PROLONG) {
      V4<float> u = {{v.x, v.y, v.z, v.w}};
      add_prolonged(u, ec, Nc, i0, jj, z);
      v = make_float4(u.v[0], u.v[1], u.v[2], u.v[3]);
    }
    return v;
  };
  const int zb = z0 == 0 ? N - 1 : z0 - 1;
  float4 cm = fld(zb, j);
  float4 c0 = fld(z0, j);
#pragma unroll 1
  for (int t = 0; t < zc; ++t) {
    const int z = z0 + t;
    const int zn = z + 1 == N ? 0 : z + 1;
    const float4 cp = fld(zn, j);
    const size_t row = at(z, j);
    const float4 ym = fld(z, jm), yp = fld(z, jp);
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MODE != kZPre) a = ld(aux, row + i0);
    float xl = __shfl_up_sync(0xffffffffu, c0.w, 1);
    float xr = __shfl_down_sync(0xffffffffu, c0.x, 1);
    if (lane == 0) xl = __ldg(field + row + il) + (PROLONG ? prolonged_at(ec, Nc, il, j, z) : 0.f);
    if (lane == 31) xr = __ldg(field + row + ir) + (PROLONG ? prolonged_at(ec, Nc, ir, j, z) : 0.f);
    const float c[4] = {c0.x, c0.y, c0.z, c0.w};
    const float ymv[4] = {ym.x, ym.y, ym.z, ym.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w};
    const float zmv[4] = {cm.x, cm.y, cm.z, cm.w}, zpv[4] = {cp.x, cp.y, cp.z, cp.w};
    const float av[4] = {a.x, a.y, a.z, a.w};
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float l = q == 0 ? xl : c[q - 1];
      const float r = q == 3 ? xr : c[q + 1];
      const float s = ((l + r) + (ymv[q] + ypv[q])) + (zmv[q] + zpv[q]);
      const float ax = 6.0f * c[q] - s;
      o[q] = MODE == kZPre ? w * (2.0f * c[q] - w * ax) : (MODE == kZResid ? av[q] - ax : c[q] + w * (av[q] - ax));
    }
    *reinterpret_cast<float4*>(out + row + i0) = make_float4(o[0], o[1], o[2], o[3]);
    if (PROLONG && MODE == kZResid) *reinterpret_cast<float4*>(xout + row + i0) = c0;
    cm = c0;
    c0 = cp;
  }
}

// rc = 4 R res onto the coarse grid Nf/2 (Nf % 4 == 0): each thread the
// coarse pair (2P, 2P+1) of row J of plane K = blockIdx.y, from the fine
// float4 at x = 4P and the scalar at 4P - 1 of each of the 9 fine rows.
__global__ void __launch_bounds__(256) k_mg_restrict2(const float* __restrict__ res, float* __restrict__ rc, int Nf,
                                                      const int* done) {
  if (done && *done) return;
  const int Nc = Nf >> 1, Np = Nc >> 1;
  const unsigned per_plane = (unsigned)Np * (unsigned)Nc;
  const int K = blockIdx.y;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < per_plane; q += gridDim.x * blockDim.x) {
    const int J = (int)(q / (unsigned)Np), P = (int)(q - (unsigned)J * (unsigned)Np);
    const int i0 = 4 * P, im = i0 == 0 ? Nf - 1 : i0 - 1;
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int oz = -1; oz <= 1; ++oz) {
      const size_t zb = (size_t)wrapi(2 * K + oz, Nf) * Nf;
      const float wz = oz ? 0.25f : 0.5f;
      float b0 = 0.f, b1 = 0.f;
#pragma unroll
      for (int oy = -1; oy <= 1; ++oy) {
        const float* row = res + (zb + (size_t)wrapi(2 * J + oy, Nf)) * Nf;
        const float wy = oy ? 0.25f : 0.5f;
        const float4 v = __ldg(reinterpret_cast<const float4*>(row + i0));
        const float m = __ldg(row + im);
        b0 = fmaf(wy, 0.25f * m + 0.5f * v.x + 0.25f * v.y, b0);
        b1 = fmaf(wy, 0.25f * v.y + 0.5f * v.z + 0.25f * v.w, b1);
      }
      a0 = fmaf(wz, b0, a0);
      a1 = fmaf(wz, b1, a1);
    }
    *reinterpret_cast<float2*>(rc + ((size_t)K * Nc + J) * Nc + 2 * P) = make_float2(4.0f * a0, 4.0f * a1);
  }
}

// ---------------------------------------------------------------------------
// Per-cell kernels (any even N)
// ---------------------------------------------------------------------------
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

// y = x.
__global__ void __launch_bounds__(256) k_mg_copy(const float* __restrict__ x, float* __restrict__ y, size_t n,
                                                 const int* done) {
  if (done && *done) return;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    y[c] = x[c];
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

// The cells c = t, t + nt, t + 2 nt, ... of an N^3 grid (t = threadIdx.x)
// with their coordinates (i, j, k), advanced by additions with carries
// instead of three divisions per cell.
struct CellWalk {
  int c, i, j, k, di, dj, dk, n, N, nt;
  __device__ __forceinline__ CellWalk(int N_, int nt_) : N(N_), nt(nt_) {
    n = N * N * N;
    c = threadIdx.x;
    i = c % N;
    j = (c / N) % N;
    k = c / (N * N);
    di = nt % N;
    dj = (nt / N) % N;
    dk = nt / (N * N);
  }
  __device__ __forceinline__ bool ok() const { return c < n; }
  __device__ __forceinline__ void next() {
    c += nt;
    i += di;
    int carry = 0;
    if (i >= N) {
      i -= N;
      carry = 1;
    }
    j += dj + carry;
    carry = 0;
    if (j >= N) {
      j -= N;
      carry = 1;
    }
    k += dk + carry;
  }
};

// One damped Jacobi sweep out = x + w (r - A^ x) (x_zero: x = 0) over the
// threads [0, nt), then a barrier of those threads (the block, or warp 0).
template <bool WARP>
__device__ __forceinline__ void sm_sweep(const float* x, const float* r, float* out, int N, bool x_zero) {
  const int n = N * N * N;
  const float w = kOmega / 6.0f;
  const int nt = WARP ? 32 : (int)blockDim.x;
  if (!WARP || threadIdx.x < 32) {
    if (x_zero) {
      for (int c = threadIdx.x; c < n; c += nt) out[c] = w * r[c];
    } else {
      for (CellWalk q(N, nt); q.ok(); q.next())
        out[q.c] = x[q.c] + w * (r[q.c] - apply_hat(x, N, q.i, q.j, q.k));
    }
  }
  if (WARP) __syncwarp();
  else __syncthreads();
}

// nu sweeps on level (x, r) with scratch t, ping-ponging x -> t -> x; the
// result ends in x (one copy when nu is odd).
template <bool WARP>
__device__ __forceinline__ void sm_smooth(float* x, const float* r, float* t, int N, int nu, bool from_zero) {
  for (int s = 0; s < nu; ++s) {
    const bool into_t = (s % 2) == 0;
    sm_sweep<WARP>(into_t ? x : t, r, into_t ? t : x, N, from_zero && s == 0);
  }
  if (nu % 2) {
    const int n = N * N * N, nt = WARP ? 32 : (int)blockDim.x;
    if (!WARP || threadIdx.x < 32)
      for (int c = threadIdx.x; c < n; c += nt) x[c] = t[c];
    if (WARP) __syncwarp();
    else __syncthreads();
  }
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
    sm_smooth<false>(x, r, t, N, nu, true);
    for (CellWalk q(N, blockDim.x); q.ok(); q.next()) t[q.c] = r[q.c] - apply_hat(x, N, q.i, q.j, q.k);
    __syncthreads();
    const int Nc = S.N[l + 1];
    float* rc = R + S.off[l + 1];
    for (CellWalk q(Nc, blockDim.x); q.ok(); q.next()) {
      const int c = q.c, I = q.i, J = q.j, K = q.k;
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
  // coarsest: damped Jacobi sweeps from zero (one warp when the level is tiny)
  {
    const int l = S.n - 1, N = S.N[l];
    float *x = X + S.off[l], *r = R + S.off[l], *t = T + S.off[l];
    if (N * N * N <= 256) {
      sm_smooth<true>(x, r, t, N, kCoarseSweeps, true);
      __syncthreads();
    } else {
      sm_smooth<false>(x, r, t, N, kCoarseSweeps, true);
    }
  }
  // up: prolong-add, post-smooth
  for (int l = S.n - 2; l >= 0; --l) {
    const int N = S.N[l], n = N * N * N, Nc = S.N[l + 1];
    float *x = X + S.off[l], *r = R + S.off[l], *t = T + S.off[l];
    const float* ec = X + S.off[l + 1];
    for (CellWalk q(N, blockDim.x); q.ok(); q.next()) {
      const int c = q.c, i = q.i, j = q.j, k = q.k;
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
    sm_smooth<false>(x, r, t, N, nu, false);
  }
  for (int c = threadIdx.x; c < n0; c += blockDim.x) x_out[c] = X[c];
}

}  // namespace mg
}  // namespace pic
