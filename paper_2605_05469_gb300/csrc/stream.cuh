// Plane-streaming machinery for the periodic 7-point stencil (Sec. 3.2).
//
// A slab is TY full x-rows (TY a divisor of N chosen by the host to fit the
// kernel's thread limit and the shared-memory budget,
// so a slab plane is at most 1024 cells). Persistent blocks each take an even
// contiguous share of the (slab, plane) work list and walk its planes in z.
// For every plane a block
// needs the slab rows plus one halo row on each side (periodic in y); these
// are contiguous runs in memory, so each plane arrives as one to three bulk
// copies issued by one thread on the TMA engine into a ring of S
// shared-memory stages, completion tracked by one mbarrier per stage. The
// x-neighbours wrap inside the row, the z-neighbours are the previous and
// next stages. Each thread owns 4 consecutive x-cells of one slab row.
#pragma once
#include "common.cuh"

namespace pic {

struct StreamGeo {
  int N;        // grid size
  int TY;       // rows per slab
  int rows;     // rows held per stage: TY + 2, or N when TY == N (halo by wrap)
  int nyt;      // N / TY slabs
  int S;        // raw stages
  int threads;  // N * TY / 4 threads that own cells
  int blocks;   // persistent grid size
  long total;   // nyt * N plane-tiles of work
};

// Slab height: the largest divisor of N with at most 1024 cells per slab plane.
inline StreamGeo make_stream_geo(int N, int S, int TY) {
  StreamGeo g;
  g.N = N;
  g.TY = TY;
  g.rows = (g.TY == N) ? N : g.TY + 2;
  g.nyt = N / g.TY;
  g.threads = N * g.TY / 4;
  g.total = (long)g.nyt * N;
  g.S = S;
  g.blocks = 1;
  return g;
}

// Persistent grid: `slots` resident blocks, but at least 4 planes per block.
inline void set_stream_blocks(StreamGeo& g, int slots) {
  long b = g.total / 4;
  if (b < 1) b = 1;
  g.blocks = (int)(slots < b ? slots : b);
}

// One contiguous run of planes of one slab, handled by one block.
struct Slab {
  int N, TY, ZC, rows, S;
  int j0, z0;       // first slab row, first output plane
  int ty, x0;       // this thread's row within the slab and first x
  int srow;         // this thread's row index inside a stage
  int rm, rp;       // stage rows of its y-1 and y+1 neighbours
  bool active;      // thread owns cells (threadIdx.x < threads)
};

__device__ __forceinline__ Slab make_slab(const StreamGeo& g, int yt, int z0, int zc) {
  Slab s;
  s.N = g.N; s.TY = g.TY; s.ZC = zc; s.rows = g.rows; s.S = g.S;
  s.j0 = yt * g.TY;
  s.z0 = z0;
  const int c = threadIdx.x * 4;
  s.active = threadIdx.x < g.threads;
  s.ty = s.active ? c / g.N : 0;
  s.x0 = s.active ? c % g.N : 0;
  if (g.TY == g.N) {
    s.srow = s.ty;
    s.rm = (s.ty == 0) ? g.N - 1 : s.ty - 1;
    s.rp = (s.ty == g.N - 1) ? 0 : s.ty + 1;
  } else {
    s.srow = s.ty + 1;
    s.rm = s.ty;
    s.rp = s.ty + 2;
  }
  return s;
}

// The block's share [b T / P, (b+1) T / P) of the plane-tiles in slab-major
// order, visited as runs that stay inside one slab: calls f(yt, z0, zc).
template <typename F>
__device__ __forceinline__ void for_each_run(const StreamGeo& g, F f) {
  long a = (long)blockIdx.x * g.total / gridDim.x;
  const long e = (long)(blockIdx.x + 1) * g.total / gridDim.x;
  while (a < e) {
    const int yt = (int)(a / g.N), z0 = (int)(a % g.N);
    long stop = (long)(yt + 1) * g.N;
    if (stop > e) stop = e;
    f(yt, z0, (int)(stop - a));
    a = stop;
  }
}

// Global plane index of load l (l = 0 is the plane before the first output).
__device__ __forceinline__ int load_plane(const Slab& s, int l) {
  int z = s.z0 - 1 + l;
  if (z < 0) z += s.N;
  if (z >= s.N) z -= s.N;
  return z;
}

__device__ __forceinline__ size_t stage_elems(const Slab& s) { return (size_t)s.rows * s.N; }

// Issue the bulk copies of plane `z` of `src` into the stage buffer `dst`.
template <typename T>
__device__ __forceinline__ void issue_plane(T* dst, const T* src, const Slab& s, int z, uint64_t* bar) {
  const size_t N = s.N;
  const T* plane = src + (size_t)z * N * N;
  if (s.TY == s.N) {
    bulk_g2s(dst, plane, (uint32_t)(N * N * sizeof(T)), bar);
  } else {
    const int jl = (s.j0 == 0) ? s.N - 1 : s.j0 - 1;
    const int jh = (s.j0 + s.TY == s.N) ? 0 : s.j0 + s.TY;
    bulk_g2s(dst, plane + (size_t)jl * N, (uint32_t)(N * sizeof(T)), bar);
    bulk_g2s(dst + N, plane + (size_t)s.j0 * N, (uint32_t)(s.TY * N * sizeof(T)), bar);
    bulk_g2s(dst + (size_t)(s.TY + 1) * N, plane + (size_t)jh * N, (uint32_t)(N * sizeof(T)), bar);
  }
}

template <typename T>
__device__ __forceinline__ uint32_t plane_bytes(const Slab& s) {
  return (uint32_t)(stage_elems(s) * sizeof(T));
}

// 4 consecutive values.
template <typename T>
struct V4 {
  T v[4];
};

__device__ __forceinline__ V4<float> ld4(const float* p) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& x) {
  *reinterpret_cast<float4*>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& x) {
  reinterpret_cast<double2*>(p)[0] = make_double2(x.v[0], x.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(x.v[2], x.v[3]);
}
__device__ __forceinline__ V4<float> ldg4(const float* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ldg4(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {{a.x, a.y, b.x, b.y}};
}

// Scaled operator h^2 A = 6 I - (sum of the 6 periodic neighbours) on this
// thread's 4 cells. prev/cur/next are the stage buffers of planes z-1, z, z+1.
// Returns the centre values in `c`.
template <typename T>
__device__ __forceinline__ V4<T> stencil4(const T* prev, const T* cur, const T* next, const Slab& s, V4<T>& c) {
  const int N = s.N;
  const T* row = cur + (size_t)s.srow * N;
  c = ld4(row + s.x0);
  const T xm = row[s.x0 == 0 ? N - 1 : s.x0 - 1];
  const T xp = row[s.x0 + 4 == N ? 0 : s.x0 + 4];
  const V4<T> ym = ld4(cur + (size_t)s.rm * N + s.x0);
  const V4<T> yp = ld4(cur + (size_t)s.rp * N + s.x0);
  const V4<T> zm = ld4(prev + (size_t)s.srow * N + s.x0);
  const V4<T> zp = ld4(next + (size_t)s.srow * N + s.x0);
  V4<T> o;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const T l = (i == 0) ? xm : c.v[i - 1];
    const T r = (i == 3) ? xp : c.v[i + 1];
    const T sum = ((l + r) + (ym.v[i] + yp.v[i])) + (zm.v[i] + zp.v[i]);
    o.v[i] = (T)6 * c.v[i] - sum;
  }
  return o;
}

// Global offset of this thread's first cell in output plane t of the slab.
__device__ __forceinline__ size_t cell_offset(const Slab& s, int t) {
  const size_t N = s.N;
  return ((size_t)(s.z0 + t) * N + (size_t)(s.j0 + s.ty)) * N + s.x0;
}

}  // namespace pic
