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

// Persistent grid: `slots` resident blocks, but at least `min_planes` planes
// per block (each block re-reads two halo planes per run).
inline void set_stream_blocks(StreamGeo& g, int slots, int min_planes = 4) {
  long b = g.total / min_planes;
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

constexpr int kMaxStages = 8;
// Block sizes of the plane-streaming kernels (4 cells per thread). Small
// blocks, several per SM, overlap one another's per-plane barrier and copy
// waits; the tall-slab form of the direction kernel (one 1024-thread block
// per SM) re-reads fewer halo rows, which pays once N >= 512 (measured).
constexpr int kStreamSmall = 256;
constexpr int kStreamTall = 1024;

// Layout of one stage: vector 0 (type A) then optional vector 1 (type B),
// each rows*N elements; stage size rounded up to 128 bytes.
template <typename A, typename B, int NV>
struct StageLayout {
  size_t e, bytes;
  __host__ __device__ StageLayout(int rows, int N) {
    e = (size_t)rows * N;
    size_t b = e * sizeof(A) + (NV == 2 ? e * sizeof(B) : 0);
    bytes = (b + 127) & ~(size_t)127;
  }
  __device__ A* v0(unsigned char* base, int st) const { return reinterpret_cast<A*>(base + st * bytes); }
  __device__ B* v1(unsigned char* base, int st) const {
    return reinterpret_cast<B*>(base + st * bytes + e * sizeof(A));
  }
};

// Streams the block's runs of planes through the ring of raw TMA stages.
// For every arriving plane l of a run, each thread transforms 4 consecutive
// cells (its own, plus one halo-row chunk for the threads on the slab's first
// and last row):
//   ingest(st, e, s, z) -> V4<TP>   transformed values at stage element
//                             offset e of global plane z,
// writes them to plane buffer l % 3 (x-y neighbours of other threads) and
// keeps its own cells in a register queue (centre and z-neighbours). After a
// single barrier the raw stage is refilled and output plane t = l - 2 runs:
//   body(s, t, pb, zm, c, zp) pb = plane buffer of plane t (x-y neighbours),
//                             zm/c/zp = own cells at planes t-1, t, t+1.
//   start(s)                  once per run before its first plane (prefetch).
// Three plane buffers make one barrier per plane sufficient. mbarrier phases
// continue across runs; every issued copy is waited for before the next run.
template <typename TP, typename A, typename B, int NV, typename Start, typename Ingest, typename Body>
__device__ __forceinline__ bool stream_slab(const StreamGeo& g, unsigned char* smem, uint64_t* bars, const A* src0,
                                            const B* src1, int* err, Start start, Ingest ingest, Body body) {
  const StageLayout<A, B, NV> lay(g.rows, g.N);
  const size_t pb_elems = (size_t)g.rows * g.N;
  TP* pbuf = reinterpret_cast<TP*>(smem + (size_t)g.S * lay.bytes);
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int st = 0; st < g.S; ++st) mbar_init(&bars[st], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t base = 0;  // loads issued (and consumed) in earlier runs
  bool ok = true;
  for_each_run(g, [&](int yt, int z0, int zc) {
    if (!ok) return;
    const Slab s = make_slab(g, yt, z0, zc);
    const int nload = s.ZC + 2;
    const uint32_t tx = plane_bytes<A>(s) + (NV == 2 ? plane_bytes<B>(s) : 0u);
    auto issue = [&](int l) {
      const uint32_t L = base + (uint32_t)l;
      const int st = (int)(L % (uint32_t)s.S);
      const int z = load_plane(s, l);
      mbar_arrive_expect_tx(&bars[st], tx);
      issue_plane(lay.v0(smem, st), src0, s, z, &bars[st]);
      if (NV == 2) issue_plane(lay.v1(smem, st), src1, s, z, &bars[st]);
    };
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      const int pre = nload < s.S ? nload : s.S;
      for (int l = 0; l < pre; ++l) issue(l);
    }
    if (s.active) start(s);
    // halo-row chunks owned by this thread (stage rows 0 and TY+1; with
    // TY == 1 the same thread owns both)
    const bool halo_lo = s.TY != s.N && s.active && s.ty == 0;
    const bool halo_hi = s.TY != s.N && s.active && s.ty == s.TY - 1;
    const size_t own = (size_t)s.srow * s.N + s.x0;
    const size_t hal_lo = (size_t)s.x0;
    const size_t hal_hi = (size_t)(s.TY + 1) * s.N + s.x0;
    V4<TP> q0, q1, q2;
    for (int l = 0; l < nload; ++l) {
      const uint32_t L = base + (uint32_t)l;
      const int st = (int)(L % (uint32_t)s.S);
      if (!mbar_wait_bounded(&bars[st], (L / (uint32_t)s.S) & 1u, err)) abort_flag = 1;
      TP* pb = pbuf + (size_t)(L % 3u) * pb_elems;
      if (s.active) {
        const int zl = load_plane(s, l);
        q0 = q1;
        q1 = q2;
        q2 = ingest(st, own, s, zl);
        st4(pb + own, q2);
        if (halo_lo) st4(pb + hal_lo, ingest(st, hal_lo, s, zl));
        if (halo_hi) st4(pb + hal_hi, ingest(st, hal_hi, s, zl));
      }
      __syncthreads();
      if (abort_flag) {
        ok = false;
        return;
      }
      if (threadIdx.x == 0 && l + s.S < nload) {
        fence_proxy_async_smem();
        issue(l + s.S);
      }
      if (l >= 2 && s.active) body(s, l - 2, pbuf + (size_t)((L + 2u) % 3u) * pb_elems, q0, q1, q2);
    }
    base += (uint32_t)nload;
  });
  return ok;
}

// Bytes of dynamic shared memory for stream_slab: S raw stages + 3 plane buffers.
template <typename TP, typename A, typename B, int NV>
__host__ __device__ inline size_t stream_smem_bytes(int rows, int N, int S) {
  const StageLayout<A, B, NV> lay(rows, N);
  return (size_t)S * lay.bytes + 3 * (size_t)rows * N * sizeof(TP);
}

// x-y neighbours from the plane buffer, z-neighbours and centre from registers:
// returns 6 c - (sum of the 6 neighbours) on the thread's 4 cells.
template <typename T>
__device__ __forceinline__ V4<T> stencil_q(const T* pb, const Slab& s, const V4<T>& zm, const V4<T>& c,
                                           const V4<T>& zp) {
  const int N = s.N;
  const T* row = pb + (size_t)s.srow * N;
  const T xm = row[s.x0 == 0 ? N - 1 : s.x0 - 1];
  const T xp = row[s.x0 + 4 == N ? 0 : s.x0 + 4];
  const V4<T> ym = ld4(pb + (size_t)s.rm * N + s.x0);
  const V4<T> yp = ld4(pb + (size_t)s.rp * N + s.x0);
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

}  // namespace pic
