// Red-black SSOR preconditioner, the paper's PCG configuration (Sec. 4.1:
// INNER = 4, OUTER = 2, damping w = pi/2). z = M r starts from
// z = 0 and repeats OUTER times: INNER forward SOR sweeps (red nodes, then
// black), then INNER backward sweeps (black, then red). Nodes are red when
// i + j + k is even; every 7-point neighbour of a node has the other colour,
// so a half-sweep updates its colour in place from the other colour's values:
//   z_i <- (1 - w) z_i + w (r_i + sum of the 6 neighbours) / 6
// in the scaled units of (h^2 A) z = r. FP32.
#include "ctx.h"
#include "ssor.h"

namespace pic {
namespace {

constexpr float kSsorOmega = 1.57079632679489662f;  // pi / 2
constexpr int kSsorInner = 4, kSsorOuter = 2;

// One half-sweep over the nodes of colour `colour` (0 red, 1 black); each
// thread takes 4 consecutive x nodes (two of each colour) and stores only
// the two of its colour, so no thread writes a value another thread reads.
// first: z is zero on entry (the first half-sweep: z = w r / 6 on the colour,
// 0 elsewhere).
__global__ void __launch_bounds__(256) k_ssor_half(float* z, const float* __restrict__ r, int N, int colour,
                                                   float w, int first, const int* done) {
  if (done && *done) return;
  const int Nq = N >> 2;
  const size_t nq = (size_t)Nq * N * N;
  const float w6 = w / 6.0f, keep = 1.0f - w;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (size_t)gridDim.x * blockDim.x) {
    const unsigned row = (unsigned)(q / (unsigned)Nq);
    const int i0 = 4 * (int)(q - (size_t)row * Nq);
    const int j = (int)(row % (unsigned)N), k = (int)(row / (unsigned)N);
    const size_t base = (size_t)row * N + i0;
    // the cells of this colour among i0 .. i0+3: offsets a and a + 2
    const int a = ((i0 + j + k) & 1) == colour ? 0 : 1;
    const float4 rv = __ldg(reinterpret_cast<const float4*>(r + base));
    const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
    if (first) {
      z[base + a] = w6 * rr[a];
      z[base + a + 2] = w6 * rr[a + 2];
      z[base + (a ^ 1)] = 0.0f;
      z[base + (a ^ 1) + 2] = 0.0f;
      continue;
    }
    const float4 cv = *reinterpret_cast<const float4*>(z + base);
    const float c[4] = {cv.x, cv.y, cv.z, cv.w};
    const size_t rowN = (size_t)row * N;
    const float xm = z[rowN + (i0 == 0 ? N - 1 : i0 - 1)];
    const float xp = z[rowN + (i0 + 4 == N ? 0 : i0 + 4)];
    const size_t pl = (size_t)k * N * N;
    const int jm = j == 0 ? N - 1 : j - 1, jp = j == N - 1 ? 0 : j + 1;
    const int km = k == 0 ? N - 1 : k - 1, kp = k == N - 1 ? 0 : k + 1;
    const float4 ym = *reinterpret_cast<const float4*>(z + pl + (size_t)jm * N + i0);
    const float4 yp = *reinterpret_cast<const float4*>(z + pl + (size_t)jp * N + i0);
    const float4 zm = *reinterpret_cast<const float4*>(z + ((size_t)km * N + j) * N + i0);
    const float4 zp = *reinterpret_cast<const float4*>(z + ((size_t)kp * N + j) * N + i0);
    const float ymv[4] = {ym.x, ym.y, ym.z, ym.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w};
    const float zmv[4] = {zm.x, zm.y, zm.z, zm.w}, zpv[4] = {zp.x, zp.y, zp.z, zp.w};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int o = a + 2 * t;
      const float l = o == 0 ? xm : c[o - 1];
      const float rgt = o == 3 ? xp : c[o + 1];
      const float s = ((l + rgt) + (ymv[o] + ypv[o])) + (zmv[o] + zpv[o]);
      z[base + o] = keep * c[o] + w6 * (rr[o] + s);
    }
  }
}

// The same half-sweep as a z-march (N % 128 == 0): a 32 x 8 block over a tile
// of 128 x-cells by 8 rows, each thread 4 x-cells of one row marching up zc
// planes with the planes below and above in registers. A node's neighbours
// all have the other colour, which this half-sweep does not write, so the
// values carried from plane to plane stay valid; each thread stores only the
// two cells of its colour.
__global__ void __launch_bounds__(256) k_ssor_zmarch(float* z, const float* __restrict__ r, int N, int colour,
                                                     float w, int zc, const int* done) {
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
  const float w6 = w / 6.0f, keep = 1.0f - w;
  auto at = [&](int zz, int jj) { return (size_t)zz * NN + (size_t)jj * N; };
  auto ld = [&](size_t off) { return *reinterpret_cast<const float4*>(z + off); };
  const int zb = z0 == 0 ? N - 1 : z0 - 1;
  float4 cm = ld(at(zb, j) + i0), c0 = ld(at(z0, j) + i0);
#pragma unroll 1
  for (int t = 0; t < zc; ++t) {
    const int zz = z0 + t;
    const int zn = zz + 1 == N ? 0 : zz + 1;
    const float4 cp = ld(at(zn, j) + i0);
    const size_t row = at(zz, j);
    const float4 ym = ld(at(zz, jm) + i0), yp = ld(at(zz, jp) + i0);
    const float4 rv = __ldg(reinterpret_cast<const float4*>(r + row + i0));
    float xl = __shfl_up_sync(0xffffffffu, c0.w, 1);
    float xr = __shfl_down_sync(0xffffffffu, c0.x, 1);
    if (lane == 0) xl = z[row + il];
    if (lane == 31) xr = z[row + ir];
    const int a = ((i0 + j + zz) & 1) == colour ? 0 : 1;
    const float c[4] = {c0.x, c0.y, c0.z, c0.w};
    const float ymv[4] = {ym.x, ym.y, ym.z, ym.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w};
    const float zmv[4] = {cm.x, cm.y, cm.z, cm.w}, zpv[4] = {cp.x, cp.y, cp.z, cp.w};
    const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int o = a + 2 * q;
      const float l = o == 0 ? xl : c[o - 1];
      const float rg = o == 3 ? xr : c[o + 1];
      const float sn = ((l + rg) + (ymv[o] + ypv[o])) + (zmv[o] + zpv[o]);
      z[row + i0 + o] = keep * c[o] + w6 * (rr[o] + sn);
    }
    cm = c0;
    c0 = cp;
  }
}

}  // namespace

int ssor_apply(pic_ctx* c, const float* r, float* z, const int* done) {
  const int N = c->N;
  if (N % 4) return PIC_EINVAL;
  const size_t nq = (size_t)(N / 4) * N * N;
  size_t b = (nq + 255) / 256;
  const size_t cap = (size_t)c->sms * 8;
  const unsigned grid = (unsigned)(b < cap ? b : cap);
  bool first = true;
  const bool zm = N % 128 == 0;
  const unsigned tiles = (unsigned)(N / 128) * (unsigned)(N / 8);
  int zc = 16;
  while (zm && zc > 4 && (long)tiles * (N / zc) < 4L * c->sms) zc /= 2;
  auto half = [&](int colour) {
    if (zm && !first)
      launch(c, k_ssor_zmarch, dim3(tiles, N / zc), dim3(32, 8), 0, z, r, N, colour, kSsorOmega, zc, done);
    else
      launch(c, k_ssor_half, grid, 256, 0, z, r, N, colour, kSsorOmega, first ? 1 : 0, done);
    first = false;
  };
  for (int o = 0; o < kSsorOuter; ++o) {
    for (int i = 0; i < kSsorInner; ++i) {
      half(0);
      half(1);
    }
    for (int i = 0; i < kSsorInner; ++i) {
      half(1);
      half(0);
    }
  }
  CK(cudaGetLastError());
  return PIC_OK;
}

}  // namespace pic

extern "C" int pic_ssor_apply(pic_ctx* c, const float* r, float* z) {
  if (!c || !r || !z) return PIC_EINVAL;
  if (!c->has_grid) return PIC_ESTATE;
  return pic::ssor_apply(c, r, z, nullptr);
}
