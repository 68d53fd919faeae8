// Red-black SSOR preconditioner, the paper's PCG configuration (Sec. 4.1:
// four inner and two outer iterations, damping pi/2). z = M r starts from
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

}  // namespace

int ssor_apply(pic_ctx* c, const float* r, float* z, const int* done) {
  const int N = c->N;
  if (N % 4) return PIC_EINVAL;
  const size_t nq = (size_t)(N / 4) * N * N;
  size_t b = (nq + 255) / 256;
  const size_t cap = (size_t)c->sms * 8;
  const unsigned grid = (unsigned)(b < cap ? b : cap);
  bool first = true;
  auto half = [&](int colour) {
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
