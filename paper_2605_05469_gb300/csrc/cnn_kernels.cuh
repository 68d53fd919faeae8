// Kernels of the learned preconditioner: a 4-layer 3x3x3 conv3d network
// (1 -> 16 -> 16 -> 16 -> 1 channels, no biases, identity activations) with
// periodic wrap whose layers 3 and 4 are the adjoints of layers 2 and 1, so
// N = G^T G is symmetric positive semi-definite (a learned factorised sparse
// approximate inverse); its training (data and weight gradients, loss, Adam)
// and crop extraction. The paper solves the Poisson system with
// preconditioned CG (Sec. 3.2); this learned preconditioner is used inside
// flexible CG.
//
// Convolutions run on the 5th-generation tensor cores as implicit GEMMs:
// one CTA owns an 8 (x) x 16 (y) x 4 (z) output tile; M = 128 output cells of
// one z-plane, N = 16 output channels, K = 16 input channels per tap, 27 taps
// accumulated into one FP32 TMEM accumulator per plane (4 planes = 64 TMEM
// columns). Activations are BF16 channels-last; the CTA stores its halo tile
// (10 x 18 x 6 cells) as two 8-channel planes so that each tap's A operand is
// the tile shifted by a constant: a no-swizzle K-major shared-memory
// descriptor with start = cell (tz, ty, tx) of the tile, SBO = one tile row
// (10 cells x 16 B, the next 8 output cells in y) and LBO = the 8-channel
// plane stride. One thread issues the 27 x 4 tcgen05.mma; tcgen05.commit
// signals an mbarrier; the 4 warps read their 32 TMEM lanes back with
// tcgen05.ld and apply the epilogue. One-channel inputs (the first layer and
// the last layer's data gradient) use an im2col A tile (27 taps padded to
// K = 32, two MMAs per plane).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace pic {
namespace cnn {

constexpr int kLayers = 4;
constexpr int kWeights = 14688;  // 16*27 + 16*16*27 + 16*16*27 + 16*27
constexpr int kLayerOff[5] = {0, 432, 7344, 14256, 14688};

// Output tile and halo tile of one CTA.
constexpr int TX = 8, TY = 16, ZT = 4;
constexpr int HX = TX + 2, HY = TY + 2, HZ = ZT + 2;
constexpr int HCELLS = HX * HY * HZ;  // 1080
constexpr int CHUNK = HCELLS * 16;    // bytes of one 8-channel BF16 plane: 17280
constexpr int W16_BYTES = 27 * 512;   // 27 taps x (16 x 16 BF16) canonical
constexpr int W1_BYTES = 1024;        // 16 x 32 BF16 canonical (im2col K)
constexpr int IM2COL_PLANE = 8192;    // 128 rows x 32 K BF16
constexpr int kThreads = 128;

// Epilogue modes.
enum : int {
  OUT_BF16 = 0,        // bf16 x16 = acc
  OUT_SCALED_F32 = 2,  // f32 x1  = scale * acc[channel 0]
  OUT_RAW_F32 = 3,     // f32 x16 = acc (tests)
};

// Per-launch scale taken from a device scalar: 1, 1/sqrt(*src * mul), or sqrt(*src * mul).
enum : int { SCALE_ONE = 0, SCALE_RSQRT = 1, SCALE_SQRT = 2 };

__device__ __forceinline__ float scale_from(const double* src, double mul, int mode) {
  if (mode == SCALE_ONE || src == nullptr) return 1.f;
  const double v = *src * mul;
  if (!(v > 0.0)) return 0.f;
  return mode == SCALE_RSQRT ? (float)(1.0 / sqrt(v)) : (float)sqrt(v);
}

struct ConvParams {
  int NX, NY, NZ, B;       // per-sample grid (periodic) and batch
  const void* in;          // CIN 16: bf16 [cells][16]; CIN 1: f32 [cells]
  void* out;
  const unsigned char* w;     // canonical BF16 weights of this conv
  const double* in_scale_src;  // CIN 1 input multiplier (see scale_from)
  double in_scale_mul;
  int in_scale_mode;
  const double* out_scale_src;  // OUT_SCALED_F32 multiplier
  double out_scale_mul;
  int out_scale_mode;
  int* err;
};

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D F32, A/B BF16, both K-major, N = 16, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Canonical K-major no-swizzle byte offset of element (row, k) of a matrix
// whose core matrices are (row/8, k/8) at (row/8) * 128 + (k/8) * lbo.
__device__ __forceinline__ int canon_off(int row, int k, int lbo) {
  return (row >> 3) * 128 + (k >> 3) * lbo + (row & 7) * 16 + (k & 7) * 2;
}

template <int CIN>
__global__ void __launch_bounds__(kThreads) k_conv_tc(ConvParams P, int mode) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t mma_bar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = P.NX / TX, tiles_y = P.NY / TY, tiles_z = P.NZ / ZT;
  int t = blockIdx.x;
  const int bx = t % tiles_x; t /= tiles_x;
  const int by = t % tiles_y; t /= tiles_y;
  const int bz = t % tiles_z; t /= tiles_z;
  const int b = t;
  const int x0 = bx * TX, y0 = by * TY, z0 = bz * ZT;
  const size_t sample = (size_t)P.NX * P.NY * P.NZ;
  const size_t sbase = (size_t)b * sample;

  constexpr int A_BYTES = CIN == 16 ? 2 * CHUNK : ZT * IM2COL_PLANE;
  constexpr int W_BYTES = CIN == 16 ? W16_BYTES : W1_BYTES;
  unsigned char* sA = smem;
  unsigned char* sW = smem + A_BYTES;
  float* sF = reinterpret_cast<float*>(smem + A_BYTES + W_BYTES);  // CIN 1: f32 halo tile

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&mma_bar, 1);
    fence_mbar_init();
  }
  // weights
  {
    const uint4* src = reinterpret_cast<const uint4*>(P.w);
    uint4* dst = reinterpret_cast<uint4*>(sW);
    for (int i = tid; i < W_BYTES / 16; i += kThreads) dst[i] = __ldg(src + i);
  }
  if (CIN == 16) {
    const uint4* in = reinterpret_cast<const uint4*>(P.in);
    for (int c = tid; c < HCELLS; c += kThreads) {
      const int hx = c % HX, hy = (c / HX) % HY, hz = c / (HX * HY);
      const int gx = wrap(x0 - 1 + hx, P.NX), gy = wrap(y0 - 1 + hy, P.NY), gz = wrap(z0 - 1 + hz, P.NZ);
      const size_t cell = sbase + ((size_t)gz * P.NY + gy) * P.NX + gx;
      const uint4 lo = __ldg(in + 2 * cell), hi = __ldg(in + 2 * cell + 1);
      reinterpret_cast<uint4*>(sA)[c] = lo;
      reinterpret_cast<uint4*>(sA + CHUNK)[c] = hi;
    }
  } else {
    const float* in = reinterpret_cast<const float*>(P.in);
    const float sc = scale_from(P.in_scale_src, P.in_scale_mul, P.in_scale_mode);
    for (int c = tid; c < HCELLS; c += kThreads) {
      const int hx = c % HX, hy = (c / HX) % HY, hz = c / (HX * HY);
      const int gx = wrap(x0 - 1 + hx, P.NX), gy = wrap(y0 - 1 + hy, P.NY), gz = wrap(z0 - 1 + hz, P.NZ);
      sF[c] = sc * __ldg(in + sbase + ((size_t)gz * P.NY + gy) * P.NX + gx);
    }
    __syncthreads();
    // im2col: row m = ly * 8 + lx, k = tz * 9 + ty * 3 + tx (k >= 27 zero)
    const int m = tid, lx = m & 7, ly = m >> 3;
    for (int zt = 0; zt < ZT; ++zt) {
      unsigned char* plane = sA + zt * IM2COL_PLANE;
      for (int k = 0; k < 32; ++k) {
        float v = 0.f;
        if (k < 27) {
          const int tz = k / 9, ty = (k / 3) % 3, tx = k % 3;
          v = sF[((zt + tz) * HY + (ly + ty)) * HX + (lx + tx)];
        }
        *reinterpret_cast<__nv_bfloat16*>(plane + canon_off(m, k, 2048)) = __float2bfloat16_rn(v);
      }
    }
  }
  // make the generic-proxy shared-memory writes visible to the tensor cores
  fence_proxy_async_smem();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (tid == 0) {
    const uint32_t a0 = smem_u32(sA), w0 = smem_u32(sW);
    for (int zt = 0; zt < ZT; ++zt) {
      const uint32_t d = tmem + (uint32_t)(zt * 16);
      if (CIN == 16) {
        for (int tap = 0; tap < 27; ++tap) {
          const int tz = tap / 9, ty = (tap / 3) % 3, tx = tap % 3;
          const uint32_t a = a0 + (uint32_t)((((zt + tz) * HY + ty) * HX + tx) * 16);
          mma_bf16(d, smem_desc(a, CHUNK, HX * 16), smem_desc(w0 + tap * 512, 256, 128), tap > 0);
        }
      } else {
        for (int q = 0; q < 2; ++q) {
          const uint32_t a = a0 + (uint32_t)(zt * IM2COL_PLANE + q * 2 * 2048);
          mma_bf16(d, smem_desc(a, 2048, 128), smem_desc(w0 + q * 2 * 256, 256, 128), q > 0);
        }
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&mma_bar))
                 : "memory");
  }
  const bool done = mbar_wait_bounded(&mma_bar, 0, P.err);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (done) {
    const int m = warp * 32 + lane, lx = m & 7, ly = m >> 3;
    const float osc = mode == OUT_SCALED_F32 ? scale_from(P.out_scale_src, P.out_scale_mul, P.out_scale_mode) : 1.f;
    for (int zt = 0; zt < ZT; ++zt) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(zt * 16), v);
      const size_t cell = sbase + ((size_t)(z0 + zt) * P.NY + (y0 + ly)) * P.NX + (x0 + lx);
      if (mode == OUT_BF16) {
        __align__(16) __nv_bfloat16 o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) o[i] = __float2bfloat16_rn(v[i]);
        uint4* op = reinterpret_cast<uint4*>(P.out) + 2 * cell;
        op[0] = reinterpret_cast<const uint4*>(o)[0];
        op[1] = reinterpret_cast<const uint4*>(o)[1];
      } else if (mode == OUT_SCALED_F32) {
        reinterpret_cast<float*>(P.out)[cell] = osc * v[0];
      } else {
        float4* op = reinterpret_cast<float4*>(P.out) + 4 * cell;
#pragma unroll
        for (int i = 0; i < 4; ++i) op[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

template <int CIN>
constexpr size_t conv_smem_bytes() {
  return CIN == 16 ? (size_t)2 * CHUNK + W16_BYTES : (size_t)ZT * IM2COL_PLANE + W1_BYTES + HCELLS * 4;
}

// ---------------------------------------------------------------------------
// Weight packing: FP32 master weights (oracle layout w[o][c][tz][ty][tx] per
// layer, concatenated) -> canonical BF16 tiles for the forward convs and for
// the data-gradient convs (flipped taps, in/out channels swapped).
// Layout of `packed`: fwd1 (1 KB) | fwd2, fwd3, fwd4 (13.5 KB each) |
//                     bwd4 (1 KB) | bwd3, bwd2 (13.5 KB each)
// ---------------------------------------------------------------------------
constexpr int kPackFwd1 = 0;
constexpr int kPackFwd2 = kPackFwd1 + W1_BYTES;
constexpr int kPackFwd3 = kPackFwd2 + W16_BYTES;
constexpr int kPackFwd4 = kPackFwd3 + W16_BYTES;
constexpr int kPackBwd4 = kPackFwd4 + W16_BYTES;
constexpr int kPackBwd3 = kPackBwd4 + W1_BYTES;
constexpr int kPackBwd2 = kPackBwd3 + W16_BYTES;
constexpr int kPackBytes = kPackBwd2 + W16_BYTES;

__device__ __forceinline__ void put(unsigned char* base, int off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

__global__ void k_pack_weights(const float* __restrict__ w, unsigned char* __restrict__ packed) {
  const float* w1 = w + kLayerOff[0];
  const float* w2 = w + kLayerOff[1];
  const float* w3 = w + kLayerOff[2];
  const float* w4 = w + kLayerOff[3];
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 16 * 32; i += stride) {
    const int n = i / 32, k = i % 32;
    // fwd1: B[n = out][k = tap]
    put(packed + kPackFwd1, canon_off(n, k, 256), k < 27 ? w1[n * 27 + k] : 0.f);
    // bwd4: B[n = c (input channel of layer 4)][k = flipped tap]
    put(packed + kPackBwd4, canon_off(n, k, 256), k < 27 ? w4[n * 27 + (26 - k)] : 0.f);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 27 * 256; i += stride) {
    const int tap = i / 256, n = (i / 16) % 16, k = i % 16;
    const int off = tap * 512 + canon_off(n, k, 256);
    // forward: B_tap[n = out][k = in] = w[o = n][c = k][tap]
    put(packed + kPackFwd2, off, w2[(n * 16 + k) * 27 + tap]);
    put(packed + kPackFwd3, off, w3[(n * 16 + k) * 27 + tap]);
    put(packed + kPackFwd4, off, n == 0 ? w4[k * 27 + tap] : 0.f);
    // data gradient: B_tap'[n = c][k = o] = w[o = k][c = n][26 - tap']
    put(packed + kPackBwd3, off, w3[(k * 16 + n) * 27 + (26 - tap)]);
    put(packed + kPackBwd2, off, w2[(k * 16 + n) * 27 + (26 - tap)]);
  }
}

// ---------------------------------------------------------------------------
// Tying of layers 3 and 4 to the adjoints of layers 2 and 1:
//   adj(w)[c][o][t] = w[o][c][26 - t].
// k_tie_weights: w3 = adj(w2), w4 = adj(w1).
// k_tie_grads:   g1 += adj(g4), g2 += adj(g3), then g3 = adj(g2), g4 = adj(g1)
//                (the gradient of the tied network, repeated in all slots so
//                that an elementwise optimiser keeps the tie).
// ---------------------------------------------------------------------------
__global__ void k_tie_weights(float* w) {
  float* w1 = w + kLayerOff[0];
  float* w2 = w + kLayerOff[1];
  float* w3 = w + kLayerOff[2];
  float* w4 = w + kLayerOff[3];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 16 * 16 * 27; i += gridDim.x * blockDim.x) {
    const int o = i / (16 * 27), c = (i / 27) % 16, t = i % 27;
    w3[(c * 16 + o) * 27 + (26 - t)] = w2[i];
    if (i < 16 * 27) {
      const int oo = i / 27, tt = i % 27;
      w4[oo * 27 + (26 - tt)] = w1[i];
    }
  }
}

__global__ void k_tie_grads(float* g) {
  // one thread per (free) weight of layers 1 and 2; each pair is read and
  // written by exactly one thread
  float* g1 = g + kLayerOff[0];
  float* g2 = g + kLayerOff[1];
  float* g3 = g + kLayerOff[2];
  float* g4 = g + kLayerOff[3];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 16 * 16 * 27; i += gridDim.x * blockDim.x) {
    const int o = i / (16 * 27), c = (i / 27) % 16, t = i % 27;
    const int j = (c * 16 + o) * 27 + (26 - t);
    const float v = g2[i] + g3[j];
    g2[i] = v;
    g3[j] = v;
    if (i < 16 * 27) {
      const int oo = i / 27, tt = i % 27;
      const int jj = oo * 27 + (26 - tt);
      const float u = g1[i] + g4[jj];
      g1[i] = u;
      g4[jj] = u;
    }
  }
}

// ---------------------------------------------------------------------------
// Inference through the composed kernel. The network is linear, so
// N x = G^T G x is one 9x9x9 convolution: with g_o[s] (o = 0..15, s in
// [0, 5)^3) the kernel of output channel o of G = conv(w2) o conv(w1),
//   g_o[s] = sum_m sum_{t1 + t2 = s} w2[o][m][t2] w1[m][0][t1],
// N x[p] = sum_d K[d] x[p + d], d in [-4, 4]^3,
//   K[d] = sum_o sum_{s - s' = d} g_o[s] g_o[s'],
// symmetric (K[d] = K[-d]). k_compose builds K (FP32, 729 values) from the
// master weights; k_apply_k applies it with periodic wrap on the CUDA cores:
// 729 FMA per cell instead of the 14 688 MACs per cell of the 4 layers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_compose(const float* __restrict__ w, float* __restrict__ K) {
  __shared__ float g[16 * 125];
  const float* w1 = w + kLayerOff[0];
  const float* w2 = w + kLayerOff[1];
  for (int i = threadIdx.x; i < 16 * 125; i += blockDim.x) {
    const int o = i / 125, sidx = i % 125;
    const int sz = sidx / 25, sy = (sidx / 5) % 5, sx = sidx % 5;
    float acc = 0.f;
    for (int t1 = 0; t1 < 27; ++t1) {
      const int az = t1 / 9, ay = (t1 / 3) % 3, ax = t1 % 3;
      const int bz = sz - az, by = sy - ay, bx = sx - ax;
      if (bz < 0 || bz > 2 || by < 0 || by > 2 || bx < 0 || bx > 2) continue;
      const int t2 = (bz * 3 + by) * 3 + bx;
      for (int m = 0; m < 16; ++m) acc = fmaf(w2[(o * 16 + m) * 27 + t2], w1[m * 27 + t1], acc);
    }
    g[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 729; i += blockDim.x) {
    const int dz = i / 81 - 4, dy = (i / 9) % 9 - 4, dx = i % 9 - 4;
    float acc = 0.f;
    for (int sidx = 0; sidx < 125; ++sidx) {
      const int sz = sidx / 25, sy = (sidx / 5) % 5, sx = sidx % 5;
      const int qz = sz - dz, qy = sy - dy, qx = sx - dx;  // s' = s - d
      if (qz < 0 || qz > 4 || qy < 0 || qy > 4 || qx < 0 || qx > 4) continue;
      const int q = (qz * 5 + qy) * 5 + qx;
      for (int o = 0; o < 16; ++o) acc = fmaf(g[o * 125 + sidx], g[o * 125 + q], acc);
    }
    K[i] = acc;
  }
}

constexpr int KX = 32, KY = 8, KZ = 16;                     // outputs per CTA
constexpr int KHX = KX + 8, KHY = KY + 8, KHZ = KZ + 8;     // input tile with the 4-cell halo
constexpr size_t kApplySmem = (size_t)KHZ * KHY * KHX * sizeof(float);  // 60 KB

// The composed kernel travels as a launch parameter (constant bank), so with
// the tap loops fully unrolled every FMA reads its coefficient from there.
struct K729 {
  float k[729];
};

// z = K * r on an N^3 periodic grid, N % 32 == 0. Each thread owns one (x, y)
// column of KZ outputs; for every (dy, dx) it loads the KZ + 8 input values of
// its column once from shared memory and uses each for up to 9 dz.
__global__ void __launch_bounds__(256) k_apply_k(const float* __restrict__ r, float* __restrict__ z, int N,
                                                 const K729 K) {
  extern __shared__ __align__(16) float tile[];  // [KHZ][KHY][KHX]
  const int tx = threadIdx.x % KX, ty = threadIdx.x / KX;
  const int bx = blockIdx.x % (N / KX), rest = blockIdx.x / (N / KX);
  const int by = rest % (N / KY), bz = rest / (N / KY);
  const int x0 = bx * KX, y0 = by * KY, z0 = bz * KZ;
  for (int i = threadIdx.x; i < KHZ * KHY * KHX; i += blockDim.x) {
    const int hx = i % KHX, hy = (i / KHX) % KHY, hz = i / (KHX * KHY);
    const int gx = wrap(x0 - 4 + hx, N), gy = wrap(y0 - 4 + hy, N), gz = wrap(z0 - 4 + hz, N);
    tile[i] = __ldg(r + ((size_t)gz * N + gy) * N + gx);
  }
  __syncthreads();
  float acc[KZ];
#pragma unroll
  for (int j = 0; j < KZ; ++j) acc[j] = 0.f;
#pragma unroll
  for (int dy = 0; dy < 9; ++dy) {
#pragma unroll
    for (int dx = 0; dx < 9; ++dx) {
      float v[KZ + 8];
#pragma unroll
      for (int k = 0; k < KZ + 8; ++k) v[k] = tile[(k * KHY + ty + dy) * KHX + tx + dx];
#pragma unroll
      for (int dz = 0; dz < 9; ++dz) {
        const float kd = K.k[(dz * 9 + dy) * 9 + dx];
#pragma unroll
        for (int j = 0; j < KZ; ++j) acc[j] = fmaf(kd, v[j + dz], acc[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < KZ; ++j) z[((size_t)(z0 + j) * N + (y0 + ty)) * N + (x0 + tx)] = acc[j];
}

// ---------------------------------------------------------------------------
// The composed 9^3 kernel on the tensor cores.
//
// For fixed (dz, dy) the x-direction sum over dx of K[dz][dy][dx] r[x + dx - 4]
// for 16 consecutive outputs x0..x0+15 is a product with the 32 x 16 Toeplitz
// matrix T_{dz,dy}[k][n] = K[dz][dy][k - n] (0 <= k - n <= 8, else 0) of the
// 32 inputs x0-4..x0+27. The A operand holds one input plane z' of a column
// of 128 output rows y0..y0+127 (136 input rows with the y halo, BF16, x
// along K); the row offset dy is a descriptor offset. The B operand for one dy
// stacks the nine T_{dz,dy} along N (N = 144), so one MMA gives the
// contributions of input plane z' to the nine output planes p = z' - dz + 4
// at once, in nine groups of 16 TMEM columns. The output planes live in a
// TMEM ring of 16-column slots whose slot index decreases with p: group dz of
// the MMA of plane z' lands in the slot of p = z' - dz + 4, so the dz sum is
// accumulated by the tensor core itself; an output plane is final once input
// plane p + 4 has been multiplied, and the epilogue reads it out. Per input
// plane: 9 dy x 2 K-steps of 16 = 18 MMAs (M 128, N <= 144). The epilogue
// zeroes a slot after reading it, so every MMA accumulates.
//
// Work: the unit is one output plane of one column (16 x 128 cells); CTA k of
// G takes units [k U / G, (k + 1) U / G) of the U = (N/16)(N/128) N units in
// column-major order, which are one or two runs of consecutive planes of a
// column; a run of planes [pa, pb) streams input planes pa-4 .. pb+3.
// Warp-specialised pipeline: producer warps stream input planes through a
// ring of FP32 stages (cp.async, three planes ahead) and convert them into a
// ring of BF16 A operands; one thread issues the MMAs as operands become
// ready; epilogue warps write each output plane back once its last input
// plane has been multiplied. mbarrier rings hand each plane from one role to
// the next, so the tensor cores are fed several planes ahead.
// ---------------------------------------------------------------------------
namespace tck {
constexpr int BX = 16;                    // x outputs per Toeplitz group
constexpr int BY = 128;                   // y outputs per column (the 128 TMEM lanes)
constexpr int AROWS = BY + 8;             // input rows y0-4 .. y0+131
// one 8-element K chunk of an input plane; the extra 64 B put chunks 1 and 3
// on the other half of the shared-memory banks for the fill
constexpr int CHUNK_B = AROWS * 16 + 64;  // 2240
constexpr int SLOT_B = 4 * CHUNK_B;       // 8960: one BF16 input plane, 32 x-inputs
constexpr int BROWS = 9 * 16;             // N rows of the B operand of one dy: (dz, n)
constexpr int BCHUNK_B = BROWS * 16;      // 2304
constexpr int BDY_B = 4 * BCHUNK_B;       // 9216
constexpr int B_BYTES = 9 * BDY_B;        // 82944: all 81 Toeplitz matrices
// TMEM: 32 physical slots of 16 columns (all 512 columns). Output planes
// take ring slots (-v) mod 24; a plane's nine groups start at a ring slot
// s < 24 and run on into physical slots up to s + 8 <= 31, so slots 24..31
// shadow ring slots 0..7 and no MMA ever wraps. An output with ring slot
// r <= 7 may hold partial sums in r and r + 24; the epilogue adds both.
constexpr int TSLOTS = 24;
constexpr int PSLOTS = 32;
constexpr int TMEM_COLS = PSLOTS * 16;    // 512: all of the SM's tensor memory
// warp roles: warp 0 issues the MMAs, warps 1-4 read the finished output
// planes out of TMEM (warp w reaches TMEM lanes 32 (w % 4) .. + 31), warps
// 5-12 load and convert the input planes
constexpr int EPI_WARP0 = 1, PROD_WARP0 = 5, NWARPS = 13;
constexpr int THREADS = NWARPS * 32;      // 416
constexpr int PTHREADS = 256;             // producer threads
constexpr int LOADS = (AROWS * 8 + PTHREADS - 1) / PTHREADS;  // 16-byte pieces per producer per plane (5)
constexpr int ASLOTS = 4;                 // BF16 A operands (input planes ready for the tensor cores)
constexpr int TILE_OUT_B = BY * BX * 4;   // 8192: one output plane's 128 x 16 FP32 block
// the fused form's epilogue operands r, q, p, x of one output plane's block,
// double-buffered (cp.async two planes ahead)
constexpr int EPI_PLANE_B = 4 * TILE_OUT_B;
template <bool FUSED>
constexpr int epi_bufs() { return FUSED ? 2 : 0; }
// an output plane's TMEM slots (zeroed by the epilogue after it reads them)
// are taken again by the output plane TSLOTS later, whose first term comes
// from the input plane TSLOTS - 8 input planes after the one that completed it
constexpr int SLOT_REUSE_LAG = TSLOTS - 8;
constexpr int ERING = 32;                 // plane handshakes between the MMA issuer and the epilogue
template <bool FUSED>
constexpr size_t smem_bytes() {
  return (size_t)B_BYTES + ASLOTS * SLOT_B + TILE_OUT_B + epi_bufs<FUSED>() * EPI_PLANE_B;
}  // 126976 plain, 192512 fused
static_assert(smem_bytes<false>() > 114 * 1024 && smem_bytes<true>() <= 226 * 1024, "one CTA per SM");
static_assert(ERING > SLOT_REUSE_LAG, "the issuer must not lap the epilogue handshakes");
}  // namespace tck

// Packed B operand (global, built when K changes): for each dy, the canonical
// K-major N x K matrix with row n' = dz * 16 + n and column k, element
// T_{dz,dy}[k][n] = K[dz][dy][k - n].
__global__ void __launch_bounds__(256) k_pack_toeplitz(const float* __restrict__ K, unsigned char* __restrict__ Bg) {
  using namespace tck;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 9 * BROWS * 32; i += gridDim.x * blockDim.x) {
    const int dy = i / (BROWS * 32), np = (i / 32) % BROWS, k = i % 32;
    const int dz = np / 16, n = np % 16, dx = k - n;
    const float v = (dx >= 0 && dx <= 8) ? K[(dz * 9 + dy) * 9 + dx] : 0.f;
    const int off = dy * BDY_B + (np >> 3) * 128 + (k >> 3) * BCHUNK_B + (np & 7) * 16 + (k & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(Bg + off) = __float2bfloat16_rn(v);
  }
}

// kind::f16 instruction descriptor: D F32, A/B BF16, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

// D += A B^T (the accumulator is always read: the epilogue zeroes each TMEM
// slot before it is reused, so no MMA needs the overwrite form).
__device__ __forceinline__ void mma_acc(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 1, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc));
}

// All 18 MMAs of one input plane, straight-line: for each dy and K-step q the
// A operand is the plane shifted by dy rows and advanced by 16 x-inputs, the
// B operand the dz groups dz_lo.. of T_{., dy}. Every offset is a
// compile-time constant added to the base descriptors, so the issue stream
// carries no branches (branches between the MMAs of a plane cost the issuing
// thread more than the MMAs themselves).
__device__ __forceinline__ void tc_issue_plane(uint64_t ad0, uint64_t b0, uint32_t d0, uint32_t idesc) {
  using namespace tck;
#pragma unroll
  for (int dy = 0; dy < 9; ++dy) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint64_t a = ad0 + (uint64_t)((dy * 16 + q * 2 * CHUNK_B) >> 4);
      const uint64_t bo = (uint64_t)((dy * BDY_B + q * 2 * BCHUNK_B) >> 4);
      mma_acc(d0, a, b0 + bo, idesc);
    }
  }
}

// Ring slot of output number v (v >= 0 counts the CTA's output planes;
// 32-bit: a CTA holds a few thousand, and a 64-bit modulo on the issue path
// costs more than the MMAs it feeds).
__device__ __forceinline__ int tc_ring_slot(int v) { return (tck::TSLOTS - v % tck::TSLOTS) % tck::TSLOTS; }

// One input plane of the CTA's stream: column `col`, run of output planes
// [pa, pb), input plane z (unwrapped, pa-4 <= z <= pb+3).
struct TcPlane {
  int col, pa, pb, z;
};

// Work order of the persistent tensor-core kernels. The C columns (output
// blocks of one x-range and 128 rows, numbered x-block fastest) are dealt out
// whole and round-robin: CTA b takes columns b, b + G, ... for R = C / G
// rounds, so the G CTAs resident at a time walk G neighbouring columns
// through z together and share in L2 the rows of r that their windows
// overlap (a contiguous split of the (column, plane) units puts neighbouring
// columns at unrelated depths, and r is read from DRAM again for each; the
// change measured 980 -> 820 us for the 8-wide form at 512^3). The C - R G
// leftover columns' units are split contiguously. Output planes are numbered
// by a CTA-local counter that runs on across the CTA's runs.
struct TcWork {
  int N, R, G, b;
  int tcol0;    // first leftover column
  long tb, te;  // this CTA's share of the leftover units
};

__device__ __forceinline__ TcWork tc_work(int N, int C) {
  TcWork W;
  W.N = N;
  W.G = gridDim.x;
  W.b = blockIdx.x;
  W.R = C / W.G;
  W.tcol0 = W.R * W.G;
  const long TU = (long)(C - W.tcol0) * N;
  W.tb = TU * W.b / W.G;
  W.te = TU * (W.b + 1) / W.G;
  return W;
}

__device__ __forceinline__ bool tc_has_work(const TcWork& W) { return W.R > 0 || W.tb < W.te; }

struct TcCur {
  TcPlane P;  // column, run [pa, pb), input plane z
  int k;      // run index: k < R whole columns, then leftover runs
  long u;     // next leftover unit
  int vbase;  // output planes of the earlier runs
};

__device__ __forceinline__ bool tc_run(const TcWork& W, TcCur& c) {
  if (c.k < W.R) {
    c.P.col = W.b + c.k * W.G;
    c.P.pa = 0;
    c.P.pb = W.N;
  } else {
    if (c.u >= W.te) return false;
    c.P.col = W.tcol0 + (int)(c.u / W.N);
    c.P.pa = (int)(c.u % W.N);
    c.P.pb = (int)min((long)W.N, (long)c.P.pa + (W.te - c.u));
  }
  c.P.z = c.P.pa - 4;
  return true;
}

__device__ __forceinline__ bool tc_start(const TcWork& W, TcCur& c) {
  c.k = 0;
  c.u = W.tb;
  c.vbase = 0;
  return tc_has_work(W) && tc_run(W, c);
}

// Next input plane: z + 1 within the run (pa - 4 .. pb + 3), else the next run.
__device__ __forceinline__ bool tc_next(const TcWork& W, TcCur& c) {
  if (c.P.z + 1 < c.P.pb + 4) {
    ++c.P.z;
    return true;
  }
  const int len = c.P.pb - c.P.pa;
  c.vbase += len;
  if (c.k >= W.R) c.u += len;
  ++c.k;
  return tc_run(W, c);
}

__device__ __forceinline__ void tc_origin(const TcPlane& P, int N, int& x0, int& y0) {
  const int nbx = N / tck::BX;
  x0 = (P.col % nbx) * tck::BX;
  y0 = (P.col / nbx) * tck::BY;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Producer thread t moves the 16-byte pieces t + 256 i (i < 5) of every
// input plane: x-inputs 4 g .. 4 g + 3 with g = t % 8 (the same for all its
// pieces) of rows t / 8 + 32 i. Its source offsets within a plane depend on
// the column only and are recomputed when the column changes. Planes are
// loaded into registers two planes ahead of their conversion.
struct TcRows {
  int col;
  int off[tck::LOADS];  // (gy * N + gx) of each piece; -1 past the last row
};

__device__ __forceinline__ void tc_rows(const TcPlane& P, int N, int ptid, TcRows& R) {
  using namespace tck;
  int x0, y0;
  tc_origin(P, N, x0, y0);
  R.col = P.col;
  // 4-float pieces never straddle the periodic wrap (x0 - 4 is a multiple of 4)
  const int gx = wrap(x0 - 4 + 4 * (ptid & 7), N);
#pragma unroll
  for (int i = 0; i < LOADS; ++i) {
    const int row = (ptid >> 3) + 32 * i;
    R.off[i] = row < AROWS ? wrap(y0 - 4 + row, N) * N + gx : -1;
  }
}

// One input plane's pieces of r (and, fused, of q) in registers.
template <bool FUSED>
struct TcIn {
  float4 r[tck::LOADS];
  float4 q[FUSED ? tck::LOADS : 1];
};

template <bool FUSED>
__device__ __forceinline__ void tc_load(const TcPlane& P, const float* __restrict__ r, const float* __restrict__ q,
                                        int N, int ptid, TcRows& R, TcIn<FUSED>& in) {
  using namespace tck;
  if (R.col != P.col) tc_rows(P, N, ptid, R);
  const size_t plane = (size_t)wrap(P.z, N) * N * N;
#pragma unroll
  for (int i = 0; i < LOADS; ++i) {
    if (R.off[i] >= 0) {
      in.r[i] = __ldg(reinterpret_cast<const float4*>(r + plane + R.off[i]));
      if (FUSED) in.q[i] = __ldg(reinterpret_cast<const float4*>(q + plane + R.off[i]));
    }
  }
}

// Registers -> BF16 canonical K-major A operand: x-input k = 4 g .. 4 g + 3
// goes to K-chunk k / 8 at byte (k % 8) * 2 of its row. With FUSED the
// operand is the updated residual r - alpha q.
template <bool FUSED>
__device__ __forceinline__ void tc_store(const TcIn<FUSED>& in, unsigned char* slot, int ptid, float alpha) {
  using namespace tck;
  const int g = ptid & 7;
  unsigned char* dst = slot + (g >> 1) * CHUNK_B + (ptid >> 3) * 16 + (g & 1) * 8;
#pragma unroll
  for (int i = 0; i < LOADS; ++i) {
    if ((ptid >> 3) + 32 * i < AROWS) {
      float4 v = in.r[i];
      if (FUSED) {
        const float4 qv = in.q[i];
        v.x = fmaf(-alpha, qv.x, v.x);
        v.y = fmaf(-alpha, qv.y, v.y);
        v.z = fmaf(-alpha, qv.z, v.z);
        v.w = fmaf(-alpha, qv.w, v.w);
      }
      __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
      uint2 packed;
      packed.x = *reinterpret_cast<uint32_t*>(&lo);
      packed.y = *reinterpret_cast<uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(dst + i * 32 * 16) = packed;  // 32 rows further
    }
  }
}

// Zero 16 columns of the calling thread's TMEM lane (32x32b shape: each
// thread of the warp owns one lane) and wait for the store.
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  const uint32_t z0 = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(z0)
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// The CG update fused in front of the preconditioner (flexible CG, one
// iteration): with q = A p from the direction kernel,
//   r' = r - alpha q,  x' = x + alpha p  (x read as zero after a reliable
//   update folded it),  z = N r',
// and the reductions (r', r'), (r', z), (z, q), (r', q) that the update's
// convergence test and the next direction need. r' goes to a second buffer:
// neighbouring CTAs still read r as their halo.
struct TcFcg {
  const float* q;
  const float* p;
  float* x;
  float* r_new;
  Scalars* sc;
  double* partials;
  unsigned* counter;
  int only_redo;  // plain form: run only when a reliable update replaced r
};

struct TcDots {
  CompSum rr, rz, zq, rq;
};

// Epilogue thread et (0..127) moves float4 f = et + 128 k (k < 4) of the
// plane's 128 x 16 block: row f / 4, x-quarter f % 4.
__device__ __forceinline__ size_t tc_epi_offset(const TcPlane& P, int N, int et, int k) {
  int x0, y0;
  tc_origin(P, N, x0, y0);
  const int f = et + 128 * k;
  return ((size_t)(P.z - 4) * N + (size_t)(y0 + (f >> 2))) * N + x0 + 4 * (f & 3);
}

// The fused epilogue's operands r, q, p, x for the owned cells of the output
// plane that P completes, copied two planes ahead (they do not depend on the
// MMAs) into one of two shared-memory buffers: [array][f] float4 per buffer,
// each thread its own pieces. One cp.async group per plane, always committed.
__device__ __forceinline__ void tc_epi_fetch(const TcPlane& P, const float* __restrict__ r, int N, const TcFcg& F,
                                             bool x_zero, float4* buf) {
  if (P.z - 4 >= P.pa) {
    const int et = threadIdx.x - tck::EPI_WARP0 * 32;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int f = et + 128 * k;
      const size_t off = tc_epi_offset(P, N, et, k);
      cp_async16(buf + f, r + off);
      cp_async16(buf + 512 + f, F.q + off);
      cp_async16(buf + 1024 + f, F.p + off);
      if (!x_zero) cp_async16(buf + 1536 + f, F.x + off);
    }
  }
  cp_async_commit();
}

// Float4 slot of (row, c4) in the epilogue's transpose tile: XOR-swizzled so
// that both the row-per-thread writes and the coalesced reads are free of
// shared-memory bank conflicts.
__device__ __forceinline__ int tc_tile_idx(int row, int c4) { return row * 4 + (c4 ^ ((row >> 1) & 3)); }

__device__ __forceinline__ void tc_epi_barrier() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Output plane p = P.z - 4 is complete once input plane P.z has been
// multiplied. Epilogue warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows y),
// all 16 columns (x) of the slot, into a shared-memory tile; the 128
// epilogue threads then move the plane's 128 x 16 block to and from global
// memory four threads per 64-byte row segment (coalesced).
template <bool FUSED>
__device__ __forceinline__ void tc_epilogue(const TcPlane& P, float* __restrict__ z, int N, uint32_t tmem,
                                            int vbase, const TcFcg& F, float alpha, bool x_zero, TcDots& D,
                                            float4* tile, const float4* ops) {
  using namespace tck;
  const int p = P.z - 4;
  if (p < P.pa) return;  // an input plane of the lower halo: no output completes (uniform)
  const int s = tc_ring_slot(vbase + p - P.pa);
  const int et = threadIdx.x - EPI_WARP0 * 32;  // 0..127
  const int quarter = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
  const int row = quarter * 32 + lane;          // TMEM lane = y row of the block
  float o[16];
  const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(s * 16);
  tmem_ld16(ta, o);
  tmem_zero16(ta);  // the slot's next output plane starts from zero
  if (s + TSLOTS < PSLOTS) {
    // partial sums of the planes whose groups ran into the shadow slot
    float o2[16];
    const uint32_t tb = ta + (uint32_t)(TSLOTS * 16);
    tmem_ld16(tb, o2);
    tmem_zero16(tb);
#pragma unroll
    for (int i = 0; i < 16; ++i) o[i] += o2[i];
  }
  tc_epi_barrier();  // the previous plane's reads of the tile are done
#pragma unroll
  for (int c4 = 0; c4 < 4; ++c4)
    tile[tc_tile_idx(row, c4)] = make_float4(o[4 * c4], o[4 * c4 + 1], o[4 * c4 + 2], o[4 * c4 + 3]);
  tc_epi_barrier();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int f = et + 128 * k;
    const size_t off = tc_epi_offset(P, N, et, k);
    const float4 zv = tile[tc_tile_idx(f >> 2, f & 3)];
    *reinterpret_cast<float4*>(z + off) = zv;
    if (!FUSED) continue;
    float4 rv = ops[f], xv = x_zero ? make_float4(0.f, 0.f, 0.f, 0.f) : ops[1536 + f];
    const float4 qv = ops[512 + f], pv = ops[1024 + f];
    const float* q4 = &qv.x;
    const float* p4 = &pv.x;
    const float* z4 = &zv.x;
    float* r4 = &rv.x;
    float* x4 = &xv.x;
    float prr = 0.f, prz = 0.f, pzq = 0.f, prq = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      r4[i] = fmaf(-alpha, q4[i], r4[i]);  // the same value the producers fed the tensor cores
      x4[i] = fmaf(alpha, p4[i], x4[i]);
      prr = fmaf(r4[i], r4[i], prr);
      prz = fmaf(r4[i], z4[i], prz);
      pzq = fmaf(z4[i], q4[i], pzq);
      prq = fmaf(r4[i], q4[i], prq);
    }
    D.rr.add(prr);
    D.rz.add(prz);
    D.zq.add(pzq);
    D.rq.add(prq);
    *reinterpret_cast<float4*>(F.r_new + off) = rv;
    *reinterpret_cast<float4*>(F.x + off) = xv;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up as soon as another role has given up.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, int* err, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0) {
      if (*abort_flag) return false;
      if (global_timer_ns() - t0 > kWaitBudgetNs) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        *abort_flag = 1;
        return false;
      }
    }
  }
}

template <bool FUSED>
__global__ void __launch_bounds__(tck::THREADS, 1) k_apply_k_tc(const float* __restrict__ r, float* __restrict__ z,
                                                                int N, const unsigned char* __restrict__ Bg,
                                                                int* err, TcFcg F) {
  using namespace tck;
  if (F.sc) {
    if (F.sc->done) return;
    if (!FUSED && F.only_redo && !F.sc->redo) return;
  }
  const float alpha = FUSED ? (float)F.sc->alpha : 0.f;
  const bool x_zero = FUSED && F.sc->x32_reset != 0;
  TcDots dots;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ __align__(8) uint64_t a_full[ASLOTS], a_empty[ASLOTS], acc_full[ERING], acc_empty[ERING], b_bar;
  unsigned char* Bs = smem;                                         // B_BYTES
  unsigned char* slots = smem + B_BYTES;                            // ASLOTS x SLOT_B (BF16 A operands)
  float4* tile = reinterpret_cast<float4*>(slots + ASLOTS * SLOT_B);  // TILE_OUT_B (epilogue transpose)
  float4* ebuf = tile + TILE_OUT_B / 16;                            // fused: 2 x EPI_PLANE_B
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcWork W = tc_work(N, (N / BX) * (N / BY));
  const bool has_work = tc_has_work(W);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    // one arrival per producer / epilogue warp (per-thread arrivals on one
    // barrier word serialise)
    for (int i = 0; i < ASLOTS; ++i) {
      mbar_init(&a_full[i], PTHREADS / 32);
      mbar_init(&a_empty[i], 1);
    }
    for (int i = 0; i < ERING; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);
    }
    mbar_init(&b_bar, 1);
    fence_mbar_init();
    if (has_work) {
      mbar_arrive_expect_tx(&b_bar, B_BYTES);
      bulk_g2s(Bs, Bg, B_BYTES, &b_bar);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (warp >= EPI_WARP0 && warp < PROD_WARP0) {
    // every MMA accumulates: start from zeroed slots
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    for (int c = 0; c < TMEM_COLS; c += 16) tmem_zero16(lane_base + (uint32_t)c);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (warp == 0) {
    // ---- MMA issuer: one thread ----
    if (lane == 0 && has_work) {
      TcCur c;
      bool have = tc_start(W, c);
      const TcPlane& P = c.P;
      const bool b_ok = tc_wait(&b_bar, 0, err, &abort_flag);
      const uint64_t bd0 = smem_desc(smem_u32(Bs), BCHUNK_B, 128);
      for (uint32_t j = 0; have && b_ok; ++j) {
        const uint32_t sa = j % ASLOTS;
        if (!tc_wait(&a_full[sa], (j / ASLOTS) & 1u, err, &abort_flag)) break;
        if (j >= (uint32_t)SLOT_REUSE_LAG) {
          const uint32_t e = j - SLOT_REUSE_LAG;
          if (!tc_wait(&acc_empty[e % ERING], (e / ERING) & 1u, err, &abort_flag)) break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // groups dz_lo..dz_hi feed output planes z + 4 - dz inside [pa, pb)
        const int dz_lo = max(0, P.z + 4 - (P.pb - 1)), dz_hi = min(8, P.z + 4 - P.pa);
        const int s_lo = tc_ring_slot(c.vbase + (P.z + 4 - dz_lo - P.pa));
        const int ng = dz_hi - dz_lo + 1;
        const uint64_t ad0 = smem_desc(smem_u32(slots + sa * SLOT_B), CHUNK_B, 128);
        const uint64_t b0 = bd0 + (uint64_t)(dz_lo * 16);  // 16 B-rows per group = 256 B
        tc_issue_plane(ad0, b0, tmem + (uint32_t)(s_lo * 16), idesc_n(16 * ng));
        // both arrive once every MMA issued so far has completed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&a_empty[sa]))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&acc_full[j % ERING]))
                     : "memory");
        have = tc_next(W, c);
      }
      if (!b_ok) abort_flag = 1;
    }
    __syncwarp();
  } else if (warp < PROD_WARP0) {
    // ---- epilogue: 128 threads ----
    TcCur c;
    bool have = tc_start(W, c);
    constexpr int EB = EPI_PLANE_B / 16;  // float4 per operand buffer
    TcCur ahead = c;
    bool have_a = have;
    if (FUSED) {
      // operands of planes 0 and 1 in flight
      for (int b = 0; b < 2; ++b) {
        if (have_a) {
          tc_epi_fetch(ahead.P, r, N, F, x_zero, ebuf + b * EB);
          have_a = tc_next(W, ahead);
        } else {
          cp_async_commit();
        }
      }
    }
    for (uint32_t j = 0; have; ++j) {
      if (FUSED) cp_async_wait<1>();  // plane j's operands (own pieces)
      // warp-uniform: a lane that gave up takes its whole warp out
      if (!__all_sync(0xffffffffu, tc_wait(&acc_full[j % ERING], (j / ERING) & 1u, err, &abort_flag))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      tc_epilogue<FUSED>(c.P, z, N, tmem, c.vbase, F, alpha, x_zero, dots, tile, ebuf + (j & 1u) * EB);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[j % ERING]);
      if (FUSED) {
        // refill the buffer plane j used with plane j + 2
        if (have_a) {
          tc_epi_fetch(ahead.P, r, N, F, x_zero, ebuf + (j & 1u) * EB);
          have_a = tc_next(W, ahead);
        } else {
          cp_async_commit();
        }
      }
      have = tc_next(W, c);
    }
    if (FUSED) cp_async_wait<0>();
  } else {
    // ---- producers: 256 threads, two planes in registers ahead of conversion ----
    const int ptid = tid - PROD_WARP0 * 32;
    TcRows rows;
    rows.col = -1;
    TcIn<FUSED> in0, in1;
    TcCur cur, ahead;
    bool have = tc_start(W, cur);
    ahead = cur;
    bool have_a = have;
    if (have_a) {
      tc_load<FUSED>(ahead.P, r, F.q, N, ptid, rows, in0);
      have_a = tc_next(W, ahead);
    }
    if (have_a) {
      tc_load<FUSED>(ahead.P, r, F.q, N, ptid, rows, in1);
      have_a = tc_next(W, ahead);
    }
    uint32_t j = 0;
    // plane j from buffer `in`, which is then refilled with plane j + 2
    auto step = [&](TcIn<FUSED>& in) -> bool {
      const uint32_t sa = j % ASLOTS;
      bool ok = true;
      if (j >= (uint32_t)ASLOTS) {
        // the MMAs of plane j - ASLOTS, which read this A slot, are done
        const uint32_t k = j - ASLOTS;
        ok = tc_wait(&a_empty[sa], (k / ASLOTS) & 1u, err, &abort_flag);
      }
      if (!__all_sync(0xffffffffu, ok)) return false;  // warp-uniform
      tc_store<FUSED>(in, slots + sa * SLOT_B, ptid, alpha);
      fence_proxy_async_smem();  // the BF16 writes, visible to the tensor cores
      __syncwarp();
      if (lane == 0) mbar_arrive(&a_full[sa]);
      if (have_a) {
        tc_load<FUSED>(ahead.P, r, F.q, N, ptid, rows, in);
        have_a = tc_next(W, ahead);
      }
      ++j;
      return true;
    };
    while (have) {
      if (!step(in0)) break;
      if (!(have = tc_next(W, cur))) break;
      if (!step(in1)) break;
      have = tc_next(W, cur);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  if (FUSED) {
    double v[4] = {dots.rr.value(), dots.rz.value(), dots.zq.value(), dots.rq.value()}, tot[4];
    if (grid_reduce_last<4>(v, F.partials, F.counter, tot) && threadIdx.x == 0) {
      Scalars* sc = F.sc;
      // the update's bookkeeping (convergence and the reliable-update trigger)
      const double rr = tot[0];
      sc->x32_reset = 0;
      sc->rr_prev = sc->rr;
      sc->rr = rr;
      sc->iter += 1;
      if (!isfinite(rr)) {
        sc->done = 3;
      } else {
        if (rr <= sc->tol2) {
          sc->need_update = 1;
          sc->final_check = 1;
        } else if (rr <= sc->delta2 * sc->rmax2) {
          sc->need_update = 1;
        }
        if (!sc->need_update && sc->iter >= sc->maxit) sc->done = 2;
      }
      // the next direction: beta = -(z, q) / (p, q), with the descent guard
      double rz = tot[1], zq = tot[2];
      sc->fallback_now = 0;
      if (!(rz > 0.0) || !isfinite(rz) || !isfinite(zq)) {
        sc->fallback_now = 1;
        sc->fallbacks += 1;
        rz = rr / 6.0;
        zq = tot[3] / 6.0;
      }
      sc->beta = -zq / sc->pq;
      sc->rz = rz;
      if (!isfinite(sc->beta) && !sc->done) sc->done = 3;
    }
  }
}

// ---------------------------------------------------------------------------
// One layer of the network in FP32 on the CUDA cores (the training test mode):
// periodic within each D^3 crop of the batch, activations FP32 (one value a
// cell for one channel, 16 channel-last values a cell for sixteen), weights
// the FP32 master copy w[out][in][tz][ty][tx]. ADJ applies the layer's
// adjoint (the data gradient): channels transposed and taps flipped,
//   forward  out[o][p] = sum_{c,t} w[o][c][t] in[c][p + t - 1],
//   adjoint  out[c][p] = sum_{o,t} w[o][c][t] in[o][p - t + 1],
// with CIN / COUT the channels this call reads / writes. One thread per
// output value.
// ---------------------------------------------------------------------------
template <int CIN, int COUT, bool ADJ>
__global__ void __launch_bounds__(256) k_conv_f32(const float* __restrict__ in, float* __restrict__ out,
                                                  const float* __restrict__ w, int D, long cells) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cells * COUT) return;
  const int o = (int)(t % COUT);
  const long cell = t / COUT;
  const long D3 = (long)D * D * D;
  const long b = cell / D3, r = cell % D3;
  const int x = (int)(r % D), y = (int)((r / D) % D), z = (int)(r / ((long)D * D));
  float acc = 0.f;
  for (int tz = 0; tz < 3; ++tz)
    for (int ty = 0; ty < 3; ++ty)
      for (int tx = 0; tx < 3; ++tx) {
        const int dz = ADJ ? 1 - tz : tz - 1, dy = ADJ ? 1 - ty : ty - 1, dx = ADJ ? 1 - tx : tx - 1;
        const long src = b * D3 + ((long)wrap(z + dz, D) * D + wrap(y + dy, D)) * D + wrap(x + dx, D);
        const int tap = (tz * 3 + ty) * 3 + tx;
        for (int c = 0; c < CIN; ++c) {
          const float wv = ADJ ? w[(c * COUT + o) * 27 + tap] : w[(o * CIN + c) * 27 + tap];
          acc = fmaf(wv, in[src * CIN + c], acc);
        }
      }
  out[cell * COUT + o] = acc;
}

// ---------------------------------------------------------------------------
// Weight gradient on CUDA cores, FP32:
//   dW[o][c][tap] += sum_cells gz[cell][o] * a[cell + tap - 1][c]
// gz: COUT channels (f32 if COUT == 1 else bf16 x16); a: CIN channels (f32 if
// CIN == 1 else bf16 x16). One CTA per 8 x 16 x 4 tile; 4 x 4 register blocks.
// ---------------------------------------------------------------------------
template <int CIN, int COUT, bool F32 = false>
__global__ void __launch_bounds__(256) k_wgrad(const void* __restrict__ gz_, const void* __restrict__ a_, int NX,
                                               int NY, int NZ, float* __restrict__ dW) {
  constexpr int CP = CIN < 4 ? 4 : CIN, OP = COUT < 4 ? 4 : COUT;
  __shared__ __align__(16) float sa[HCELLS * CP];
  __shared__ __align__(16) float sg[TX * TY * ZT * OP];
  const int tiles_x = NX / TX, tiles_y = NY / TY, tiles_z = NZ / ZT;
  int t = blockIdx.x;
  const int bx = t % tiles_x; t /= tiles_x;
  const int by = t % tiles_y; t /= tiles_y;
  const int bz = t % tiles_z; t /= tiles_z;
  const int b = t;
  const int x0 = bx * TX, y0 = by * TY, z0 = bz * ZT;
  const size_t sbase = (size_t)b * NX * NY * NZ;
  for (int c = threadIdx.x; c < HCELLS; c += blockDim.x) {
    const int hx = c % HX, hy = (c / HX) % HY, hz = c / (HX * HY);
    const size_t cell = sbase + ((size_t)wrap(z0 - 1 + hz, NZ) * NY + wrap(y0 - 1 + hy, NY)) * NX + wrap(x0 - 1 + hx, NX);
    if (CIN == 1) {
      sa[c * CP] = reinterpret_cast<const float*>(a_)[cell];
      sa[c * CP + 1] = sa[c * CP + 2] = sa[c * CP + 3] = 0.f;
    } else if (F32) {
      const float* ap = reinterpret_cast<const float*>(a_) + 16 * cell;
      for (int i = 0; i < 16; ++i) sa[c * CP + i] = ap[i];
    } else {
      const __nv_bfloat16* ap = reinterpret_cast<const __nv_bfloat16*>(a_) + 16 * cell;
      for (int i = 0; i < 16; ++i) sa[c * CP + i] = __bfloat162float(ap[i]);
    }
  }
  for (int c = threadIdx.x; c < TX * TY * ZT; c += blockDim.x) {
    const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
    const size_t cell = sbase + ((size_t)(z0 + lz) * NY + (y0 + ly)) * NX + (x0 + lx);
    if (COUT == 1) {
      sg[c * OP] = reinterpret_cast<const float*>(gz_)[cell];
      sg[c * OP + 1] = sg[c * OP + 2] = sg[c * OP + 3] = 0.f;
    } else if (F32) {
      const float* gp = reinterpret_cast<const float*>(gz_) + 16 * cell;
      for (int i = 0; i < 16; ++i) sg[c * OP + i] = gp[i];
    } else {
      const __nv_bfloat16* gp = reinterpret_cast<const __nv_bfloat16*>(gz_) + 16 * cell;
      for (int i = 0; i < 16; ++i) sg[c * OP + i] = __bfloat162float(gp[i]);
    }
  }
  __syncthreads();
  constexpr int NOB = OP / 4, NCB = CP / 4, ITEMS = 27 * NOB * NCB;
  for (int it = threadIdx.x; it < ITEMS; it += blockDim.x) {
    const int tap = it / (NOB * NCB), ob = (it / NCB) % NOB, cb = it % NCB;
    const int tz = tap / 9, ty = (tap / 3) % 3, tx = tap % 3;
    float acc[4][4] = {};
    for (int c = 0; c < TX * TY * ZT; ++c) {
      const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
      const float4 g = *reinterpret_cast<const float4*>(&sg[c * OP + ob * 4]);
      const int hc = ((lz + tz) * HY + (ly + ty)) * HX + (lx + tx);
      const float4 a = *reinterpret_cast<const float4*>(&sa[hc * CP + cb * 4]);
      const float gv[4] = {g.x, g.y, g.z, g.w}, av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(gv[i], av[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int o = ob * 4 + i;
      if (o >= COUT) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cc = cb * 4 + j;
        if (cc >= CIN) continue;
        atomicAdd(&dW[(o * CIN + cc) * 27 + tap], acc[i][j]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Training loss per crop: energy norm plus residual norm of d = y - t,
//   L_b = E(d) / E(t) + |A_I d|^2 / |A_I t|^2,
// E(d) = sum over grid edges inside R4 (cells at least 4 from every face) of
// the squared difference across the edge, A_I d = 6 d_i - sum_nb d_j on R5
// (at least 5 from every face). Pass 1: q = A_I d, num_e[b] += E(d),
// num_r[b] += |q|^2. Pass 2: gy = (2 sum_{j in R4 nb of i} (d_i - d_j) / E(t)
// + 2 A_I^T q / |A_I t|^2) / B.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool in_interior(int x, int y, int z, int D, int border) {
  return x >= border && x < D - border && y >= border && y < D - border && z >= border && z < D - border;
}

// 6 v_i - sum of the 6 neighbours of i inside the crop (absent ones count 0).
__device__ __forceinline__ float crop_stencil(const float* v, int x, int y, int z, int D) {
  const size_t i = ((size_t)z * D + y) * D + x;
  float s = 6.f * v[i];
  if (x > 0) s -= v[i - 1];
  if (x < D - 1) s -= v[i + 1];
  if (y > 0) s -= v[i - D];
  if (y < D - 1) s -= v[i + D];
  if (z > 0) s -= v[i - (size_t)D * D];
  if (z < D - 1) s -= v[i + (size_t)D * D];
  return s;
}

__global__ void k_loss_q(const float* __restrict__ y, const float* __restrict__ tgt, int D, float* __restrict__ q,
                         double* num_e, double* num_r) {
  const size_t per = (size_t)D * D * D;
  const int b = blockIdx.y;
  const float* yb = y + (size_t)b * per;
  const float* tb = tgt + (size_t)b * per;
  double ae = 0.0, ar = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % D), yy = (int)((i / D) % D), z = (int)(i / ((size_t)D * D));
    float v = 0.f;
    if (in_interior(x, yy, z, D, 4)) {
      const float di = yb[i] - tb[i];
      // forward edges inside R4, each once
      if (in_interior(x + 1, yy, z, D, 4)) {
        const float dd = di - (yb[i + 1] - tb[i + 1]);
        ae += (double)dd * dd;
      }
      if (in_interior(x, yy + 1, z, D, 4)) {
        const float dd = di - (yb[i + D] - tb[i + D]);
        ae += (double)dd * dd;
      }
      if (in_interior(x, yy, z + 1, D, 4)) {
        const float dd = di - (yb[i + (size_t)D * D] - tb[i + (size_t)D * D]);
        ae += (double)dd * dd;
      }
      if (in_interior(x, yy, z, D, 5)) {
        float s = 6.f * di;
        s -= yb[i - 1] - tb[i - 1];
        s -= yb[i + 1] - tb[i + 1];
        s -= yb[i - D] - tb[i - D];
        s -= yb[i + D] - tb[i + D];
        s -= yb[i - (size_t)D * D] - tb[i - (size_t)D * D];
        s -= yb[i + (size_t)D * D] - tb[i + (size_t)D * D];
        v = s;
        ar += (double)v * v;
      }
    }
    q[(size_t)b * per + i] = v;
  }
  __shared__ double red[32];
  const double se = block_sum(ae, red);
  const double sr = block_sum(ar, red);
  if (threadIdx.x == 0) {
    atomicAdd(&num_e[b], se);
    atomicAdd(&num_r[b], sr);
  }
}

__global__ void k_loss_grad(const float* __restrict__ y, const float* __restrict__ tgt,
                            const float* __restrict__ q, int D, int B, const double* __restrict__ den_e,
                            const double* __restrict__ den_r, float* __restrict__ gy) {
  const size_t per = (size_t)D * D * D;
  const int b = blockIdx.y;
  const float* yb = y + (size_t)b * per;
  const float* tb = tgt + (size_t)b * per;
  const float fe = (float)(2.0 / (den_e[b] * B)), fr = (float)(2.0 / (den_r[b] * B));
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % D), yy = (int)((i / D) % D), z = (int)(i / ((size_t)D * D));
    float g = fr * crop_stencil(q + (size_t)b * per, x, yy, z, D);
    if (in_interior(x, yy, z, D, 4)) {
      const float di = yb[i] - tb[i];
      float gs = 0.f;
      const int ox[6] = {1, -1, 0, 0, 0, 0}, oy[6] = {0, 0, 1, -1, 0, 0}, oz[6] = {0, 0, 0, 0, 1, -1};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int xn = x + ox[k], yn = yy + oy[k], zn = z + oz[k];
        if (!in_interior(xn, yn, zn, D, 4)) continue;
        const size_t j = ((size_t)zn * D + yn) * D + xn;
        gs += di - (yb[j] - tb[j]);
      }
      g += fe * gs;
    }
    gy[(size_t)b * per + i] = g;
  }
}

// den_e[b] = E(t) over R4 edges, den_r[b] = |A_I t|^2 over R5.
__global__ void k_crops_den(const float* __restrict__ t, int D, double* den_e, double* den_r) {
  const size_t per = (size_t)D * D * D;
  const int b = blockIdx.y;
  const float* tb = t + (size_t)b * per;
  double ae = 0.0, ar = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % D), yy = (int)((i / D) % D), z = (int)(i / ((size_t)D * D));
    if (!in_interior(x, yy, z, D, 4)) continue;
    const float ti = tb[i];
    if (in_interior(x + 1, yy, z, D, 4)) {
      const float d = ti - tb[i + 1];
      ae += (double)d * d;
    }
    if (in_interior(x, yy + 1, z, D, 4)) {
      const float d = ti - tb[i + D];
      ae += (double)d * d;
    }
    if (in_interior(x, yy, z + 1, D, 4)) {
      const float d = ti - tb[i + (size_t)D * D];
      ae += (double)d * d;
    }
    if (in_interior(x, yy, z, D, 5)) {
      const float v = crop_stencil(tb, x, yy, z, D);
      ar += (double)v * v;
    }
  }
  __shared__ double red[32];
  const double se = block_sum(ae, red);
  const double sr = block_sum(ar, red);
  if (threadIdx.x == 0) {
    atomicAdd(&den_e[b], se);
    atomicAdd(&den_r[b], sr);
  }
}

// ---------------------------------------------------------------------------
// Crops at periodic origins, in FP32, of a residual field r and an error
// e = a - b (a = converged solution, b = CG iterate): pass 1 gathers and
// accumulates ss[b] = sum r^2 (whole crop); pass 2 scales x = r / s and
// t = e / (s h2) with s = RMS(r crop); k_crops_den then gives E(t) and |A_I t|^2.
// ---------------------------------------------------------------------------
__global__ void k_crops_gather_diff(const double* __restrict__ fr, const double* __restrict__ fa,
                                    const double* __restrict__ fb, int N, const int* __restrict__ origins, int D,
                                    float* __restrict__ xr, float* __restrict__ xe, double* ss) {
  const size_t per = (size_t)D * D * D;
  const int b = blockIdx.y;
  const int ox = origins[3 * b], oy = origins[3 * b + 1], oz = origins[3 * b + 2];
  double s1 = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % D), y = (int)((i / D) % D), z = (int)(i / ((size_t)D * D));
    const size_t src = ((size_t)((oz + z) % N) * N + (size_t)((oy + y) % N)) * N + (size_t)((ox + x) % N);
    const double rv = fr[src], ev = fa[src] - fb[src];
    xr[(size_t)b * per + i] = (float)rv;
    xe[(size_t)b * per + i] = (float)ev;
    s1 += rv * rv;
  }
  __shared__ double red[32];
  const double a = block_sum(s1, red);
  if (threadIdx.x == 0) atomicAdd(&ss[b], a);
}

__global__ void k_crops_scale(float* xr, float* xe, int D, double h2, const double* ss) {
  const size_t per = (size_t)D * D * D;
  const int b = blockIdx.y;
  const double s = sqrt(ss[b] / (double)per);
  const float ir = s > 0.0 ? (float)(1.0 / s) : 0.f;
  const float ie = s > 0.0 ? (float)(1.0 / (s * h2)) : 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    xr[(size_t)b * per + i] *= ir;
    xe[(size_t)b * per + i] *= ie;
  }
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba 2015) on the FP32 master weights; gradients are zeroed.
// ---------------------------------------------------------------------------
__global__ void k_adam(float* w, float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    w[i] -= lr * mh / (sqrtf(vh) + eps);
    g[i] = 0.f;
  }
}

}  // namespace cnn
}  // namespace pic
