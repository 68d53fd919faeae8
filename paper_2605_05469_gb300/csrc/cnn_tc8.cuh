// The composed 9^3 preconditioner kernel on the tensor cores, 8-wide form.
//
// z = K * r (periodic), K the 9^3 composition of the linear network. For a
// fixed (dz, dy) the 9-tap x-sum of 8 consecutive outputs x0..x0+7 reads the
// 16 inputs x0-4..x0+11: a product with a 16 x 8 Toeplitz matrix
// T_{dz,dy}[k][n] = K[dz][dy][k - n] (0 <= k - n <= 8), dense enough that one
// K = 16 step of tcgen05.mma carries it (9 of every 16 products are taps,
// against 9 of 32 in the 16-wide form, which needs K = 32 for its 24 inputs).
// One MMA per (input plane, dy): M = 128 outputs in y (the TMEM lanes), A =
// the BF16 input plane's 136 x 16 (y x x) window shifted by dy rows, B = the
// nine T_{dz,dy} stacked along N. N = 72 is not a legal shape for M = 128
// (N must be a multiple of 16), so the stack carries a tenth, all-zero group
// in front: N = 80, and the zero group's columns receive A x 0 = 0.
//
// TMEM: 64 physical slots of 8 columns. Output planes (numbered by a
// CTA-local counter v) take ring slot s(v) = (-v) mod 55 and physical slot s + 1;
// an input plane's groups for outputs v_hi, v_hi - 1, ... occupy consecutive
// physical slots from s(v_hi) + 1, running on into the shadow slots 56..63
// (which alias ring slots 0..7; the epilogue adds both) instead of wrapping.
// The zero group lands on physical slot s(v_hi), the primary slot of output
// v_hi + 1 (not started, or beyond the CTA's range) or the unused slot 0.
// Runs of planes cut the group list at both ends; an odd count of groups is
// padded by the zero group in front when the list starts at dz = 0, and
// otherwise split into a [zero, dz_lo] pair from a separate B stack and the
// even remainder, so that no zero group ever touches the slot of an output
// whose epilogue may be reading it. The slot of the output v_hi + 1 is last
// used by output v_hi + 1 - 55, complete 46 input planes earlier: the issuer
// waits for that epilogue before it issues an input plane's MMAs.
//
// Opt-in (PIC_CNN_APPLY_TC8), not the default: the denser operand does not
// pay on GB300. Measured at 512^3 (phase timers per role): one thread issues
// a tcgen05.mma in ~80 cycles whatever N is (N = 16 .. 144 alike, N = 256
// ~93), so the 9 MMAs of an 8-wide plane cost about what the 18 of a
// 16-wide plane cost per output; its per-thread loads of twice as many
// planes per output add the rest (833 us against 470 us for the 16-wide form).
#pragma once
#include "cnn_kernels.cuh"

namespace pic {
namespace cnn {

namespace tc8 {
constexpr int BX = 8;                      // x outputs per column
constexpr int BY = 128;                    // y outputs per column (TMEM lanes)
constexpr int AROWS = BY + 8;              // input rows y0-4 .. y0+131
constexpr int CHUNK_B = AROWS * 16 + 64;   // one 8-input K chunk of a plane (2240)
constexpr int SLOT_B = 2 * CHUNK_B;        // one BF16 input plane, 16 x-inputs
constexpr int ASLOTS = 12;                 // input planes ready for the tensor cores
constexpr int MAIN_ROWS = 80;              // zero group + dz 0..8, 8 rows each
constexpr int MAIN_CHUNK_B = MAIN_ROWS * 16;
constexpr int MAIN_DY_B = 2 * MAIN_CHUNK_B;
constexpr int MAIN_B = 9 * MAIN_DY_B;      // 23040
constexpr int SOLO_ROWS = 16;              // zero group + one dz
constexpr int SOLO_CHUNK_B = SOLO_ROWS * 16;
constexpr int SOLO_DY_B = 2 * SOLO_CHUNK_B;
constexpr int SOLO_D_B = 9 * SOLO_DY_B;    // one dz (1..8), all dy
constexpr int SOLO_B = 8 * SOLO_D_B;       // 36864
constexpr int B_BYTES = MAIN_B + SOLO_B;   // 59904
constexpr int TSLOTS = 55;
constexpr int PSLOTS = 64;
constexpr int TMEM_COLS = PSLOTS * 8;      // 512: all of the SM's tensor memory
constexpr int SLOT_REUSE_LAG = TSLOTS - 9;
constexpr int ERING = 64;
constexpr int EPI_WARP0 = 1, PROD_WARP0 = 5, NWARPS = 13;
constexpr int THREADS = NWARPS * 32;       // 416
constexpr int PTHREADS = 256;
constexpr int LOADS = (AROWS * 4 + PTHREADS - 1) / PTHREADS;  // 16-byte pieces per producer per plane (3)
constexpr int AHEAD = 4;                   // input planes in producer registers
constexpr int TILE_OUT_B = BY * BX * 4;    // 4096: one output plane's 128 x 8 block
constexpr size_t SMEM = (size_t)B_BYTES + ASLOTS * SLOT_B + TILE_OUT_B;  // 117760
static_assert(SMEM > 114 * 1024 && SMEM <= 226 * 1024, "one CTA per SM (the kernel takes all 512 TMEM columns)");
static_assert(ERING > SLOT_REUSE_LAG, "the issuer must not lap the epilogue handshakes");
static_assert(TSLOTS + 9 == PSLOTS, "ring slots + zero/shadow slots fill the tensor memory");
static_assert(B_BYTES % 16 == 0 && (B_BYTES + ASLOTS * SLOT_B) % 16 == 0, "bulk copy and descriptor alignment");
}  // namespace tc8

// Packed B stacks (global, built when K changes). Main stack, for each dy: the
// canonical K-major 80 x 16 matrix with rows 0..7 zero and row 8 + 8 dz + n,
// column k holding T_{dz,dy}[k][n]. Solo stacks d = 1..8, for each dy: 16 x 16,
// rows 0..7 zero and rows 8..15 = T_{d,dy}.
__global__ void __launch_bounds__(256) k_pack_toeplitz8(const float* __restrict__ K, unsigned char* __restrict__ Bg) {
  using namespace tc8;
  constexpr int kMain = 9 * MAIN_ROWS * 16, kSolo = 8 * 9 * SOLO_ROWS * 16;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMain + kSolo; i += gridDim.x * blockDim.x) {
    int dz, dy, row, k, off;
    if (i < kMain) {
      dy = i / (MAIN_ROWS * 16);
      row = (i / 16) % MAIN_ROWS;
      k = i % 16;
      dz = row / 8 - 1;
      off = dy * MAIN_DY_B + (k >> 3) * MAIN_CHUNK_B + row * 16 + (k & 7) * 2;
    } else {
      const int j = i - kMain;
      const int d = j / (9 * SOLO_ROWS * 16) + 1;
      dy = (j / (SOLO_ROWS * 16)) % 9;
      row = (j / 16) % SOLO_ROWS;
      k = j % 16;
      dz = row < 8 ? -1 : d;
      off = MAIN_B + (d - 1) * SOLO_D_B + dy * SOLO_DY_B + (k >> 3) * SOLO_CHUNK_B + row * 16 + (k & 7) * 2;
    }
    const int dx = k - (row & 7);
    const float v = (dz >= 0 && dx >= 0 && dx <= 8) ? K[(dz * 9 + dy) * 9 + dx] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(Bg + off) = __float2bfloat16_rn(v);
  }
}

// Ring slot of the CTA's output plane number v (32-bit: a CTA holds a few
// thousand output planes; a 64-bit modulo on the issue path costs more than
// the MMAs it feeds).
__device__ __forceinline__ int tc8_ring_slot(int v) { return (tc8::TSLOTS - v % tc8::TSLOTS) % tc8::TSLOTS; }

__device__ __forceinline__ void tc8_origin(const TcPlane& P, int N, int& x0, int& y0) {
  const int nbx = N / tc8::BX;
  x0 = (P.col % nbx) * tc8::BX;
  y0 = (P.col / nbx) * tc8::BY;
}

// Nine MMAs of one B stack (one per dy): A shifted by dy rows, B advanced by
// one dy block; offsets are compile-time constants added to the descriptors.
template <int DY_B>
__device__ __forceinline__ void tc8_issue(uint64_t ad0, uint64_t b0, uint32_t d, uint32_t idesc) {
#pragma unroll
  for (int dy = 0; dy < 9; ++dy) mma_acc(d, ad0 + (uint64_t)dy, b0 + (uint64_t)((dy * DY_B) >> 4), idesc);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_zero8(uint32_t taddr) {
  const uint32_t z0 = 0u;
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr), "r"(z0)
               : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Producer thread t moves the 16-byte pieces t + 256 i (i < 3) of every input
// plane: x-inputs 4 g .. 4 g + 3 with g = t % 4 of rows t / 4 + 64 i.
struct Tc8Rows {
  int col;
  int off[tc8::LOADS];  // (gy * N + gx) of each piece; -1 past the last row
};

__device__ __forceinline__ void tc8_rows(const TcPlane& P, int N, int ptid, Tc8Rows& R) {
  using namespace tc8;
  int x0, y0;
  tc8_origin(P, N, x0, y0);
  R.col = P.col;
  // 4-float pieces never straddle the periodic wrap (x0 - 4 is a multiple of 4)
  const int gx = wrap(x0 - 4 + 4 * (ptid & 3), N);
#pragma unroll
  for (int i = 0; i < LOADS; ++i) {
    const int row = (ptid >> 2) + 64 * i;
    R.off[i] = row < AROWS ? wrap(y0 - 4 + row, N) * N + gx : -1;
  }
}

struct Tc8In {
  float4 r[tc8::LOADS];
};

__device__ __forceinline__ void tc8_load(const TcPlane& P, const float* __restrict__ r, int N, int ptid, Tc8Rows& R,
                                         Tc8In& in) {
  using namespace tc8;
  if (R.col != P.col) tc8_rows(P, N, ptid, R);
  const size_t plane = (size_t)wrap(P.z, N) * N * N;
#pragma unroll
  for (int i = 0; i < LOADS; ++i)
    if (R.off[i] >= 0) in.r[i] = __ldg(reinterpret_cast<const float4*>(r + plane + R.off[i]));
}

// Registers -> BF16 canonical K-major A operand: x-input k = 4 g .. 4 g + 3
// goes to K-chunk k / 8 at byte (k % 8) * 2 of its row.
__device__ __forceinline__ void tc8_store(const Tc8In& in, unsigned char* slot, int ptid) {
  using namespace tc8;
  const int g = ptid & 3;
  unsigned char* dst = slot + (g >> 1) * CHUNK_B + (ptid >> 2) * 16 + (g & 1) * 8;
#pragma unroll
  for (int i = 0; i < LOADS; ++i) {
    if ((ptid >> 2) + 64 * i < AROWS) {
      const float4 v = in.r[i];
      __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
      uint2 packed;
      packed.x = *reinterpret_cast<uint32_t*>(&lo);
      packed.y = *reinterpret_cast<uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(dst + i * 64 * 16) = packed;  // 64 rows further
    }
  }
}

// Float4 slot of (row, half) in the epilogue's transpose tile, XOR-swizzled:
// the row-per-thread writes and the coalesced reads are both conflict-free.
__device__ __forceinline__ int tc8_tile_idx(int row, int c) { return row * 2 + (c ^ ((row >> 2) & 1)); }

// Output plane p = P.z - 4 is complete once input plane P.z has been
// multiplied. Epilogue warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows y)
// and the slot's 8 columns (x), adds the shadow slot's partial sums, zeroes
// both, and the 128 epilogue threads write the 128 x 8 block two threads per
// 32-byte row segment.
__device__ __forceinline__ void tc8_epilogue(const TcCur& c, float* __restrict__ z, int N, uint32_t tmem,
                                             float4* tile) {
  using namespace tc8;
  const TcPlane& P = c.P;
  const int p = P.z - 4;
  if (p < P.pa) return;  // an input plane of the lower halo: no output completes (uniform)
  const int s = tc8_ring_slot(c.vbase + p - P.pa);
  const int et = threadIdx.x - EPI_WARP0 * 32;
  const int quarter = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
  const int row = quarter * 32 + lane;
  const uint32_t lanes = (uint32_t)(quarter * 32) << 16;
  float o[8];
  const uint32_t ta = tmem + lanes + (uint32_t)((s + 1) * 8);
  tmem_ld8(ta, o);
  tmem_zero8(ta);  // the slot's next output plane starts from zero
  if (s + TSLOTS + 1 < PSLOTS) {
    float o2[8];
    const uint32_t tb = tmem + lanes + (uint32_t)((s + TSLOTS + 1) * 8);
    tmem_ld8(tb, o2);
    tmem_zero8(tb);
#pragma unroll
    for (int i = 0; i < 8; ++i) o[i] += o2[i];
  }
  tc_epi_barrier();  // the previous plane's reads of the tile are done
  tile[tc8_tile_idx(row, 0)] = make_float4(o[0], o[1], o[2], o[3]);
  tile[tc8_tile_idx(row, 1)] = make_float4(o[4], o[5], o[6], o[7]);
  tc_epi_barrier();
  int x0, y0;
  tc8_origin(P, N, x0, y0);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int f = et + 128 * k;
    const int rr = f >> 1, c = f & 1;
    const size_t off = ((size_t)p * N + (size_t)(y0 + rr)) * N + x0 + 4 * c;
    *reinterpret_cast<float4*>(z + off) = tile[tc8_tile_idx(rr, c)];
  }
}

// z = K * r with the 8-wide Toeplitz form; persistent, one CTA per SM, in
// the work order of TcWork (whole columns round-robin). Warp 0 issues the MMAs,
// warps 1-4 drain finished output planes, warps 5-12 load and convert r.
// Every wait is bounded: on a timeout the kernel records DEV_ERR_TIMEOUT,
// every role leaves its loop, and the TMEM is freed.
__global__ void __launch_bounds__(tc8::THREADS, 1) k_apply_k_tc8(const float* __restrict__ r, float* __restrict__ z,
                                                                 int N, const unsigned char* __restrict__ Bg,
                                                                 int* err, const Scalars* sc) {
  using namespace tc8;
  if (sc && sc->done) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ __align__(8) uint64_t a_full[ASLOTS], a_empty[ASLOTS], acc_full[ERING], acc_empty[ERING], b_bar;
  unsigned char* Bs = smem;                                           // B_BYTES
  unsigned char* slots = smem + B_BYTES;                              // ASLOTS x SLOT_B
  float4* tile = reinterpret_cast<float4*>(slots + ASLOTS * SLOT_B);  // TILE_OUT_B
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
    // barrier word serialise and cost more than a plane's MMAs)
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
      const uint64_t bmain = smem_desc(smem_u32(Bs), MAIN_CHUNK_B, 128);
      const uint64_t bsolo = smem_desc(smem_u32(Bs + MAIN_B), SOLO_CHUNK_B, 128);
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
        const int ng = dz_hi - dz_lo + 1;
        const int v_hi = c.vbase + (P.z + 4 - dz_lo - P.pa);
        const uint32_t d_lo = tmem + (uint32_t)((tc8_ring_slot(v_hi) + 1) * 8);  // group dz_lo's columns
        const uint64_t ad0 = smem_desc(smem_u32(slots + sa * SLOT_B), CHUNK_B, 128);
        if (!(ng & 1)) {
          tc8_issue<MAIN_DY_B>(ad0, bmain + (uint64_t)(((dz_lo + 1) * 128) >> 4), d_lo, idesc_n(8 * ng));
        } else if (dz_lo == 0) {
          tc8_issue<MAIN_DY_B>(ad0, bmain, d_lo - 8u, idesc_n(8 * ng + 8));
        } else {
          tc8_issue<SOLO_DY_B>(ad0, bsolo + (uint64_t)(((dz_lo - 1) * SOLO_D_B) >> 4), d_lo - 8u, idesc_n(16));
          if (ng > 1)
            tc8_issue<MAIN_DY_B>(ad0, bmain + (uint64_t)(((dz_lo + 2) * 128) >> 4), d_lo + 8u, idesc_n(8 * ng - 8));
        }
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
    for (uint32_t j = 0; have; ++j) {
      // warp-uniform: a lane that gave up takes its whole warp out
      if (!__all_sync(0xffffffffu, tc_wait(&acc_full[j % ERING], (j / ERING) & 1u, err, &abort_flag))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      tc8_epilogue(c, z, N, tmem, tile);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[j % ERING]);
      have = tc_next(W, c);
    }
  } else {
    // ---- producers: 256 threads, AHEAD planes in registers ahead of conversion ----
    const int ptid = tid - PROD_WARP0 * 32;
    Tc8Rows rows;
    rows.col = -1;
    Tc8In in[AHEAD];
    TcCur cur, ahead;
    bool go = tc_start(W, cur);
    ahead = cur;
    bool have_a = go;
#pragma unroll
    for (int k = 0; k < AHEAD; ++k) {
      if (have_a) {
        tc8_load(ahead.P, r, N, ptid, rows, in[k]);
        have_a = tc_next(W, ahead);
      }
    }
    uint32_t j = 0;
    // plane j from buffer in[j % AHEAD], which is then refilled with plane j + AHEAD
    while (go) {
#pragma unroll
      for (int k = 0; k < AHEAD; ++k) {
        if (go) {
          const uint32_t sa = j % ASLOTS;
          bool ok = true;
          if (j >= (uint32_t)ASLOTS) {
            // the MMAs of plane j - ASLOTS, which read this A slot, are done
            const uint32_t kk = j - ASLOTS;
            ok = tc_wait(&a_empty[sa], (kk / ASLOTS) & 1u, err, &abort_flag);
          }
          if (!__all_sync(0xffffffffu, ok)) {  // warp-uniform
            go = false;
          } else {
            tc8_store(in[k], slots + sa * SLOT_B, ptid);
            fence_proxy_async_smem();  // the BF16 writes, visible to the tensor cores
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_full[sa]);
            if (have_a) {
              tc8_load(ahead.P, r, N, ptid, rows, in[k]);
              have_a = tc_next(W, ahead);
            }
            ++j;
            go = tc_next(W, cur);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace cnn
}  // namespace pic
