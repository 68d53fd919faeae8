// Host-side choice of the plane-streaming geometry (slab height, raw stages,
// persistent grid) for a kernel built on stream_slab, on any N^3 grid.
#pragma once
#include "ctx.h"
#include "stream.cuh"

namespace pic {

// dynamic shared memory of one plane-streaming block: small blocks leave room
// for at least three (FP32) or two (FP64) blocks per SM, a tall block has the SM
constexpr size_t kSmemBudget32 = 72 * 1024;
constexpr size_t kSmemBudget64 = 110 * 1024;
constexpr size_t kSmemTall = 220 * 1024;
constexpr size_t kSmemMax = 226 * 1024;

// The tallest slab (largest divisor TY of N) whose block fits the thread cap
// and, with three raw stages and three plane buffers, the block's shared-memory
// budget: the halo rows re-read per plane are (TY + 2) / TY of the slab. If
// none fits the budget, the tallest that fits the SM. Then as many raw stages
// as the budget allows (at least three, at most kMaxStages). The persistent
// grid is the resident blocks of `kernel`, but at least `min_planes` planes
// per block. Sets the kernel's dynamic shared-memory limit to the size
// returned in *smem. budget_bytes (0: the defaults above) replaces the
// shared-memory budget of a small block.
template <typename TP, typename A, typename B, int NV, typename K>
int slab_geometry(pic_ctx* c, int N, K kernel, StreamGeo* out, size_t* smem, bool tall = false,
                  int min_planes = 4, size_t budget_bytes = 0) {
  if (N < 4 || N % 4) return PIC_EINVAL;
  const int cap = tall ? kStreamTall : kStreamSmall;
  const size_t budget = tall ? kSmemTall
                             : (budget_bytes ? budget_bytes : (sizeof(TP) == 8 ? kSmemBudget64 : kSmemBudget32));
  StreamGeo g{};
  bool found = false;
  for (int pass = 0; pass < 2 && !found; ++pass) {
    const size_t lim = pass == 0 ? budget : kSmemMax;
    for (int ty = N; ty >= 1 && !found; --ty) {
      if (N % ty || (long)N * ty / 4 > cap) continue;
      StreamGeo t = make_stream_geo(N, 3, ty);
      if (stream_smem_bytes<TP, A, B, NV>(t.rows, t.N, 3) <= lim) {
        g = t;
        found = true;
      }
    }
  }
  if (!found) return PIC_EINVAL;
  const StageLayout<A, B, NV> lay(g.rows, g.N);
  const size_t pb = 3 * (size_t)g.rows * g.N * sizeof(TP);
  int S = budget > pb ? (int)((budget - pb) / lay.bytes) : 0;
  if (S < 3) S = 3;
  if (S > kMaxStages) S = kMaxStages;
  g.S = S;
  *smem = stream_smem_bytes<TP, A, B, NV>(g.rows, g.N, S);
  CK(cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
  CK(cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                          (int)cudaSharedmemCarveoutMaxShared));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, round32(g.threads), *smem));
  if (per_sm < 1) return PIC_EINVAL;
  set_stream_blocks(g, per_sm * c->sms, min_planes);
  *out = g;
  return PIC_OK;
}

}  // namespace pic
