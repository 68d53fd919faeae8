// Learned preconditioner: weights, training primitives and inference behind
// the C ABI (include/pic.h). The network and its kernels are described in
// cnn_kernels.cuh; this file owns the buffers and sequences the launches.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "cnn.h"
#include "cnn_kernels.cuh"
#include "cnn_tc8.cuh"
#include "ctx.h"

namespace pic {

struct CnnState {
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, grads, Adam moments
  unsigned char* packed = nullptr;                                // canonical BF16 tiles
  bool has_weights = false;
  int adam_t = 0;
  // training: activations of the last forward (B x D^3 cells)
  size_t train_cells = 0;
  __nv_bfloat16 *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *ga = nullptr, *gb = nullptr;
  // the FP32 test mode of the training convs (PIC_CNN_TRAIN_FP32)
  int train_prec = 0;
  size_t f32_cells = 0;
  float *f1 = nullptr, *f2 = nullptr, *f3 = nullptr, *fa = nullptr, *fb = nullptr;
  const float* last_x = nullptr;
  int last_B = 0, last_D = 0;
  // inference ping-pong activations at N^3
  size_t inf_cells = 0;
  __nv_bfloat16 *i1 = nullptr, *i2 = nullptr;
  // crops / loss scratch
  int bmax = 0;
  double* sums = nullptr;  // [5 * bmax]: ss, den_e, den_r, num_e, num_r
  int* origins = nullptr;  // [3 * bmax]
  double* sums_host = nullptr;
  float* q = nullptr;      // loss: A_I (y - t)
  size_t q_cells = 0;
  float* K = nullptr;      // composed 9^3 kernel of N = G^T G (FP32)
  unsigned char* Bt = nullptr;  // its 81 Toeplitz matrices, packed BF16 B operand (16-wide form)
  unsigned char* Bt8 = nullptr; // the 8-wide form's zero-led B stacks
  cnn::K729 K_host;        // its host copy (launch parameter)
  bool K_stale = true;     // the device kernel changed since the host copy
};

}  // namespace pic

using namespace pic;
using namespace pic::cnn;

namespace {


int ensure_state(pic_ctx* c) {
  if (c->cnn) return PIC_OK;
  CnnState* s = new (std::nothrow) CnnState();
  if (!s) return PIC_ENOMEM;
  int e;
  if ((e = dalloc(&s->w, kWeights)) || (e = dalloc(&s->g, kWeights)) || (e = dalloc(&s->m, kWeights)) ||
      (e = dalloc(&s->v, kWeights)) || (e = dalloc(&s->packed, (size_t)kPackBytes)) || (e = dalloc(&s->K, 729)) ||
      (e = dalloc(&s->Bt, (size_t)tck::B_BYTES)) || (e = dalloc(&s->Bt8, (size_t)tc8::B_BYTES))) {
    cnn_state_free(s);
    return e;
  }
  if (cudaMemset(s->g, 0, kWeights * 4) != cudaSuccess || cudaMemset(s->m, 0, kWeights * 4) != cudaSuccess ||
      cudaMemset(s->v, 0, kWeights * 4) != cudaSuccess) {
    cnn_state_free(s);
    return PIC_ECUDA;
  }
  c->cnn = s;
  return PIC_OK;
}

int ensure_train(pic_ctx* c, size_t cells) {
  CnnState* s = c->cnn;
  if (s->train_cells >= cells) return PIC_OK;
  dfree(s->a1); dfree(s->a2); dfree(s->a3); dfree(s->ga); dfree(s->gb);
  s->train_cells = 0;
  int e;
  if ((e = dalloc(&s->a1, 16 * cells)) || (e = dalloc(&s->a2, 16 * cells)) || (e = dalloc(&s->a3, 16 * cells)) ||
      (e = dalloc(&s->ga, 16 * cells)) || (e = dalloc(&s->gb, 16 * cells)))
    return e;
  s->train_cells = cells;
  return PIC_OK;
}

int ensure_train_f32(pic_ctx* c, size_t cells) {
  CnnState* s = c->cnn;
  if (s->f32_cells >= cells) return PIC_OK;
  dfree(s->f1); dfree(s->f2); dfree(s->f3); dfree(s->fa); dfree(s->fb);
  s->f32_cells = 0;
  int e;
  if ((e = dalloc(&s->f1, 16 * cells)) || (e = dalloc(&s->f2, 16 * cells)) || (e = dalloc(&s->f3, 16 * cells)) ||
      (e = dalloc(&s->fa, 16 * cells)) || (e = dalloc(&s->fb, 16 * cells)))
    return e;
  s->f32_cells = cells;
  return PIC_OK;
}

template <int CIN, int COUT, bool ADJ>
int conv_f32(pic_ctx* c, const float* in, float* out, int layer, int D, int B) {
  const long cells = (long)B * D * D * D;
  launch(c, k_conv_f32<CIN, COUT, ADJ>, (unsigned)((cells * COUT + 255) / 256), 256, 0, in, out,
         (const float*)(c->cnn->w + kLayerOff[layer]), D, cells);
  CK(cudaGetLastError());
  return PIC_OK;
}

int ensure_batch(pic_ctx* c, int B) {
  CnnState* s = c->cnn;
  if (s->bmax >= B) return PIC_OK;
  dfree(s->sums); dfree(s->origins);
  if (s->sums_host) cudaFreeHost(s->sums_host);
  s->sums_host = nullptr;
  s->bmax = 0;
  int e;
  if ((e = dalloc(&s->sums, 5 * (size_t)B)) || (e = dalloc(&s->origins, 3 * (size_t)B))) return e;
  if (cudaMallocHost(&s->sums_host, 5 * (size_t)B * sizeof(double)) != cudaSuccess) return PIC_ENOMEM;
  s->bmax = B;
  return PIC_OK;
}

bool dims_ok(int NX, int NY, int NZ) {
  return NX >= TX && NY >= TY && NZ >= ZT && NX % TX == 0 && NY % TY == 0 && NZ % ZT == 0;
}

template <int CIN>
int conv(pic_ctx* c, const void* in, void* out, const unsigned char* w, int mode, int NX, int NY, int NZ, int B,
         const double* in_src = nullptr, double in_mul = 0.0, int in_mode = SCALE_ONE,
         const double* out_src = nullptr, double out_mul = 0.0, int out_mode = SCALE_ONE) {
  static bool configured = false;
  const size_t smem = conv_smem_bytes<CIN>();
  if (!configured) {
    CK(cudaFuncSetAttribute((const void*)k_conv_tc<CIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  ConvParams P;
  P.NX = NX; P.NY = NY; P.NZ = NZ; P.B = B;
  P.in = in; P.out = out; P.w = w;
  P.in_scale_src = in_src; P.in_scale_mul = in_mul; P.in_scale_mode = in_mode;
  P.out_scale_src = out_src; P.out_scale_mul = out_mul; P.out_scale_mode = out_mode;
  P.err = c->err;
  const long tiles = (long)(NX / TX) * (NY / TY) * (NZ / ZT) * B;
  launch(c, k_conv_tc<CIN>, (unsigned)tiles, kThreads, smem, P, mode);
  CK(cudaGetLastError());
  return PIC_OK;
}

template <int CIN, int COUT, bool F32 = false>
int wgrad(pic_ctx* c, const void* gz, const void* a, int D, int B, float* dW) {
  const long tiles = (long)(D / TX) * (D / TY) * (D / ZT) * B;
  launch(c, k_wgrad<CIN, COUT, F32>, (unsigned)tiles, 256, 0, gz, a, D, D, D, dW);
  CK(cudaGetLastError());
  return PIC_OK;
}

int repack(pic_ctx* c) {
  launch(c, k_tie_weights, 27, 256, 0, c->cnn->w);
  launch(c, k_pack_weights, 32, 256, 0, (const float*)c->cnn->w, c->cnn->packed);
  launch(c, k_compose, 1, 256, 0, (const float*)c->cnn->w, c->cnn->K);
  launch(c, k_pack_toeplitz, 41, 256, 0, (const float*)c->cnn->K, c->cnn->Bt);
  launch(c, k_pack_toeplitz8, 117, 256, 0, (const float*)c->cnn->K, c->cnn->Bt8);
  c->cnn->K_stale = true;
  CK(cudaGetLastError());
  return PIC_OK;
}

}  // namespace

namespace pic {

void cnn_state_free(CnnState* s) {
  if (!s) return;
  dfree(s->w); dfree(s->g); dfree(s->m); dfree(s->v); dfree(s->packed); dfree(s->K); dfree(s->Bt); dfree(s->Bt8);
  dfree(s->a1); dfree(s->a2); dfree(s->a3); dfree(s->ga); dfree(s->gb);
  dfree(s->f1); dfree(s->f2); dfree(s->f3); dfree(s->fa); dfree(s->fb);
  dfree(s->i1); dfree(s->i2);
  dfree(s->sums); dfree(s->origins); dfree(s->q);
  if (s->sums_host) cudaFreeHost(s->sums_host);
  delete s;
}

bool cnn_ready(const pic_ctx* c) { return c->cnn && c->cnn->has_weights; }

bool cnn_tc_ok(const pic_ctx* c) {
  return c->N % tck::BY == 0 && (c->cnn_apply_mode == PIC_CNN_APPLY_TC || c->cnn_apply_mode == PIC_CNN_APPLY_TC_FUSED ||
                                 c->cnn_apply_mode == PIC_CNN_APPLY_TC8);
}

bool cnn_fused_ok(const pic_ctx* c) { return c->N % tck::BY == 0 && c->cnn_apply_mode == PIC_CNN_APPLY_TC_FUSED; }

// The composed kernel on the tensor cores, persistent: one CTA per SM, each a
// contiguous range of output planes.
template <bool FUSED>
int launch_tc(pic_ctx* c, const float* r, float* z, const TcFcg& F) {
  static bool configured = false;
  if (!configured) {
    CK(cudaFuncSetAttribute((const void*)k_apply_k_tc<FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)tck::smem_bytes<FUSED>()));
    configured = true;
  }
  const int N = c->N;
  const long units = (long)(N / tck::BX) * (N / tck::BY) * N;
  const unsigned grid = (unsigned)(units < c->sms ? units : c->sms);
  launch(c, k_apply_k_tc<FUSED>, grid, tck::THREADS, tck::smem_bytes<FUSED>(), r, z, N,
         (const unsigned char*)c->cnn->Bt, c->err, F);
  CK(cudaGetLastError());
  return PIC_OK;
}

// The 8-wide composed kernel (opt-in, PIC_CNN_APPLY_TC8), persistent like the
// 16-wide one. With `stop` (the solver's scalars) it returns at once once the
// solve has finished, like the solver's other kernels.
int launch_tc8(pic_ctx* c, const float* r, float* z, const Scalars* stop) {
  static bool configured = false;
  if (!configured) {
    CK(cudaFuncSetAttribute((const void*)k_apply_k_tc8, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)tc8::SMEM));
    configured = true;
  }
  const int N = c->N;
  const long units = (long)(N / tc8::BX) * (N / tc8::BY) * N;
  const unsigned grid = (unsigned)(units < c->sms ? units : c->sms);
  launch(c, k_apply_k_tc8, grid, tc8::THREADS, tc8::SMEM, r, z, N, (const unsigned char*)c->cnn->Bt8, c->err, stop);
  CK(cudaGetLastError());
  return PIC_OK;
}

int cnn_apply_fused(pic_ctx* c, const float* r, float* r_new, float* z, const float* q, const float* p, float* x) {
  if (!cnn_fused_ok(c)) return PIC_EINVAL;
  TcFcg F{q, p, x, r_new, c->sc, c->partials, c->counter, 0};
  return launch_tc<true>(c, r, z, F);
}

int cnn_apply_redo(pic_ctx* c, const float* r, float* z) {
  if (!cnn_tc_ok(c)) return PIC_EINVAL;
  TcFcg F{};
  F.sc = c->sc;
  F.only_redo = 1;
  return launch_tc<false>(c, r, z, F);
}

int cnn_apply(pic_ctx* c, const float* r, float* z, const double* rr, size_t n) {
  CnnState* s = c->cnn;
  const int N = c->N;
  // linear network: z = s N(r / s) = N r, one composed 9^3 convolution
  if (cnn_tc_ok(c)) {
    // inside a solve (rr given) the kernel skips its work once the solve is done
    const Scalars* stop = rr ? c->sc : nullptr;
    if (c->cnn_apply_mode == PIC_CNN_APPLY_TC8) return launch_tc8(c, r, z, stop);
    TcFcg F{};
    F.sc = const_cast<Scalars*>(stop);
    return launch_tc<false>(c, r, z, F);
  }
  // grids that are not a multiple of 128 run the FP32 composed kernel in TC mode
  if (N % KX == 0 && c->cnn_apply_mode != PIC_CNN_APPLY_LAYERS) {
    static bool configured = false;
    if (!configured) {
      CK(cudaFuncSetAttribute((const void*)k_apply_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApplySmem));
      configured = true;
    }
    if (s->K_stale) {
      CK(cudaMemcpyAsync(s->K_host.k, s->K, sizeof(s->K_host.k), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      s->K_stale = false;
    }
    const unsigned blocks = (unsigned)((N / KX) * (N / KY) * (N / KZ));
    launch(c, k_apply_k, blocks, KX * KY, kApplySmem, r, z, N, s->K_host);
    CK(cudaGetLastError());
    return PIC_OK;
  }
  if (!dims_ok(N, N, N)) return PIC_EINVAL;
  if (s->inf_cells < n) {
    dfree(s->i1); dfree(s->i2);
    s->inf_cells = 0;
    int e;
    if ((e = dalloc(&s->i1, 16 * n)) || (e = dalloc(&s->i2, 16 * n))) return e;
    s->inf_cells = n;
  }
  const double inv_n = 1.0 / (double)n;
  int e;
  // z = s N(r / s), s = RMS(r) = sqrt(rr / n)
  if ((e = conv<1>(c, r, s->i1, s->packed + kPackFwd1, OUT_BF16, N, N, N, 1, rr, inv_n, SCALE_RSQRT))) return e;
  if ((e = conv<16>(c, s->i1, s->i2, s->packed + kPackFwd2, OUT_BF16, N, N, N, 1))) return e;
  if ((e = conv<16>(c, s->i2, s->i1, s->packed + kPackFwd3, OUT_BF16, N, N, N, 1))) return e;
  return conv<16>(c, s->i1, z, s->packed + kPackFwd4, OUT_SCALED_F32, N, N, N, 1, nullptr, 0.0, SCALE_ONE, rr,
                  inv_n, SCALE_SQRT);
}

int cnn_state_get(pic_ctx* c, float* dev3, int* adam_t) {
  if (!cnn_ready(c)) return PIC_ESTATE;
  CnnState* s = c->cnn;
  CK(cudaMemcpyAsync(dev3, s->w, kWeights * 4, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(dev3 + kWeights, s->m, kWeights * 4, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(dev3 + 2 * kWeights, s->v, kWeights * 4, cudaMemcpyDeviceToDevice, c->stream));
  *adam_t = s->adam_t;
  return PIC_OK;
}

int cnn_state_set(pic_ctx* c, const float* dev3, int adam_t) {
  int e;
  if ((e = ensure_state(c))) return e;
  CnnState* s = c->cnn;
  CK(cudaMemcpyAsync(s->w, dev3, kWeights * 4, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(s->m, dev3 + kWeights, kWeights * 4, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(s->v, dev3 + 2 * kWeights, kWeights * 4, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemsetAsync(s->g, 0, kWeights * 4, c->stream));
  s->adam_t = adam_t;
  if ((e = repack(c))) return e;
  s->has_weights = true;
  return PIC_OK;
}

}  // namespace pic

namespace {

// Weights file: a 32-byte header (magic, format version, weight count, Adam
// step count, FNV-1a 64-bit hash of the payload) and the payload: the FP32
// master weights, then Adam's m and v, PIC_CNN_WEIGHTS floats each,
// little-endian.
constexpr char kFileMagic[8] = {'P', 'I', 'C', 'C', 'N', 'N', '1', '\n'};
constexpr uint32_t kFileVersion = 1;

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t count;
  int64_t adam_t;
  uint64_t hash;
};
static_assert(sizeof(FileHeader) == 32, "weights file header");

uint64_t fnv1a64(const unsigned char* p, size_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

}  // namespace

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

int pic_cnn_set_weights(pic_ctx* c, const float* w_host) {
  if (!c || !w_host) return PIC_EINVAL;
  int e;
  if ((e = ensure_state(c))) return e;
  CK(cudaMemcpyAsync(c->cnn->w, w_host, kWeights * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->cnn->g, 0, kWeights * 4, c->stream));
  CK(cudaMemsetAsync(c->cnn->m, 0, kWeights * 4, c->stream));
  CK(cudaMemsetAsync(c->cnn->v, 0, kWeights * 4, c->stream));
  c->cnn->adam_t = 0;
  if ((e = repack(c))) return e;
  CK(cudaStreamSynchronize(c->stream));
  c->cnn->has_weights = true;
  return PIC_OK;
}

int pic_cnn_get_weights(pic_ctx* c, float* w_host) {
  if (!c || !w_host) return PIC_EINVAL;
  if (!cnn_ready(c)) return PIC_ESTATE;
  CK(cudaMemcpyAsync(w_host, c->cnn->w, kWeights * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

int pic_cnn_get_grads(pic_ctx* c, float* g_host) {
  if (!c || !g_host) return PIC_EINVAL;
  if (!cnn_ready(c)) return PIC_ESTATE;
  CK(cudaMemcpyAsync(g_host, c->cnn->g, kWeights * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

int pic_cnn_conv_raw(pic_ctx* c, int which, const void* in, float* out, int B, int D) {
  if (!c || !in || !out || B < 1 || which < 0 || which > 6) return PIC_EINVAL;
  if (!dims_ok(D, D, D)) return PIC_EINVAL;
  if (!cnn_ready(c)) return PIC_ESTATE;
  static const int offs[7] = {kPackFwd1, kPackFwd2, kPackFwd3, kPackFwd4, kPackBwd4, kPackBwd3, kPackBwd2};
  const unsigned char* w = c->cnn->packed + offs[which];
  if (which == 0 || which == 4) return conv<1>(c, in, out, w, OUT_RAW_F32, D, D, D, B);
  return conv<16>(c, in, out, w, OUT_RAW_F32, D, D, D, B);
}

int pic_cnn_apply(pic_ctx* c, const float* r, float* z) {
  if (!c || !r || !z) return PIC_EINVAL;
  if (!c->has_grid) return PIC_ESTATE;
  if (!cnn_ready(c)) return PIC_ESTATE;
  return cnn_apply(c, r, z, nullptr, c->n);
}

int pic_cnn_set_apply(pic_ctx* c, int mode) {
  if (!c || mode < PIC_CNN_APPLY_TC || mode > PIC_CNN_APPLY_TC8) return PIC_EINVAL;
  c->cnn_apply_mode = mode;
  return PIC_OK;
}

int pic_cnn_forward(pic_ctx* c, const float* x, float* y, int B, int D) {
  if (!c || !x || !y || B < 1) return PIC_EINVAL;
  if (!dims_ok(D, D, D)) return PIC_EINVAL;
  if (!cnn_ready(c)) return PIC_ESTATE;
  CnnState* s = c->cnn;
  const size_t cells = (size_t)B * D * D * D;
  int e;
  if (s->train_prec == PIC_CNN_TRAIN_FP32) {
    if ((e = ensure_train_f32(c, cells))) return e;
    if ((e = conv_f32<1, 16, false>(c, x, s->f1, 0, D, B))) return e;
    if ((e = conv_f32<16, 16, false>(c, s->f1, s->f2, 1, D, B))) return e;
    if ((e = conv_f32<16, 16, false>(c, s->f2, s->f3, 2, D, B))) return e;
    if ((e = conv_f32<16, 1, false>(c, s->f3, y, 3, D, B))) return e;
    s->last_x = x;
    s->last_B = B;
    s->last_D = D;
    return PIC_OK;
  }
  if ((e = ensure_train(c, cells))) return e;
  if ((e = conv<1>(c, x, s->a1, s->packed + kPackFwd1, OUT_BF16, D, D, D, B))) return e;
  if ((e = conv<16>(c, s->a1, s->a2, s->packed + kPackFwd2, OUT_BF16, D, D, D, B))) return e;
  if ((e = conv<16>(c, s->a2, s->a3, s->packed + kPackFwd3, OUT_BF16, D, D, D, B))) return e;
  if ((e = conv<16>(c, s->a3, y, s->packed + kPackFwd4, OUT_SCALED_F32, D, D, D, B))) return e;
  s->last_x = x;
  s->last_B = B;
  s->last_D = D;
  return PIC_OK;
}

int pic_cnn_backward(pic_ctx* c, const float* gy, int B, int D) {
  if (!c || !gy) return PIC_EINVAL;
  if (!cnn_ready(c)) return PIC_ESTATE;
  CnnState* s = c->cnn;
  if (B != s->last_B || D != s->last_D || !s->last_x) return PIC_ESTATE;
  float* g4 = s->g + kLayerOff[3];
  float* g3 = s->g + kLayerOff[2];
  float* g2 = s->g + kLayerOff[1];
  float* g1 = s->g + kLayerOff[0];
  int e;
  // the activations are the identity, so each data gradient is the adjoint
  // conv of the layer's own gradient; weight gradients per layer, then tied
  if (s->train_prec == PIC_CNN_TRAIN_FP32) {
    if (s->f32_cells < (size_t)B * D * D * D) return PIC_ESTATE;
    if ((e = wgrad<16, 1, true>(c, gy, s->f3, D, B, g4))) return e;
    if ((e = conv_f32<1, 16, true>(c, gy, s->fa, 3, D, B))) return e;
    if ((e = wgrad<16, 16, true>(c, s->fa, s->f2, D, B, g3))) return e;
    if ((e = conv_f32<16, 16, true>(c, s->fa, s->fb, 2, D, B))) return e;
    if ((e = wgrad<16, 16, true>(c, s->fb, s->f1, D, B, g2))) return e;
    if ((e = conv_f32<16, 16, true>(c, s->fb, s->fa, 1, D, B))) return e;
    if ((e = wgrad<1, 16, true>(c, s->fa, s->last_x, D, B, g1))) return e;
    launch(c, k_tie_grads, 27, 256, 0, s->g);
    CK(cudaGetLastError());
    return PIC_OK;
  }
  if ((e = wgrad<16, 1>(c, gy, s->a3, D, B, g4))) return e;
  if ((e = conv<1>(c, gy, s->ga, s->packed + kPackBwd4, OUT_BF16, D, D, D, B))) return e;
  if ((e = wgrad<16, 16>(c, s->ga, s->a2, D, B, g3))) return e;
  if ((e = conv<16>(c, s->ga, s->gb, s->packed + kPackBwd3, OUT_BF16, D, D, D, B))) return e;
  if ((e = wgrad<16, 16>(c, s->gb, s->a1, D, B, g2))) return e;
  if ((e = conv<16>(c, s->gb, s->ga, s->packed + kPackBwd2, OUT_BF16, D, D, D, B))) return e;
  if ((e = wgrad<1, 16>(c, s->ga, s->last_x, D, B, g1))) return e;
  launch(c, k_tie_grads, 27, 256, 0, s->g);
  CK(cudaGetLastError());
  return PIC_OK;
}

int pic_cnn_save(pic_ctx* c, const char* path) {
  if (!c || !path) return PIC_EINVAL;
  if (!cnn_ready(c)) return PIC_ESTATE;
  CnnState* s = c->cnn;
  float* host = static_cast<float*>(malloc(3 * kWeights * sizeof(float)));
  if (!host) return PIC_ENOMEM;
  cudaError_t ce = cudaMemcpyAsync(host, s->w, kWeights * 4, cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(host + kWeights, s->m, kWeights * 4, cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(host + 2 * kWeights, s->v, kWeights * 4, cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  if (ce != cudaSuccess) {
    free(host);
    return PIC_ECUDA;
  }
  FileHeader hd;
  memcpy(hd.magic, kFileMagic, 8);
  hd.version = kFileVersion;
  hd.count = kWeights;
  hd.adam_t = s->adam_t;
  hd.hash = fnv1a64(reinterpret_cast<const unsigned char*>(host), 3 * kWeights * sizeof(float));
  FILE* f = fopen(path, "wb");
  int rc = PIC_OK;
  if (!f) {
    rc = PIC_EINVAL;
  } else {
    if (fwrite(&hd, sizeof(hd), 1, f) != 1 || fwrite(host, sizeof(float), 3 * kWeights, f) != 3 * (size_t)kWeights)
      rc = PIC_EINVAL;
    if (fclose(f) != 0) rc = PIC_EINVAL;
  }
  free(host);
  return rc;
}

int pic_cnn_load(pic_ctx* c, const char* path) {
  if (!c || !path) return PIC_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return PIC_EINVAL;
  FileHeader hd;
  float* host = static_cast<float*>(malloc(3 * kWeights * sizeof(float)));
  int rc = PIC_OK;
  if (!host) {
    rc = PIC_ENOMEM;
  } else if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, kFileMagic, 8) != 0 ||
             hd.version != kFileVersion || hd.count != (uint32_t)kWeights || hd.adam_t < 0 ||
             hd.adam_t > 0x7fffffff || fread(host, sizeof(float), 3 * kWeights, f) != 3 * (size_t)kWeights ||
             fnv1a64(reinterpret_cast<const unsigned char*>(host), 3 * kWeights * sizeof(float)) != hd.hash) {
    rc = PIC_EINVAL;
  }
  fclose(f);
  if (rc != PIC_OK) {
    free(host);
    return rc;
  }
  int e;
  if ((e = ensure_state(c))) {
    free(host);
    return e;
  }
  CnnState* s = c->cnn;
  cudaError_t ce = cudaMemcpyAsync(s->w, host, kWeights * 4, cudaMemcpyHostToDevice, c->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->m, host + kWeights, kWeights * 4, cudaMemcpyHostToDevice, c->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(s->v, host + 2 * kWeights, kWeights * 4, cudaMemcpyHostToDevice, c->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(s->g, 0, kWeights * 4, c->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);  // the host buffer is freed next
  free(host);
  if (ce != cudaSuccess) return PIC_ECUDA;
  s->adam_t = (int)hd.adam_t;
  if ((e = repack(c))) return e;
  CK(cudaStreamSynchronize(c->stream));
  s->has_weights = true;
  return PIC_OK;
}

int pic_cnn_set_train_precision(pic_ctx* c, int mode) {
  if (!c || (mode != PIC_CNN_TRAIN_BF16 && mode != PIC_CNN_TRAIN_FP32)) return PIC_EINVAL;
  int e;
  if ((e = ensure_state(c))) return e;
  c->cnn->train_prec = mode;
  c->cnn->last_x = nullptr;  // a backward pass needs a forward pass in the same mode
  return PIC_OK;
}

int pic_cnn_make_batch(pic_ctx* c, const double* r, const double* a, const double* b, const int* origins_host,
                       int B, int D, float* x, float* t, double h2) {
  if (!c || !r || !a || !b || !origins_host || !x || !t || B < 1 || D < 16 || D % 16 != 0) return PIC_EINVAL;
  if (!c->has_grid) return PIC_ESTATE;
  int e;
  if ((e = ensure_state(c)) || (e = ensure_batch(c, B))) return e;
  for (int i = 0; i < 3 * B; ++i)
    if (origins_host[i] < 0 || origins_host[i] >= c->N) return PIC_EINVAL;
  CnnState* s = c->cnn;
  CK(cudaMemcpyAsync(s->origins, origins_host, 3 * (size_t)B * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));  // origins_host may be reused by the caller
  CK(cudaMemsetAsync(s->sums, 0, 5 * (size_t)B * sizeof(double), c->stream));
  dim3 grid(64, B);
  // e = a - b: the crop kernel reads the error as the difference of two fields
  k_crops_gather_diff<<<grid, 256, 0, c->stream>>>(r, a, b, c->N, s->origins, D, x, t, s->sums);
  ++c->launches;
  k_crops_scale<<<grid, 256, 0, c->stream>>>(x, t, D, h2, s->sums);
  ++c->launches;
  k_crops_den<<<grid, 256, 0, c->stream>>>(t, D, s->sums + B, s->sums + 2 * B);
  ++c->launches;
  CK(cudaGetLastError());
  return PIC_OK;
}

int pic_cnn_loss(pic_ctx* c, const float* y, const float* t, int B, int D, float* gy, double* loss_host) {
  if (!c || !y || !t || !gy || !loss_host || B < 1) return PIC_EINVAL;
  if (!c->cnn || c->cnn->bmax < B) return PIC_ESTATE;
  CnnState* s = c->cnn;
  const size_t cells = (size_t)B * D * D * D;
  if (s->q_cells < cells) {
    dfree(s->q);
    s->q_cells = 0;
    int e;
    if ((e = dalloc(&s->q, cells))) return e;
    s->q_cells = cells;
  }
  CK(cudaMemsetAsync(s->sums + 3 * B, 0, 2 * (size_t)B * sizeof(double), c->stream));
  dim3 grid(64, B);
  k_loss_q<<<grid, 256, 0, c->stream>>>(y, t, D, s->q, s->sums + 3 * B, s->sums + 4 * B);
  ++c->launches;
  k_loss_grad<<<grid, 256, 0, c->stream>>>(y, t, s->q, D, B, s->sums + B, s->sums + 2 * B, gy);
  ++c->launches;
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(s->sums_host, s->sums, 5 * (size_t)B * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double L = 0.0;
  for (int b = 0; b < B; ++b)
    L += s->sums_host[3 * B + b] / s->sums_host[B + b] + s->sums_host[4 * B + b] / s->sums_host[2 * B + b];
  *loss_host = L / B;
  return PIC_OK;
}

int pic_cnn_adam(pic_ctx* c, double lr) {
  if (!c || !(lr > 0.0)) return PIC_EINVAL;
  if (!cnn_ready(c)) return PIC_ESTATE;
  CnnState* s = c->cnn;
  s->adam_t += 1;
  const double b1 = 0.9, b2 = 0.999;
  launch(c, k_adam, 58, 256, 0, s->w, s->g, s->m, s->v, kWeights, (float)lr, (float)b1, (float)b2, 1e-8f,
         (float)(1.0 - pow(b1, s->adam_t)), (float)(1.0 - pow(b2, s->adam_t)));
  CK(cudaGetLastError());
  return repack(c);
}

}  // extern "C"
