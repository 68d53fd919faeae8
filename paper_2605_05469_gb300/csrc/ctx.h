// Internal: the context behind the C ABI and the host helpers shared by the
// library's translation units (not part of the public interface).
#pragma once
#include "common.cuh"

namespace pic {

struct CnnState;  // learned-preconditioner state, see cnn.cu
struct MgState;   // multigrid hierarchy, see mg.cu
struct FftState;  // spectral solve plans and buffers, see fft.cu
struct PifState;  // particle-in-Fourier plans and buffers, see pif.cu

struct SolverWs {
  // FP64 reference solve
  double *x = nullptr, *r = nullptr, *p[2] = {nullptr, nullptr}, *q = nullptr;
  // mixed
  double* xm[2] = {nullptr, nullptr};
  float *x32 = nullptr, *r32 = nullptr, *p32[2] = {nullptr, nullptr};
  // flexible CG with the learned preconditioner
  float* z32[2] = {nullptr, nullptr};
  float* q32 = nullptr;  // A p of the last direction
  float* r32b = nullptr; // second FP32 residual: the fused update writes r' while r is still read as halo
  // shared
  double* b = nullptr;
};

// A pool of CUDA event pairs recorded on the context stream; flushed (elapsed
// times summed) once the stream has passed them.
struct EventPool {
  static constexpr int kCap = 1024;
  cudaEvent_t ev[kCap][2] = {};
  int n = 0;         // pending pairs
  int count = 0;     // flushed pairs
  double ms = 0.0;   // flushed total
  bool ready = false;
  bool init() {
    for (int i = 0; i < kCap; ++i)
      for (int j = 0; j < 2; ++j)
        if (cudaEventCreate(&ev[i][j]) != cudaSuccess) return false;
    ready = true;
    return true;
  }
  void destroy() {
    for (int i = 0; i < kCap; ++i)
      for (int j = 0; j < 2; ++j)
        if (ev[i][j]) cudaEventDestroy(ev[i][j]);
    ready = false;
  }
  void flush() {
    for (int i = 0; i < n; ++i) {
      float t = 0.f;
      if (cudaEventSynchronize(ev[i][1]) == cudaSuccess && cudaEventElapsedTime(&t, ev[i][0], ev[i][1]) == cudaSuccess) {
        ms += t;
        ++count;
      }
    }
    n = 0;
  }
  // Start a pair; returns its slot or -1 when profiling is off.
  int begin(cudaStream_t st) {
    if (!ready) return -1;
    if (n == kCap) flush();
    cudaEventRecord(ev[n][0], st);
    return n++;
  }
  void end(int slot, cudaStream_t st) {
    if (slot >= 0) cudaEventRecord(ev[slot][1], st);
  }
  void reset() { n = 0; count = 0; ms = 0.0; }
};

}  // namespace pic

struct pic_ctx {
  cudaStream_t stream = nullptr;
  int device = 0, sms = 0;
  // geometry
  bool has_grid = false;
  int N = 0;
  size_t n = 0;
  double L = 0, h = 0, alpha = 0, k = 0;
  int ppc = 0;
  uint64_t np = 0;
  pic::Grid grid{};
  // particles
  pic::PRec* prec[2] = {nullptr, nullptr};  // particle records, current sort order and scratch
  int cur = 0;
  uint32_t *counts = nullptr, *offsets = nullptr, *chunks = nullptr;
  bool keys_valid = false, sorted = false, half_step = false;
  float2* E = nullptr;    // 4 n: E_x, E_y, E_z at the nodes and phi, double-float
  float2* dep = nullptr;  // 8 n: per cell, the CIC charge of its particles at each of its 8 corners
  // solver
  pic::SolverWs ws;
  pic::Scalars* sc = nullptr;
  pic::Scalars* sc_host = nullptr;  // pinned, 2 slots
  double* partials = nullptr;
  size_t partials_len = 0;
  unsigned* counter = nullptr;
  int* err = nullptr;
  int* err_host = nullptr;   // pinned
  double* out3 = nullptr;    // device, 3 doubles
  double* out3_host = nullptr;  // pinned
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, batch_ev[2] = {nullptr, nullptr};
  // tracing
  int64_t launches = 0;
  bool prof_on = false;
  pic::EventPool* phase = nullptr;  // [PIC_NPHASE]
  pic::EventPool* ker = nullptr;    // [PIC_NKER]
  int ker_prec[PIC_NKER] = {};
  // learned preconditioner (weights, activations, optimiser state)
  pic::CnnState* cnn = nullptr;
  int cnn_apply_mode = 0;  // PIC_CNN_APPLY_*
  // multigrid preconditioner (level buffers)
  pic::MgState* mg = nullptr;
  pic::FftState* fft = nullptr;
  pic::PifState* pif = nullptr;
  double* pif_E = nullptr;  // 3 np: the particle-in-Fourier field, current particle order
  // host <-> device particle transfers: two FP64 staging buffers of up to
  // kStageParticles particles each (6 blocks), the copies on their own stream
  // so that one chunk's copy overlaps the neighbouring chunk's conversion
  // kernel (io_ev: [b] copy through buffer b done, [2 + b] kernel on buffer b
  // done, [4] the context stream's work before the transfer), and a device
  // flag for rejected input
  double* stage = nullptr;
  cudaStream_t io_stream = nullptr;
  cudaEvent_t io_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int* io_flag = nullptr;
};

namespace pic {

// The CUDA error behind the calling thread's last PIC_ECUDA (pic_cuda_error).
inline thread_local cudaError_t g_last_cuda_error = cudaSuccess;

// A failed CUDA call: recorded for pic_cuda_error, and the runtime's own
// last-error state is cleared so it does not surface in a later call.
#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) {                      \
      pic::g_last_cuda_error = e_;                \
      cudaGetLastError();                         \
      return PIC_ECUDA;                           \
    }                                             \
  } while (0)

template <typename T>
inline int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return PIC_OK;
  if (cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return PIC_ENOMEM;
  }
  return PIC_OK;
}

template <typename T>
inline void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

inline int round32(int t) { return ((t + 31) / 32) * 32; }

// Every kernel goes through here: launched on the context stream and counted.
template <typename... KArgs, typename... Args>
void launch(pic_ctx* c, void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, Args... args) {
  kernel<<<grid, block, smem, c->stream>>>(args...);
  ++c->launches;
}
template <typename... KArgs, typename... Args>
void launch(pic_ctx* c, void (*kernel)(KArgs...), dim3 grid, unsigned block, size_t smem, Args... args) {
  kernel<<<grid, block, smem, c->stream>>>(args...);
  ++c->launches;
}
template <typename... KArgs, typename... Args>
void launch(pic_ctx* c, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, Args... args) {
  kernel<<<grid, block, smem, c->stream>>>(args...);
  ++c->launches;
}

// Phase timer around one public call (no-op unless profiling is on).
struct PhaseScope {
  pic_ctx* c;
  int phase, slot;
  PhaseScope(pic_ctx* cc, int ph) : c(cc), phase(ph), slot(-1) {
    if (c->prof_on) slot = c->phase[phase].begin(c->stream);
  }
  ~PhaseScope() {
    if (slot >= 0) c->phase[phase].end(slot, c->stream);
  }
};

}  // namespace pic
