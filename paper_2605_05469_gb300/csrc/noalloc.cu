// pic_field_energy_noalloc: the field-energy reduction for callers that
// cannot allocate device memory.
//
// Some callers are not allowed to call cudaMalloc at all: a host code that
// hands this library a fixed device-memory budget at start-up and owns every
// byte after that (a coupled multi-physics driver, a service sharing the GPU
// under a hard quota), or a latency-critical stepping loop that must not call
// cudaMalloc/cudaFree because those calls can synchronise the whole device.
// They cannot create a pic_ctx (which allocates its workspace), so this entry
// point takes only the caller's input and output buffers. Its reduction
// scratch (per-block partial sums and the last-block counter) lives in a
// file-scope __device__ array of fixed size, which every GPU that loads the
// library keeps until the process exits.
#include <math.h>

#include "common.cuh"

using namespace pic;

namespace {

constexpr int kNoAllocMaxBlocks = 2048;                          // grid of the reduction
constexpr size_t kNoAllocPartialBytes = (size_t)kNoAllocMaxBlocks * 3 * sizeof(double);
constexpr size_t kNoAllocScratchBytes = kNoAllocPartialBytes + 256;  // + counter, padded

// Shared by every call on a device; holds the last call's partial sums.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array in the current device's context. The
// name g_noalloc_scratch in host code is only a host-side stand-in, so the
// address is looked up with cudaGetSymbolAddress, with the device current, on
// every call: the lookup allocates nothing, and a cached address would go
// stale when the module is reloaded at another address (after
// cudaDeviceReset, or under another driver context).
int scratch_for_current_device(unsigned char** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return PIC_ECUDA;
  }
  *out = static_cast<unsigned char*>(p);
  return PIC_OK;
}

// Same reduction as the context's field-energy kernel (E = -grad phi by
// central differences, W_d = h^3 sum E_d^2 = (h/4) sum (phi_{i-1} - phi_{i+1})^2
// along d), with its partial sums and counter in the caller-free scratch.
__global__ void __launch_bounds__(256) k_field_energy_static(const double* __restrict__ phi, int N, double h,
                                                             double* out3, double* partials, unsigned* counter) {
  const size_t Ns = N, n = Ns * Ns * Ns;
  double a[3] = {0.0, 0.0, 0.0};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
    const int ix = (int)(c % Ns), iy = (int)((c / Ns) % Ns), iz = (int)(c / (Ns * Ns));
    const size_t row = c - ix, pl = c - (size_t)iy * Ns, col = c - (size_t)iz * Ns * Ns;
    const double dx = __ldg(phi + row + (ix == 0 ? N - 1 : ix - 1)) - __ldg(phi + row + (ix == N - 1 ? 0 : ix + 1));
    const double dy = __ldg(phi + pl + (size_t)(iy == 0 ? N - 1 : iy - 1) * Ns) -
                      __ldg(phi + pl + (size_t)(iy == N - 1 ? 0 : iy + 1) * Ns);
    const double dz = __ldg(phi + col + (size_t)(iz == 0 ? N - 1 : iz - 1) * Ns * Ns) -
                      __ldg(phi + col + (size_t)(iz == N - 1 ? 0 : iz + 1) * Ns * Ns);
    a[0] = fma(dx, dx, a[0]);
    a[1] = fma(dy, dy, a[1]);
    a[2] = fma(dz, dz, a[2]);
  }
  double tot[3];
  if (grid_reduce_last<3>(a, partials, counter, tot) && threadIdx.x == 0) {
    const double f = 0.25 * h;
    out3[0] = f * tot[0];
    out3[1] = f * tot[1];
    out3[2] = f * tot[2];
  }
}

}  // namespace

extern "C" int pic_field_energy_noalloc(const double* phi, int N, double k, double* out_w, void* cuda_stream) {
  if (!phi || !out_w || ((uintptr_t)phi % 16) != 0) return PIC_EINVAL;
  if (N < 8 || N > 1024 || N % 8 != 0 || !(k > 0.0)) return PIC_EINVAL;
  unsigned char* scratch = nullptr;
  int e = scratch_for_current_device(&scratch);
  if (e) return e;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PIC_ECUDA;
  const size_t n = (size_t)N * N * N;
  size_t blocks = (n / 4 + 255) / 256;
  if (blocks > (size_t)sms * 4) blocks = (size_t)sms * 4;
  if (blocks > (size_t)kNoAllocMaxBlocks) blocks = kNoAllocMaxBlocks;
  double* partials = reinterpret_cast<double*>(scratch);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNoAllocPartialBytes);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the counter must start at zero (a call that failed part-way could leave it set)
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), st) != cudaSuccess) return PIC_ECUDA;
  const double L = 2.0 * M_PI / k;
  k_field_energy_static<<<(unsigned)blocks, 256, 0, st>>>(phi, N, L / N, out_w, partials, counter);
  if (cudaGetLastError() != cudaSuccess) return PIC_ECUDA;
  return PIC_OK;
}
