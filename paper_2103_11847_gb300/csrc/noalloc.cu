// tc_fro_norm_noalloc: the Frobenius norm reduction without any device
// allocation, for callers that cannot call cudaMalloc. Examples are code
// whose device memory belongs to another allocator (a framework pool that
// has reserved the device), and code on a path where the implicit device
// synchronisation of cudaMalloc/cudaFree is not acceptable.
//
// It runs the same kernel shape as the norm reduction used by the solvers (same
// grid, same per-thread FP32 partial sums, same FP64 tree in CTA order), but
// its per-CTA partials and arrival ticket live in the file-scope array below
// instead of in a plan's workspace. Every GPU that loads this library holds
// the array until the process exits.
#include <mutex>

#include "tc_device.cuh"

namespace {

constexpr int NT = 256;
constexpr unsigned kMaxBlocks = 152 * 32;  // the solvers' cap on reduction CTAs
// Largest input: at most 64 elements per thread in the FP32 per-thread sums.
constexpr size_t kMaxElems = (size_t)kMaxBlocks * NT * 64;
// Scratch: kMaxBlocks FP64 partials, then the ticket (39 KB in all).
constexpr size_t kScratchBytes = kMaxBlocks * sizeof(double) + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Same grid as the solvers' reduction pass (16 elements per thread, capped).
unsigned grid_for(size_t n) {
  size_t b = (n + (size_t)NT * 16 - 1) / ((size_t)NT * 16);
  if (b < 1) b = 1;
  if (b > kMaxBlocks) b = kMaxBlocks;
  return (unsigned)b;
}

__global__ void __launch_bounds__(NT)
k_fro_norm_static(const float* __restrict__ x, size_t n, double* out, unsigned char* scratch) {
  Red red;
  red.out = out;
  red.sqrt_out = 1;
  red.partials = reinterpret_cast<double*>(scratch);
  red.ticket = reinterpret_cast<unsigned*>(scratch + kMaxBlocks * sizeof(double));
  float s = 0.f;
  const size_t stride = (size_t)gridDim.x * NT;
  for (size_t i = (size_t)blockIdx.x * NT + threadIdx.x; i < n; i += stride) {
    const float v = x[i];
    s = fmaf(v, v, s);
  }
  reduce_finish(s, red);
}

// Device address of g_scratch on the current device, looked up once per device.
int scratch_for_current_device(unsigned char** ptr) {
  int dev = 0;
  TC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return TC_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    TC_CUDA(cudaGetSymbolAddress(&p, g_scratch));
    g_scratch_ptr[dev] = p;
  }
  *ptr = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return TC_OK;
}

}  // namespace

extern "C" int tc_fro_norm_noalloc(const float* X, size_t n, double* out, tc_stream_t stream) {
  if (!X || !out || n == 0) return TC_EINVAL;
  if (n > kMaxElems) {
    tc_set_message("tc_fro_norm_noalloc: n exceeds the maximum of 79691776 elements");
    return TC_EINVAL;
  }
  unsigned char* scratch = nullptr;
  TC_TRY(scratch_for_current_device(&scratch));
  cudaStream_t st = (cudaStream_t)stream;
  // The ticket must be zero when the launch starts; the previous call left it
  // zero, but a call cut short by an error would not have.
  TC_CUDA(cudaMemsetAsync(scratch + kMaxBlocks * sizeof(double), 0, sizeof(unsigned), st));
  k_fro_norm_static<<<grid_for(n), NT, 0, st>>>(X, n, out, scratch);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
