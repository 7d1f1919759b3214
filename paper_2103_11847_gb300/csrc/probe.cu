// Peak-rate probes: the FP32 FFMA, FP64 DFMA and tcgen05 (TF32, BF16) issue
// rates of the device, which the roofline fractions of the FFMA-bound and
// TF32 kernels divide by. The paper has no counterpart. Each probe runs a
// fixed amount of independent arithmetic whose count the caller knows; the
// caller times the launch with CUDA events.
#include "tc_device.cuh"
#include "tcgen05.cuh"

namespace {

using namespace tc5;

constexpr int FMA_CHAINS = 8;  // independent accumulators a thread

// `iters` rounds of FMA_CHAINS independent FMAs a thread (2 flops each).
// The result goes to sink[0] only if it is impossible (never), which keeps
// the arithmetic alive without a store per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b, float* sink) {
  T x[FMA_CHAINS];
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) s += x[c];
  if (s == (T)-12345.678) sink[0] = (float)s;
}

// One CTA a SM (its shared memory request keeps others off the SM): thread
// 0 issues `iters` rounds of four 128 x 256 x K MMAs
// (K = 16 BF16 or 8 TF32 values, one 128-byte swizzled slab of A and B),
// accumulating into 256 tensor-memory columns, then waits (bounded) for them.
template <int KIND>
__global__ void __launch_bounds__(128, 1) k_mma_probe(int iters, int* status) {
  constexpr int BM = 128, BN = 256;
  constexpr uint32_t FMT = KIND == 0 ? 1u : 2u;
  constexpr int ES = KIND == 0 ? 2 : 4, UK = KIND == 0 ? 16 : 8;
  constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  extern __shared__ uint8_t pr_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(pr_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;                   // BM rows of 128 bytes
  uint8_t* sB = base + BM * 128;        // BN rows of 128 bytes
  uint64_t* done = reinterpret_cast<uint64_t*>(sB + BN * 128);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  // operands: a small constant in every element (the values do not matter)
  for (int i = threadIdx.x; i < (BM + BN) * 128 / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(base)[i] = KIND == 0 ? 0x3c003c00u : 0x3c000000u;
  if (threadIdx.x == 0) {
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tslot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (threadIdx.x == 0) {
    const uint32_t a0 = su32(sA), b0 = su32(sB);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int kk = 0; kk < 128 / (UK * ES); ++kk)
        umma<KIND>(tmem, smem_desc(a0 + kk * UK * ES, 16, 1024),
                   smem_desc(b0 + kk * UK * ES, 16, 1024), IDESC, (it | kk) != 0);
    }
    umma_commit(done);
    if (!mbar_wait(done, 0)) atomicExch(status, TC_ETIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN)
                 : "memory");
}

// More than half an SM's shared memory, so that no two probe CTAs share an SM.
constexpr size_t kProbeSmem = 120 * 1024;

}  // namespace

extern "C" int tc_peak_probe(int kind, int iters, int* status, tc_stream_t stream) {
  if (!status || iters < 1 || iters > (1 << 24) || kind < 0 || kind > 3) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  TC_CUDA(cudaGetDevice(&dev));
  TC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (kind == 0 || kind == 1) {
    // eight CTAs of 256 threads a SM: every FP32 (FP64) lane busy
    if (kind == 0)
      k_fma_probe<float><<<nsm * 8, 256, 0, st>>>(iters, 1.0000001f, 1e-7f,
                                                  reinterpret_cast<float*>(status));
    else
      k_fma_probe<double><<<nsm * 8, 256, 0, st>>>(iters, 1.0000000001, 1e-12,
                                                   reinterpret_cast<float*>(status));
  } else {
    auto fn = kind == 2 ? k_mma_probe<1> : k_mma_probe<0>;
    TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kProbeSmem));
    fn<<<nsm, 128, kProbeSmem, st>>>(iters, status);
  }
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
