// Device-side helpers shared by the kernels: epilogue coefficients and the
// deterministic two-level FP64 reduction.
#pragma once

#include "tc_internal.cuh"

// (ca, cp) of the epilogue rule, computed by thread 0 in FP64 and broadcast.
// A zero denominator gives a zero coefficient: that is how a Golub-Kahan
// breakdown (beta or alpha = 0) produces a zero tensor instead of Inf/NaN.
__device__ __forceinline__ void coef_compute(const Coef& c, float* sh2) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double ca = 1.0, cp = 0.0;
    switch (c.rule) {
      case COEF_RESID: ca = -1.0; cp = 1.0; break;
      case COEF_GK: {
        double s0 = *c.s0, s1 = *c.s1;
        ca = (s0 != 0.0) ? 1.0 / s0 : 0.0;
        cp = (s1 != 0.0) ? -s0 / s1 : 0.0;
        break;
      }
      case COEF_INV: {
        double s0 = *c.s0;
        ca = (s0 != 0.0) ? 1.0 / s0 : 0.0;
        break;
      }
      case COEF_NEG: ca = -1.0; break;
      case COEF_AXPY: cp = -*c.s0; break;
      default: break;
    }
    sh2[0] = (float)ca;
    sh2[1] = (float)cp;
  }
}

// Programmatic dependent launch. A kernel launched with the programmatic
// stream-serialization attribute may start while its predecessor finishes;
// pdl_wait() blocks until every predecessor grid has completed and its
// memory is visible, so it comes before the first read of anything a
// predecessor wrote. pdl_trigger() lets the next launch start being
// scheduled (it still waits in its own pdl_wait()). Both are no-ops for a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduce one value per thread over the CTA (fixed FP32 tree: a CTA sums at
// most a few thousand FP32 terms), store the CTA partial in FP64, and let the
// last CTA to arrive sum all partials in CTA order in FP64. The ticket is an
// acquire-release atomic: it publishes this CTA's partial and, for the last
// CTA, makes every other partial visible. Must be called by every thread of
// every CTA of the launch.
__device__ __forceinline__ void reduce_finish(float v, const Red& red) {
  __shared__ double sh_w[32];
  __shared__ int sh_last;
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  v = warp_sum_f(v);
  if ((tid & 31) == 0) sh_w[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    float wf = (tid < (nthr + 31) / 32) ? (float)sh_w[tid] : 0.f;
    wf = warp_sum_f(wf);
    if (tid == 0) {
      red.partials[bid] = (double)wf;
      unsigned t;
      asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(t) : "l"(red.ticket) : "memory");
      sh_last = (t == nblk - 1);
    }
  }
  __syncthreads();
  if (!sh_last) return;
  double acc = 0.0;
  for (unsigned i = tid; i < nblk; i += nthr) acc += __ldcg(red.partials + i);
  acc = warp_sum(acc);
  if ((tid & 31) == 0) sh_w[tid >> 5] = acc;
  __syncthreads();
  if (tid < 32) {
    double w = (tid < (nthr + 31) / 32) ? sh_w[tid] : 0.0;
    w = warp_sum(w);
    if (tid == 0) {
      if (red.status && !isfinite(w)) *red.status = TC_ENONFINITE;
      *red.out = red.sqrt_out ? sqrt(w) : w;
      *red.ticket = 0u;
    }
  }
}
