// Device-side helpers shared by the kernels: epilogue coefficients and the
// deterministic two-level FP64 reduction.
#pragma once

#include "tc_internal.cuh"

// FP64 reciprocal and inverse square root by Newton's method from the
// hardware estimates: y <- y (2 - x y) and y <- y (3/2 - x y^2 / 2), each step
// doubling the correct bits. A few dependent FMAs, where the IEEE division
// and square root are long sequences on this part's scarce FP64 units.
// The estimates flush subnormal inputs and results to zero, so the Newton
// form serves |x| in [DBL_MIN, 2^1000] only (where x, 1/x and 1/sqrt(x) are
// all normal); everything else (zero, subnormals, huge values, Inf, NaN)
// takes the IEEE operations. Within that range the results are within a few
// ulp of the correctly rounded ones (checked against host FP64 and long double
// references by tc_check_recip).
constexpr double kNewtonLo = 2.2250738585072014e-308;  // DBL_MIN
constexpr double kNewtonHi = 1.0715086071862673e301;   // 2^1000

__device__ __forceinline__ double rcp_newton(double x) {
  const double ax = fabs(x);
  if (!(ax >= kNewtonLo && ax <= kNewtonHi)) return 1.0 / x;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

__device__ __forceinline__ double rsqrt_newton(double x) {
  if (!(x >= kNewtonLo && x <= kNewtonHi)) return 1.0 / sqrt(x);
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double h = 0.5 * x;
#pragma unroll
  for (int i = 0; i < 3; ++i) y = y * fma(-h * y, y, 1.5);
  return y;
}

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
        ca = (s0 != 0.0) ? rcp_newton(s0) : 0.0;
        cp = (s1 != 0.0) ? -s0 * rcp_newton(s1) : 0.0;
        break;
      }
      case COEF_INV: {
        double s0 = *c.s0;
        ca = (s0 != 0.0) ? rcp_newton(s0) : 0.0;
        break;
      }
      case COEF_NEG: ca = -1.0; break;
      case COEF_AXPY: cp = -*c.s0; break;
      case COEF_ADD: cp = 1.0; break;
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
// reduce_finish_n: the same with the CTA's index among the nblk CTAs that
// share red's partials and ticket given explicitly (grouped launches, where
// one launch holds the CTAs of many reductions). Both return, to every
// thread, whether this CTA was the last to arrive (the one that wrote the
// result).
__device__ __forceinline__ bool reduce_finish_n(float v, const Red& red, unsigned bid,
                                                unsigned nblk) {
  __shared__ double sh_w[32];
  __shared__ int sh_last;
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
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
  if (!sh_last) return false;
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
  return true;
}

__device__ __forceinline__ bool reduce_finish(float v, const Red& red) {
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  return reduce_finish_n(v, red, bid, nblk);
}

// LSQR step scalars (Algorithm 6 steps (c)-(g), 0-based step j):
//   rho = hypot(rhobar_j, beta_{j+1}), c = rhobar_j/rho, s = beta_{j+1}/rho,
//   theta = s alpha_{j+1}, rhobar_{j+1} = c alpha_{j+1},
//   phi = c phibar_j, phibar_{j+1} = -s phibar_j,
//   X += (phi/rho) W,  W = V_{j+1} - (theta/rho) W,  V_{j+1} = V~/alpha_{j+1}.
// Called by one thread per CTA: every CTA derives the same values from the
// same device scalars; `writer` (one thread of the grid) stores index j+1 of
// the state, the history, the flags and done_out. sh = (phi/rho, 1/alpha,
// theta/rho); returns the stop decision (breakdown, convergence, non-finite,
// or the learned stop index reached).
__device__ __forceinline__ bool lsqr_step_scalars(const LsqrStep& u, float* sh, bool writer) {
  const int j = u.j;
  const double b = u.beta[j + 1], a = u.alpha[j + 1];
  const double rb = u.rhobar[j], pb = u.phibar[j];
  const double r2 = fma(rb, rb, b * b);
  // Newton's range (normal r2 up to 2^1000); else the IEEE path: zeros,
  // subnormals, Inf, NaN, and squares that would overflow
  const bool plain = r2 >= kNewtonLo && r2 <= kNewtonHi;
  const double irho = plain ? rsqrt_newton(r2) : 1.0 / hypot(rb, b);
  const double rho = plain ? r2 * irho : hypot(rb, b);
  const double c = rb * irho, s = b * irho;
  const double theta = s * a;
  const double phi = c * pb;
  const double pbn = -s * pb;
  const bool finite = isfinite(a) && isfinite(b) && isfinite(rho);
  const bool brk = (a == 0.0);
  const bool conv = fabs(pbn) < u.tol || (u.stop_at && *u.stop_at > 0 && j + 1 >= *u.stop_at);
  sh[0] = (float)(phi * irho);
  sh[1] = brk ? 0.f : (float)rcp_newton(a);
  sh[2] = (float)(theta * irho);
  const bool stop = brk || conv || !finite;
  if (writer) {
    u.rhobar[j + 1] = c * a;
    u.phibar[j + 1] = pbn;
    if (u.rgiv) {  // R_k and f_k of Q_k [C~_k beta_1 e_1] (§3.3): rho, theta, phi
      u.rgiv[3 * j] = rho;
      u.rgiv[3 * j + 1] = theta;
      u.rgiv[3 * j + 2] = phi;
    }
    if (u.phibar_hist) u.phibar_hist[j] = fabs(pbn);
    u.flags[1] = j + 1;
    if (!finite) u.flags[2] = TC_ENONFINITE;
    else if (brk) u.flags[2] = TC_EBREAKDOWN;
    else if (conv) u.flags[2] = 1;
    *u.done_out = stop ? 1 : 0;
  }
  return stop;
}

// The vector part of an LSQR step on elements [beg, end), by the threads of
// one CTA (nt threads), four loads in flight per thread. A step without
// vectors (X null: the iterate is formed from the kept basis at the end of
// the solve) does nothing here.
__device__ __forceinline__ void lsqr_step_vectors(const LsqrStep& u, size_t beg, size_t end,
                                                  float cx, float cv, float cw, bool stop,
                                                  int nt) {
  if (!u.X) return;
  for (size_t i0 = beg + threadIdx.x; i0 < end; i0 += 4 * (size_t)nt) {
    float w[4], x[4], v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const size_t i = i0 + (size_t)q * nt;
      w[q] = i < end ? u.W[i] : 0.f;
      x[q] = i < end ? u.X[i] : 0.f;
      v[q] = i < end ? u.V[i] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const size_t i = i0 + (size_t)q * nt;
      if (i >= end) break;
      u.X[i] = fmaf(cx, w[q], x[q]);
      if (!stop) {
        const float vn = cv * v[q];
        u.W[i] = fmaf(-cw, w[q], vn);
        if (u.basis_slot) u.basis_slot[i] = vn;
      }
    }
  }
}
