// Whole-tensor passes of the Krylov iterations (HBM-bound): norms and inner
// products (Definition 2.2), scaled copies, the LSQR update of Algorithm 6
// steps (c)-(g), the basis combination V (*) y (§3.1, eq. (xm)), and one
// modified Gram-Schmidt pass of Algorithm 2 fused with the next inner product.
#include "tc_device.cuh"

namespace {

constexpr int NT = 256;

unsigned grid_for(size_t n, int per_thread) {
  size_t b = (n + (size_t)NT * per_thread - 1) / ((size_t)NT * per_thread);
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

__global__ void __launch_bounds__(NT)
k_reduce(const float* __restrict__ x, const float* __restrict__ other, size_t n, Red red,
         const int* skip) {
  if (skip && *skip) return;
  float s = 0.f;
  const size_t stride = (size_t)gridDim.x * NT;
  for (size_t i = (size_t)blockIdx.x * NT + threadIdx.x; i < n; i += stride) {
    const float v = x[i];
    s = fmaf(v, other ? other[i] : v, s);
  }
  reduce_finish(s, red);
}

__global__ void __launch_bounds__(NT)
k_scale(const float* __restrict__ in, float* out, size_t n, Coef c, const float* prev,
        const int* skip) {
  if (skip && *skip) return;
  __shared__ float sh[2];
  coef_compute(c, sh);
  __syncthreads();
  const float ca = sh[0], cp = sh[1];
  const size_t stride = (size_t)gridDim.x * NT;
  for (size_t i = (size_t)blockIdx.x * NT + threadIdx.x; i < n; i += stride) {
    float o = ca * in[i];
    if (prev) o = fmaf(cp, prev[i], o);
    out[i] = o;
  }
}

// One LSQR step as its own launch (lsqr_step_scalars, lsqr_step_vectors):
// X += (phi / rho) W; V_{j+1} = V / alpha; W = V_{j+1} - (theta / rho) W.
// One wave of CTAs strides over the tensor in units of T (float4 when every
// pointer is 16-byte aligned and n % 4 == 0, else float), UPT units a thread
// per pass, the next pass's loads issued before this pass's stores. Thread
// 0's FP64 scalar chain runs once a CTA, while the first pass's loads are in
// flight; CTA 0 writes the state.
constexpr int UPT = 2;
int g_sms = 152;             // SM count of the device (set by vec_init)
int g_upd_ctas[2] = {4, 4};  // resident k_lsqr_update CTAs per SM: float, float4

__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 mul4(float a, float4 x) {
  return make_float4(a * x.x, a * x.y, a * x.z, a * x.w);
}
__device__ __forceinline__ float fma4(float a, float x, float y) { return fmaf(a, x, y); }
__device__ __forceinline__ float mul4(float a, float x) { return a * x; }

template <typename T>
__global__ void __launch_bounds__(NT) k_lsqr_update(LsqrStep u) {
  pdl_wait();
  if (*u.done_in) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *u.done_out = 1;
    return;
  }
  __shared__ float sh[3];
  __shared__ int sh_stop;
  constexpr int EL = sizeof(T) / sizeof(float);
  const size_t nu = u.n / EL;  // units; EL == 4 only when n % 4 == 0
  T* X = reinterpret_cast<T*>(u.X);
  T* W = reinterpret_cast<T*>(u.W);
  const T* V = reinterpret_cast<const T*>(u.V);
  T* Vs = reinterpret_cast<T*>(u.basis_slot);
  const size_t per = (size_t)NT * UPT, stride = (size_t)gridDim.x * per;
  size_t cta = (size_t)blockIdx.x * per;
  T w[UPT], x[UPT], v[UPT];
#pragma unroll
  for (int q = 0; q < UPT; ++q) {
    const size_t i = cta + threadIdx.x + (size_t)q * NT;
    if (i < nu) {
      w[q] = W[i];
      x[q] = X[i];
      v[q] = V[i];
    }
  }
  pdl_trigger();
  if (threadIdx.x == 0) sh_stop = lsqr_step_scalars(u, sh, blockIdx.x == 0);
  __syncthreads();
  const float cx = sh[0], cv = sh[1], cw = sh[2];
  const bool stop = sh_stop;
  while (cta < nu) {
    const size_t nxt = cta + stride;
    T w2[UPT], x2[UPT], v2[UPT];
#pragma unroll
    for (int q = 0; q < UPT; ++q) {
      const size_t i = nxt + threadIdx.x + (size_t)q * NT;
      if (i < nu) {
        w2[q] = W[i];
        x2[q] = X[i];
        v2[q] = V[i];
      }
    }
#pragma unroll
    for (int q = 0; q < UPT; ++q) {
      const size_t i = cta + threadIdx.x + (size_t)q * NT;
      if (i < nu) {
        X[i] = fma4(cx, w[q], x[q]);
        if (!stop) {
          const T vn = mul4(cv, v[q]);
          W[i] = fma4(-cw, w[q], vn);
          if (Vs) Vs[i] = vn;
        }
      }
      w[q] = w2[q];
      x[q] = x2[q];
      v[q] = v2[q];
    }
    cta = nxt;
  }
}

// The scalars of one LSQR step (lsqr_step_scalars), one thread.
__global__ void k_lsqr_scalars(LsqrStep u) {
  if (*u.done_in) {
    *u.done_out = 1;
    return;
  }
  float sh[3];
  lsqr_step_scalars(u, sh, true);
}

// y = R^{-1} f by back substitution: R upper bidiagonal with diagonal
// rho_1..rho_k and superdiagonal theta_2..theta_k, f = (phi_1..phi_k), from
// rg = (rho_j, theta_{j+1}, phi_j) interleaved; zero beyond k. One thread.
__global__ void k_lsqr_coeffs(const double* __restrict__ rg, const int* kdev, int kmax,
                              double* y) {
  const int k = kdev ? max(0, min(*kdev, kmax)) : kmax;
  for (int i = kmax - 1; i >= k; --i) y[i] = 0.0;
  double yi = 0.0;
  for (int i = k - 1; i >= 0; --i) {
    const double num = rg[3 * i + 2] - (i + 1 < k ? rg[3 * i + 1] * yi : 0.0);
    yi = num / rg[3 * i];
    y[i] = yi;
  }
}

// X = sum_i (y_i / d_i) B_i and X2 = sum_i (y2_i / d_i) B_i over i < k in one
// pass over the basis (same order and loads as k_combine).
template <bool VEC>
__global__ void __launch_bounds__(NT)
k_combine2(float* X, float* X2, const float* __restrict__ basis, size_t stride, int kmax,
           const int* kdev, const double* __restrict__ y, const double* __restrict__ y2,
           const double* __restrict__ d, size_t n) {
  __shared__ float ys[TC_MAX_PROJ], ys2[TC_MAX_PROJ];
  const int k = kdev ? max(0, min(*kdev, kmax)) : kmax;
  for (int i = threadIdx.x; i < k; i += NT) {
    const double dv = d ? d[i] : 1.0;
    ys[i] = (float)(y[i] / dv);
    ys2[i] = (float)(y2[i] / dv);
  }
  __syncthreads();
  const size_t e = 4 * ((size_t)blockIdx.x * NT + threadIdx.x);
  if (e >= n) return;
  if (VEC && e + 3 < n) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    for (int q0 = 0; q0 < k; q0 += 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = q0 + u < k ? __ldg(reinterpret_cast<const float4*>(basis + (size_t)(q0 + u) * stride + e))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (q0 + u >= k) break;
        const float c = ys[q0 + u], c2 = ys2[q0 + u];
        a.x = fmaf(c, v[u].x, a.x);
        a.y = fmaf(c, v[u].y, a.y);
        a.z = fmaf(c, v[u].z, a.z);
        a.w = fmaf(c, v[u].w, a.w);
        b.x = fmaf(c2, v[u].x, b.x);
        b.y = fmaf(c2, v[u].y, b.y);
        b.z = fmaf(c2, v[u].z, b.z);
        b.w = fmaf(c2, v[u].w, b.w);
      }
    }
    *reinterpret_cast<float4*>(X + e) = a;
    *reinterpret_cast<float4*>(X2 + e) = b;
    return;
  }
  for (size_t i = e; i < e + 4 && i < n; ++i) {
    float a = 0.f, b = 0.f;
    for (int q = 0; q < k; ++q) {
      const float v = __ldg(basis + (size_t)q * stride + i);
      a = fmaf(ys[q], v, a);
      b = fmaf(ys2[q], v, b);
    }
    X[i] = a;
    X2[i] = b;
  }
}

// X = X0 + sum_{i<k} y_i V_i (V_i at basis + i*stride); k read from the device.
// Thread t owns elements 4t..4t+3 and keeps eight basis loads in flight; the
// sum runs in the order i = 0, 1, .., k-1 for every element. VEC: 16-byte
// aligned tensors and stride % 4 == 0.
template <bool VEC>
__global__ void __launch_bounds__(NT)
k_combine(float* X, const float* X0, const float* __restrict__ basis, size_t stride, int kmax,
          const int* kdev, const double* __restrict__ y, size_t n, const int* skip) {
  if (skip && *skip) return;
  __shared__ float ys[TC_MAX_PROJ];
  const int k = kdev ? min(*kdev, kmax) : kmax;
  for (int i = threadIdx.x; i < k; i += NT) ys[i] = (float)y[i];
  __syncthreads();
  const size_t e = 4 * ((size_t)blockIdx.x * NT + threadIdx.x);
  if (e >= n) return;
  if (VEC && e + 3 < n) {
    float4 acc = X0 ? *reinterpret_cast<const float4*>(X0 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q0 = 0; q0 < k; q0 += 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = q0 + u < k ? __ldg(reinterpret_cast<const float4*>(basis + (size_t)(q0 + u) * stride + e))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (q0 + u >= k) break;
        const float c = ys[q0 + u];
        acc.x = fmaf(c, v[u].x, acc.x);
        acc.y = fmaf(c, v[u].y, acc.y);
        acc.z = fmaf(c, v[u].z, acc.z);
        acc.w = fmaf(c, v[u].w, acc.w);
      }
    }
    *reinterpret_cast<float4*>(X + e) = acc;
    return;
  }
  for (size_t i = e; i < e + 4 && i < n; ++i) {
    float acc = X0 ? X0[i] : 0.f;
    for (int q = 0; q < k; ++q) acc = fmaf(ys[q], __ldg(basis + (size_t)q * stride + i), acc);
    X[i] = acc;
  }
}

// The Krylov epilogue as its own pass: out = ca * in + cp * prev (prev may
// alias out), then the fused reduction of out. Used by the transform-domain
// products, whose slice GEMMs store plainly. Each thread keeps UNR float4
// loads of every operand in flight; one element is read and written by one
// thread only, so prev aliasing out is safe.
constexpr int UNR = 4;
__global__ void __launch_bounds__(NT)
k_epi(const float* __restrict__ in, float* out, size_t n, Epi ep, int vec) {
  if (ep.skip && *ep.skip) return;
  __shared__ float sh[2];
  coef_compute(ep.coef, sh);
  __syncthreads();
  const float ca = sh[0], cp = sh[1];
  float local = 0.f;
  const size_t gt = (size_t)blockIdx.x * NT + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * NT;
  size_t done = 0;
  if (vec) {
    const size_t n4 = n / 4;
    const float4* in4 = reinterpret_cast<const float4*>(in);
    const float4* pv4 = reinterpret_cast<const float4*>(ep.prev);
    const float4* ot4 = reinterpret_cast<const float4*>(ep.red.other);
    float4* out4 = reinterpret_cast<float4*>(out);
    for (size_t i0 = gt; i0 < n4; i0 += UNR * stride) {
      float4 v[UNR], pv[UNR], ov[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const size_t i = i0 + u * stride;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        v[u] = i < n4 ? in4[i] : z;
        pv[u] = (ep.prev && i < n4) ? pv4[i] : z;
        ov[u] = (ep.red.other && i < n4) ? ot4[i] : z;
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const size_t i = i0 + u * stride;
        if (i >= n4) break;
        float4 o = make_float4(ca * v[u].x, ca * v[u].y, ca * v[u].z, ca * v[u].w);
        if (ep.prev) {
          o.x = fmaf(cp, pv[u].x, o.x); o.y = fmaf(cp, pv[u].y, o.y);
          o.z = fmaf(cp, pv[u].z, o.z); o.w = fmaf(cp, pv[u].w, o.w);
        }
        out4[i] = o;
        if (ep.red.out) {
          const float4 q = ep.red.other ? ov[u] : o;
          local = fmaf(o.x, q.x, fmaf(o.y, q.y, fmaf(o.z, q.z, fmaf(o.w, q.w, local))));
        }
      }
    }
    done = 4 * n4;
  }
  for (size_t i = done + gt; i < n; i += stride) {
    float o = ca * in[i];
    if (ep.prev) o = fmaf(cp, ep.prev[i], o);
    out[i] = o;
    if (ep.red.out) local = fmaf(o, ep.red.other ? ep.red.other[i] : o, local);
  }
  if (ep.red.out) reduce_finish(local, ep.red);
}

// Algorithm 2 step 3(b): W -= h V_i, then <V_next, W> (or ||W||^2) for the next step.
__global__ void __launch_bounds__(NT)
k_mgs_pass(float* W, const float* __restrict__ Vi, const double* h, const float* Vnext,
           size_t n, Red red, const int* skip) {
  if (skip && *skip) return;
  __shared__ float sh_h;
  if (threadIdx.x == 0) sh_h = (float)(*h);
  __syncthreads();
  const float hh = sh_h;
  float s = 0.f;
  const size_t st = (size_t)gridDim.x * NT;
  for (size_t i = (size_t)blockIdx.x * NT + threadIdx.x; i < n; i += st) {
    const float w = fmaf(-hh, Vi[i], W[i]);
    W[i] = w;
    s = fmaf(w, Vnext ? Vnext[i] : w, s);
  }
  reduce_finish(s, red);
}

}  // namespace

// The vector passes need no shared memory; asking for the largest shared
// carveout keeps the SM in the split the GEMM launches around them use, so
// consecutive launches of a solve do not reconfigure the L1/shared split.
int vec_init() {
  const int c = cudaSharedmemCarveoutMaxShared;
  TC_CUDA(cudaFuncSetAttribute(k_reduce, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_scale, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_lsqr_update<float>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_lsqr_update<float4>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  int dev = 0;
  TC_CUDA(cudaGetDevice(&dev));
  TC_CUDA(cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev));
  TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_upd_ctas[0], k_lsqr_update<float>,
                                                        NT, 0));
  TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_upd_ctas[1], k_lsqr_update<float4>,
                                                        NT, 0));
  TC_CUDA(cudaFuncSetAttribute(k_combine<true>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_combine<false>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_combine2<true>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_combine2<false>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_mgs_pass, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_epi, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  return TC_OK;
}

int launch_epi(const float* in, float* out, size_t n, const Epi& ep, cudaStream_t st) {
  auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  const int vec = al(in) && al(out) && (!ep.prev || al(ep.prev)) &&
                  (!ep.red.other || al(ep.red.other));
  k_epi<<<grid_for(n, 4 * UNR), NT, 0, st>>>(in, out, n, ep, vec);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_reduce(const float* x, const float* other, size_t n, const Red& red,
                  const int* skip, cudaStream_t st) {
  k_reduce<<<grid_for(n, 16), NT, 0, st>>>(x, other, n, red, skip);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_scale(const float* in, float* out, size_t n, const Coef& c, const float* prev,
                 const int* skip, cudaStream_t st) {
  k_scale<<<grid_for(n, 8), NT, 0, st>>>(in, out, n, c, prev, skip);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_lsqr_update(const LsqrStep& step, cudaStream_t st) {
  auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  const bool vec = step.n % 4 == 0 && al(step.X) && al(step.W) && al(step.V) &&
                   (!step.basis_slot || al(step.basis_slot));
  const size_t units = vec ? step.n / 4 : step.n;
  size_t blocks = (units + (size_t)NT * UPT - 1) / ((size_t)NT * UPT);
  const size_t wave = (size_t)g_sms * (size_t)(g_upd_ctas[vec ? 1 : 0] > 0 ? g_upd_ctas[vec ? 1 : 0] : 1);
  if (blocks > wave) blocks = wave;
  if (blocks < 1) blocks = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(NT);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (vec)
    TC_CUDA(cudaLaunchKernelEx(&cfg, k_lsqr_update<float4>, step));
  else
    TC_CUDA(cudaLaunchKernelEx(&cfg, k_lsqr_update<float>, step));
  return TC_OK;
}

int launch_combine(float* X, const float* X0, const float* basis, size_t stride, int kmax,
                   const int* kdev, const double* y, size_t n, const int* skip,
                   cudaStream_t st) {
  TC_CHECK(kmax <= TC_MAX_PROJ);
  auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  const bool vec = stride % 4 == 0 && al(X) && al(basis) && (!X0 || al(X0));
  const size_t blocks = (n + 4 * (size_t)NT - 1) / (4 * (size_t)NT);
  TC_CHECK(blocks >= 1 && blocks <= 0x7fffffffULL);
  if (vec)
    k_combine<true><<<(unsigned)blocks, NT, 0, st>>>(X, X0, basis, stride, kmax, kdev, y, n, skip);
  else
    k_combine<false><<<(unsigned)blocks, NT, 0, st>>>(X, X0, basis, stride, kmax, kdev, y, n, skip);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_lsqr_scalars(const LsqrStep& step, cudaStream_t st) {
  k_lsqr_scalars<<<1, 1, 0, st>>>(step);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_lsqr_coeffs(const double* rg, const int* kdev, int kmax, double* y, cudaStream_t st) {
  TC_CHECK(kmax >= 1 && kmax <= TC_MAX_PROJ);
  k_lsqr_coeffs<<<1, 1, 0, st>>>(rg, kdev, kmax, y);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_combine2(float* X, const double* y, float* X2, const double* y2, const double* d,
                    const float* basis, size_t stride, int kmax, const int* kdev, size_t n,
                    cudaStream_t st) {
  TC_CHECK(kmax <= TC_MAX_PROJ);
  auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  const bool vec = stride % 4 == 0 && al(X) && al(X2) && al(basis);
  const size_t blocks = (n + 4 * (size_t)NT - 1) / (4 * (size_t)NT);
  TC_CHECK(blocks >= 1 && blocks <= 0x7fffffffULL);
  if (vec)
    k_combine2<true><<<(unsigned)blocks, NT, 0, st>>>(X, X2, basis, stride, kmax, kdev, y, y2, d, n);
  else
    k_combine2<false><<<(unsigned)blocks, NT, 0, st>>>(X, X2, basis, stride, kmax, kdev, y, y2, d, n);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_mgs_pass(float* W, const float* Vi, const double* h, const float* Vnext,
                    size_t n, const Red& red, const int* skip, cudaStream_t st) {
  k_mgs_pass<<<grid_for(n, 16), NT, 0, st>>>(W, Vi, h, Vnext, n, red, skip);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

namespace {
// The FP64 reciprocal and inverse square root of the step and coefficient
// scalars (rcp_newton, rsqrt_newton), evaluated elementwise for their test.
__global__ void k_check_recip(const double* __restrict__ x, size_t n, double* rcp,
                              double* rsq) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    rcp[i] = rcp_newton(v);
    rsq[i] = v > 0.0 ? rsqrt_newton(v) : 0.0;
  }
}
}  // namespace

extern "C" int tc_check_recip(const double* x, size_t n, double* rcp, double* rsqrt_out,
                              tc_stream_t stream) {
  if (!x || !rcp || !rsqrt_out || n < 1 || n > ((size_t)1 << 28)) return TC_EINVAL;
  const size_t blocks = (n + 255) / 256;
  k_check_recip<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(
      x, n, rcp, rsqrt_out);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

