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

// LSQR, Algorithm 6 steps (c)-(g) for iteration j (0-based; the paper's j+1):
//   rho = hypot(rhobar_j, beta_{j+1}), c = rhobar_j/rho, s = beta_{j+1}/rho,
//   theta = s alpha_{j+1}, rhobar_{j+1} = c alpha_{j+1},
//   phi = c phibar_j, phibar_{j+1} = -s phibar_j,
//   X += (phi/rho) W,  W = V_{j+1} - (theta/rho) W,  V_{j+1} = Vt/alpha_{j+1}.
// Every CTA derives the same scalars from alpha[j+1], beta[j+1], rhobar[j],
// phibar[j]; CTA 0 writes index j+1 of the state, so no CTA reads a value
// another CTA of this launch writes. Each thread loads its UPT elements of W,
// X and V before thread 0's FP64 scalar chain, so the two latencies overlap.
// done_in (= done[j]) gates the launch; done_out (= done[j+1], read by every
// launch of the next step and by nothing in this one) is written by CTA 0.
// flags: [1] iterations, [2] status.
constexpr int UPT = 4;
__global__ void __launch_bounds__(NT)
k_lsqr_update(float* __restrict__ X, float* __restrict__ W, const float* __restrict__ V,
              float* __restrict__ basis_slot, size_t n, const double* alpha,
              const double* beta, double* rhobar, double* phibar, double* phibar_hist,
              double* rgiv, int j, double tol, int* flags, const int* done_in, int* done_out,
              const int* stop_at) {
  pdl_wait();
  if (*done_in) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *done_out = 1;
    return;
  }
  __shared__ float sh[4];
  __shared__ int sh_stop;
  const size_t base = (size_t)blockIdx.x * (NT * UPT) + threadIdx.x;
  float w[UPT], x[UPT], v[UPT];
#pragma unroll
  for (int u = 0; u < UPT; ++u) {
    const size_t i = base + (size_t)u * NT;
    w[u] = i < n ? W[i] : 0.f;
    x[u] = i < n ? X[i] : 0.f;
    v[u] = i < n ? V[i] : 0.f;
  }
  pdl_trigger();
  if (threadIdx.x == 0) {
    const double b = beta[j + 1], a = alpha[j + 1];
    const double rb = rhobar[j], pb = phibar[j];
    const double rho = hypot(rb, b);
    const double irho = 1.0 / rho;
    const double c = rb * irho, s = b * irho;
    const double theta = s * a;
    const double phi = c * pb;
    const double pbn = -s * pb;
    const bool finite = isfinite(a) && isfinite(b) && isfinite(rho);
    const bool brk = (a == 0.0);
    // converged, or reached the step count a learned predictor chose
    const bool conv = fabs(pbn) < tol || (stop_at && *stop_at > 0 && j + 1 >= *stop_at);
    sh[0] = (float)(phi * irho);
    sh[1] = brk ? 0.f : (float)(1.0 / a);
    sh[2] = (float)(theta * irho);
    sh_stop = brk || conv || !finite;
    if (blockIdx.x == 0) {
      rhobar[j + 1] = c * a;
      phibar[j + 1] = pbn;
      if (rgiv) {  // R_k and f_k of Q_k [C~_k beta_1 e_1] (§3.3): rho, theta, phi
        rgiv[3 * j] = rho;
        rgiv[3 * j + 1] = theta;
        rgiv[3 * j + 2] = phi;
      }
      if (phibar_hist) phibar_hist[j] = fabs(pbn);
      flags[1] = j + 1;
      if (!finite) flags[2] = TC_ENONFINITE;
      else if (brk) flags[2] = TC_EBREAKDOWN;
      else if (conv) flags[2] = 1;
      *done_out = (!finite || brk || conv) ? 1 : 0;
    }
  }
  __syncthreads();
  const float cx = sh[0], cv = sh[1], cw = sh[2];
  const bool stop = sh_stop;
#pragma unroll
  for (int u = 0; u < UPT; ++u) {
    const size_t i = base + (size_t)u * NT;
    if (i >= n) break;
    X[i] = fmaf(cx, w[u], x[u]);
    if (!stop) {
      const float vn = cv * v[u];
      W[i] = fmaf(-cw, w[u], vn);
      if (basis_slot) basis_slot[i] = vn;
    }
  }
}

// X = X0 + sum_{i<k} y_i V_i (V_i at basis + i*stride); k read from the device.
__global__ void __launch_bounds__(NT)
k_combine(float* X, const float* X0, const float* __restrict__ basis, size_t stride, int kmax,
          const int* kdev, const double* __restrict__ y, size_t n, const int* skip) {
  if (skip && *skip) return;
  __shared__ float ys[TC_MAX_PROJ];
  const int k = kdev ? min(*kdev, kmax) : kmax;
  for (int i = threadIdx.x; i < k; i += NT) ys[i] = (float)y[i];
  __syncthreads();
  const size_t st = (size_t)gridDim.x * NT;
  for (size_t i = (size_t)blockIdx.x * NT + threadIdx.x; i < n; i += st) {
    float acc = X0 ? X0[i] : 0.f;
    for (int q = 0; q < k; ++q) acc = fmaf(ys[q], __ldg(basis + q * stride + i), acc);
    X[i] = acc;
  }
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
  TC_CUDA(cudaFuncSetAttribute(k_lsqr_update, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_combine, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_mgs_pass, cudaFuncAttributePreferredSharedMemoryCarveout, c));
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

int launch_lsqr_update(float* X, float* W, const float* V, float* basis_slot, size_t n,
                       double* alpha, double* beta, double* rhobar, double* phibar,
                       double* phibar_hist, double* rgiv, int j, double tol, int* flags,
                       const int* done_in, int* done_out, cudaStream_t st,
                       const int* stop_at) {
  const size_t blocks = (n + (size_t)NT * UPT - 1) / ((size_t)NT * UPT);
  TC_CHECK(blocks >= 1 && blocks <= 0x7fffffffULL);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(NT);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TC_CUDA(cudaLaunchKernelEx(&cfg, k_lsqr_update, X, W, V, basis_slot, n, alpha, beta, rhobar,
                             phibar, phibar_hist, rgiv, j, tol, flags, done_in, done_out,
                             stop_at));
  return TC_OK;
}

int launch_combine(float* X, const float* X0, const float* basis, size_t stride, int kmax,
                   const int* kdev, const double* y, size_t n, const int* skip,
                   cudaStream_t st) {
  TC_CHECK(kmax <= TC_MAX_PROJ);
  k_combine<<<grid_for(n, 8), NT, 0, st>>>(X, X0, basis, stride, kmax, kdev, y, n, skip);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_mgs_pass(float* W, const float* Vi, const double* h, const float* Vnext,
                    size_t n, const Red& red, const int* skip, cudaStream_t st) {
  k_mgs_pass<<<grid_for(n, 16), NT, 0, st>>>(W, Vi, h, Vnext, n, red, skip);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
