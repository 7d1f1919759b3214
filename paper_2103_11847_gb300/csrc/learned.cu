// The learned stop index and lambda around c-LSQR: features of the first
// steps, the network on the device, training labels from exact errors, and
// the learned solve (see include/tcprod.h for the contract). The paper has no
// counterpart; the labels and the fallback use its quantities: the bidiagonal
// alpha, beta (Algorithm 4), the LSQR rotations rho, theta, phi, phibar
// (§3.3) and GCV (eq. (gcv2)).
#include <cuda_bf16.h>

#include "gcv_eval.cuh"
#include "mlp.cuh"

namespace {

constexpr int NGRID_L = 48;   // lambda values per stop index when labelling
constexpr int KSTEP = 2;      // candidate stop indices 4, 6, .., kmax

// The 36 features: log(alpha_i / beta_1), log(beta_{i+1} / beta_1),
// log(|phibar_{i+1}| / beta_1), i = 1..12 (alpha[0] = alpha_1, beta[0] = beta_1).
__device__ void features(const double* alpha, const double* beta, const double* phibar, float* f) {
  const double b1 = beta[0];
  for (int i = 0; i < MLP_FEAT_STEPS; ++i) {
    f[i] = (float)log(alpha[i] / b1);
    f[MLP_FEAT_STEPS + i] = (float)log(beta[i + 1] / b1);
    f[2 * MLP_FEAT_STEPS + i] = (float)log(fabs(phibar[i + 1]) / b1);
  }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

// Features -> normalise -> network -> denormalise -> lambda, stop index.
// One CTA of 64 threads.
__global__ void __launch_bounds__(MLP_HID)
k_learned_predict(const __nv_bfloat16* __restrict__ Wb, const float* __restrict__ theta,
                  const float* __restrict__ norm, const double* alpha, const double* beta,
                  const double* phibar, int kmax, double* lam_pred, int* stop_at) {
  constexpr int NI = MLP_IN, NH = MLP_HID, NO = MLP_OUT;
  constexpr int OB1 = NI * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH * NO;
  __shared__ float x[NI], h1[NH], h2[NH], out[NO];
  const int j = threadIdx.x;
  if (j == 0) {
    features(alpha, beta, phibar, x);
    for (int i = 0; i < NI; ++i) x[i] = (x[i] - norm[i]) / norm[NI + i];
  }
  __syncthreads();
  float z = theta[OB1 + j];
  for (int i = 0; i < NI; ++i) z = fmaf(x[i], __bfloat162float(Wb[i * NH + j]), z);
  h1[j] = gelu(z);
  __syncthreads();
  z = theta[OB2 + j];
  for (int i = 0; i < NH; ++i) z = fmaf(h1[i], __bfloat162float(Wb[OW2 + i * NH + j]), z);
  h2[j] = gelu(z);
  __syncthreads();
  if (j < NO) {
    float o = theta[OB3 + j];
    for (int i = 0; i < NH; ++i) o = fmaf(h2[i], __bfloat162float(Wb[OW3 + i * NO + j]), o);
    out[j] = o * norm[2 * NI + NO + j] + norm[2 * NI + j];
  }
  __syncthreads();
  if (j == 0) {
    *lam_pred = exp((double)out[0]);
    int k = (int)lrint(out[1]);
    k = max(MLP_FEAT_STEPS + 1, min(k, kmax));
    *stop_at = k;
  }
}

// Gram matrix of the kept basis and its inner products with X_true:
// G[a][b] = <V_a, V_b> (a <= b), c[a] = <V_a, X_true>, xx = ||X_true||^2.
// One CTA per entry, FP32 per-thread sums, FP64 tree: deterministic.
__global__ void __launch_bounds__(256)
k_gram(const float* __restrict__ V, size_t stride, size_t n, const float* __restrict__ Xt,
       int kmax, double* G, double* c, double* xx) {
  __shared__ double wsum[8];
  const int npairs = kmax * (kmax + 1) / 2;
  int q = blockIdx.x;
  const float *u, *v;
  double* dst;
  double* mirror = nullptr;
  if (q < npairs) {
    int a = 0;
    while (q >= kmax - a) {
      q -= kmax - a;
      ++a;
    }
    const int b = a + q;
    u = V + (size_t)a * stride;
    v = V + (size_t)b * stride;
    dst = G + (size_t)a * kmax + b;
    mirror = G + (size_t)b * kmax + a;
  } else if (q < npairs + kmax) {
    const int a = q - npairs;
    u = V + (size_t)a * stride;
    v = Xt;
    dst = c + a;
  } else {
    u = Xt;
    v = Xt;
    dst = xx;
  }
  float s = 0.f;
  for (size_t i = threadIdx.x; i < n; i += 256) s = fmaf(__ldg(u + i), __ldg(v + i), s);
  double d = s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += wsum[w];
    *dst = t;
    if (mirror) *mirror = t;  // the lower triangle
  }
}

// Labels: error(k, lambda) = y^T G_k y - 2 c_k^T y + ||X||^2 with
// y = y_k(lambda) from the rotations, on the grid k = 4, 6, .., kmax and
// NGRID_L log-spaced lambda in [1e-6, 1] ||C~_kmax||_F. CTA ki takes k = 4 +
// KSTEP ki, thread li one lambda (the O(k^2) FP64 work of the grid spread over
// the SMs); err[ki * NGRID_L + li].
__device__ double label_scale(const double* alpha, const double* beta, int kmax) {
  double s2 = 0.0;
  for (int j = 0; j < kmax; ++j) s2 += alpha[j] * alpha[j] + beta[j + 1] * beta[j + 1];
  return sqrt(s2);
}

__global__ void __launch_bounds__(64)
k_label_err(const double* rg, const double* alpha, const double* beta, const double* G,
            const double* c, const double* xx, int kmax, double* err) {
  __shared__ double sh_s;
  const int ki = blockIdx.x, li = threadIdx.x;
  if (li == 0) sh_s = label_scale(alpha, beta, kmax);
  __syncthreads();
  if (li >= NGRID_L) return;
  const double lo = log(sh_s) - 6.0 * log(10.0), hi = log(sh_s);
  const int k = 4 + KSTEP * ki;
  const double lam = exp(lo + (hi - lo) * li / (NGRID_L - 1));
  double y[TC_MAX_PROJ];
  gcv_bd_eval(rg, k, 0.0, lam, TC_GCV_FULL, y);
  double e = *xx;
  for (int a = 0; a < k; ++a) {
    double gy = 0.0;
    for (int b = 0; b < k; ++b) gy += G[(size_t)a * kmax + b] * y[b];
    e += y[a] * (gy - 2.0 * c[a]);
  }
  err[ki * NGRID_L + li] = e;
}

// The labels from the error grid: k_opt = the smallest k whose best error
// over lambda is within 1% of the best over all k, lambda_opt its minimiser;
// and the features of the first MLP_FEAT_STEPS steps. One thread.
__global__ void k_label_pick(const double* alpha, const double* beta, const double* phibar,
                             const double* err, int kmax, float* feat, float* target) {
  const int nk = (kmax - 4) / KSTEP + 1;
  const double s = label_scale(alpha, beta, kmax);
  const double lo = log(s) - 6.0 * log(10.0), hi = log(s);
  features(alpha, beta, phibar, feat);
  double best = INFINITY;
  for (int t = 0; t < nk * NGRID_L; ++t) best = fmin(best, err[t]);
  int kbest = nk - 1;
  for (int ki = 0; ki < nk; ++ki) {
    double m = INFINITY;
    for (int li = 0; li < NGRID_L; ++li) m = fmin(m, err[ki * NGRID_L + li]);
    if (m <= best * 1.0201) {  // error within 1%: squared errors within 1.01^2
      kbest = ki;
      break;
    }
  }
  int lb = 0;
  for (int li = 1; li < NGRID_L; ++li)
    if (err[kbest * NGRID_L + li] < err[kbest * NGRID_L + lb]) lb = li;
  target[0] = (float)(lo + (hi - lo) * lb / (NGRID_L - 1));
  target[1] = (float)(4 + KSTEP * kbest);
}

}  // namespace

int launch_learned_predict(const tc_mlp* m, const double* alpha, const double* beta,
                           const double* phibar, int kmax, double* lam_pred, int* stop_at,
                           cudaStream_t st) {
  k_learned_predict<<<1, MLP_HID, 0, st>>>(mlp_weights(m), mlp_theta(m), mlp_norm(m), alpha, beta,
                                           phibar, kmax, lam_pred, stop_at);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

extern "C" int tc_lsqr_label(tc_plan* p, const float* C, const float* X_true, int kmax, float* feat,
                             float* target, tc_stream_t stream) {
  if (!p || !C || !X_true || !feat || !target) return TC_EINVAL;
  if (kmax < MLP_FEAT_STEPS + 1 || kmax > TC_MAX_PROJ) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  TC_TRY(ensure_lsqr(p, kmax, true));
  // aux: X, X_reg (FP32), then G (kmax^2), c (kmax), ||X_true||^2, the error
  // grid (FP64), info
  const int nk = (kmax - 4) / KSTEP + 1;
  const size_t offG = ((2 * p->Tx * sizeof(float)) + 255) / 256 * 256;
  const size_t need =
      offG + ((size_t)kmax * kmax + kmax + 1 + (size_t)nk * NGRID_L) * sizeof(double) + 256;
  if (!p->aux || p->aux_bytes < need) {
    if (p->aux) cudaFree(p->aux);
    p->aux = nullptr;
    p->aux_bytes = 0;
    if (cudaMalloc(&p->aux, need) != cudaSuccess) return TC_ENOMEM;
    p->aux_bytes = need;
  }
  unsigned char* base = static_cast<unsigned char*>(p->aux);
  float* X = reinterpret_cast<float*>(base);
  float* Xr = X + p->Tx;
  double* G = reinterpret_cast<double*>(base + offG);
  double* c = G + (size_t)kmax * kmax;
  double* xx = c + kmax;
  double* err = xx + 1;
  tc_solve_info* info =
      reinterpret_cast<tc_solve_info*>(base + (need - 256 + 0));  // 256-byte slot at the end
  LsqrArgs a{C, X, Xr, kmax, 0.0, 0.0, nullptr, info};
  a.spatial_basis = 1;  // the labels compare the basis with X_true
  TC_TRY(lsqr_enqueue(p, a, st));
  const size_t L = (size_t)kmax + 2;
  double* alpha = p->dscal;
  double* beta = alpha + L;
  double* phibar = beta + 2 * L;
  double* rgiv = phibar + L;
  const int blocks = kmax * (kmax + 1) / 2 + kmax + 1;
  k_gram<<<blocks, 256, 0, st>>>(p->basis, p->Tx, p->Tx, X_true, kmax, G, c, xx);
  TC_CUDA(cudaGetLastError());
  k_label_err<<<nk, 64, 0, st>>>(rgiv, alpha, beta, G, c, xx, kmax, err);
  TC_CUDA(cudaGetLastError());
  k_label_pick<<<1, 1, 0, st>>>(alpha, beta, phibar, err, kmax, feat, target);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

extern "C" int tc_lsqr_c_learned(tc_plan* p, const tc_mlp* m, const float* C, float* X,
                                 float* X_reg, int kmax, double gcv_factor, tc_solve_info* info,
                                 tc_stream_t stream) {
  if (!p || !m || !C || !X || !X_reg || !info) return TC_EINVAL;
  if (kmax < MLP_FEAT_STEPS + 1 || kmax > TC_MAX_PROJ || !(gcv_factor >= 1.0)) return TC_EINVAL;
  TC_TRY(ensure_lsqr(p, kmax, true));
  LsqrArgs a{C, X, X_reg, kmax, 0.0, -1.0, nullptr, info, m, gcv_factor};
  return lsqr_enqueue(p, a, (cudaStream_t)stream);
}
