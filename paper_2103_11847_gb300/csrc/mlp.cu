// The learned-lambda network: 36 -> 64 -> 64 -> 2 with GELU, FP32 master
// weights, BF16 weight copies used by the forward pass, FP32 accumulation.
// It maps features of the first c-LSQR steps to (log lambda, stop index) and
// stands in for the GCV search of §3.1 and the stopping choice of §3.3. The
// paper has no such network.
//
// Parameters are one flat FP32 vector, W1 (36 x 64, row-major in x out), b1,
// W2 (64 x 64), b2, W3 (64 x 2), b3. The loss is (1/2B) sum (out - t)^2. All
// reductions over the batch run in a fixed order, so training is deterministic.
#include <cuda_bf16.h>

#include <new>
#include <vector>

#include "tc_device.cuh"
#include "mlp.cuh"

namespace {

constexpr int NI = MLP_IN, NH = MLP_HID, NO = MLP_OUT;
constexpr int OW1 = 0, OB1 = OW1 + NI * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NO;
static_assert(OB3 + NO == MLP_NPARAMS, "parameter layout");

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// One CTA of 64 threads per sample: z1, h1, z2, h2, out (saved for backward).
__global__ void __launch_bounds__(NH)
k_mlp_fwd(const float* __restrict__ X, int B, const __nv_bfloat16* __restrict__ Wb,
          const float* __restrict__ theta, float* Z1, float* H1, float* Z2, float* H2, float* OUT) {
  __shared__ float x[NI], h1[NH], h2[NH];
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= B) return;
  for (int i = j; i < NI; i += NH) x[i] = X[(size_t)b * NI + i];
  __syncthreads();
  float z = theta[OB1 + j];
  for (int i = 0; i < NI; ++i) z = fmaf(x[i], __bfloat162float(Wb[OW1 + i * NH + j]), z);
  h1[j] = gelu(z);
  if (Z1) { Z1[(size_t)b * NH + j] = z; H1[(size_t)b * NH + j] = h1[j]; }
  __syncthreads();
  z = theta[OB2 + j];
  for (int i = 0; i < NH; ++i) z = fmaf(h1[i], __bfloat162float(Wb[OW2 + i * NH + j]), z);
  h2[j] = gelu(z);
  if (Z2) { Z2[(size_t)b * NH + j] = z; H2[(size_t)b * NH + j] = h2[j]; }
  __syncthreads();
  if (j < NO) {
    float o = theta[OB3 + j];
    for (int i = 0; i < NH; ++i) o = fmaf(h2[i], __bfloat162float(Wb[OW3 + i * NO + j]), o);
    OUT[(size_t)b * NO + j] = o;
  }
}

// Backward through the activations, one CTA per sample: D = (out - t) / B,
// dZ2 = (D W3^T) * gelu'(z2), dZ1 = (dZ2 W2^T) * gelu'(z1); per-sample loss.
__global__ void __launch_bounds__(NH)
k_mlp_bwd_act(const float* __restrict__ T, int B, const __nv_bfloat16* __restrict__ Wb,
              const float* Z1, const float* Z2, const float* OUT, float* D, float* dZ1,
              float* dZ2, float* lossb) {
  __shared__ float d[NO], dz2[NH];
  const int b = blockIdx.x, j = threadIdx.x;
  if (j < NO) {
    const float r = OUT[(size_t)b * NO + j] - T[(size_t)b * NO + j];
    d[j] = r / B;
    D[(size_t)b * NO + j] = r / B;
  }
  if (j == 0) {
    float l = 0.f;
    for (int o = 0; o < NO; ++o) {
      const float r = OUT[(size_t)b * NO + o] - T[(size_t)b * NO + o];
      l = fmaf(r, r, l);
    }
    lossb[b] = 0.5f * l / B;
  }
  __syncthreads();
  float g = 0.f;
  for (int o = 0; o < NO; ++o) g = fmaf(d[o], __bfloat162float(Wb[OW3 + j * NO + o]), g);
  dz2[j] = g * gelu_d(Z2[(size_t)b * NH + j]);
  dZ2[(size_t)b * NH + j] = dz2[j];
  __syncthreads();
  g = 0.f;
  for (int k = 0; k < NH; ++k) g = fmaf(dz2[k], __bfloat162float(Wb[OW2 + j * NH + k]), g);
  dZ1[(size_t)b * NH + j] = g * gelu_d(Z1[(size_t)b * NH + j]);
}

// Weight gradients, one thread per parameter, batch summed in order.
__global__ void k_mlp_bwd_w(const float* __restrict__ X, int B, const float* H1, const float* H2,
                            const float* D, const float* dZ1, const float* dZ2,
                            const float* lossb, float* grad, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss) {
    float l = 0.f;
    for (int b = 0; b < B; ++b) l += lossb[b];
    *loss = l;
  }
  if (p >= MLP_NPARAMS) return;
  float s = 0.f;
  if (p < OB1) {
    const int i = p / NH, j = p % NH;
    for (int b = 0; b < B; ++b) s = fmaf(X[(size_t)b * NI + i], dZ1[(size_t)b * NH + j], s);
  } else if (p < OW2) {
    const int j = p - OB1;
    for (int b = 0; b < B; ++b) s += dZ1[(size_t)b * NH + j];
  } else if (p < OB2) {
    const int i = (p - OW2) / NH, j = (p - OW2) % NH;
    for (int b = 0; b < B; ++b) s = fmaf(H1[(size_t)b * NH + i], dZ2[(size_t)b * NH + j], s);
  } else if (p < OW3) {
    const int j = p - OB2;
    for (int b = 0; b < B; ++b) s += dZ2[(size_t)b * NH + j];
  } else if (p < OB3) {
    const int i = (p - OW3) / NO, o = (p - OW3) % NO;
    for (int b = 0; b < B; ++b) s = fmaf(H2[(size_t)b * NH + i], D[(size_t)b * NO + o], s);
  } else {
    const int o = p - OB3;
    for (int b = 0; b < B; ++b) s += D[(size_t)b * NO + o];
  }
  grad[p] = s;
}

// Adam (bias-corrected); refreshes the BF16 copies of the weight matrices.
__global__ void k_adam(float* theta, const float* grad, float* m, float* v, int t, float lr,
                       __nv_bfloat16* Wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAMS) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float g = grad[p];
  const float mm = b1 * m[p] + (1.f - b1) * g;
  const float vv = b2 * v[p] + (1.f - b2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.f - powf(b1, (float)t));
  const float vh = vv / (1.f - powf(b2, (float)t));
  const float th = theta[p] - lr * mh / (sqrtf(vh) + eps);
  theta[p] = th;
  Wb[p] = __float2bfloat16_rn(th);
}

__global__ void k_to_bf16(const float* theta, __nv_bfloat16* Wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < MLP_NPARAMS) Wb[p] = __float2bfloat16_rn(theta[p]);
}

// Deterministic pseudo-random initialisation (splitmix64), scaled by 1/sqrt(fan_in).
__global__ void k_init(float* theta, unsigned long long seed) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAMS) return;
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(p + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const float u = (float)((z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;  // U(-1, 1)
  float scale = 0.f;
  if (p < OB1) scale = rsqrtf((float)NI);
  else if (p >= OW2 && p < OB2) scale = rsqrtf((float)NH);
  else if (p >= OW3 && p < OB3) scale = rsqrtf((float)NH);
  theta[p] = u * scale * 1.7320508f;  // unit variance times 1/sqrt(fan_in)
}

}  // namespace

struct tc_mlp {
  float* theta = nullptr;  // FP32 master parameters
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* Wb = nullptr;  // BF16 copy (biases too, unused)
  float* norm = nullptr;        // x mean[36], x std[36], t mean[2], t std[2]
  float* work = nullptr;        // activations for up to kMaxB samples
  float* loss = nullptr;
  int step = 0;
};

namespace {
constexpr int kMaxB = 1024;
constexpr size_t kWork = (size_t)kMaxB * (4 * NH + 2 * NO + NH * 2 + 1);
}  // namespace

extern "C" int tc_mlp_create(tc_mlp** out, unsigned long long seed, tc_stream_t stream) {
  if (!out) return TC_EINVAL;
  tc_mlp* m = new (std::nothrow) tc_mlp();
  if (!m) return TC_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  bool ok = cudaMalloc(&m->theta, MLP_NPARAMS * 4) == cudaSuccess &&
            cudaMalloc(&m->m, MLP_NPARAMS * 4) == cudaSuccess &&
            cudaMalloc(&m->v, MLP_NPARAMS * 4) == cudaSuccess &&
            cudaMalloc(&m->grad, MLP_NPARAMS * 4) == cudaSuccess &&
            cudaMalloc(&m->Wb, MLP_NPARAMS * 2) == cudaSuccess &&
            cudaMalloc(&m->norm, MLP_NORM * 4) == cudaSuccess &&
            cudaMalloc(&m->work, kWork * 4) == cudaSuccess &&
            cudaMalloc(&m->loss, 4) == cudaSuccess;
  if (!ok) {
    tc_mlp_destroy(m);
    return TC_ENOMEM;
  }
  TC_CUDA(cudaMemsetAsync(m->m, 0, MLP_NPARAMS * 4, st));
  TC_CUDA(cudaMemsetAsync(m->v, 0, MLP_NPARAMS * 4, st));
  std::vector<float> nrm(MLP_NORM, 0.f);
  for (int i = 0; i < MLP_IN; ++i) nrm[MLP_IN + i] = 1.f;
  nrm[2 * MLP_IN + 2] = nrm[2 * MLP_IN + 3] = 1.f;
  TC_CUDA(cudaMemcpyAsync(m->norm, nrm.data(), MLP_NORM * 4, cudaMemcpyHostToDevice, st));
  k_init<<<(MLP_NPARAMS + 255) / 256, 256, 0, st>>>(m->theta, seed);
  k_to_bf16<<<(MLP_NPARAMS + 255) / 256, 256, 0, st>>>(m->theta, m->Wb);
  TC_CUDA(cudaGetLastError());
  TC_CUDA(cudaStreamSynchronize(st));
  *out = m;
  return TC_OK;
}

extern "C" int tc_mlp_destroy(tc_mlp* m) {
  if (!m) return TC_EINVAL;
  void* ps[] = {m->theta, m->m, m->v, m->grad, m->Wb, m->norm, m->work, m->loss};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete m;
  return TC_OK;
}

extern "C" int tc_mlp_set_params(tc_mlp* m, const float* theta, const float* norm,
                                 tc_stream_t stream) {
  if (!m || (!theta && !norm)) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (theta) {
    TC_CUDA(cudaMemcpyAsync(m->theta, theta, MLP_NPARAMS * 4, cudaMemcpyDeviceToDevice, st));
    k_to_bf16<<<(MLP_NPARAMS + 255) / 256, 256, 0, st>>>(m->theta, m->Wb);
    TC_CUDA(cudaGetLastError());
    TC_CUDA(cudaMemsetAsync(m->m, 0, MLP_NPARAMS * 4, st));
    TC_CUDA(cudaMemsetAsync(m->v, 0, MLP_NPARAMS * 4, st));
    m->step = 0;
  }
  if (norm) TC_CUDA(cudaMemcpyAsync(m->norm, norm, MLP_NORM * 4, cudaMemcpyDeviceToDevice, st));
  return TC_OK;
}

extern "C" int tc_mlp_get_params(tc_mlp* m, float* theta, float* norm, tc_stream_t stream) {
  if (!m || (!theta && !norm)) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (theta) TC_CUDA(cudaMemcpyAsync(theta, m->theta, MLP_NPARAMS * 4, cudaMemcpyDeviceToDevice, st));
  if (norm) TC_CUDA(cudaMemcpyAsync(norm, m->norm, MLP_NORM * 4, cudaMemcpyDeviceToDevice, st));
  return TC_OK;
}

namespace {
int fwd_bwd(tc_mlp* m, const float* X, const float* T, int B, float* grad, float* loss,
            cudaStream_t st) {
  float* Z1 = m->work;
  float* H1 = Z1 + (size_t)kMaxB * NH;
  float* Z2 = H1 + (size_t)kMaxB * NH;
  float* H2 = Z2 + (size_t)kMaxB * NH;
  float* OUT = H2 + (size_t)kMaxB * NH;
  float* D = OUT + (size_t)kMaxB * NO;
  float* dZ1 = D + (size_t)kMaxB * NO;
  float* dZ2 = dZ1 + (size_t)kMaxB * NH;
  float* lossb = dZ2 + (size_t)kMaxB * NH;
  k_mlp_fwd<<<B, NH, 0, st>>>(X, B, m->Wb, m->theta, Z1, H1, Z2, H2, OUT);
  k_mlp_bwd_act<<<B, NH, 0, st>>>(T, B, m->Wb, Z1, Z2, OUT, D, dZ1, dZ2, lossb);
  k_mlp_bwd_w<<<(MLP_NPARAMS + 255) / 256, 256, 0, st>>>(X, B, H1, H2, D, dZ1, dZ2, lossb, grad,
                                                         loss);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
}  // namespace

extern "C" int tc_mlp_loss_grad(tc_mlp* m, const float* X, const float* T, int B, float* loss,
                                float* grad, tc_stream_t stream) {
  if (!m || !X || !T || !grad || B < 1 || B > kMaxB) return TC_EINVAL;
  return fwd_bwd(m, X, T, B, grad, loss, (cudaStream_t)stream);
}

extern "C" int tc_mlp_forward(tc_mlp* m, const float* X, int B, float* Y, tc_stream_t stream) {
  if (!m || !X || !Y || B < 1) return TC_EINVAL;
  k_mlp_fwd<<<B, NH, 0, (cudaStream_t)stream>>>(X, B, m->Wb, m->theta, nullptr, nullptr, nullptr,
                                                nullptr, Y);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

extern "C" int tc_mlp_train(tc_mlp* m, const float* X, const float* T, int N, int batch, int steps,
                            float lr, float* loss_hist, tc_stream_t stream) {
  if (!m || !X || !T || N < 1 || batch < 1 || batch > kMaxB || steps < 1 || !(lr > 0.f))
    return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int off = 0;
  for (int s = 0; s < steps; ++s) {
    const int B = (off + batch <= N) ? batch : N - off;
    TC_TRY(fwd_bwd(m, X + (size_t)off * MLP_IN, T + (size_t)off * MLP_OUT, B, m->grad,
                   loss_hist ? loss_hist + s : m->loss, st));
    ++m->step;
    k_adam<<<(MLP_NPARAMS + 255) / 256, 256, 0, st>>>(m->theta, m->grad, m->m, m->v, m->step, lr,
                                                      m->Wb);
    TC_CUDA(cudaGetLastError());
    off += B;
    if (off >= N) off = 0;
  }
  return TC_OK;
}

namespace {
// Column means and standard deviations of R (N x ncol) into stats[0..ncol)
// and stats[ncol..2 ncol); then R_out = (R - mean) / std. One CTA per column.
__global__ void k_colstats(const float* R, int N, int ncol, float* mean, float* stdv, float* R_out) {
  __shared__ double s1[256], s2[256];
  const int c = blockIdx.x, t = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (int i = t; i < N; i += 256) {
    const double v = R[(size_t)i * ncol + c];
    a += v;
    b += v * v;
  }
  s1[t] = a;
  s2[t] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) {
      s1[t] += s1[t + o];
      s2[t] += s2[t + o];
    }
    __syncthreads();
  }
  __shared__ float mu, sd;
  if (t == 0) {
    const double m = s1[0] / N;
    const double var = fmax(s2[0] / N - m * m, 0.0);
    mu = (float)m;
    sd = (float)(var > 1e-12 ? sqrt(var) : 1.0);
    mean[c] = mu;
    stdv[c] = sd;
  }
  __syncthreads();
  for (int i = t; i < N; i += 256) R_out[(size_t)i * ncol + c] = (R[(size_t)i * ncol + c] - mu) / sd;
}
}  // namespace

extern "C" int tc_mlp_fit_norm(tc_mlp* m, const float* Xraw, const float* Traw, int N, float* Xn,
                               float* Tn, tc_stream_t stream) {
  if (!m || !Xraw || !Traw || !Xn || !Tn || N < 2) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  k_colstats<<<MLP_IN, 256, 0, st>>>(Xraw, N, MLP_IN, m->norm, m->norm + MLP_IN, Xn);
  k_colstats<<<MLP_OUT, 256, 0, st>>>(Traw, N, MLP_OUT, m->norm + 2 * MLP_IN,
                                       m->norm + 2 * MLP_IN + MLP_OUT, Tn);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// device-side inference used by the learned solve (learned.cu)
const __nv_bfloat16* mlp_weights(const tc_mlp* m) { return m->Wb; }
const float* mlp_theta(const tc_mlp* m) { return m->theta; }
const float* mlp_norm(const tc_mlp* m) { return m->norm; }
