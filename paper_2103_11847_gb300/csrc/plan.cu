// Plans and the two products of the library (Algorithm 1 with the transform M
// of Remark 2.1, and its adjoint), plus the error strings of the C ABI.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "tc_device.cuh"
#include "umma.cuh"

namespace {
thread_local char g_err[512] = "";

// Orthonormal DCT-II matrix C_n (eq. (dft1), §2.1), 0-based indices.
void dct2(int n, std::vector<double>& C) {
  const double pi = 3.14159265358979323846;
  C.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      C[(size_t)i * n + j] = std::sqrt((i == 0 ? 1.0 : 2.0) / n) *
                             std::cos(i * (2.0 * j + 1.0) * pi / (2.0 * n));
}

// M = W^{-1} C (I + Z) and its inverse M^{-1} = (I + Z)^{-1} C^T W in FP64
// (Remark 2.1). (I + Z)^{-1} is upper triangular with entries (-1)^{c-r}, so
// the inverse is formed in closed form rather than by a factorisation.
void transform_pair(int n, std::vector<double>& M, std::vector<double>& Mi) {
  std::vector<double> C;
  dct2(n, C);
  M.assign((size_t)n * n, 0.0);
  Mi.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    const double w = C[(size_t)i * n];
    for (int j = 0; j < n; ++j) {
      const double cij = C[(size_t)i * n + j] + (j > 0 ? C[(size_t)i * n + j - 1] : 0.0);
      M[(size_t)i * n + j] = cij / w;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int r = i; r < n; ++r) s += (((r - i) & 1) ? -1.0 : 1.0) * C[(size_t)j * n + r];
      Mi[(size_t)i * n + j] = s * C[(size_t)j * n];
    }
}

__global__ void k_transpose_slices(const float* __restrict__ in, float* out, int R, int Cc,
                                   const int* skip) {
  if (skip && *skip) return;
  __shared__ float t[32][33];
  const size_t so = (size_t)blockIdx.z * R * Cc;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < Cc) t[i][threadIdx.x] = in[so + (size_t)r * Cc + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < Cc) out[so + (size_t)c * R + r] = t[threadIdx.x][i];
  }
}

int transpose_slices(const float* in, float* out, int R, int Cc, int n3, cudaStream_t st,
                     const int* skip = nullptr) {
  dim3 grid((Cc + 31) / 32, (R + 31) / 32, n3);
  k_transpose_slices<<<grid, dim3(32, 8), 0, st>>>(in, out, R, Cc, skip);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

template <class T>
int dalloc(T** p, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    tc_set_error("cudaMalloc", e);
    return TC_ENOMEM;
  }
  return TC_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

bool fused(const tc_plan* p) { return p->n3 <= TC_MAX_FUSED && p->opts.precision == TC_FP32; }
bool lowp(const tc_plan* p) { return p->opts.precision != TC_FP32; }
bool x3(const tc_plan* p) { return p->opts.precision == TC_BF16X3; }
// operand type of the plan's tensor-core GEMMs (RoundKind)
int rkind(const tc_plan* p) {
  return x3(p) ? ROUND_BF16X3 : (p->opts.precision == TC_BF16 ? ROUND_BF16 : ROUND_TF32);
}
// where the rounded operand of the tensor-core GEMMs lives
void* lowop(const tc_plan* p) { return x3(p) ? p->lowX : (void*)p->tmp1; }
}  // namespace

void tc_set_error(const char* what, cudaError_t e) {
  std::snprintf(g_err, sizeof(g_err), "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
}

void tc_set_message(const char* msg) { std::snprintf(g_err, sizeof(g_err), "%s", msg); }

extern "C" const char* tc_last_error(void) { return g_err; }
extern "C" const char* tc_version(void) { return "tcprod 0.1 (sm_103a)"; }

Red make_red(tc_plan* p, double* out, int sqrt_out, const float* other, int* status) {
  Red r;
  r.out = out;
  r.sqrt_out = sqrt_out;
  r.other = other;
  r.partials = p->scratch.partials;
  r.ticket = p->scratch.tickets;
  r.status = status;
  return r;
}

namespace {
// The right factor of a two-sided product on the tensor cores: the first
// GEMM's result T (FP32, tmp2, `n` values) is rounded to the GEMM input type
// into the operand buffer (free once the first GEMM has read its operand;
// TF32: T is already K-major as the left operand), then tmp2 = T_k B~_k (or
// T_k B~_k^T) by the second GEMM `m`.
int right_factor(tc_plan* p, const UmmaMaps& m, size_t n, int* err, const int* skip,
                 cudaStream_t st) {
  TC_TRY(launch_round(p->tmp2, lowop(p), n, rkind(p), st, skip));
  return launch_umma(m, p->tmp2, err, skip, st);
}
}  // namespace

// Y = A *c X [*c B] with the epilogue `ep` on the last stage.
int cprod_epi(tc_plan* p, const float* X, float* Y, const Epi& ep, cudaStream_t st,
              const LsqrStep* step, const Chain* ch) {
  const bool ready = ch && ch->in_ready && p->store_bf16;
  const float* next_T = (ch && p->store_bf16) ? ch->next_T : nullptr;
  const int n1 = p->n1, n2 = p->n2, s = p->s, n3 = p->n3;
  if (fused(p) && p->two_sided && cprod2_fits(s))  // the step runs inside the product
    return launch_cprod2(p->AhT, X, p->Bh, Y, n1, n2, s, n3, p->hM, p->hMinv, ep,
                         step ? *step : LsqrStep{}, st);
  if (step) TC_TRY(step->X ? launch_lsqr_update(*step, st) : launch_lsqr_scalars(*step, st));
  Epi mid;
  mid.skip = ep.skip;
  if (fused(p)) {
    if (!p->two_sided)
      return launch_slice_gemm(p->Ah, X, Y, n1, s, n2, n3, p->hM, p->hMinv, ep, st);
    TC_TRY(launch_slice_gemm(p->Ah, X, p->tmp1, n1, s, n2, n3, p->hM, nullptr, mid, st));
    return launch_slice_gemm(p->tmp1, p->Bh, Y, n1, s, s, n3, nullptr, p->hMinv, ep, st);
  }
  if (lowp(p)) {  // transform to the GEMM input type, tcgen05 slice GEMMs, transform back
    int* err = ep.red.status ? ep.red.status : p->dev_err;
    const bool tct = n3 > TC_TUBE_MIN_N3;
    const size_t P = (size_t)n2 * s;
    if (ready) {  // the pass back of the product before wrote bf16(X x_3 M)
    } else if (tct) {
      TC_TRY(launch_mode3_tc_lowp(X, lowop(p), p->dM, n3, P, rkind(p), ep.skip, err, st));
    } else if (x3(p)) {  // the exact FP32 pass, then the three planes
      TC_TRY(launch_mode3(X, p->tmp2, p->dM, n3, P, mid, st));
      TC_TRY(launch_round(p->tmp2, p->lowX, P * n3, ROUND_BF16X3, st, ep.skip));
    } else {
      TC_TRY(launch_mode3_lowp(X, p->tmp1, p->dM, n3, P, rkind(p) == ROUND_BF16, ep.skip, st));
    }
    if (p->tmp3) TC_TRY(transpose_slices(p->tmp1, p->tmp3, n2, s, n3, st, ep.skip));
    if (p->store_bf16) {  // BF16 slice products, read back by the BF16-input pass
      TC_TRY(launch_umma(*p->umf, p->tmp2, err, ep.skip, st, true));
      if (next_T)
        return launch_mode3_tc_chain(p->tmp2, Y, p->dMinv, lowop(p), next_T, n3, (size_t)n1 * s,
                                     ep, err, st, nullptr);
      return launch_mode3_tc_inb(p->tmp2, Y, p->dMinv, n3, (size_t)n1 * s, ep, err, st, nullptr);
    }
    TC_TRY(launch_umma(*p->umf, p->tmp2, err, ep.skip, st));
    if (p->two_sided) TC_TRY(right_factor(p, *p->umf2, (size_t)n1 * s * n3, err, ep.skip, st));
    return tct ? launch_mode3_tc(p->tmp2, Y, p->dMinv, n3, (size_t)n1 * s, ep, err, st, x3(p))
               : launch_mode3(p->tmp2, Y, p->dMinv, n3, (size_t)n1 * s, ep, st);
  }
  TC_TRY(launch_mode3(X, p->tmp1, p->dM, n3, (size_t)n2 * s, mid, st));
  TC_TRY(launch_slice_gemm(p->Ah, p->tmp1, p->tmp2, n1, s, n2, n3, nullptr, nullptr, mid, st));
  const float* src = p->tmp2;
  if (p->two_sided) {
    TC_TRY(launch_slice_gemm(p->tmp2, p->Bh, p->tmp1, n1, s, s, n3, nullptr, nullptr, mid, st));
    src = p->tmp1;
  }
  return launch_mode3(src, Y, p->dMinv, n3, (size_t)n1 * s, ep, st);
}

// Transform-domain products (ORTHODCT plans off the fused route): the
// operand and result stay in the transform domain, so a product is the slice
// GEMMs plus the epilogue pass. The DCT is orthogonal, so Definition 2.2's
// inner products and norms are the same there, and LSQR can run on the
// transformed tensors throughout.
bool td_route(const tc_plan* p) {
  return p->opts.product == TC_ORTHODCT && !fused(p) && p->opts.route != TC_ROUTE_SPATIAL;
}

// Dual-domain route (TH product, BF16, one-sided, 32 < n3 <= 64): V is kept
// as V x_3 M^{-T} and U as U x_3 M. The forward product is facewise in the
// M domain and the exact adjoint (M^T [A~_k^T (Y x_3 M^{-T})_k]) is facewise
// in the M^{-T} domain, so each product is one slice GEMM plus one change of
// domain, by G = M^{-T} M^{-1} (U) or G^{-1} = M M^T (V); the norm of the
// spatial tensor is ||U x_3 M^{-1}|| (||V x_3 M^T||), formed in the same pass.
bool thd_route(const tc_plan* p) {
  return p->opts.product == TC_TH && p->opts.precision == TC_BF16 && !p->two_sided &&
         p->n3 > TC_TUBE_MIN_N3 && p->n3 <= 64 && p->opts.route == TC_ROUTE_DUAL;
}

int cprod_td(tc_plan* p, const float* Xt, float* Yt, const Epi& ep, cudaStream_t st) {
  const int n1 = p->n1, n2 = p->n2, s = p->s, n3 = p->n3;
  Epi mid;
  mid.skip = ep.skip;
  const float* src = p->tmp2;
  if (lowp(p)) {
    int* err = ep.red.status ? ep.red.status : p->dev_err;
    TC_TRY(launch_round(Xt, lowop(p), (size_t)n2 * s * n3, rkind(p), st, ep.skip));
    if (p->tmp3) TC_TRY(transpose_slices(p->tmp1, p->tmp3, n2, s, n3, st, ep.skip));
    TC_TRY(launch_umma(*p->umf, p->tmp2, err, ep.skip, st));
    if (p->two_sided) TC_TRY(right_factor(p, *p->umf2, (size_t)n1 * s * n3, err, ep.skip, st));
  } else {
    TC_TRY(launch_slice_gemm(p->Ah, Xt, p->tmp2, n1, s, n2, n3, nullptr, nullptr, mid, st));
    if (p->two_sided) {
      TC_TRY(launch_slice_gemm(p->tmp2, p->Bh, p->tmp1, n1, s, s, n3, nullptr, nullptr, mid, st));
      src = p->tmp1;
    }
  }
  return launch_epi(src, Yt, p->Ty, ep, st);
}

// BF16 transform-domain products with the epilogue in the GEMM store (plans
// with umf_td): the forward GEMM reads bf16(V~) from lowV and writes U~ and
// bf16(U~) to lowU; the adjoint reads lowU and writes V~ and lowV.
int cprod_tdf(tc_plan* p, float* Yt, const Epi& ep, cudaStream_t st) {
  int* err = ep.red.status ? ep.red.status : p->dev_err;
  return launch_umma_epi(*p->umf_td, Yt, static_cast<__nv_bfloat16*>(p->lowU), ep, err, st);
}

int adjoint_tdf(tc_plan* p, float* Xt, const Epi& ep, cudaStream_t st) {
  int* err = ep.red.status ? ep.red.status : p->dev_err;
  return launch_umma_epi(*p->uma_td, Xt, static_cast<__nv_bfloat16*>(p->lowV), ep, err, st);
}

// Dual-domain products (thd_route). Forward: U^ = ca A~ V^ + cp prev in the
// M domain (the GEMM reads bf16(V^) from lowV, the Krylov update is in its
// store), then one pass writes lowU = bf16(U^ x_3 G), the adjoint's operand
// in the M^{-T} domain, and reduces ||U^ x_3 M^{-1}||^2 = ||U||^2 into
// ep.red. Adjoint: V' = ca A~^T U' + cp prev in the M^{-T} domain, then
// lowV = bf16(V' x_3 G^{-1}) and ||V' x_3 M^T||^2 = ||V||^2; `after` (an
// LSQR step's scalars) runs once that norm is in place.
int cprod_thd(tc_plan* p, float* Yt, const Epi& ep, cudaStream_t st) {
  int* err = ep.red.status ? ep.red.status : p->dev_err;
  Epi g = ep;
  g.red = Red{};
  TC_TRY(launch_umma_epi(*p->umf_td, Yt, nullptr, g, err, st));
  Epi n;
  n.red = ep.red;
  n.skip = ep.skip;
  return launch_mode3_tc_norm(Yt, p->lowU, p->dG, p->dMinv, p->n3, (size_t)p->n1 * p->s, n, err,
                              st, nullptr);
}

int adjoint_thd(tc_plan* p, float* Xt, const Epi& ep, cudaStream_t st, const LsqrStep* after) {
  int* err = ep.red.status ? ep.red.status : p->dev_err;
  Epi g = ep;
  g.red = Red{};
  TC_TRY(launch_umma_epi(*p->uma_td, Xt, nullptr, g, err, st));
  Epi n;
  n.red = ep.red;
  n.skip = ep.skip;
  return launch_mode3_tc_norm(Xt, p->lowV, p->dGi, p->dMT, p->n3, (size_t)p->n2 * p->s, n, err,
                              st, after);
}

int adjoint_td(tc_plan* p, const float* Yt, float* Xt, const Epi& ep, cudaStream_t st) {
  const int n1 = p->n1, n2 = p->n2, s = p->s, n3 = p->n3;
  Epi mid;
  mid.skip = ep.skip;
  const float* src = p->tmp2;
  if (lowp(p)) {
    int* err = ep.red.status ? ep.red.status : p->dev_err;
    TC_TRY(launch_round(Yt, lowop(p), (size_t)n1 * s * n3, rkind(p), st, ep.skip));
    if (p->tmp3) TC_TRY(transpose_slices(p->tmp1, p->tmp3, n1, s, n3, st, ep.skip));
    TC_TRY(launch_umma(*p->uma, p->tmp2, err, ep.skip, st));
    if (p->two_sided) TC_TRY(right_factor(p, *p->uma2, (size_t)n2 * s * n3, err, ep.skip, st));
  } else {
    TC_TRY(launch_slice_gemm(p->AhT, Yt, p->tmp2, n2, s, n1, n3, nullptr, nullptr, mid, st));
    if (p->two_sided) {
      TC_TRY(launch_slice_gemm(p->tmp2, p->BhT, p->tmp1, n2, s, s, n3, nullptr, nullptr, mid, st));
      src = p->tmp1;
    }
  }
  return launch_epi(src, Xt, p->Tx, ep, st);
}

// X = M^T [ A~_k^T (M^{-T} Y)_k (B~_k^T) ] with the epilogue `ep` on the last stage.
int adjoint_epi(tc_plan* p, const float* Y, float* X, const Epi& ep, cudaStream_t st,
                const LsqrStep* after, const Chain* ch) {
  if (after && !(lowp(p) && p->n3 > TC_TUBE_MIN_N3)) {  // the step's own launch after the product
    TC_TRY(adjoint_epi(p, Y, X, ep, st, nullptr, ch));
    return launch_lsqr_scalars(*after, st);
  }
  const bool ready = ch && ch->in_ready && p->store_bf16;
  const float* next_T = (ch && p->store_bf16) ? ch->next_T : nullptr;
  const int n1 = p->n1, n2 = p->n2, s = p->s, n3 = p->n3;
  Epi mid;
  mid.skip = ep.skip;
  if (fused(p)) {
    if (!p->two_sided)
      return launch_slice_gemm(p->AhT, Y, X, n2, s, n1, n3, p->hMinvT, p->hMT, ep, st);
    if (cprod2_fits(s))
      return launch_cprod2(p->Ah, Y, p->BhT, X, n2, n1, s, n3, p->hMinvT, p->hMT, ep,
                           LsqrStep{}, st);
    TC_TRY(launch_slice_gemm(p->AhT, Y, p->tmp1, n2, s, n1, n3, p->hMinvT, nullptr, mid, st));
    return launch_slice_gemm(p->tmp1, p->BhT, X, n2, s, s, n3, nullptr, p->hMT, ep, st);
  }
  if (lowp(p)) {
    int* err = ep.red.status ? ep.red.status : p->dev_err;
    const bool tct = n3 > TC_TUBE_MIN_N3;
    const size_t P = (size_t)n1 * s;
    if (ready) {  // the pass back of the product before wrote bf16(Y x_3 M^{-T})
    } else if (tct) {
      TC_TRY(launch_mode3_tc_lowp(Y, lowop(p), p->dMinvT, n3, P, rkind(p), ep.skip, err, st));
    } else if (x3(p)) {
      TC_TRY(launch_mode3(Y, p->tmp2, p->dMinvT, n3, P, mid, st));
      TC_TRY(launch_round(p->tmp2, p->lowX, P * n3, ROUND_BF16X3, st, ep.skip));
    } else {
      TC_TRY(launch_mode3_lowp(Y, p->tmp1, p->dMinvT, n3, P, rkind(p) == ROUND_BF16, ep.skip,
                               st));
    }
    if (p->store_bf16) {  // BF16 slice products, read back by the BF16-input pass
      TC_TRY(launch_umma(*p->uma, p->tmp2, err, ep.skip, st, true));
      if (next_T)
        return launch_mode3_tc_chain(p->tmp2, X, p->dMT, lowop(p), next_T, n3, (size_t)n2 * s,
                                     ep, err, st, after);
      return launch_mode3_tc_inb(p->tmp2, X, p->dMT, n3, (size_t)n2 * s, ep, err, st, after);
    }
    if (p->tmp3) TC_TRY(transpose_slices(p->tmp1, p->tmp3, n1, s, n3, st, ep.skip));
    TC_TRY(launch_umma(*p->uma, p->tmp2, err, ep.skip, st));
    if (p->two_sided) TC_TRY(right_factor(p, *p->uma2, (size_t)n2 * s * n3, err, ep.skip, st));
    return tct ? launch_mode3_tc(p->tmp2, X, p->dMT, n3, (size_t)n2 * s, ep, err, st, x3(p), after)
               : launch_mode3(p->tmp2, X, p->dMT, n3, (size_t)n2 * s, ep, st);
  }
  TC_TRY(launch_mode3(Y, p->tmp1, p->dMinvT, n3, (size_t)n1 * s, mid, st));
  TC_TRY(launch_slice_gemm(p->AhT, p->tmp1, p->tmp2, n2, s, n1, n3, nullptr, nullptr, mid, st));
  const float* src = p->tmp2;
  if (p->two_sided) {
    TC_TRY(launch_slice_gemm(p->tmp2, p->BhT, p->tmp1, n2, s, s, n3, nullptr, nullptr, mid, st));
    src = p->tmp1;
  }
  return launch_mode3(src, X, p->dMT, n3, (size_t)n2 * s, ep, st);
}

namespace {
// ORTHODCT (Algorithm 1 as printed): M = C_{n3}, M^{-1} = C_{n3}^T.
void transform_pair_orthodct(int n, std::vector<double>& M, std::vector<double>& Mi) {
  dct2(n, M);
  Mi.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Mi[(size_t)i * n + j] = M[(size_t)j * n + i];
}

int plan_build(tc_plan* p, const float* A, const float* B, cudaStream_t st) {
  const int n1 = p->n1, n2 = p->n2, s = p->s, n3 = p->n3;
  std::vector<double> M, Mi;
  if (p->opts.product == TC_ORTHODCT)
    transform_pair_orthodct(n3, M, Mi);
  else
    transform_pair(n3, M, Mi);
  // M Mi must be the identity; anything else is a bug in the closed forms.
  for (int i = 0; i < n3; ++i)
    for (int j = 0; j < n3; ++j) {
      double t = 0.0;
      for (int r = 0; r < n3; ++r) t += M[(size_t)i * n3 + r] * Mi[(size_t)r * n3 + j];
      if (std::fabs(t - (i == j ? 1.0 : 0.0)) > 1e-9) return TC_EINVAL;
    }
  const size_t nn = (size_t)n3 * n3;
  std::vector<float> fM(nn), fMi(nn), fMiT(nn), fMT(nn);
  for (int i = 0; i < n3; ++i)
    for (int j = 0; j < n3; ++j) {
      fM[(size_t)i * n3 + j] = (float)M[(size_t)i * n3 + j];
      fMi[(size_t)i * n3 + j] = (float)Mi[(size_t)i * n3 + j];
      fMiT[(size_t)i * n3 + j] = (float)Mi[(size_t)j * n3 + i];
      fMT[(size_t)i * n3 + j] = (float)M[(size_t)j * n3 + i];
    }
  if (n3 <= TC_MAX_FUSED) {
    std::memcpy(p->hM, fM.data(), nn * sizeof(float));
    std::memcpy(p->hMinv, fMi.data(), nn * sizeof(float));
    std::memcpy(p->hMinvT, fMiT.data(), nn * sizeof(float));
    std::memcpy(p->hMT, fMT.data(), nn * sizeof(float));
  }
  TC_TRY(dalloc(&p->dM, nn));
  TC_TRY(dalloc(&p->dMinv, nn));
  TC_TRY(dalloc(&p->dMinvT, nn));
  TC_TRY(dalloc(&p->dMT, nn));
  TC_CUDA(cudaMemcpyAsync(p->dM, fM.data(), nn * 4, cudaMemcpyHostToDevice, st));
  TC_CUDA(cudaMemcpyAsync(p->dMinv, fMi.data(), nn * 4, cudaMemcpyHostToDevice, st));
  TC_CUDA(cudaMemcpyAsync(p->dMinvT, fMiT.data(), nn * 4, cudaMemcpyHostToDevice, st));
  TC_CUDA(cudaMemcpyAsync(p->dMT, fMT.data(), nn * 4, cudaMemcpyHostToDevice, st));
  if (thd_route(p)) {  // G = M^{-T} M^{-1} and G^{-1} = M M^T, formed in FP64
    std::vector<float> fG(nn), fGi(nn);
    for (int i = 0; i < n3; ++i)
      for (int j = 0; j < n3; ++j) {
        double g = 0.0, gi = 0.0;
        for (int r = 0; r < n3; ++r) {
          g += Mi[(size_t)r * n3 + i] * Mi[(size_t)r * n3 + j];
          gi += M[(size_t)i * n3 + r] * M[(size_t)j * n3 + r];
        }
        fG[(size_t)i * n3 + j] = (float)g;
        fGi[(size_t)i * n3 + j] = (float)gi;
      }
    TC_TRY(dalloc(&p->dG, nn));
    TC_TRY(dalloc(&p->dGi, nn));
    TC_CUDA(cudaMemcpyAsync(p->dG, fG.data(), nn * 4, cudaMemcpyHostToDevice, st));
    TC_CUDA(cudaMemcpyAsync(p->dGi, fGi.data(), nn * 4, cudaMemcpyHostToDevice, st));
  }

  const size_t TA = (size_t)n3 * n1 * n2;
  TC_TRY(dalloc(&p->Ah, TA));
  TC_TRY(dalloc(&p->AhT, TA));
  Epi none;
  TC_TRY(launch_mode3(A, p->Ah, p->dM, n3, (size_t)n1 * n2, none, st));
  TC_TRY(transpose_slices(p->Ah, p->AhT, n1, n2, n3, st));
  if (B) {
    const size_t TB = (size_t)n3 * s * s;
    TC_TRY(dalloc(&p->Bh, TB));
    TC_TRY(dalloc(&p->BhT, TB));
    TC_TRY(launch_mode3(B, p->Bh, p->dM, n3, (size_t)s * s, none, st));
    TC_TRY(transpose_slices(p->Bh, p->BhT, s, s, n3, st));
  }
  p->tmp_elems = p->Tx > p->Ty ? p->Tx : p->Ty;
  TC_TRY(dalloc(&p->tmp1, p->tmp_elems));
  TC_TRY(dalloc(&p->tmp2, p->tmp_elems));
  if (p->opts.store == TC_STORE_BF16) {
    p->store_bf16 = tube_inb_ok(p->tmp2, n3, (size_t)(n1 > n2 ? n1 : n2) * s);
    if (!p->store_bf16) return TC_EUNSUPPORTED;
  }
  // partials: one per CTA of the largest reducing launch (vector passes are
  // capped at 152*32 CTAs, transform passes use P/128, fused GEMMs tiles).
  size_t np = 152 * 32 + 64;
  const size_t big = (p->tmp_elems / n3 + 127) / 128 + 64;
  if (big > np) np = big;
  // fused GEMMs: 32 x 32 tiles times a K split of up to 8
  const size_t tiles = (size_t)((n1 > n2 ? n1 : n2) + 31) / 32 * ((s + 31) / 32) * 8 + 64;
  if (tiles > np) np = tiles;
  TC_TRY(dalloc(&p->dev_err, 1));
  TC_CUDA(cudaMemsetAsync(p->dev_err, 0, sizeof(int), st));
  if (lowp(p)) {
    const int bf16 = p->opts.precision != TC_TF32;  // BF16 operands (one plane or three)
    const int ns = x3(p) ? 3 : 1;
    const size_t es = bf16 ? 2 : 4;
    TC_CUDA(cudaMalloc(&p->AhL, TA * es * ns));
    TC_CUDA(cudaMalloc(&p->AhTL, TA * es * ns));
    TC_TRY(launch_round(p->Ah, p->AhL, TA, rkind(p), st));
    TC_TRY(launch_round(p->AhT, p->AhTL, TA, rkind(p), st));
    if (ns == 3) TC_CUDA(cudaMalloc(&p->lowX, p->tmp_elems * 2 * 3));
    p->umf = new UmmaMaps();
    p->uma = new UmmaMaps();
    const int kind = bf16 ? 0 : 1;
    // TF32 reads B K-major: the transformed operand is transposed per slice into tmp3
    if (!bf16) TC_TRY(dalloc(&p->tmp3, p->tmp_elems));
    const void* bop = bf16 ? lowop(p) : (const void*)p->tmp3;
    TC_TRY(make_umma_maps(p->umf, kind, p->AhL, bop, n1, s, n2, n3, ns));
    TC_TRY(make_umma_maps(p->uma, kind, p->AhTL, bop, n2, s, n1, n3, ns));
    if (B) {
      // second GEMMs: left operand T in the operand buffer (K = s contiguous);
      // B operand K x N with N contiguous (BF16): B~ forward, B~^T adjoint;
      // N x K with K contiguous (TF32): B~^T forward, B~ adjoint
      const size_t TB = (size_t)n3 * s * s;
      TC_CUDA(cudaMalloc(&p->BfL, TB * es * ns));
      TC_CUDA(cudaMalloc(&p->BaL, TB * es * ns));
      TC_TRY(launch_round(bf16 ? p->Bh : p->BhT, p->BfL, TB, rkind(p), st));
      TC_TRY(launch_round(bf16 ? p->BhT : p->Bh, p->BaL, TB, rkind(p), st));
      p->umf2 = new UmmaMaps();
      p->uma2 = new UmmaMaps();
      TC_TRY(make_umma_maps(p->umf2, kind, lowop(p), p->BfL, n1, s, s, n3, ns));
      TC_TRY(make_umma_maps(p->uma2, kind, lowop(p), p->BaL, n2, s, s, n3, ns));
    }
    if (bf16 && ((p->opts.product == TC_ORTHODCT && !B) || thd_route(p))) {
      // transform-domain LSQR with the epilogue in the GEMM: the forward and
      // adjoint GEMMs read separate BF16 operands (lowV: V~, n2 x s; lowU:
      // U~, n1 x s), each written by the other product (ORTHODCT: by its
      // GEMM's store; dual-domain route: by its change-of-domain pass)
      TC_CUDA(cudaMalloc(&p->lowV, (size_t)n2 * s * n3 * 2 * ns));
      TC_CUDA(cudaMalloc(&p->lowU, (size_t)n1 * s * n3 * 2 * ns));
      p->umf_td = new UmmaMaps();
      p->uma_td = new UmmaMaps();
      TC_TRY(make_umma_maps(p->umf_td, 0, p->AhL, p->lowV, n1, s, n2, n3, ns));
      TC_TRY(make_umma_maps(p->uma_td, 0, p->AhTL, p->lowU, n2, s, n1, n3, ns));
    }
  }
  TC_TRY(dalloc(&p->scratch.partials, np));
  TC_TRY(dalloc(&p->scratch.tickets, 16));
  p->scratch.npartials = np;
  TC_CUDA(cudaMemsetAsync(p->scratch.tickets, 0, 16 * sizeof(unsigned), st));
  TC_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  TC_CUDA(cudaStreamSynchronize(st));
  return TC_OK;
}
}  // namespace

extern "C" int tc_plan_destroy(tc_plan* p) {
  if (!p) return TC_EINVAL;
  if (p->lsqr_graph) cudaGraphExecDestroy(p->lsqr_graph);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  float* fs[] = {p->Ah, p->AhT, p->Bh, p->BhT, p->dM, p->dMinv, p->dMinvT, p->dMT, p->dG, p->dGi,
                 p->tmp1, p->tmp2, p->tmp3, p->lsqr_U, p->lsqr_V, p->lsqr_W, p->basis,
                 p->gm_basis, p->lsqr_Ct, p->lsqr_Xt};
  for (float* f : fs) dfree(f);
  dfree(p->scratch.partials);
  dfree(p->scratch.tickets);
  dfree(p->dscal);
  dfree(p->iflags);
  dfree(p->lsqr_done);
  dfree(p->gm_dscal);
  dfree(p->gm_flags);
  dfree(p->dev_err);
  dfree(p->aux);
  dfree(p->AhL);
  dfree(p->AhTL);
  delete p->umf;
  delete p->uma;
  delete p->umf_td;
  delete p->uma_td;
  delete p->umf2;
  delete p->uma2;
  dfree(p->BfL);
  dfree(p->BaL);
  dfree(p->lowX);
  dfree(p->lowV);
  dfree(p->lowU);
  delete p;
  return TC_OK;
}

extern "C" int tc_plan_create(tc_plan** out, int n1, int n2, int s, int n3, const float* A,
                              const float* B, const tc_opts* opts, tc_stream_t stream) {
  if (!out || !A) return TC_EINVAL;
  *out = nullptr;
  if (n1 < 1 || n2 < 1 || s < 1 || n3 < 1 || n3 > TC_MAX_N3) return TC_EINVAL;
  if ((long long)n1 * n2 * n3 > (1LL << 34) || (long long)(n1 > n2 ? n1 : n2) * s * n3 > (1LL << 34))
    return TC_EINVAL;
  tc_opts o{};
  o.precision = TC_FP32;
  o.gcv_variant = TC_GCV_PAPER;
  o.use_graphs = 1;
  if (opts) {
    o = *opts;
    for (int r : o.reserved)
      if (r != 0) return TC_EINVAL;
    if (o.precision != TC_FP32 && o.precision != TC_TF32 && o.precision != TC_BF16 &&
        o.precision != TC_BF16X3)
      return TC_EINVAL;
    if (o.gcv_variant != TC_GCV_PAPER && o.gcv_variant != TC_GCV_FULL) return TC_EINVAL;
    if (o.product != TC_TH && o.product != TC_ORTHODCT) return TC_EINVAL;
    if (o.route != TC_ROUTE_AUTO && o.route != TC_ROUTE_SPATIAL && o.route != TC_ROUTE_DUAL)
      return TC_EINVAL;
    if (o.store != TC_STORE_F32 && o.store != TC_STORE_BF16) return TC_EINVAL;
    // BF16-stored slice products: BF16 plans, one-sided, with the tensor-core
    // passes (32 < n3 <= 64)
    if (o.store == TC_STORE_BF16 &&
        (o.precision != TC_BF16 || B || n3 <= TC_TUBE_MIN_N3 || n3 > 64))
      return TC_EUNSUPPORTED;
  }
  if (o.precision != TC_FP32) {
    // tensor-core forms: every dimension a multiple of 8 (16-byte rows for
    // TMA), the transform passes of the unfused route
    if (n1 % 8 || n2 % 8 || s % 8) return TC_EUNSUPPORTED;
  }
  static int inited = 0;
  if (!inited) {
    TC_TRY(tc_kernels_init());
    TC_TRY(umma_init());
    inited = 1;
  }
  tc_plan* p = new (std::nothrow) tc_plan();
  if (!p) return TC_ENOMEM;
  p->n1 = n1; p->n2 = n2; p->s = s; p->n3 = n3;
  p->two_sided = (B != nullptr);
  p->opts = o;
  p->Tx = (size_t)n2 * s * n3;
  p->Ty = (size_t)n1 * s * n3;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return TC_ECUDA;
  }
  const int r = plan_build(p, A, B, (cudaStream_t)stream);
  if (r != TC_OK) {
    tc_plan_destroy(p);
    return r;
  }
  *out = p;
  return TC_OK;
}

extern "C" int tc_cprod(tc_plan* p, const float* X, float* Y, tc_stream_t stream) {
  if (!p || !X || !Y || (const void*)X == (const void*)Y) return TC_EINVAL;
  Epi ep;
  return cprod_epi(p, X, Y, ep, (cudaStream_t)stream);
}

extern "C" int tc_cprod_adjoint(tc_plan* p, const float* Y, float* X, tc_stream_t stream) {
  if (!p || !X || !Y || (const void*)X == (const void*)Y) return TC_EINVAL;
  Epi ep;
  return adjoint_epi(p, Y, X, ep, (cudaStream_t)stream);
}

extern "C" int tc_slice_gemm(tc_plan* p, const void* Xh, float* Yh, int adjoint,
                             tc_stream_t stream) {
  if (!p || !Xh || !Yh || (const void*)Xh == (const void*)Yh) return TC_EINVAL;
  if (p->two_sided) return TC_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const int M = adjoint ? p->n2 : p->n1, K = adjoint ? p->n1 : p->n2;
  if (!lowp(p)) {
    Epi none;
    return launch_slice_gemm(adjoint ? p->AhT : p->Ah, static_cast<const float*>(Xh), Yh, M,
                             p->s, K, p->n3, nullptr, nullptr, none, st);
  }
  const void* bop = Xh;
  if (p->tmp3) {  // TF32: K-major copy of the operand
    TC_TRY(transpose_slices(static_cast<const float*>(Xh), p->tmp3, K, p->s, p->n3, st));
    bop = p->tmp3;
  }
  UmmaMaps m;
  TC_TRY(make_umma_maps(&m, p->opts.precision == TC_TF32 ? 1 : 0, adjoint ? p->AhTL : p->AhL, bop,
                        M, p->s, K, p->n3, x3(p) ? 3 : 1));
  return launch_umma(m, Yh, p->dev_err, nullptr, st);
}

extern "C" int tc_slice_gemm_gk(tc_plan* p, const void* Xh, float* Yh, int adjoint,
                                const double* s0, const double* s1, const float* prev,
                                double* sumsq, tc_stream_t stream) {
  if (!p || !Xh || !Yh || !s0 || (const void*)Xh == (const void*)Yh) return TC_EINVAL;
  if (p->two_sided || p->opts.precision != TC_BF16) return TC_EUNSUPPORTED;
  if (prev && !s1) return TC_EINVAL;
  const int M = adjoint ? p->n2 : p->n1, K = adjoint ? p->n1 : p->n2;
  UmmaMaps m;
  TC_TRY(make_umma_maps(&m, 0, adjoint ? p->AhTL : p->AhL, Xh, M, p->s, K, p->n3, 1));
  Epi ep;
  ep.coef.rule = prev ? COEF_GK : COEF_INV;
  ep.coef.s0 = s0;
  ep.coef.s1 = s1;
  ep.prev = prev;
  if (sumsq) ep.red = make_red(p, sumsq, 0, nullptr, nullptr);
  return launch_umma_epi(m, Yh, nullptr, ep, p->dev_err, (cudaStream_t)stream);
}

extern "C" int tc_transform(tc_plan* p, int which, const float* in, float* out, size_t P,
                            const float* prev, double* sumsq, tc_stream_t stream) {
  if (!p || !in || !out || (const void*)in == (const void*)out) return TC_EINVAL;
  if (which < TC_M || which > TC_MT || P < 1 || P * (size_t)p->n3 > p->tmp_elems)
    return TC_EINVAL;
  if (prev && (prev == out || prev == in)) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const float* T = which == TC_M ? p->dM : which == TC_MINV ? p->dMinv
                   : which == TC_MINVT ? p->dMinvT : p->dMT;
  Epi ep;
  if (prev) {
    ep.coef.rule = COEF_ADD;
    ep.prev = prev;
  }
  if (sumsq) ep.red = make_red(p, sumsq, 0, nullptr, nullptr);
  // the pass the plan's products run: tcgen05 for tensor-core plans above
  // TC_TUBE_MIN_N3 (three BF16 planes for TC_BF16X3), the FP32 pass otherwise
  if (lowp(p) && p->n3 > TC_TUBE_MIN_N3)
    return launch_mode3_tc(in, out, T, p->n3, P, ep, p->dev_err, st, x3(p));
  return launch_mode3(in, out, T, p->n3, P, ep, st);
}

extern "C" int tc_transform_dual(tc_plan* p, int which, const float* in, void* out, size_t P,
                                 double* sumsq, tc_stream_t stream) {
  if (!p || !in || !out || !sumsq || (const void*)in == out) return TC_EINVAL;
  if ((which != TC_DUAL_U && which != TC_DUAL_V) || P < 1 || P * (size_t)p->n3 > p->tmp_elems)
    return TC_EINVAL;
  if (!thd_route(p)) return TC_EUNSUPPORTED;
  if (P % 8 || (reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
    return TC_EINVAL;
  Epi ep;
  ep.red = make_red(p, sumsq, 0, nullptr, nullptr);
  const bool u = which == TC_DUAL_U;
  return launch_mode3_tc_norm(in, out, u ? p->dG : p->dGi, u ? p->dMinv : p->dMT, p->n3, P, ep,
                              p->dev_err, (cudaStream_t)stream, nullptr);
}

extern "C" int tc_transform_bf16in(tc_plan* p, int which, const void* in, float* out, size_t P,
                                   const float* prev, double* sumsq, int which_next, void* nxt,
                                   tc_stream_t stream) {
  if (!p || !in || !out || (const void*)in == (const void*)out) return TC_EINVAL;
  if (which < TC_M || which > TC_MT || P < 1 || P * (size_t)p->n3 > p->tmp_elems)
    return TC_EINVAL;
  if (prev && prev == out) return TC_EINVAL;
  if (nxt && (which_next < TC_M || which_next > TC_MT || nxt == (void*)out || nxt == in ||
              (const void*)nxt == (const void*)prev))
    return TC_EINVAL;
  if (!p->store_bf16) return TC_EUNSUPPORTED;
  auto pick = [&](int w) {
    return w == TC_M ? p->dM : w == TC_MINV ? p->dMinv : w == TC_MINVT ? p->dMinvT : p->dMT;
  };
  const float* T = pick(which);
  Epi ep;
  if (prev) {
    ep.coef.rule = COEF_ADD;
    ep.prev = prev;
  }
  if (sumsq) ep.red = make_red(p, sumsq, 0, nullptr, nullptr);
  if (nxt)
    return launch_mode3_tc_chain(in, out, T, nxt, pick(which_next), p->n3, P, ep, p->dev_err,
                                 (cudaStream_t)stream, nullptr);
  return launch_mode3_tc_inb(in, out, T, p->n3, P, ep, p->dev_err, (cudaStream_t)stream,
                             nullptr);
}

extern "C" int tc_plan_status(tc_plan* p, int* status) {
  if (!p || !status) return TC_EINVAL;
  TC_CUDA(cudaMemcpy(status, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  return TC_OK;
}

