// Mode-3 transform pass for n3 > TC_MAX_FUSED (Remark 2.1: X~ = X x_3 T with
// T one of M, M^{-1}, M^{-T}, M^T): out[k][p] = ca * sum_l T[k][l] in[l][p]
// + cp * prev[k][p], with the fused reduction of the epilogue. Each CTA owns
// 128 consecutive pixels p of every slice: warp w computes the KPW contiguous
// outputs k = w*KPW .. w*KPW + KPW - 1 (coefficients read as float4
// broadcasts) and lane q the pixels 4q..4q+3. T is staged in shared memory
// once. The CTA's whole input block (every slice of its 128 pixels, 32 KB at
// n3 = 64) is requested at once with cp.async in groups of 16 slices, and
// each group is consumed as it lands, so a CTA keeps its whole input in
// flight. HBM traffic is one read of `in` (and `prev`) and one write of `out`.
#include <cuda_bf16.h>

#include "tc_device.cuh"
#include "tcgen05.cuh"
#include "umma.cuh"

namespace {

// Output element of a transform pass: FP32 (with the Krylov epilogue), or the
// low-precision operand of a tensor-core GEMM: BF16 (round to nearest even)
// or FP32 holding a TF32 value (round to nearest, ties away, as cvt.rna).
enum OutKind { OUT_F32 = 0, OUT_BF16 = 1, OUT_TF32 = 2, OUT_BF16X3 = 3 };

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

constexpr int PB = 128;  // pixels per CTA
constexpr int LC = 16;   // input slices per cp.async group

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;  // zero-fill when out of range
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(n)
               : "memory");
}

// Dynamic shared memory of k_mode3<KPW, .>: T^T (8 KPW x 8 KPW) and the whole
// input block (8 KPW slices x PB pixels).
template <int KPW>
constexpr size_t mode3_smem() { return (size_t)(8 * KPW) * (8 * KPW + PB) * sizeof(float); }

__device__ __forceinline__ void cp_wait_upto(int n) {  // at most n groups pending
  if (n <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
  else if (n == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
  else if (n == 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
  else asm volatile("cp.async.wait_group 3;" ::: "memory");
}

template <int KPW, int OUT>
__global__ void __launch_bounds__(256, 3)
k_mode3(const float* __restrict__ in, void* out_v, const float* __restrict__ T, int n3,
        size_t P, Epi ep) {
  if (ep.skip && *ep.skip) return;
  // ts: T transposed (ts[l][k] = T[k][l]), loaded once; xs: the CTA's whole
  // input block, every slice of its PB pixels, requested at once in groups of
  // LC slices so that all of it is in flight while the first groups compute
  extern __shared__ __align__(16) float m3_smem[];
  float(*ts)[8 * KPW] = reinterpret_cast<float(*)[8 * KPW]>(m3_smem);
  float(*xs)[PB] = reinterpret_cast<float(*)[PB]>(m3_smem + (8 * KPW) * (8 * KPW));
  __shared__ float sh_coef[2];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const size_t p0 = (size_t)blockIdx.x * PB;
  // float4 path: whole groups of 4 pixels and 16-byte aligned tensors
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  const bool vec = (P % 4 == 0) && al16(in) && al16(out_v) && (!ep.prev || al16(ep.prev)) &&
                   (!ep.red.other || al16(ep.red.other));
  float acc[KPW][4];
#pragma unroll
  for (int q = 0; q < KPW; ++q)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[q][e] = 0.f;

  const int nch = (n3 + LC - 1) / LC;  // <= 4 (n3 <= 64)
  for (int c = 0; c < nch; ++c) {
    const int l0 = c * LC, lc_n = min(LC, n3 - l0);
    if (vec) {
      for (int idx = tid; idx < LC * PB / 4; idx += 256) {
        const int lc = idx / (PB / 4), px = (idx % (PB / 4)) * 4;
        const size_t p = p0 + px;
        if (lc < lc_n) {
          const bool ok = p < P;
          cp_async16(&xs[l0 + lc][px], ok ? in + (size_t)(l0 + lc) * P + p : in, ok);
        }
      }
    } else {
      for (int idx = tid; idx < LC * PB; idx += 256) {
        const int lc = idx / PB, px = idx % PB;
        const size_t p = p0 + px;
        if (lc < lc_n) xs[l0 + lc][px] = p < P ? __ldg(in + (size_t)(l0 + lc) * P + p) : 0.f;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int idx = tid; idx < n3 * 8 * KPW; idx += 256) {
    const int l = idx / (8 * KPW), k = idx % (8 * KPW);
    ts[l][k] = (k < n3) ? __ldg(T + (size_t)k * n3 + l) : 0.f;
  }
  for (int c = 0; c < nch; ++c) {
    cp_wait_upto(nch - 1 - c);  // this thread's copies of group c have landed
    __syncthreads();            // everyone's, and T
    const int l0 = c * LC, lc_n = min(LC, n3 - l0);
    for (int lc = 0; lc < lc_n; ++lc) {
      const float4 x = *reinterpret_cast<const float4*>(&xs[l0 + lc][lane * 4]);
      float t[KPW];  // warp w owns the contiguous outputs k = w*KPW .. w*KPW + KPW - 1
      if (KPW % 4 == 0) {
#pragma unroll
        for (int q = 0; q < KPW; q += 4) {
          const float4 tv = *reinterpret_cast<const float4*>(&ts[l0 + lc][w * KPW + q]);
          t[q] = tv.x; t[q + 1] = tv.y; t[q + 2] = tv.z; t[q + 3] = tv.w;
        }
      } else {
#pragma unroll
        for (int q = 0; q < KPW; ++q) t[q] = ts[l0 + lc][w * KPW + q];
      }
#pragma unroll
      for (int q = 0; q < KPW; ++q) {
        acc[q][0] = fmaf(t[q], x.x, acc[q][0]);
        acc[q][1] = fmaf(t[q], x.y, acc[q][1]);
        acc[q][2] = fmaf(t[q], x.z, acc[q][2]);
        acc[q][3] = fmaf(t[q], x.w, acc[q][3]);
      }
    }
  }

  if (OUT != OUT_F32) {  // operand of a tensor-core GEMM: store only
#pragma unroll
    for (int q = 0; q < KPW; ++q) {
      const int k = w * KPW + q;
      if (k >= n3) continue;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const size_t p = p0 + lane * 4 + e;
        if (p < P) {
          const size_t idx = (size_t)k * P + p;
          if (OUT == OUT_BF16)
            static_cast<__nv_bfloat16*>(out_v)[idx] = __float2bfloat16_rn(acc[q][e]);
          else
            static_cast<float*>(out_v)[idx] = round_tf32(acc[q][e]);
        }
      }
    }
    return;
  }
  float* out = static_cast<float*>(out_v);
  coef_compute(ep.coef, sh_coef);
  __syncthreads();
  const float ca = sh_coef[0], cp = sh_coef[1];
  float local = 0.f;
#pragma unroll
  for (int q = 0; q < KPW; ++q) {
    const int k = w * KPW + q;
    if (k >= n3) continue;
    const size_t pb = p0 + lane * 4;
    if (vec && pb + 4 <= P) {
      const size_t idx = (size_t)k * P + pb;
      float4 o = make_float4(ca * acc[q][0], ca * acc[q][1], ca * acc[q][2], ca * acc[q][3]);
      if (ep.prev) {
        const float4 pv = *reinterpret_cast<const float4*>(ep.prev + idx);
        o.x = fmaf(cp, pv.x, o.x); o.y = fmaf(cp, pv.y, o.y);
        o.z = fmaf(cp, pv.z, o.z); o.w = fmaf(cp, pv.w, o.w);
      }
      *reinterpret_cast<float4*>(out + idx) = o;
      if (ep.red.out) {
        if (ep.red.other) {
          const float4 ov = *reinterpret_cast<const float4*>(ep.red.other + idx);
          local = fmaf(o.x, ov.x, fmaf(o.y, ov.y, fmaf(o.z, ov.z, fmaf(o.w, ov.w, local))));
        } else {
          local = fmaf(o.x, o.x, fmaf(o.y, o.y, fmaf(o.z, o.z, fmaf(o.w, o.w, local))));
        }
      }
      continue;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const size_t p = pb + e;
      if (p < P) {
        const size_t idx = (size_t)k * P + p;
        float o = ca * acc[q][e];
        if (ep.prev) o = fmaf(cp, ep.prev[idx], o);
        out[idx] = o;
        if (ep.red.out) local = fmaf(o, ep.red.other ? ep.red.other[idx] : o, local);
      }
    }
  }
  if (ep.red.out) reduce_finish(local, ep.red);
}

template <int KPW, int OUT>
int run(const float* in, void* out, const float* T, int n3, size_t P, const Epi& ep,
        cudaStream_t st) {
  const size_t blocks = (P + PB - 1) / PB;
  k_mode3<KPW, OUT><<<(unsigned)blocks, 256, mode3_smem<KPW>(), st>>>(in, out, T, n3, P, ep);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

template <int OUT>
int pick(const float* in, void* out, const float* T, int n3, size_t P, const Epi& ep,
         cudaStream_t st) {
  if (n3 <= 8) return run<1, OUT>(in, out, T, n3, P, ep, st);
  if (n3 <= 16) return run<2, OUT>(in, out, T, n3, P, ep, st);
  if (n3 <= 32) return run<4, OUT>(in, out, T, n3, P, ep, st);
  return run<8, OUT>(in, out, T, n3, P, ep, st);
}

// Elementwise rounding to the GEMM input type; four elements per thread and
// iteration when in is 16-byte aligned (the output then is 8- or 16-byte
// aligned too), with four such groups of loads in flight. OUT_BF16X3 writes
// three BF16 planes of n values each: bf16(x), then bf16 of what each plane
// leaves (the planes of the FP32-level form).
__global__ void k_round(const float* __restrict__ in, void* out, size_t n, int kind,
                        const int* skip) {
  if (skip && *skip) return;
  const size_t st = (size_t)gridDim.x * blockDim.x;
  const size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t done = 0;
  __nv_bfloat16* o16 = static_cast<__nv_bfloat16*>(out);
  if ((reinterpret_cast<uintptr_t>(in) & 15) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0 &&
      (kind != OUT_BF16X3 || n % 4 == 0)) {
    const size_t n4 = n / 4;
    for (size_t i0 = gt; i0 < n4; i0 += 4 * st) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const size_t i = i0 + u * st;
        v[u] = i < n4 ? reinterpret_cast<const float4*>(in)[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const size_t i = i0 + u * st;
        if (i >= n4) break;
        if (kind == OUT_BF16 || kind == OUT_BF16X3) {
          float4 r = v[u];
          for (int q = 0; q < (kind == OUT_BF16X3 ? 3 : 1); ++q) {
            const __nv_bfloat162 lo = __floats2bfloat162_rn(r.x, r.y);
            const __nv_bfloat162 hi = __floats2bfloat162_rn(r.z, r.w);
            uint2 pk;
            pk.x = *reinterpret_cast<const uint32_t*>(&lo);
            pk.y = *reinterpret_cast<const uint32_t*>(&hi);
            reinterpret_cast<uint2*>(o16 + q * n)[i] = pk;
            r.x -= __low2float(lo);
            r.y -= __high2float(lo);
            r.z -= __low2float(hi);
            r.w -= __high2float(hi);
          }
        } else {
          reinterpret_cast<float4*>(out)[i] = make_float4(round_tf32(v[u].x), round_tf32(v[u].y),
                                                          round_tf32(v[u].z), round_tf32(v[u].w));
        }
      }
    }
    done = 4 * n4;
  }
  for (size_t i = done + gt; i < n; i += st) {
    if (kind == OUT_BF16 || kind == OUT_BF16X3) {
      float r = in[i];
      for (int q = 0; q < (kind == OUT_BF16X3 ? 3 : 1); ++q) {
        const __nv_bfloat16 b = __float2bfloat16_rn(r);
        o16[q * n + i] = b;
        r -= __bfloat162float(b);
      }
    } else {
      static_cast<float*>(out)[i] = round_tf32(in[i]);
    }
  }
}

// ---------------------------------------------------------- tensor cores ----
// Mode-3 transform on the tcgen05 tensor cores, for the TF32 and BF16
// precision forms: out[k][p] = sum_l T[k][l] in[l][p] (+ the Krylov
// epilogue) as the transposed product D = in^T T^T. One CTA a tile of TP =
// 128 pixels: A = in^T (128 pixels x 64 slices), MN-major straight from the
// slice layout; B = T (64 outputs x 64 slices), K-major; D = 128 pixels x 64
// outputs in tensor memory, lane = pixel, so each store (and prev load) of a
// warp is 32 consecutive pixels of one slice. n3 < 64 pads K and N with zeros.
// Both operands are split into NS BF16 planes: x_0 = bf16(x), then each next
// plane rounds what the ones before leave, x_s = bf16(x - x_0 - .. - x_{s-1})
// (each difference is exact in FP32). D accumulates the products x_i y_j with
// i + j < NS in FP32 (kind::f16):
// * NS = 2 (TF32 and BF16 forms): 3 products, relative error near 2^-16 a term;
// * NS = 3 (the FP32-level form): 6 products, near 2^-27 a term, below FP32
//   rounding; the tensor cores' FP32 accumulation then sets the error.
// Shared memory holds the operand planes in the 128-byte swizzled layouts the
// descriptors name (16-byte chunk j of row r at chunk j ^ (r & 7)).
// The kernel is persistent, 4 (NS = 2) or 3 (NS = 3) CTAs a SM, each looping
// over tiles. B is split once a CTA. Once a tile's MMAs have completed, the
// next tile's FP32 input is copied (cp.async) into the first 32 KB of the A
// planes while this tile's epilogue runs. The reduction runs once a CTA.
constexpr int TP = 128, TK = 64, TNT = 128;
int g_tube_sms = 152;  // SM count of the device (set by transform_init)
constexpr uint32_t TA_BYTES = TP * TK * 2;  // one BF16 plane of A: 16 KB
constexpr uint32_t TB_BYTES = TK * TK * 2;  // one BF16 plane of B: 8 KB

constexpr size_t tube_smem(int ns) { return 1024 + ns * (TA_BYTES + TB_BYTES) + 16; }
constexpr int tube_ctas(int ns) { return ns == 2 ? 4 : 3; }  // resident CTAs a SM

// product p of the split operands: planes (tube_pa(p), tube_pb(p)), the
// products with i + j = 0, 1, 2 in that order
__device__ __forceinline__ int tube_pa(int p) { return p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0); }
__device__ __forceinline__ int tube_pb(int p) { return p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0); }

// NS planes of eight values, packed as eight BF16 each
template <int NS>
__device__ __forceinline__ void split8(const float* x, uint4* pl) {
  float r[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) r[e] = x[e];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(r[2 * j], r[2 * j + 1]);
      w[j] = *reinterpret_cast<const uint32_t*>(&b);
      r[2 * j] -= __low2float(b);
      r[2 * j + 1] -= __high2float(b);
    }
    pl[s] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int OUT, int NS>
__global__ void __launch_bounds__(TNT, tube_ctas(NS))
k_tube(const float* __restrict__ in, void* out_v, const float* __restrict__ T, int n3, size_t P,
       Epi ep, int* err) {
  constexpr int NPASS = NS == 2 ? 3 : 6;
  using namespace tc5;
  // D F32; A, B BF16; A MN-major, B K-major; N = 64, M = 128
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (0u << 16) |
                             ((uint32_t)(TK >> 3) << 17) | ((uint32_t)(TP >> 4) << 24);
  if (ep.skip && *ep.skip) return;
  extern __shared__ uint8_t tube_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(tube_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;  // NS A planes; between tiles, the FP32 staging of the next input tile
  float* stg = reinterpret_cast<float*>(base);  // [TK][TP] FP32, 32 KB: the first two planes
  uint8_t* sB = base + NS * TA_BYTES;           // NS B planes
  uint64_t* done = reinterpret_cast<uint64_t*>(sB + NS * TB_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ float sh_coef[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t ntile = (P + TP - 1) / TP;
  const bool vec = P % 4 == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0;

  // Input tile t into the staging buffer: unit u = tid + 128 i is slice l =
  // u / 16, pixels 8 (u % 16) + 0..7; each thread later reads its own units.
  auto stage = [&](size_t t) {
    const size_t p0 = t * TP;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int u = tid + TNT * i, l = u >> 4, px = 8 * (u & 15);
      float* dst = stg + l * TP + px;
      const size_t p = p0 + px;
      if (vec) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const bool ok = l < n3 && p + 4 * h + 4 <= P;
          cp_async16(dst + 4 * h, ok ? in + (size_t)l * P + p + 4 * h : in, ok);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[e] = (l < n3 && p + e < P) ? in[(size_t)l * P + p + e] : 0.f;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (blockIdx.x < ntile) stage(blockIdx.x);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tslot)),
                 "r"(TK)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (OUT == OUT_F32) coef_compute(ep.coef, sh_coef);
  // B = T, once a CTA: unit u = tid + 128 j is row n = u / 8 (output k), slices 8 (u % 8) + 0..7
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int u = tid + TNT * j, n = u >> 3, c = u & 7;
    float t[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int l = 8 * c + e;
      t[e] = (n < n3 && l < n3) ? __ldg(T + (size_t)n * n3 + l) : 0.f;
    }
    uint4 pl[NS];
    split8<NS>(t, pl);
    const uint32_t off = n * 128 + ((c ^ (n & 7)) << 4);
#pragma unroll
    for (int q = 0; q < NS; ++q) *reinterpret_cast<uint4*>(sB + q * TB_BYTES + off) = pl[q];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const float ca = OUT == OUT_F32 ? sh_coef[0] : 1.f, cp = OUT == OUT_F32 ? sh_coef[1] : 0.f;
  float local = 0.f;
  bool ok = true;
  uint32_t phase = 0;

  for (size_t t = blockIdx.x; t < ntile && ok; t += gridDim.x, phase ^= 1u) {
    const size_t p0 = t * TP;
    // staged input -> registers -> split into the A halves (same bytes)
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    float x[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int u = tid + TNT * i, l = u >> 4, px = 8 * (u & 15);
      const float4 a = *reinterpret_cast<const float4*>(stg + l * TP + px);
      const float4 b = *reinterpret_cast<const float4*>(stg + l * TP + px + 4);
      x[i][0] = a.x; x[i][1] = a.y; x[i][2] = a.z; x[i][3] = a.w;
      x[i][4] = b.x; x[i][5] = b.y; x[i][6] = b.z; x[i][7] = b.w;
    }
    __syncthreads();  // every thread has its staged values
    // A = in^T, MN-major: pixel chunk c of slice l in atom column c / 8, row l
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int u = tid + TNT * i, l = u >> 4, c = u & 15;
      uint4 pl[NS];
      split8<NS>(x[i], pl);
      const uint32_t off = (c >> 3) * (TA_BYTES / 2) + l * 128 + (((c & 7) ^ (l & 7)) << 4);
#pragma unroll
      for (int q = 0; q < NS; ++q) *reinterpret_cast<uint4*>(sA + q * TA_BYTES + off) = pl[q];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
#pragma unroll
      for (int pass = 0; pass < NPASS; ++pass) {
        const uint32_t a0 = su32(sA + tube_pa(pass) * TA_BYTES);
        const uint32_t b0 = su32(sB + tube_pb(pass) * TB_BYTES);
#pragma unroll
        for (int kk = 0; kk < TK / 16; ++kk)
          umma<0>(tmem, smem_desc(a0 + kk * 16 * 128, TA_BYTES / 2, 1024),
                  smem_desc(b0 + kk * 16 * 2, 16, 1024), IDESC, (pass | kk) != 0);
      }
      umma_commit(done);
    }

    // epilogue: thread = pixel p0 + 32 warp + lane = tensor-memory lane 32 warp + lane
    const size_t p = p0 + 32 * warp + lane;
    const bool live = p < P;
    float pv[2][32];  // prev of outputs 32 h + j
    auto load_prev = [&](int h) {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        pv[h][j] = (OUT == OUT_F32 && ep.prev && live && 32 * h + j < n3)
                       ? ep.prev[(size_t)(32 * h + j) * P + p]
                       : 0.f;
    };
    load_prev(0);  // does not depend on the MMAs
    ok = __syncthreads_and(mbar_wait(done, phase));
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the MMAs have read the A halves: stage the next tile there now
    if (t + gridDim.x < ntile) stage(t + gridDim.x);
#pragma unroll
    for (int h = 0; h < TK / 32; ++h) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * h), v);
      if (h + 1 < TK / 32) load_prev(h + 1);  // in flight while this half is stored
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int k = 32 * h + j;
        if (k >= n3 || !live) continue;
        const size_t idx = (size_t)k * P + p;
        if (OUT == OUT_BF16) {
          static_cast<__nv_bfloat16*>(out_v)[idx] = __float2bfloat16_rn(v[j]);
        } else if (OUT == OUT_BF16X3) {  // three planes of n3 P values
          __nv_bfloat16* o3 = static_cast<__nv_bfloat16*>(out_v);
          const __nv_bfloat16 y0 = __float2bfloat16_rn(v[j]);
          const float r1 = v[j] - __bfloat162float(y0);
          const __nv_bfloat16 y1 = __float2bfloat16_rn(r1);
          o3[idx] = y0;
          o3[(size_t)n3 * P + idx] = y1;
          o3[2 * (size_t)n3 * P + idx] = __float2bfloat16_rn(r1 - __bfloat162float(y1));
        } else if (OUT == OUT_TF32) {
          static_cast<float*>(out_v)[idx] = round_tf32(v[j]);
        } else {
          float o = ca * v[j];
          if (ep.prev) o = fmaf(cp, pv[h][j], o);
          static_cast<float*>(out_v)[idx] = o;
          if (ep.red.out) local = fmaf(o, ep.red.other ? ep.red.other[idx] : o, local);
        }
      }
    }
    // the next tile's MMAs overwrite the accumulator after the next barrier
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  if (!ok && tid == 0) {
    // The MMAs of the tile whose wait gave up may still read sA/sB and write
    // the accumulator: wait (bounded) once more for their commit before the
    // tensor memory is freed and the CTA's shared memory is released.
    mbar_wait(done, phase);
    atomicExch(err, TC_ETIMEOUT);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // no copy outlives the CTA
  if (OUT == OUT_F32 && ep.red.out) reduce_finish(local, ep.red);  // every thread of every CTA
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TK)
                 : "memory");
}

// ------------------------------------------- TMA-streamed tensor-core pass --
// The same transform (D = in^T T^T per tile of TP = 128 pixels, operands
// split into NS BF16 planes, FP32 accumulation) as a warp-specialised
// persistent kernel, one CTA per SM, every tile moved by TMA through two
// rings of 32 KB slots:
//   warp 0 (one lane): input producer; loads tile t's input box [n3 slices x
//     128 pixels] into input slot t % NI;
//   warp 2 (one lane): prev producer; loads tile t's prev box into output
//     slot t % 2 once that slot's previous store has read it (without prev
//     it only hands the slot on);
//   warps 3..10: split the staged input into the NS BF16 planes of A (same
//     swizzled MN-major layout as k_tube; zero for slices >= n3). With two
//     planes (32 KB, the slot's size) the split is written over the slot
//     itself once all eight warps have read it, so A is as deep as the input
//     ring and the split of the next tile does not wait for these MMAs; the
//     three planes of the FP32-level form go to a separate A buffer;
//   warp 1 (one lane): tcgen05.mma into accumulator buffer t % 2 (2 x 64
//     tensor-memory columns); one commit frees the input slot (or the A
//     buffer), another hands the accumulator to the epilogue;
//   warps 11..18: epilogue; thread = pixel = tensor-memory lane, two warps a
//     lane quadrant, each taking 32 of the 64 outputs. It writes ca v + cp
//     prev over prev in the output slot (or the GEMM operand's BF16 or TF32
//     tile), and one thread stores the slot by TMA and frees it once the
//     store has read it.
// Eight warps split and eight write back, so that the ALU work of both stays
// behind the loads (with four each, the split alone took about a tile period).
// (The three-plane BF16 operand of the FP32-level form, 48 KB a tile, does
// not fit a slot; k_tube writes it.)
// So input loads run up to NI tiles ahead and prev loads and stores overlap
// the split and the MMAs of the next tiles. Requirements (checked by the
// launcher, else k_tube runs): P % 8 == 0 (16-byte rows of the FP32 and BF16
// boxes), 16-byte aligned tensors, no dot-product reduction.
// NRM (BF16 output, two planes): a second matrix N multiplies the same A
// planes into a second pair of accumulators, and the epilogue sums the
// squares of in x_3 N into ep.red instead of storing them. The dual-domain
// iteration (transform-domain LSQR under the TH product) uses it to form the
// next GEMM operand, bf16(in x_3 G), and the Frobenius norm of the spatial
// tensor, ||in x_3 N||_F, in one pass over `in`.
// INB (FP32 output, two B planes): the input is BF16 and lands by TMA (128-byte
// swizzle, two boxes of 64 pixels x 64 slices) directly in the A operand's
// layout, one plane, so no converter stage runs; two MMA passes (B hi, lo).
constexpr int TT_NT = 608;
constexpr uint32_t TT_SLOT = TK * TP * 4;  // one FP32 box of 64 x 128: 32 KB
// Slots: two planes (A in the input slot) 3 input + 3 output, or 4 + 4
// half-size output slots for a BF16 output (16 KB a tile); three planes (a
// separate A buffer, larger B) 2 + 2.
constexpr int tube_tma_in(int ns, int out, bool inb = false) {
  return inb ? 6 : (ns == 3 ? 2 : (out == OUT_BF16 ? 4 : 3));
}
constexpr int tube_tma_out(int ns, int out) { return ns == 3 ? 2 : (out == OUT_BF16 ? 4 : 3); }
constexpr uint32_t tube_tma_oslot(int out) { return out == OUT_BF16 ? TT_SLOT / 2 : TT_SLOT; }
constexpr size_t tube_tma_smem(int ns, int out, bool nrm = false, bool inb = false) {
  return 1024 + tube_tma_in(ns, out, inb) * (inb ? TA_BYTES : TT_SLOT) +
         tube_tma_out(ns, out) * tube_tma_oslot(out) + (ns == 3 ? ns * TA_BYTES : 0) +
         (nrm ? 2 : 1) * ns * TB_BYTES + (3 * tube_tma_in(ns, out, inb) + 3 * tube_tma_out(ns, out) + 7) * 8 +
         16;
}

template <int OUT, int NS, bool NRM = false, bool INB = false>
__global__ void __launch_bounds__(TT_NT, 1)
k_tube_tma(const __grid_constant__ CUtensorMap tmIn, const __grid_constant__ CUtensorMap tmPrev,
           const __grid_constant__ CUtensorMap tmOut, const float* __restrict__ T,
           const float* __restrict__ N, int n3, size_t P, int has_prev, Epi ep, int* err,
           LsqrStep after) {
  static_assert(!INB || (OUT == OUT_F32 && NS == 2 && !NRM), "BF16 input: the pass back");
  constexpr int NPASS = INB ? 2 : (NS == 2 ? 3 : 6);  // INB: A (one plane) x B hi, lo
  constexpr int NI = tube_tma_in(NS, OUT, INB), NO = tube_tma_out(NS, OUT);
  constexpr uint32_t ISLOT = INB ? TA_BYTES : TT_SLOT;  // one input slot
  constexpr uint32_t OSLOT = tube_tma_oslot(OUT);
  constexpr bool INPLACE = NS == 2;  // A planes over the input slot
  constexpr bool RED = OUT == OUT_F32 || NRM;  // the pass reduces into ep.red
  constexpr uint32_t NCOL = NRM ? 4 * TK : 2 * TK;  // tensor-memory columns
  static_assert(!NRM || (OUT == OUT_BF16 && NS == 2), "the norm pass writes a BF16 operand");
  using namespace tc5;
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (0u << 16) |
                             ((uint32_t)(TK >> 3) << 17) | ((uint32_t)(TP >> 4) << 24);
  // `after` (alpha non-null): the scalars of an LSQR step that need this
  // pass's norm, run by the CTA that finishes the norm (see the end); a
  // skipped pass still hands the done flag on
  if (ep.skip && *ep.skip) {
    if (after.alpha && blockIdx.x == 0 && threadIdx.x == 0) *after.done_out = 1;
    return;
  }
  extern __shared__ uint8_t tt_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(tt_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sin = base;                    // NI input slots
  uint8_t* sout = base + NI * ISLOT;      // NO prev / output slots
  uint8_t* sAx = sout + NO * OSLOT;       // three planes: the A buffer
  uint8_t* sB = sAx + (INPLACE ? 0 : NS * TA_BYTES);  // NS B planes (NRM: then N's NS planes)
  uint64_t* ifull = reinterpret_cast<uint64_t*>(sB + (NRM ? 2 : 1) * NS * TB_BYTES);  // [NI] input loaded
  uint64_t* iempty = ifull + NI;          // [NI] input split (8 converter warps)
  // A planes written (8 converter warps), one barrier an input slot: the
  // converters may run up to NI tiles ahead of the MMAs when A is in place,
  // more than one barrier's phase parity can tell apart
  uint64_t* afull = iempty + NI;          // [NI]
  uint64_t* ofull = afull + NI;           // [NO] output slot holds prev (or is free)
  uint64_t* oempty = ofull + NO;          // [NO] output slot stored (read by the TMA store)
  uint64_t* owrit = oempty + NO;          // [NO] output tile written (8 epilogue warps)
  uint64_t* aempty = owrit + NO;          // the A buffer read by the MMAs (three planes)
  uint64_t* dfull = aempty + 1;           // [2] accumulator ready
  uint64_t* dempty = aempty + 3;          // [2] accumulator drained (8 epilogue warps)
  uint64_t* fin = aempty + 5;             // every MMA of this CTA completed
  uint64_t* cread = aempty + 6;           // the input slot read (8 converter warps)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(aempty + 7);
  __shared__ int sh_fail;
  __shared__ float sh_coef[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntile = (int)((P + TP - 1) / TP);
  const uint32_t box = (uint32_t)n3 * TP * 4;  // bytes of one FP32 box
  static_assert(OUT != OUT_BF16X3, "the three-plane operand is k_tube's");

  if (tid == 0) {
    for (int b = 0; b < NI; ++b) {
      mbar_init(ifull + b, 1);
      mbar_init(iempty + b, (INPLACE || INB) ? 1 : 8);
      mbar_init(afull + b, 8);
    }
    for (int b = 0; b < NO; ++b) {
      mbar_init(ofull + b, 1);
      mbar_init(oempty + b, 1);
      mbar_init(owrit + b, 8);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(dfull + b, 1);
      mbar_init(dempty + b, 8);
    }
    mbar_init(aempty, 1);
    mbar_init(fin, 1);
    mbar_init(cread, 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh_fail = 0;
  }
  if (OUT == OUT_F32) coef_compute(ep.coef, sh_coef);
  if (warp >= 3 && warp < 11) {  // B = T once: unit u is row n = u / 8, slices 8 (u % 8) + 0..7
    const int ct = tid - 96;
#pragma unroll
    for (int j = 0; j < (NRM ? 4 : 2); ++j) {  // NRM: j >= 2 stages N
      const int u = ct + 256 * (j & 1), n = u >> 3, c = u & 7;
      const float* src = j < 2 ? T : N;
      uint8_t* dst = sB + (j < 2 ? 0 : NS * TB_BYTES);
      float t[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int l = 8 * c + e;
        t[e] = (n < n3 && l < n3) ? __ldg(src + (size_t)n * n3 + l) : 0.f;
      }
      uint4 pl[NS];
      split8<NS>(t, pl);
      const uint32_t off = n * 128 + ((c ^ (n & 7)) << 4);
#pragma unroll
      for (int q = 0; q < NS; ++q) *reinterpret_cast<uint4*>(dst + q * TB_BYTES + off) = pl[q];
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tslot)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  volatile int* vfail = &sh_fail;
  float local = 0.f;
  int issued = 0, issued_p = 0;  // tiles whose input (prev) loads were issued

  if (warp == 0) {
    if (lane == 0) {
      int i = 0;
      for (int t = blockIdx.x; t < ntile && !*vfail; t += gridDim.x, ++i) {
        const int s = i % NI;
        const uint32_t u = (uint32_t)(i / NI) & 1u;
        if (!mbar_wait(iempty + s, u ^ 1u)) {
          *vfail = 1;
          break;
        }
        if (INB) {  // two 64-pixel halves of the BF16 A operand, 128-byte swizzle
          mbar_expect_tx(ifull + s, TA_BYTES);
          tma_load_3d(sin + s * ISLOT, &tmIn, t * TP, 0, 0, ifull + s);
          tma_load_3d(sin + s * ISLOT + TA_BYTES / 2, &tmIn, t * TP + TP / 2, 0, 0, ifull + s);
        } else {
          mbar_expect_tx(ifull + s, box);
          tma_load_2d(sin + s * TT_SLOT, &tmIn, t * TP, 0, ifull + s);
        }
        issued = i + 1;
      }
    }
  } else if (warp == 2) {
    if (lane == 0) {
      int i = 0;
      for (int t = blockIdx.x; t < ntile && !*vfail; t += gridDim.x, ++i) {
        const int s = i % NO;
        const uint32_t u = (uint32_t)(i / NO) & 1u;
        if (!mbar_wait(oempty + s, u ^ 1u)) {
          *vfail = 1;
          break;
        }
        if (has_prev) {
          mbar_expect_tx(ofull + s, box);
          tma_load_2d(sout + s * OSLOT, &tmPrev, t * TP, 0, ofull + s);
          issued_p = i + 1;
        } else {
          mbar_arrive(ofull + s);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int i = 0;
      for (int t = blockIdx.x; t < ntile && !*vfail; t += gridDim.x, ++i) {
        const int d = i & 1;
        const uint32_t u = (uint32_t)(i >> 1) & 1u;
        if (!mbar_wait((INB ? ifull : afull) + i % NI, (uint32_t)(i / NI) & 1u) ||
            !mbar_wait(dempty + d, u ^ 1u)) {
          *vfail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(d * TK);
        uint8_t* sA = INPLACE ? sin + (i % NI) * ISLOT : sAx;
#pragma unroll
        for (int m = 0; m < (NRM ? 2 : 1); ++m) {  // m = 1: N into the second pair
#pragma unroll
          for (int pass = 0; pass < NPASS; ++pass) {
            const uint32_t a0 = su32(sA + tube_pa(pass) * TA_BYTES);
            const uint32_t b0 = su32(sB + (m * NS + tube_pb(pass)) * TB_BYTES);
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk)
              umma<0>(acc + (uint32_t)(m * 2 * TK),
                      smem_desc(a0 + kk * 16 * 128, TA_BYTES / 2, 1024),
                      smem_desc(b0 + kk * 16 * 2, 16, 1024), IDESC, (pass | kk) != 0);
          }
        }
        umma_commit(INPLACE ? iempty + (i % NI) : aempty);  // the A planes are read
        umma_commit(dfull + d);
      }
      umma_commit(fin);
    }
  } else if (warp < 11) {  // converters (none with INB: the input is the A operand)
    const int ct = tid - 96;
    int i = 0;
    for (int t = blockIdx.x; t < ntile && !INB; t += gridDim.x, ++i) {
      if (__any_sync(0xffffffffu, *vfail)) break;
      const int s = i % NI;
      const uint32_t u = (uint32_t)(i / NI) & 1u;
      bool ok = mbar_wait(ifull + s, u);
      if (!INPLACE) ok = ok && mbar_wait(aempty, ((uint32_t)i & 1u) ^ 1u);
      if (!__all_sync(0xffffffffu, ok)) {
        *vfail = 1;
        break;
      }
      uint8_t* slot = sin + s * TT_SLOT;
      const float* stg = reinterpret_cast<const float*>(slot);
      float x[4][8];  // four units: slice l, pixels 8 c .. 8 c + 7
#pragma unroll
      for (int i8 = 0; i8 < 4; ++i8) {
        const int uu = ct + 256 * i8, l = uu >> 4, c = uu & 15;
        if (l < n3) {
          const float4 a = *reinterpret_cast<const float4*>(stg + l * TP + 8 * c);
          const float4 b = *reinterpret_cast<const float4*>(stg + l * TP + 8 * c + 4);
          x[i8][0] = a.x; x[i8][1] = a.y; x[i8][2] = a.z; x[i8][3] = a.w;
          x[i8][4] = b.x; x[i8][5] = b.y; x[i8][6] = b.z; x[i8][7] = b.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) x[i8][e] = 0.f;
        }
      }
      if (INPLACE) {  // every warp has read the slot before any writes over it
        __syncwarp();
        if (lane == 0) mbar_arrive(cread);
        if (!__all_sync(0xffffffffu, mbar_wait(cread, (uint32_t)i & 1u))) {
          *vfail = 1;
          break;
        }
      }
      uint8_t* sA = INPLACE ? slot : sAx;
#pragma unroll
      for (int i8 = 0; i8 < 4; ++i8) {
        const int uu = ct + 256 * i8, l = uu >> 4, c = uu & 15;
        uint4 pl[NS];
        split8<NS>(x[i8], pl);
        const uint32_t off = (c >> 3) * (TA_BYTES / 2) + l * 128 + (((c & 7) ^ (l & 7)) << 4);
#pragma unroll
        for (int q = 0; q < NS; ++q) *reinterpret_cast<uint4*>(sA + q * TA_BYTES + off) = pl[q];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(afull + s);
        if (!INPLACE) mbar_arrive(iempty + s);  // this warp has read the input slot
      }
    }
  } else {  // epilogue warps 11..18: tensor-memory lanes 32 (warp % 4) .., columns 32 hh ..
    const int qd = warp & 3, hh = (warp - 11) >> 2, px = 32 * qd + lane, et = tid - 352;
    const float ca = OUT == OUT_F32 ? sh_coef[0] : 1.f, cp = OUT == OUT_F32 ? sh_coef[1] : 0.f;
    int i = 0;
    for (int t = blockIdx.x; t < ntile; t += gridDim.x, ++i) {
      if (__any_sync(0xffffffffu, *vfail)) break;
      const int s = i % NO, d = i & 1;
      const uint32_t u = (uint32_t)(i / NO) & 1u, ud = (uint32_t)(i >> 1) & 1u;
      bool ok = mbar_wait(dfull + d, ud);
      ok = ok && mbar_wait(ofull + s, u);
      if (!__all_sync(0xffffffffu, ok)) {
        *vfail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint8_t* so = sout + s * OSLOT;  // prev in, output out (same element, same thread)
      const size_t p = (size_t)t * TP + px;
      const bool live = p < P;
      {
        const int h = hh;
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(d * TK + 32 * h), v);
        if (NRM) {  // the squares of in x_3 N (the second pair) into the norm
          float w[32];
          tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(2 * TK + d * TK + 32 * h), w);
          if (live) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (32 * h + j < n3) local = fmaf(w[j], w[j], local);
          }
        }
        // this warp's part of the accumulator is read: hand it back
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(dempty + d);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int k = 32 * h + j;
          if (k >= n3) continue;
          const int o = k * TP + px;
          if (OUT == OUT_BF16) {
            reinterpret_cast<__nv_bfloat16*>(so)[o] = __float2bfloat16_rn(v[j]);
          } else if (OUT == OUT_TF32) {
            reinterpret_cast<float*>(so)[o] = round_tf32(v[j]);
          } else {
            float* f = reinterpret_cast<float*>(so);
            float y = ca * v[j];
            if (has_prev) y = fmaf(cp, f[o], y);
            f[o] = y;
            if (live) local = fmaf(y, y, local);
          }
        }
      }
      // every thread's writes to the async proxy, one arrival a warp; the
      // storing thread waits (bounded) for all eight warps (a failed wait
      // only raises the flag: each warp leaves the loop at its next check)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(owrit + s);
      // One store stays in flight: once this tile's store is issued, the
      // previous one has read its slot, which goes back to the prev producer.
      if (et == 0) {
        if (mbar_wait(owrit + s, u)) {
          tma_store_2d(&tmOut, t * TP, 0, so);
          bulk_commit();
          if (i > 0) {
            bulk_wait_read1();
            mbar_arrive(oempty + (i - 1) % NO);
          }
        } else {
          *vfail = 1;
        }
      }
    }
    if (et == 0) {  // the last store's slot (and every store) done
      bulk_wait_all();
      if (i > 0 && !*vfail) mbar_arrive(oempty + (i - 1) % NO);
    }
  }

  // wind down: every thread of the CTA
  __syncthreads();
  const bool failed = *vfail != 0;
  if (warp == 1 && lane == 0) mbar_wait(fin, 0);  // the MMAs have finished with TMEM
  if (failed && warp == 0 && lane == 0) {          // let the input loads this CTA issued land
    for (int g = (issued > NI ? issued - NI : 0); g < issued; ++g)
      mbar_wait(ifull + g % NI, (uint32_t)(g / NI) & 1u);
    atomicExch(err, TC_ETIMEOUT);
  }
  if (failed && warp == 2 && lane == 0) {  // and the prev loads
    for (int g = (issued_p > NO ? issued_p - NO : 0); g < issued_p; ++g)
      mbar_wait(ofull + g % NO, (uint32_t)(g / NO) & 1u);
  }
  if (RED && ep.red.out) {  // every thread of every CTA
    const bool last = reduce_finish(local, ep.red);
    if (last && after.alpha && tid == 0) {  // the norm is in place: the step's scalars
      if (*after.done_in) {
        *after.done_out = 1;
      } else {
        float sh[3];
        lsqr_step_scalars(after, sh, true);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL)
                 : "memory");
}

// ------------------------------------------------------- chained pass back --
// The pass back from BF16 slice products (as k_tube_tma<OUT_F32, 2, INB>):
// y = ca (in x_3 T) + cp prev, written in FP32 with its norm, and in the same
// pass nxt = bf16(y x_3 T2), the next product's GEMM operand (the transform
// that product would start with), so that product skips its own first pass.
// Roles (640 threads, one CTA a SM):
//   warp 0 (one lane): BF16 input by TMA straight into the A1 operand;
//   warp 2 (one lane): the y ring: the first CH_NO prev loads, then per tile
//     the TMA store of y and, once the store and the eight splitter warps
//     have read the slot (nine arrivals), the prev load CH_NO tiles ahead
//     into it;
//   warp 1 (one lane): MMA1 (A1 x T, two passes) into acc1[i & 1], then
//     MMA2 of the previous tile (A2 x T2, three passes) into acc2;
//   warps 11..18: epilogue: y from acc1 and prev over prev in the y slot,
//     norm;
//   warps 3..10: split y (FP32, from the y slot) into the two BF16 planes of
//     A2; drain acc2 of the tile before to BF16 into the nxt slot;
//   warp 19 (one lane): the TMA store of the nxt slot, which it frees once
//     the store has read it.
// Both store threads wait for their store's reads at once, and each splitter
// warp hands its part of the y slot back itself: a split or a drain that
// waited for a store or for the other warps held up the tile after it
// (measured).
constexpr int CH_NI = 3, CH_NO = 3, CH_NT = TT_NT + 32;
constexpr size_t tube_chain_smem() {
  return 1024 + CH_NI * TA_BYTES + CH_NO * TT_SLOT + 2 * TA_BYTES + TT_SLOT / 2 +
         4 * TB_BYTES + (3 * CH_NI + 3 * CH_NO + 16) * 8 + 16;
}

__global__ void __launch_bounds__(CH_NT, 1)
k_tube_chain(const __grid_constant__ CUtensorMap tmIn, const __grid_constant__ CUtensorMap tmPrev,
             const __grid_constant__ CUtensorMap tmOut, const __grid_constant__ CUtensorMap tmNxt,
             const float* __restrict__ T, const float* __restrict__ T2, int n3, size_t P,
             int has_prev, Epi ep, int* err, LsqrStep after) {
  using namespace tc5;
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (0u << 16) |
                             ((uint32_t)(TK >> 3) << 17) | ((uint32_t)(TP >> 4) << 24);
  if (ep.skip && *ep.skip) {
    if (after.alpha && blockIdx.x == 0 && threadIdx.x == 0) *after.done_out = 1;
    return;
  }
  extern __shared__ uint8_t ch_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(ch_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sin = base;                          // CH_NI BF16 A1 slots (16 KB)
  uint8_t* sy = sin + CH_NI * TA_BYTES;         // CH_NO prev / y slots (32 KB)
  uint8_t* sA2 = sy + CH_NO * TT_SLOT;          // the two planes of A2
  uint8_t* sN = sA2 + 2 * TA_BYTES;             // the nxt slot (BF16, 16 KB)
  uint8_t* sB = sN + TT_SLOT / 2;               // T's two planes, then T2's
  uint64_t* ifull = reinterpret_cast<uint64_t*>(sB + 4 * TB_BYTES);  // [NI] input landed
  uint64_t* iempty = ifull + CH_NI;             // [NI] MMA1 read the input
  uint64_t* ofull = iempty + CH_NI;             // [NO] y slot holds prev (or is free)
  uint64_t* oempty = ofull + CH_NO;             // [NO] stored and split (two arrivals)
  uint64_t* owrit = oempty + CH_NO;             // [NO] y written (8 epilogue warps)
  uint64_t* dfull = owrit + CH_NO;              // [2] acc1 ready
  uint64_t* dempty = dfull + 2;                 // [2] acc1 drained (8 epilogue warps)
  uint64_t* efull = dempty + 2;                 // [2] acc2 ready
  uint64_t* eempty = efull + 2;                 // [2] acc2 drained (8 splitter warps)
  uint64_t* a2full = eempty + 2;                // A2 written (8 splitter warps)
  uint64_t* a2empty = a2full + 1;               // MMA2 read A2
  uint64_t* nwrit = a2empty + 1;                // nxt slot written (8 splitter warps)
  uint64_t* nfree = nwrit + 1;                  // nxt slot read by its store
  uint64_t* fin = nfree + 1;                    // every MMA of this CTA completed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
  __shared__ int sh_fail;
  __shared__ float sh_coef[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntile = (int)((P + TP - 1) / TP);
  const uint32_t box = (uint32_t)n3 * TP * 4;  // bytes of one FP32 prev box

  if (tid == 0) {
    for (int b = 0; b < CH_NI; ++b) {
      mbar_init(ifull + b, 1);
      mbar_init(iempty + b, 1);
    }
    for (int b = 0; b < CH_NO; ++b) {
      mbar_init(ofull + b, 1);
      mbar_init(oempty + b, 9);
      mbar_init(owrit + b, 8);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(dfull + b, 1);
      mbar_init(dempty + b, 8);
      mbar_init(efull + b, 1);
      mbar_init(eempty + b, 8);
    }
    mbar_init(a2full, 8);
    mbar_init(a2empty, 1);
    mbar_init(nwrit, 8);
    mbar_init(nfree, 1);
    mbar_init(fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh_fail = 0;
  }
  coef_compute(ep.coef, sh_coef);
  if (warp >= 3 && warp < 11) {  // T and T2, two planes each
    const int ct = tid - 96;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int u = ct + 256 * (j & 1), n = u >> 3, c = u & 7;
      const float* src = j < 2 ? T : T2;
      uint8_t* dst = sB + (j < 2 ? 0 : 2 * TB_BYTES);
      float t[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int l = 8 * c + e;
        t[e] = (n < n3 && l < n3) ? __ldg(src + (size_t)n * n3 + l) : 0.f;
      }
      uint4 pl[2];
      split8<2>(t, pl);
      const uint32_t off = n * 128 + ((c ^ (n & 7)) << 4);
#pragma unroll
      for (int q = 0; q < 2; ++q) *reinterpret_cast<uint4*>(dst + q * TB_BYTES + off) = pl[q];
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tslot)),
                 "r"(4 * TK)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;  // acc1: columns 0, TK; acc2: 2 TK, 3 TK
  volatile int* vfail = &sh_fail;
  float local = 0.f;
  int issued = 0, issued_p = 0;

  if (warp == 0) {
    if (lane == 0) {
      int i = 0;
      for (int t = blockIdx.x; t < ntile && !*vfail; t += gridDim.x, ++i) {
        const int s = i % CH_NI;
        if (!mbar_wait(iempty + s, ((uint32_t)(i / CH_NI) & 1u) ^ 1u)) {
          *vfail = 1;
          break;
        }
        mbar_expect_tx(ifull + s, TA_BYTES);
        tma_load_3d(sin + s * TA_BYTES, &tmIn, t * TP, 0, 0, ifull + s);
        tma_load_3d(sin + s * TA_BYTES + TA_BYTES / 2, &tmIn, t * TP + TP / 2, 0, 0, ifull + s);
        issued = i + 1;
      }
    }
  } else if (warp == 2) {
    if (lane == 0) {  // the y ring: prev loads CH_NO tiles ahead of the stores of y
      const int nmine = (int)blockIdx.x < ntile
                            ? (ntile - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                            : 0;
      auto load = [&](int k) -> bool {
        const int s = k % CH_NO;
        if (!mbar_wait(oempty + s, ((uint32_t)(k / CH_NO) & 1u) ^ 1u)) return false;
        if (has_prev) {
          mbar_expect_tx(ofull + s, box);
          tma_load_2d(sy + s * TT_SLOT, &tmPrev, ((int)blockIdx.x + k * (int)gridDim.x) * TP, 0,
                      ofull + s);
          issued_p = k + 1;
        } else {
          mbar_arrive(ofull + s);
        }
        return true;
      };
      int il = 0;
      for (; il < CH_NO && il < nmine; ++il)
        if (!load(il)) {
          *vfail = 1;
          break;
        }
      for (int i = 0; i < nmine && !*vfail; ++i) {
        const int s = i % CH_NO;
        if (!mbar_wait(owrit + s, (uint32_t)(i / CH_NO) & 1u)) {
          *vfail = 1;
          break;
        }
        tma_store_2d(&tmOut, ((int)blockIdx.x + i * (int)gridDim.x) * TP, 0, sy + s * TT_SLOT);
        bulk_commit();
        bulk_wait_read();
        mbar_arrive(oempty + s);
        if (il < nmine) {
          if (!load(il)) {
            *vfail = 1;
            break;
          }
          ++il;
        }
      }
      bulk_wait_all();
    }
  } else if (warp == 1) {
    if (lane == 0) {
      auto mma2 = [&](int k) -> bool {  // tile k's A2 x T2 into acc2[k & 1]
        const int e = k & 1;
        if (!mbar_wait(a2full, (uint32_t)k & 1u) ||
            !mbar_wait(eempty + e, ((uint32_t)(k >> 1) & 1u) ^ 1u))
          return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)((2 + e) * TK);
#pragma unroll
        for (int pass = 0; pass < 3; ++pass) {
          const uint32_t a0 = su32(sA2 + tube_pa(pass) * TA_BYTES);
          const uint32_t b0 = su32(sB + (2 + tube_pb(pass)) * TB_BYTES);
#pragma unroll
          for (int kk = 0; kk < TK / 16; ++kk)
            umma<0>(acc, smem_desc(a0 + kk * 16 * 128, TA_BYTES / 2, 1024),
                    smem_desc(b0 + kk * 16 * 2, 16, 1024), IDESC, (pass | kk) != 0);
        }
        umma_commit(a2empty);
        umma_commit(efull + e);
        return true;
      };
      int i = 0;
      for (int t = blockIdx.x; t < ntile && !*vfail; t += gridDim.x, ++i) {
        const int d = i & 1;
        if (!mbar_wait(ifull + i % CH_NI, (uint32_t)(i / CH_NI) & 1u) ||
            !mbar_wait(dempty + d, ((uint32_t)(i >> 1) & 1u) ^ 1u)) {
          *vfail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(d * TK);
        const uint32_t a0s = su32(sin + (i % CH_NI) * TA_BYTES);
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          const uint32_t b0 = su32(sB + pass * TB_BYTES);
#pragma unroll
          for (int kk = 0; kk < TK / 16; ++kk)
            umma<0>(acc, smem_desc(a0s + kk * 16 * 128, TA_BYTES / 2, 1024),
                    smem_desc(b0 + kk * 16 * 2, 16, 1024), IDESC, (pass | kk) != 0);
        }
        umma_commit(iempty + i % CH_NI);
        umma_commit(dfull + d);
        if (i > 0 && !mma2(i - 1)) {
          *vfail = 1;
          break;
        }
      }
      if (i > 0 && !*vfail && !mma2(i - 1)) *vfail = 1;
      umma_commit(fin);
    }
  } else if (warp < 11) {  // splitters / nxt drain
    const int ct = tid - 96;
    const int qd = warp & 3, hh = (warp - 3) >> 2, px = 32 * qd + lane;
    auto drain = [&](int k) -> bool {  // tile k of acc2 to nxt
      const int e = k & 1;
      bool ok = mbar_wait(efull + e, (uint32_t)(k >> 1) & 1u);
      ok = ok && (k == 0 || mbar_wait(nfree, (uint32_t)(k - 1) & 1u));  // sN read by its store
      if (!__all_sync(0xffffffffu, ok)) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)((2 + e) * TK + 32 * hh), v);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(eempty + e);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int kq = 32 * hh + j;
        if (kq < n3) reinterpret_cast<__nv_bfloat16*>(sN)[kq * TP + px] = __float2bfloat16_rn(v[j]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(nwrit);
      return true;
    };
    int i = 0;
    for (int t = blockIdx.x; t < ntile; t += gridDim.x, ++i) {
      if (__any_sync(0xffffffffu, *vfail)) break;
      const int s = i % CH_NO;
      // y of tile i written; A2 free (MMA2 of tile i - 1 read it)
      bool ok = mbar_wait(owrit + s, (uint32_t)(i / CH_NO) & 1u);
      ok = ok && (i == 0 || mbar_wait(a2empty, ((uint32_t)(i - 1) & 1u)));
      if (!__all_sync(0xffffffffu, ok)) {
        *vfail = 1;
        break;
      }
      const float* stg = reinterpret_cast<const float*>(sy + s * TT_SLOT);
#pragma unroll
      for (int i8 = 0; i8 < 4; ++i8) {
        const int uu = ct + 256 * i8, l = uu >> 4, c = uu & 15;
        float x[8];
        if (l < n3) {
          const float4 a = *reinterpret_cast<const float4*>(stg + l * TP + 8 * c);
          const float4 b = *reinterpret_cast<const float4*>(stg + l * TP + 8 * c + 4);
          x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
          x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) x[e] = 0.f;
        }
        uint4 pl[2];
        split8<2>(x, pl);
        const uint32_t off = (c >> 3) * (TA_BYTES / 2) + l * 128 + (((c & 7) ^ (l & 7)) << 4);
#pragma unroll
        for (int q = 0; q < 2; ++q) *reinterpret_cast<uint4*>(sA2 + q * TA_BYTES + off) = pl[q];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(a2full);
        mbar_arrive(oempty + s);  // this warp has read its part of the y slot
      }
      if (i > 0 && !drain(i - 1)) {
        *vfail = 1;
        break;
      }
    }
    if (i > 0 && !*vfail && !drain(i - 1)) *vfail = 1;
  } else if (warp < 19) {  // epilogue warps 11..18
    const int qd = warp & 3, hh = (warp - 11) >> 2, px = 32 * qd + lane;
    const float ca = sh_coef[0], cp = sh_coef[1];
    int i = 0;
    for (int t = blockIdx.x; t < ntile; t += gridDim.x, ++i) {
      if (__any_sync(0xffffffffu, *vfail)) break;
      const int s = i % CH_NO, d = i & 1;
      bool ok = mbar_wait(dfull + d, (uint32_t)(i >> 1) & 1u);
      ok = ok && mbar_wait(ofull + s, (uint32_t)(i / CH_NO) & 1u);
      if (!__all_sync(0xffffffffu, ok)) {
        *vfail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* f = reinterpret_cast<float*>(sy + s * TT_SLOT);
      const bool live = (size_t)t * TP + px < P;
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(d * TK + 32 * hh), v);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(dempty + d);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int k = 32 * hh + j;
        if (k >= n3) continue;
        const int o = k * TP + px;
        float y = ca * v[j];
        if (has_prev) y = fmaf(cp, f[o], y);
        f[o] = y;
        if (live) local = fmaf(y, y, local);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(owrit + s);
    }
  } else if (lane == 0) {  // warp 19: the nxt stores, one tile at a time
    int k = 0;
    for (int t = blockIdx.x; t < ntile && !*vfail; t += gridDim.x, ++k) {
      if (!mbar_wait(nwrit, (uint32_t)k & 1u)) {
        *vfail = 1;
        break;
      }
      tma_store_2d(&tmNxt, t * TP, 0, sN);
      bulk_commit();
      bulk_wait_read();
      mbar_arrive(nfree);
    }
    bulk_wait_all();
  }

  __syncthreads();
  const bool failed = *vfail != 0;
  if (warp == 1 && lane == 0) mbar_wait(fin, 0);
  if (failed && warp == 0 && lane == 0) {
    for (int g = (issued > CH_NI ? issued - CH_NI : 0); g < issued; ++g)
      mbar_wait(ifull + g % CH_NI, (uint32_t)(g / CH_NI) & 1u);
    atomicExch(err, TC_ETIMEOUT);
  }
  if (failed && warp == 2 && lane == 0) {
    for (int g = (issued_p > CH_NO ? issued_p - CH_NO : 0); g < issued_p; ++g)
      mbar_wait(ofull + g % CH_NO, (uint32_t)(g / CH_NO) & 1u);
  }
  if (ep.red.out) {
    const bool last = reduce_finish(local, ep.red);
    if (last && after.alpha && tid == 0) {
      if (*after.done_in) {
        *after.done_out = 1;
      } else {
        float sh[3];
        lsqr_step_scalars(after, sh, true);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * TK)
                 : "memory");
}

// The TMA form when its requirements hold: P % 8 == 0 (16-byte rows of the
// FP32 and BF16 boxes), 16-byte aligned tensors, no dot-product reduction.
bool tube_tma_ok(const float* in, const void* out, size_t P, const Epi& ep) {
  auto al = [](const void* q) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  return P % 8 == 0 && P / TP < (1u << 30) && al(in) && al(out) && al(ep.prev) &&
         ep.red.other == nullptr;
}

template <int OUT, int NS, bool NRM = false>
int run_tube_tma(const float* in, void* out, const float* T, int n3, size_t P, const Epi& ep,
                 int* err, cudaStream_t st, const LsqrStep& after = LsqrStep{},
                 const float* N = nullptr) {
  CUtensorMap mi, mp, mo;
  TC_TRY(make_tmap_2d(&mi, in, 0, P, (size_t)n3, TP, n3));
  const int hp = (OUT == OUT_F32 && ep.prev) ? 1 : 0;
  if (hp)
    TC_TRY(make_tmap_2d(&mp, ep.prev, 0, P, (size_t)n3, TP, n3));
  else
    mp = mi;
  TC_TRY(make_tmap_2d(&mo, out, OUT == OUT_BF16 ? 1 : 0, P, (size_t)n3, TP, n3));
  const size_t ntile = (P + TP - 1) / TP;
  const unsigned grid = (unsigned)(ntile < (size_t)g_tube_sms ? ntile : (size_t)g_tube_sms);
  k_tube_tma<OUT, NS, NRM><<<grid, TT_NT, tube_tma_smem(NS, OUT, NRM), st>>>(
      mi, mp, mo, T, N, n3, P, hp, ep, err, after);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

}  // namespace

int launch_mode3(const float* in, float* out, const float* T_dev, int n3, size_t P,
                 const Epi& ep, cudaStream_t st) {
  TC_CHECK(n3 >= 1 && n3 <= TC_MAX_N3);
  return pick<OUT_F32>(in, out, T_dev, n3, P, ep, st);
}

int launch_mode3_lowp(const float* in, void* out, const float* T_dev, int n3, size_t P,
                      int bf16, const int* skip, cudaStream_t st) {
  TC_CHECK(n3 >= 1 && n3 <= TC_MAX_N3);
  Epi ep;
  ep.skip = skip;
  return bf16 ? pick<OUT_BF16>(in, out, T_dev, n3, P, ep, st)
              : pick<OUT_TF32>(in, out, T_dev, n3, P, ep, st);
}

namespace {
template <int KPW>
int init_kpw() {
  for (auto fn : {k_mode3<KPW, OUT_F32>, k_mode3<KPW, OUT_BF16>, k_mode3<KPW, OUT_TF32>})
    TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mode3_smem<KPW>()));
  return TC_OK;
}
}  // namespace

namespace {

// persistent grid: tube_ctas(ns) CTAs a SM, no more than one a tile
unsigned tube_grid(size_t P, int ns) {
  const size_t tiles = (P + TP - 1) / TP, cap = (size_t)tube_ctas(ns) * g_tube_sms;
  return (unsigned)(tiles < 1 ? 1 : (tiles < cap ? tiles : cap));
}
}  // namespace

int launch_mode3_tc(const float* in, float* out, const float* T_dev, int n3, size_t P,
                    const Epi& ep, int* err, cudaStream_t st, int split3, const LsqrStep* after) {
  TC_CHECK(n3 >= 1 && n3 <= TK);
  TC_CHECK(!after || (after->alpha && !after->X && ep.red.out));  // scalars after a norm only
  if (tube_tma_ok(in, out, P, ep))
    return split3 ? run_tube_tma<OUT_F32, 3>(in, out, T_dev, n3, P, ep, err, st,
                                             after ? *after : LsqrStep{})
                  : run_tube_tma<OUT_F32, 2>(in, out, T_dev, n3, P, ep, err, st,
                                             after ? *after : LsqrStep{});
  if (split3)
    k_tube<OUT_F32, 3><<<tube_grid(P, 3), TNT, tube_smem(3), st>>>(in, out, T_dev, n3, P, ep, err);
  else
    k_tube<OUT_F32, 2><<<tube_grid(P, 2), TNT, tube_smem(2), st>>>(in, out, T_dev, n3, P, ep, err);
  TC_CUDA(cudaGetLastError());
  if (after) TC_TRY(launch_lsqr_scalars(*after, st));  // its own launch after the pass
  return TC_OK;
}

int launch_mode3_tc_inb(const void* in, float* out, const float* T_dev, int n3, size_t P,
                        const Epi& ep, int* err, cudaStream_t st, const LsqrStep* after) {
  TC_CHECK(n3 > 0 && n3 <= TK);
  TC_CHECK(!after || (after->alpha && !after->X && ep.red.out));
  auto al = [](const void* q) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  // the input map's inner extent is an int: P < 2^31
  if (P % 8 || P >= (1u << 31) || !al(in) || !al(out) || !al(ep.prev) || ep.red.other)
    return TC_EUNSUPPORTED;
  CUtensorMap mi, mp, mo;
  // BF16 input as a 3-D map (P, n3, 1), box 64 pixels x 64 slices, 128-byte
  // swizzle: the A operand's layout; slices >= n3 read as zero
  TC_TRY(make_tmap(&mi, in, 1, (int)P, n3, 1, TP / 2, TK));
  const int hp = ep.prev ? 1 : 0;
  if (hp)
    TC_TRY(make_tmap_2d(&mp, ep.prev, 0, P, (size_t)n3, TP, n3));
  TC_TRY(make_tmap_2d(&mo, out, 0, P, (size_t)n3, TP, n3));
  if (!hp) mp = mo;
  const size_t ntile = (P + TP - 1) / TP;
  const unsigned grid = (unsigned)(ntile < (size_t)g_tube_sms ? ntile : (size_t)g_tube_sms);
  k_tube_tma<OUT_F32, 2, false, true><<<grid, TT_NT, tube_tma_smem(2, OUT_F32, false, true), st>>>(
      mi, mp, mo, T_dev, nullptr, n3, P, hp, ep, err, after ? *after : LsqrStep{});
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_mode3_tc_chain(const void* in, float* out, const float* T_dev, void* nxt,
                          const float* T2_dev, int n3, size_t P, const Epi& ep, int* err,
                          cudaStream_t st, const LsqrStep* after) {
  TC_CHECK(n3 > 0 && n3 <= TK && nxt && T2_dev);
  TC_CHECK(!after || (after->alpha && !after->X && ep.red.out));
  auto al = [](const void* q) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  if (P % 8 || P >= (1u << 31) || !al(in) || !al(out) || !al(nxt) || !al(ep.prev) ||
      ep.red.other)
    return TC_EUNSUPPORTED;
  CUtensorMap mi, mp, mo, mn;
  TC_TRY(make_tmap(&mi, in, 1, (int)P, n3, 1, TP / 2, TK));
  const int hp = ep.prev ? 1 : 0;
  TC_TRY(make_tmap_2d(&mo, out, 0, P, (size_t)n3, TP, n3));
  if (hp)
    TC_TRY(make_tmap_2d(&mp, ep.prev, 0, P, (size_t)n3, TP, n3));
  else
    mp = mo;
  TC_TRY(make_tmap_2d(&mn, nxt, 1, P, (size_t)n3, TP, n3));
  const size_t ntile = (P + TP - 1) / TP;
  const unsigned grid = (unsigned)(ntile < (size_t)g_tube_sms ? ntile : (size_t)g_tube_sms);
  k_tube_chain<<<grid, CH_NT, tube_chain_smem(), st>>>(mi, mp, mo, mn, T_dev, T2_dev, n3, P, hp,
                                                       ep, err, after ? *after : LsqrStep{});
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// Whether the BF16-input pass takes this plan's shapes: the encoder accepts
// the input map (box of 64 slices over n3 of them).
bool tube_inb_ok(const void* buf, int n3, size_t P) {
  if (n3 <= TC_TUBE_MIN_N3 || n3 > TK || P % 8 || P >= (1u << 31)) return false;
  if (reinterpret_cast<uintptr_t>(buf) & 15) return false;
  CUtensorMap m;
  return make_tmap(&m, buf, 1, (int)P, n3, 1, TP / 2, TK) == TC_OK;
}

int launch_mode3_tc_norm(const float* in, void* out, const float* T_dev, const float* N_dev,
                         int n3, size_t P, const Epi& ep, int* err, cudaStream_t st,
                         const LsqrStep* after) {
  TC_CHECK(n3 > 0 && n3 <= TK && ep.red.out && !ep.prev);
  TC_CHECK(!after || (after->alpha && !after->X));
  if (!tube_tma_ok(in, out, P, ep)) return TC_EUNSUPPORTED;
  return run_tube_tma<OUT_BF16, 2, true>(in, out, T_dev, n3, P, ep, err, st,
                                         after ? *after : LsqrStep{}, N_dev);
}

int launch_mode3_tc_lowp(const float* in, void* out, const float* T_dev, int n3, size_t P,
                         int kind, const int* skip, int* err, cudaStream_t st) {
  TC_CHECK(n3 >= 1 && n3 <= TK);
  Epi ep;
  ep.skip = skip;
  // the three-plane operand (48 KB a tile, stored directly by the TMA form)
  // measured faster on k_tube's four CTAs a SM
  if (kind != ROUND_BF16X3 && tube_tma_ok(in, out, P, ep)) {
    if (kind == ROUND_BF16) return run_tube_tma<OUT_BF16, 2>(in, out, T_dev, n3, P, ep, err, st);
    return run_tube_tma<OUT_TF32, 2>(in, out, T_dev, n3, P, ep, err, st);
  }
  if (kind == ROUND_BF16X3)
    k_tube<OUT_BF16X3, 3><<<tube_grid(P, 3), TNT, tube_smem(3), st>>>(in, out, T_dev, n3, P, ep,
                                                                        err);
  else if (kind == ROUND_BF16)
    k_tube<OUT_BF16, 2><<<tube_grid(P, 2), TNT, tube_smem(2), st>>>(in, out, T_dev, n3, P, ep, err);
  else
    k_tube<OUT_TF32, 2><<<tube_grid(P, 2), TNT, tube_smem(2), st>>>(in, out, T_dev, n3, P, ep, err);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int transform_init() {
  // several CTAs of 50 (NS = 2) or 73 KB (NS = 3) a SM need the largest carveout
  for (auto fn : {k_tube<OUT_F32, 2>, k_tube<OUT_BF16, 2>, k_tube<OUT_TF32, 2>}) {
    TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tube_smem(2)));
    TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
  }
  TC_CUDA(cudaFuncSetAttribute(k_tube_tma<OUT_F32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tube_tma_smem(2, OUT_F32)));
  TC_CUDA(cudaFuncSetAttribute(k_tube_tma<OUT_BF16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tube_tma_smem(2, OUT_BF16)));
  TC_CUDA(cudaFuncSetAttribute(k_tube_tma<OUT_TF32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tube_tma_smem(2, OUT_TF32)));
  TC_CUDA(cudaFuncSetAttribute(k_tube_tma<OUT_F32, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tube_tma_smem(3, OUT_F32)));
  TC_CUDA(cudaFuncSetAttribute(k_tube_chain, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tube_chain_smem()));
  TC_CUDA(cudaFuncSetAttribute(k_tube_tma<OUT_F32, 2, false, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tube_tma_smem(2, OUT_F32, false, true)));
  TC_CUDA(cudaFuncSetAttribute(k_tube_tma<OUT_BF16, 2, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tube_tma_smem(2, OUT_BF16, true)));
  for (auto fn : {k_tube<OUT_F32, 3>, k_tube<OUT_BF16X3, 3>}) {
    TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tube_smem(3)));
    TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
  }
  int dev = 0;
  TC_CUDA(cudaGetDevice(&dev));
  TC_CUDA(cudaDeviceGetAttribute(&g_tube_sms, cudaDevAttrMultiProcessorCount, dev));
  TC_TRY(init_kpw<1>());
  TC_TRY(init_kpw<2>());
  TC_TRY(init_kpw<4>());
  TC_TRY(init_kpw<8>());
  return TC_OK;
}

int launch_round(const float* in, void* out, size_t n, int kind, cudaStream_t st,
                 const int* skip) {
  TC_CHECK(kind == ROUND_TF32 || kind == ROUND_BF16 || kind == ROUND_BF16X3);
  k_round<<<152 * 8, 256, 0, st>>>(
      in, out, n, kind == ROUND_BF16X3 ? OUT_BF16X3 : (kind == ROUND_BF16 ? OUT_BF16 : OUT_TF32),
      skip);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
