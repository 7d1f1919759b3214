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
int g_tube_sms = 152;  // SM count of the device (set by transform_init)

// persistent grid: tube_ctas(ns) CTAs a SM, no more than one a tile
unsigned tube_grid(size_t P, int ns) {
  const size_t tiles = (P + TP - 1) / TP, cap = (size_t)tube_ctas(ns) * g_tube_sms;
  return (unsigned)(tiles < 1 ? 1 : (tiles < cap ? tiles : cap));
}
}  // namespace

int launch_mode3_tc(const float* in, float* out, const float* T_dev, int n3, size_t P,
                    const Epi& ep, int* err, cudaStream_t st, int split3) {
  TC_CHECK(n3 >= 1 && n3 <= TK);
  if (split3)
    k_tube<OUT_F32, 3><<<tube_grid(P, 3), TNT, tube_smem(3), st>>>(in, out, T_dev, n3, P, ep, err);
  else
    k_tube<OUT_F32, 2><<<tube_grid(P, 2), TNT, tube_smem(2), st>>>(in, out, T_dev, n3, P, ep, err);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_mode3_tc_lowp(const float* in, void* out, const float* T_dev, int n3, size_t P,
                         int kind, const int* skip, int* err, cudaStream_t st) {
  TC_CHECK(n3 >= 1 && n3 <= TK);
  Epi ep;
  ep.skip = skip;
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
