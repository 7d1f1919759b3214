// Frontal-slice GEMMs on the 5th-generation tensor cores (tcgen05), for the
// TF32 and BF16 precision forms of the c-product (Algorithm 1, step 2):
//   D_z = A_z B_z,  A_z: M x K (K contiguous), B_z: K x N (N contiguous),
//   D_z: M x N FP32, for every slice z.
//
// A persistent kernel, two CTAs per SM, each looping over 128 x 128 output
// tiles (tile t, t + gridDim.x, ...; columns fastest, then rows, then slices).
// The FP32 accumulator is double-buffered in tensor memory (2 x 128 columns
// a CTA, the SM's 512 between two CTAs), so the store of one tile overlaps
// the MMAs of the next:
//   warp 0, one lane : TMA producer (cp.async.bulk.tensor.3d, 128B swizzle)
//                      over every (tile, K block) of the CTA, into a
//                      STAGES-deep ring of (A, B) stages in shared memory;
//   warp 1, one lane : tcgen05.mma (kind::f16 with BF16 inputs, or
//                      kind::tf32) into accumulator buffer (i & 1) of the
//                      CTA's i-th tile; tcgen05.commit releases each stage
//                      and then hands the buffer to the epilogue;
//   warps 2..5       : epilogue; warp w reads tensor-memory lanes
//                      32 (w % 4) .. + 31, the lanes that warp may access.
// A is read K-major. B is read MN-major straight from the row-major K x N
// operand for BF16. For TF32 it is read K-major from a per-slice transposed
// copy (N x K): kind::tf32 with an MN-major B left the accumulator unchanged
// on this part. Each CTA fetches its own tiles (no cluster multicast).
//
// Every mbarrier wait is bounded. A wait that gives up raises *err, ends every
// role's loop, and the CTA waits (bounded) for the copies and MMAs it issued,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "tc_device.cuh"
#include "tcgen05.cuh"
#include "umma.cuh"

namespace {

using namespace tc5;

constexpr int BM = 128, BN = 128, STAGES = 3;  // 105 KB smem: 2 CTAs per SM (NPAIR 1)
constexpr uint32_t A_BYTES = BM * 128;   // 128 rows of one 128-byte K slab
constexpr uint32_t B_BYTES = 128 * BN;   // (128 / elem) K rows x BN columns

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
int g_nsm = 0;  // SMs of the device (persistent grid size: 2 CTAs per SM)

// KIND 0: BF16 inputs (kind::f16), KIND 1: TF32 inputs (kind::tf32).
// BKMAJ: B given as N x K per slice (K contiguous) instead of K x N.
// EPI: the Krylov epilogue in the store: D = ca * acc + cp * prev (prev may
// alias D; each element is read and written by one thread), an optional BF16
// copy of D into dlow (the next GEMM's operand), and the fused reduction of D.
// Without EPI the accumulator is stored as is.
constexpr int NT = 192;  // warps 0, 1: producer, MMA; warps 2..5: epilogue

// Stages: three of one (A, B) K block (two CTAs a SM); for the split
// products (NPAIR = 6), two of all three planes of both operands (96 KB a
// stage, one CTA a SM), so each plane is loaded once per K block.
__host__ __device__ constexpr int stage_planes(int npair) { return npair == 6 ? 3 : 1; }
__host__ __device__ constexpr int stage_count(int npair) { return npair == 6 ? 2 : STAGES; }

size_t smem_bytes(int npair = 1) {
  const int pl = stage_planes(npair), ns = stage_count(npair);
  return 1024 + ns * pl * (A_BYTES + B_BYTES) + 4 * 32 * 16 * 4 + (2 * ns + 5) * 8 + 16;
}


// Split-operand products (NPAIR = 6): A and B are each given as three BF16
// planes, x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0
// - x1)), stacked as slices p Z + z of one map. D accumulates the six products
// x_i y_j with i + j <= 2. The dropped terms and the residual of the split are
// near 2^-27 relative; the FP32 accumulation in the tensor core then sets the
// error (about 1e-6 relative at K = 64..512, a few times FFMA's).
__device__ __forceinline__ int pair_a(int p) { return p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0); }
__device__ __forceinline__ int pair_b(int p) { return p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0); }

// OUTB (plain store, BF16 inputs): D holds BF16 values (one rounding of the
// FP32 accumulator), for a consumer that reads BF16.
template <int KIND, int BKMAJ, bool EPI, int NPAIR = 1, bool OUTB = false>
__global__ void __launch_bounds__(NT, NPAIR == 6 ? 1 : 2)
k_umma_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            float* D, int M, int N, int K, int Z, int* err, const int* skip, Epi ep,
            __nv_bfloat16* dlow) {
  constexpr int ES = KIND == 0 ? 2 : 4;
  constexpr int BKE = 128 / ES;
  constexpr int UK = KIND == 0 ? 16 : 8;
  constexpr int NATOM = 128 / ES;
  constexpr int NBOX = BN / NATOM;
  constexpr uint32_t B_COL = BKE * 128;
  constexpr uint32_t FMT = KIND == 0 ? 1u : 2u;
  constexpr uint32_t BMAJ = BKMAJ ? 0u : 1u;
  constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) | (0u << 15) | (BMAJ << 16) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static_assert(!OUTB || (!EPI && KIND == 0), "BF16 store: the plain BF16 GEMM");
  constexpr int PL = stage_planes(NPAIR), NST = stage_count(NPAIR);
  constexpr uint32_t SA = PL * A_BYTES, SB = PL * B_BYTES;  // one stage's A, B bytes
  if (skip && *skip) return;
  const size_t zmn = (size_t)Z * M * N;  // values of one output plane
  extern __shared__ uint8_t dsm_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + NST * SA;
  float* sE = reinterpret_cast<float*>(sB + NST * SB);  // 4 warps x 32 x 16 floats
  uint64_t* full = reinterpret_cast<uint64_t*>(sE + 4 * 32 * 16);
  uint64_t* empty = full + NST;
  uint64_t* accf = empty + NST;  // [2]: accumulator buffer ready for the epilogue
  uint64_t* acce = accf + 2;        // [2]: accumulator buffer drained by the epilogue
  uint64_t* fin = acce + 2;         // every MMA of this CTA completed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
  __shared__ int sh_fail;
  __shared__ float sh_coef[2];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  const int ntile = tm * tn * Z;
  const int nk = (K + BKE - 1) / BKE;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf + b, 1);
      mbar_init(acce + b, 4);  // one arrival per epilogue warp
    }
    mbar_init(fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh_fail = 0;
  }
  if (EPI && threadIdx.x == 64) {  // an epilogue thread, idle until the first tile
    double ca = 1.0, cp = 0.0;
    const Coef& c = ep.coef;
    if (c.rule == COEF_GK) {
      const double s0 = *c.s0, s1 = *c.s1;
      ca = (s0 != 0.0) ? 1.0 / s0 : 0.0;
      cp = (s1 != 0.0) ? -s0 / s1 : 0.0;
    } else if (c.rule == COEF_INV) {
      const double s0 = *c.s0;
      ca = (s0 != 0.0) ? 1.0 / s0 : 0.0;
    } else if (c.rule == COEF_RESID) {
      ca = -1.0;
      cp = 1.0;
    } else if (c.rule == COEF_NEG) {
      ca = -1.0;
    } else if (c.rule == COEF_AXPY) {
      cp = -*c.s0;
    }
    sh_coef[0] = (float)ca;
    sh_coef[1] = (float)cp;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tslot)),
                 "r"(2 * BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  volatile int* vfail = &sh_fail;
  float local = 0.f;
  int issued = 0;  // producer: K blocks armed (for the bounded drain on failure)

  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      for (int t = blockIdx.x; t < ntile && !*vfail; t += gridDim.x) {
        const int z = t / (tm * tn), r = t % (tm * tn);
        const int m0 = (r / tn) * BM, n0 = (r % tn) * BN;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % NST;
          const uint32_t ph = (g / NST) & 1;
          if (!mbar_wait(empty + s, ph ^ 1)) {
            *vfail = 1;
            break;
          }
          mbar_expect_tx(full + s, SA + SB);
#pragma unroll
          for (int pl = 0; pl < PL; ++pl) {  // operand plane pl: slice pl Z + z
            const int zp = pl * Z + z;
            tma_load_3d(sA + s * SA + pl * A_BYTES, &tmA, kb * BKE, m0, zp, full + s);
            uint8_t* sb = sB + s * SB + pl * B_BYTES;
            if (BKMAJ) {
              tma_load_3d(sb, &tmB, kb * BKE, n0, zp, full + s);
            } else {
#pragma unroll
              for (int bx = 0; bx < NBOX; ++bx)
                tma_load_3d(sb + bx * B_COL, &tmB, n0 + bx * NATOM, kb * BKE, zp, full + s);
            }
          }
          issued = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int g = 0, i = 0;
      for (int t = blockIdx.x; t < ntile && !*vfail; t += gridDim.x, ++i) {
        const int b = i & 1, u = i >> 1;
        if (!mbar_wait(acce + b, (uint32_t)(u & 1) ^ 1u)) {
          *vfail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(b * BN);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % NST;
          const uint32_t ph = (g / NST) & 1;
          if (!mbar_wait(full + s, ph)) {
            *vfail = 1;
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int pr = 0; pr < NPAIR; ++pr) {  // product of planes (pair_a, pair_b)
            const uint32_t a0 = su32(sA + s * SA + pair_a(pr) * A_BYTES);
            const uint32_t b0 = su32(sB + s * SB + pair_b(pr) * B_BYTES);
#pragma unroll
            for (int kk = 0; kk < BKE / UK; ++kk) {
              const uint64_t ad = smem_desc(a0 + kk * UK * ES, 16, 1024);
              const uint64_t bd = BKMAJ ? smem_desc(b0 + kk * UK * ES, 16, 1024)
                                        : smem_desc(b0 + kk * UK * 128, B_COL, 1024);
              umma<KIND>(acc, ad, bd, IDESC, (kb | pr | kk) != 0);
            }
          }
          umma_commit(empty + s);
        }
        if (!ok) break;
        umma_commit(accf + b);
      }
      umma_commit(fin);  // completes once every MMA issued above has
    }
  } else {  // epilogue warps 2..5
    // Each 32-row x 16-column chunk goes tensor memory -> registers (one row
    // a lane) -> shared memory -> registers in a coalesced layout: lane l takes
    // float4 (l & 3) of rows 8 i + (l >> 2), so a warp instruction covers 8
    // rows x 64 contiguous bytes of D, prev and dlow instead of 32 rows x 16.
    // The float4 slot of (row r, quad j) is j ^ ((r >> 1) & 3): conflict-free
    // on both sides.
    const int eq = warp & 3;  // tensor-memory lanes 32 eq .. 32 eq + 31
    float* sw = sE + eq * (32 * 16);
    const int rsub = lane >> 2, jq = lane & 3;
    const bool nvec = (N & 3) == 0;
    int i = 0;  // the loop exit and the waits are warp-uniform: tcgen05.ld is .sync.aligned
    for (int t = blockIdx.x; t < ntile && !__any_sync(0xffffffffu, *vfail); t += gridDim.x, ++i) {
      const int b = i & 1, u = i >> 1;
      const int z = t / (tm * tn), r = t % (tm * tn);
      const int m0 = (r / tn) * BM + eq * 32, n0 = (r % tn) * BN;
      const size_t zoff = (size_t)z * M * N;
      // prev of chunk c (rows 8 i + rsub, columns 16 c + 4 jq) sits in
      // pre[4 (c % PD) + i], loaded PD chunks ahead; the first PD chunks load
      // before the wait, as they do not depend on this tile's MMAs.
      constexpr int NCH = BN / 16, PD = 3;
      float4 pre[EPI ? 4 * PD : 1];
      auto load_prev = [&](int c, int ii) {
        const int row = m0 + 8 * ii + rsub, col = n0 + 16 * c + 4 * jq;
        const bool whole = ep.prev && nvec && row < M && col + 4 <= N;
        return whole ? *reinterpret_cast<const float4*>(ep.prev + zoff + (size_t)row * N + col)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
      };
      if (EPI) {
#pragma unroll
        for (int q = 0; q < 4 * PD; ++q) pre[q] = load_prev(q >> 2, q & 3);
      }
      if (!__all_sync(0xffffffffu, mbar_wait(accf + b, (uint32_t)(u & 1)))) {
        *vfail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float ca = EPI ? sh_coef[0] : 1.f, cp = EPI ? sh_coef[1] : 0.f;
      const uint32_t tacc = tmem + ((uint32_t)(eq * 32) << 16) + (uint32_t)(b * BN);
      uint32_t rg[2][16];  // chunk c in rg[c & 1]; chunk c + 1 loads while c is stored
      tmem_ld16_issue(tacc, rg[0]);
      tmem_ld16_wait(rg[0]);
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const uint32_t* v = rg[c & 1];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          *reinterpret_cast<float4*>(sw + lane * 16 + 4 * (j ^ ((lane >> 1) & 3))) =
              make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                          __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
        __syncwarp();
        if (c + 1 < NCH) tmem_ld16_issue(tacc + (uint32_t)((c + 1) * 16), rg[(c + 1) & 1]);
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
          const int rr = 8 * ii + rsub;
          float4 y = *reinterpret_cast<const float4*>(sw + rr * 16 + 4 * (jq ^ ((rr >> 1) & 3)));
          const int row = m0 + rr, col = n0 + 16 * c + 4 * jq;
          if (row >= M || col >= N) continue;
          const size_t o = zoff + (size_t)row * N + col;
          if (nvec) {  // col + 4 <= N
            if (EPI) {
              if (ep.prev) {
                const float4 pv = pre[4 * (c % PD) + ii];
                y.x = fmaf(cp, pv.x, ca * y.x);
                y.y = fmaf(cp, pv.y, ca * y.y);
                y.z = fmaf(cp, pv.z, ca * y.z);
                y.w = fmaf(cp, pv.w, ca * y.w);
              } else {
                y.x *= ca;
                y.y *= ca;
                y.z *= ca;
                y.w *= ca;
              }
              if (ep.red.out) {
                const float4 ov = ep.red.other
                                      ? *reinterpret_cast<const float4*>(ep.red.other + o)
                                      : y;
                local = fmaf(y.x, ov.x, fmaf(y.y, ov.y, fmaf(y.z, ov.z, fmaf(y.w, ov.w, local))));
              }
            }
            if (OUTB) {
              const __nv_bfloat162 lo = __floats2bfloat162_rn(y.x, y.y);
              const __nv_bfloat162 hi = __floats2bfloat162_rn(y.z, y.w);
              uint2 pk;
              pk.x = *reinterpret_cast<const uint32_t*>(&lo);
              pk.y = *reinterpret_cast<const uint32_t*>(&hi);
              *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(D) + o) = pk;
            } else {
              *reinterpret_cast<float4*>(D + o) = y;
            }
            if (EPI && dlow) {  // PL planes of the next operand, Z M N values apart
              float4 r = y;
#pragma unroll
              for (int pl = 0; pl < PL; ++pl) {
                const __nv_bfloat162 lo = __floats2bfloat162_rn(r.x, r.y);
                const __nv_bfloat162 hi = __floats2bfloat162_rn(r.z, r.w);
                uint2 pk;
                pk.x = *reinterpret_cast<const uint32_t*>(&lo);
                pk.y = *reinterpret_cast<const uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(dlow + pl * zmn + o) = pk;
                r.x -= __low2float(lo);
                r.y -= __high2float(lo);
                r.z -= __low2float(hi);
                r.w -= __high2float(hi);
              }
            }
          } else {  // ragged row length: element by element
            const float ys[4] = {y.x, y.y, y.z, y.w};
            for (int e = 0; e < 4 && col + e < N; ++e) {
              float w = ys[e];
              if (EPI) {
                w *= ca;
                if (ep.prev) w = fmaf(cp, ep.prev[o + e], w);
                if (ep.red.out) local = fmaf(w, ep.red.other ? ep.red.other[o + e] : w, local);
              }
              if (OUTB)
                reinterpret_cast<__nv_bfloat16*>(D)[o + e] = __float2bfloat16_rn(w);
              else
                D[o + e] = w;
              if (EPI && dlow) {
                float r = w;
#pragma unroll
                for (int pl = 0; pl < PL; ++pl) {
                  const __nv_bfloat16 b = __float2bfloat16_rn(r);
                  dlow[pl * zmn + o + e] = b;
                  r -= __bfloat162float(b);
                }
              }
            }
          }
        }
        if (EPI && c + PD < NCH) {
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) pre[4 * (c % PD) + ii] = load_prev(c + PD, ii);
        }
        __syncwarp();  // the next chunk overwrites sw
        if (c + 1 < NCH) tmem_ld16_wait(rg[(c + 1) & 1]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(acce + b);  // this warp's lanes of buffer b are free
    }
  }

  // wind down: every thread of the CTA
  __syncthreads();
  const bool failed = *vfail != 0;
  if (warp == 1 && lane == 0) mbar_wait(fin, 0);  // the MMAs have finished with TMEM
  if (failed && warp == 0 && lane == 0) {          // let the copies this CTA issued land
    for (int g = (issued > NST ? issued - NST : 0); g < issued; ++g)
      mbar_wait(full + g % NST, (g / NST) & 1);
    atomicExch(err, TC_ETIMEOUT);
  }
  if (EPI && ep.red.out) reduce_finish(local, ep.red);  // every thread of every CTA
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN)
                 : "memory");
}

}  // namespace

namespace {
// One bounded wait on an mbarrier that nothing arrives on: the phase of
// parity 0 never completes, so the wait gives up after `spins` polls and the
// status is TC_ETIMEOUT. This is the path every wait of the tcgen05 kernels
// takes when its copies or MMAs do not arrive.
__global__ void k_wait_check(int spins, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool done = mbar_wait_n(&bar, 0, spins);
  if (threadIdx.x == 0) *status = done ? TC_OK : TC_ETIMEOUT;
}
}  // namespace

extern "C" int tc_check_bounded_wait(int spins, int* status, tc_stream_t stream) {
  if (!status || spins < 1 || spins > (1 << 20)) return TC_EINVAL;
  k_wait_check<<<1, 32, 0, (cudaStream_t)stream>>>(spins, status);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int umma_init() {
  for (auto fn : {k_umma_gemm<0, 0, false>, k_umma_gemm<1, 1, false>, k_umma_gemm<0, 0, true>,
                  k_umma_gemm<0, 0, false, 6>, k_umma_gemm<0, 0, true, 6>,
                  k_umma_gemm<0, 0, false, 1, true>}) {
    const int npair =
        (fn == k_umma_gemm<0, 0, false, 6> || fn == k_umma_gemm<0, 0, true, 6>) ? 6 : 1;
    TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes(npair)));
    // two CTAs of 105 KB (or one of 201 KB) a SM need the largest carveout
    TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
  }
  int dev = 0;
  TC_CUDA(cudaGetDevice(&dev));
  TC_CUDA(cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev));
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    TC_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return TC_EUNSUPPORTED;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return TC_OK;
}

// 3-D tiled map over `slices` row-major matrices rows x inner, box
// (box_inner, box_rows, 1), 128-byte swizzle, zero fill out of bounds.
int make_tmap(CUtensorMap* map, const void* base, int bf16, int inner, int rows, int slices,
              int box_inner, int box_rows) {
  if (!g_encode) return TC_EUNSUPPORTED;
  const cuuint64_t es = bf16 ? 2 : 4;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || ((cuuint64_t)inner * es) % 16 != 0)
    return TC_EINVAL;
  cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)slices};
  cuuint64_t strides[2] = {(cuuint64_t)inner * es, (cuuint64_t)inner * rows * es};
  cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? TC_OK : TC_EINVAL;
}

int make_tmap_2d(CUtensorMap* map, const void* base, int bf16, size_t inner, size_t rows,
                 int box_inner, int box_rows) {
  if (!g_encode) return TC_EUNSUPPORTED;
  const cuuint64_t es = bf16 ? 2 : 4;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || ((cuuint64_t)inner * es) % 16 != 0 ||
      ((cuuint64_t)box_inner * es) % 16 != 0 || box_inner > 256 || box_rows > 256)
    return TC_EINVAL;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)inner * es};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? TC_OK : TC_EINVAL;
}

// A operand: M x K per slice, K contiguous. B operand: K x N with N contiguous
// (BF16), or its transpose N x K with K contiguous (TF32).
int make_umma_maps(UmmaMaps* m, int kind, const void* A, const void* B, int M, int N, int K,
                   int slices, int nsplit) {
  const int bf16 = kind == 0;
  const int bke = bf16 ? 64 : 32;
  TC_CHECK(nsplit == 1 || (nsplit == 3 && bf16));
  TC_TRY(make_tmap(&m->a, A, bf16, K, M, slices * nsplit, bke, BM));
  if (bf16)
    TC_TRY(make_tmap(&m->b, B, bf16, N, K, slices * nsplit, 64, bke));
  else
    TC_TRY(make_tmap(&m->b, B, bf16, K, N, slices * nsplit, bke, BN));
  m->M = M;
  m->N = N;
  m->K = K;
  m->slices = slices;
  m->kind = kind;
  m->nsplit = nsplit;
  return TC_OK;
}

namespace {
unsigned grid_size(const UmmaMaps& m) {
  const long tiles = (long)((m.N + BN - 1) / BN) * ((m.M + BM - 1) / BM) * m.slices;
  const long cap = (m.nsplit == 3 ? 1L : 2L) * (g_nsm > 0 ? g_nsm : 152);  // CTAs a SM
  return (unsigned)(tiles < cap ? tiles : cap);
}
}  // namespace

int launch_umma(const UmmaMaps& m, float* D, int* err, const int* skip, cudaStream_t st,
                bool out_bf16) {
  Epi none;
  TC_CHECK(!out_bf16 || (m.kind == 0 && m.nsplit == 1));
  if (out_bf16)
    k_umma_gemm<0, 0, false, 1, true><<<grid_size(m), NT, smem_bytes(), st>>>(
        m.a, m.b, D, m.M, m.N, m.K, m.slices, err, skip, none, nullptr);
  else if (m.nsplit == 3)
    k_umma_gemm<0, 0, false, 6><<<grid_size(m), NT, smem_bytes(6), st>>>(
        m.a, m.b, D, m.M, m.N, m.K, m.slices, err, skip, none, nullptr);
  else if (m.kind == 0)
    k_umma_gemm<0, 0, false><<<grid_size(m), NT, smem_bytes(), st>>>(
        m.a, m.b, D, m.M, m.N, m.K, m.slices, err, skip, none, nullptr);
  else
    k_umma_gemm<1, 1, false><<<grid_size(m), NT, smem_bytes(), st>>>(
        m.a, m.b, D, m.M, m.N, m.K, m.slices, err, skip, none, nullptr);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_umma_epi(const UmmaMaps& m, float* D, __nv_bfloat16* dlow, const Epi& ep, int* err,
                    cudaStream_t st) {
  TC_CHECK(m.kind == 0);
  if (m.nsplit == 3)
    k_umma_gemm<0, 0, true, 6><<<grid_size(m), NT, smem_bytes(6), st>>>(
        m.a, m.b, D, m.M, m.N, m.K, m.slices, err, ep.skip, ep, dlow);
  else
    k_umma_gemm<0, 0, true><<<grid_size(m), NT, smem_bytes(), st>>>(
        m.a, m.b, D, m.M, m.N, m.K, m.slices, err, ep.skip, ep, dlow);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
