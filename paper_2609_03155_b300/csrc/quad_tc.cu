// Quadrature contractions on the 5th-generation tensor cores (tcgen05,
// kind::tf32, FP32 accumulators in tensor memory).
//
// The real matrices of the element pass (M = V^T V, C = Cu^T Cu, P = V^T PhiL,
// Q = Cu^T PhiL, sums over the volume quadrature points of the scaled basis
// values, Sec. 2.3 / Algorithm 2) are dense contractions over K = 3 n_q.  In the
// reduced-precision modes they run here instead of the FP64 GEMM:
//   DPG_PREC_TF32    one TF32 product per term (operands rounded to TF32),
//   DPG_PREC_3XTF32  a = a_hi + a_lo with a_hi = tf32(a), a_lo = tf32(a - a_hi);
//                    a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (about FP32 accuracy).
// Everything after the contraction (G, B, the Cholesky factorisation, the
// condensation, CG residuals) stays FP64.
//
// One CTA (128 threads) computes a 128 x 128 tile of C for one element.  Per
// 32-wide K step the threads stage the operand tiles from the FP64 arrays into
// shared memory in the K-major core-matrix layout (8 rows x 16 bytes per core
// matrix, no swizzle), one elected thread issues the MMAs (M = 128, N = 128,
// K = 8 each) and commits them to an mbarrier, and the CTA waits on it before
// the next step overwrites the tiles.  The accumulator lives in tensor memory
// (128 lanes x 128 FP32 columns); the epilogue reads it with tcgen05.ld and
// writes FP64.  Every wait is bounded in time: on a timeout the CTA records an
// error, waits once more (bounded) for its MMAs, frees its tensor memory if
// they completed (else leaves it allocated) and returns.
#include <cstdint>

#include "dpg_internal.h"

namespace dpg {

namespace {

constexpr int TC_M = 128, TC_N = 128, TC_K = 32;  // CTA tile and K step
constexpr int TILE_BYTES = TC_M * TC_K * 4;       // one FP32 operand tile (16 KB)
constexpr int LBO = (TC_M / 8) * 128;             // K-adjacent core matrices (2048 B)
constexpr int SBO = 128;                          // M/N-adjacent core matrices
constexpr uint32_t TMEM_COLS = 256;               // allocation (N = 128 used)
constexpr unsigned long long WAIT_NS = 100000000ull;  // an mbarrier wait gives up after 100 ms

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, the fixed version bits 46..48 = 0b001, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(LBO >> 4) << 16;
  d |= (uint64_t)(SBO >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ unsigned long long tc_global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the mbarrier phase, bounded in time (WAIT_NS on the global
// nanosecond timer, whatever each try_wait's own suspension); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const unsigned long long t0 = tc_global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (done) return true;
    if (tc_global_ns() - t0 > WAIT_NS) return false;
  }
}

// Stage rows [r0, r0 + 128) x K [k0, k0 + 32) of X^T (X: Kd x ncol row-major
// FP64, row stride ld) into the K-major core layout: element (row t, k) at
// byte (k / 4) * LBO + t * 16 + (k % 4) * 4.  Thread t owns row t and writes
// 16-byte vectors (consecutive threads, consecutive vectors).
template <int SPLIT>
__device__ __forceinline__ void stage_tile(const double* __restrict__ X, int ld, int ncol, int Kd, int r0, int k0,
                                           float* hi, float* lo) {
  const int t = threadIdx.x;
  const int col = r0 + t;
  const bool in = col < ncol;
#pragma unroll
  for (int c = 0; c < TC_K / 4; ++c) {
    float h4[4], l4[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + 4 * c + j;
      const double a = (in && k < Kd) ? X[(size_t)k * ld + col] : 0.0;
      const float h = tf32_round((float)a);
      h4[j] = h;
      l4[j] = SPLIT == 3 ? tf32_round((float)(a - (double)h)) : 0.0f;
    }
    *reinterpret_cast<float4*>(reinterpret_cast<char*>(hi) + c * LBO + t * 16) = make_float4(h4[0], h4[1], h4[2], h4[3]);
    if (SPLIT == 3)
      *reinterpret_cast<float4*>(reinterpret_cast<char*>(lo) + c * LBO + t * 16) =
          make_float4(l4[0], l4[1], l4[2], l4[3]);
  }
}

}  // namespace

// C[b] (Ma x Nb, row-major, ldc) = A[b]^T B[b], A[b]: Kd x Ma (lda), B[b]: Kd x Nb (ldb), FP64.
// upper_only: tiles strictly below the diagonal are skipped (symmetric products).
template <int SPLIT>
__global__ void __launch_bounds__(128) k_gemm_tn_tc(int Ma, int Nb, int Kd, const double* __restrict__ A, int lda,
                                                    long long sA, const double* __restrict__ B, int ldb,
                                                    long long sB, double* C, int ldc, long long sC, int upper_only,
                                                    int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
  if (upper_only && n0 + TC_N <= m0) return;
  const int b = blockIdx.z;
  const double* Ab = A + b * sA;
  const double* Bb = B + b * sB;
  double* Cb = C + b * sC;
  float* Ahi = reinterpret_cast<float*>(smem);
  float* Bhi = reinterpret_cast<float*>(smem + TILE_BYTES);
  float* Alo = reinterpret_cast<float*>(smem + 2 * TILE_BYTES);
  float* Blo = reinterpret_cast<float*>(smem + 3 * TILE_BYTES);
  const int warp = threadIdx.x >> 5;
  const uint32_t mbar_a = smem_u32(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_tf32(TC_M, TC_N);
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < Kd && ok; k0 += TC_K) {
    stage_tile<SPLIT>(Ab, lda, Ma, Kd, m0, k0, Ahi, Alo);
    stage_tile<SPLIT>(Bb, ldb, Nb, Kd, n0, k0, Bhi, Blo);
    // generic-proxy stores -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int j = 0; j < TC_K / 8; ++j) {
        const uint32_t off = (uint32_t)(2 * j * LBO);  // K = 8: two core matrices along K
        const uint32_t acc0 = (k0 > 0 || j > 0) ? 1u : 0u;
        mma_tf32(tmem, smem_desc(smem_u32(Ahi) + off), smem_desc(smem_u32(Bhi) + off), idesc, acc0);
        if (SPLIT == 3) {
          mma_tf32(tmem, smem_desc(smem_u32(Ahi) + off), smem_desc(smem_u32(Blo) + off), idesc, 1u);
          mma_tf32(tmem, smem_desc(smem_u32(Alo) + off), smem_desc(smem_u32(Bhi) + off), idesc, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a));
    }
    // every thread waits; the CTA goes on only if all saw the phase complete
    ok = __syncthreads_and(mbar_wait(mbar_a, phase) ? 1 : 0) != 0;
    phase ^= 1u;
  }
  bool drained = true;
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    // once more (bounded) for the MMAs in flight; if they still have not
    // completed, the tensor memory they write is left allocated rather than
    // freed under them (the host reports DPG_ERR_TIMEOUT either way)
    drained = __syncthreads_and(mbar_wait(mbar_a, phase ^ 1u) ? 1 : 0) != 0;
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: warp w owns accumulator lanes (rows) 32 w .. 32 w + 31
    const int row = m0 + 32 * warp + (threadIdx.x & 31);
#pragma unroll 1
    for (int c0 = 0; c0 < TC_N; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < Ma) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col < Nb) Cb[(size_t)row * ldc + col] = (double)__uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0 && drained) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// Dynamic shared memory: four operand tiles plus slack that keeps every
// descriptor-addressed byte inside the allocation.
constexpr size_t TC_SMEM = 6 * (size_t)TILE_BYTES;

// Dynamic shared memory limits of both variants (once, outside any capture).
int tc_init() {
  if (cudaFuncSetAttribute(k_gemm_tn_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(k_gemm_tn_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM) != cudaSuccess)
    return DPG_ERR_CUDA;
  return DPG_OK;
}

int gemm_tn_tc(int split, int Ma, int Nb, int Kd, const double* A, int lda, long long sA, const double* B, int ldb,
               long long sB, double* C, int ldc, long long sC, int batch, int upper_only, int* err, cudaStream_t s) {
  dim3 grid((Nb + TC_N - 1) / TC_N, (Ma + TC_M - 1) / TC_M, batch);
  if (split == 3)
    k_gemm_tn_tc<3><<<grid, 128, TC_SMEM, s>>>(Ma, Nb, Kd, A, lda, sA, B, ldb, sB, C, ldc, sC, upper_only, err);
  else
    k_gemm_tn_tc<1><<<grid, 128, TC_SMEM, s>>>(Ma, Nb, Kd, A, lda, sA, B, ldb, sB, C, ldc, sC, upper_only, err);
  return cudaGetLastError() == cudaSuccess ? DPG_OK : DPG_ERR_CUDA;
}

}  // namespace dpg
