// Element factorisation with the trailing updates on the tensor cores, at FP64
// accuracy (the augmented partial Cholesky of the element pass, Sec. 2.3,
// Eq. linear_system).
//
// Same algorithm, inputs and outputs as k_factor (element.cu): one CTA per
// element, a blocked right-looking partial Cholesky of the augmented Hermitian
// matrix [[G, B_K], [B_K^H, 0]] (lower triangle, column-major) in panels of 32
// columns, n_v positive pivots, a sign flip of the trailing block, n_u further
// pivots.  The diagonal block (unblocked Cholesky) and the panel triangular
// solve run in FP64 exactly as in k_factor.  The trailing update
//     A[i][j] -= sum_k P[i][k] conj(P[j][k])      (i >= j >= k1)
// which is ~95 % of the arithmetic, runs on tcgen05 FP16 MMAs with FP32
// accumulation through an error-free splitting of the panel into small
// integers (the splitting idea of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 2012), with fixed 8-bit digits:
//
//  * every panel row i gets a power of two 2^e_i > max_k |P[i][k]| (real and
//    imaginary parts together) and is written as integers
//    X[i][k] = round(P[i][k] 2^(55 - e_i)), |X| <= 2^55, split into 7 balanced
//    base-256 digits q_0..q_6 in [-128, 128]:
//        P[i][k] = 2^e_i sum_t q_t[i][k] 2^(-7 - 8 t)  + O(2^(e_i - 56));
//  * digits are exact in FP16, their products exact in FP32, and the products
//    of one level s = a + b (digit pairs (a, b)) summed over K <= 64 stay
//    below 2^24 in magnitude (at most 7 pairs x 64 terms x 2^14), so each
//    level's FP32 accumulator in tensor memory holds an exact integer V_s;
//  * levels s = 0..6 are kept (28 digit pairs); the epilogue combines them in
//    64-bit integers, T = sum_s V_s 2^(8 (5 - s)) (the last level shifted
//    right; |T| < 2^61), rounds T 2^(e_i + e_j - 54) once to FP64 and
//    subtracts it from the trailing matrix with one FP64 operation.
//
// The error of one update is about 2^-57 2^e_i 2^e_j K (rounding of the
// digits, the dropped levels s >= 7 and the last level's shift), below the
// FP64 dot product's own rounding bound.  Complex panels (K = 64 reals per
// row: real parts, then imaginary parts) give the real part of P P^H from
// [Re P, Im P] [Re P, Im P]^T and the imaginary part from
// [Im P, -Re P] [Re P, Im P]^T, the minus sign by the MMA's negate-A bit.
//
// Data flow per panel: the thread that solves a panel row also writes its
// digits (FP16, in the K-major core-matrix layout of the MMA operands) to a
// per-element scratch area; the trailing lower triangle is then covered by
// 128-row x NJ-column tiles (NJ = 32 real, 16 complex): the 128-row operand is
// copied from the scratch into shared memory once per row block, the NJ-row
// operand per tile (or taken from the row block on diagonal tiles), one thread
// issues the 28 (x 2 or x 8) MMAs into 7 (x 2) accumulators of tensor memory
// (224 columns per tile, two tiles in flight), and all threads run the
// epilogue, which overlaps the next tile's MMAs.  Every wait on the MMAs is
// bounded in time; on a timeout the CTA records it and returns.
#include <cuda_fp16.h>

#include <cstdint>

#include "dpg_internal.h"

namespace dpg {

namespace {

constexpr int TB = 32;          // panel width
constexpr int TM = 128;         // rows of a trailing tile (MMA M)
constexpr int NSL = 7;          // digits per value
constexpr int NLEV = 7;         // digit levels kept (a + b < NLEV)
constexpr int FT_THREADS = 256;
constexpr uint32_t FT_TMEM_COLS = 512;
constexpr unsigned long long FT_WAIT_NS = 100000000ull;  // a wait on the MMAs gives up after 100 ms

template <typename T> struct TcCfg;
template <> struct TcCfg<double> {
  static constexpr int K = 32;      // reals per panel row
  static constexpr int NJ = 32;     // tile columns
  static constexpr int PARTS = 1;   // accumulator sets (real)
  static_assert(NSL * (K / 8) * NJ <= 4 * FT_THREADS, "one J-operand copy is at most four per thread");
};
template <> struct TcCfg<double2> {
  static constexpr int K = 64;      // real parts, then imaginary parts
  static constexpr int NJ = 16;
  static constexpr int PARTS = 2;   // real and imaginary part of P P^H
};
// tensor-memory columns of one tile's accumulators: 7 levels x NJ x parts = 224
constexpr int BUFC = 224;

__device__ __forceinline__ uint32_t ft_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long ft_global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor, K-major without swizzle: start address,
// leading (K-adjacent core matrices) and stride (M/N-adjacent core matrices)
// byte offsets in 16-byte units, the fixed version bits 46..48 = 0b001.
__device__ __forceinline__ uint64_t ft_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D F32 (bits 4-5 = 1), A and B F16
// (bits 7-9, 10-12 = 0), negate A (bit 13), both K-major, N >> 3 at bits
// 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t ft_idesc(int M, int N, bool neg_a) {
  return (1u << 4) | (neg_a ? (1u << 13) : 0u) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void ft_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool ft_mbar_wait(uint32_t mbar, uint32_t parity) {
  const unsigned long long t0 = ft_global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (done) return true;
    if (ft_global_ns() - t0 > FT_WAIT_NS) return false;
  }
}

__device__ __forceinline__ void ft_tmem_ld16(uint32_t taddr, uint32_t v[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

// Scalar operations of the FP64 parts (diagonal block, panel solve).
template <typename T> struct Fs;
template <> struct Fs<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double re(double a) { return a; }
  __device__ static double real(double r) { return r; }
  __device__ static double neg(double a) { return -a; }
  __device__ static double sub(double a, double b) { return a - b; }
  __device__ static double scale(double a, double s) { return a * s; }
  __device__ static double mul_conj(double a, double b) { return a * b; }
  __device__ static double amax(double a) { return fabs(a); }
};
template <> struct Fs<double2> {
  __device__ static double2 zero() { return make_double2(0.0, 0.0); }
  __device__ static double re(double2 a) { return a.x; }
  __device__ static double2 real(double r) { return make_double2(r, 0.0); }
  __device__ static double2 neg(double2 a) { return make_double2(-a.x, -a.y); }
  __device__ static double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
  __device__ static double2 scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
  __device__ static double2 mul_conj(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
  }
  __device__ static double amax(double2 a) { return fmax(fabs(a.x), fabs(a.y)); }
};

// v 2^(55 - e) rounded to an integer (half away from zero) for |v| < 2^e,
// from the bits of v (no FP64 arithmetic).
__device__ __forceinline__ long long fixed55(double v, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7ff);
  if (be == 0) return 0;  // zero (and subnormals, below every row scale used here)
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const int sh = be - 1020 - e;  // v = mant 2^(be - 1075); times 2^(55 - e)
  unsigned long long mag = 0;
  if (sh >= 0)
    mag = mant << sh;  // sh <= 2 because |v| < 2^e
  else if (sh > -64)
    mag = ((mant >> (-sh - 1)) + 1) >> 1;
  return (b >> 63) ? -(long long)mag : (long long)mag;
}

// Exponent e with max < 2^e (0 for max = 0).
__device__ __forceinline__ int row_exponent(double m) {
  if (!(m > 0.0)) return 0;
  const int be = (int)(((unsigned long long)__double_as_longlong(m) >> 52) & 0x7ff);
  return be == 0 ? -1022 : be - 1022;
}

// Seven balanced base-256 digits of X (|X| < 2^55), most significant first.
__device__ __forceinline__ void digits7(long long X, int d[NSL]) {
#pragma unroll
  for (int t = NSL - 1; t >= 1; --t) {
    int lo = (int)(X & 0xff);
    lo -= (lo & 0x80) << 1;  // to [-128, 127]
    d[t] = lo;
    X = (X - lo) >> 8;
  }
  d[0] = (int)X;  // |d_0| <= 128
}

__device__ __forceinline__ uint32_t pack_half2(int a, int b) {
  // small integers to FP32 exactly (magic-number addition), then one packed conversion
  const float fa = __int_as_float(0x4B400000 + a) - 12582912.0f;
  const float fb = __int_as_float(0x4B400000 + b) - 12582912.0f;
  const __half2 h = __floats2half2_rn(fa, fb);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Digits of 8 consecutive values (one 16-byte K chunk) into the scratch:
// slice t, chunk kc, row rho at ((t KC + kc) RP + rho) 16 bytes.
__device__ __forceinline__ void write_chunk(uint8_t* Q, int KC, int RP, int kc, int rho, const double v[8], int e) {
  int d[8][NSL];
#pragma unroll
  for (int j = 0; j < 8; ++j) digits7(fixed55(v[j], e), d[j]);
#pragma unroll
  for (int t = 0; t < NSL; ++t) {
    uint4 u;
    u.x = pack_half2(d[0][t], d[1][t]);
    u.y = pack_half2(d[2][t], d[3][t]);
    u.z = pack_half2(d[4][t], d[5][t]);
    u.w = pack_half2(d[6][t], d[7][t]);
    *reinterpret_cast<uint4*>(Q + ((size_t)(t * KC + kc) * RP + rho) * 16) = u;
  }
}

// v 2^E rounded to the nearest FP64 (ties away from zero), from the integer's
// bits; no FP64 arithmetic except where the exponent leaves the normal range.
__device__ __forceinline__ double scaled_i64(long long v, int E) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long m = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll((long long)m);
  m <<= lz;  // leading one at bit 63
  int ex = E + 63 - lz;
  unsigned long long r = m + 0x400ull;  // round at bit 11
  if (r < m) {                          // carried out of bit 63
    r = 0x8000000000000000ull;
    ++ex;
  }
  if (ex < -1022 || ex > 1023) return ldexp((double)v, E);
  const unsigned long long bits = sgn | ((unsigned long long)(ex + 1023) << 52) | ((r >> 11) & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// Accumulate one level of 16 FP32 exact integers into 64-bit sums.
template <bool MAGIC>
__device__ __forceinline__ void acc_level(const uint32_t v[16], int s, long long acc[16]) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    int x;
    if (MAGIC)  // |V| < 2^22: integer bits by adding 1.5 * 2^23
      x = __float_as_int(__uint_as_float(v[j]) + 12582912.0f) - 0x4B400000;
    else
      x = __float2int_rn(__uint_as_float(v[j]));
    if (s <= 5)
      acc[j] += (long long)x << (8 * (5 - s));
    else
      acc[j] += (long long)(x >> 8);
  }
}

}  // namespace

// The factorisation of one element's augmented matrix A (N x N,
// column-major, lower triangle used) by the calling CTA.  The caller owns the
// tensor memory (tmem, 512 columns) and the MMA completion barrier; `phase`
// carries the barrier's parity from call to call.  Returns FT_DONE unless a
// wait on the MMAs gave up, with FT_BAD added on a non-positive pivot.
constexpr int FT_DONE = 1, FT_BAD = 2;
template <typename T>
__device__ __forceinline__ int ft_factor(int N, int nact, int nv, int npiv, T* A, uint8_t* Q, int RP, uint32_t tmem,
                                         uint32_t mbar_a, uint32_t& phase) {
  __shared__ int bad;
  using O = Fs<T>;
  using Cf = TcCfg<T>;
  constexpr int KR = Cf::K, NJ = Cf::NJ, KC = KR / 8;
  constexpr int ISLICE = TM * KR * 2;  // bytes of one digit slice of the row block
  constexpr int JSLICE = NJ * KR * 2;
  constexpr uint32_t LBO_I = TM * 16, LBO_J = NJ * 16;
  extern __shared__ __align__(1024) unsigned char ftsm[];
  unsigned char* sI = ftsm;
  unsigned char* sJ = ftsm + NSL * ISLICE;  // two buffers
  T* sD = reinterpret_cast<T*>(sJ + 2 * NSL * JSLICE);
  int* s_exp = reinterpret_cast<int*>(sD + TB * TB);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) bad = 0;  // first read after the diagonal block's barriers
  bool ok = true;
  for (int k0 = 0; k0 < npiv && ok;) {
    const int stage_end = (k0 < nv) ? nv : npiv;
    const int w = min(TB, stage_end - k0);
    const int k1 = k0 + w;
    if (k0 == nv) {
      // sign flip: the trailing block now holds -A_full; negate it (lower part)
      __syncthreads();
      const size_t R = N - nv;
      for (size_t t = tid; t < R * R; t += blockDim.x) {
        int jj = (int)(t / R), ii = (int)(t - (size_t)jj * R);
        if (ii >= jj) {
          T* p = &A[(size_t)(nv + ii) + (size_t)(nv + jj) * N];
          *p = O::neg(*p);
        }
      }
      __syncthreads();
    }
    // --- diagonal block (FP64): load, factor (unblocked), store
    for (int t = tid; t < w * w; t += blockDim.x) {
      int jj = t / w, ii = t - jj * w;
      sD[ii + jj * TB] = (ii >= jj) ? A[(size_t)(k0 + ii) + (size_t)(k0 + jj) * N] : O::zero();
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
      if (tid == 0) {
        double dv = O::re(sD[j + j * TB]);
        if (!(dv > 0.0)) {
          bad = 1;
          dv = 1e-300;
        }
        sD[j + j * TB] = O::real(sqrt(dv));
      }
      __syncthreads();
      const double ljj = O::re(sD[j + j * TB]);
      for (int ii = j + 1 + tid; ii < w; ii += blockDim.x) sD[ii + j * TB] = O::scale(sD[ii + j * TB], 1.0 / ljj);
      __syncthreads();
      const int rem = w - j - 1;
      for (int t = tid; t < rem * rem; t += blockDim.x) {
        int cc = j + 1 + t / rem, ii = j + 1 + t % rem;
        if (ii >= cc) sD[ii + cc * TB] = O::sub(sD[ii + cc * TB], O::mul_conj(sD[ii + j * TB], sD[cc + j * TB]));
      }
      __syncthreads();
    }
    for (int t = tid; t < w * w; t += blockDim.x) {
      int jj = t / w, ii = t - jj * w;
      if (ii >= jj) A[(size_t)(k0 + ii) + (size_t)(k0 + jj) * N] = sD[ii + jj * TB];
    }
    // --- panel rows [k1, nact) of columns [k0, k1): X L_D^H = P (one row per
    // thread, FP64), then the row's scale and digits; rows up to the next
    // multiple of TM get zero digits
    const int R = nact - k1;
    const int Rp = (R + TM - 1) / TM * TM;
    for (int rho = tid; rho < Rp; rho += blockDim.x) {
      const int row = k1 + rho;
      T x[TB];
#pragma unroll
      for (int j = 0; j < TB; ++j) x[j] = O::zero();
      if (rho < R) {
#pragma unroll
        for (int j = 0; j < TB; ++j)
          if (j < w) x[j] = A[(size_t)row + (size_t)(k0 + j) * N];
#pragma unroll
        for (int j = 0; j < TB; ++j) {
          if (j < w) {
            T v = x[j];
#pragma unroll
            for (int kk = 0; kk < TB; ++kk)
              if (kk < j) v = O::sub(v, O::mul_conj(x[kk], sD[j + kk * TB]));
            x[j] = O::scale(v, 1.0 / O::re(sD[j + j * TB]));
          }
        }
#pragma unroll
        for (int j = 0; j < TB; ++j)
          if (j < w) A[(size_t)row + (size_t)(k0 + j) * N] = x[j];
      }
      double m = 0.0;
#pragma unroll
      for (int j = 0; j < TB; ++j) m = fmax(m, O::amax(x[j]));
      const int e = row_exponent(m);
      s_exp[rho] = e;
#pragma unroll
      for (int kc = 0; kc < TB / 8; ++kc) {
        double v[8];
        if constexpr (sizeof(T) == sizeof(double)) {
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = Fs<double>::re(reinterpret_cast<const double*>(x)[8 * kc + j]);
          write_chunk(Q, KC, RP, kc, rho, v, e);
        } else {
          const double2* xc = reinterpret_cast<const double2*>(x);
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = xc[8 * kc + j].x;
          write_chunk(Q, KC, RP, kc, rho, v, e);
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = xc[8 * kc + j].y;
          write_chunk(Q, KC, RP, kc + TB / 8, rho, v, e);
        }
      }
    }
    __syncthreads();
    // --- trailing update of the lower triangle of rows/cols [k1, nact) on the
    // tensor cores, pipelined over the tiles of a row block: the J operand of
    // tile j + 1 is copied while the MMAs of tile j run, and the epilogue of
    // tile j runs while the MMAs of tile j + 1 run (two accumulator sets in
    // tensor memory, two J buffers; at most one MMA group in flight at a wait)
    for (int rhoI = 0; rhoI < R && ok; rhoI += TM) {
      // row block operand: slice t, chunk kc = 2 KB contiguous in the scratch
      // four independent loads per thread in flight
      for (int q0 = tid; q0 < NSL * KC * TM; q0 += 4 * FT_THREADS) {
        uint4 u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int q = q0 + k * FT_THREADS, r16 = q % TM, tk = q / TM;  // tk = t * KC + kc
          if (q < NSL * KC * TM) u[k] = *reinterpret_cast<const uint4*>(Q + ((size_t)tk * RP + rhoI + r16) * 16);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int q = q0 + k * FT_THREADS, r16 = q % TM, tk = q / TM;
          const int t = tk / KC, kc = tk - t * KC;
          if (q < NSL * KC * TM) *reinterpret_cast<uint4*>(sI + t * ISLICE + kc * LBO_I + r16 * 16) = u[k];
        }
      }
      const int nJ = (min(rhoI + TM, R) + NJ - 1) / NJ;
      auto load_J = [&](int j) {
        const int rhoJ = j * NJ;
        if (rhoJ >= rhoI) return;  // diagonal tiles take B from the row block
        unsigned char* dst = sJ + (j & 1) * (NSL * JSLICE);
        // NSL KC NJ = 896 copies (real and complex): up to four per thread
        uint4 u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int q = tid + k * FT_THREADS, r16 = q % NJ, tk = q / NJ;
          if (q < NSL * KC * NJ) u[k] = *reinterpret_cast<const uint4*>(Q + ((size_t)tk * RP + rhoJ + r16) * 16);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int q = tid + k * FT_THREADS, r16 = q % NJ, tk = q / NJ;
          const int t = tk / KC, kc = tk - t * KC;
          if (q < NSL * KC * NJ) *reinterpret_cast<uint4*>(dst + t * JSLICE + kc * LBO_J + r16 * 16) = u[k];
        }
      };
      auto issue = [&](int j) {  // one thread: all digit-pair MMAs of tile j, then one commit
        const int rhoJ = j * NJ;
        const bool diag = rhoJ >= rhoI;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t aI = ft_smem_u32(sI);
        const uint32_t bJ = diag ? aI + (uint32_t)((rhoJ - rhoI) * 16) : ft_smem_u32(sJ + (j & 1) * (NSL * JSLICE));
        const uint32_t bslice = diag ? ISLICE : JSLICE, lbo_b = diag ? LBO_I : LBO_J;
        const uint32_t id_pos = ft_idesc(TM, NJ, false), id_neg = ft_idesc(TM, NJ, true);
        const uint32_t buf = tmem + (uint32_t)((j & 1) * BUFC);
#pragma unroll 1
        for (int sl = 0; sl < NLEV; ++sl) {
          const uint32_t dre = buf + (uint32_t)(sl * NJ);
          const uint32_t dim = buf + (uint32_t)((NLEV + sl) * NJ);
          uint32_t first_re = 0, first_im = 0;
#pragma unroll 1
          for (int a = 0; a <= sl; ++a) {
            const int b = sl - a;
            const uint32_t abase = aI + (uint32_t)(a * ISLICE), bbase = bJ + (uint32_t)(b * bslice);
            // real part: all K steps of 16 (two 16-byte chunks each)
#pragma unroll
            for (int kk = 0; kk < KC / 2; ++kk) {
              ft_mma(dre, ft_desc(abase + kk * 2 * LBO_I, LBO_I, 128), ft_desc(bbase + kk * 2 * lbo_b, lbo_b, 128),
                     id_pos, first_re);
              first_re = 1;
            }
            if (Cf::PARTS == 2) {
              // imaginary part: Im P_I (Re P_J)^T - Re P_I (Im P_J)^T
#pragma unroll
              for (int kk = 0; kk < KC / 4; ++kk) {
                ft_mma(dim, ft_desc(abase + (kk + KC / 4) * 2 * LBO_I, LBO_I, 128),
                       ft_desc(bbase + kk * 2 * lbo_b, lbo_b, 128), id_pos, first_im);
                first_im = 1;
                ft_mma(dim, ft_desc(abase + kk * 2 * LBO_I, LBO_I, 128),
                       ft_desc(bbase + (kk + KC / 4) * 2 * lbo_b, lbo_b, 128), id_neg, 1u);
              }
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a));
      };
      // epilogue of tile j: warp w reads accumulator lanes 32 (w % 4) .. + 31
      // (tile rows) and 16 columns: real, column half w / 4; complex, all 16
      // columns of the real (w < 4) or imaginary (w >= 4) part
      auto epilogue = [&](int j) {
        const int rhoJ = j * NJ;
        const int qd = warp & 3, hsel = warp >> 2;
        const int rho = rhoI + 32 * qd + lane;
        const int row = k1 + rho;
        const int cbase = (Cf::PARTS == 2) ? 0 : hsel * 16;
        const uint32_t base = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)((j & 1) * BUFC) +
                              ((Cf::PARTS == 2) ? (uint32_t)(hsel * NLEV * NJ) : 0u) + (uint32_t)cbase;
        long long acc[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) acc[jj] = 0;
#pragma unroll
        for (int sl = 0; sl < NLEV; ++sl) {
          uint32_t v[16];
          ft_tmem_ld16(base + (uint32_t)(sl * NJ), v);
          acc_level<Cf::PARTS == 1>(v, sl, acc);
        }
        if (rho < R) {
          // all 16 loads of the trailing entries first, then the updates (the
          // entries are distinct, so the loads need not wait on the stores)
          const int er = s_exp[rho];
          double* p0 = reinterpret_cast<double*>(&A[(size_t)row + (size_t)(k1 + rhoJ + cbase) * N]) +
                       ((Cf::PARTS == 2) ? hsel : 0);
          constexpr size_t cstride = (size_t)(sizeof(T) / sizeof(double));
          double cv[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj)
            if (rhoJ + cbase + jj <= rho) cv[jj] = p0[(size_t)jj * N * cstride];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int cr = rhoJ + cbase + jj;  // column, relative to k1
            if (cr <= rho) p0[(size_t)jj * N * cstride] = cv[jj] - scaled_i64(acc[jj], er + s_exp[cr] - 54);
          }
        }
      };
      load_J(0);
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      if (tid == 0) issue(0);
      for (int j = 0; j < nJ; ++j) {
        if (j + 1 < nJ) load_J(j + 1);  // its buffer was read by the MMAs of tile j - 1 (completed)
        asm volatile("fence.proxy.async.shared::cta;");
        ok = __syncthreads_and(ft_mbar_wait(mbar_a, phase) ? 1 : 0) != 0;  // MMAs of tile j done
        phase ^= 1u;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // the accumulator set of tile j + 1 was drained by the epilogue of tile j - 1
        if (tid == 0 && j + 1 < nJ) issue(j + 1);
        epilogue(j);
        asm volatile("tcgen05.fence::before_thread_sync;");
      }
      __syncthreads();  // the row block operand is reloaded next
    }
    __syncthreads();
    k0 = k1;
  }
  __syncthreads();
  return (ok ? FT_DONE : 0) | (bad ? FT_BAD : 0);
}

// CTA setup of the factorisation kernels: tensor memory and the MMA barrier.
__device__ __forceinline__ uint32_t ft_setup(uint32_t* tmem_slot, uint32_t mbar_a) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ft_smem_u32(tmem_slot)),
                 "r"(FT_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  return *tmem_slot;
}

// CTA teardown: after a failed wait, one more bounded wait for the MMAs in
// flight; tensor memory is released only when nothing can still write it.
__device__ __forceinline__ void ft_finish(bool ok, uint32_t tmem, uint32_t mbar_a, uint32_t phase, int* tc_err) {
  bool drained = true;
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(tc_err, 1);
    drained = __syncthreads_and(ft_mbar_wait(mbar_a, phase ^ 1u) ? 1 : 0) != 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0 && drained) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FT_TMEM_COLS));
  }
}

__device__ __forceinline__ unsigned int ft_smid() {
  unsigned int r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// One CTA per element of a chunk.  stamps (optional): per element the SM, and
// the start and end of its factorisation (global timer, ns).
template <typename T>
__global__ void __launch_bounds__(FT_THREADS, 1)
    k_factor_tc(int N, int nact, int nv, int npiv, const int* __restrict__ ids, T* K, int* status, int* tc_err,
                uint8_t* qscr, long long qstride, int RP, unsigned long long* stamps) {
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ unsigned long long s_t0;
  const int slot = blockIdx.x;
  const uint32_t mbar_a = ft_smem_u32(&mbar);
  const uint32_t tmem = ft_setup(&tmem_slot, mbar_a);
  if (threadIdx.x == 0) s_t0 = ft_global_ns();
  uint32_t phase = 0;
  const int res = ft_factor<T>(N, nact, nv, npiv, K + (size_t)slot * N * N, qscr + (size_t)slot * qstride, RP, tmem,
                               mbar_a, phase);
  const bool ok = (res & FT_DONE) != 0;
  if (threadIdx.x == 0 && stamps) {
    stamps[3 * (size_t)slot] = ft_smid();
    stamps[3 * (size_t)slot + 1] = s_t0;
    stamps[3 * (size_t)slot + 2] = ft_global_ns();
  }
  ft_finish(ok, tmem, mbar_a, phase, tc_err);
  if (threadIdx.x == 0 && (res & FT_BAD)) status[ids[slot]] = 1;
}

// Persistent factorisation of a work list of one arithmetic (real or
// complex) that mixes trial orders: one CTA per SM takes the next item of the
// list (ordered longest first by the host) until the list is exhausted.  Each
// item's matrix sits at its byte offset in the arena; the digit scratch is per
// CTA.  stamps: per item the SM and the start and end times.
template <typename T>
__global__ void __launch_bounds__(FT_THREADS, 1)
    k_factor_tc_queue(const FtItem* __restrict__ items, int nitems, int* counter, unsigned char* arena, int* status,
                      int* tc_err, uint8_t* qscr, long long qstride, unsigned long long* stamps) {
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_item;
  __shared__ unsigned long long s_t0;
  const uint32_t mbar_a = ft_smem_u32(&mbar);
  const uint32_t tmem = ft_setup(&tmem_slot, mbar_a);
  uint8_t* Q = qscr + (size_t)blockIdx.x * qstride;
  uint32_t phase = 0;
  bool ok = true;
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int w = s_item;
    __syncthreads();  // every thread has its item before the next one is fetched
    if (w >= nitems) break;
    const FtItem it = items[w];
    if (threadIdx.x == 0) s_t0 = ft_global_ns();
    const int res = ft_factor<T>(it.N, it.nact, it.nv, it.npiv, reinterpret_cast<T*>(arena + it.koff), Q,
                                 (it.N + TM - 1) / TM * TM, tmem, mbar_a, phase);
    ok = (res & FT_DONE) != 0;
    if (threadIdx.x == 0) {
      if (res & FT_BAD) status[it.elem] = 1;
      if (stamps) {
        stamps[3 * (size_t)w] = ft_smid();
        stamps[3 * (size_t)w + 1] = s_t0;
        stamps[3 * (size_t)w + 2] = ft_global_ns();
      }
    }
    __syncthreads();
    if (!ok) break;
  }
  ft_finish(ok, tmem, mbar_a, phase, tc_err);
}

// Rows of the digit scratch for an augmented size N (multiple of TM).
static int ft_rows(int N) { return (N + TM - 1) / TM * TM; }

size_t factor_tc_scratch_bytes(int N, bool cplx) {
  const int KR = cplx ? TcCfg<double2>::K : TcCfg<double>::K;
  return (size_t)NSL * (KR / 8) * ft_rows(N) * 16;
}

static size_t ft_smem(bool cplx) {
  if (cplx)
    return (size_t)NSL * TM * TcCfg<double2>::K * 2 + 2 * (size_t)NSL * TcCfg<double2>::NJ * TcCfg<double2>::K * 2 +
           sizeof(double2) * TB * TB;
  return (size_t)NSL * TM * TcCfg<double>::K * 2 + 2 * (size_t)NSL * TcCfg<double>::NJ * TcCfg<double>::K * 2 +
         sizeof(double) * TB * TB;
}

// the row-exponent array rides after the fixed part; 3328 rows covers N <= 3315 (p = 4)
constexpr int FT_MAX_RP = 3328;

int factor_tc_init() {
  constexpr size_t exp_bytes = sizeof(int) * FT_MAX_RP;
  if (cudaFuncSetAttribute(k_factor_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(ft_smem(false) + exp_bytes)) != cudaSuccess ||
      cudaFuncSetAttribute(k_factor_tc<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(ft_smem(true) + exp_bytes)) != cudaSuccess ||
      cudaFuncSetAttribute(k_factor_tc_queue<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(ft_smem(false) + exp_bytes)) != cudaSuccess ||
      cudaFuncSetAttribute(k_factor_tc_queue<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(ft_smem(true) + exp_bytes)) != cudaSuccess)
    return DPG_ERR_CUDA;
  return DPG_OK;
}

int factor_tc_launch(bool cplx, int count, int N, int nact, int nv, int npiv, const int* ids, void* K, int* status,
                     int* tc_err, uint8_t* qscr, cudaStream_t s, unsigned long long* stamps) {
  const int RP = ft_rows(N);
  if (RP > FT_MAX_RP) return DPG_ERR_UNSUPPORTED;
  const size_t smem = ft_smem(cplx) + sizeof(int) * (size_t)RP;
  const long long qstride = (long long)factor_tc_scratch_bytes(N, cplx);
  if (cplx)
    k_factor_tc<double2><<<count, FT_THREADS, smem, s>>>(N, nact, nv, npiv, ids, static_cast<double2*>(K), status,
                                                         tc_err, qscr, qstride, RP, stamps);
  else
    k_factor_tc<double><<<count, FT_THREADS, smem, s>>>(N, nact, nv, npiv, ids, static_cast<double*>(K), status,
                                                        tc_err, qscr, qstride, RP, stamps);
  return cudaGetLastError() == cudaSuccess ? DPG_OK : DPG_ERR_CUDA;
}

// Digit scratch of one persistent CTA (the largest item it can meet).
size_t factor_tc_queue_scratch_bytes(int Nmax) { return factor_tc_scratch_bytes(Nmax, true); }

int factor_tc_queue_launch(bool cplx, const FtItem* items, int nitems, int Nmax, int* counter, void* arena,
                           int* status, int* tc_err, uint8_t* qscr, unsigned long long* stamps, int grid,
                           cudaStream_t s) {
  if (nitems <= 0) return DPG_OK;
  if (ft_rows(Nmax) > FT_MAX_RP) return DPG_ERR_UNSUPPORTED;
  const size_t smem = ft_smem(cplx) + sizeof(int) * (size_t)ft_rows(Nmax);
  const long long qstride = (long long)factor_tc_queue_scratch_bytes(Nmax);
  if (cudaMemsetAsync(counter, 0, sizeof(int), s) != cudaSuccess) return DPG_ERR_CUDA;
  const int g = grid < nitems ? grid : nitems;
  unsigned char* ar = static_cast<unsigned char*>(arena);
  if (cplx)
    k_factor_tc_queue<double2><<<g, FT_THREADS, smem, s>>>(items, nitems, counter, ar, status, tc_err, qscr, qstride,
                                                           stamps);
  else
    k_factor_tc_queue<double><<<g, FT_THREADS, smem, s>>>(items, nitems, counter, ar, status, tc_err, qscr, qstride,
                                                          stamps);
  return cudaGetLastError() == cudaSuccess ? DPG_OK : DPG_ERR_CUDA;
}

}  // namespace dpg
