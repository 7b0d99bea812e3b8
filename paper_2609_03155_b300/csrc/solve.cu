// Assembly (DistributeLocalToGlobal of Algorithm 2), conjugate gradients on the
// condensed trace system (Sec. 2.3 end), and local recovery with the residual
// estimator (Sec. 2.3).  complex FP64 unless stated.
#include <cmath>
#include <cstring>
#include <mutex>

#include "dpg_internal.h"

namespace dpg {

__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ------------------------------------------------------------ assembly --
// Position of column gj in row gi (entity column lists are sorted), or -1.
__device__ __forceinline__ int64_t csr_pos(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ row2blk,
                                           const int4* __restrict__ blk, const int64_t* __restrict__ colptr,
                                           const int32_t* __restrict__ cols, int gi, int gj) {
  const int b = row2blk[gi];
  const int W = blk[b].z;
  const int32_t* c = cols + colptr[b];
  int lo = 0, hi = W - 1;
  if (W <= 0) return -1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (c[mid] < gj)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (c[lo] == gj) ? rowptr[gi] + lo : -1;
}

// One block per element of one colour: elements of a colour share no
// unknowns, so the plain read-modify-write below has no race and the sum
// order per entry is the fixed colour order.
// off: the element's trace-map offsets; soff: its store offsets (the same
// table, or the slot-based one of the streaming mode).
__global__ void __launch_bounds__(256) k_assemble(int nh, const int* __restrict__ elems, const ElemOff* __restrict__ off,
                                                  const ElemOff* __restrict__ soff,
                                                  const int32_t* __restrict__ l2g, const double2* __restrict__ xfix,
                                                  const double2* __restrict__ Sst, const double2* __restrict__ sst,
                                                  const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ row2blk, const int4* __restrict__ blk,
                                                  const int64_t* __restrict__ colptr, const int32_t* __restrict__ cols,
                                                  double2* val, double2* b) {
  const int e = elems[blockIdx.x];
  const ElemOff of = off[e];
  const int32_t* g = l2g + of.h;
  const double2* Se = Sst + soff[e].S;
  sst += soff[e].h;
  xfix += of.h;
  for (int t = threadIdx.x; t < nh * nh; t += blockDim.x) {
    const int i = t / nh, j = t - i * nh;
    const int gi = g[i], gj = g[j];
    if (gi < 0 || gj < 0) continue;
    const int64_t pos = csr_pos(rowptr, row2blk, blk, colptr, cols, gi, gj);
    if (pos >= 0) val[pos] = c_add(val[pos], Se[t]);
  }
  for (int i = threadIdx.x; i < nh; i += blockDim.x) {
    const int gi = g[i];
    if (gi < 0) continue;
    double2 acc = sst[i];
    for (int j = 0; j < nh; ++j)
      if (g[j] == -1) {  // Dirichlet lifting: b -= S_{i,fixed} x_D
        double2 pr = c_mul(Se[(size_t)i * nh + j], xfix[j]);
        acc.x -= pr.x;
        acc.y -= pr.y;
      }
    b[gi] = c_add(b[gi], acc);
  }
}

// Assembly of one colour-homogeneous chunk as it is condensed (streaming mode).
int assemble_chunk(dpg_handle* h, int g, const int* ids, int count, cudaStream_t s) {
  k_assemble<<<count, 256, 0, s>>>(h->grp[g].sz.n_h, ids, h->d_off, h->d_soff, h->d_l2g, h->d_xfix, h->d_S, h->d_s,
                                   h->d_rowptr, h->d_row2blk, h->d_blk, h->d_blk_colptr, h->d_cols, h->d_val, h->d_b);
  h->launches += 1;
  DPG_CUDA_TRY(h, cudaGetLastError());
  return DPG_OK;
}

void system_changed(dpg_handle* h) {
  h->have_system = true;
  h->have_val32 = false;
  h->have_val32h = false;
  h->have_ebe = false;
  h->have_valdw = false;
  h->have_binvdw = false;
  h->have_dinv = false;
  h->have_binv = false;
}

int assemble_system(dpg_handle* h, cudaStream_t s) {
  if (h->stream) return DPG_OK;  // assembled by the element pass
  DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_val, 0, sizeof(double2) * h->nnz, s));
  DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_b, 0, sizeof(double2) * h->n, s));
  // colour by colour; within a colour one launch per order group (the
  // elements of one colour share no unknowns, whatever their group)
  for (int c = 0; c < h->ncolor; ++c)
    for (const Group& G : h->grp) {
      const int cnt = G.color_off[c + 1] - G.color_off[c];
      if (cnt == 0) continue;
      k_assemble<<<cnt, 256, 0, s>>>(G.sz.n_h, G.d_color_elems + G.color_off[c], h->d_off, h->d_off, h->d_l2g,
                                     h->d_xfix,
                                     h->d_S, h->d_s, h->d_rowptr, h->d_row2blk, h->d_blk, h->d_blk_colptr, h->d_cols,
                                     h->d_val, h->d_b);
      h->launches += 1;
    }
  DPG_CUDA_TRY(h, cudaGetLastError());
  system_changed(h);
  return DPG_OK;
}

// ------------------------------------------------------------------ CG --
// Conjugate gradients on the Hermitian positive definite trace system
// (Sec. 2.3 end), optionally preconditioned by the diagonal (Jacobi) or by
// the inverses of the entity diagonal blocks (each mesh entity's E-hat and
// H-hat unknowns together).  One persistent cooperative kernel runs a whole
// (inner) solve: three bounded grid barriers per iteration, every reduction
// summed in a fixed order by every block (deterministic, identical scalars).
struct SysView {
  int64_t n;
  int nblk;
  const int64_t* rowptr;
  const int32_t* row2blk;
  const int4* blk;
  const int64_t* colptr;
  const int32_t* cols;
  const int64_t* binv_ptr;
  int dmax;  // rows of the largest entity block
  // Hermitian half storage (FP32 inner solves)
  const int64_t* rowptr_h;
  const int64_t* toff;
  const int64_t* rev_ptr;
  const int64_t* rev_off;
  // element-by-element operator (FP32 inner solves): per element the upper
  // triangle of 32 x 32 tiles of S_K, its slots (trace map) and, per row, the
  // slots that carry it
  int ne;
  int ebe_nbmax;              // 32-row blocks of the largest element
  const float2* ebe;          // tiles, element by element
  const int64_t* ebe_toff;    // per element: first tile entry (ne + 1)
  const int64_t* ebe_hoff;    // per element: first slot (ne + 1)
  const int32_t* l2g;         // per slot: global row (negative: fixed)
  const int64_t* ebe_rptr;    // per row: first entry of its slot list (n + 1)
  const int32_t* ebe_ridx;    // slot lists, ascending
  float2* ebe_ys;             // per slot: the element product
  int ebe_stages;             // staging buffers per warp of the bulk-copy variant
};

struct CgState {          // device-resident
  double tol2;            // in: stop when ||r||^2 <= tol2
  int max_iter;           // in
  int status;             // out: 0 ok, 1 a barrier timed out
  int iters;              // out
  double rr, rz;          // out
  unsigned int bar[2];    // grid barrier counter / generation
  unsigned long long wait_ns;  // in: a barrier wait gives up after this long
  int hold;               // in: test hook, no barrier ever releases (every wait runs out)
  int cont;               // in: continue the previous solve's direction p (reliable update)
  double rz_prev;         // in: r^H z at the end of the previous solve (cont)
};

constexpr int CG_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded grid-wide barrier for a cooperative launch.  Returns false when a
// wait gave up (state->status set); callers then leave the kernel.  The wait
// is bounded in time (st->wait_ns on the global nanosecond timer), not in
// polls.  Every block arrives at every barrier once, so after a timeout the
// last arriving block still resets the counter and all blocks leave.
__device__ __forceinline__ bool grid_barrier(CgState* st, unsigned int& gen) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int target = gen + 1;
    __threadfence();
    const unsigned int arrived = atomicAdd(&st->bar[0], 1u) + 1u;
    if (arrived == gridDim.x && !st->hold) {
      st->bar[0] = 0u;
      __threadfence();
      atomicExch(&st->bar[1], target);
    } else {
      const unsigned long long t0 = global_ns(), limit = st->wait_ns;
      while (*((volatile unsigned int*)&st->bar[1]) != target) {
        if (global_ns() - t0 > limit) {  // something is broken: give up
          atomicExch(&st->status, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  ++gen;
  return *((volatile int*)&st->status) == 0;
}

// Block-level sum of (a, b) into red[slot*G + block] pairs, then every block
// sums all partials in index order.  All threads get the totals.
template <typename R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-lane partials are in the solve precision R (FP32 for the inner solves of
// iterative refinement, whose tolerance is ~1e-3); each warp's total is widened
// to FP64 once, and block / grid sums are FP64 in a fixed order.
template <typename R>
__device__ __forceinline__ void block_partial(R a_r, R b_r, double* red_a, double* red_b) {
  __shared__ double sw[2][CG_THREADS / 32];
  const double a = (double)warp_sum_r(a_r);
  const double b = (double)warp_sum_r(b_r);
  if ((threadIdx.x & 31) == 0) {
    sw[0][threadIdx.x >> 5] = a;
    sw[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0, tb = 0;
    for (int k = 0; k < CG_THREADS / 32; ++k) {
      ta += sw[0][k];
      tb += sw[1][k];
    }
    red_a[blockIdx.x] = ta;
    if (red_b) red_b[blockIdx.x] = tb;
  }
}

// One warp of each block sums the per-block partials (FP64, fixed order: lane
// strides then the shuffle tree), so every block obtains identical totals
// while the FP64 pipe (2 DFMA/clk/SM on B300) sees one warp's work, not eight.
__device__ __forceinline__ void grid_total(const double* red_a, const double* red_b, double& ta, double& tb) {
  __shared__ double sw[2];
  if (threadIdx.x < 32) {
    double a = 0, b = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += 32) {
      a += ((volatile const double*)red_a)[k];
      if (red_b) b += ((volatile const double*)red_b)[k];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) {
      sw[0] = a;
      sw[1] = b;
    }
  }
  __syncthreads();
  ta = sw[0];
  tb = sw[1];
  __syncthreads();
}

template <typename V> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };
__device__ __forceinline__ double2 mkv(double a, double b, double2*) { return make_double2(a, b); }
__device__ __forceinline__ float2 mkv(double a, double b, float2*) { return make_float2((float)a, (float)b); }
__device__ __forceinline__ float2 mkv(float a, float b, float2*) { return make_float2(a, b); }

// y_row = (A x)_row by one warp; the row's columns are its entity's list.
// Products and the row sum in the matrix precision Mv.
template <typename V, typename Mv>
__device__ __forceinline__ V row_spmv(const SysView& S, int64_t row, const Mv* __restrict__ val, const V* __restrict__ x) {
  using R = typename RealOf<Mv>::T;
  const int lane = threadIdx.x & 31;
  const int b = S.row2blk[row];
  const int W = S.blk[b].z;
  const int32_t* c = S.cols + S.colptr[b];
  const Mv* v = val + S.rowptr[row];
  R ar = 0, ai = 0;
  int k = lane;
  // four independent column chains in flight per lane
  for (; k + 96 < W; k += 128) {
    const int c0 = c[k], c1 = c[k + 32], c2 = c[k + 64], c3 = c[k + 96];
    const Mv a0 = v[k], a1 = v[k + 32], a2 = v[k + 64], a3 = v[k + 96];
    const V x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
    ar = fma(a0.x, (R)x0.x, fma(-a0.y, (R)x0.y, ar));
    ai = fma(a0.x, (R)x0.y, fma(a0.y, (R)x0.x, ai));
    ar = fma(a1.x, (R)x1.x, fma(-a1.y, (R)x1.y, ar));
    ai = fma(a1.x, (R)x1.y, fma(a1.y, (R)x1.x, ai));
    ar = fma(a2.x, (R)x2.x, fma(-a2.y, (R)x2.y, ar));
    ai = fma(a2.x, (R)x2.y, fma(a2.y, (R)x2.x, ai));
    ar = fma(a3.x, (R)x3.x, fma(-a3.y, (R)x3.y, ar));
    ai = fma(a3.x, (R)x3.y, fma(a3.y, (R)x3.x, ai));
  }
  for (; k < W; k += 32) {
    const Mv a = v[k];
    const V xv = x[c[k]];
    ar = fma(a.x, (R)xv.x, fma(-a.y, (R)xv.y, ar));
    ai = fma(a.x, (R)xv.y, fma(a.y, (R)xv.x, ai));
  }
  R yr = ar, yi = ai;
  // warp sum in the matrix precision
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    yr += __shfl_xor_sync(0xffffffffu, yr, o);
    yi += __shfl_xor_sync(0xffffffffu, yi, o);
  }
  return mkv(yr, yi, (V*)nullptr);
}

// z = M^{-1} r on the rows of block b (precond 0: copy, 1: Jacobi, 2: block
// inverse) by one warp; rs is this warp's shared staging area (>= rows of the
// largest block).  The block inverse is Hermitian, so row j read contiguously
// gives column j: z_i = sum_j conj(Binv[j][i]) r_j with coalesced loads.
// Returns the partial sums ||r||^2 and Re(r^H z) (per lane, FP64).
template <typename V>
__device__ __forceinline__ void block_precond(const SysView& S, int b, int precond, const V* __restrict__ r, V* z,
                                              const typename RealOf<V>::T* __restrict__ dinv,
                                              const V* __restrict__ binv, V* rs, typename RealOf<V>::T& rr,
                                              typename RealOf<V>::T& rz) {
  using R = typename RealOf<V>::T;
  const int lane = threadIdx.x & 31;
  const int4 B = S.blk[b];
  if (precond == 2) {
    for (int i = lane; i < B.y; i += 32) rs[i] = r[B.x + i];
    __syncwarp();
    const V* Bi = binv + S.binv_ptr[b];
    for (int i0 = 0; i0 < B.y; i0 += 32) {
      const int i = i0 + lane;
      R zr = 0, zi = 0;
      if (i < B.y) {
        for (int j = 0; j < B.y; ++j) {
          const V a = Bi[(size_t)j * B.y + i];  // conj of Binv[i][j]
          const V rj = rs[j];
          zr = fma(a.x, rj.x, fma(a.y, rj.y, zr));
          zi = fma(a.x, rj.y, fma(-a.y, rj.x, zi));
        }
        const V ri = rs[i];
        const V zv = mkv(zr, zi, (V*)nullptr);
        z[B.x + i] = zv;
        rr += ri.x * ri.x + ri.y * ri.y;
        rz += ri.x * zr + ri.y * zi;
      }
    }
    __syncwarp();
    return;
  }
  for (int i = lane; i < B.y; i += 32) {
    const int64_t row = B.x + i;
    const V ri = r[row];
    V zi = ri;
    if (precond == 1) {
      const R d = dinv[row];
      zi.x = d * ri.x;
      zi.y = d * ri.y;
    }
    z[row] = zi;
    rr += ri.x * ri.x + ri.y * ri.y;
    rz += ri.x * zi.x + ri.y * zi.y;
  }
}

// Half-storage SpMV, first half: block a (one warp): for each of its rows
// y_row = sum over the stored prefix (lower blocks and the diagonal block) of
// A[row][c] x_c, into y; and the conjugate-transpose partial sums of the
// strictly lower part, T[toff[a] + q] = sum_rows conj(A[row][q]) x_row, one
// per prefix position q < n_low(a).  All rows of a block share its column
// list, so each lane gathers its x_c once per window of 32 x HW positions
// (lane owns q = window + lane + 32 k) and every row then streams only its
// values; rows go in pairs so that two reductions are in flight.
constexpr int HW = 4;
template <typename V, typename Mv>
__device__ __forceinline__ void half_block_lower(const SysView& S, int a, const Mv* __restrict__ valh,
                                                 const V* __restrict__ x, V* y, V* T) {
  using R = typename RealOf<Mv>::T;
  const int lane = threadIdx.x & 31;
  const int4 B = S.blk[a];
  const int wl = B.w, Wh = B.w + B.y;
  const int32_t* c = S.cols + S.colptr[a];
  const int64_t* rp = S.rowptr_h + B.x;
  for (int q0 = 0; q0 < Wh; q0 += 32 * HW) {
    R xr[HW], xi[HW], tr[HW], ti[HW];
#pragma unroll
    for (int k = 0; k < HW; ++k) {
      const int q = q0 + lane + 32 * k;
      const V xv = q < Wh ? x[c[q]] : mkv(0.0f, 0.0f, (V*)nullptr);
      xr[k] = (R)xv.x;
      xi[k] = (R)xv.y;
      tr[k] = ti[k] = 0;
    }
    for (int i = 0; i < B.y; i += 2) {
      const bool two = i + 1 < B.y;
      const Mv* v0 = valh + rp[i];
      const Mv* v1 = valh + rp[two ? i + 1 : i];
      const V x0 = x[B.x + i];
      const V x1 = two ? x[B.x + i + 1] : mkv(0.0f, 0.0f, (V*)nullptr);
      R a0r = 0, a0i = 0, a1r = 0, a1i = 0;
#pragma unroll
      for (int k = 0; k < HW; ++k) {
        const int q = q0 + lane + 32 * k;
        if (q < Wh) {
          const Mv u0 = v0[q];
          const Mv u1 = two ? v1[q] : Mv{0, 0};
          a0r = fma(u0.x, xr[k], fma(-u0.y, xi[k], a0r));
          a0i = fma(u0.x, xi[k], fma(u0.y, xr[k], a0i));
          a1r = fma(u1.x, xr[k], fma(-u1.y, xi[k], a1r));
          a1i = fma(u1.x, xi[k], fma(u1.y, xr[k], a1i));
          if (q < wl) {  // conj(A[row][q]) x_row for both rows
            tr[k] = fma(u0.x, (R)x0.x, fma(u0.y, (R)x0.y, tr[k]));
            ti[k] = fma(u0.x, (R)x0.y, fma(-u0.y, (R)x0.x, ti[k]));
            tr[k] = fma(u1.x, (R)x1.x, fma(u1.y, (R)x1.y, tr[k]));
            ti[k] = fma(u1.x, (R)x1.y, fma(-u1.y, (R)x1.x, ti[k]));
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a0r += __shfl_xor_sync(0xffffffffu, a0r, o);
        a0i += __shfl_xor_sync(0xffffffffu, a0i, o);
        a1r += __shfl_xor_sync(0xffffffffu, a1r, o);
        a1i += __shfl_xor_sync(0xffffffffu, a1i, o);
      }
      if (lane < 2 && (lane == 0 || two)) {
        const int64_t row = B.x + i + lane;
        const R ar = lane ? a1r : a0r, ai = lane ? a1i : a0i;
        if (q0 == 0) {
          y[row] = mkv(ar, ai, (V*)nullptr);
        } else {
          V yv = y[row];
          yv.x += ar;
          yv.y += ai;
          y[row] = yv;
        }
      }
    }
    V* Ta = T + S.toff[a];
#pragma unroll
    for (int k = 0; k < HW; ++k) {
      const int q = q0 + lane + 32 * k;
      if (q < wl) Ta[q] = mkv(tr[k], ti[k], (V*)nullptr);
    }
  }
}

// ------------------------------------------------- double-word FP32 arithmetic --
// A double-word (DW) number is an unevaluated sum hi + lo of two FP32 values
// (|lo| <= ulp(hi) / 2), about 48 significant bits.  The DW solver mode keeps
// the matrix, the direction vector p and the block inverses as DW pairs and
// forms every product and sum of the SpMV and the preconditioner with the
// error-free transformations of Dekker (1971) and Knuth: the product of two
// FP32 values is exact as p + fma(a, b, -p); the sum as TwoSum.  Only the
// FP32 pipes do this work (B300 runs FP64 FMA at 1/64 of FP32), while the
// values carry FP64-class accuracy, so CG keeps the convergence of FP64 CG.
__device__ __forceinline__ void dw_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (sh, sl) += (ah + al) (xh + xl), the al xl term dropped (below 2^-46 relative).
__device__ __forceinline__ void dw_mac(float& sh, float& sl, float ah, float al, float xh, float xl) {
  const float pr = ah * xh;
  const float pe = fmaf(ah, xh, -pr);  // exact error of the product
  const float lo = fmaf(ah, xl, fmaf(al, xh, pe));
  float t, e;
  dw_two_sum(sh, pr, t, e);
  sh = t;
  sl += e + lo;
}

__device__ __forceinline__ void dw_warp_sum(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    float t, e;
    dw_two_sum(h, oh, t, e);
    h = t;
    l += e + ol;
  }
}

__device__ __forceinline__ float4 dw_split(double2 v) {
  const float rh = (float)v.x, ih = (float)v.y;
  return make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
}

// y_row = (A p)_row with DW matrix values (re_hi, im_hi, re_lo, im_lo) and the
// DW copy of p; FP64 result.
__device__ __forceinline__ double2 row_spmv_dw(const SysView& S, int64_t row, const float4* __restrict__ val,
                                               const float4* __restrict__ pdw) {
  const int lane = threadIdx.x & 31;
  const int b = S.row2blk[row];
  const int W = S.blk[b].z;
  const int32_t* c = S.cols + S.colptr[b];
  const float4* v = val + S.rowptr[row];
  float rh0 = 0, rl0 = 0, ih0 = 0, il0 = 0, rh1 = 0, rl1 = 0, ih1 = 0, il1 = 0;
  int k = lane;
  for (; k + 96 < W; k += 128) {  // four column chains per lane in flight, two accumulator pairs
    const float4 a0 = v[k], a1 = v[k + 32], a2 = v[k + 64], a3 = v[k + 96];
    const int c0 = c[k], c1 = c[k + 32], c2 = c[k + 64], c3 = c[k + 96];
    const float4 x0 = pdw[c0], x1 = pdw[c1], x2 = pdw[c2], x3 = pdw[c3];
    dw_mac(rh0, rl0, a0.x, a0.z, x0.x, x0.z);
    dw_mac(rh0, rl0, -a0.y, -a0.w, x0.y, x0.w);
    dw_mac(ih0, il0, a0.x, a0.z, x0.y, x0.w);
    dw_mac(ih0, il0, a0.y, a0.w, x0.x, x0.z);
    dw_mac(rh1, rl1, a1.x, a1.z, x1.x, x1.z);
    dw_mac(rh1, rl1, -a1.y, -a1.w, x1.y, x1.w);
    dw_mac(ih1, il1, a1.x, a1.z, x1.y, x1.w);
    dw_mac(ih1, il1, a1.y, a1.w, x1.x, x1.z);
    dw_mac(rh0, rl0, a2.x, a2.z, x2.x, x2.z);
    dw_mac(rh0, rl0, -a2.y, -a2.w, x2.y, x2.w);
    dw_mac(ih0, il0, a2.x, a2.z, x2.y, x2.w);
    dw_mac(ih0, il0, a2.y, a2.w, x2.x, x2.z);
    dw_mac(rh1, rl1, a3.x, a3.z, x3.x, x3.z);
    dw_mac(rh1, rl1, -a3.y, -a3.w, x3.y, x3.w);
    dw_mac(ih1, il1, a3.x, a3.z, x3.y, x3.w);
    dw_mac(ih1, il1, a3.y, a3.w, x3.x, x3.z);
  }
  for (; k < W; k += 32) {
    const float4 a0 = v[k];
    const float4 x0 = pdw[c[k]];
    dw_mac(rh0, rl0, a0.x, a0.z, x0.x, x0.z);
    dw_mac(rh0, rl0, -a0.y, -a0.w, x0.y, x0.w);
    dw_mac(ih0, il0, a0.x, a0.z, x0.y, x0.w);
    dw_mac(ih0, il0, a0.y, a0.w, x0.x, x0.z);
  }
  float t, e;
  dw_two_sum(rh0, rh1, t, e);
  rh0 = t;
  rl0 += e + rl1;
  dw_two_sum(ih0, ih1, t, e);
  ih0 = t;
  il0 += e + il1;
  dw_warp_sum(rh0, rl0);
  dw_warp_sum(ih0, il0);
  return make_double2((double)rh0 + (double)rl0, (double)ih0 + (double)il0);
}

// z = M^{-1} r on the rows of block b with the DW block inverses (conj of
// Binv[i][j] read contiguously as row j); rs: this warp's DW staging of r.
__device__ __forceinline__ void block_precond_dw(const SysView& S, int b, const double2* __restrict__ r, double2* z,
                                                 const float4* __restrict__ binv, float4* rs, double& rr, double& rz) {
  const int lane = threadIdx.x & 31;
  const int4 B = S.blk[b];
  for (int i = lane; i < B.y; i += 32) rs[i] = dw_split(r[B.x + i]);
  __syncwarp();
  const float4* Bi = binv + S.binv_ptr[b];
  for (int i0 = 0; i0 < B.y; i0 += 32) {
    const int i = i0 + lane;
    if (i < B.y) {
      float zrh = 0, zrl = 0, zih = 0, zil = 0;
      for (int j = 0; j < B.y; ++j) {
        const float4 a = Bi[(size_t)j * B.y + i];  // conj of Binv[i][j]
        const float4 rj = rs[j];
        // z += conj(a) r_j: re = a.re r.re + a.im r.im, im = a.re r.im - a.im r.re
        dw_mac(zrh, zrl, a.x, a.z, rj.x, rj.z);
        dw_mac(zrh, zrl, a.y, a.w, rj.y, rj.w);
        dw_mac(zih, zil, a.x, a.z, rj.y, rj.w);
        dw_mac(zih, zil, -a.y, -a.w, rj.x, rj.z);
      }
      const double2 zv = make_double2((double)zrh + (double)zrl, (double)zih + (double)zil);
      const double2 ri = r[B.x + i];
      z[B.x + i] = zv;
      rr += ri.x * ri.x + ri.y * ri.y;
      rz += ri.x * zv.x + ri.y * zv.y;
    }
  }
  __syncwarp();
}

// One whole CG solve of A d = r0 (d = 0 at entry, r holds r0 at entry) in the
// DW mode: FP64 vectors, recurrences and reductions; DW matrix, p copy and
// block inverses (precond 2) or none (precond 0).
__global__ void __launch_bounds__(CG_THREADS, 3) k_cg_dw(SysView S, const float4* __restrict__ val, double2* x,
                                                         double2* r, double2* p, float4* pdw, double2* Ap, double2* z,
                                                         int precond, const float4* __restrict__ binv, double* red,
                                                         CgState* st) {
  extern __shared__ __align__(16) unsigned char cg_smem[];
  float4* rs = reinterpret_cast<float4*>(cg_smem) + (threadIdx.x >> 5) * S.dmax;
  const int G = gridDim.x;
  double* redA = red;
  double* redB0 = red + G;
  double* redB1 = red + 2 * G;
  const int warps = G * (CG_THREADS / 32);
  const int gw = blockIdx.x * (CG_THREADS / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  unsigned int gen = *((volatile unsigned int*)&st->bar[1]);
  const double tol2 = st->tol2;
  const int max_iter = st->max_iter;
  double rr0 = 0, rz0 = 0;
  for (int b = gw; b < S.nblk; b += warps) {
    const int4 B = S.blk[b];
    if (precond == 2) {
      block_precond_dw(S, b, r, z, binv, rs, rr0, rz0);
    } else {
      for (int i = lane; i < B.y; i += 32) {
        const double2 ri = r[B.x + i];
        z[B.x + i] = ri;
        rr0 += ri.x * ri.x + ri.y * ri.y;
        rz0 += ri.x * ri.x + ri.y * ri.y;
      }
    }
    __syncwarp();
    for (int i = lane; i < B.y; i += 32) {
      const double2 zi = z[B.x + i];
      p[B.x + i] = zi;
      pdw[B.x + i] = dw_split(zi);
      x[B.x + i] = make_double2(0.0, 0.0);
    }
  }
  block_partial(rr0, rz0, redB0, redB1);
  if (!grid_barrier(st, gen)) return;
  double rr, rz;
  grid_total(redB0, redB1, rr, rz);
  int it = 0;
  bool done = rr <= tol2;
  while (!done && it < max_iter) {
    double pap = 0;
    for (int64_t row = gw; row < S.n; row += warps) {
      const double2 y = row_spmv_dw(S, row, val, pdw);
      if (lane == 0) {
        Ap[row] = y;
        const double2 pr = p[row];
        pap += pr.x * y.x + pr.y * y.y;
      }
    }
    block_partial(pap, 0.0, redA, nullptr);
    if (!grid_barrier(st, gen)) return;
    double tpap, dummy;
    grid_total(redA, nullptr, tpap, dummy);
    const double alpha = rz / tpap;
    double rr2 = 0, rz2 = 0;
    for (int b = gw; b < S.nblk; b += warps) {
      const int4 B = S.blk[b];
      for (int i = lane; i < B.y; i += 32) {
        const int64_t row = B.x + i;
        double2 xv = x[row], rv = r[row];
        const double2 pv = p[row], av = Ap[row];
        xv.x = fma(alpha, pv.x, xv.x);
        xv.y = fma(alpha, pv.y, xv.y);
        rv.x = fma(-alpha, av.x, rv.x);
        rv.y = fma(-alpha, av.y, rv.y);
        x[row] = xv;
        r[row] = rv;
      }
      __syncwarp();
      if (precond == 2) {
        block_precond_dw(S, b, r, z, binv, rs, rr2, rz2);
      } else {
        for (int i = lane; i < B.y; i += 32) {
          const double2 ri = r[B.x + i];
          z[B.x + i] = ri;
          rr2 += ri.x * ri.x + ri.y * ri.y;
          rz2 += ri.x * ri.x + ri.y * ri.y;
        }
      }
    }
    block_partial(rr2, rz2, redB0, redB1);
    if (!grid_barrier(st, gen)) return;
    double trr, trz;
    grid_total(redB0, redB1, trr, trz);
    const double beta = trz / rz;
    rz = trz;
    rr = trr;
    ++it;
    if (rr <= tol2) break;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)G * blockDim.x) {
      const double2 zv = z[i];
      double2 pv = p[i];
      pv.x = fma(beta, pv.x, zv.x);
      pv.y = fma(beta, pv.y, zv.y);
      p[i] = pv;
      pdw[i] = dw_split(pv);
    }
    if (!grid_barrier(st, gen)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->iters = it;
    st->rr = rr;
    st->rz = rz;
  }
}

__global__ void k_to_dw(int64_t n, const double2* __restrict__ a, float4* b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = dw_split(a[i]);
}

// One whole CG solve of A x = r0 (x = 0 at entry, r holds r0 at entry).
// V: precision of the vectors and recurrences; Mv: precision of the stored
// matrix and of the SpMV products (FP32 values with FP64 recurrences keeps the
// convergence rate of FP64 CG at the bandwidth of an FP32 matrix).
// Element-by-element product y_K = S_K x_K of one element by one warp, FP32.
// The element's S_K (Hermitian, n_h rows) is stored as the upper triangle of
// 32 x 32 tiles (I <= J, row-major, I-major order; diagonal tiles whole, zero
// padding past n_h).  Lane l holds column l of a tile, loaded one row per
// step (coalesced): the column part of an off-diagonal tile,
// y_J[l] += sum_i conj(a_il) x_I[i], stays in the lane; the row part,
// y_I[i] += sum_l a_il x_J[l], is summed across the warp by a transposing
// reduction (5 exchange steps, 31 shuffles per component) that leaves row l's
// sum in lane l.  Every sum has one fixed order.  xs, ya: this warp's shared
// staging of x_K and y_K (nbmax x 32 entries each).  y_K goes to the slots.
// One tile (I, J) of an element's product: t points at its 32 x 32 values
// (global or shared memory), xs at the element's x_K, ya at its y_K.
__device__ __forceinline__ void ebe_tile(const float2* __restrict__ t, int I, int J, const float2* xs, float2* ya) {
  const int lane = threadIdx.x & 31;
  const float2 xj = xs[J * 32 + lane];
  float pr[32], pi[32];
  float cr = 0.0f, ci = 0.0f;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const float2 a = t[i * 32 + lane];
    const float2 xi = xs[I * 32 + i];
    cr = fmaf(a.x, xi.x, fmaf(a.y, xi.y, cr));   // conj(a) x_i
    ci = fmaf(a.x, xi.y, fmaf(-a.y, xi.x, ci));
    pr[i] = fmaf(a.x, xj.x, -a.y * xj.y);         // a x_j
    pi[i] = fmaf(a.x, xj.y, a.y * xj.x);
  }
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) {
    const bool up = (lane & sh) != 0;
#pragma unroll
    for (int k = 0; k < sh; ++k) {
      const float sr = up ? pr[k] : pr[k + sh], si = up ? pi[k] : pi[k + sh];
      const float kr = up ? pr[k + sh] : pr[k], ki = up ? pi[k + sh] : pi[k];
      pr[k] = kr + __shfl_xor_sync(0xffffffffu, sr, sh);
      pi[k] = ki + __shfl_xor_sync(0xffffffffu, si, sh);
    }
  }
  float2 yr = ya[I * 32 + lane];
  yr.x += pr[0];
  yr.y += pi[0];
  ya[I * 32 + lane] = yr;
  if (J > I) {
    float2 yc = ya[J * 32 + lane];
    yc.x += cr;
    yc.y += ci;
    ya[J * 32 + lane] = yc;
  }
}

// x_K of element e into xs (zero past n_h and on fixed unknowns), y_K = 0.
__device__ __forceinline__ int ebe_begin(const SysView& S, int e, const float2* __restrict__ p, float2* xs,
                                         float2* ya, int64_t& h0) {
  const int lane = threadIdx.x & 31;
  h0 = S.ebe_hoff[e];
  const int nh = (int)(S.ebe_hoff[e + 1] - h0);
  const int nb = (nh + 31) >> 5;
  for (int i = lane; i < nb * 32; i += 32) {
    float2 v = make_float2(0.0f, 0.0f);
    if (i < nh) {
      const int g = S.l2g[h0 + i];
      if (g >= 0) v = p[g];
    }
    xs[i] = v;
    ya[i] = make_float2(0.0f, 0.0f);
  }
  __syncwarp();
  return nh;
}

__device__ __forceinline__ void ebe_end(const SysView& S, int64_t h0, int nh, const float2* ya) {
  __syncwarp();
  for (int i = threadIdx.x & 31; i < nh; i += 32) S.ebe_ys[h0 + i] = ya[i];
  __syncwarp();
}

__device__ __forceinline__ void ebe_element(const SysView& S, int e, const float2* __restrict__ p, float2* xs,
                                            float2* ya) {
  int64_t h0;
  const int nh = ebe_begin(S, e, p, xs, ya, h0);
  const int nb = (nh + 31) >> 5;
  const float2* t = S.ebe + S.ebe_toff[e];
  for (int I = 0; I < nb; ++I)
    for (int J = I; J < nb; ++J, t += 1024) ebe_tile(t, I, J, xs, ya);
  ebe_end(S, h0, nh, ya);
}

__device__ __forceinline__ uint32_t cg_smem_u32(const void* q) { return (uint32_t)__cvta_generic_to_shared(q); }

// Bounded wait on an mbarrier phase (false: the limit ran out).
__device__ __forceinline__ bool cg_mbar_wait(uint32_t mbar, uint32_t parity, unsigned long long limit) {
  const unsigned long long t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (done) return true;
    if (global_ns() - t0 > limit) return false;
  }
}

// The element products of this warp's elements (e = gw, gw + warps, ...) with
// the tiles staged through shared memory by the bulk-copy engine: a ring of
// `stages` 8 KB buffers, one mbarrier each; lane 0 keeps up to `stages` tile
// copies in flight, across element boundaries, and refills a buffer once the
// warp has consumed it.  tiles_done: tiles this warp consumed so far in the
// launch (it fixes every buffer's mbarrier parity).
__device__ __forceinline__ void ebe_pass_bulk(const SysView& S, const float2* __restrict__ p, float2* xs, float2* ya,
                                              float2* ring, uint64_t* mbar, int gw, int warps, uint32_t& tiles_done,
                                              CgState* st) {
  const int lane = threadIdx.x & 31;
  const int nst = S.ebe_stages;
  int pe = gw, pk = 0;
  uint32_t pn = tiles_done, cn = tiles_done;
  auto ntiles = [&](int e) {
    const int nb = (int)((S.ebe_hoff[e + 1] - S.ebe_hoff[e] + 31) >> 5);
    return nb * (nb + 1) / 2;
  };
  auto produce = [&]() {
    if (lane != 0) return;
    while (pn < cn + (uint32_t)nst && pe < S.ne) {
      const int stg = (int)(pn % (uint32_t)nst);
      const uint32_t mb = cg_smem_u32(mbar + stg);
      const float2* src = S.ebe + S.ebe_toff[pe] + (int64_t)pk * 1024;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(8192) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       cg_smem_u32(ring + (size_t)stg * 1024)),
                   "l"(src), "r"(8192), "r"(mb)
                   : "memory");
      ++pn;
      if (++pk == ntiles(pe)) {
        pk = 0;
        pe += warps;
      }
    }
  };
  produce();
  for (int e = gw; e < S.ne; e += warps) {
    int64_t h0;
    const int nh = ebe_begin(S, e, p, xs, ya, h0);
    const int nb = (nh + 31) >> 5;
    for (int I = 0; I < nb; ++I)
      for (int J = I; J < nb; ++J) {
        const int stg = (int)(cn % (uint32_t)nst);
        if (!cg_mbar_wait(cg_smem_u32(mbar + stg), (cn / (uint32_t)nst) & 1u, st->wait_ns) && lane == 0)
          atomicExch(&st->status, 1);
        ebe_tile(ring + (size_t)stg * 1024, I, J, xs, ya);
        __syncwarp();
        // the buffer's generic-proxy reads come before the next bulk copy into it
        if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ++cn;
        produce();
      }
    ebe_end(S, h0, nh, ya);
  }
  tiles_done = cn;
}

// SP: the SpMV of the inner solve: 0 rows of the CSR, 1 Hermitian half
// storage, 2 element by element.
template <typename V, typename Mv, int SP>
__global__ void __launch_bounds__(CG_THREADS, SP == 1 ? 4 : (SP == 2 ? 2 : (SP == 3 ? 1 : 5))) k_cg_persistent(SysView S, const Mv* __restrict__ val, V* x, V* r, V* p,
                                                             V* Ap, V* z, int precond,
                                                             const typename RealOf<V>::T* __restrict__ dinv,
                                                             const V* __restrict__ binv, double* red, CgState* st,
                                                             V* T) {
  using R = typename RealOf<V>::T;
  extern __shared__ __align__(16) unsigned char cg_smem[];
  V* rs = reinterpret_cast<V*>(cg_smem) + (threadIdx.x >> 5) * S.dmax;
  const int G = gridDim.x;
  double* redA = red;          // pAp partials
  double* redB0 = red + G;     // rr partials
  double* redB1 = red + 2 * G; // rz partials
  const int warps = G * (CG_THREADS / 32);
  const int gw = blockIdx.x * (CG_THREADS / 32) + (threadIdx.x >> 5);
  unsigned int gen = *((volatile unsigned int*)&st->bar[1]);
  const double tol2 = st->tol2;
  const int max_iter = st->max_iter;
  // bulk-copy staging of the element tiles (SP = 3): per warp up to four
  // mbarriers, one per staging buffer, and the count of tiles it consumed
  __shared__ __align__(8) uint64_t ebe_mbar[(CG_THREADS / 32) * 4];
  uint32_t ebe_tiles_done = 0;
  if constexpr (SP == 3) {
    if ((threadIdx.x & 31) == 0) {
      for (int k = 0; k < S.ebe_stages; ++k)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cg_smem_u32(ebe_mbar + (threadIdx.x >> 5) * 4 + k)));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
  }
  // phase 0: z = M^{-1} r, x = 0, and p = z; or, continuing the previous
  // solve after its residual was replaced by the true one (reliable update),
  // p = z + beta p with beta = r^H z / (r^H z)_previous
  const bool cont = st->cont != 0;
  R rr0 = 0, rz0 = 0;
  for (int b = gw; b < S.nblk; b += warps) {
    block_precond<V>(S, b, precond, r, z, dinv, binv, rs, rr0, rz0);
    __syncwarp();
    const int4 B = S.blk[b];
    for (int i = threadIdx.x & 31; i < B.y; i += 32) {
      if (!cont) p[B.x + i] = z[B.x + i];
      x[B.x + i] = mkv(0.0, 0.0, (V*)nullptr);
    }
  }
  block_partial(rr0, rz0, redB0, redB1);
  if (!grid_barrier(st, gen)) return;
  double rr, rz;
  grid_total(redB0, redB1, rr, rz);
  if (cont) {
    const R beta0 = (R)(rz / st->rz_prev);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)G * blockDim.x) {
      const V zv = z[i];
      V pv = p[i];
      pv.x = fma(beta0, pv.x, zv.x);
      pv.y = fma(beta0, pv.y, zv.y);
      p[i] = pv;
    }
    if (!grid_barrier(st, gen)) return;
  }
  int it = 0;
  bool done = rr <= tol2;
  while (!done && it < max_iter) {
    // A: Ap = A p and Re(p^H A p)
    R pap = 0;
    if constexpr (SP == 2 || SP == 3) {
      // element products into the slots, then each row the sum of its slots
      float2* xs = reinterpret_cast<float2*>(cg_smem + (CG_THREADS / 32) * (size_t)S.dmax * sizeof(V)) +
                   (size_t)(threadIdx.x >> 5) * 2 * 32 * S.ebe_nbmax;
      float2* ya = xs + 32 * S.ebe_nbmax;
      if constexpr (SP == 3) {
        const size_t base = ((CG_THREADS / 32) * (size_t)S.dmax * sizeof(V) +
                             (CG_THREADS / 32) * 2 * 32 * (size_t)S.ebe_nbmax * sizeof(float2) + 127) / 128 * 128;
        float2* ring = reinterpret_cast<float2*>(cg_smem + base) + (size_t)(threadIdx.x >> 5) * S.ebe_stages * 1024;
        ebe_pass_bulk(S, reinterpret_cast<const float2*>(p), xs, ya, ring, ebe_mbar + (threadIdx.x >> 5) * 4, gw,
                      warps, ebe_tiles_done, st);
      } else {
        for (int e = gw; e < S.ne; e += warps) ebe_element(S, e, reinterpret_cast<const float2*>(p), xs, ya);
      }
      if (!grid_barrier(st, gen)) return;
      for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < S.n; row += (int64_t)G * blockDim.x) {
        float yr = 0.0f, yi = 0.0f;
        for (int64_t k = S.ebe_rptr[row]; k < S.ebe_rptr[row + 1]; ++k) {
          const float2 v = S.ebe_ys[S.ebe_ridx[k]];
          yr += v.x;
          yi += v.y;
        }
        const V y = mkv(yr, yi, (V*)nullptr);
        Ap[row] = y;
        const V pr = p[row];
        pap += pr.x * y.x + pr.y * y.y;
      }
    } else if constexpr (SP == 1) {
      // lower blocks and diagonal blocks, conjugate-transpose partial sums
      for (int b = gw; b < S.nblk; b += warps) half_block_lower<V, Mv>(S, b, val, p, Ap, T);
      if (!grid_barrier(st, gen)) return;
      // the upper blocks: the partial sums of the upper neighbours, in list order
      for (int b = gw; b < S.nblk; b += warps) {
        const int4 B = S.blk[b];
        const int64_t k0 = S.rev_ptr[b], k1 = S.rev_ptr[b + 1];
        for (int i = threadIdx.x & 31; i < B.y; i += 32) {
          const int64_t row = B.x + i;
          V yv = Ap[row];
          int64_t k = k0;
          for (; k + 3 < k1; k += 4) {  // four independent loads in flight, summed in list order
            const int64_t o0 = S.rev_off[k], o1 = S.rev_off[k + 1], o2 = S.rev_off[k + 2], o3 = S.rev_off[k + 3];
            const V t0 = T[o0 + i], t1 = T[o1 + i], t2 = T[o2 + i], t3 = T[o3 + i];
            yv.x += t0.x;
            yv.y += t0.y;
            yv.x += t1.x;
            yv.y += t1.y;
            yv.x += t2.x;
            yv.y += t2.y;
            yv.x += t3.x;
            yv.y += t3.y;
          }
          for (; k < k1; ++k) {
            const V t = T[S.rev_off[k] + i];
            yv.x += t.x;
            yv.y += t.y;
          }
          Ap[row] = yv;
          const V pr = p[row];
          pap += pr.x * yv.x + pr.y * yv.y;
        }
      }
    } else {
      for (int64_t row = gw; row < S.n; row += warps) {
        const V y = row_spmv<V, Mv>(S, row, val, p);
        if ((threadIdx.x & 31) == 0) {
          Ap[row] = y;
          const V pr = p[row];
          pap += pr.x * y.x + pr.y * y.y;
        }
      }
    }
    block_partial(pap, (R)0, redA, nullptr);
    if (!grid_barrier(st, gen)) return;
    double tpap, dummy;
    grid_total(redA, nullptr, tpap, dummy);
    const R alpha = (R)(rz / tpap);
    // B: x += alpha p, r -= alpha Ap, z = M^{-1} r
    R rr2 = 0, rz2 = 0;
    for (int b = gw; b < S.nblk; b += warps) {
      const int4 B = S.blk[b];
      for (int i = threadIdx.x & 31; i < B.y; i += 32) {
        const int64_t row = B.x + i;
        V xv = x[row], rv = r[row];
        const V pv = p[row], av = Ap[row];
        xv.x = fma(alpha, pv.x, xv.x);
        xv.y = fma(alpha, pv.y, xv.y);
        rv.x = fma(-alpha, av.x, rv.x);
        rv.y = fma(-alpha, av.y, rv.y);
        x[row] = xv;
        r[row] = rv;
      }
      __syncwarp();
      block_precond<V>(S, b, precond, r, z, dinv, binv, rs, rr2, rz2);
    }
    block_partial(rr2, rz2, redB0, redB1);
    if (!grid_barrier(st, gen)) return;
    double trr, trz;
    grid_total(redB0, redB1, trr, trz);
    const R beta = (R)(trz / rz);
    rz = trz;
    rr = trr;
    ++it;
    if (rr <= tol2) break;
    // C: p = z + beta p
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)G * blockDim.x) {
      const V zv = z[i];
      V pv = p[i];
      pv.x = fma(beta, pv.x, zv.x);
      pv.y = fma(beta, pv.y, zv.y);
      p[i] = pv;
    }
    if (!grid_barrier(st, gen)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->iters = it;
    st->rr = rr;
    st->rz = rz;
  }
}

// r = b - A x in FP64 (x may be NULL for x = 0); ||r||^2 summed in block order.
__global__ void __launch_bounds__(CG_THREADS) k_residual(SysView S, const double2* __restrict__ val,
                                                         const double2* __restrict__ x, const double2* __restrict__ b,
                                                         double2* r, double* red, double* out) {
  const int warps = gridDim.x * (CG_THREADS / 32);
  const int gw = blockIdx.x * (CG_THREADS / 32) + (threadIdx.x >> 5);
  double acc = 0.0;
  for (int64_t row = gw; row < S.n; row += warps) {
    const double2 ax = x ? row_spmv<double2, double2>(S, row, val, x) : make_double2(0.0, 0.0);
    if ((threadIdx.x & 31) == 0) {
      const double2 bv = b[row];
      const double2 rv = make_double2(bv.x - ax.x, bv.y - ax.y);
      r[row] = rv;
      acc += rv.x * rv.x + rv.y * rv.y;
    }
  }
  block_partial(acc, 0.0, red, nullptr);
  // the caller sums red[0..G) with k_sum_red
}

__global__ void k_sum_red(int G, const double* __restrict__ red, double* out) {
  __shared__ double sw[32];
  double a = 0;
  for (int k = threadIdx.x; k < G; k += blockDim.x) a += red[k];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sw[k];
    *out = t;
  }
}

__global__ void k_to_f32(int64_t n, const double2* __restrict__ a, float2* b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void k_add_correction64(int64_t n, double2* x, const double2* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i].x += d[i].x;
    x[i].y += d[i].y;
  }
}

__global__ void k_add_correction(int64_t n, double2* x, const float2* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i].x += (double)d[i].x;
    x[i].y += (double)d[i].y;
  }
}

// Diagonal and entity-block inverses.  One CTA per entity block: the
// diagonal sub-block (the block's own columns are contiguous in its list
// from position blk.w) is inverted by Gauss-Jordan elimination (Hermitian
// positive definite, no pivoting needed) in shared memory.
__global__ void __launch_bounds__(128) k_block_inverse(SysView S, const double2* __restrict__ val, double2* binv,
                                                       float2* binv32, double* dinv, float* dinv32) {
  extern __shared__ double2 sm[];
  const int b = blockIdx.x;
  const int4 B = S.blk[b];
  const int d = B.y;
  double2* A = sm;          // d x d
  double2* Iv = sm + d * d; // d x d
  for (int t = threadIdx.x; t < d * d; t += blockDim.x) {
    const int i = t / d, j = t - i * d;
    A[t] = val[S.rowptr[B.x + i] + B.w + j];
    Iv[t] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double a = A[i * d + i].x;
    const double di = a > 0 ? 1.0 / a : 1.0;
    dinv[B.x + i] = di;
    dinv32[B.x + i] = (float)di;
  }
  for (int k = 0; k < d; ++k) {
    __syncthreads();
    const double2 piv = A[k * d + k];
    const double pm = piv.x * piv.x + piv.y * piv.y;
    const double2 ip = make_double2(piv.x / pm, -piv.y / pm);
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
      A[k * d + j] = c_mul(A[k * d + j], ip);
      Iv[k * d + j] = c_mul(Iv[k * d + j], ip);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < d * d; t += blockDim.x) {
      const int i = t / d, j = t - i * d;
      if (i == k) continue;
      const double2 f = A[i * d + k];
      const double2 ak = A[k * d + j], ik = Iv[k * d + j];
      // row i -= f * row k (A's column k is read before it is overwritten: f uses column k, j loops)
      if (j != k) {
        const double2 pa = c_mul(f, ak);
        A[i * d + j] = make_double2(A[i * d + j].x - pa.x, A[i * d + j].y - pa.y);
      }
      const double2 pi = c_mul(f, ik);
      Iv[i * d + j] = make_double2(Iv[i * d + j].x - pi.x, Iv[i * d + j].y - pi.y);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x)
      if (i != k) A[i * d + k] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int64_t o = S.binv_ptr[b];
  for (int t = threadIdx.x; t < d * d; t += blockDim.x) {
    binv[o + t] = Iv[t];
    binv32[o + t] = make_float2((float)Iv[t].x, (float)Iv[t].y);
  }
}

static SysView sys_view(dpg_handle* h) {
  SysView v;
  v.n = h->n;
  v.nblk = h->nblk;
  v.rowptr = h->d_rowptr;
  v.row2blk = h->d_row2blk;
  v.blk = h->d_blk;
  v.colptr = h->d_blk_colptr;
  v.cols = h->d_cols;
  v.binv_ptr = h->d_binv_ptr;
  v.dmax = h->blk_dmax;
  v.rowptr_h = h->d_rowptr_h;
  v.toff = h->d_toff;
  v.rev_ptr = h->d_rev_ptr;
  v.rev_off = h->d_rev_off;
  v.ne = h->ne;
  v.ebe_nbmax = h->ebe_nbmax;
  v.ebe = h->d_ebe;
  v.ebe_toff = h->d_ebe_toff;
  v.ebe_hoff = h->d_ebe_hoff;
  v.l2g = h->d_l2g;
  v.ebe_rptr = h->d_ebe_rptr;
  v.ebe_ridx = h->d_ebe_ridx;
  v.ebe_ys = h->d_ebe_ys;
  v.ebe_stages = h->ebe_stages;
  return v;
}

static int ensure_buf(dpg_handle* h, void** p, size_t bytes) {
  if (*p) return DPG_OK;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->err = "CG buffer allocation of " + std::to_string(bytes) + " bytes failed";
    return DPG_ERR_NOMEM;
  }
  return DPG_OK;
}

// Grid of a persistent cooperative CG kernel: every block resident (at most 8 per SM).
static int persistent_grid(dpg_handle* h, const void* kernel, size_t smem, int* grid) {
  int dev = 0, sms = 0, per = 0, coop = 0;
  DPG_CUDA_TRY(h, cudaGetDevice(&dev));
  DPG_CUDA_TRY(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DPG_CUDA_TRY(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) {
    h->err = "device does not support cooperative launches";
    return DPG_ERR_UNSUPPORTED;
  }
  if (smem > 48 * 1024)
    DPG_CUDA_TRY(h, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DPG_CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, CG_THREADS, smem));
  *grid = std::max(1, std::min(per, 8) * sms);
  return DPG_OK;
}

// One cooperative launch of a persistent CG kernel whose last argument is the
// CgState; the state is initialised before and read back after the solve.
static int launch_persistent(dpg_handle* h, const void* kernel, void** args, CgState** st_arg, size_t smem,
                             double tol2, int max_iter, bool fp32, cudaStream_t s, int* iters, double* rr_out,
                             int cont = 0, double rz_prev = 0.0, double* rz_out = nullptr) {
  int grid = 0;
  int rc = persistent_grid(h, kernel, smem, &grid);
  if (rc) return rc;
  CgState host{};
  host.tol2 = tol2;
  host.max_iter = max_iter;
  host.wait_ns = (unsigned long long)h->wait_ns;
  host.hold = h->wait_hold ? 1 : 0;
  host.cont = cont;
  host.rz_prev = rz_prev;
  CgState* st = static_cast<CgState*>(h->d_cgstate);
  *st_arg = st;
  DPG_CUDA_TRY(h, cudaMemcpyAsync(st, &host, sizeof(CgState), cudaMemcpyHostToDevice, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->timing) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  DPG_CUDA_TRY(h, cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(CG_THREADS), args, smem, s));
  h->launches += 1;
  if (h->timing) cudaEventRecord(e1, s);
  DPG_CUDA_TRY(h, cudaMemcpyAsync(&host, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  if (h->timing) {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->cgk_ms += ms;
    h->cgk_launches += 1;
    h->cgk_iters += host.iters;
    if (fp32) h->cgk_fp32 = true;
  }
  if (host.status != 0) {
    h->err = "a grid barrier of the CG kernel timed out";
    return DPG_ERR_TIMEOUT;
  }
  *iters = host.iters;
  *rr_out = host.rr;
  if (rz_out) *rz_out = host.rz;
  return DPG_OK;
}

// One persistent solve of A d = r0 (d = 0 at entry; r holds r0 at entry).
template <typename V, typename Mv, int SP>
static int run_persistent(dpg_handle* h, const Mv* val, V* x, V* r, V* p, V* Ap, V* z, int precond,
                          const typename RealOf<V>::T* dinv, const V* binv, double tol2, int max_iter,
                          cudaStream_t s, int* iters, double* rr_out, V* T = nullptr, int cont = 0,
                          double rz_prev = 0.0, double* rz_out = nullptr) {
  size_t smem = (CG_THREADS / 32) * (size_t)std::max(1, h->blk_dmax) * sizeof(V);
  if (SP == 2 || SP == 3) smem += (CG_THREADS / 32) * 2 * 32 * (size_t)h->ebe_nbmax * sizeof(float2);  // x_K, y_K
  if (SP == 3) smem = (smem + 127) / 128 * 128 + (CG_THREADS / 32) * (size_t)h->ebe_stages * 8192;  // tile staging
  SysView S = sys_view(h);
  double* red = h->d_red;
  CgState* st = nullptr;
  void* args[] = {&S, &val, &x, &r, &p, &Ap, &z, &precond, &dinv, &binv, &red, &st, &T};
  return launch_persistent(h, (const void*)k_cg_persistent<V, Mv, SP>, args, &st, smem, tol2, max_iter,
                           sizeof(Mv) == sizeof(float2), s, iters, rr_out, cont, rz_prev, rz_out);
}

// The same in the double-word mode (k_cg_dw).
static int run_dw(dpg_handle* h, double2* x, double2* r, int precond, double tol2, int max_iter, cudaStream_t s,
                  int* iters, double* rr_out) {
  const size_t smem = (CG_THREADS / 32) * (size_t)std::max(1, h->blk_dmax) * sizeof(float4);
  SysView S = sys_view(h);
  const float4* val = h->d_valdw;
  double2 *p = h->d_p, *Ap = h->d_Ap, *z = h->d_zv;
  float4* pdw = h->d_pdw;
  const float4* binv = h->d_binvdw;
  double* red = h->d_red;
  CgState* st = nullptr;
  void* args[] = {&S, &val, &x, &r, &p, &pdw, &Ap, &z, &precond, &binv, &red, &st};
  return launch_persistent(h, (const void*)k_cg_dw, args, &st, smem, tol2, max_iter, false, s, iters, rr_out);
}

static int residual(dpg_handle* h, const double2* x, const double2* b, double2* r, cudaStream_t s, double* rr) {
  SysView S = sys_view(h);
  const int G = 1184;
  k_residual<<<G, CG_THREADS, 0, s>>>(S, h->d_val, x, b, r, h->d_red, nullptr);
  k_sum_red<<<1, 1024, 0, s>>>(G, h->d_red, h->d_red + 3 * 4096);
  h->launches += 2;
  DPG_CUDA_TRY(h, cudaMemcpyAsync(rr, h->d_red + 3 * 4096, sizeof(double), cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  return DPG_OK;
}

static int prepare_preconditioner(dpg_handle* h, cudaStream_t s) {
  if (h->have_binv) return DPG_OK;
  if (!h->d_binv_ptr) {
    std::vector<int64_t> ptr(h->nblk + 1, 0);
    int dmax = 0;
    for (int b = 0; b < h->nblk; ++b) {
      ptr[b + 1] = ptr[b] + (int64_t)h->blk[b].y * h->blk[b].y;
      dmax = std::max(dmax, h->blk[b].y);
    }
    h->binv_dmax = dmax;
    int rc = 0;
    rc |= ensure_buf(h, (void**)&h->d_binv_ptr, sizeof(int64_t) * (h->nblk + 1));
    rc |= ensure_buf(h, (void**)&h->d_binv, sizeof(double2) * ptr[h->nblk]);
    rc |= ensure_buf(h, (void**)&h->d_binv32, sizeof(float2) * ptr[h->nblk]);
    rc |= ensure_buf(h, (void**)&h->d_dinv, sizeof(double) * h->n);
    rc |= ensure_buf(h, (void**)&h->d_dinv32, sizeof(float) * h->n);
    if (rc) return DPG_ERR_NOMEM;
    DPG_CUDA_TRY(h, cudaMemcpy(h->d_binv_ptr, ptr.data(), sizeof(int64_t) * ptr.size(), cudaMemcpyHostToDevice));
  }
  const size_t smem = sizeof(double2) * 2 * (size_t)h->binv_dmax * h->binv_dmax;
  if (smem > 48 * 1024)
    DPG_CUDA_TRY(h, cudaFuncSetAttribute(k_block_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_block_inverse<<<h->nblk, 128, smem, s>>>(sys_view(h), h->d_val, h->d_binv, h->d_binv32, h->d_dinv, h->d_dinv32);
  h->launches += 1;
  DPG_CUDA_TRY(h, cudaGetLastError());
  h->have_binv = true;
  h->have_dinv = true;
  return DPG_OK;
}

// Element-by-element FP32 operator: per element the upper-triangle 32 x 32
// tiles of its stored S_K (row-major n_h x n_h, FP64), zero past n_h.
__global__ void __launch_bounds__(256) k_ebe_pack(const ElemOff* __restrict__ off, const int64_t* __restrict__ toff,
                                                  const double2* __restrict__ Sst, float2* ebe) {
  const int e = blockIdx.x;
  const int nh = (int)(off[e + 1].h - off[e].h), nb = (nh + 31) >> 5;
  const double2* Se = Sst + off[e].S;
  float2* t = ebe + toff[e];
  const int ntile = nb * (nb + 1) / 2;
  for (int64_t q = threadIdx.x; q < (int64_t)ntile * 1024; q += blockDim.x) {
    int k = (int)(q >> 10);
    const int ij = (int)(q & 1023), i = ij >> 5, j = ij & 31;
    int I = 0;
    while (k >= nb - I) {  // tile k of the I-major upper triangle
      k -= nb - I;
      ++I;
    }
    const int J = I + k;
    const int row = I * 32 + i, col = J * 32 + j;
    float2 v = make_float2(0.0f, 0.0f);
    if (row < nh && col < nh) {
      const double2 a = Se[(size_t)row * nh + col];
      v = make_float2((float)a.x, (float)a.y);
    }
    t[q] = v;
  }
}

// Index structures of the element-by-element operator (once per mesh): tile
// and slot offsets per element, and per row its slots in ascending order.
static int build_ebe_index(dpg_handle* h) {
  if (h->have_ebe_idx) return DPG_OK;
  const int ne = h->ne;
  std::vector<int64_t> toff(ne + 1, 0), hoff(ne + 1, 0);
  int nbmax = 1;
  for (int e = 0; e < ne; ++e) {
    const int nh = (int)(h->off[e + 1].h - h->off[e].h), nb = (nh + 31) / 32;
    nbmax = std::max(nbmax, nb);
    toff[e + 1] = toff[e] + (int64_t)nb * (nb + 1) / 2 * 1024;
    hoff[e] = h->off[e].h;
  }
  hoff[ne] = h->off[ne].h;
  const int64_t slots = hoff[ne];
  if (slots >= ((int64_t)1 << 31)) {
    h->err = "too many trace slots for the element-by-element operator";
    return DPG_ERR_UNSUPPORTED;
  }
  std::vector<int64_t> rptr(h->n + 1, 0);
  for (int64_t q = 0; q < slots; ++q)
    if (h->l2g[q] >= 0) rptr[h->l2g[q] + 1] += 1;
  for (int64_t i = 0; i < h->n; ++i) rptr[i + 1] += rptr[i];
  std::vector<int32_t> ridx(std::max<int64_t>(1, rptr[h->n]));
  std::vector<int64_t> fill(rptr.begin(), rptr.end() - 1);
  for (int64_t q = 0; q < slots; ++q)
    if (h->l2g[q] >= 0) ridx[fill[h->l2g[q]]++] = (int32_t)q;
  int rc = 0;
  rc |= ensure_buf(h, (void**)&h->d_ebe, sizeof(float2) * std::max<int64_t>(1, toff[ne]));
  rc |= ensure_buf(h, (void**)&h->d_ebe_toff, sizeof(int64_t) * (ne + 1));
  rc |= ensure_buf(h, (void**)&h->d_ebe_hoff, sizeof(int64_t) * (ne + 1));
  rc |= ensure_buf(h, (void**)&h->d_ebe_rptr, sizeof(int64_t) * (h->n + 1));
  rc |= ensure_buf(h, (void**)&h->d_ebe_ridx, sizeof(int32_t) * ridx.size());
  rc |= ensure_buf(h, (void**)&h->d_ebe_ys, sizeof(float2) * std::max<int64_t>(1, slots));
  if (rc) return DPG_ERR_NOMEM;
  DPG_CUDA_TRY(h, cudaMemcpy(h->d_ebe_toff, toff.data(), sizeof(int64_t) * toff.size(), cudaMemcpyHostToDevice));
  DPG_CUDA_TRY(h, cudaMemcpy(h->d_ebe_hoff, hoff.data(), sizeof(int64_t) * hoff.size(), cudaMemcpyHostToDevice));
  DPG_CUDA_TRY(h, cudaMemcpy(h->d_ebe_rptr, rptr.data(), sizeof(int64_t) * rptr.size(), cudaMemcpyHostToDevice));
  DPG_CUDA_TRY(h, cudaMemcpy(h->d_ebe_ridx, ridx.data(), sizeof(int32_t) * ridx.size(), cudaMemcpyHostToDevice));
  h->ebe_nbmax = nbmax;
  // staging buffers per warp of the bulk-copy variant: three, or two when the
  // x_K / y_K staging of the largest element leaves no room for three
  {
    const size_t fixed = (CG_THREADS / 32) * ((size_t)std::max(1, h->blk_dmax) * sizeof(float2) +
                                              2 * 32 * (size_t)nbmax * sizeof(float2)) + 128;
    h->ebe_stages = fixed + (CG_THREADS / 32) * 3 * 8192 <= 227 * 1024 ? 3 : 2;
  }
  h->ebe_tiles = toff[ne];
  h->ebe_slots = slots;
  h->ebe_links = rptr[h->n];
  h->have_ebe_idx = true;
  return DPG_OK;
}

// Hermitian half storage of the FP32 inner matrix: row pointers of the stored
// prefixes, the partial-sum offsets per block and, per block b, the T offsets
// of b's segments in its upper neighbours' partial sums (in block order, so
// every sum is taken in one fixed order).  Host-side construction, once.
static int build_half(dpg_handle* h) {
  if (h->have_half) return DPG_OK;
  const int nb = h->nblk;
  std::vector<int32_t> row2blk(h->n);
  for (int b = 0; b < nb; ++b)
    for (int i = 0; i < h->blk[b].y; ++i) row2blk[h->blk[b].x + i] = b;
  std::vector<int64_t> rowptr_h(h->n + 1, 0), toff(nb + 1, 0);
  int wmax = 0;
  for (int b = 0; b < nb; ++b) {
    const int4& B = h->blk[b];
    const int Wh = B.w + B.y;
    wmax = std::max(wmax, Wh);
    for (int i = 0; i < B.y; ++i) rowptr_h[B.x + i + 1] = Wh;
    toff[b + 1] = toff[b] + B.w;
  }
  for (int64_t i = 0; i < h->n; ++i) rowptr_h[i + 1] += rowptr_h[i];
  std::vector<std::vector<int64_t>> rev(nb);
  for (int a = 0; a < nb; ++a) {
    const int4& A = h->blk[a];
    const int32_t* c = &h->cols[h->blk_colptr[a]];
    for (int q = 0; q < A.w; ++q) {
      const int b = row2blk[c[q]];
      if (c[q] == h->blk[b].x) rev[b].push_back(toff[a] + q);  // first column of b's segment
    }
  }
  std::vector<int64_t> rev_ptr(nb + 1, 0), rev_off;
  for (int b = 0; b < nb; ++b) {
    rev_ptr[b + 1] = rev_ptr[b] + (int64_t)rev[b].size();
    rev_off.insert(rev_off.end(), rev[b].begin(), rev[b].end());
  }
  h->nnz_h = rowptr_h[h->n];
  h->t_len = toff[nb];
  h->rev_len = (int64_t)rev_off.size();
  h->half_wmax = wmax;
  int rc = 0;
  rc |= ensure_buf(h, (void**)&h->d_rowptr_h, sizeof(int64_t) * (h->n + 1));
  rc |= ensure_buf(h, (void**)&h->d_toff, sizeof(int64_t) * (nb + 1));
  rc |= ensure_buf(h, (void**)&h->d_rev_ptr, sizeof(int64_t) * (nb + 1));
  rc |= ensure_buf(h, (void**)&h->d_rev_off, sizeof(int64_t) * std::max<int64_t>(1, h->rev_len));
  rc |= ensure_buf(h, (void**)&h->d_val32h, sizeof(float2) * h->nnz_h);
  rc |= ensure_buf(h, (void**)&h->d_T, sizeof(float2) * std::max<int64_t>(1, h->t_len));
  if (rc) return DPG_ERR_NOMEM;
  DPG_CUDA_TRY(h, cudaMemcpy(h->d_rowptr_h, rowptr_h.data(), sizeof(int64_t) * rowptr_h.size(), cudaMemcpyHostToDevice));
  DPG_CUDA_TRY(h, cudaMemcpy(h->d_toff, toff.data(), sizeof(int64_t) * toff.size(), cudaMemcpyHostToDevice));
  DPG_CUDA_TRY(h, cudaMemcpy(h->d_rev_ptr, rev_ptr.data(), sizeof(int64_t) * rev_ptr.size(), cudaMemcpyHostToDevice));
  if (!rev_off.empty())
    DPG_CUDA_TRY(h, cudaMemcpy(h->d_rev_off, rev_off.data(), sizeof(int64_t) * rev_off.size(), cudaMemcpyHostToDevice));
  h->have_half = true;
  return DPG_OK;
}

// FP32 copy of each row's stored prefix (one warp per row).
__global__ void __launch_bounds__(256) k_to_f32_half(SysView S, const double2* __restrict__ val, float2* valh) {
  const int warps = gridDim.x * (blockDim.x / 32);
  const int lane = threadIdx.x & 31;
  for (int64_t row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); row < S.n; row += warps) {
    const int4 B = S.blk[S.row2blk[row]];
    const int Wh = B.w + B.y;
    const double2* v = val + S.rowptr[row];
    float2* o = valh + S.rowptr_h[row];
    for (int q = lane; q < Wh; q += 32) o[q] = make_float2((float)v[q].x, (float)v[q].y);
  }
}

// Algorithmic bytes of one CG iteration: the matrix values (16 B per complex
// non-zero in FP64, 8 B in FP32), the per-entity column lists, the
// preconditioner data, and the vector traffic of the three phases
// (SpMV reads p once and writes Ap; the update reads x, r, p, Ap and writes
// x, r, z; the direction update reads z, p and writes p): 13 vector passes.
int64_t cg_bytes_per_iteration(const dpg_handle* h, int mode) {
  const bool ir = (mode & DPG_CG_IR_FP32) != 0;
  const bool v64 = ir && (mode & DPG_CG_IR_V64);
  const int64_t mb = ir ? 8 : 16, vb = (ir && !v64) ? 8 : 16;  // DW: 16 B values (two FP32 pairs), FP64 vectors
  int64_t ncol = (int64_t)h->cols.size();
  int64_t bytes = 0;
  if (ir && (mode & DPG_CG_EBE)) {
    // element by element: the tiles, per slot the x gather, the trace map, the
    // product written and read back, its index in the row lists; per row the
    // list pointer; the vector passes
    int64_t tiles = 0;
    for (int e = 0; e < h->ne; ++e) {
      const int64_t nb = (h->off[e + 1].h - h->off[e].h + 31) / 32;
      tiles += nb * (nb + 1) / 2 * 1024;
    }
    const int64_t slots = h->off[h->ne].h;
    bytes = 8 * tiles + slots * (8 + 4 + 8 + 8 + 4) + 8 * (h->n + 1) + 13 * vb * h->n;
  } else if (ir && (mode & DPG_CG_HALF)) {
    // half storage: stored prefixes, their column lists, the partial sums T
    // (written once, read once) and their offsets
    int64_t nh = 0, ncol_h = 0, tl = 0;
    for (const int4& B : h->blk) {
      nh += (int64_t)B.y * (B.w + B.y);
      ncol_h += B.w + B.y;
      tl += B.w;
    }
    bytes = mb * nh + 4 * ncol_h + 2 * vb * tl + 8 * h->rev_len + 14 * vb * h->n;
  } else {
    bytes = mb * h->nnz + 4 * ncol + 13 * vb * h->n;
  }
  if (mode & DPG_CG_BLOCK_JACOBI) {
    int64_t inv = 0;
    for (const int4& B : h->blk) inv += (int64_t)B.y * B.y;
    bytes += vb * inv;
  } else if (mode & DPG_CG_JACOBI) {
    bytes += (ir ? 4 : 8) * h->n;
  }
  return bytes;
}

int cg_solve(dpg_handle* h, int mode, double rtol, double atol, int max_iter, double inner_rtol, double2* x,
             const double2* b, dpg_cg_report* rep, cudaStream_t s) {
  if (!h->have_system) {
    h->err = "dpg_cg_solve before dpg_assemble";
    return DPG_ERR_STATE;
  }
  if (!x || max_iter <= 0 || !(rtol >= 0) || !(atol >= 0)) {
    h->err = "bad CG arguments";
    return DPG_ERR_ARG;
  }
  if (mode & ~(DPG_CG_IR_FP32 | DPG_CG_JACOBI | DPG_CG_BLOCK_JACOBI | DPG_CG_X0 | DPG_CG_HALF | DPG_CG_IR_V64 |
               DPG_CG_DW | DPG_CG_EBE | DPG_CG_RELIABLE | DPG_CG_EBE_BULK) ||
      ((mode & DPG_CG_EBE_BULK) && !(mode & DPG_CG_EBE)) ||
      ((mode & DPG_CG_RELIABLE) && !(mode & DPG_CG_IR_FP32)) ||
      ((mode & DPG_CG_HALF) && (mode & DPG_CG_IR_V64)) ||
      ((mode & DPG_CG_EBE) && (!(mode & DPG_CG_IR_FP32) || (mode & (DPG_CG_HALF | DPG_CG_IR_V64)))) ||
      ((mode & DPG_CG_DW) && (mode & (DPG_CG_IR_FP32 | DPG_CG_JACOBI))) ||
      ((mode & DPG_CG_JACOBI) && (mode & DPG_CG_BLOCK_JACOBI))) {
    h->err = "unknown CG mode";
    return DPG_ERR_ARG;
  }
  const bool ir = (mode & DPG_CG_IR_FP32) != 0;
  const int precond = (mode & DPG_CG_BLOCK_JACOBI) ? 2 : ((mode & DPG_CG_JACOBI) ? 1 : 0);
  const size_t n = h->n;
  int rc = 0;
  rc |= ensure_buf(h, (void**)&h->d_r, sizeof(double2) * n);
  rc |= ensure_buf(h, (void**)&h->d_p, sizeof(double2) * n);
  rc |= ensure_buf(h, (void**)&h->d_Ap, sizeof(double2) * n);
  rc |= ensure_buf(h, (void**)&h->d_zv, sizeof(double2) * n);
  rc |= ensure_buf(h, (void**)&h->d_d64, sizeof(double2) * n);
  rc |= ensure_buf(h, (void**)&h->d_red, sizeof(double) * (3 * 4096 + 8));
  rc |= ensure_buf(h, (void**)&h->d_cgstate, sizeof(CgState));
  if (ir) {
    rc |= ensure_buf(h, (void**)&h->d_r32, sizeof(float2) * n);
    rc |= ensure_buf(h, (void**)&h->d_p32, sizeof(float2) * n);
    rc |= ensure_buf(h, (void**)&h->d_Ap32, sizeof(float2) * n);
    rc |= ensure_buf(h, (void**)&h->d_x32, sizeof(float2) * n);
    rc |= ensure_buf(h, (void**)&h->d_z32, sizeof(float2) * n);
  }
  if (rc) return DPG_ERR_NOMEM;
  const bool half = ir && (mode & DPG_CG_HALF) && !(mode & DPG_CG_IR_V64);
  const bool ebe = ir && (mode & DPG_CG_EBE);
  if (ebe && h->stream) {
    h->err = "the element-by-element operator reads every element's S_K; streaming keeps chunk stores only";
    return DPG_ERR_UNSUPPORTED;
  }
  const bool dw = (mode & DPG_CG_DW) != 0;
  if (dw) {
    rc |= ensure_buf(h, (void**)&h->d_valdw, sizeof(float4) * h->nnz);
    rc |= ensure_buf(h, (void**)&h->d_pdw, sizeof(float4) * n);
    if (rc) return DPG_ERR_NOMEM;
  }
  if (half) {
    rc = build_half(h);
    if (rc) return rc;
  } else if (ebe) {
    rc = build_ebe_index(h);
    if (rc) return rc;
  } else if (ir) {
    rc = ensure_buf(h, (void**)&h->d_val32, sizeof(float2) * h->nnz);
    if (rc) return rc;
  }
  const double2* rhs = b ? b : h->d_b;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, s);
  if (precond) {
    rc = prepare_preconditioner(h, s);
    if (rc) return rc;
  }
  if (dw && !h->have_valdw) {
    k_to_dw<<<1184, 256, 0, s>>>(h->nnz, h->d_val, h->d_valdw);
    h->launches += 1;
    h->have_valdw = true;
  }
  if (dw && precond == 2 && !h->have_binvdw) {
    int64_t inv = 0;
    for (const int4& B : h->blk) inv += (int64_t)B.y * B.y;
    rc = ensure_buf(h, (void**)&h->d_binvdw, sizeof(float4) * inv);
    if (rc) return rc;
    k_to_dw<<<1184, 256, 0, s>>>(inv, h->d_binv, h->d_binvdw);
    h->launches += 1;
    h->have_binvdw = true;
  }
  if (half && !h->have_val32h) {
    k_to_f32_half<<<1184, 256, 0, s>>>(sys_view(h), h->d_val, h->d_val32h);
    h->launches += 1;
    h->have_val32h = true;
  }
  if (ebe && !h->have_ebe) {
    k_ebe_pack<<<h->ne, 256, 0, s>>>(h->d_off, h->d_ebe_toff, h->d_S, h->d_ebe);
    h->launches += 1;
    DPG_CUDA_TRY(h, cudaGetLastError());
    h->have_ebe = true;
  }
  if (ir && !half && !ebe && !h->have_val32) {
    k_to_f32<<<1184, 256, 0, s>>>(h->nnz, h->d_val, h->d_val32);
    h->launches += 1;
    h->have_val32 = true;
  }
  // ||b|| (and r = b for x0 = 0)
  double bb = 0;
  rc = residual(h, nullptr, rhs, h->d_r, s, &bb);
  if (rc) return rc;
  const double bnorm = std::sqrt(bb);
  const double tol = std::max(rtol * bnorm, atol);
  int total_iters = 0, outer = 0;
  // Outer loop: solve A d = r for the current true residual, x += d, recompute
  // r = b - A x in FP64.  With FP32 inner solves this is iterative refinement
  // (inner tolerance inner_rtol); with FP64 inner solves the first pass already
  // targets the final tolerance and further passes only replace a recursive
  // residual that drifted from the true one.
  double rnorm = bnorm;
  if (mode & DPG_CG_X0) {  // warm start: r = b - A x for the caller's x
    double r2 = 0;
    rc = residual(h, x, rhs, h->d_r, s, &r2);
    if (rc) return rc;
    rnorm = std::sqrt(r2);
  } else {
    DPG_CUDA_TRY(h, cudaMemsetAsync(x, 0, sizeof(double2) * n, s));
  }
  bool conv = rnorm <= tol;
  const int max_outer = ir ? 100 : 8;
  // reliable updates: every inner solve after the first continues the previous
  // one's search direction (p = z + beta p) from the replaced true residual
  const bool reliable = (mode & DPG_CG_RELIABLE) != 0;
  double rz_last = 0.0;
  while (!conv && total_iters < max_iter && outer < max_outer) {
    int it = 0;
    double rr = 0;
    const int cont = (reliable && outer > 0 && rz_last > 0.0) ? 1 : 0;
    if (dw) {
      const double itol = 0.5 * tol;
      rc = run_dw(h, h->d_d64, h->d_r, precond, itol * itol, max_iter - total_iters, s, &it, &rr);
      if (rc) return rc;
      k_add_correction64<<<1184, 256, 0, s>>>((int64_t)n, x, h->d_d64);
    } else if (ir && (mode & DPG_CG_IR_V64)) {
      // inner CG over the FP32 matrix (FP32 products) with FP64 vectors and recurrences
      const double itol = std::max(inner_rtol * rnorm, 0.5 * tol);
      rc = run_persistent<double2, float2, 0>(h, h->d_val32, h->d_d64, h->d_r, h->d_p, h->d_Ap, h->d_zv, precond,
                                              h->d_dinv, h->d_binv, itol * itol, max_iter - total_iters, s, &it,
                                              &rr, nullptr, cont, rz_last, &rz_last);
      if (rc) return rc;
      k_add_correction64<<<1184, 256, 0, s>>>((int64_t)n, x, h->d_d64);
    } else if (ir) {
      const double itol = std::max(inner_rtol * rnorm, 0.5 * tol);
      k_to_f32<<<1184, 256, 0, s>>>((int64_t)n, h->d_r, h->d_r32);
      h->launches += 1;
      if (half)
        rc = run_persistent<float2, float2, 1>(h, h->d_val32h, h->d_x32, h->d_r32, h->d_p32, h->d_Ap32, h->d_z32,
                                               precond, h->d_dinv32, h->d_binv32, itol * itol,
                                               max_iter - total_iters, s, &it, &rr, h->d_T, cont, rz_last,
                                               &rz_last);
      else if (ebe && (mode & DPG_CG_EBE_BULK))
        rc = run_persistent<float2, float2, 3>(h, (const float2*)nullptr, h->d_x32, h->d_r32, h->d_p32, h->d_Ap32,
                                               h->d_z32, precond, h->d_dinv32, h->d_binv32, itol * itol,
                                               max_iter - total_iters, s, &it, &rr, nullptr, cont, rz_last,
                                               &rz_last);
      else if (ebe)
        rc = run_persistent<float2, float2, 2>(h, (const float2*)nullptr, h->d_x32, h->d_r32, h->d_p32, h->d_Ap32,
                                               h->d_z32, precond, h->d_dinv32, h->d_binv32, itol * itol,
                                               max_iter - total_iters, s, &it, &rr, nullptr, cont, rz_last,
                                               &rz_last);
      else
        rc = run_persistent<float2, float2, 0>(h, h->d_val32, h->d_x32, h->d_r32, h->d_p32, h->d_Ap32, h->d_z32,
                                               precond, h->d_dinv32, h->d_binv32, itol * itol,
                                               max_iter - total_iters, s, &it, &rr, nullptr, cont, rz_last,
                                               &rz_last);
      if (rc) return rc;
      k_add_correction<<<1184, 256, 0, s>>>((int64_t)n, x, h->d_x32);
    } else {
      const double itol = 0.5 * tol;
      rc = run_persistent<double2, double2, false>(h, h->d_val, h->d_d64, h->d_r, h->d_p, h->d_Ap, h->d_zv, precond,
                                            h->d_dinv, h->d_binv, itol * itol, max_iter - total_iters, s, &it, &rr);
      if (rc) return rc;
      k_add_correction64<<<1184, 256, 0, s>>>((int64_t)n, x, h->d_d64);
    }
    h->launches += 1;
    total_iters += it;
    ++outer;
    double r2 = 0;
    rc = residual(h, x, rhs, h->d_r, s, &r2);
    if (rc) return rc;
    rnorm = std::sqrt(r2);
    conv = rnorm <= tol;
    if (it == 0) break;
  }
  // final true residual in FP64
  double res2 = 0;
  rc = residual(h, x, rhs, h->d_Ap, s, &res2);
  if (rc) return rc;
  cudaEventRecord(t1, s);
  cudaEventSynchronize(t1);
  float ms = 0;
  cudaEventElapsedTime(&ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  const double res = std::sqrt(res2);
  const double rel = bnorm > 0 ? res / bnorm : 0.0;
  // the recursive residual of plain CG may sit a hair below the true one
  const bool converged = res <= tol;
  h->cg_ms += ms;
  h->cg_iters += total_iters;
  if (rep) {
    rep->iterations = total_iters;
    rep->outer = outer;
    rep->rel_residual = rel;
    rep->ms = ms;
    rep->converged = converged ? 1 : 0;
  }
  if (!converged) {
    h->err = "CG did not reach the tolerance within max_iter";
    return DPG_ERR_NOT_CONVERGED;
  }
  return DPG_OK;
}

// ------------------------------------------------------------ estimate --
__global__ void k_sqrt_sum(int n, const double* __restrict__ eta2, double* eta, double* total) {
  __shared__ double sw[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = eta2[i];  // >= 0 (the recompute pass clamps and counts negatives)
    if (eta) eta[i] = sqrt(v);
    acc += v;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sw[k];
    *total = t;
  }
}

// u (optional), eta_K^2 into eta2[0, ne) and their sum into eta2[ne]; the
// host value (if asked) after a synchronisation that also reports a timed-out
// tensor-core wait of the recompute pass.
static int estimate_into(dpg_handle* h, const double2* xhat, double2* u, double* eta, double* eta_global,
                         double* eta2, cudaStream_t s) {
  if (!eta && !eta_global) {  // recovery only
    if (u) {
      const int rc = recover_u(h, xhat, u, s);
      if (rc) return rc;
    }
    DPG_CUDA_TRY(h, cudaGetLastError());
    return DPG_OK;
  }
  int rc = estimate_pass(h, xhat, u, eta2, s);
  if (rc) return rc;
  k_sqrt_sum<<<1, 1024, 0, s>>>(h->ne, eta2, eta, eta2 + h->ne);
  h->launches += 1;
  DPG_CUDA_TRY(h, cudaGetLastError());
  if (eta_global) {
    double tot = 0;
    int terr = 0;
    DPG_CUDA_TRY(h, cudaMemcpyAsync(&tot, eta2 + h->ne, sizeof(double), cudaMemcpyDeviceToHost, s));
    DPG_CUDA_TRY(h, cudaMemcpyAsync(&terr, h->d_status + h->ne, sizeof(int), cudaMemcpyDeviceToHost, s));
    DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
    if (terr) {
      h->err = "a tensor-core wait of the estimator gave up";
      return DPG_ERR_TIMEOUT;
    }
    *eta_global = std::sqrt(std::max(tot, 0.0));
  }
  return DPG_OK;
}

int estimate(dpg_handle* h, const double2* xhat, double2* u, double* eta, double* eta_global, cudaStream_t s) {
  if (!h->have_elements) {
    h->err = "dpg_estimate before dpg_element_batch";
    return DPG_ERR_STATE;
  }
  if (!xhat) {
    h->err = "null xhat";
    return DPG_ERR_ARG;
  }
  double* d_eta2 = nullptr;
  if (eta || eta_global) DPG_CUDA_TRY(h, cudaMallocAsync(&d_eta2, sizeof(double) * (h->ne + 1), s));
  const int rc = estimate_into(h, xhat, u, eta, eta_global, d_eta2, s);
  if (d_eta2) cudaFreeAsync(d_eta2, s);
  return rc;
}

int estimate_negatives(dpg_handle* h, int* count) {
  if (!h->d_est_neg) {
    *count = 0;
    return DPG_OK;
  }
  DPG_CUDA_TRY(h, cudaMemcpy(count, h->d_est_neg, sizeof(int), cudaMemcpyDeviceToHost));
  return DPG_OK;
}

// ------------------------------------------------ allocation-free estimate --
// Variant of estimate() for callers that must not allocate device memory at
// call time (for example a process whose device memory is committed to its
// own pool up front, or a loop that may not wait on an allocator).  Its only
// scratch, the per-element eta_K^2 values and their sum, lives in the
// file-scope array below, which every GPU that loads this library holds until
// the process exits (8 MiB).  Nothing in it has to start at zero: every call
// overwrites the first n_elem + 1 entries before reading them.  All calls
// share the array, so calls that overlap on the GPU (different streams or
// different handles on the same device) race on it.
constexpr int NOALLOC_MAX_ELEMS = (1 << 20) - 1;
static __device__ __align__(256) double g_noalloc_eta2[NOALLOC_MAX_ELEMS + 1];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
}  // namespace

// Device address of the scratch array on the current device.  The first call
// on a device looks it up with cudaGetSymbolAddress (the host-side name of a
// __device__ array is not a device address); later calls reuse it.
static int noalloc_scratch(dpg_handle* h, double** out) {
  int dev = 0;
  DPG_CUDA_TRY(h, cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    h->err = "device index beyond the allocation-free table";
    return DPG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_eta2);
    if (e != cudaSuccess || !p) {
      h->err = std::string("cudaGetSymbolAddress of the estimate scratch: ") + cudaGetErrorString(e);
      return DPG_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return DPG_OK;
}

int estimate_noalloc(dpg_handle* h, const double2* xhat, double2* u, double* eta, double* eta_global,
                     cudaStream_t s) {
  if (!h->have_elements) {
    h->err = "dpg_estimate_noalloc before dpg_element_batch";
    return DPG_ERR_STATE;
  }
  if (!xhat) {
    h->err = "null xhat";
    return DPG_ERR_ARG;
  }
  if (h->ne > NOALLOC_MAX_ELEMS) {
    h->err = "dpg_estimate_noalloc supports at most " + std::to_string(NOALLOC_MAX_ELEMS) +
             " elements; this mesh has " + std::to_string(h->ne) + " (use dpg_estimate)";
    return DPG_ERR_ARG;
  }
  double* scratch = nullptr;
  int rc = noalloc_scratch(h, &scratch);
  if (rc) return rc;
  // the recompute pass runs in the handle's chunk workspace, allocated at setup
  return estimate_into(h, xhat, u, eta, eta_global, scratch, s);
}

}  // namespace dpg
