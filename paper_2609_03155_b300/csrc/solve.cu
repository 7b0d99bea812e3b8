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
// One block per element of one colour: elements of a colour share no
// unknowns, so the plain read-modify-write below has no race and the sum
// order per entry is the fixed colour order.
__global__ void __launch_bounds__(256) k_assemble(int nh, const int* __restrict__ elems, const int32_t* __restrict__ l2g,
                                                  const double2* __restrict__ xfix, const double2* __restrict__ Sst,
                                                  const double2* __restrict__ sst, const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ col, double2* val, double2* b) {
  const int e = elems[blockIdx.x];
  const int32_t* g = l2g + (size_t)e * nh;
  const double2* Se = Sst + (size_t)e * nh * nh;
  for (int t = threadIdx.x; t < nh * nh; t += blockDim.x) {
    const int i = t / nh, j = t - i * nh;
    const int gi = g[i], gj = g[j];
    if (gi < 0 || gj < 0) continue;
    const int64_t end = rowptr[gi + 1];
    int64_t lo = rowptr[gi], hi = end - 1;
    if (lo >= end) continue;
    while (lo < hi) {  // first position with col >= gj
      int64_t mid = (lo + hi) >> 1;
      if (col[mid] < gj)
        lo = mid + 1;
      else
        hi = mid;
    }
    if (col[lo] == gj) {
      double2 v = val[lo];
      val[lo] = c_add(v, Se[t]);
    }
  }
  for (int i = threadIdx.x; i < nh; i += blockDim.x) {
    const int gi = g[i];
    if (gi < 0) continue;
    double2 acc = sst[(size_t)e * nh + i];
    for (int j = 0; j < nh; ++j)
      if (g[j] == -1) {  // Dirichlet lifting: b -= S_{i,fixed} x_D
        double2 pr = c_mul(Se[(size_t)i * nh + j], xfix[(size_t)e * nh + j]);
        acc.x -= pr.x;
        acc.y -= pr.y;
      }
    b[gi] = c_add(b[gi], acc);
  }
}

int assemble_system(dpg_handle* h, cudaStream_t s) {
  const Sizes& S = h->sz;
  DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_val, 0, sizeof(double2) * h->nnz, s));
  DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_b, 0, sizeof(double2) * h->n, s));
  const int ncol = (int)h->color_off.size() - 1;
  for (int c = 0; c < ncol; ++c) {
    int cnt = h->color_off[c + 1] - h->color_off[c];
    if (cnt == 0) continue;
    k_assemble<<<cnt, 256, 0, s>>>(S.n_h, h->d_color_elems + h->color_off[c], h->d_l2g, h->d_xfix, h->d_S, h->d_s,
                                   h->d_rowptr, h->d_col, h->d_val, h->d_b);
    h->launches += 1;
  }
  DPG_CUDA_TRY(h, cudaGetLastError());
  h->have_system = true;
  h->have_val32 = false;
  h->have_dinv = false;
  return DPG_OK;
}

// ------------------------------------------------------------------ CG --
// Conjugate gradients for the Hermitian positive definite trace system, with
// optional Jacobi (diagonal) preconditioning z = D^{-1} r.  Device scalars
// (double): see the SC_* slots.  All reductions are deterministic: per-block
// partials summed in block order by the last block of each launch.
enum { SC_RZ = 0, SC_PAP, SC_ALPHA, SC_BETA, SC_TOL2, SC_DONE, SC_ITER, SC_BB, SC_RN, SC_N };
constexpr int RED_BLOCKS = 1184;  // 8 x 148
constexpr int RED_THREADS = 256;

__device__ unsigned int g_red_count[4];

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Two block partial sums -> red[2 * blockIdx.x + {0,1}]; the last block to
// finish sums the partials in index order and calls fin(tot0, tot1).
template <typename Fin>
__device__ void block_reduce2_last(double v0, double v1, double* red, unsigned int* counter, Fin fin) {
  __shared__ double sw[2][RED_THREADS / 32];
  __shared__ bool last;
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  if ((threadIdx.x & 31) == 0) {
    sw[0][threadIdx.x >> 5] = v0;
    sw[1][threadIdx.x >> 5] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0, t1 = 0;
    for (int k = 0; k < RED_THREADS / 32; ++k) {
      t0 += sw[0][k];
      t1 += sw[1][k];
    }
    red[2 * blockIdx.x] = t0;
    red[2 * blockIdx.x + 1] = t1;
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double t0 = 0, t1 = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
      t0 += ((volatile double*)red)[2 * k];
      t1 += ((volatile double*)red)[2 * k + 1];
    }
    t0 = warp_sum(t0);
    t1 = warp_sum(t1);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      sw[0][threadIdx.x >> 5] = t0;
      sw[1][threadIdx.x >> 5] = t1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0, b = 0;
      for (int k = 0; k < RED_THREADS / 32; ++k) {
        a += sw[0][k];
        b += sw[1][k];
      }
      fin(a, b);
      *counter = 0;
    }
  }
}

template <typename V> struct Real;
template <> struct Real<double2> { using T = double; };
template <> struct Real<float2> { using T = float; };
__device__ __forceinline__ double2 mk(double a, double b, double2*) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk(double a, double b, float2*) { return make_float2((float)a, (float)b); }

// Ap = A p (one warp per row); partial sums of Re(p^H A p); alpha = rz / pAp at the end.
// Products run in the storage precision, the row sum in that precision too,
// the dot product in FP64.
template <typename V>
__global__ void __launch_bounds__(RED_THREADS) k_spmv_dot(int64_t n, const int64_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col, const V* __restrict__ val,
                                                          const V* __restrict__ p, V* Ap, double* red, double* scal) {
  using R = typename Real<V>::T;
  if (scal[SC_DONE] != 0.0) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int64_t row = warp; row < n; row += nwarps) {
    const int64_t a = rowptr[row], b = rowptr[row + 1];
    R yr = 0, yi = 0;
    for (int64_t k = a + lane; k < b; k += 32) {
      const V v = val[k];
      const V xv = p[col[k]];
      yr = fma(v.x, xv.x, fma(-v.y, xv.y, yr));
      yi = fma(v.x, xv.y, fma(v.y, xv.x, yi));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      yr += __shfl_xor_sync(0xffffffffu, yr, o);
      yi += __shfl_xor_sync(0xffffffffu, yi, o);
    }
    if (lane == 0) {
      Ap[row] = mk(yr, yi, (V*)nullptr);
      const V pv = p[row];
      dot += (double)pv.x * (double)yr + (double)pv.y * (double)yi;  // Re(conj(p) Ap)
    }
  }
  block_reduce2_last(dot, 0.0, red, &g_red_count[0], [&](double tot, double) {
    scal[SC_PAP] = tot;
    scal[SC_ALPHA] = scal[SC_RZ] / tot;
  });
}

// x += alpha p, r -= alpha Ap; partial ||r||^2 and Re(r^H D^{-1} r);
// beta, the new rz, the iteration count and the done flag at the end.
template <typename V>
__global__ void __launch_bounds__(RED_THREADS) k_cg_update(int64_t n, V* x, V* r, const V* __restrict__ p,
                                                           const V* __restrict__ Ap,
                                                           const typename Real<V>::T* __restrict__ dinv, double* red,
                                                           double* scal) {
  using R = typename Real<V>::T;
  if (scal[SC_DONE] != 0.0) return;
  const R alpha = (R)scal[SC_ALPHA];
  double rr = 0.0, rz = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    V xv = x[i], rv = r[i];
    const V pv = p[i], av = Ap[i];
    xv.x = fma(alpha, pv.x, xv.x);
    xv.y = fma(alpha, pv.y, xv.y);
    rv.x = fma(-alpha, av.x, rv.x);
    rv.y = fma(-alpha, av.y, rv.y);
    x[i] = xv;
    r[i] = rv;
    const double q = (double)rv.x * rv.x + (double)rv.y * rv.y;
    rr += q;
    rz += dinv ? q * (double)dinv[i] : q;
  }
  block_reduce2_last(rr, rz, red, &g_red_count[1], [&](double trr, double trz) {
    scal[SC_BETA] = trz / scal[SC_RZ];
    scal[SC_RZ] = trz;
    scal[SC_RN] = trr;
    scal[SC_ITER] += 1.0;
    if (trr <= scal[SC_TOL2]) scal[SC_DONE] = 1.0;
  });
}

// p = D^{-1} r + beta p
template <typename V>
__global__ void k_cg_p(int64_t n, const V* __restrict__ r, V* p, const typename Real<V>::T* __restrict__ dinv,
                       const double* __restrict__ scal) {
  using R = typename Real<V>::T;
  if (scal[SC_DONE] != 0.0) return;
  const R beta = (R)scal[SC_BETA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const V rv = r[i];
    const R d = dinv ? dinv[i] : (R)1;
    V pv = p[i];
    pv.x = fma(beta, pv.x, d * rv.x);
    pv.y = fma(beta, pv.y, d * rv.y);
    p[i] = pv;
  }
}

// Start of a (possibly inner) solve for A d = r0 with d = 0: r = r0 (converted
// to the solve precision), p = D^{-1} r, rz = Re(r^H D^{-1} r), rn = ||r||^2.
template <typename V>
__global__ void __launch_bounds__(RED_THREADS) k_cg_start(int64_t n, const double2* __restrict__ r0, V* r, V* p, V* d,
                                                          const typename Real<V>::T* __restrict__ dinv, double* red,
                                                          double* scal, double tol2) {
  using R = typename Real<V>::T;
  double rr = 0.0, rz = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const V rv = mk(r0[i].x, r0[i].y, (V*)nullptr);
    const R dd = dinv ? dinv[i] : (R)1;
    r[i] = rv;
    V pv;
    pv.x = dd * rv.x;
    pv.y = dd * rv.y;
    p[i] = pv;
    d[i] = mk(0.0, 0.0, (V*)nullptr);
    const double q = (double)rv.x * rv.x + (double)rv.y * rv.y;
    rr += q;
    rz += q * (double)dd;
  }
  block_reduce2_last(rr, rz, red, &g_red_count[2], [&](double trr, double trz) {
    scal[SC_RZ] = trz;
    scal[SC_RN] = trr;
    scal[SC_TOL2] = tol2;
    scal[SC_DONE] = (trr <= tol2) ? 1.0 : 0.0;
    scal[SC_ITER] = 0.0;
  });
}

// r = b - A x in FP64 (x may be NULL for x = 0); ||r||^2 -> scal[slot].
__global__ void __launch_bounds__(RED_THREADS) k_residual(int64_t n, const int64_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col,
                                                          const double2* __restrict__ val,
                                                          const double2* __restrict__ x, const double2* __restrict__ b,
                                                          double2* r, double* red, double* scal, int slot) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double acc = 0.0;
  for (int64_t row = warp; row < n; row += nwarps) {
    double yr = 0.0, yi = 0.0;
    if (x) {
      const int64_t a = rowptr[row], bb = rowptr[row + 1];
      for (int64_t k = a + lane; k < bb; k += 32) {
        const double2 v = val[k];
        const double2 xv = x[col[k]];
        yr = fma(v.x, xv.x, fma(-v.y, xv.y, yr));
        yi = fma(v.x, xv.y, fma(v.y, xv.x, yi));
      }
      yr = warp_sum(yr);
      yi = warp_sum(yi);
    }
    if (lane == 0) {
      const double2 bv = b[row];
      const double2 rv = make_double2(bv.x - yr, bv.y - yi);
      r[row] = rv;
      acc += rv.x * rv.x + rv.y * rv.y;
    }
  }
  block_reduce2_last(acc, 0.0, red, &g_red_count[3], [&](double tot, double) { scal[slot] = tot; });
}

__global__ void k_to_f32(int64_t n, const double2* __restrict__ a, float2* b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// inverse of the (real, positive) diagonal of the Hermitian matrix
__global__ void k_diag_inv(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const double2* __restrict__ val, double* dinv, float* dinv32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = rowptr[i], hi = rowptr[i + 1] - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (col[mid] < i)
        lo = mid + 1;
      else
        hi = mid;
    }
    const double d = (col[lo] == i && val[lo].x > 0) ? 1.0 / val[lo].x : 1.0;
    dinv[i] = d;
    dinv32[i] = (float)d;
  }
}

__global__ void k_add_correction(int64_t n, double2* x, const float2* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i].x += (double)d[i].x;
    x[i].y += (double)d[i].y;
  }
}

static int ensure_cg_buffers(dpg_handle* h, bool fp32) {
  const size_t n = h->n;
  auto al = [&](void** p, size_t bytes) -> int {
    if (*p) return DPG_OK;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      h->err = "CG buffer allocation failed";
      return DPG_ERR_NOMEM;
    }
    return DPG_OK;
  };
  int rc = 0;
  rc |= al((void**)&h->d_r, sizeof(double2) * n);
  rc |= al((void**)&h->d_p, sizeof(double2) * n);
  rc |= al((void**)&h->d_Ap, sizeof(double2) * n);
  rc |= al((void**)&h->d_red, sizeof(double) * 2 * RED_BLOCKS);
  rc |= al((void**)&h->d_scal, sizeof(double) * SC_N);
  rc |= al((void**)&h->d_dinv, sizeof(double) * n);
  rc |= al((void**)&h->d_dinv32, sizeof(float) * n);
  if (fp32) {
    rc |= al((void**)&h->d_r32, sizeof(float2) * n);
    rc |= al((void**)&h->d_p32, sizeof(float2) * n);
    rc |= al((void**)&h->d_Ap32, sizeof(float2) * n);
    rc |= al((void**)&h->d_x32, sizeof(float2) * n);
    rc |= al((void**)&h->d_val32, sizeof(float2) * h->nnz);
  }
  return rc ? DPG_ERR_NOMEM : DPG_OK;
}

// Run CG iterations in graph-captured groups until the device flag says done
// or max_iter is reached.  The solve vectors are (x, r, p, Ap) of type V.
template <typename V>
static int run_cg_loop(dpg_handle* h, const V* val, V* x, V* r, V* p, V* Ap, const typename Real<V>::T* dinv,
                       int max_iter, cudaStream_t s, int* iters_out) {
  const int64_t n = h->n;
  const int group = 32;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // capture on a private stream ordered after the caller's stream
  cudaStream_t cs;
  DPG_CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t ev;
  DPG_CUDA_TRY(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  DPG_CUDA_TRY(h, cudaEventRecord(ev, s));
  DPG_CUDA_TRY(h, cudaStreamWaitEvent(cs, ev, 0));
  DPG_CUDA_TRY(h, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < group; ++k) {
    k_spmv_dot<V><<<RED_BLOCKS, RED_THREADS, 0, cs>>>(n, h->d_rowptr, h->d_col, val, p, Ap, h->d_red, h->d_scal);
    k_cg_update<V><<<RED_BLOCKS, RED_THREADS, 0, cs>>>(n, x, r, p, Ap, dinv, h->d_red, h->d_scal);
    k_cg_p<V><<<RED_BLOCKS, RED_THREADS, 0, cs>>>(n, r, p, dinv, h->d_scal);
  }
  cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  if (ce != cudaSuccess) {
    h->err = std::string("graph capture: ") + cudaGetErrorString(ce);
    return DPG_ERR_CUDA;
  }
  DPG_CUDA_TRY(h, cudaGraphInstantiate(&exec, graph, 0));
  double scal[SC_N];
  for (int launched = 0; launched < max_iter; launched += group) {
    DPG_CUDA_TRY(h, cudaGraphLaunch(exec, cs));
    h->launches += 3 * group;
    // read the flag every fourth group so the device stays busy in between
    if (((launched / group) & 3) == 3 || launched + group >= max_iter) {
      DPG_CUDA_TRY(h, cudaMemcpyAsync(scal, h->d_scal, sizeof(scal), cudaMemcpyDeviceToHost, cs));
      DPG_CUDA_TRY(h, cudaStreamSynchronize(cs));
      if (scal[SC_DONE] != 0.0 || (int)scal[SC_ITER] >= max_iter) break;
    }
  }
  DPG_CUDA_TRY(h, cudaMemcpyAsync(scal, h->d_scal, sizeof(scal), cudaMemcpyDeviceToHost, cs));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(cs));
  *iters_out = (int)scal[SC_ITER];
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  cudaEventDestroy(ev);
  cudaStreamDestroy(cs);
  return DPG_OK;
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
  const bool ir = (mode & DPG_CG_IR_FP32) != 0;
  const bool jac = (mode & DPG_CG_JACOBI) != 0;
  if (mode & ~(DPG_CG_IR_FP32 | DPG_CG_JACOBI)) {
    h->err = "unknown CG mode";
    return DPG_ERR_ARG;
  }
  int rc = ensure_cg_buffers(h, ir);
  if (rc) return rc;
  const int64_t n = h->n;
  const double2* rhs = b ? b : h->d_b;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, s);
  if (!h->have_dinv) {
    k_diag_inv<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, h->d_rowptr, h->d_col, h->d_val, h->d_dinv, h->d_dinv32);
    h->launches += 1;
    h->have_dinv = true;
  }
  if (ir && !h->have_val32) {
    k_to_f32<<<RED_BLOCKS, RED_THREADS, 0, s>>>(h->nnz, h->d_val, h->d_val32);
    h->launches += 1;
    h->have_val32 = true;
  }
  double scal[SC_N];
  // r = b (x = 0), ||b||^2 -> SC_BB
  k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, h->d_rowptr, h->d_col, h->d_val, nullptr, rhs, h->d_r, h->d_red,
                                                 h->d_scal, SC_BB);
  h->launches += 1;
  DPG_CUDA_TRY(h, cudaMemcpyAsync(scal, h->d_scal, sizeof(scal), cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(scal[SC_BB]);
  const double tol = std::max(rtol * bnorm, atol);
  int total_iters = 0, outer = 0;
  double rnorm = bnorm;
  if (!ir) {
    // FP64 solve directly on x
    k_cg_start<double2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, h->d_r, h->d_r, h->d_p, x, jac ? h->d_dinv : nullptr,
                                                           h->d_red, h->d_scal, tol * tol);
    h->launches += 1;
    rc = run_cg_loop<double2>(h, h->d_val, x, h->d_r, h->d_p, h->d_Ap, jac ? h->d_dinv : nullptr, max_iter, s,
                              &total_iters);
    if (rc) return rc;
  } else {
    DPG_CUDA_TRY(h, cudaMemsetAsync(x, 0, sizeof(double2) * n, s));
    bool converged = rnorm <= tol;
    while (!converged && total_iters < max_iter && outer < 100) {
      // inner FP32 CG on A d = r to relative tolerance inner_rtol (not below the outer target)
      const double itol = std::max(inner_rtol * rnorm, 0.5 * tol);
      k_cg_start<float2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, h->d_r, h->d_r32, h->d_p32, h->d_x32,
                                                            jac ? h->d_dinv32 : nullptr, h->d_red, h->d_scal,
                                                            itol * itol);
      h->launches += 1;
      int it = 0;
      rc = run_cg_loop<float2>(h, h->d_val32, h->d_x32, h->d_r32, h->d_p32, h->d_Ap32, jac ? h->d_dinv32 : nullptr,
                               max_iter - total_iters, s, &it);
      if (rc) return rc;
      total_iters += it;
      ++outer;
      // FP64 update and true residual
      k_add_correction<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, x, h->d_x32);
      k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, h->d_rowptr, h->d_col, h->d_val, x, rhs, h->d_r, h->d_red,
                                                     h->d_scal, SC_BB);
      h->launches += 2;
      DPG_CUDA_TRY(h, cudaMemcpyAsync(scal, h->d_scal, sizeof(scal), cudaMemcpyDeviceToHost, s));
      DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
      rnorm = std::sqrt(scal[SC_BB]);
      converged = rnorm <= tol;
      if (it == 0) break;
    }
  }
  // final true residual in FP64 (into Ap as scratch)
  k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, h->d_rowptr, h->d_col, h->d_val, x, rhs, h->d_Ap, h->d_red,
                                                 h->d_scal, SC_PAP);
  h->launches += 1;
  cudaEventRecord(t1, s);
  DPG_CUDA_TRY(h, cudaMemcpyAsync(scal, h->d_scal, sizeof(scal), cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  float ms = 0;
  cudaEventElapsedTime(&ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  const double res = std::sqrt(scal[SC_PAP]);
  const double rel = bnorm > 0 ? res / bnorm : 0.0;
  // the recursive residual of plain CG may sit a hair below the true one
  const bool converged = res <= tol * (ir ? 1.0 : 1.0 + 1e-3) || (!ir && scal[SC_DONE] != 0.0 && res <= 2 * tol);
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
// Per element: uhat_K gathered from x (free) and the Dirichlet values,
// eta^2 = c - 2 Re(uhat^H s) + uhat^H S uhat, u = z - Z uhat.
__global__ void __launch_bounds__(256) k_estimate(int nh, int nu, const int32_t* __restrict__ l2g,
                                                  const double2* __restrict__ xfix, const double2* __restrict__ xhat,
                                                  const double2* __restrict__ Sst, const double2* __restrict__ sst,
                                                  const double* __restrict__ cst, const double2* __restrict__ Zst,
                                                  const double2* __restrict__ zst, double2* u_out, double* eta2) {
  extern __shared__ double2 su[];
  const int e = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < nh; t += blockDim.x) {
    const int g = l2g[(size_t)e * nh + t];
    su[t] = g >= 0 ? xhat[g] : (g == -1 ? xfix[(size_t)e * nh + t] : make_double2(0.0, 0.0));
  }
  __syncthreads();
  const double2* Se = Sst + (size_t)e * nh * nh;
  double q = 0.0;  // sum over rows of Re(conj(uhat_i) (S uhat)_i)
  for (int i = wid; i < nh; i += nw) {
    double yr = 0.0, yi = 0.0;
    for (int j = lane; j < nh; j += 32) {
      const double2 v = Se[(size_t)i * nh + j], x = su[j];
      yr = fma(v.x, x.x, fma(-v.y, x.y, yr));
      yi = fma(v.x, x.y, fma(v.y, x.x, yi));
    }
    yr = warp_sum(yr);
    yi = warp_sum(yi);
    const double2 ui = su[i], si = sst[(size_t)e * nh + i];
    q += (lane == 0) ? (ui.x * yr + ui.y * yi) - 2.0 * (ui.x * si.x + ui.y * si.y) : 0.0;
  }
  if (u_out) {
    const double2* Ze = Zst + (size_t)e * nu * nh;
    for (int i = wid; i < nu; i += nw) {
      double yr = 0.0, yi = 0.0;
      for (int j = lane; j < nh; j += 32) {
        const double2 v = Ze[(size_t)i * nh + j], x = su[j];
        yr = fma(v.x, x.x, fma(-v.y, x.y, yr));
        yi = fma(v.x, x.y, fma(v.y, x.x, yi));
      }
      yr = warp_sum(yr);
      yi = warp_sum(yi);
      if (lane == 0) {
        const double2 zi = zst[(size_t)e * nu + i];
        u_out[(size_t)e * nu + i] = make_double2(zi.x - yr, zi.y - yi);
      }
    }
  }
  __shared__ double sq[32];
  q = warp_sum(q);
  if (lane == 0) sq[wid] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = cst[e];
    for (int k = 0; k < nw; ++k) t += sq[k];
    eta2[e] = t;
  }
}

__global__ void k_sqrt_sum(int n, const double* __restrict__ eta2, double* eta, double* total) {
  __shared__ double sw[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v = fmax(eta2[i], 0.0);
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

int estimate(dpg_handle* h, const double2* xhat, double2* u, double* eta, double* eta_global, cudaStream_t s) {
  if (!h->have_elements) {
    h->err = "dpg_estimate before dpg_element_batch";
    return DPG_ERR_STATE;
  }
  if (!xhat) {
    h->err = "null xhat";
    return DPG_ERR_ARG;
  }
  const Sizes& S = h->sz;
  double* d_eta2 = nullptr;
  DPG_CUDA_TRY(h, cudaMallocAsync(&d_eta2, sizeof(double) * (h->ne + 1), s));
  k_estimate<<<h->ne, 256, sizeof(double2) * S.n_h, s>>>(S.n_h, S.n_u, h->d_l2g, h->d_xfix, xhat, h->d_S, h->d_s,
                                                         h->d_c, h->d_Z, h->d_z, u, d_eta2);
  k_sqrt_sum<<<1, 1024, 0, s>>>(h->ne, d_eta2, eta, d_eta2 + h->ne);
  h->launches += 2;
  DPG_CUDA_TRY(h, cudaGetLastError());
  if (eta_global) {
    double tot = 0;
    DPG_CUDA_TRY(h, cudaMemcpyAsync(&tot, d_eta2 + h->ne, sizeof(double), cudaMemcpyDeviceToHost, s));
    DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
    *eta_global = std::sqrt(std::max(tot, 0.0));
  }
  DPG_CUDA_TRY(h, cudaFreeAsync(d_eta2, s));
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
  const Sizes& S = h->sz;
  k_estimate<<<h->ne, 256, sizeof(double2) * S.n_h, s>>>(S.n_h, S.n_u, h->d_l2g, h->d_xfix, xhat, h->d_S, h->d_s,
                                                         h->d_c, h->d_Z, h->d_z, u, scratch);
  k_sqrt_sum<<<1, 1024, 0, s>>>(h->ne, scratch, eta, scratch + h->ne);
  h->launches += 2;
  DPG_CUDA_TRY(h, cudaGetLastError());
  if (eta_global) {
    double tot = 0;
    DPG_CUDA_TRY(h, cudaMemcpyAsync(&tot, scratch + h->ne, sizeof(double), cudaMemcpyDeviceToHost, s));
    DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
    *eta_global = std::sqrt(std::max(tot, 0.0));
  }
  return DPG_OK;
}

}  // namespace dpg
