// Assembly (DistributeLocalToGlobal of Algorithm 2), conjugate gradients on the
// condensed trace system (Sec. 2.3 end), and local recovery with the residual
// estimator (Sec. 2.3).  complex FP64 unless stated.
#include <cmath>
#include <cstring>

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
  }
  DPG_CUDA_TRY(h, cudaGetLastError());
  h->have_system = true;
  h->have_val32 = false;
  return DPG_OK;
}

// ------------------------------------------------------------------ CG --
// Device scalars (double): [0] rr, [1] pAp, [2] alpha, [3] beta, [4] tol^2,
// [5] done flag, [6] iterations, [7] rr of b.
enum { SC_RR = 0, SC_PAP, SC_ALPHA, SC_BETA, SC_TOL2, SC_DONE, SC_ITER, SC_BB, SC_N };
constexpr int RED_BLOCKS = 1184;  // 8 x 148
constexpr int RED_THREADS = 256;

__device__ unsigned int g_red_count[4];

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block partial -> red[blockIdx.x]; the last block to finish sums the partials
// in index order (deterministic) and calls fin(total) on thread 0.
template <typename Fin>
__device__ void block_reduce_last(double v, double* red, unsigned int* counter, Fin fin) {
  __shared__ double sw[RED_THREADS / 32];
  __shared__ bool last;
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < RED_THREADS / 32; ++k) t += sw[k];
    red[blockIdx.x] = t;
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double t = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) t += ((volatile double*)red)[k];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0;
      for (int k = 0; k < RED_THREADS / 32; ++k) tot += sw[k];
      fin(tot);
      *counter = 0;
    }
  }
}

// Ap = A p (warp per row) and the partial sums of Re(p^H A p); alpha at the end.
__global__ void __launch_bounds__(RED_THREADS) k_spmv_dot(int64_t n, const int64_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col,
                                                          const double2* __restrict__ val,
                                                          const double2* __restrict__ p, double2* Ap, double* red,
                                                          double* scal) {
  if (scal[SC_DONE] != 0.0) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int64_t row = warp; row < n; row += nwarps) {
    const int64_t a = rowptr[row], b = rowptr[row + 1];
    double yr = 0.0, yi = 0.0;
    for (int64_t k = a + lane; k < b; k += 32) {
      const double2 v = val[k];
      const double2 xv = p[col[k]];
      yr = fma(v.x, xv.x, fma(-v.y, xv.y, yr));
      yi = fma(v.x, xv.y, fma(v.y, xv.x, yi));
    }
    yr = warp_sum(yr);
    yi = warp_sum(yi);
    if (lane == 0) {
      Ap[row] = make_double2(yr, yi);
      const double2 pv = p[row];
      dot += pv.x * yr + pv.y * yi;  // Re(conj(p) Ap)
    }
  }
  block_reduce_last(dot, red, &g_red_count[0], [&](double tot) {
    scal[SC_PAP] = tot;
    scal[SC_ALPHA] = scal[SC_RR] / tot;
  });
}

// x += alpha p, r -= alpha Ap, partial r^H r; beta, done flag and counter at the end.
__global__ void __launch_bounds__(RED_THREADS) k_cg_update(int64_t n, double2* x, double2* r, const double2* __restrict__ p,
                                                           const double2* __restrict__ Ap, double* red, double* scal) {
  if (scal[SC_DONE] != 0.0) return;
  const double alpha = scal[SC_ALPHA];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 xv = x[i], rv = r[i];
    const double2 pv = p[i], av = Ap[i];
    xv.x = fma(alpha, pv.x, xv.x);
    xv.y = fma(alpha, pv.y, xv.y);
    rv.x = fma(-alpha, av.x, rv.x);
    rv.y = fma(-alpha, av.y, rv.y);
    x[i] = xv;
    r[i] = rv;
    acc += rv.x * rv.x + rv.y * rv.y;
  }
  block_reduce_last(acc, red, &g_red_count[1], [&](double tot) {
    scal[SC_BETA] = tot / scal[SC_RR];
    scal[SC_RR] = tot;
    scal[SC_ITER] += 1.0;
    if (tot <= scal[SC_TOL2]) scal[SC_DONE] = 1.0;
  });
}

__global__ void k_cg_p(int64_t n, const double2* __restrict__ r, double2* p, const double* __restrict__ scal) {
  if (scal[SC_DONE] != 0.0) return;
  const double beta = scal[SC_BETA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 rv = r[i];
    double2 pv = p[i];
    pv.x = fma(beta, pv.x, rv.x);
    pv.y = fma(beta, pv.y, rv.y);
    p[i] = pv;
  }
}

// r = b - A x (FP64), partial ||r||^2 -> scal[SC_RR]; also copies r to p when setp.
__global__ void __launch_bounds__(RED_THREADS) k_residual(int64_t n, const int64_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col,
                                                          const double2* __restrict__ val,
                                                          const double2* __restrict__ x, const double2* __restrict__ b,
                                                          double2* r, double2* p, int use_x, double* red, double* scal,
                                                          int slot) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double acc = 0.0;
  for (int64_t row = warp; row < n; row += nwarps) {
    double yr = 0.0, yi = 0.0;
    if (use_x) {
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
      if (p) p[row] = rv;
      acc += rv.x * rv.x + rv.y * rv.y;
    }
  }
  block_reduce_last(acc, red, &g_red_count[2], [&](double tot) { scal[slot] = tot; });
}

__global__ void k_set_scalars(double* scal, double tol2) {
  scal[SC_TOL2] = tol2;
  scal[SC_DONE] = 0.0;
  scal[SC_ITER] = 0.0;
}

// ---------------------------------------------------- FP32 inner solve --
// Same recurrences in FP32 storage with FP32 products and FP64 reductions.
__global__ void k_to_f32(int64_t n, const double2* __restrict__ a, float2* b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void __launch_bounds__(RED_THREADS) k_spmv_dot32(int64_t n, const int64_t* __restrict__ rowptr,
                                                            const int32_t* __restrict__ col,
                                                            const float2* __restrict__ val,
                                                            const float2* __restrict__ p, float2* Ap, double* red,
                                                            double* scal) {
  if (scal[SC_DONE] != 0.0) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int64_t row = warp; row < n; row += nwarps) {
    const int64_t a = rowptr[row], b = rowptr[row + 1];
    float yr = 0.f, yi = 0.f;
    for (int64_t k = a + lane; k < b; k += 32) {
      const float2 v = val[k];
      const float2 xv = p[col[k]];
      yr = fmaf(v.x, xv.x, fmaf(-v.y, xv.y, yr));
      yi = fmaf(v.x, xv.y, fmaf(v.y, xv.x, yi));
    }
    double dr = warp_sum((double)yr), di = warp_sum((double)yi);
    if (lane == 0) {
      Ap[row] = make_float2((float)dr, (float)di);
      const float2 pv = p[row];
      dot += (double)pv.x * dr + (double)pv.y * di;
    }
  }
  block_reduce_last(dot, red, &g_red_count[0], [&](double tot) {
    scal[SC_PAP] = tot;
    scal[SC_ALPHA] = scal[SC_RR] / tot;
  });
}

__global__ void __launch_bounds__(RED_THREADS) k_cg_update32(int64_t n, float2* x, float2* r, const float2* __restrict__ p,
                                                             const float2* __restrict__ Ap, double* red, double* scal) {
  if (scal[SC_DONE] != 0.0) return;
  const float alpha = (float)scal[SC_ALPHA];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float2 xv = x[i], rv = r[i];
    const float2 pv = p[i], av = Ap[i];
    xv.x = fmaf(alpha, pv.x, xv.x);
    xv.y = fmaf(alpha, pv.y, xv.y);
    rv.x = fmaf(-alpha, av.x, rv.x);
    rv.y = fmaf(-alpha, av.y, rv.y);
    x[i] = xv;
    r[i] = rv;
    acc += (double)rv.x * rv.x + (double)rv.y * rv.y;
  }
  block_reduce_last(acc, red, &g_red_count[1], [&](double tot) {
    scal[SC_BETA] = tot / scal[SC_RR];
    scal[SC_RR] = tot;
    scal[SC_ITER] += 1.0;
    if (tot <= scal[SC_TOL2]) scal[SC_DONE] = 1.0;
  });
}

__global__ void k_cg_p32(int64_t n, const float2* __restrict__ r, float2* p, const double* __restrict__ scal) {
  if (scal[SC_DONE] != 0.0) return;
  const float beta = (float)scal[SC_BETA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 rv = r[i];
    float2 pv = p[i];
    pv.x = fmaf(beta, pv.x, rv.x);
    pv.y = fmaf(beta, pv.y, rv.y);
    p[i] = pv;
  }
}

// r32 = r / ||r|| scaling is not needed: the inner system is solved for the
// correction d with A d = r (r in FP32), starting at d = 0.
__global__ void k_inner_start(int64_t n, const double2* __restrict__ r, float2* r32, float2* p32, float2* x32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float2 v = make_float2((float)r[i].x, (float)r[i].y);
    r32[i] = v;
    p32[i] = v;
    x32[i] = make_float2(0.f, 0.f);
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
  rc |= al((void**)&h->d_red, sizeof(double) * RED_BLOCKS);
  rc |= al((void**)&h->d_scal, sizeof(double) * SC_N);
  if (fp32) {
    rc |= al((void**)&h->d_r32, sizeof(float2) * n);
    rc |= al((void**)&h->d_p32, sizeof(float2) * n);
    rc |= al((void**)&h->d_Ap32, sizeof(float2) * n);
    rc |= al((void**)&h->d_x32, sizeof(float2) * n);
    rc |= al((void**)&h->d_val32, sizeof(float2) * h->nnz);
  }
  return rc ? DPG_ERR_NOMEM : DPG_OK;
}

// Run CG iterations in graph-captured groups of `group` until the device flag
// says done or max_iter is reached.  Returns the iteration count.
static int run_cg_loop(dpg_handle* h, bool fp32, int max_iter, cudaStream_t s, int* iters_out) {
  const int64_t n = h->n;
  const int group = 32;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // capture on a private stream so the caller's legacy stream can be used too
  cudaStream_t cs;
  DPG_CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t ev;
  DPG_CUDA_TRY(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  DPG_CUDA_TRY(h, cudaEventRecord(ev, s));
  DPG_CUDA_TRY(h, cudaStreamWaitEvent(cs, ev, 0));
  DPG_CUDA_TRY(h, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const int vb = RED_BLOCKS;
  for (int k = 0; k < group; ++k) {
    if (!fp32) {
      k_spmv_dot<<<RED_BLOCKS, RED_THREADS, 0, cs>>>(n, h->d_rowptr, h->d_col, h->d_val, h->d_p, h->d_Ap, h->d_red,
                                                      h->d_scal);
      k_cg_update<<<vb, RED_THREADS, 0, cs>>>(n, h->d_xw, h->d_r, h->d_p, h->d_Ap, h->d_red, h->d_scal);
      k_cg_p<<<vb, RED_THREADS, 0, cs>>>(n, h->d_r, h->d_p, h->d_scal);
    } else {
      k_spmv_dot32<<<RED_BLOCKS, RED_THREADS, 0, cs>>>(n, h->d_rowptr, h->d_col, h->d_val32, h->d_p32, h->d_Ap32,
                                                        h->d_red, h->d_scal);
      k_cg_update32<<<vb, RED_THREADS, 0, cs>>>(n, h->d_x32, h->d_r32, h->d_p32, h->d_Ap32, h->d_red, h->d_scal);
      k_cg_p32<<<vb, RED_THREADS, 0, cs>>>(n, h->d_r32, h->d_p32, h->d_scal);
    }
  }
  cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  if (ce != cudaSuccess) {
    h->err = std::string("graph capture: ") + cudaGetErrorString(ce);
    return DPG_ERR_CUDA;
  }
  DPG_CUDA_TRY(h, cudaGraphInstantiate(&exec, graph, 0));
  double scal[SC_N];
  int done_iters = 0;
  for (int launched = 0; launched < max_iter; launched += group) {
    DPG_CUDA_TRY(h, cudaGraphLaunch(exec, cs));
    // check every few groups to keep the device busy between host reads
    if (((launched / group) & 3) == 3 || launched + group >= max_iter) {
      DPG_CUDA_TRY(h, cudaMemcpyAsync(scal, h->d_scal, sizeof(scal), cudaMemcpyDeviceToHost, cs));
      DPG_CUDA_TRY(h, cudaStreamSynchronize(cs));
      done_iters = (int)scal[SC_ITER];
      if (scal[SC_DONE] != 0.0 || done_iters >= max_iter) break;
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
  const bool ir = (mode == DPG_CG_IR_FP32);
  if (mode != DPG_CG_FP64 && !ir) {
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
  DPG_CUDA_TRY(h, cudaMemsetAsync(x, 0, sizeof(double2) * n, s));
  h->d_xw = x;
  double scal[SC_N];
  // ||b||^2 into SC_BB (r = b, x = 0)
  k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, h->d_rowptr, h->d_col, h->d_val, x, rhs, h->d_r, h->d_p, 0,
                                                 h->d_red, h->d_scal, SC_BB);
  DPG_CUDA_TRY(h, cudaMemcpyAsync(scal, h->d_scal, sizeof(scal), cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(scal[SC_BB]);
  const double tol = std::max(rtol * bnorm, atol);
  int total_iters = 0, outer = 0;
  double rnorm = bnorm;
  bool converged = rnorm <= tol;
  if (!ir) {
    if (!converged) {
      // rr = ||b||^2
      k_set_scalars<<<1, 1, 0, s>>>(h->d_scal, tol * tol);
      DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_scal + SC_RR, h->d_scal + SC_BB, sizeof(double), cudaMemcpyDeviceToDevice, s));
      rc = run_cg_loop(h, false, max_iter, s, &total_iters);
      if (rc) return rc;
    }
  } else {
    if (!h->have_val32) {
      k_to_f32<<<RED_BLOCKS, RED_THREADS, 0, s>>>(h->nnz, h->d_val, h->d_val32);
      h->have_val32 = true;
    }
    // residual r = b (x = 0) already in d_r
    while (!converged && total_iters < max_iter && outer < 100) {
      // inner FP32 CG on A d = r to relative tolerance inner_rtol
      k_inner_start<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, h->d_r, h->d_r32, h->d_p32, h->d_x32);
      const double rr0 = rnorm * rnorm;
      const double itol = std::max(inner_rtol * rnorm, 0.5 * tol);
      k_set_scalars<<<1, 1, 0, s>>>(h->d_scal, itol * itol);
      DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_scal + SC_RR, &rr0, sizeof(double), cudaMemcpyHostToDevice, s));
      int it = 0;
      rc = run_cg_loop(h, true, max_iter - total_iters, s, &it);
      if (rc) return rc;
      total_iters += it;
      ++outer;
      k_add_correction<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, x, h->d_x32);
      k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, h->d_rowptr, h->d_col, h->d_val, x, rhs, h->d_r, nullptr, 1,
                                                     h->d_red, h->d_scal, SC_BB + 0);
      DPG_CUDA_TRY(h, cudaMemcpyAsync(scal, h->d_scal, sizeof(scal), cudaMemcpyDeviceToHost, s));
      DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
      rnorm = std::sqrt(scal[SC_BB]);
      converged = rnorm <= tol;
      if (it == 0) break;
    }
  }
  // final true residual in FP64
  k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, h->d_rowptr, h->d_col, h->d_val, x, rhs, h->d_Ap, nullptr, 1,
                                                 h->d_red, h->d_scal, SC_PAP);
  cudaEventRecord(t1, s);
  DPG_CUDA_TRY(h, cudaMemcpyAsync(scal, h->d_scal, sizeof(scal), cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  float ms = 0;
  cudaEventElapsedTime(&ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  const double rel = bnorm > 0 ? std::sqrt(scal[SC_PAP]) / bnorm : 0.0;
  converged = std::sqrt(scal[SC_PAP]) <= tol * (ir ? 1.0 : 1.0 + 1e-6) || (!ir && scal[SC_DONE] != 0.0);
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

}  // namespace dpg
