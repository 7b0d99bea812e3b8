// extern "C" entry points of libdpg (declared in include/dpg.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "dpg_internal.h"

using namespace dpg;

// NVTX range around each entry point (visible to nsys / ncu range filters;
// free when no tool is attached).
namespace {
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};
}  // namespace

static cudaStream_t S_(dpg_stream s) { return reinterpret_cast<cudaStream_t>(s); }
static thread_local std::string g_setup_err;

static void free_all(dpg_handle* h) {
  free_plan(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  h->cap_stream = nullptr;
  for (Group& G : h->grp) {
    void* gb[] = {G.d_Xref, G.d_Tf, G.d_Tall, G.d_trfun, G.d_elems, G.d_color_elems};
    for (void* b : gb)
      if (b) cudaFree(b);
  }
  void* bufs[] = {h->d_X,     h->d_eps,   h->d_mu,   h->d_fbc,   h->d_off,   h->d_sig,  h->d_rsig,
                  h->d_rint,  h->d_l2g,   h->d_xfix, h->d_rdbl,  h->d_robin, h->d_status, h->d_S,
                  h->d_s,     h->d_c,     h->d_Z,    h->d_z,     h->d_rowptr, h->d_row2blk, h->d_val,
                  h->d_b,     h->d_val32, h->d_r,    h->d_p,     h->d_Ap,    h->d_r32,  h->d_p32,
                  h->d_Ap32,  h->d_x32,   h->d_red,  h->d_cgstate,  h->ws.K,    h->ws.V,   h->ws.Cu,
                  h->ws.PhiL, h->ws.MC,   h->ws.ids, h->ws.FV,   h->ws.FR,   h->ws.rent, h->ws.WQ,
                  h->d_dinv,  h->d_dinv32, h->d_L1, h->d_u, h->d_zg, h->d_gc, h->d_lam, h->d_rhs_adj,
                  h->d_Pk, h->d_blk, h->d_blk_colptr, h->d_cols, h->d_binv_ptr, h->d_binv, h->d_binv32,
                  h->d_zv, h->d_z32, h->d_d64, h->ws.Q, h->d_est_neg,
                  h->d_rowptr_h, h->d_toff, h->d_rev_ptr, h->d_rev_off, h->d_val32h, h->d_T,
                  h->d_valdw, h->d_pdw, h->d_binvdw, h->d_ebe, h->d_ebe_toff, h->d_ebe_hoff, h->d_ebe_rptr,
                  h->d_ebe_ridx, h->d_ebe_ys, h->d_Xst, h->d_xst_off};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (h->d_soff && h->d_soff != h->d_off) cudaFree(h->d_soff);
}

extern "C" int dpg_setup_mesh(dpg_handle** out, const dpg_mesh_desc* m, const dpg_params* prm, dpg_stream st) {
  Range range_("dpg_setup_mesh");
  if (!out) return DPG_ERR_ARG;
  *out = nullptr;
  dpg_handle* h = new (std::nothrow) dpg_handle();
  if (!h) return DPG_ERR_NOMEM;
  cudaStream_t s = S_(st);
  int rc = build_mesh(h, m, prm, s);
  if (rc == DPG_OK) {
    set_default_caps(h, prm->chunk);
    rc = alloc_workspace(h);
  }
  if (rc == DPG_OK) rc = init_kernel_attributes(h);
  for (int g = 0; rc == DPG_OK && g < (int)h->grp.size(); ++g) rc = compute_reference_matrices(h, g, s);
  if (rc != DPG_OK) {
    // keep the message on a static buffer for dpg_last_error(NULL)
    free_all(h);
    g_setup_err = h->err;
    delete h;
    return rc;
  }
  *out = h;
  return DPG_OK;
}

extern "C" int dpg_element_batch(dpg_handle* h, int32_t pass, dpg_stream st) {
  Range range_("dpg_element_batch");
  if (!h) return DPG_ERR_ARG;
  if (pass != DPG_PASS_ASSEMBLE) {
    h->err = "unknown element pass";
    return DPG_ERR_ARG;
  }
  cudaStream_t s = S_(st);
  h->have_elements = false;
  h->have_system = false;
  // per-element pivot flags and the tensor-core timeout flag start clear on
  // every pass, so one failed pass does not poison the next
  DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int) * (h->ne + 1), s));
  // the launch plan of every order group (lossless elements in real
  // arithmetic, the others in complex arithmetic), replayed as a CUDA graph
  int rc = element_pass(h, s);
  if (rc) return rc;
  // pivot check
  std::vector<int> status(h->ne);
  DPG_CUDA_TRY(h, cudaMemcpyAsync(status.data(), h->d_status, sizeof(int) * h->ne, cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  if (h->timing && h->bucketed && h->factor_arith == DPG_FACTOR_TC_SPLIT) {
    for (const WavePlan& wp : h->waves) {  // one persistent launch per wave
      float ms = 0;
      DPG_CUDA_TRY(h, cudaEventElapsedTime(&ms, wp.ev0, wp.ev1));
      h->factor_ms += ms;
      h->factor_launches += (wp.nitems > wp.nitems_real) + (wp.nitems_real > 0);
      h->factor_elements += wp.nitems;
      h->factor_elements_real += wp.nitems_real;
    }
  } else if (h->timing) {
    for (const ChunkPlan& cp : h->plan) {
      float ms = 0;
      DPG_CUDA_TRY(h, cudaEventElapsedTime(&ms, cp.ev0, cp.ev1));
      h->factor_ms += ms;
      h->factor_launches += 1;
      h->factor_elements += cp.count;
      if (cp.real) {
        h->factor_ms_real += ms;
        h->factor_elements_real += cp.count;
      }
    }
  }
  for (int e = 0; e < h->ne; ++e)
    if (status[e]) {
      h->err = "non-positive pivot in element " + std::to_string(e);
      return DPG_ERR_NOT_HPD;
    }
  {
    int terr = 0;
    DPG_CUDA_TRY(h, cudaMemcpy(&terr, h->d_status + h->ne, sizeof(int), cudaMemcpyDeviceToHost));
    if (terr) {
      h->err = "a tensor-core kernel of the element pass gave up waiting for its MMAs";
      return DPG_ERR_TIMEOUT;
    }
  }
  // only a pass whose every pivot was positive feeds assembly and estimation
  h->have_elements = true;
  h->xst_valid = h->d_Xst != nullptr && !h->stream;
  if (h->stream) system_changed(h);  // assembled during the pass
  return DPG_OK;
}

extern "C" int dpg_assemble(dpg_handle* h, dpg_stream st) {
  Range range_("dpg_assemble");
  if (!h) return DPG_ERR_ARG;
  if (!h->have_elements) {
    h->err = "dpg_assemble before dpg_element_batch";
    return DPG_ERR_STATE;
  }
  return assemble_system(h, S_(st));
}

extern "C" int dpg_cg_solve(dpg_handle* h, int32_t mode, double rtol, double atol, int32_t max_iter,
                            double inner_rtol, dpg_complex* x, const dpg_complex* b, dpg_cg_report* rep,
                            dpg_stream st) {
  Range range_("dpg_cg_solve");
  if (!h) return DPG_ERR_ARG;
  return cg_solve(h, mode, rtol, atol, max_iter, inner_rtol, reinterpret_cast<double2*>(x),
                  reinterpret_cast<const double2*>(b), rep, S_(st));
}

extern "C" int dpg_estimate(dpg_handle* h, const dpg_complex* xhat, dpg_complex* u, double* eta, double* eta_global,
                            dpg_stream st) {
  Range range_("dpg_estimate");
  if (!h) return DPG_ERR_ARG;
  return estimate(h, reinterpret_cast<const double2*>(xhat), reinterpret_cast<double2*>(u), eta, eta_global, S_(st));
}

// Fixed-fraction marking of Sec. 4.2 (host logic after one copy of eta).
extern "C" int dpg_mark_fraction(dpg_handle* h, const double* eta, double refine_frac, double coarsen_frac,
                                 int32_t power, int8_t* marks, dpg_stream st) {
  Range range_("dpg_mark_fraction");
  if (!h || !eta || !marks || !(refine_frac >= 0.0 && refine_frac <= 1.0) ||
      !(coarsen_frac >= 0.0 && coarsen_frac <= 1.0) || (power != 1 && power != 2))
    return DPG_ERR_ARG;
  const int ne = h->ne;
  std::vector<double> e2(ne);
  cudaStream_t s = S_(st);
  DPG_CUDA_TRY(h, cudaMemcpyAsync(e2.data(), eta, sizeof(double) * ne, cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  double total = 0.0;
  for (int e = 0; e < ne; ++e) {
    e2[e] = power == 2 ? e2[e] * e2[e] : std::fabs(e2[e]);
    total += e2[e];
  }
  std::memset(marks, 0, (size_t)ne);
  if (ne == 0 || !(total > 0.0)) return DPG_OK;
  std::vector<int> order(ne);
  for (int e = 0; e < ne; ++e) order[e] = e;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return e2[a] > e2[b] || (e2[a] == e2[b] && a < b); });
  double acc = 0.0;
  for (int k = 0; k < ne && acc < refine_frac * total; ++k) {  // largest first, up to the crossing cell
    marks[order[k]] = 1;
    acc += e2[order[k]];
  }
  acc = 0.0;
  for (int k = ne - 1; k >= 0; --k) {  // smallest first, within the coarsening share
    const int e = order[k];
    if (marks[e] == 1 || acc + e2[e] > coarsen_frac * total) break;
    marks[e] = -1;
    acc += e2[e];
  }
  return DPG_OK;
}

extern "C" int dpg_estimate_clamped(dpg_handle* h, int32_t* count) {
  if (!h || !count) return DPG_ERR_ARG;
  int c = 0;
  int rc = estimate_negatives(h, &c);
  *count = c;
  return rc;
}

extern "C" int dpg_estimate_noalloc(dpg_handle* h, const dpg_complex* xhat, dpg_complex* u, double* eta,
                                    double* eta_global, dpg_stream st) {
  Range range_("dpg_estimate_noalloc");
  if (!h) return DPG_ERR_ARG;
  return estimate_noalloc(h, reinterpret_cast<const double2*>(xhat), reinterpret_cast<double2*>(u), eta, eta_global,
                          S_(st));
}

extern "C" int dpg_grad_eps(dpg_handle* h, const dpg_complex* xhat, const uint8_t* obstacle_mask, double* P,
                            double* dP_deps_re, double* dP_deps_im, int32_t cg_mode, double cg_rtol, int32_t max_iter,
                            dpg_stream st) {
  Range range_("dpg_grad_eps");
  if (!h) return DPG_ERR_ARG;
  if (h->stream) {
    h->err = "dpg_grad_eps needs the stored condensation data (not kept with DPG_FLAG_STREAM)";
    return DPG_ERR_UNSUPPORTED;
  }
  return grad_eps(h, reinterpret_cast<const double2*>(xhat), obstacle_mask, P, dP_deps_re, dP_deps_im, cg_mode, cg_rtol,
                  max_iter, S_(st));
}

extern "C" int dpg_power(dpg_handle* h, const dpg_complex* xhat, double* q, double* flux, dpg_stream st) {
  Range range_("dpg_power");
  if (!h) return DPG_ERR_ARG;
  return power(h, reinterpret_cast<const double2*>(xhat), q, flux, S_(st));
}

extern "C" int dpg_sizes(dpg_handle* h, int64_t* n, int64_t* nnz, int32_t* n_elem, int32_t* n_v, int32_t* n_u,
                         int32_t* n_h) {
  if (!h) return DPG_ERR_ARG;
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  if (n_elem) *n_elem = h->ne;
  if (n_v) *n_v = h->szmax.n_v;
  if (n_u) *n_u = h->szmax.n_u;
  if (n_h) *n_h = h->szmax.n_h;
  return DPG_OK;
}

extern "C" int dpg_element_layout(dpg_handle* h, int8_t* p, int64_t* u_off, int64_t* h_off) {
  if (!h) return DPG_ERR_ARG;
  for (int e = 0; e < h->ne; ++e)
    if (p) p[e] = (int8_t)h->grp[h->elem_grp[e]].p;
  for (int e = 0; e <= h->ne; ++e) {
    if (u_off) u_off[e] = h->off[e].u;
    if (h_off) h_off[e] = h->off[e].h;
  }
  return DPG_OK;
}

extern "C" int dpg_trace_map(dpg_handle* h, int32_t* map, dpg_complex* fixed_val) {
  if (!h) return DPG_ERR_ARG;
  if (map) std::memcpy(map, h->l2g.data(), sizeof(int32_t) * h->l2g.size());
  if (fixed_val)
    DPG_CUDA_TRY(h, cudaMemcpy(fixed_val, h->d_xfix, sizeof(double2) * h->l2g.size(), cudaMemcpyDeviceToHost));
  return DPG_OK;
}

extern "C" int dpg_element_dump(dpg_handle* h, const int32_t* ids, int32_t n_ids, dpg_complex* G, dpg_complex* B,
                                dpg_complex* Bh, dpg_complex* l, dpg_complex* Sout, dpg_complex* sout, dpg_stream st) {
  Range range_("dpg_element_dump");
  if (!h || !ids || n_ids <= 0) return DPG_ERR_ARG;
  cudaStream_t s = S_(st);
  for (int k = 0; k < n_ids; ++k)
    if (ids[k] < 0 || ids[k] >= h->ne) {
      h->err = "element id out of range";
      return DPG_ERR_ARG;
    }
  const int g = h->elem_grp[ids[0]];
  for (int k = 0; k < n_ids; ++k)
    if (h->elem_grp[ids[k]] != g) {
      h->err = "dpg_element_dump: the elements must share one trial degree";
      return DPG_ERR_ARG;
    }
  const Sizes& S = h->grp[g].sz;
  const int cap = h->grp[g].cap;
  const int N = S.N, nv = S.n_v, nu = S.n_u, nh = S.n_h;
  std::vector<double2> Kh((size_t)N * N);
  for (int k0 = 0; k0 < n_ids; k0 += cap) {
    const int cnt = std::min(cap, n_ids - k0);
    int rc = run_element_chunk(h, g, ids + k0, cnt, s, false, false);
    if (rc) return rc;
    for (int k = 0; k < cnt; ++k) {
      DPG_CUDA_TRY(h, cudaMemcpyAsync(Kh.data(), h->ws.K + (size_t)k * N * N, sizeof(double2) * N * N,
                                      cudaMemcpyDeviceToHost, s));
      DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
      const size_t q = (size_t)(k0 + k);
      auto at = [&](int i, int j) { return Kh[(size_t)i + (size_t)j * N]; };
      if (G)
        for (int i = 0; i < nv; ++i)
          for (int j = 0; j < nv; ++j) {
            double2 v = at(i, j);
            G[q * nv * nv + (size_t)i * nv + j] = {v.x, v.y};
          }
      if (B)
        for (int i = 0; i < nv; ++i)
          for (int u = 0; u < nu; ++u) {
            double2 v = at(nv + u, i);
            B[q * nv * nu + (size_t)i * nu + u] = {v.x, -v.y};
          }
      if (Bh)
        for (int i = 0; i < nv; ++i)
          for (int t = 0; t < nh; ++t) {
            double2 v = at(nv + nu + t, i);
            Bh[q * nv * nh + (size_t)i * nh + t] = {v.x, -v.y};
          }
      if (l)
        for (int i = 0; i < nv; ++i) {
          double2 v = at(N - 1, i);
          l[q * nv + i] = {v.x, -v.y};
        }
    }
    if ((Sout || sout) && h->stream) {
      // chunk-sized stores: one element at a time, read from its slot
      for (int k = 0; k < cnt; ++k) {
        const int e = ids[k0 + k];
        rc = run_element_chunk(h, g, &e, 1, s, true, true, h->allow_real && h->is_real[e]);
        if (rc) return rc;
        const size_t q = (size_t)(k0 + k);
        if (Sout)
          DPG_CUDA_TRY(h, cudaMemcpyAsync(Sout + q * nh * nh, h->d_S + h->soff_host[e].S, sizeof(double2) * nh * nh,
                                          cudaMemcpyDeviceToHost, s));
        if (sout)
          DPG_CUDA_TRY(h, cudaMemcpyAsync(sout + q * nh, h->d_s + h->soff_host[e].h, sizeof(double2) * nh,
                                          cudaMemcpyDeviceToHost, s));
        DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
      }
    } else if (Sout || sout) {
      std::vector<int> re, cx;
      for (int k = 0; k < cnt; ++k) (h->allow_real && h->is_real[ids[k0 + k]] ? re : cx).push_back(ids[k0 + k]);
      if (!re.empty()) {
        rc = run_element_chunk(h, g, re.data(), (int)re.size(), s, true, true, true);
        if (rc) return rc;
      }
      if (!cx.empty()) {
        rc = run_element_chunk(h, g, cx.data(), (int)cx.size(), s, true, true, false);
        if (rc) return rc;
      }
      for (int k = 0; k < cnt; ++k) {
        const size_t q = (size_t)(k0 + k);
        if (Sout)
          DPG_CUDA_TRY(h, cudaMemcpyAsync(Sout + q * nh * nh, h->d_S + h->off[ids[k0 + k]].S,
                                          sizeof(double2) * nh * nh, cudaMemcpyDeviceToHost, s));
        if (sout)
          DPG_CUDA_TRY(h, cudaMemcpyAsync(sout + q * nh, h->d_s + h->off[ids[k0 + k]].h, sizeof(double2) * nh,
                                          cudaMemcpyDeviceToHost, s));
      }
      DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
    }
  }
  return DPG_OK;
}

extern "C" int dpg_csr_copy(dpg_handle* h, int64_t* row_ptr, int32_t* col, dpg_complex* val, dpg_complex* b,
                            dpg_stream st) {
  Range range_("dpg_csr_copy");
  if (!h) return DPG_ERR_ARG;
  if (!h->have_system && (val || b)) {
    h->err = "dpg_csr_copy of values before dpg_assemble";
    return DPG_ERR_STATE;
  }
  cudaStream_t s = S_(st);
  if (row_ptr)
    DPG_CUDA_TRY(h, cudaMemcpyAsync(row_ptr, h->d_rowptr, sizeof(int64_t) * (h->n + 1), cudaMemcpyDeviceToHost, s));
  if (col) {  // expand the per-entity column lists
    std::vector<int64_t> rp(h->n + 1);
    DPG_CUDA_TRY(h, cudaMemcpy(rp.data(), h->d_rowptr, sizeof(int64_t) * (h->n + 1), cudaMemcpyDeviceToHost));
    for (int b = 0; b < h->nblk; ++b) {
      const int4 B = h->blk[b];
      for (int i = 0; i < B.y; ++i)
        std::memcpy(col + rp[B.x + i], &h->cols[h->blk_colptr[b]], sizeof(int32_t) * B.z);
    }
  }
  if (val) DPG_CUDA_TRY(h, cudaMemcpyAsync(val, h->d_val, sizeof(double2) * h->nnz, cudaMemcpyDeviceToHost, s));
  if (b) DPG_CUDA_TRY(h, cudaMemcpyAsync(b, h->d_b, sizeof(double2) * h->n, cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  return DPG_OK;
}

// Throughput probe: independent FMA chains, each thread writes one output.
template <typename T>
__global__ void k_fma_probe(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x * 1e-7 + k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" int dpg_probe_peaks(double* fp64, double* fp32, dpg_stream st) {
  cudaStream_t s = S_(st);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DPG_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * blocks * threads) != cudaSuccess) return DPG_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0, best64 = 1e30f, best32 = 1e30f;
  const int it64 = 100, it32 = 1000;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_probe<double><<<blocks, threads, 0, s>>>(d, it64, 0.999999, 1e-9);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best64 = std::min(best64, ms);
    cudaEventRecord(e0, s);
    k_fma_probe<float><<<blocks, threads, 0, s>>>((float*)d, it32, 0.999999f, 1e-9f);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best32 = std::min(best32, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (cudaGetLastError() != cudaSuccess) return DPG_ERR_CUDA;
  const double n = (double)blocks * threads * 64.0 * 2.0;
  if (fp64) *fp64 = n * it64 / (best64 * 1e-3);
  if (fp32) *fp32 = n * it32 / (best32 * 1e-3);
  return DPG_OK;
}

extern "C" int dpg_tc_gemm(int32_t split, int32_t Ma, int32_t Nb, int32_t Kd, const double* A, const double* B,
                           double* C, int32_t upper_only) {
  Range range_("dpg_tc_gemm");
  if ((split != 1 && split != 3) || Ma <= 0 || Nb <= 0 || Kd <= 0 || !A || !B || !C) return DPG_ERR_ARG;
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  int* derr = nullptr;
  const size_t nA = (size_t)Kd * Ma, nB = (size_t)Kd * Nb, nC = (size_t)Ma * Nb;
  if (cudaMalloc(&dA, nA * 8) != cudaSuccess || cudaMalloc(&dB, nB * 8) != cudaSuccess ||
      cudaMalloc(&dC, nC * 8) != cudaSuccess || cudaMalloc(&derr, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(derr);
    return DPG_ERR_NOMEM;
  }
  int rc = tc_init(), herr = 0;
  if (rc == DPG_OK && (cudaMemcpy(dA, A, nA * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dB, B, nB * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dC, C, nC * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(derr, 0, sizeof(int)) != cudaSuccess))
    rc = DPG_ERR_CUDA;
  if (rc == DPG_OK) rc = gemm_tn_tc(split, Ma, Nb, Kd, dA, Ma, 0, dB, Nb, 0, dC, Nb, 0, 1, upper_only, derr, nullptr);
  if (rc == DPG_OK && cudaDeviceSynchronize() != cudaSuccess) rc = DPG_ERR_CUDA;
  if (rc == DPG_OK && cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = DPG_ERR_CUDA;
  if (rc == DPG_OK && herr) rc = DPG_ERR_TIMEOUT;
  if (rc == DPG_OK && cudaMemcpy(C, dC, nC * 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = DPG_ERR_CUDA;
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  cudaFree(derr);
  return rc;
}

extern "C" int dpg_update_elements(dpg_handle* h, const double* corners, const dpg_complex* eps, const dpg_complex* mu,
                                   dpg_stream st) {
  Range range_("dpg_update_elements");
  if (!h) return DPG_ERR_ARG;
  cudaStream_t s = S_(st);
  if (corners)
    DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_X, corners, sizeof(double) * 24 * (size_t)h->ne, cudaMemcpyHostToDevice, s));
  if (eps) DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_eps, eps, sizeof(double2) * h->ne, cudaMemcpyHostToDevice, s));
  if (mu) DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_mu, mu, sizeof(double2) * h->ne, cudaMemcpyHostToDevice, s));
  if (eps || mu) {  // re-classify lossless elements (host copies read now)
    if (eps) h->eps_host.assign(eps, eps + h->ne);
    if (mu) h->mu_host.assign(mu, mu + h->ne);
    bool changed = false;
    for (int e = 0; e < h->ne; ++e) {
      const char r = h->eps_host[e].im == 0.0 && h->mu_host[e].im == 0.0 && !h->robin_face[e];
      changed |= r != h->is_real[e];
      h->is_real[e] = r;
    }
    if (changed) {
      classify_elements(h);
      h->plan_valid = false;  // the real / complex chunks change
    }
  }
  h->have_elements = false;
  h->have_system = false;
  return DPG_OK;
}

extern "C" int dpg_timing_enable(dpg_handle* h, int32_t enable) {
  if (!h) return DPG_ERR_ARG;
  h->timing = enable != 0;
  h->factor_ms = h->cg_ms = h->factor_ms_real = h->cgk_ms = 0;
  h->factor_launches = h->factor_elements = h->cg_iters = h->launches = h->factor_elements_real = 0;
  h->cgk_launches = h->cgk_iters = 0;
  return DPG_OK;
}

extern "C" int dpg_cg_bytes_per_iteration(dpg_handle* h, int32_t mode, int64_t* bytes) {
  if (!h || !bytes) return DPG_ERR_ARG;
  *bytes = cg_bytes_per_iteration(h, mode);
  return DPG_OK;
}

extern "C" int dpg_set_estimator_store(dpg_handle* h, int32_t enable);

extern "C" int dpg_set_real_path(dpg_handle* h, int32_t enable) {
  if (!h) return DPG_ERR_ARG;
  if (h->allow_real == (enable != 0)) return DPG_OK;
  h->plan_valid = false;
  h->allow_real = enable != 0;
  if (h->d_Xst) {  // X is sized by each element's arithmetic
    dpg_set_estimator_store(h, 0);
    const int rc = dpg_set_estimator_store(h, 1);
    if (rc) return rc;
  }
  if (h->bucketed) {  // the waves' lists change with the arithmetic split
    set_default_caps(h, h->chunk_req);
    return alloc_workspace(h);
  }
  return DPG_OK;
}

extern "C" int dpg_set_estimator_store(dpg_handle* h, int32_t enable) {
  if (!h) return DPG_ERR_ARG;
  if ((h->d_Xst != nullptr) == (enable != 0)) return DPG_OK;
  h->xst_valid = false;
  h->graph_valid = false;  // the element pass gains or loses its X extraction
  if (!enable) {
    cudaFree(h->d_Xst);
    cudaFree(h->d_xst_off);
    h->d_Xst = nullptr;
    h->d_xst_off = nullptr;
    return DPG_OK;
  }
  if (h->stream) {
    h->err = "streaming keeps no per-element data; the estimator condenses each chunk again";
    return DPG_ERR_UNSUPPORTED;
  }
  std::vector<int64_t> xoff(h->ne + 1, 0);
  for (int e = 0; e < h->ne; ++e) {
    const Sizes& S = h->grp[h->elem_grp[e]].sz;
    const int64_t vals = (int64_t)S.n_v * (S.N - S.n_v);
    xoff[e + 1] = xoff[e] + ((h->allow_real && h->is_real[e]) ? vals : 2 * vals);
  }
  if (cudaMalloc(&h->d_Xst, sizeof(double) * std::max<int64_t>(1, xoff[h->ne])) != cudaSuccess ||
      cudaMalloc(&h->d_xst_off, sizeof(int64_t) * (h->ne + 1)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(h->d_Xst);
    h->d_Xst = nullptr;
    h->d_xst_off = nullptr;
    h->err = "allocation of the stored-factor estimator data (" + std::to_string(8 * xoff[h->ne]) +
             " bytes) failed";
    return DPG_ERR_NOMEM;
  }
  DPG_CUDA_TRY(h, cudaMemcpy(h->d_xst_off, xoff.data(), sizeof(int64_t) * xoff.size(), cudaMemcpyHostToDevice));
  h->have_elements = false;  // the next element pass writes X
  return DPG_OK;
}

extern "C" int dpg_set_bucketed(dpg_handle* h, int32_t enable) {
  if (!h) return DPG_ERR_ARG;
  if (h->bucketed == (enable != 0)) return DPG_OK;
  h->bucketed = enable != 0;
  h->have_elements = false;
  h->have_system = false;
  set_default_caps(h, h->chunk_req);
  return alloc_workspace(h);  // the K arena and the plan (waves) change
}

extern "C" int dpg_factor_balance(dpg_handle* h, double* busy, double* span_ms, int64_t* items) {
  if (!h || !busy || !span_ms || !items) return DPG_ERR_ARG;
  if (!h->d_stamps || h->n_stamps <= 0) {
    h->err = "no element pass has run on the current plan";
    return DPG_ERR_STATE;
  }
  std::vector<unsigned long long> st(3 * (size_t)h->n_stamps);
  DPG_CUDA_TRY(h, cudaMemcpy(st.data(), h->d_stamps, sizeof(unsigned long long) * st.size(), cudaMemcpyDeviceToHost));
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // launches: the waves (bucketed) or the chunks, each a range of stamps
  std::vector<std::pair<int64_t, int64_t>> ranges;
  if (h->bucketed && h->factor_arith == DPG_FACTOR_TC_SPLIT)
    for (const WavePlan& wp : h->waves) {  // the complex and the real launch of the wave
      const int64_t mid = wp.item_off + (wp.nitems - wp.nitems_real);
      ranges.push_back({wp.item_off, mid});
      ranges.push_back({mid, wp.item_off + wp.nitems});
    }
  else
    for (const ChunkPlan& cp : h->plan) ranges.push_back({cp.ids_off, cp.ids_off + cp.count});
  double work = 0, span = 0;
  int64_t n = 0;
  for (const auto& r : ranges) {
    unsigned long long lo = ~0ull, hi = 0;
    for (int64_t k = r.first; k < r.second; ++k) {
      const unsigned long long t0 = st[3 * k + 1], t1 = st[3 * k + 2];
      if (t0 == 0 || t1 < t0) {
        h->err = "the last element pass left no factorisation stamps (FP64-pipe factorisation?)";
        return DPG_ERR_STATE;
      }
      lo = std::min(lo, t0);
      hi = std::max(hi, t1);
      work += (double)(t1 - t0);
      ++n;
    }
    if (r.second > r.first) span += (double)(hi - lo);
  }
  *busy = span > 0 ? work / (span * sms) : 0.0;
  *span_ms = span * 1e-6;
  *items = n;
  return DPG_OK;
}

extern "C" int dpg_set_factor_arith(dpg_handle* h, int32_t arith) {
  if (!h || (arith != DPG_FACTOR_FP64 && arith != DPG_FACTOR_TC_SPLIT)) return DPG_ERR_ARG;
  if (arith == h->factor_arith) return DPG_OK;
  h->factor_arith = arith;
  h->have_elements = false;
  h->have_system = false;
  return alloc_workspace(h);  // the digit scratch; invalidates the launch plan and its graph
}

extern "C" int dpg_set_wait_limit(dpg_handle* h, int64_t wait_ns, int32_t hold) {
  if (!h || wait_ns <= 0) return DPG_ERR_ARG;
  h->wait_ns = wait_ns;
  h->wait_hold = hold != 0;
  return DPG_OK;
}

extern "C" int dpg_set_graph(dpg_handle* h, int32_t enable) {
  if (!h) return DPG_ERR_ARG;
  h->use_graph = enable != 0;
  return DPG_OK;
}

extern "C" int dpg_autotune(dpg_handle* h, double max_workspace_bytes, int32_t* caps, float* ms_per_element,
                            dpg_stream st) {
  Range range_("dpg_autotune");
  if (!h || !(max_workspace_bytes > 0)) return DPG_ERR_ARG;
  if (h->stream) {
    h->err = "dpg_autotune is not available with DPG_FLAG_STREAM";
    return DPG_ERR_UNSUPPORTED;
  }
  int rc = autotune(h, max_workspace_bytes, caps, ms_per_element, S_(st));
  h->have_elements = false;
  h->have_system = false;
  return rc;
}

extern "C" int dpg_group_info(dpg_handle* h, int32_t* n_groups, int32_t* p, int32_t* n_elem, int32_t* cap) {
  if (!h) return DPG_ERR_ARG;
  if (n_groups) *n_groups = (int32_t)h->grp.size();
  for (size_t g = 0; g < h->grp.size(); ++g) {
    if (p) p[g] = h->grp[g].p;
    if (n_elem) n_elem[g] = (int32_t)h->grp[g].elems.size();
    if (cap) cap[g] = h->grp[g].cap;
  }
  return DPG_OK;
}

extern "C" int dpg_timing_get(dpg_handle* h, dpg_timing* out) {
  if (!h || !out) return DPG_ERR_ARG;
  out->factor_ms = h->factor_ms;
  out->factor_launches = h->factor_launches;
  out->factor_elements = h->factor_elements;
  out->cg_ms = h->cg_ms;
  out->cg_iterations = h->cg_iters;
  out->kernel_launches = h->launches;
  out->factor_ms_real = h->factor_ms_real;
  out->factor_elements_real = h->factor_elements_real;
  out->cg_kernel_ms = h->cgk_ms;
  out->cg_kernel_launches = h->cgk_launches;
  out->cg_kernel_iterations = h->cgk_iters;
  return DPG_OK;
}

extern "C" const char* dpg_last_error(dpg_handle* h) {
  if (!h) return g_setup_err.c_str();  // the last failed dpg_setup_mesh on this thread
  return h->err.c_str();
}

extern "C" void dpg_destroy(dpg_handle* h) {
  if (!h) return;
  free_all(h);
  delete h;
}
