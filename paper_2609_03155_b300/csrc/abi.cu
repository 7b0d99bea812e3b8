// extern "C" entry points of libdpg (declared in include/dpg.h).
#include <algorithm>
#include <cstring>
#include <new>

#include "dpg_internal.h"

using namespace dpg;

static cudaStream_t S_(dpg_stream s) { return reinterpret_cast<cudaStream_t>(s); }
static thread_local std::string g_setup_err;

static void free_all(dpg_handle* h) {
  void* bufs[] = {h->d_X,     h->d_eps,   h->d_mu,   h->d_fbc,   h->d_Xref,  h->d_Tf,   h->d_Tall,
                  h->d_trfun, h->d_l2g,   h->d_xfix, h->d_color_elems, h->d_robin, h->d_status, h->d_S,
                  h->d_s,     h->d_c,     h->d_Z,    h->d_z,     h->d_rowptr, h->d_row2blk, h->d_val,
                  h->d_b,     h->d_val32, h->d_r,    h->d_p,     h->d_Ap,    h->d_r32,  h->d_p32,
                  h->d_Ap32,  h->d_x32,   h->d_red,  h->d_cgstate,  h->ws.K,    h->ws.V,   h->ws.Cu,
                  h->ws.PhiL, h->ws.MC,   h->ws.ids, h->ws.FV,   h->ws.FR,   h->ws.rent,
                  h->d_dinv,  h->d_dinv32, h->d_L1, h->d_u, h->d_zg, h->d_gc, h->d_lam, h->d_rhs_adj,
                  h->d_Pk, h->d_blk, h->d_blk_colptr, h->d_cols, h->d_binv_ptr, h->d_binv, h->d_binv32,
                  h->d_zv, h->d_z32, h->d_d64};
  for (void* b : bufs)
    if (b) cudaFree(b);
}

extern "C" int dpg_setup_mesh(dpg_handle** out, const dpg_mesh_desc* m, const dpg_params* prm, dpg_stream st) {
  if (!out) return DPG_ERR_ARG;
  *out = nullptr;
  dpg_handle* h = new (std::nothrow) dpg_handle();
  if (!h) return DPG_ERR_NOMEM;
  cudaStream_t s = S_(st);
  int rc = build_mesh(h, m, prm, s);
  if (rc == DPG_OK) {
    const Sizes& S = h->sz;
    size_t per = sizeof(double2) * (size_t)S.N * S.N + sizeof(double) * 3 * (size_t)S.nq * (2 * S.n_f + 3 * S.nL) +
                 sizeof(double) * (2 * (size_t)S.n_f * S.n_f + 2 * (size_t)S.n_f * 3 * S.nL);
    size_t budget = (size_t)12 << 30;
    int cap = (int)std::max<size_t>(1, budget / per);
    if (prm->chunk > 0) cap = prm->chunk;
    if (cap >= 148 && prm->chunk <= 0) cap = cap / 148 * 148;
    cap = std::min(cap, h->ne);
    cap = std::max(cap, 1);
    rc = alloc_workspace(h, cap);
    if (rc == DPG_OK) rc = compute_reference_matrices(h, s);
  }
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
  if (!h) return DPG_ERR_ARG;
  if (pass != DPG_PASS_ASSEMBLE) {
    h->err = "unknown element pass";
    return DPG_ERR_ARG;
  }
  cudaStream_t s = S_(st);
  const int cap = h->ws.cap;
  // lossless elements in real arithmetic, the others in complex arithmetic
  std::vector<int> all;
  const std::vector<int>* lists[2];
  if (h->allow_real) {
    lists[0] = &h->real_elems;
    lists[1] = &h->cplx_elems;
  } else {
    all.resize(h->ne);
    for (int e = 0; e < h->ne; ++e) all[e] = e;
    lists[0] = &all;
    lists[1] = nullptr;
  }
  for (int li = 0; li < 2; ++li) {
    if (!lists[li]) continue;
    const std::vector<int>& L = *lists[li];
    const bool real = h->allow_real && li == 0;
    for (size_t c0 = 0; c0 < L.size(); c0 += cap) {
      const int cnt = (int)std::min<size_t>(cap, L.size() - c0);
      int rc = run_element_chunk(h, L.data() + c0, cnt, s, true, true, real);
      if (rc) return rc;
    }
  }
  h->have_elements = true;
  h->have_system = false;
  // pivot check
  std::vector<int> status(h->ne);
  DPG_CUDA_TRY(h, cudaMemcpyAsync(status.data(), h->d_status, sizeof(int) * h->ne, cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  for (size_t k = 0; k < h->factor_events.size(); ++k) {
    float ms = 0;
    cudaEventElapsedTime(&ms, h->factor_events[k].first, h->factor_events[k].second);
    h->factor_ms += ms;
    h->factor_launches += 1;
    h->factor_elements += h->factor_counts[k];
    if (h->factor_real[k]) {
      h->factor_ms_real += ms;
      h->factor_elements_real += h->factor_counts[k];
    }
    cudaEventDestroy(h->factor_events[k].first);
    cudaEventDestroy(h->factor_events[k].second);
  }
  h->factor_events.clear();
  h->factor_counts.clear();
  h->factor_real.clear();
  for (int e = 0; e < h->ne; ++e)
    if (status[e]) {
      h->err = "non-positive pivot in element " + std::to_string(e);
      return DPG_ERR_NOT_HPD;
    }
  return DPG_OK;
}

extern "C" int dpg_assemble(dpg_handle* h, dpg_stream st) {
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
  if (!h) return DPG_ERR_ARG;
  return cg_solve(h, mode, rtol, atol, max_iter, inner_rtol, reinterpret_cast<double2*>(x),
                  reinterpret_cast<const double2*>(b), rep, S_(st));
}

extern "C" int dpg_estimate(dpg_handle* h, const dpg_complex* xhat, dpg_complex* u, double* eta, double* eta_global,
                            dpg_stream st) {
  if (!h) return DPG_ERR_ARG;
  return estimate(h, reinterpret_cast<const double2*>(xhat), reinterpret_cast<double2*>(u), eta, eta_global, S_(st));
}

extern "C" int dpg_estimate_noalloc(dpg_handle* h, const dpg_complex* xhat, dpg_complex* u, double* eta,
                                    double* eta_global, dpg_stream st) {
  if (!h) return DPG_ERR_ARG;
  return estimate_noalloc(h, reinterpret_cast<const double2*>(xhat), reinterpret_cast<double2*>(u), eta, eta_global,
                          S_(st));
}

extern "C" int dpg_grad_eps(dpg_handle* h, const dpg_complex* xhat, const uint8_t* obstacle_mask, double* P,
                            double* dP_deps_re, double* dP_deps_im, int32_t cg_mode, double cg_rtol, int32_t max_iter,
                            dpg_stream st) {
  if (!h) return DPG_ERR_ARG;
  return grad_eps(h, reinterpret_cast<const double2*>(xhat), obstacle_mask, P, dP_deps_re, dP_deps_im, cg_mode, cg_rtol,
                  max_iter, S_(st));
}

extern "C" int dpg_sizes(dpg_handle* h, int64_t* n, int64_t* nnz, int32_t* n_elem, int32_t* n_v, int32_t* n_u,
                         int32_t* n_h) {
  if (!h) return DPG_ERR_ARG;
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  if (n_elem) *n_elem = h->ne;
  if (n_v) *n_v = h->sz.n_v;
  if (n_u) *n_u = h->sz.n_u;
  if (n_h) *n_h = h->sz.n_h;
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
  if (!h || !ids || n_ids <= 0) return DPG_ERR_ARG;
  cudaStream_t s = S_(st);
  const Sizes& S = h->sz;
  const int N = S.N, nv = S.n_v, nu = S.n_u, nh = S.n_h;
  for (int k = 0; k < n_ids; ++k)
    if (ids[k] < 0 || ids[k] >= h->ne) {
      h->err = "element id out of range";
      return DPG_ERR_ARG;
    }
  std::vector<double2> Kh((size_t)N * N);
  for (int k0 = 0; k0 < n_ids; k0 += h->ws.cap) {
    const int cnt = std::min(h->ws.cap, n_ids - k0);
    int rc = run_element_chunk(h, ids + k0, cnt, s, false, false);
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
    if (Sout || sout) {
      std::vector<int> re, cx;
      for (int k = 0; k < cnt; ++k) (h->allow_real && h->is_real[ids[k0 + k]] ? re : cx).push_back(ids[k0 + k]);
      if (!re.empty()) {
        rc = run_element_chunk(h, re.data(), (int)re.size(), s, true, true, true);
        if (rc) return rc;
      }
      if (!cx.empty()) {
        rc = run_element_chunk(h, cx.data(), (int)cx.size(), s, true, true, false);
        if (rc) return rc;
      }
      for (int k = 0; k < cnt; ++k) {
        const size_t q = (size_t)(k0 + k);
        if (Sout)
          DPG_CUDA_TRY(h, cudaMemcpyAsync(Sout + q * nh * nh, h->d_S + (size_t)ids[k0 + k] * nh * nh,
                                          sizeof(double2) * nh * nh, cudaMemcpyDeviceToHost, s));
        if (sout)
          DPG_CUDA_TRY(h, cudaMemcpyAsync(sout + q * nh, h->d_s + (size_t)ids[k0 + k] * nh, sizeof(double2) * nh,
                                          cudaMemcpyDeviceToHost, s));
      }
      DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
    }
  }
  return DPG_OK;
}

extern "C" int dpg_csr_copy(dpg_handle* h, int64_t* row_ptr, int32_t* col, dpg_complex* val, dpg_complex* b,
                            dpg_stream st) {
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

extern "C" int dpg_update_elements(dpg_handle* h, const double* corners, const dpg_complex* eps, const dpg_complex* mu,
                                   dpg_stream st) {
  if (!h) return DPG_ERR_ARG;
  cudaStream_t s = S_(st);
  if (corners)
    DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_X, corners, sizeof(double) * 24 * (size_t)h->ne, cudaMemcpyHostToDevice, s));
  if (eps) DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_eps, eps, sizeof(double2) * h->ne, cudaMemcpyHostToDevice, s));
  if (mu) DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_mu, mu, sizeof(double2) * h->ne, cudaMemcpyHostToDevice, s));
  if (eps || mu) {  // re-classify lossless elements (host copies read now)
    if (eps) h->eps_host.assign(eps, eps + h->ne);
    if (mu) h->mu_host.assign(mu, mu + h->ne);
    h->real_elems.clear();
    h->cplx_elems.clear();
    for (int e = 0; e < h->ne; ++e) {
      const bool real = h->eps_host[e].im == 0.0 && h->mu_host[e].im == 0.0 && !h->robin_face[e];
      h->is_real[e] = real;
      (real ? h->real_elems : h->cplx_elems).push_back(e);
    }
  }
  h->have_elements = false;
  h->have_system = false;
  return DPG_OK;
}

extern "C" int dpg_timing_enable(dpg_handle* h, int32_t enable) {
  if (!h) return DPG_ERR_ARG;
  h->timing = enable != 0;
  h->factor_ms = h->cg_ms = h->factor_ms_real = 0;
  h->factor_launches = h->factor_elements = h->cg_iters = h->launches = h->factor_elements_real = 0;
  return DPG_OK;
}

extern "C" int dpg_set_real_path(dpg_handle* h, int32_t enable) {
  if (!h) return DPG_ERR_ARG;
  h->allow_real = enable != 0;
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
