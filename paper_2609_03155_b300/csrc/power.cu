// Electromagnetic power of a solution (Sec. 3.2): per-element dissipated power
// int_K Q_em dV with Q_em = 1/2 omega (Im eps |E|^2 + Im mu |H|^2) (dimensionless,
// the conductivity being part of Im eps), and the Poynting flux
// int Re(E x conj(H)) . n_out dA through the Robin faces of each Robin group
// (the port flux that sets the reference field E0 of Eq. power_scaling).
// Both use the interior fields u_K and the element pass's Gauss-Legendre rule.
#include <cmath>

#include "dpg_internal.h"

namespace dpg {

namespace {

__device__ __forceinline__ void p_geom(const double* X, const double xi[3], double J[3][3]) {
  for (int a = 0; a < 3; ++a) J[a][0] = J[a][1] = J[a][2] = 0.0;
  for (int v = 0; v < 8; ++v) {
    const double f0 = (v & 1) ? xi[0] : 1.0 - xi[0], d0 = (v & 1) ? 1.0 : -1.0;
    const double f1 = (v & 2) ? xi[1] : 1.0 - xi[1], d1 = (v & 2) ? 1.0 : -1.0;
    const double f2 = (v & 4) ? xi[2] : 1.0 - xi[2], d2 = (v & 4) ? 1.0 : -1.0;
    for (int a = 0; a < 3; ++a) {
      J[a][0] += d0 * f1 * f2 * X[3 * v + a];
      J[a][1] += f0 * d1 * f2 * X[3 * v + a];
      J[a][2] += f0 * f1 * d2 * X[3 * v + a];
    }
  }
}

__device__ __forceinline__ double p_det(const double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// E and H at the extended 1D point indices qi (Lagrange values of the L^2 family).
__device__ __forceinline__ void p_fields(const Tables& T, int p1, int nL, const double2* u, const int qi[3],
                                         double2 E[3], double2 H[3]) {
  for (int d = 0; d < 3; ++d) E[d] = H[d] = make_double2(0.0, 0.0);
  for (int l = 0; l < nL; ++l) {
    const int l0 = l % p1, l1 = (l / p1) % p1, l2 = l / (p1 * p1);
    const double L = T.val[F_L2][qi[0]][l0] * T.val[F_L2][qi[1]][l1] * T.val[F_L2][qi[2]][l2];
    for (int d = 0; d < 3; ++d) {
      const double2 e = u[d * nL + l], hh = u[(3 + d) * nL + l];
      E[d].x += L * e.x;
      E[d].y += L * e.y;
      H[d].x += L * hh.x;
      H[d].y += L * hh.y;
    }
  }
}

__device__ __forceinline__ double p_block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
  return t;
}

}  // namespace

// One block per element of one order group.
__global__ void __launch_bounds__(256) k_power_vol(const __grid_constant__ Tables T, Sizes S, double omega,
                                                   const int* __restrict__ elems, const ElemOff* __restrict__ off,
                                                   const double* __restrict__ Xall, const double2* __restrict__ eps,
                                                   const double2* __restrict__ mu, const double2* __restrict__ u,
                                                   double* q) {
  __shared__ double sX[24];
  __shared__ double red[8];
  const int e = elems[blockIdx.x];
  if (threadIdx.x < 24) sX[threadIdx.x] = Xall[(size_t)e * 24 + threadIdx.x];
  __syncthreads();
  const double2* ue = u + off[e].u;
  const int nq1 = S.nq1, p1 = S.p + 1;
  double aE = 0.0, aH = 0.0;
  for (int k = threadIdx.x; k < S.nq; k += blockDim.x) {
    const int qi[3] = {k % nq1, (k / nq1) % nq1, k / (nq1 * nq1)};
    const double xi[3] = {T.pt[qi[0]], T.pt[qi[1]], T.pt[qi[2]]};
    double J[3][3];
    p_geom(sX, xi, J);
    const double wd = T.w[qi[0]] * T.w[qi[1]] * T.w[qi[2]] * p_det(J);
    double2 E[3], H[3];
    p_fields(T, p1, S.nL, ue, qi, E, H);
    for (int d = 0; d < 3; ++d) {
      aE += wd * (E[d].x * E[d].x + E[d].y * E[d].y);
      aH += wd * (H[d].x * H[d].x + H[d].y * H[d].y);
    }
  }
  aE = p_block_sum(aE, red);
  aH = p_block_sum(aH, red);
  if (threadIdx.x == 0) q[e] = 0.5 * omega * (eps[e].y * aE + mu[e].y * aH);
}

// One block per (element, face) entry: int Re(E x conj(H)) . (det J J^{-T} N_ref) dxi.
__global__ void __launch_bounds__(256) k_power_face(const __grid_constant__ Tables T, Sizes S,
                                                    const int* __restrict__ ent, const ElemOff* __restrict__ off,
                                                    const double* __restrict__ Xall, const double2* __restrict__ u,
                                                    double* flux) {
  __shared__ double sX[24];
  __shared__ double red[8];
  const int e = ent[2 * blockIdx.x], f = ent[2 * blockIdx.x + 1];
  const int d = f >> 1, sd = f & 1;
  if (threadIdx.x < 24) sX[threadIdx.x] = Xall[(size_t)e * 24 + threadIdx.x];
  __syncthreads();
  const double2* ue = u + off[e].u;
  const int nq1 = S.nq1, p1 = S.p + 1;
  const int a = (d == 0) ? 1 : 0, b = (d == 2) ? 1 : 2;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nq1 * nq1; k += blockDim.x) {
    const int ta = k % nq1, tb = k / nq1;
    int qi[3];
    qi[d] = nq1 + sd;  // extended point xi_d = sd
    qi[a] = ta;
    qi[b] = tb;
    const double xi[3] = {T.pt[qi[0]], T.pt[qi[1]], T.pt[qi[2]]};
    double J[3][3];
    p_geom(sX, xi, J);
    const double det = p_det(J);
    // det J J^{-T} N_ref = (2 sd - 1) times row d of the cofactor matrix of J
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    const double sg = sd ? 1.0 : -1.0;
    double nv[3];
    for (int c = 0; c < 3; ++c) {
      const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      nv[c] = sg * (J[c1][d1] * J[c2][d2] - J[c1][d2] * J[c2][d1]);
    }
    (void)det;
    double2 E[3], H[3];
    p_fields(T, p1, S.nL, ue, qi, E, H);
    // Re(E x conj(H))
    double Sv[3];
    for (int c = 0; c < 3; ++c) {
      const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      Sv[c] = (E[c1].x * H[c2].x + E[c1].y * H[c2].y) - (E[c2].x * H[c1].x + E[c2].y * H[c1].y);
    }
    acc += T.w[ta] * T.w[tb] * (Sv[0] * nv[0] + Sv[1] * nv[1] + Sv[2] * nv[2]);
  }
  acc = p_block_sum(acc, red);
  if (threadIdx.x == 0) flux[blockIdx.x] = acc;
}

static int ensure_dev(dpg_handle* h, void** p, size_t bytes) {
  if (*p) return DPG_OK;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->err = "power buffer allocation failed";
    return DPG_ERR_NOMEM;
  }
  return DPG_OK;
}

int power(dpg_handle* h, const double2* xhat, double* q, double* flux_host, cudaStream_t s) {
  if (!h->have_elements) {
    h->err = "dpg_power before dpg_element_batch";
    return DPG_ERR_STATE;
  }
  if (!xhat) {
    h->err = "null xhat";
    return DPG_ERR_ARG;
  }
  const ElemOff tot = h->off[h->ne];
  int rc = ensure_dev(h, (void**)&h->d_u, sizeof(double2) * tot.u);
  if (rc) return rc;
  rc = estimate(h, xhat, h->d_u, nullptr, nullptr, s);
  if (rc) return rc;
  if (q) {
    for (const Group& G : h->grp) {
      k_power_vol<<<(int)G.elems.size(), 256, 0, s>>>(G.tab, G.sz, h->omega, G.d_elems, h->d_off, h->d_X, h->d_eps,
                                                      h->d_mu, h->d_u, q);
      h->launches += 1;
    }
    DPG_CUDA_TRY(h, cudaGetLastError());
  }
  if (flux_host) {
    const int nrob = (int)h->robin.size();
    for (int k = 0; k < nrob; ++k) flux_host[k] = 0.0;
    // Robin entries per order group, in entry order
    for (int g = 0; g < (int)h->grp.size(); ++g) {
      std::vector<int> ent, grp_of;
      for (const RobinEntry& re : h->robin_entries)
        if (h->elem_grp[re.elem] == g) {
          ent.push_back(re.elem);
          ent.push_back(re.face);
          grp_of.push_back(re.grp);
        }
      const int n = (int)grp_of.size();
      if (n == 0) continue;
      int* d_ent = nullptr;
      double* d_flux = nullptr;
      DPG_CUDA_TRY(h, cudaMallocAsync(&d_ent, sizeof(int) * ent.size(), s));
      DPG_CUDA_TRY(h, cudaMallocAsync(&d_flux, sizeof(double) * n, s));
      DPG_CUDA_TRY(h, cudaMemcpyAsync(d_ent, ent.data(), sizeof(int) * ent.size(), cudaMemcpyHostToDevice, s));
      k_power_face<<<n, 256, 0, s>>>(h->grp[g].tab, h->grp[g].sz, d_ent, h->d_off, h->d_X, h->d_u, d_flux);
      h->launches += 1;
      DPG_CUDA_TRY(h, cudaGetLastError());
      std::vector<double> fl(n);
      DPG_CUDA_TRY(h, cudaMemcpyAsync(fl.data(), d_flux, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
      DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
      DPG_CUDA_TRY(h, cudaFreeAsync(d_ent, s));
      DPG_CUDA_TRY(h, cudaFreeAsync(d_flux, s));
      for (int k = 0; k < n; ++k) flux_host[grp_of[k]] += fl[k];
    }
  }
  return DPG_OK;
}

}  // namespace dpg
