// Absorbed power of an obstacle and its adjoint gradient with respect to the
// per-element permittivity (the paper has no adjoint; this serves the
// reactor-optimisation use of the solver).
//
// P = 1/2 omega sum_{K in obstacle} Im(eps_K) int_K |E|^2 (the electric-loss
// term of Q_em, Sec. 3.2, dimensionless).  DPG minimises
// J(w) = sum_K ||l_K - B_K w_K||^2_{G_K^{-1}}; with g = dP/d conj(w) and the
// adjoint A lambda = g (same Hermitian system, condensed like Eq. linear_system),
//   dP/ds = dP/ds|explicit + 2 Re((B' lambda)^H psi - mu^H G' psi - mu^H B' w),
//   psi = G^{-1}(l - B_K w), mu = G^{-1} B_K lambda,
// for s = Re eps_K (c = i w, a = 2 w^2 Re eps) and s = Im eps_K (c = -w,
// a = 2 w^2 Im eps):  B' = c P on the (F, E) block,
// G' = [[a M, c X^T], [conj(c) X, 0]] (rows/cols F, I).
#include <cmath>

#include "dpg_internal.h"

namespace dpg {

__device__ __forceinline__ double2 a_cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 a_cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double a_wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Gather element-local trace values of a global vector (free entries), fixed
// values (fix != nullptr) or zero.
__device__ __forceinline__ double2 gather_trace(const int32_t* l2g, const double2* fix, const double2* x, size_t k) {
  const int g = l2g[k];
  if (g >= 0) return x[g];
  if (g == -1 && fix) return fix[k];
  return make_double2(0.0, 0.0);
}

// Per element: E at the volume points from u_E, g_u = 1/2 w Im(eps) M_E u_E,
// e_K = 1/2 w u_E^H M_E u_E (explicit d P / d Im eps), P_K = Im(eps) e_K,
// zg = M1^{-1} g_u (through the stored Cholesky factor L1 of M1) and the
// condensed adjoint load gc = -Z^H g_u.  Elements outside the obstacle get zeros.
__global__ void __launch_bounds__(256) k_adj_source(const __grid_constant__ Tables T, Sizes S, double omega,
                                                    const int* __restrict__ elems, const ElemOff* __restrict__ off,
                                                    const double* __restrict__ Xall, const double2* __restrict__ eps_all,
                                                    const uint8_t* __restrict__ mask, const double2* __restrict__ u,
                                                    const double2* __restrict__ L1st, const double2* __restrict__ Zst,
                                                    double2* zg, double2* gc, double* Pk, double* ek) {
  extern __shared__ double2 sh[];
  const int e = elems[blockIdx.x];
  const ElemOff of = off[e];
  const int nu = S.n_u, nh = S.n_h, nL = S.nL, nq = S.nq, nq1 = S.nq1, p1 = S.p + 1;
  double2* g = sh;            // n_u
  double2* Eq = g + nu;       // 3 nq (E at the points, times w det J)
  __shared__ double sX[24];
  __shared__ double sred[8];
  if (!mask[e]) {
    for (int t = threadIdx.x; t < nu; t += blockDim.x) zg[of.u + t] = make_double2(0.0, 0.0);
    for (int t = threadIdx.x; t < nh; t += blockDim.x) gc[of.h + t] = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
      Pk[e] = 0.0;
      ek[e] = 0.0;
    }
    return;
  }
  if (threadIdx.x < 24) sX[threadIdx.x] = Xall[(size_t)e * 24 + threadIdx.x];
  __syncthreads();
  const double2* ue = u + of.u;
  // E(q) w det J
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const int qi[3] = {q % nq1, (q / nq1) % nq1, q / (nq1 * nq1)};
    const double xi[3] = {T.pt[qi[0]], T.pt[qi[1]], T.pt[qi[2]]};
    double J[3][3];
    for (int a = 0; a < 3; ++a) J[a][0] = J[a][1] = J[a][2] = 0.0;
    for (int v = 0; v < 8; ++v) {
      double f0 = (v & 1) ? xi[0] : 1.0 - xi[0], d0 = (v & 1) ? 1.0 : -1.0;
      double f1 = (v & 2) ? xi[1] : 1.0 - xi[1], d1 = (v & 2) ? 1.0 : -1.0;
      double f2 = (v & 4) ? xi[2] : 1.0 - xi[2], d2 = (v & 4) ? 1.0 : -1.0;
      for (int a = 0; a < 3; ++a) {
        J[a][0] += d0 * f1 * f2 * sX[3 * v + a];
        J[a][1] += f0 * d1 * f2 * sX[3 * v + a];
        J[a][2] += f0 * f1 * d2 * sX[3 * v + a];
      }
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    const double wd = T.w[qi[0]] * T.w[qi[1]] * T.w[qi[2]] * det;
    for (int d = 0; d < 3; ++d) {
      double2 E = make_double2(0.0, 0.0);
      for (int l = 0; l < nL; ++l) {
        const int l0 = l % p1, l1 = (l / p1) % p1, l2 = l / (p1 * p1);
        const double L = T.val[F_L2][qi[0]][l0] * T.val[F_L2][qi[1]][l1] * T.val[F_L2][qi[2]][l2];
        E.x += L * ue[d * nL + l].x;
        E.y += L * ue[d * nL + l].y;
      }
      Eq[3 * q + d] = make_double2(E.x * wd, E.y * wd);
    }
  }
  __syncthreads();
  const double2 eps = eps_all[e];
  const double half_w = 0.5 * omega;
  // (M_E u_E)_{d,l} = sum_q w det J L_l(q) E_d(q)
  double part = 0.0;
  for (int t = threadIdx.x; t < nu; t += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (t < 3 * nL) {
      const int d = t / nL, l = t - d * nL;
      const int l0 = l % p1, l1 = (l / p1) % p1, l2 = l / (p1 * p1);
      for (int q = 0; q < nq; ++q) {
        const int qi0 = q % nq1, qi1 = (q / nq1) % nq1, qi2 = q / (nq1 * nq1);
        const double L = T.val[F_L2][qi0][l0] * T.val[F_L2][qi1][l1] * T.val[F_L2][qi2][l2];
        v.x += L * Eq[3 * q + d].x;
        v.y += L * Eq[3 * q + d].y;
      }
      part += ue[t].x * v.x + ue[t].y * v.y;  // Re(conj(u) M u)
    }
    g[t] = make_double2(half_w * eps.y * v.x, half_w * eps.y * v.y);
  }
  part = a_wsum(part);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += sred[k];
    ek[e] = half_w * tot;
    Pk[e] = eps.y * half_w * tot;
  }
  // gc = -Z^H g  (Z: n_u x n_h row-major)
  const double2* Ze = Zst + of.Z;
  for (int t = threadIdx.x; t < nh; t += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < nu; ++k) {
      const double2 z = Ze[(size_t)k * nh + t];
      const double2 gk = g[k];
      acc.x += z.x * gk.x + z.y * gk.y;  // conj(z) g
      acc.y += z.x * gk.y - z.y * gk.x;
    }
    gc[of.h + t] = make_double2(-acc.x, -acc.y);
  }
  __syncthreads();
  // zg = L1^{-H} L1^{-1} g  (L1 row-major lower, n_u x n_u), one thread
  if (threadIdx.x == 0) {
    const double2* L = L1st + of.L1;
    double2* z = zg + of.u;
    for (int i = 0; i < nu; ++i) {  // forward
      double2 v = g[i];
      for (int k = 0; k < i; ++k) {
        const double2 pr = a_cmul(L[(size_t)i * nu + k], z[k]);
        v.x -= pr.x;
        v.y -= pr.y;
      }
      const double d = L[(size_t)i * nu + i].x;
      z[i] = make_double2(v.x / d, v.y / d);
    }
    for (int i = nu - 1; i >= 0; --i) {  // backward with L1^H
      double2 v = z[i];
      for (int k = i + 1; k < nu; ++k) {
        const double2 pr = a_cmul(a_cconj(L[(size_t)k * nu + i]), z[k]);
        v.x -= pr.x;
        v.y -= pr.y;
      }
      const double d = L[(size_t)i * nu + i].x;
      z[i] = make_double2(v.x / d, v.y / d);
    }
  }
}

// rhs[g_i] += gc[e][i] for the elements of one colour (free entries only)
__global__ void k_adj_scatter(int nh, const int* __restrict__ elems, const ElemOff* __restrict__ off,
                              const int32_t* __restrict__ l2g, const double2* __restrict__ gc, double2* rhs) {
  const int e = elems[blockIdx.x];
  const int64_t o = off[e].h;
  for (int i = threadIdx.x; i < nh; i += blockDim.x) {
    const int g = l2g[o + i];
    if (g >= 0) {
      const double2 v = gc[o + i];
      rhs[g].x += v.x;
      rhs[g].y += v.y;
    }
  }
}

__global__ void k_sum_serial(int n, const double* __restrict__ v, double* out) {
  __shared__ double sw[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += v[i];
  acc = a_wsum(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sw[k];
    *out = t;
  }
}

// Block-wide sum of two doubles (all threads get the result).
__device__ void block_sum2(double& a, double& b, double* red) {
  a = a_wsum(a);
  b = a_wsum(b);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[2 * (threadIdx.x >> 5)] = a;
    red[2 * (threadIdx.x >> 5) + 1] = b;
  }
  __syncthreads();
  a = b = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
    a += red[2 * k];
    b += red[2 * k + 1];
  }
  __syncthreads();
}

// Gradient of one element (one CTA).  K holds the formed augmented matrix with
// its G block replaced by the Cholesky factor L (lower, column-major, ld N).
__global__ void __launch_bounds__(256) k_adj_grad(Sizes S, double omega, const int* __restrict__ ids,
                                                  const ElemOff* __restrict__ off, const int* __restrict__ sig,
                                                  const RSig* __restrict__ rsig, const int32_t* __restrict__ rint,
                                                  const double* __restrict__ rdbl,
                                                  const double2* __restrict__ eps_all, const double2* __restrict__ K,
                                                  const double* __restrict__ MC, const double* __restrict__ Xref,
                                                  const int32_t* __restrict__ l2g, const double2* __restrict__ xfix,
                                                  const double2* __restrict__ xhat, const double2* __restrict__ lam,
                                                  const double2* __restrict__ u, const double2* __restrict__ zg,
                                                  const double2* __restrict__ Zst, const double* __restrict__ ek,
                                                  const uint8_t* __restrict__ mask, double* dre, double* dim) {
  extern __shared__ double2 sh[];
  const int slot = blockIdx.x;
  const int e = ids[slot];
  const ElemOff of = off[e];
  const int N = S.N, nv = S.n_v, nu = S.n_u, nh = S.n_h, nf = S.n_f, m = nu + nh, nL3 = 3 * S.nL;
  double2* w = sh;          // m
  double2* lm = w + m;      // m
  double2* r = lm + m;      // n_v  (becomes psi)
  double2* bl = r + nv;     // n_v  (becomes mu)
  __shared__ double red[16];
  const double2* A = K + (size_t)slot * N * N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // 1. w = (u, uhat), lambda = (zg - Z lambda_h, lambda_h), in the trace slots
  for (int t = threadIdx.x; t < nh; t += blockDim.x) {
    const size_t k = (size_t)of.h + t;
    w[nu + t] = gather_trace(l2g, xfix, xhat, k);
    lm[nu + t] = gather_trace(l2g, nullptr, lam, k);
  }
  for (int t = threadIdx.x; t < nu; t += blockDim.x) w[t] = u[of.u + t];
  __syncthreads();
  const double2* Ze = Zst + of.Z;
  for (int i = wid; i < nu; i += nw) {
    double ar = 0.0, ai = 0.0;
    for (int j = lane; j < nh; j += 32) {
      const double2 z = Ze[(size_t)i * nh + j], l = lm[nu + j];
      ar += z.x * l.x - z.y * l.y;
      ai += z.x * l.y + z.y * l.x;
    }
    ar = a_wsum(ar);
    ai = a_wsum(ai);
    if (lane == 0) {
      const double2 zgi = zg[of.u + i];
      lm[i] = make_double2(zgi.x - ar, zgi.y - ai);
    }
  }
  __syncthreads();
  // restricted elements: element trace coefficients from the slots, uhat_K = R uhat
  const int sg = sig[e];
  if (sg >= 0) {
    const RSig R = rsig[sg];
    const int32_t* rp = rint + R.rptr;
    const int32_t* ri = rint + R.ridx;
    const double* rw = rdbl + R.rw;
    const int nt = nh / 2;
    for (int t = threadIdx.x; t < nh; t += blockDim.x) {
      r[t] = w[nu + t];
      bl[t] = lm[nu + t];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nh; t += blockDim.x) {
      const int tt = t < nt ? t : t - nt, base = t < nt ? 0 : nt;
      double2 aw = make_double2(0.0, 0.0), al = make_double2(0.0, 0.0);
      for (int k = rp[tt]; k < rp[tt + 1]; ++k) {
        const double2 x = r[base + ri[k]], y = bl[base + ri[k]];
        aw.x = fma(rw[k], x.x, aw.x);
        aw.y = fma(rw[k], x.y, aw.y);
        al.x = fma(rw[k], y.x, al.x);
        al.y = fma(rw[k], y.y, al.y);
      }
      w[nu + t] = aw;
      lm[nu + t] = al;
    }
    __syncthreads();
  }
  // 2. r = l - B_K w, bl = B_K lambda;  B_K[i][j] = conj(A[nv + j][i]), l_i = conj(A[N-1][i])
  for (int i = wid; i < nv; i += nw) {
    double rr = 0, ri = 0, br = 0, bi = 0;
    const double2* col = A + (size_t)i * N + nv;
    for (int j = lane; j < m; j += 32) {
      const double2 b = a_cconj(col[j]);
      const double2 wj = w[j], lj = lm[j];
      rr += b.x * wj.x - b.y * wj.y;
      ri += b.x * wj.y + b.y * wj.x;
      br += b.x * lj.x - b.y * lj.y;
      bi += b.x * lj.y + b.y * lj.x;
    }
    rr = a_wsum(rr);
    ri = a_wsum(ri);
    br = a_wsum(br);
    bi = a_wsum(bi);
    if (lane == 0) {
      const double2 li = a_cconj(A[(size_t)(N - 1) + (size_t)i * N]);
      r[i] = make_double2(li.x - rr, li.y - ri);
      bl[i] = make_double2(br, bi);
    }
  }
  __syncthreads();
  // 3. forward substitution L y = (r, bl), column sweep
  for (int j = 0; j < nv; ++j) {
    const double d = A[(size_t)j + (size_t)j * N].x;
    const double2 yr = make_double2(r[j].x / d, r[j].y / d), yb = make_double2(bl[j].x / d, bl[j].y / d);
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nv; i += blockDim.x) {
      const double2 L = A[(size_t)i + (size_t)j * N];
      const double2 pr = a_cmul(L, yr), pb = a_cmul(L, yb);
      r[i].x -= pr.x;
      r[i].y -= pr.y;
      bl[i].x -= pb.x;
      bl[i].y -= pb.y;
    }
    if (threadIdx.x == 0) {
      r[j] = yr;
      bl[j] = yb;
    }
    __syncthreads();
  }
  // backward substitution L^H z = y: z_j = (y_j - sum_{i>j} conj(L_ij) z_i) / L_jj
  for (int j = nv - 1; j >= 0; --j) {
    double ar = 0, ai = 0, br = 0, bi = 0;
    for (int i = j + 1 + threadIdx.x; i < nv; i += blockDim.x) {
      const double2 L = a_cconj(A[(size_t)i + (size_t)j * N]);
      const double2 pr = a_cmul(L, r[i]), pb = a_cmul(L, bl[i]);
      ar += pr.x;
      ai += pr.y;
      br += pb.x;
      bi += pb.y;
    }
    block_sum2(ar, ai, red);
    block_sum2(br, bi, red);
    if (threadIdx.x == 0) {
      const double d = A[(size_t)j + (size_t)j * N].x;
      r[j] = make_double2((r[j].x - ar) / d, (r[j].y - ai) / d);
      bl[j] = make_double2((bl[j].x - br) / d, (bl[j].y - bi) / d);
    }
    __syncthreads();
  }
  // 4. dot products with the real quadrature matrices: psi = r, mu = bl
  const double* M = MC + (size_t)slot * (2 * (size_t)nf * nf + 2 * (size_t)nf * nL3);
  const double* P = M + 2 * (size_t)nf * nf;
  // d1 = (P lam_E)^H psi_F, d2 = mu_F^H M psi_F, d3 = mu_F^H X^T psi_I, d4 = mu_I^H X psi_F, d5 = mu_F^H P w_E
  double d1r = 0, d1i = 0, d2r = 0, d2i = 0, d3r = 0, d3i = 0, d4r = 0, d4i = 0, d5r = 0, d5i = 0;
  for (int i = threadIdx.x; i < nf; i += blockDim.x) {
    double2 pl = make_double2(0, 0), pw = make_double2(0, 0), mp = make_double2(0, 0), xt = make_double2(0, 0),
            xp = make_double2(0, 0);
    for (int k = 0; k < nL3; ++k) {
      const double pv = P[(size_t)i * nL3 + k];
      pl.x += pv * lm[k].x;
      pl.y += pv * lm[k].y;
      pw.x += pv * w[k].x;
      pw.y += pv * w[k].y;
    }
    for (int k = 0; k < nf; ++k) {
      const double mv = M[(size_t)min(k, i) * nf + max(k, i)];  // M symmetric, upper triangle stored
      const double xt_ = Xref[(size_t)k * nf + i];    // (X^T)[i][k] = X[k][i]
      const double x_ = Xref[(size_t)i * nf + k];     // X[i][k]
      mp.x += mv * r[k].x;
      mp.y += mv * r[k].y;
      xt.x += xt_ * r[nf + k].x;
      xt.y += xt_ * r[nf + k].y;
      xp.x += x_ * r[k].x;
      xp.y += x_ * r[k].y;
    }
    const double2 psi = r[i], muF = bl[i], muI = bl[nf + i];
    // conj(a) b
    d1r += pl.x * psi.x + pl.y * psi.y;
    d1i += pl.x * psi.y - pl.y * psi.x;
    d2r += muF.x * mp.x + muF.y * mp.y;
    d2i += muF.x * mp.y - muF.y * mp.x;
    d3r += muF.x * xt.x + muF.y * xt.y;
    d3i += muF.x * xt.y - muF.y * xt.x;
    d4r += muI.x * xp.x + muI.y * xp.y;
    d4i += muI.x * xp.y - muI.y * xp.x;
    d5r += muF.x * pw.x + muF.y * pw.y;
    d5i += muF.x * pw.y - muF.y * pw.x;
  }
  block_sum2(d1r, d1i, red);
  block_sum2(d2r, d2i, red);
  block_sum2(d3r, d3i, red);
  block_sum2(d4r, d4i, red);
  block_sum2(d5r, d5i, red);
  if (threadIdx.x == 0) {
    const double2 eps = eps_all[e];
    const double2 d1 = make_double2(d1r, d1i), d2 = make_double2(d2r, d2i), d3 = make_double2(d3r, d3i),
                  d4 = make_double2(d4r, d4i), d5 = make_double2(d5r, d5i);
    for (int which = 0; which < 2; ++which) {
      // c = i w (Re eps) or -w (Im eps); a = 2 w^2 Re eps or 2 w^2 Im eps
      const double2 c = which == 0 ? make_double2(0.0, omega) : make_double2(-omega, 0.0);
      const double a = 2.0 * omega * omega * (which == 0 ? eps.x : eps.y);
      const double2 t1 = a_cmul(a_cconj(c), d1);
      const double2 t2a = make_double2(a * d2.x, a * d2.y);
      const double2 t2b = a_cmul(c, d3), t2c = a_cmul(a_cconj(c), d4);
      const double2 t3 = a_cmul(c, d5);
      const double val = 2.0 * (t1.x - t2a.x - t2b.x - t2c.x - t3.x);
      if (which == 0)
        dre[e] = val;
      else
        dim[e] = val + (mask[e] ? ek[e] : 0.0);
    }
  }
}

static int ensure(dpg_handle* h, void** p, size_t bytes) {
  if (*p) return DPG_OK;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->err = "adjoint buffer allocation failed";
    return DPG_ERR_NOMEM;
  }
  return DPG_OK;
}

int grad_eps(dpg_handle* h, const double2* xhat, const uint8_t* mask, double* P_host, double* dre, double* dim,
             int cg_mode, double cg_rtol, int max_iter, cudaStream_t s) {
  if (!h->have_system || !h->have_elements) {
    h->err = "dpg_grad_eps needs dpg_element_batch and dpg_assemble first";
    return DPG_ERR_STATE;
  }
  if (!h->d_L1) {
    h->err = "dpg_grad_eps needs DPG_FLAG_ADJOINT at dpg_setup_mesh (the M1 factors are kept for it)";
    return DPG_ERR_STATE;
  }
  if (!xhat || !mask || (!dre) != (!dim)) {
    h->err = "bad dpg_grad_eps arguments";
    return DPG_ERR_ARG;
  }
  const size_t ne = h->ne;
  const ElemOff tot = h->off[ne];
  int rc = 0;
  rc |= ensure(h, (void**)&h->d_u, sizeof(double2) * tot.u);
  rc |= ensure(h, (void**)&h->d_zg, sizeof(double2) * tot.u);
  rc |= ensure(h, (void**)&h->d_gc, sizeof(double2) * tot.h);
  rc |= ensure(h, (void**)&h->d_Pk, sizeof(double) * (2 * ne + 1));
  rc |= ensure(h, (void**)&h->d_lam, sizeof(double2) * h->n);
  rc |= ensure(h, (void**)&h->d_rhs_adj, sizeof(double2) * h->n);
  if (rc) return DPG_ERR_NOMEM;
  rc = recover_u(h, xhat, h->d_u, s);
  if (rc) return rc;
  double* Pk = h->d_Pk;
  double* ekv = h->d_Pk + ne;
  for (const Group& G : h->grp) {
    const Sizes& S = G.sz;
    const size_t sh_src = sizeof(double2) * (S.n_u + 3 * (size_t)S.nq);
    if (sh_src > 48 * 1024)
      DPG_CUDA_TRY(h, cudaFuncSetAttribute(k_adj_source, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_src));
    k_adj_source<<<(int)G.elems.size(), 256, sh_src, s>>>(G.tab, S, h->omega, G.d_elems, h->d_off, h->d_X, h->d_eps,
                                                          mask, h->d_u, h->d_L1, h->d_Z, h->d_zg, h->d_gc, Pk, ekv);
    h->launches += 1;
  }
  k_sum_serial<<<1, 1024, 0, s>>>((int)ne, Pk, h->d_Pk + 2 * ne);
  h->launches += 1;
  DPG_CUDA_TRY(h, cudaGetLastError());
  if (P_host) {
    DPG_CUDA_TRY(h, cudaMemcpyAsync(P_host, h->d_Pk + 2 * ne, sizeof(double), cudaMemcpyDeviceToHost, s));
    DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  }
  if (!dre) return DPG_OK;
  // condensed adjoint load, colour by colour (deterministic)
  DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_rhs_adj, 0, sizeof(double2) * h->n, s));
  for (int c = 0; c < h->ncolor; ++c)
    for (const Group& G : h->grp) {
      const int cnt = G.color_off[c + 1] - G.color_off[c];
      if (cnt == 0) continue;
      k_adj_scatter<<<cnt, 256, 0, s>>>(G.sz.n_h, G.d_color_elems + G.color_off[c], h->d_off, h->d_l2g, h->d_gc,
                                        h->d_rhs_adj);
      h->launches += 1;
    }
  dpg_cg_report rep{};
  rc = cg_solve(h, cg_mode, cg_rtol, 0.0, max_iter, 1e-4, h->d_lam, h->d_rhs_adj, &rep, s);
  if (rc) return rc;
  // gradient pass: re-form K, factor G only, evaluate the derivative terms;
  // the pivot flags start clear so a failed factorisation here is reported
  DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int) * ne, s));
  Workspace& wsp = h->ws;
  for (int gi = 0; gi < (int)h->grp.size(); ++gi) {
    const Group& G = h->grp[gi];
    const Sizes& S = G.sz;
    const size_t smem_grad = sizeof(double2) * (2 * (size_t)(S.n_u + S.n_h) + 2 * (size_t)S.n_v);
    if (smem_grad > 48 * 1024)
      DPG_CUDA_TRY(h, cudaFuncSetAttribute(k_adj_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_grad));
    for (size_t c0 = 0; c0 < G.elems.size(); c0 += G.cap) {
      const int cnt = (int)std::min<size_t>(G.cap, G.elems.size() - c0);
      rc = run_element_chunk(h, gi, G.elems.data() + c0, cnt, s, false, false);
      if (rc) return rc;
      rc = factor_gram_only(h, gi, cnt, s);
      if (rc) return rc;
      k_adj_grad<<<cnt, 256, smem_grad, s>>>(S, h->omega, wsp.ids, h->d_off, h->d_sig, h->d_rsig, h->d_rint,
                                             h->d_rdbl, h->d_eps, wsp.K, wsp.MC, G.d_Xref, h->d_l2g, h->d_xfix, xhat,
                                             h->d_lam, h->d_u, h->d_zg, h->d_Z, ekv, mask, dre, dim);
      h->launches += 1;
      DPG_CUDA_TRY(h, cudaGetLastError());
    }
  }
  std::vector<int> status(ne);
  DPG_CUDA_TRY(h, cudaMemcpyAsync(status.data(), h->d_status, sizeof(int) * ne, cudaMemcpyDeviceToHost, s));
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  for (size_t e = 0; e < ne; ++e)
    if (status[e]) {
      h->err = "non-positive pivot of G_K in the gradient pass, element " + std::to_string(e);
      return DPG_ERR_NOT_HPD;
    }
  return DPG_OK;
}

}  // namespace dpg
