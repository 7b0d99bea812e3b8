// Element pass of the DPG method on sm_103a, complex FP64 (Sec. 2.3, Algorithm 2).
//
// Per element K the pass builds the augmented Hermitian matrix
//
//        [ G_K        B_K   B-hat_K   0 ]      columns/rows: test (n_v),
//   K =  [ B_K^H      0     0         0 ]      interior trial (n_u),
//        [ B-hat_K^H  0     0         0 ]      trace (n_h), load (1);
//        [ l_K^H      0     0         0 ]      the load is the last row.
//
// and eliminates it by one blocked right-looking partial Cholesky: n_v positive
// pivots (G = L L^H), a sign flip of the trailing block, which then holds
// A_full = [B B-hat l]^H G^{-1} [B B-hat l], and n_u further pivots (M1 = L1 L1^H).
// The remaining trailing block is [[S_K, s_K], [s_K^H, c_K]] with
// S_K = M3 - M2^H M1^{-1} M2 and s_K = (M5 - M2^H M1^{-1} M4) l of Eq. (linear_system),
// and c_K = l^H G^{-1} l - (M4 l)^H M1^{-1} M4 l, the constant of the element's
// residual quadratic.  Below L1 sit (L1^{-1} M2)^H and (L1^{-1} M4 l)^H.
//
// G_K and B_K come from real quadrature contractions (batched FP64 GEMMs) of
// weighted, Piola-mapped basis values: with s_q = sqrt(w_q det J_q),
//   M = V^T V, C = Cu^T Cu, P = V^T PhiL, Q = Cu^T PhiL, X = Cu^T V (metric free),
// and G_FF = C + (|w eps|^2 + alpha) M, G_II = C + (|w mu|^2 + alpha) M,
// G_FI = i w conj(mu) X + i w eps X^T (+ Robin terms), B = [[i w eps P, Q], [Q, -i w mu P]]
// (Eq. test_inner_product and Eq. bilinear_form with real basis functions and
// conjugation on the first argument).  The skeleton pairing of Eq.
// (trace_pairing) is metric free for covariant Piola functions and Nanson's
// formula, so B-hat comes from reference face matrices T_f.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "dpg_internal.h"
#include "geom.cuh"

namespace dpg {

// ---------------------------------------------------------------- helpers --
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// Test function i of the order-rt Nedelec space: component and 1D indices.
__device__ __forceinline__ void test_index(int i, int rt, int& c, int ii[3]) {
  const int nc = rt * (rt + 1) * (rt + 1);
  c = i / nc;
  int rem = i - c * nc;
  int n0 = (c == 0) ? rt : rt + 1;
  int n1 = (c == 1) ? rt : rt + 1;
  ii[0] = rem % n0;
  rem /= n0;
  ii[1] = rem % n1;
  ii[2] = rem / n1;
}

// Value f and reference gradient of the scalar factor of a Nedelec function
// (component c, 1D indices ii) at the extended-grid point (q0, q1, q2).
// fo/fc: open/closed family of the space (F_OPEN_T/F_CLOSED_T or F_OPEN_R/F_CLOSED_R).
__device__ __forceinline__ void ned_eval(const Tables& T, int fo, int fc, int c, const int ii[3],
                                         const int q[3], double& f, double g[3]) {
  double v[3], d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int fam = (k == c) ? fo : fc;
    v[k] = T.val[fam][q[k]][ii[k]];
    d[k] = T.der[fam][q[k]][ii[k]];
  }
  f = v[0] * v[1] * v[2];
  g[0] = d[0] * v[1] * v[2];
  g[1] = v[0] * d[1] * v[2];
  g[2] = v[0] * v[1] * d[2];
}

// reference curl of f e_c: grad f x e_c
__device__ __forceinline__ void ref_curl(int c, const double g[3], double cu[3]) {
  if (c == 0) {
    cu[0] = 0.0; cu[1] = g[2]; cu[2] = -g[1];
  } else if (c == 1) {
    cu[0] = -g[2]; cu[1] = 0.0; cu[2] = g[0];
  } else {
    cu[0] = g[1]; cu[1] = -g[0]; cu[2] = 0.0;
  }
}

// complex square root, principal branch
__device__ __forceinline__ double2 csqrt(double2 z) {
  double m = hypot(z.x, z.y);
  double re = sqrt(0.5 * (m + z.x));
  double im = sqrt(0.5 * fmax(m - z.x, 0.0));
  return make_double2(re, z.y < 0 ? -im : im);
}

// TE_mn mode of Sec. 4.1 at x (guide [0,a] x [0,b], propagation along +x3).
__device__ void te_fields(const dpg_robin_group& g, double omega, const double x[3], double2 E[3],
                          double2 H[3]) {
  const double pi = 3.14159265358979323846;
  double k1 = g.m * pi / g.a, k2 = g.n * pi / g.b, kc2 = k1 * k1 + k2 * k2;
  double2 eps = make_double2(g.eps_re, g.eps_im), mu = make_double2(g.mu_re, g.mu_im);
  double2 em = cmul(eps, mu);
  double2 k3 = csqrt(make_double2(omega * omega * em.x - kc2, omega * omega * em.y));
  double sn, cs;
  sincos(k3.x * x[2], &sn, &cs);
  double dec = exp(-k3.y * x[2]);
  double2 ph = make_double2(cs * dec, sn * dec);  // e^{i k3 x3}
  double s1, c1, s2, c2;
  sincos(k1 * x[0], &s1, &c1);
  sincos(k2 * x[1], &s2, &c2);
  double2 pre = cscale(cmul(make_double2(0.0, omega), mu), 1.0 / kc2);  // i w mu / kc^2
  E[0] = cmul(cscale(pre, -k2 * c1 * s2), ph);
  E[1] = cmul(cscale(pre, k1 * s1 * c2), ph);
  E[2] = make_double2(0.0, 0.0);
  double2 ik3 = make_double2(-k3.y, k3.x);  // i k3
  H[0] = cmul(cscale(ik3, -k1 / kc2 * s1 * c2), ph);
  H[1] = cmul(cscale(ik3, -k2 / kc2 * c1 * s2), ph);
  H[2] = cscale(ph, c1 * c2);
}

// ------------------------------------------------- volume basis arrays --
// V[(q*3+a)][i] = s_q (J^{-T} e_c f_i)_a, Cu[(q*3+a)][i] = s_q (J curl_ref / det J)_a,
// PhiL[(q*3+a)][d*nL+l] = delta_ad s_q L_l(q).
constexpr int QB = 8;

__global__ void __launch_bounds__(256) k_vol_arrays(const __grid_constant__ Tables T, Sizes S, const double* __restrict__ Xall,
                                                    const int* __restrict__ ids, double* V, double* Cu, double* PhiL) {
  const int slot = blockIdx.y;
  const int e = ids[slot];
  __shared__ double sX[24];
  __shared__ double sJi[QB][9], sJs[QB][9], sw[QB];  // J^{-1}, J/detJ scaled, s_q
  if (threadIdx.x < 24) sX[threadIdx.x] = Xall[(size_t)e * 24 + threadIdx.x];
  __syncthreads();
  const int nq1 = S.nq1, nq = S.nq;
  const int q0b = blockIdx.x * QB;
  if (threadIdx.x < QB) {
    int q = q0b + threadIdx.x;
    if (q < nq) {
      int qi[3] = {q % nq1, (q / nq1) % nq1, q / (nq1 * nq1)};
      double xi[3] = {T.pt[qi[0]], T.pt[qi[1]], T.pt[qi[2]]};
      double J[3][3], x[3], Ji[3][3];
      geom(sX, xi, J, x);
      double det = inv3(J, Ji);
      double s = sqrt(T.w[qi[0]] * T.w[qi[1]] * T.w[qi[2]] * det);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          sJi[threadIdx.x][3 * a + b] = Ji[a][b];
          sJs[threadIdx.x][3 * a + b] = J[a][b] * (s / det);
        }
      sw[threadIdx.x] = s;
    }
  }
  __syncthreads();
  const size_t nf = S.n_f;
  const size_t stride = (size_t)3 * nq * nf;
  double* Ve = V + slot * stride;
  double* Ce = Cu + slot * stride;
  const int nqb = min(QB, nq - q0b);
  for (int idx = threadIdx.x; idx < nqb * S.n_f; idx += blockDim.x) {
    int ql = idx / S.n_f, i = idx - ql * S.n_f;
    int q = q0b + ql;
    int qi[3] = {q % nq1, (q / nq1) % nq1, q / (nq1 * nq1)};
    int c, ii[3];
    test_index(i, S.rt, c, ii);
    double f, g[3], cr[3];
    ned_eval(T, F_OPEN_T, F_CLOSED_T, c, ii, qi, f, g);
    ref_curl(c, g, cr);
    const double* Ji = sJi[ql];
    const double* Js = sJs[ql];
    double s = sw[ql];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Ve[((size_t)q * 3 + a) * nf + i] = s * Ji[3 * c + a] * f;  // (J^{-T})_{a c} = (J^{-1})_{c a}
      Ce[((size_t)q * 3 + a) * nf + i] = Js[3 * a + 0] * cr[0] + Js[3 * a + 1] * cr[1] + Js[3 * a + 2] * cr[2];
    }
  }
  const int nL = S.nL, w3 = 3 * nL;
  double* Pe = PhiL + slot * (size_t)3 * nq * w3;
  for (int idx = threadIdx.x; idx < nqb * 3 * w3; idx += blockDim.x) {
    int ql = idx / (3 * w3), rem = idx - ql * 3 * w3;
    int a = rem / w3, col = rem - a * w3;
    int d = col / nL, l = col - d * nL;
    int q = q0b + ql;
    int qi[3] = {q % nq1, (q / nq1) % nq1, q / (nq1 * nq1)};
    int p1 = S.p + 1;
    int l0 = l % p1, l1 = (l / p1) % p1, l2 = l / (p1 * p1);
    double v = 0.0;
    if (a == d) v = sw[ql] * T.val[F_L2][qi[0]][l0] * T.val[F_L2][qi[1]][l1] * T.val[F_L2][qi[2]][l2];
    Pe[((size_t)q * 3 + a) * w3 + col] = v;
  }
}

// --------------------------------------------------------- face arrays --
// Per (element, face) entry: columns [Vt (n_f) | Nx (n_f) | Pt (nt) | NxP (nt) | g_re | g_im],
// rows (qf*3+a), all scaled by sqrt(w dS):  Vt = tangential test values,
// Nx = n x test, Pt = tangential trace values, NxP = n x trace, g = Robin datum.
__global__ void __launch_bounds__(256) k_face_arrays(const __grid_constant__ Tables T, Sizes S, const double* __restrict__ Xall,
                                                     const int* __restrict__ rent, const dpg_robin_group* __restrict__ groups,
                                                     const int* __restrict__ trfun, double omega, int use_unit_cube,
                                                     double* FV) {
  const int ent = blockIdx.y;
  const int e = rent[4 * ent + 3], f = rent[4 * ent + 1], grp = rent[4 * ent + 2];
  const int d = f >> 1, sd = f & 1;
  const int nq1 = S.nq1, nqf = S.nqf;
  const int W = 2 * S.n_f + 2 * S.nt + 2;
  __shared__ double sX[24];
  __shared__ double sJi[9], sn[3], ssw;
  __shared__ int sq[3];
  if (threadIdx.x < 24) {
    if (use_unit_cube) {
      int v = threadIdx.x / 3, a = threadIdx.x % 3;
      sX[threadIdx.x] = (double)((v >> a) & 1);
    } else {
      sX[threadIdx.x] = Xall[(size_t)e * 24 + threadIdx.x];
    }
  }
  double* Fe = FV + (size_t)ent * 3 * nqf * W;
  for (int qf = 0; qf < nqf; ++qf) {
    __syncthreads();
    if (threadIdx.x == 0) {
      int ta = qf % nq1, tb = qf / nq1;
      int a = (d == 0) ? 1 : 0, b = (d == 2) ? 1 : 2;
      int qi[3];
      qi[d] = nq1 + sd;  // extended point index of xi_d = sd
      qi[a] = ta;
      qi[b] = tb;
      double xi[3] = {T.pt[qi[0]], T.pt[qi[1]], T.pt[qi[2]]};
      double J[3][3], x[3], Ji[3][3];
      geom(sX, xi, J, x);
      double det = inv3(J, Ji);
      // Nanson: n dS = det J J^{-T} N_ref, N_ref = (2 sd - 1) e_d
      double sg = sd ? 1.0 : -1.0;
      double nv[3] = {det * Ji[d][0] * sg, det * Ji[d][1] * sg, det * Ji[d][2] * sg};
      double dS = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
      for (int k = 0; k < 3; ++k) sn[k] = nv[k] / dS;
      for (int k = 0; k < 9; ++k) sJi[k] = Ji[k / 3][k % 3];
      double sw = sqrt(T.w[ta] * T.w[tb] * dS);
      ssw = sw;
      sq[0] = qi[0];
      sq[1] = qi[1];
      sq[2] = qi[2];
      // Robin datum g = n x H_TE + zinv (E_TE)_t  (port) or 0
      double2 gv[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
      if (!use_unit_cube && groups[grp].port) {
        double2 E[3], H[3];
        te_fields(groups[grp], omega, x, E, H);
        double2 zinv = make_double2(groups[grp].zinv_re, groups[grp].zinv_im);
        double2 En = cadd(cadd(cscale(E[0], sn[0]), cscale(E[1], sn[1])), cscale(E[2], sn[2]));
        double2 Et[3], nH[3];
        for (int k = 0; k < 3; ++k) Et[k] = csub(E[k], cscale(En, sn[k]));
        nH[0] = csub(cscale(H[2], sn[1]), cscale(H[1], sn[2]));
        nH[1] = csub(cscale(H[0], sn[2]), cscale(H[2], sn[0]));
        nH[2] = csub(cscale(H[1], sn[0]), cscale(H[0], sn[1]));
        for (int k = 0; k < 3; ++k) gv[k] = cadd(nH[k], cmul(zinv, Et[k]));
      }
      for (int k = 0; k < 3; ++k) {
        Fe[((size_t)qf * 3 + k) * W + W - 2] = sw * gv[k].x;
        Fe[((size_t)qf * 3 + k) * W + W - 1] = sw * gv[k].y;
      }
    }
    __syncthreads();
    const int qi[3] = {sq[0], sq[1], sq[2]};
    const double n0 = sn[0], n1 = sn[1], n2 = sn[2], sw = ssw;
    const int nfun = S.n_f + S.nt;
    for (int k = threadIdx.x; k < nfun; k += blockDim.x) {
      int c, ii[3];
      double fv, g[3];
      if (k < S.n_f) {
        test_index(k, S.rt, c, ii);
        ned_eval(T, F_OPEN_T, F_CLOSED_T, c, ii, qi, fv, g);
      } else {
        int pk = trfun[k - S.n_f];
        c = pk & 3;
        ii[0] = (pk >> 2) & 15;
        ii[1] = (pk >> 6) & 15;
        ii[2] = (pk >> 10) & 15;
        ned_eval(T, F_OPEN_R, F_CLOSED_R, c, ii, qi, fv, g);
      }
      // physical value psi = J^{-T} e_c f
      double ps[3] = {sJi[3 * c + 0] * fv, sJi[3 * c + 1] * fv, sJi[3 * c + 2] * fv};
      double pn = ps[0] * n0 + ps[1] * n1 + ps[2] * n2;
      double pt[3] = {ps[0] - pn * n0, ps[1] - pn * n1, ps[2] - pn * n2};
      double nx[3] = {n1 * ps[2] - n2 * ps[1], n2 * ps[0] - n0 * ps[2], n0 * ps[1] - n1 * ps[0]};
      int colT = (k < S.n_f) ? k : 2 * S.n_f + (k - S.n_f);      // tangential value column
      int colN = (k < S.n_f) ? S.n_f + k : 2 * S.n_f + S.nt + (k - S.n_f);  // n x value column
      for (int a = 0; a < 3; ++a) {
        Fe[((size_t)qf * 3 + a) * W + colT] = sw * pt[a];
        Fe[((size_t)qf * 3 + a) * W + colN] = sw * nx[a];
      }
    }
  }
}

// -------------------------------------------------- batched FP64 GEMM --
// C[b] (Ma x Nb, row-major, ldc) = A[b]^T B[b]; A: Kd x Ma (lda), B: Kd x Nb (ldb).
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) k_gemm_tn(int Ma, int Nb, int Kd, const double* __restrict__ A, int lda, long long sA,
                                                 const double* __restrict__ B, int ldb, long long sB, double* C, int ldc,
                                                 long long sC, int upper_only, const double* __restrict__ wk,
                                                 long long sw) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int b = blockIdx.z;
  const double* Ab = A + b * sA;
  const double* Bb = B + b * sB;
  double* Cb = C + b * sC;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  // symmetric products: tiles strictly below the diagonal are never read
  if (upper_only && n0 + GT <= m0) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < Kd; k0 += GK) {
    for (int t = threadIdx.x; t < GK * GT; t += 256) {
      int kk = t / GT, mm = t - kk * GT;
      int k = k0 + kk;
      As[kk][mm] = (k < Kd && m0 + mm < Ma) ? Ab[(size_t)k * lda + m0 + mm] : 0.0;
      Bs[kk][mm] = (k < Kd && n0 + mm < Nb) ? Bb[(size_t)k * ldb + n0 + mm] * (wk ? wk[b * sw + k] : 1.0) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty + 16 * i;
    if (m >= Ma) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n < Nb) Cb[(size_t)m * ldc + n] = acc[i][j];
    }
  }
}

// C = A^T diag(wk) B when wk is given (one weight per k, stride sw per batch entry).
static void gemm_tn(int Ma, int Nb, int Kd, const double* A, int lda, long long sA, const double* B, int ldb,
                    long long sB, double* C, int ldc, long long sC, int batch, cudaStream_t s, int upper_only = 0,
                    const double* wk = nullptr, long long sw = 0) {
  dim3 grid((Nb + GT - 1) / GT, (Ma + GT - 1) / GT, batch);
  k_gemm_tn<<<grid, 256, 0, s>>>(Ma, Nb, Kd, A, lda, sA, B, ldb, sB, C, ldc, sC, upper_only, wk, sw);
}

// ------------------------------------------------------ build K matrix --
// K (column-major, N x N) from M, C, P, Q, X_ref, T_f; full matrix written.
__global__ void __launch_bounds__(256) k_build_K(Sizes S, double omega, double alpha, const int* __restrict__ ids,
                                                 const double2* __restrict__ eps_all, const double2* __restrict__ mu_all,
                                                 const int8_t* __restrict__ fbc, const double* __restrict__ MC,
                                                 const double* __restrict__ Xref, const double* __restrict__ Tf,
                                                 const double* __restrict__ Tall, double2* K) {
  const int slot = blockIdx.y;
  const int e = ids[slot];
  const int N = S.N, nf = S.n_f, nv = S.n_v, nu = S.n_u, nt = S.nt, nL3 = 3 * S.nL;
  const double2 eps = eps_all[e], mu = mu_all[e];
  const double a1 = omega * omega * (eps.x * eps.x + eps.y * eps.y) + alpha;
  const double a2 = omega * omega * (mu.x * mu.x + mu.y * mu.y) + alpha;
  // i w mu, i w eps
  const double2 iwmu = make_double2(-omega * mu.y, omega * mu.x);
  const double2 iweps = make_double2(-omega * eps.y, omega * eps.x);
  const double* M = MC + (size_t)slot * (2 * (size_t)nf * nf + 2 * (size_t)nf * nL3);
  const double* Cm = M + (size_t)nf * nf;
  const double* P = Cm + (size_t)nf * nf;
  const double* Q = P + (size_t)nf * nL3;
  int robin_mask = 0;
  for (int f = 0; f < 6; ++f)
    if (fbc[(size_t)e * 6 + f] == DPG_BC_ROBIN) robin_mask |= 1 << f;
  double2* Ke = K + (size_t)slot * N * N;
  const size_t total = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / N), i = (int)(idx - (size_t)j * N);
    double2 v = make_double2(0.0, 0.0);
    if (j < nv && i < nv) {
      // M and C are symmetric and only their upper triangle (row <= col) is
      // computed: read [min][max] (coalesced over rows i for the lower part of K)
      if (i < nf && j < nf) {
        const size_t q = (size_t)min(i, j) * nf + max(i, j);
        v.x = Cm[q] + a1 * M[q];
      } else if (i >= nf && j >= nf) {
        const size_t q = (size_t)min(i - nf, j - nf) * nf + max(i - nf, j - nf);
        v.x = Cm[q] + a2 * M[q];
      } else if (i >= nf) {
        // G_IF[i'][j] = -i w mu X[j][i'] - i w conj(eps) X[i'][j]
        const int ip = i - nf;
        double xji = Xref[(size_t)j * nf + ip], xij = Xref[(size_t)ip * nf + j];
        v = make_double2(-(iwmu.x * xji) - (-omega * (-eps.y)) * xij, -(iwmu.y * xji) - (omega * eps.x) * xij);
      } else {
        // G_FI[i][j'] = i w conj(mu) X[i][j'] + i w eps X[j'][i]
        const int jp = j - nf;
        double xij = Xref[(size_t)i * nf + jp], xji = Xref[(size_t)jp * nf + i];
        v = make_double2((omega * mu.y) * xij + iweps.x * xji, (omega * mu.x) * xij + iweps.y * xji);
      }
    } else if (j < nv && i < nv + nu) {
      // K[nv+u][j] = conj(BK[j][u])
      const int u = i - nv;
      const bool Fj = j < nf;
      const int jj = Fj ? j : j - nf;
      if (u < nL3) {
        if (Fj) {  // conj(i w eps P)
          double pv = P[(size_t)jj * nL3 + u];
          v = make_double2(iweps.x * pv, -iweps.y * pv);
        } else {
          v.x = Q[(size_t)jj * nL3 + u];
        }
      } else {
        const int up = u - nL3;
        if (Fj) {
          v.x = Q[(size_t)jj * nL3 + up];
        } else {  // conj(-i w mu P)
          double pv = P[(size_t)jj * nL3 + up];
          v = make_double2(-iwmu.x * pv, iwmu.y * pv);
        }
      }
    } else if (j < nv && i < nv + nu + 2 * nt) {
      const int t = i - nv - nu;
      if (t < nt) {  // E-hat: <I, n x E-hat> on all faces (real)
        if (j >= nf) v.x = Tall[(size_t)(j - nf) * nt + t];
      } else {       // H-hat: <F, n x H-hat> on faces not on Gamma_R
        if (j < nf) {
          const int tp = t - nt;
          double s = Tall[(size_t)j * nt + tp];
          for (int f = 0; f < 6; ++f)
            if (robin_mask & (1 << f)) s -= Tf[((size_t)f * nf + j) * nt + tp];
          v.x = s;
        }
      }
    }
    Ke[idx] = v;
  }
}


// K of a lossless element in the phase-scaled real basis: test functions
// scaled by diag(1 on F, -i on I), trial by diag(-i on E, 1 on H, -i on
// E-hat, 1 on H-hat).  Then G_r = [[C + a1 M, w (mu X + eps X^T)], sym.],
// B_r = [[w eps P, Q], [Q, w mu P]], B-hat_r = [[0, T_F], [T_I, 0]] are real.
__global__ void __launch_bounds__(256) k_build_K_real(Sizes S, double omega, double alpha, const int* __restrict__ ids,
                                                      const double2* __restrict__ eps_all,
                                                      const double2* __restrict__ mu_all, const double* __restrict__ MC,
                                                      const double* __restrict__ Xref, const double* __restrict__ Tall,
                                                      double* K) {
  const int slot = blockIdx.y;
  const int e = ids[slot];
  const int N = S.N, nf = S.n_f, nv = S.n_v, nu = S.n_u, nt = S.nt, nL3 = 3 * S.nL;
  const double eps = eps_all[e].x, mu = mu_all[e].x;
  const double a1 = omega * omega * eps * eps + alpha, a2 = omega * omega * mu * mu + alpha;
  const double* M = MC + (size_t)slot * (2 * (size_t)nf * nf + 2 * (size_t)nf * nL3);
  const double* Cm = M + (size_t)nf * nf;
  const double* P = Cm + (size_t)nf * nf;
  const double* Q = P + (size_t)nf * nL3;
  double* Ke = K + (size_t)slot * N * N;
  const size_t total = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / N), i = (int)(idx - (size_t)j * N);
    double v = 0.0;
    if (j < nv && i < nv) {
      if (i < nf && j < nf) {
        const size_t q = (size_t)min(i, j) * nf + max(i, j);
        v = Cm[q] + a1 * M[q];
      } else if (i >= nf && j >= nf) {
        const size_t q = (size_t)min(i - nf, j - nf) * nf + max(i - nf, j - nf);
        v = Cm[q] + a2 * M[q];
      } else if (i >= nf) {  // rows I, cols F: w (mu X[j][i'] + eps X[i'][j])
        const int ip = i - nf;
        v = omega * (mu * Xref[(size_t)j * nf + ip] + eps * Xref[(size_t)ip * nf + j]);
      } else {  // rows F, cols I: w (mu X[i][j'] + eps X[j'][i])
        const int jp = j - nf;
        v = omega * (mu * Xref[(size_t)i * nf + jp] + eps * Xref[(size_t)jp * nf + i]);
      }
    } else if (j < nv && i < nv + nu) {  // K[nv+u][j] = B_r[j][u]
      const int u = i - nv;
      const bool Fj = j < nf;
      const int jj = Fj ? j : j - nf;
      if (u < nL3)
        v = Fj ? omega * eps * P[(size_t)jj * nL3 + u] : Q[(size_t)jj * nL3 + u];
      else
        v = Fj ? Q[(size_t)jj * nL3 + (u - nL3)] : omega * mu * P[(size_t)jj * nL3 + (u - nL3)];
    } else if (j < nv && i < nv + nu + 2 * nt) {
      const int t = i - nv - nu;
      if (t < nt) {
        if (j >= nf) v = Tall[(size_t)(j - nf) * nt + t];
      } else if (j < nf) {
        v = Tall[(size_t)j * nt + (t - nt)];
      }
    }
    Ke[idx] = v;
  }
}

// Robin additions (one block per element with Robin faces, its entries in order).
// FR per entry: n_f x W with W = 2 n_f + 2 nt + 2 = Vt^T [Vt | Nx | Pt | NxP | g].
__global__ void __launch_bounds__(256) k_robin_add(Sizes S, const int* __restrict__ rlist, const int* __restrict__ rent,
                                                   const dpg_robin_group* __restrict__ groups, const double* __restrict__ FR,
                                                   double2* K) {
  const int el = blockIdx.x;
  const int first = rlist[2 * el], count = rlist[2 * el + 1];
  const int N = S.N, nf = S.n_f, nv = S.n_v, nu = S.n_u, nt = S.nt;
  const int W = 2 * nf + 2 * nt + 2;
  for (int k = 0; k < count; ++k) {
    const int ent = first + k;
    const int slot = rent[4 * ent + 0], grp = rent[4 * ent + 2];
    const double2 zinv = make_double2(groups[grp].zinv_re, groups[grp].zinv_im);
    const double z2 = zinv.x * zinv.x + zinv.y * zinv.y;
    const double* Fr = FR + (size_t)ent * nf * W;
    double2* Ke = K + (size_t)slot * N * N;
    for (int idx = threadIdx.x; idx < nf * nf; idx += blockDim.x) {
      int i = idx / nf, j = idx - i * nf;  // j fastest: K rows j -> strided, acceptable (boundary only)
      double R = Fr[(size_t)i * W + j];
      double Xc_ij = Fr[(size_t)i * W + nf + j];
      double Xc_ji = Fr[(size_t)j * W + nf + i];
      // column-major K: entry (row, col) at row + col * N
      double2* g_ff = &Ke[(size_t)i + (size_t)j * N];
      g_ff->x += z2 * R;
      double2* g_ii = &Ke[(size_t)(nf + i) + (size_t)(nf + j) * N];
      g_ii->x += R;
      // G_IF[i][j] += conj(zinv) Xc[j][i]
      double2* g_if = &Ke[(size_t)(nf + i) + (size_t)j * N];
      g_if->x += zinv.x * Xc_ji;
      g_if->y += -zinv.y * Xc_ji;
      // G_FI[i][j] += zinv Xc[i][j]
      double2* g_fi = &Ke[(size_t)i + (size_t)(nf + j) * N];
      g_fi->x += zinv.x * Xc_ij;
      g_fi->y += zinv.y * Xc_ij;
    }
    for (int idx = threadIdx.x; idx < nf * nt; idx += blockDim.x) {
      int i = idx / nt, t = idx - i * nt;
      double Bt = Fr[(size_t)i * W + 2 * nf + t];
      // K[nv+nu+t][i] += conj(-zinv Bt)
      double2* kk = &Ke[(size_t)(nv + nu + t) + (size_t)i * N];
      kk->x += -zinv.x * Bt;
      kk->y += zinv.y * Bt;
    }
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
      double lre = Fr[(size_t)i * W + W - 2], lim = Fr[(size_t)i * W + W - 1];
      // l_i = -(lre + i lim);  K[N-1][i] += conj(l_i)
      double2* kk = &Ke[(size_t)(N - 1) + (size_t)i * N];
      kk->x += -lre;
      kk->y += lim;
    }
    __syncthreads();
  }
}

// --------------------------------------------- blocked partial Cholesky --
// One CTA per element.  Pivots [0, nv) with positive sign; the trailing block
// is negated after them; pivots [nv, npiv) again positive.  Lower triangle,
// column-major, leading dimension N; only rows and columns [0, nact) take part
// (nact = nv factors G alone and leaves the rows below untouched).
// Non-positive pivots set status[elem].
constexpr int NB = 32;   // panel width
constexpr int TT = 64;   // trailing tile

// Real / complex scalar operations for the factorisation kernel.
template <typename T> struct Sc;
template <> struct Sc<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double re(double a) { return a; }
  __device__ static double real(double r) { return r; }
  __device__ static double neg(double a) { return -a; }
  __device__ static double sub(double a, double b) { return a - b; }
  __device__ static double scale(double a, double s) { return a * s; }
  __device__ static double mul_conj(double a, double b) { return a * b; }  // a * conj(b)
  __device__ static void fma_conj(double& acc, double a, double b) { acc = fma(a, b, acc); }
};
template <> struct Sc<double2> {
  __device__ static double2 zero() { return make_double2(0.0, 0.0); }
  __device__ static double re(double2 a) { return a.x; }
  __device__ static double2 real(double r) { return make_double2(r, 0.0); }
  __device__ static double2 neg(double2 a) { return make_double2(-a.x, -a.y); }
  __device__ static double2 sub(double2 a, double2 b) { return csub(a, b); }
  __device__ static double2 scale(double2 a, double s) { return cscale(a, s); }
  __device__ static double2 mul_conj(double2 a, double2 b) { return cmul(a, cconj(b)); }
  __device__ static void fma_conj(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.y, b.x, fma(-a.x, b.y, acc.y));
  }
};


// Column tiles per pass of the trailing update.
template <typename T> struct FactorJW { static constexpr int value = 1; };

template <typename T>
constexpr size_t factor_smem() {
  return sizeof(T) * (NB * NB + (1 + FactorJW<T>::value) * NB * TT);
}

// A[row][col] -= sum_kk PI[kk][row] conj(PJ_j[kk][col]) for NJ adjacent
// column tiles (lower triangle only); thread (tx, ty) owns rows tx + 16 a and
// columns ty + 16 b of each tile.  The panel tiles are zero beyond column w,
// so the k loop runs the compile-time width and unrolls.
template <typename T, int NJ>
__device__ __forceinline__ void tile_update(T* A, int N, int nact, int r0, int c0, const T* sPI, const T* sPJ,
                                            int tid) {
  using O = Sc<T>;
  const int tx = tid & 15, ty = tid >> 4;
  T acc[NJ][4][4];
#pragma unroll
  for (int j = 0; j < NJ; ++j)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[j][a][b] = O::zero();
#pragma unroll
  for (int kk = 0; kk < NB; ++kk) {
    T pa[4], pb[NJ][4];
#pragma unroll
    for (int a = 0; a < 4; ++a) pa[a] = sPI[kk * TT + tx + 16 * a];
#pragma unroll
    for (int j = 0; j < NJ; ++j)
#pragma unroll
      for (int b = 0; b < 4; ++b) pb[j][b] = sPJ[j * NB * TT + kk * TT + ty + 16 * b];
#pragma unroll
    for (int j = 0; j < NJ; ++j)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) O::fma_conj(acc[j][a][b], pa[a], pb[j][b]);  // acc += pa conj(pb)
  }
#pragma unroll
  for (int j = 0; j < NJ; ++j)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int row = r0 + tx + 16 * a;
      if (row >= nact) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int col = c0 + j * TT + ty + 16 * b;
        if (col >= nact || col > row) continue;
        T* p = &A[(size_t)row + (size_t)col * N];
        *p = O::sub(*p, acc[j][a][b]);
      }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_factor(int N, int nact, int nv, int npiv, const int* __restrict__ ids,
                                                T* K, int* status) {
  using O = Sc<T>;
  extern __shared__ __align__(16) unsigned char fsm[];
  T* sD = reinterpret_cast<T*>(fsm);  // NB x NB diagonal block (column-major)
  T* sPI = sD + NB * NB;              // NB x TT panel rows of tile I ([k][row])
  T* sPJ = sPI + NB * TT;             // JW x NB x TT panel rows of the column tiles
  const int slot = blockIdx.x;
  T* A = K + (size_t)slot * N * N;
  const int tid = threadIdx.x;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  for (int k0 = 0; k0 < npiv;) {
    const int stage_end = (k0 < nv) ? nv : npiv;
    const int w = min(NB, stage_end - k0);
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
    // --- diagonal block: load, factor (unblocked), store
    for (int t = tid; t < w * w; t += blockDim.x) {
      int jj = t / w, ii = t - jj * w;
      sD[ii + jj * NB] = (ii >= jj) ? A[(size_t)(k0 + ii) + (size_t)(k0 + jj) * N] : O::zero();
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
      if (tid == 0) {
        double d = O::re(sD[j + j * NB]);
        if (!(d > 0.0)) {
          bad = 1;
          d = 1e-300;
        }
        sD[j + j * NB] = O::real(sqrt(d));
      }
      __syncthreads();
      const double ljj = O::re(sD[j + j * NB]);
      for (int ii = j + 1 + tid; ii < w; ii += blockDim.x) sD[ii + j * NB] = O::scale(sD[ii + j * NB], 1.0 / ljj);
      __syncthreads();
      // rank-1 update of the remaining lower part of the block
      const int rem = w - j - 1;
      for (int t = tid; t < rem * rem; t += blockDim.x) {
        int cc = j + 1 + t / rem, ii = j + 1 + t % rem;
        if (ii >= cc) sD[ii + cc * NB] = O::sub(sD[ii + cc * NB], O::mul_conj(sD[ii + j * NB], sD[cc + j * NB]));
      }
      __syncthreads();
    }
    for (int t = tid; t < w * w; t += blockDim.x) {
      int jj = t / w, ii = t - jj * w;
      if (ii >= jj) A[(size_t)(k0 + ii) + (size_t)(k0 + jj) * N] = sD[ii + jj * NB];
    }
    // --- panel: rows [k1, N) of columns [k0, k1): X L_D^H = P  (one row per thread)
    for (int row = k1 + tid; row < nact; row += blockDim.x) {
      T x[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < w) x[j] = A[(size_t)row + (size_t)(k0 + j) * N];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < w) {
          T v = x[j];
#pragma unroll
          for (int kk = 0; kk < NB; ++kk)
            if (kk < j) v = O::sub(v, O::mul_conj(x[kk], sD[j + kk * NB]));
          x[j] = O::scale(v, 1.0 / O::re(sD[j + j * NB]));
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < w) A[(size_t)row + (size_t)(k0 + j) * N] = x[j];
    }
    __syncthreads();
    // --- trailing update of the lower triangle of rows/cols [k1, N)
    const int R = nact - k1;
    const int ntile = (R + TT - 1) / TT;
    for (int I = 0; I < ntile; ++I) {
      const int r0 = k1 + I * TT;
      __syncthreads();
      for (int t = tid; t < NB * TT; t += blockDim.x) {
        int kk = t / TT, rr = t - kk * TT;
        sPI[kk * TT + rr] = (kk < w && r0 + rr < nact) ? A[(size_t)(r0 + rr) + (size_t)(k0 + kk) * N] : O::zero();
      }
      for (int Jt = 0; Jt <= I; ++Jt) {
        const int c0 = k1 + Jt * TT;
        __syncthreads();
        for (int t = tid; t < NB * TT; t += blockDim.x) {
          int kk = t / TT, rr = t - kk * TT;
          sPJ[kk * TT + rr] =
              (kk < w && c0 + rr < nact) ? A[(size_t)(c0 + rr) + (size_t)(k0 + kk) * N] : O::zero();
        }
        __syncthreads();
        tile_update<T, 1>(A, N, nact, r0, c0, sPI, sPJ, tid);
      }
    }
    __syncthreads();
    k0 = k1;
  }
  __syncthreads();
  if (tid == 0 && bad) status[ids[slot]] = 1;
}

// ---------------------------------------------------------- extraction --
// From the factored K of one element: S (n_h x n_h full), s, c, Z = M1^{-1} M2, z = M1^{-1} M4 l.
__global__ void __launch_bounds__(256) k_extract(Sizes S, const int* __restrict__ ids, const double2* __restrict__ K,
                                                 const ElemOff* __restrict__ off, double2* Sst, double2* sst,
                                                 double* cst, double2* Zst, double2* zst, double2* L1st) {
  const int slot = blockIdx.x;
  const int e = ids[slot];
  const ElemOff of = off[e];
  const int N = S.N, nv = S.n_v, nu = S.n_u, nh = S.n_h;
  const double2* A = K + (size_t)slot * N * N;
  const int o = nv + nu;  // first trace row
  double2* Se = Sst + of.S;
  sst += of.h;
  zst += of.u;
  for (int t = threadIdx.x; t < nh * nh; t += blockDim.x) {
    int i = t / nh, j = t - i * nh;
    Se[t] = (i >= j) ? A[(size_t)(o + i) + (size_t)(o + j) * N] : cconj(A[(size_t)(o + j) + (size_t)(o + i) * N]);
  }
  for (int t = threadIdx.x; t < nh; t += blockDim.x) sst[t] = cconj(A[(size_t)(N - 1) + (size_t)(o + t) * N]);
  if (threadIdx.x == 0) cst[e] = A[(size_t)(N - 1) + (size_t)(N - 1) * N].x;
  if (L1st) {  // Cholesky factor of M1 (row-major, lower; upper zero), kept for the adjoint
    double2* Le = L1st + of.L1;
    for (int t = threadIdx.x; t < nu * nu; t += blockDim.x) {
      const int i = t / nu, j = t - i * nu;
      Le[t] = (i >= j) ? A[(size_t)(nv + i) + (size_t)(nv + j) * N] : make_double2(0.0, 0.0);
    }
  }
  // Z: for each column t in [0, nh] (t = nh is the load) solve L1^H z = y with
  // y[u] = conj(A[o + t][nv + u]), L1[a][b] = A[nv + a][nv + b].
  double2* Ze = Zst + of.Z;
  for (int t = threadIdx.x; t <= nh; t += blockDim.x) {
    const int rowt = (t < nh) ? o + t : N - 1;
    for (int u = nu - 1; u >= 0; --u) {
      double2 v = cconj(A[(size_t)rowt + (size_t)(nv + u) * N]);
      for (int k = u + 1; k < nu; ++k) {
        double2 zk = (t < nh) ? Ze[(size_t)k * nh + t] : zst[k];
        // (L1^H)[u][k] = conj(L1[k][u])
        v = csub(v, cmul(cconj(A[(size_t)(nv + k) + (size_t)(nv + u) * N]), zk));
      }
      v = cscale(v, 1.0 / A[(size_t)(nv + u) + (size_t)(nv + u) * N].x);
      if (t < nh)
        Ze[(size_t)u * nh + t] = v;
      else
        zst[u] = v;
    }
  }
}


// Real path: the factored K of a lossless element (real eps, mu, no Robin
// face) in the phase-scaled basis.  With D_h = diag(-i on E-hat, 1 on H-hat)
// and D_u = diag(-i on E, 1 on H): S = D_h S_r D_h^H, Z = D_u Z_r D_h^H,
// L1 = D_u L1_r D_u^H; the load and therefore s, c, z vanish.
__device__ __forceinline__ double2 phase_apply(double v, bool a_imag, bool b_imag) {
  // d_a v conj(d_b) with d = -i (imag) or 1
  if (a_imag == b_imag) return make_double2(v, 0.0);
  return a_imag ? make_double2(0.0, -v) : make_double2(0.0, v);
}

__global__ void __launch_bounds__(256) k_extract_real(Sizes S, const int* __restrict__ ids, const double* __restrict__ K,
                                                      const ElemOff* __restrict__ off, double2* Sst, double2* sst,
                                                      double* cst, double2* Zst, double2* zst, double2* L1st,
                                                      double* Zscratch) {
  const int slot = blockIdx.x;
  const int e = ids[slot];
  const ElemOff of = off[e];
  const int N = S.N, nv = S.n_v, nu = S.n_u, nh = S.n_h, nt = S.nt, nE = 3 * S.nL;
  const double* A = K + (size_t)slot * N * N;
  const int o = nv + nu;
  double2* Se = Sst + of.S;
  for (int t = threadIdx.x; t < nh * nh; t += blockDim.x) {
    const int i = t / nh, j = t - i * nh;
    const double v = (i >= j) ? A[(size_t)(o + i) + (size_t)(o + j) * N] : A[(size_t)(o + j) + (size_t)(o + i) * N];
    Se[t] = phase_apply(v, i < nt, j < nt);
  }
  for (int t = threadIdx.x; t < nh; t += blockDim.x) sst[of.h + t] = make_double2(0.0, 0.0);
  for (int t = threadIdx.x; t < nu; t += blockDim.x) zst[of.u + t] = make_double2(0.0, 0.0);
  if (threadIdx.x == 0) cst[e] = 0.0;
  if (L1st) {
    double2* Le = L1st + of.L1;
    for (int t = threadIdx.x; t < nu * nu; t += blockDim.x) {
      const int i = t / nu, j = t - i * nu;
      Le[t] = (i >= j) ? phase_apply(A[(size_t)(nv + i) + (size_t)(nv + j) * N], i < nE, j < nE)
                       : make_double2(0.0, 0.0);
    }
  }
  // Z_r = L1_r^{-T} Y_r, Y_r[u][t] = A[o + t][nv + u]; real back substitution per column t
  double* Zr = Zscratch + (size_t)slot * nu * nh;
  for (int t = threadIdx.x; t < nh; t += blockDim.x) {
    for (int u = nu - 1; u >= 0; --u) {
      double v = A[(size_t)(o + t) + (size_t)(nv + u) * N];
      for (int k = u + 1; k < nu; ++k) v -= A[(size_t)(nv + k) + (size_t)(nv + u) * N] * Zr[(size_t)k * nh + t];
      Zr[(size_t)u * nh + t] = v / A[(size_t)(nv + u) + (size_t)(nv + u) * N];
    }
  }
  __syncthreads();
  double2* Ze = Zst + of.Z;
  for (int q = threadIdx.x; q < nu * nh; q += blockDim.x) {
    const int u = q / nh, t = q - u * nh;
    Ze[q] = phase_apply(Zr[q], u < nE, t < nt);
  }
}

// ----------------------------------------------------- trace restriction --
// Elements with an entity of lower order than their own: the stored condensed
// matrices become those of the element's trace slots, S <- R^T S R,
// s <- R^T s, Z <- Z R, with R = diag(R1, R1) over the E-hat and H-hat halves
// (R1 real, nt x nt, column-compressed).  The element's K slot serves as scratch
// (N^2 >= n_h^2 + n_u n_h entries).
__global__ void __launch_bounds__(256) k_restrict(int nt, int nu, const int* __restrict__ ids,
                                                  const ElemOff* __restrict__ off, const int* __restrict__ sig,
                                                  const RSig* __restrict__ rsig, const int32_t* __restrict__ rint,
                                                  const double* __restrict__ rdbl, double2* Sst, double2* sst,
                                                  double2* Zst, double2* scratch, size_t scratch_stride) {
  extern __shared__ double2 s_in[];  // n_h
  const int slot = blockIdx.x, e = ids[slot];
  const int sg = sig[e];
  if (sg < 0) return;
  const RSig R = rsig[sg];
  const int32_t* cp = rint + R.cptr;
  const int32_t* ci = rint + R.cidx;
  const double* cw = rdbl + R.cw;
  const int nh = 2 * nt;
  const ElemOff of = off[e];
  double2* Se = Sst + of.S;
  double2* Ze = Zst + of.Z;
  double2* se = sst + of.h;
  double2* T = scratch + (size_t)slot * scratch_stride;
  double2* Zn = T + (size_t)nh * nh;
  for (int t = threadIdx.x; t < nh; t += blockDim.x) s_in[t] = se[t];
  // T = S R and Zn = Z R: column c of R (half base) combines columns base + ci[k]
  for (int q = threadIdx.x; q < nh * nh; q += blockDim.x) {
    const int i = q / nh, c = q - i * nh;
    const int cc = c < nt ? c : c - nt, base = c < nt ? 0 : nt;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = cp[cc]; k < cp[cc + 1]; ++k) {
      const double2 v = Se[(size_t)i * nh + base + ci[k]];
      acc.x = fma(v.x, cw[k], acc.x);
      acc.y = fma(v.y, cw[k], acc.y);
    }
    T[q] = acc;
  }
  for (int q = threadIdx.x; q < nu * nh; q += blockDim.x) {
    const int i = q / nh, c = q - i * nh;
    const int cc = c < nt ? c : c - nt, base = c < nt ? 0 : nt;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = cp[cc]; k < cp[cc + 1]; ++k) {
      const double2 v = Ze[(size_t)i * nh + base + ci[k]];
      acc.x = fma(v.x, cw[k], acc.x);
      acc.y = fma(v.y, cw[k], acc.y);
    }
    Zn[q] = acc;
  }
  __syncthreads();
  // S = R^T T: row r of the result combines rows base + ci[k] of T
  for (int q = threadIdx.x; q < nh * nh; q += blockDim.x) {
    const int r = q / nh, c = q - r * nh;
    const int rr = r < nt ? r : r - nt, base = r < nt ? 0 : nt;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = cp[rr]; k < cp[rr + 1]; ++k) {
      const double2 v = T[(size_t)(base + ci[k]) * nh + c];
      acc.x = fma(v.x, cw[k], acc.x);
      acc.y = fma(v.y, cw[k], acc.y);
    }
    Se[q] = acc;
  }
  for (int q = threadIdx.x; q < nu * nh; q += blockDim.x) Ze[q] = Zn[q];
  for (int r = threadIdx.x; r < nh; r += blockDim.x) {
    const int rr = r < nt ? r : r - nt, base = r < nt ? 0 : nt;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = cp[rr]; k < cp[rr + 1]; ++k) {
      const double2 v = s_in[base + ci[k]];
      acc.x = fma(v.x, cw[k], acc.x);
      acc.y = fma(v.y, cw[k], acc.y);
    }
    se[r] = acc;
  }
}

// ------------------------------------------------------- orchestration --
// Per-element bytes of the chunk workspace of one group.  FP64 quadrature is
// sum-factorised (quad_sf.cu) and keeps only per-point weights and, for the
// real-path extraction, an n_u x n_h scratch; the tensor-core modes keep the
// weighted basis values at every quadrature point.
static size_t chunk_bytes(const Sizes& S, bool fp64q) {
  const size_t mc = sizeof(double) * (2 * (size_t)S.n_f * S.n_f + 2 * (size_t)S.n_f * 3 * S.nL);
  const size_t k = sizeof(double2) * (size_t)S.N * S.N + sizeof(int);
  if (fp64q)
    return k + mc + quad_sf_weight_bytes(S) + sizeof(double) * (size_t)S.n_u * S.n_h;
  return k + mc + sizeof(double) * 3 * (size_t)S.nq * (2 * S.n_f + 3 * S.nL);
}

// Default chunk capacity per group: a byte budget of 12 GB, raised to one
// element per SM when a single chunk of the group is larger (high degrees), at
// most 48 GB; a multiple of the SM count when large enough; or the caller's
// fixed chunk.
// The element lists the plan cuts into chunks: per order group, the lossless
// elements (real path, when allowed) and the others; in streaming mode each
// list split further by colour (a chunk is then colour-homogeneous).
struct ElemList {
  int g = 0;
  bool real = false;
  int colour = 0;  // streaming: the chunk colour of the list (one wave group per colour); else 0
  std::vector<int> elems;
};

static std::vector<ElemList> element_lists(const dpg_handle* h, bool real) {
  std::vector<ElemList> out;
  for (int g = 0; g < (int)h->grp.size(); ++g) {
    const Group& G = h->grp[g];
    std::vector<std::vector<int>> lists;
    if (real) {
      lists.push_back(G.real_elems);
      lists.push_back(G.cplx_elems);
    } else {
      lists.push_back(G.elems);
    }
    std::vector<int> colours(lists.size(), 0);
    if (h->stream) {
      std::vector<std::vector<int>> by_colour;
      colours.clear();
      for (const std::vector<int>& L : lists)
        for (int c = 0; c < h->ncolor; ++c) {
          std::vector<int> part;
          for (int e : L)
            if (h->elem_color[e] == c) part.push_back(e);
          if (!part.empty()) {
            by_colour.push_back(part);
            colours.push_back(c);
          }
        }
      lists = by_colour;
    }
    for (size_t k = 0; k < lists.size(); ++k) {
      std::vector<int>& L = lists[k];
      if (L.empty()) continue;
      ElemList el;
      el.g = g;
      el.real = real && h->is_real[L[0]];
      el.colour = colours[k];
      el.elems = std::move(L);
      out.push_back(std::move(el));
    }
  }
  return out;
}

// Bytes of one element's augmented matrix in the K workspace.
static size_t k_bytes(const Sizes& S, bool real) {
  return (real ? sizeof(double) : sizeof(double2)) * (size_t)S.N * S.N;
}

// Chunk of list l in wave w of the order-bucketed pass: ceil(n_l / waves) elements.
static int wave_cap(size_t n, int waves) { return (int)((n + waves - 1) / waves); }

// Waves of the order-bucketed pass, per list.  The lists form wave groups
// (one per chunk colour in streaming mode, one otherwise); a group's waves
// each take ceil(n_l / waves) elements of every list of the group.  A group
// has at least as many waves as the K arena budget (48 GB) requires, and at
// least enough that its costliest list (largest N^3, complex 4x real) puts no
// more elements into a wave than there are SMs, since an SM that got two of
// them would double the wave's span; otherwise as few as possible, so that
// the cheaper elements fill the SMs around the long ones.  With the caller's
// chunk size: the group's largest list's share of a wave.
static std::vector<int> list_waves(const dpg_handle* h, const std::vector<ElemList>& lists, int chunk, int sms) {
  int ngroup = 1;
  for (const ElemList& L : lists) ngroup = std::max(ngroup, L.colour + 1);
  std::vector<int> waves_of(ngroup, 1);
  const size_t budget = (size_t)48 << 30;
  for (int c = 0; c < ngroup; ++c) {
    size_t total = 0, nmax = 0, ncost = 0;
    double cmax = -1.0;
    for (const ElemList& L : lists) {
      if (L.colour != c) continue;
      const Sizes& S = h->grp[L.g].sz;
      total += k_bytes(S, L.real) * L.elems.size();
      nmax = std::max(nmax, L.elems.size());
      const double cost = (double)S.N * S.N * S.N * (L.real ? 1.0 : 4.0);
      if (cost > cmax) {
        cmax = cost;
        ncost = L.elems.size();
      }
    }
    if (nmax == 0) continue;
    int w;
    if (chunk > 0) {
      w = (int)((nmax + chunk - 1) / chunk);
    } else {
      const int w_mem = (int)((total + budget - 1) / budget);
      const int w_sm = (int)((ncost + sms - 1) / sms);
      w = std::max(w_mem, w_sm);
    }
    waves_of[c] = std::max(1, w);
  }
  std::vector<int> out(lists.size());
  for (size_t l = 0; l < lists.size(); ++l) out[l] = waves_of[lists[l].colour];
  return out;
}

void set_default_caps(dpg_handle* h, int chunk) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  h->chunk_req = chunk;
  if (h->bucketed) {
    const std::vector<ElemList> lists = element_lists(h, h->allow_real);
    const std::vector<int> lw = list_waves(h, lists, chunk, sms);
    h->nwaves = 0;
    for (int w : lw) h->nwaves = std::max(h->nwaves, w);
    for (Group& G : h->grp) G.cap = 1;
    for (size_t l = 0; l < lists.size(); ++l) {
      Group& G = h->grp[lists[l].g];
      G.cap = std::max(G.cap, wave_cap(lists[l].elems.size(), lw[l]));
    }
    return;
  }
  for (Group& G : h->grp) {
    const size_t per = chunk_bytes(G.sz, h->prec == DPG_PREC_FP64);
    const size_t budget = std::max((size_t)12 << 30, std::min((size_t)48 << 30, per * (size_t)sms));
    int cap = (int)std::max<size_t>(1, budget / per);
    if (chunk > 0) cap = chunk;
    if (cap >= sms && chunk <= 0) cap = cap / sms * sms;
    G.cap = std::max(1, std::min(cap, (int)G.elems.size()));
  }
}

// One workspace sized for the largest group chunk (frees the previous one).
int alloc_workspace(dpg_handle* h) {
  Workspace& w = h->ws;
  void* old[] = {w.K, w.V, w.Cu, w.PhiL, w.MC, w.ids, w.FV, w.FR, w.rent, w.WQ, w.Q};
  for (void* b : old)
    if (b) cudaFree(b);
  w = Workspace{};
  const bool fp64q = h->prec == DPG_PREC_FP64;
  size_t bK = 0, bV = 0, bCu = 0, bP = 0, bMC = 0, bFV = 0, bFR = 0, bWQ = 16, bQ = 16;
  int capmax = 1;
  for (Group& G : h->grp) {
    const Sizes& S = G.sz;
    const int cap = G.cap;
    capmax = std::max(capmax, cap);
    const size_t nq3 = 3 * (size_t)S.nq;
    bK = std::max(bK, sizeof(double2) * (size_t)S.N * S.N * cap);
    // V, Cu, PhiL: basis values at the quadrature points for the tensor-core
    // contractions; with FP64 quadrature one element's worth (the metric-free
    // reference matrices) and V doubling as the real-path extraction scratch
    const int vcap = fp64q ? 1 : cap;
    bV = std::max(bV, sizeof(double) * nq3 * S.n_f * vcap);
    if (fp64q) bV = std::max(bV, sizeof(double) * (size_t)S.n_u * S.n_h * cap);
    bCu = std::max(bCu, sizeof(double) * nq3 * S.n_f * vcap);
    bP = std::max(bP, sizeof(double) * nq3 * 3 * S.nL * vcap);
    bMC = std::max(bMC, sizeof(double) * (2 * (size_t)S.n_f * S.n_f + 2 * (size_t)S.n_f * 3 * S.nL) * cap);
    if (fp64q) bWQ = std::max(bWQ, quad_sf_weight_bytes(S) * cap);
    if (h->factor_arith == DPG_FACTOR_TC_SPLIT) bQ = std::max(bQ, factor_tc_scratch_bytes(S.N, true) * cap);
  }
  if (h->bucketed) {
    // the K arena holds one wave: every list's chunk side by side (256-byte
    // aligned slices); the persistent factorisation's digit scratch is per SM
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const std::vector<ElemList> lists = element_lists(h, h->allow_real);
    const std::vector<int> lw = list_waves(h, lists, h->chunk_req, sms);
    std::vector<size_t> arena_of(1, 0);
    int nmax = 1;
    for (size_t l = 0; l < lists.size(); ++l) {
      const ElemList& L = lists[l];
      const Sizes& S = h->grp[L.g].sz;
      if ((int)arena_of.size() <= L.colour) arena_of.resize(L.colour + 1, 0);
      arena_of[L.colour] += (k_bytes(S, L.real) * wave_cap(L.elems.size(), lw[l]) + 255) / 256 * 256;
      nmax = std::max(nmax, S.N);
    }
    for (size_t a : arena_of) bK = std::max(bK, a);
    bQ = std::max(bQ, factor_tc_queue_scratch_bytes(nmax) * (size_t)sms);
  }
  w.rcap = std::max(6, std::min(capmax * 2, std::max(6, (int)h->robin_entries.size())));
  for (Group& G : h->grp) {
    const Sizes& S = G.sz;
    const int Wf = 2 * S.n_f + 2 * S.nt + 2;
    bFV = std::max(bFV, sizeof(double) * 3 * (size_t)S.nqf * Wf * w.rcap);
    bFR = std::max(bFR, sizeof(double) * (size_t)S.n_f * Wf * w.rcap);
  }
  size_t bytes[] = {bK, bV, bCu, bP, bMC, sizeof(int) * (size_t)capmax, bFV, bFR, sizeof(int) * 4 * (size_t)w.rcap,
                    bWQ, bQ};
  void** ptrs[] = {(void**)&w.K, (void**)&w.V, (void**)&w.Cu, (void**)&w.PhiL, (void**)&w.MC, (void**)&w.ids,
                   (void**)&w.FV, (void**)&w.FR, (void**)&w.rent, (void**)&w.WQ, (void**)&w.Q};
  for (int k = 0; k < 11; ++k) {
    if (cudaMalloc(ptrs[k], bytes[k]) != cudaSuccess) {
      cudaGetLastError();
      h->err = "workspace allocation of " + std::to_string(bytes[k]) + " bytes failed";
      return DPG_ERR_NOMEM;
    }
  }
  w.cap = capmax;
  h->plan_valid = false;
  h->graph_valid = false;
  if (h->stream) {
    // chunk-sized element stores: slot k of a chunk of group g at k times the
    // group's per-element sizes
    size_t bS = 16, bs = 16, bZ = 16, bz = 16;
    for (const Group& G : h->grp) {
      const Sizes& S = G.sz;
      bS = std::max(bS, sizeof(double2) * (size_t)S.n_h * S.n_h * G.cap);
      bs = std::max(bs, sizeof(double2) * (size_t)S.n_h * G.cap);
      bZ = std::max(bZ, sizeof(double2) * (size_t)S.n_u * S.n_h * G.cap);
      bz = std::max(bz, sizeof(double2) * (size_t)S.n_u * G.cap);
    }
    void* olds[] = {h->d_S, h->d_s, h->d_Z, h->d_z};
    for (void* b : olds)
      if (b) cudaFree(b);
    h->d_S = h->d_s = h->d_Z = h->d_z = nullptr;
    if (cudaMalloc(&h->d_S, bS) != cudaSuccess || cudaMalloc(&h->d_s, bs) != cudaSuccess ||
        cudaMalloc(&h->d_Z, bZ) != cudaSuccess || cudaMalloc(&h->d_z, bz) != cudaSuccess) {
      cudaGetLastError();
      h->err = "chunk store allocation failed";
      return DPG_ERR_NOMEM;
    }
    // the slot offsets of the stores come with the plan
    return build_plan(h);
  }
  return DPG_OK;
}

// Kernel attributes set once (never inside a stream capture).
int init_kernel_attributes(dpg_handle* h) {
  const int s64 = (int)factor_smem<double>();
  const int s128 = (int)factor_smem<double2>();
  DPG_CUDA_TRY(h, cudaFuncSetAttribute(k_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64));
  DPG_CUDA_TRY(h, cudaFuncSetAttribute(k_factor<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s128));
  if (tc_init() != DPG_OK || factor_tc_init() != DPG_OK || quad_sf_init() != DPG_OK) {
    h->err = "tensor-core kernel attribute setup failed";
    return DPG_ERR_CUDA;
  }
  return DPG_OK;
}

// Robin sub-batches of a chunk: whole elements, at most rcap / 2 entries.
// Each sub-batch is (entries: slot, face, group, element id; per element:
// first entry, count).
static void robin_batches(const dpg_handle* h, const int* ids_host, int count,
                          std::vector<std::vector<int>>& rents, std::vector<std::vector<int>>& rlists) {
  std::vector<int> rent, rlist;
  auto flush = [&]() {
    if (rlist.empty()) return;
    rents.push_back(rent);
    rlists.push_back(rlist);
    rent.clear();
    rlist.clear();
  };
  for (int slot = 0; slot < count; ++slot) {
    const int e = ids_host[slot];
    const int first = h->robin_first[e];
    if (first < 0) continue;
    int cnt = 0;
    while (first + cnt < (int)h->robin_entries.size() && h->robin_entries[first + cnt].elem == e) ++cnt;
    if ((int)rent.size() / 4 + cnt > h->ws.rcap / 2) flush();
    rlist.push_back((int)rent.size() / 4);
    rlist.push_back(cnt);
    for (int k = 0; k < cnt; ++k) {
      const RobinEntry& re = h->robin_entries[first + k];
      rent.push_back(slot);
      rent.push_back(re.face);
      rent.push_back(re.grp);
      rent.push_back(e);
    }
  }
  flush();
}

// Face arrays, face GEMM and Robin terms of one sub-batch (device lists).
static int robin_launch(dpg_handle* h, int g, const int* d_rent, int nent, const int* d_rlist, int nel,
                        cudaStream_t s, double2* K) {
  Workspace& w = h->ws;
  const Group& G = h->grp[g];
  const Sizes& S = G.sz;
  const int Wf = 2 * S.n_f + 2 * S.nt + 2;
  k_face_arrays<<<dim3(1, nent), 256, 0, s>>>(G.tab, S, h->d_X, d_rent, h->d_robin, G.d_trfun, h->omega, 0, w.FV);
  gemm_tn(S.n_f, Wf, 3 * S.nqf, w.FV, Wf, (long long)3 * S.nqf * Wf, w.FV, Wf, (long long)3 * S.nqf * Wf, w.FR, Wf,
          (long long)S.n_f * Wf, nent, s);
  k_robin_add<<<nel, 256, 0, s>>>(S, d_rlist, d_rent, h->d_robin, w.FR, K);
  DPG_CUDA_TRY(h, cudaGetLastError());
  h->launches += 3;
  return DPG_OK;
}

// Robin terms of a chunk given by host ids (paths outside the plan): the
// sub-batch lists are copied to the workspace one at a time.
static int run_robin(dpg_handle* h, int g, const int* ids_host, int count, cudaStream_t s) {
  Workspace& w = h->ws;
  std::vector<std::vector<int>> rents, rlists;
  robin_batches(h, ids_host, count, rents, rlists);
  for (size_t k = 0; k < rents.size(); ++k) {
    const int nent = (int)rents[k].size() / 4;
    DPG_CUDA_TRY(h, cudaMemcpyAsync(w.rent, rents[k].data(), sizeof(int) * rents[k].size(), cudaMemcpyHostToDevice, s));
    // the element list rides after the entries (rcap / 2 entries and 2 ints per element fit 4 rcap ints)
    int* d_rlist = w.rent + 4 * nent;
    DPG_CUDA_TRY(h, cudaMemcpyAsync(d_rlist, rlists[k].data(), sizeof(int) * rlists[k].size(), cudaMemcpyHostToDevice,
                                    s));
    int rc = robin_launch(h, g, w.rent, nent, d_rlist, (int)rlists[k].size() / 2, s, w.K);
    if (rc) return rc;
    // the workspace list buffer is reused: wait for this sub-batch
    DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  }
  return DPG_OK;
}

// quad = false reuses the quadrature matrices already in the workspace (the
// same chunk was formed just before) and only forms K again.
// The stored X of a chunk's elements after their factorisation (see
// k_est_stored): column i of rows n_v..N-1 of K, contiguous in K.
template <typename T>
__global__ void __launch_bounds__(256) k_extract_x(Sizes S, const int* __restrict__ ids, const T* __restrict__ K,
                                                   const int64_t* __restrict__ xoff, double* Xst) {
  const int slot = blockIdx.x, e = ids[slot];
  const int N = S.N, nv = S.n_v, m1 = N - nv;
  const T* A = K + (size_t)slot * N * N;
  T* dst = reinterpret_cast<T*>(Xst + xoff[e]);
  for (int64_t q = threadIdx.x; q < (int64_t)nv * m1; q += blockDim.x) {
    const int i = (int)(q / m1), t = (int)(q - (int64_t)i * m1);
    dst[q] = A[(size_t)nv + t + (size_t)i * N];
  }
}

int run_element_chunk(dpg_handle* h, int g, const int* ids_host, int count, cudaStream_t s, bool factor,
                      bool extract, bool real, const ChunkPlan* cp, bool quad, bool build, void* Kc) {
  Workspace& w = h->ws;
  double2* const Kw = Kc ? static_cast<double2*>(Kc) : w.K;  // the chunk's augmented matrices
  const Group& G = h->grp[g];
  const Sizes& S = G.sz;
  if (count > G.cap) return DPG_ERR_ARG;
  // element ids of the chunk: the plan's device list, or a copy of the host list
  const int* ids = cp ? cp->d_ids + cp->ids_off : w.ids;
  if (!cp) DPG_CUDA_TRY(h, cudaMemcpyAsync(w.ids, ids_host, sizeof(int) * count, cudaMemcpyHostToDevice, s));
  if (quad) {
    if (h->prec == DPG_PREC_FP64) {
      // M, C, P, Q by sum factorisation over the tensor Gauss rule (quad_sf.cu)
      if (quad_sf_launch(G.tab, S, h->d_X, ids, count, w.WQ, w.MC, s) != DPG_OK) {
        h->err = "sum-factorised quadrature launch failed";
        return DPG_ERR_CUDA;
      }
      h->launches += 2;
    } else {
      const size_t nq3 = 3 * (size_t)S.nq;
      k_vol_arrays<<<dim3((S.nq + QB - 1) / QB, count), 256, 0, s>>>(G.tab, S, h->d_X, ids, w.V, w.Cu, w.PhiL);
      const long long sV = (long long)(nq3 * S.n_f), sP = (long long)(nq3 * 3 * S.nL);
      const int nL3 = 3 * S.nL;
      const size_t mcs = 2 * (size_t)S.n_f * S.n_f + 2 * (size_t)S.n_f * 3 * S.nL;
      const int split = h->prec == DPG_PREC_3XTF32 ? 3 : 1;
      int* terr = h->d_status + h->ne;
      int rc = 0;
      rc |= gemm_tn_tc(split, S.n_f, S.n_f, (int)nq3, w.V, S.n_f, sV, w.V, S.n_f, sV, w.MC, S.n_f, (long long)mcs,
                       count, 1, terr, s);
      rc |= gemm_tn_tc(split, S.n_f, S.n_f, (int)nq3, w.Cu, S.n_f, sV, w.Cu, S.n_f, sV, w.MC + (size_t)S.n_f * S.n_f,
                       S.n_f, (long long)mcs, count, 1, terr, s);
      rc |= gemm_tn_tc(split, S.n_f, nL3, (int)nq3, w.V, S.n_f, sV, w.PhiL, nL3, sP, w.MC + 2 * (size_t)S.n_f * S.n_f,
                       nL3, (long long)mcs, count, 0, terr, s);
      rc |= gemm_tn_tc(split, S.n_f, nL3, (int)nq3, w.Cu, S.n_f, sV, w.PhiL, nL3, sP,
                       w.MC + 2 * (size_t)S.n_f * S.n_f + (size_t)S.n_f * nL3, nL3, (long long)mcs, count, 0, terr, s);
      if (rc) {
        h->err = "tensor-core contraction launch failed";
        return DPG_ERR_CUDA;
      }
      h->launches += 5;  // basis arrays, four contractions
    }
  }
  double* Kr = reinterpret_cast<double*>(Kw);
  if (build) {
    if (real) {
      k_build_K_real<<<dim3(148, count), 256, 0, s>>>(S, h->omega, h->alpha, ids, h->d_eps, h->d_mu, w.MC,
                                                      G.d_Xref, G.d_Tall, Kr);
    } else {
      k_build_K<<<dim3(148, count), 256, 0, s>>>(S, h->omega, h->alpha, ids, h->d_eps, h->d_mu, h->d_fbc, w.MC,
                                                 G.d_Xref, G.d_Tf, G.d_Tall, Kw);
    }
    DPG_CUDA_TRY(h, cudaGetLastError());
    h->launches += 1;
    if (!real) {
      if (cp) {
        for (const int4& rb : cp->robin) {
          int rc = robin_launch(h, g, cp->d_rent + rb.x, rb.y, cp->d_rent + rb.z, rb.w, s, Kw);
          if (rc) return rc;
        }
      } else {
        int rc = run_robin(h, g, ids_host, count, s);
        if (rc) return rc;
      }
    }
  }
  if (factor) {
    const size_t smem = real ? factor_smem<double>() : factor_smem<double2>();
    const bool timed = cp && h->timing;
    // inside a stream capture an event record is only a dependency unless it
    // is marked external; then it is recorded at every graph replay
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (timed) DPG_CUDA_TRY(h, cudaStreamIsCapturing(s, &cap));
    const unsigned int rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (timed) DPG_CUDA_TRY(h, cudaEventRecordWithFlags(cp->ev0, s, rec_flags));
    if (h->factor_arith == DPG_FACTOR_TC_SPLIT) {
      // factorisation stamps of the plan's chunks (SM, start, end per element)
      unsigned long long* st = (cp && h->d_stamps && !h->bucketed) ? h->d_stamps + 3 * cp->ids_off : nullptr;
      if (factor_tc_launch(!real, count, S.N, S.N, S.n_v, S.n_v + S.n_u, ids, real ? (void*)Kr : (void*)Kw,
                           h->d_status, h->d_status + h->ne, w.Q, s, st) != DPG_OK) {
        h->err = "tensor-core factorisation launch failed";
        return DPG_ERR_CUDA;
      }
    } else if (real) {
      k_factor<double><<<count, 256, smem, s>>>(S.N, S.N, S.n_v, S.n_v + S.n_u, ids, Kr, h->d_status);
    } else {
      k_factor<double2><<<count, 256, smem, s>>>(S.N, S.N, S.n_v, S.n_v + S.n_u, ids, Kw, h->d_status);
    }
    DPG_CUDA_TRY(h, cudaGetLastError());
    h->launches += 1;
    if (timed) DPG_CUDA_TRY(h, cudaEventRecordWithFlags(cp->ev1, s, rec_flags));
  }
  if (extract) {
    if (h->d_Xst && !h->stream) {  // X = (L^{-1} [B | B-hat | l])^H for the stored-factor estimator
      if (real)
        k_extract_x<double><<<count, 256, 0, s>>>(S, ids, Kr, h->d_xst_off, h->d_Xst);
      else
        k_extract_x<double2><<<count, 256, 0, s>>>(S, ids, Kw, h->d_xst_off, h->d_Xst);
      DPG_CUDA_TRY(h, cudaGetLastError());
      h->launches += 1;
    }
    if (real)
      k_extract_real<<<count, 256, 0, s>>>(S, ids, Kr, h->d_soff, h->d_S, h->d_s, h->d_c, h->d_Z, h->d_z, h->d_L1,
                                           w.V);
    else
      k_extract<<<count, 256, 0, s>>>(S, ids, Kw, h->d_soff, h->d_S, h->d_s, h->d_c, h->d_Z, h->d_z, h->d_L1);
    DPG_CUDA_TRY(h, cudaGetLastError());
    h->launches += 1;
    bool any = cp ? cp->restricted : false;
    for (int k = 0; !cp && k < count && !any; ++k) any = h->elem_sig[ids_host[k]] >= 0;
    if (any) {
      // scratch: each element's own (already extracted) matrix slot, N^2
      // doubles on the real path and N^2 complex values otherwise
      k_restrict<<<count, 256, sizeof(double2) * S.n_h, s>>>(S.nt, S.n_u, ids, h->d_soff, h->d_sig, h->d_rsig,
                                                            h->d_rint, h->d_rdbl, h->d_S, h->d_s, h->d_Z, Kw,
                                                            real ? (size_t)S.N * S.N / 2 : (size_t)S.N * S.N);
      DPG_CUDA_TRY(h, cudaGetLastError());
      h->launches += 1;
    }
  }
  return DPG_OK;
}

// ------------------------------------------------------ pass plan / graph --
static void free_chunks(std::vector<ChunkPlan>& plan, int** d_ids, int** d_rent) {
  for (ChunkPlan& c : plan) {
    if (c.ev0) cudaEventDestroy(c.ev0);
    if (c.ev1) cudaEventDestroy(c.ev1);
  }
  plan.clear();
  if (*d_ids) cudaFree(*d_ids);
  if (*d_rent) cudaFree(*d_rent);
  *d_ids = nullptr;
  *d_rent = nullptr;
}

void free_plan(dpg_handle* h) {
  free_chunks(h->plan, &h->d_plan_ids, &h->d_plan_rent);
  for (WavePlan& wp : h->waves) {
    if (wp.ev0) cudaEventDestroy(wp.ev0);
    if (wp.ev1) cudaEventDestroy(wp.ev1);
  }
  h->waves.clear();
  void* bufs[] = {h->d_items, h->d_wave_ctr, h->d_stamps};
  for (void* b : bufs)
    if (b) cudaFree(b);
  h->d_items = nullptr;
  h->d_wave_ctr = nullptr;
  h->d_stamps = nullptr;
  h->n_stamps = 0;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  h->plan_valid = false;
  h->graph_valid = false;
}

// Chunks of every group (with real: lossless elements on the real path
// first), their device id lists and Robin sub-batches.  Synchronous.
static int make_chunks(dpg_handle* h, bool real, std::vector<ChunkPlan>& plan, int** d_ids, int** d_rent) {
  std::vector<int> ids_all, rent_all;
  std::vector<ElemOff> soff;
  if (h->stream) soff.assign(h->ne + 1, ElemOff{});
  const std::vector<ElemList> lists = element_lists(h, real);
  // (list, first element, count) of every chunk, in plan order: list by list,
  // or wave by wave (the w-th chunk of every list) when order-bucketed
  struct Cut {
    int l;
    size_t c0;
    int count;
    int wave;
  };
  std::vector<Cut> cuts;
  const bool waves = h->bucketed;
  if (waves) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const std::vector<int> lw = list_waves(h, lists, h->chunk_req, sms);
    int ngroup = 1;
    for (const ElemList& L : lists) ngroup = std::max(ngroup, L.colour + 1);
    int wave_id = 0;  // waves numbered across the groups, group by group
    for (int c = 0; c < ngroup; ++c) {
      int wg = 0;
      for (size_t l = 0; l < lists.size(); ++l)
        if (lists[l].colour == c) wg = std::max(wg, lw[l]);
      for (int w = 0; w < wg; ++w, ++wave_id)
        for (int l = 0; l < (int)lists.size(); ++l) {
          if (lists[l].colour != c) continue;
          const size_t n = lists[l].elems.size();
          const int cap = wave_cap(n, lw[l]);
          const size_t c0 = (size_t)w * cap;
          if (c0 < n) cuts.push_back({l, c0, (int)std::min<size_t>(cap, n - c0), wave_id});
        }
    }
  } else {
    for (int l = 0; l < (int)lists.size(); ++l) {
      const int cap = h->grp[lists[l].g].cap;
      for (size_t c0 = 0; c0 < lists[l].elems.size(); c0 += cap)
        cuts.push_back({l, c0, (int)std::min<size_t>(cap, lists[l].elems.size() - c0), -1});
    }
  }
  std::vector<FtItem> items;
  int64_t koff = 0;
  int cur_wave = -1;
  for (size_t ci = 0; ci < cuts.size(); ++ci) {
    const Cut& cu = cuts[ci];
    const ElemList& EL = lists[cu.l];
    const int g = EL.g;
    const Group& G = h->grp[g];
    const Sizes& S = G.sz;
    const std::vector<int>& L = EL.elems;
    const size_t c0 = cu.c0;
    ChunkPlan cp;
    cp.g = g;
    cp.real = EL.real;
    cp.count = cu.count;
    cp.ids_off = (int64_t)ids_all.size();
    ids_all.insert(ids_all.end(), L.begin() + c0, L.begin() + c0 + cp.count);
    if (waves) {
      if (cu.wave != cur_wave) {
        cur_wave = cu.wave;
        WavePlan wp;
        wp.c0 = (int)plan.size();
        wp.item_off = (int64_t)items.size();
        DPG_CUDA_TRY(h, cudaEventCreate(&wp.ev0));
        DPG_CUDA_TRY(h, cudaEventCreate(&wp.ev1));
        h->waves.push_back(wp);
        koff = 0;
      }
      WavePlan& wp = h->waves.back();
      wp.nc += 1;
      cp.koff = koff;
      const size_t eb = k_bytes(S, cp.real);
      for (int k = 0; k < cp.count; ++k) {
        FtItem it{};
        it.koff = koff + (int64_t)(eb * k);
        it.elem = L[c0 + k];
        it.cplx = cp.real ? 0 : 1;
        it.N = S.N;
        it.nact = S.N;
        it.nv = S.n_v;
        it.npiv = S.n_v + S.n_u;
        items.push_back(it);
      }
      wp.nitems += cp.count;
      if (cp.real) wp.nitems_real += cp.count;
      wp.nmax = std::max(wp.nmax, S.N);
      koff += (int64_t)((eb * cp.count + 255) / 256 * 256);
    }
    if (h->stream)
      for (int k = 0; k < cp.count; ++k) {
        ElemOff& o = soff[L[c0 + k]];
        o.S = (int64_t)k * S.n_h * S.n_h;
        o.Z = (int64_t)k * S.n_u * S.n_h;
        o.L1 = 0;
        o.h = (int64_t)k * S.n_h;
        o.u = (int64_t)k * S.n_u;
      }
    for (int k = 0; k < cp.count && !cp.restricted; ++k) cp.restricted = h->elem_sig[L[c0 + k]] >= 0;
    if (!cp.real) {
      std::vector<std::vector<int>> rents, rlists;
      robin_batches(h, L.data() + c0, cp.count, rents, rlists);
      for (size_t k = 0; k < rents.size(); ++k) {
        int4 rb;
        rb.x = (int)rent_all.size();
        rb.y = (int)rents[k].size() / 4;
        rent_all.insert(rent_all.end(), rents[k].begin(), rents[k].end());
        rb.z = (int)rent_all.size();
        rb.w = (int)rlists[k].size() / 2;
        rent_all.insert(rent_all.end(), rlists[k].begin(), rlists[k].end());
        cp.robin.push_back(rb);
      }
    }
    DPG_CUDA_TRY(h, cudaEventCreate(&cp.ev0));
    DPG_CUDA_TRY(h, cudaEventCreate(&cp.ev1));
    plan.push_back(std::move(cp));
  }
  if (waves) {
    // each wave's work list: complex items, then real ones (one persistent
    // launch each), each part longest first (by matrix size), element order
    // among equals; the order fixes nothing in the results, only which SM
    // takes which element
    for (WavePlan& wp : h->waves) {
      std::stable_sort(items.begin() + wp.item_off, items.begin() + wp.item_off + wp.nitems,
                       [](const FtItem& x, const FtItem& y) {
                         if (x.cplx != y.cplx) return x.cplx > y.cplx;
                         return x.N > y.N;
                       });
    }
    DPG_CUDA_TRY(h, cudaMalloc(&h->d_items, sizeof(FtItem) * std::max<size_t>(1, items.size())));
    if (!items.empty())
      DPG_CUDA_TRY(h, cudaMemcpy(h->d_items, items.data(), sizeof(FtItem) * items.size(), cudaMemcpyHostToDevice));
    DPG_CUDA_TRY(h, cudaMalloc(&h->d_wave_ctr, 2 * sizeof(int) * std::max<size_t>(1, h->waves.size())));
  }
  {
    h->n_stamps = waves ? (int64_t)items.size() : (int64_t)ids_all.size();
    DPG_CUDA_TRY(h, cudaMalloc(&h->d_stamps, 3 * sizeof(unsigned long long) * std::max<int64_t>(1, h->n_stamps)));
    DPG_CUDA_TRY(h, cudaMemset(h->d_stamps, 0, 3 * sizeof(unsigned long long) * std::max<int64_t>(1, h->n_stamps)));
  }
  DPG_CUDA_TRY(h, cudaMalloc(d_ids, sizeof(int) * std::max<size_t>(1, ids_all.size())));
  DPG_CUDA_TRY(h, cudaMalloc(d_rent, sizeof(int) * std::max<size_t>(1, rent_all.size())));
  if (!ids_all.empty())
    DPG_CUDA_TRY(h, cudaMemcpy(*d_ids, ids_all.data(), sizeof(int) * ids_all.size(), cudaMemcpyHostToDevice));
  if (!rent_all.empty())
    DPG_CUDA_TRY(h, cudaMemcpy(*d_rent, rent_all.data(), sizeof(int) * rent_all.size(), cudaMemcpyHostToDevice));
  for (ChunkPlan& cp : plan) {
    cp.d_ids = *d_ids;
    cp.d_rent = *d_rent;
  }
  if (h->stream) {
    DPG_CUDA_TRY(h, cudaMemcpy(h->d_soff, soff.data(), sizeof(ElemOff) * soff.size(), cudaMemcpyHostToDevice));
    h->soff_host = soff;
  }
  return DPG_OK;
}

// The element pass's plan (real path as allowed), built once per workspace;
// the estimator's recompute pass runs the same chunks.
int build_plan(dpg_handle* h) {
  free_plan(h);
  int rc = make_chunks(h, h->allow_real, h->plan, &h->d_plan_ids, &h->d_plan_rent);
  if (rc == DPG_OK && !h->d_est_neg) DPG_CUDA_TRY(h, cudaMalloc(&h->d_est_neg, sizeof(int)));
  if (rc) return rc;
  h->plan_valid = true;
  h->graph_valid = false;
  return DPG_OK;
}

// The persistent factorisation of one wave of the order-bucketed pass: one
// CTA per SM over the wave's work list (every order, real and complex,
// longest first), timed by the wave's events when timing is on.
static int factor_wave(dpg_handle* h, int wi, cudaStream_t s) {
  const WavePlan& wp = h->waves[wi];
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (h->timing) DPG_CUDA_TRY(h, cudaStreamIsCapturing(s, &cap));
  const unsigned int rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
  if (h->timing) DPG_CUDA_TRY(h, cudaEventRecordWithFlags(wp.ev0, s, rec_flags));
  // complex items (all orders) first, then the real ones
  const int ncplx = wp.nitems - wp.nitems_real;
  const int64_t off[2] = {wp.item_off, wp.item_off + ncplx};
  const int cnt[2] = {ncplx, wp.nitems_real};
  for (int k = 0; k < 2; ++k) {
    if (cnt[k] == 0) continue;
    if (factor_tc_queue_launch(k == 0, h->d_items + off[k], cnt[k], wp.nmax, h->d_wave_ctr + 2 * wi + k, h->ws.K,
                               h->d_status, h->d_status + h->ne, h->ws.Q,
                               h->d_stamps ? h->d_stamps + 3 * off[k] : nullptr, sms, s) != DPG_OK) {
      h->err = "persistent factorisation launch failed";
      return DPG_ERR_CUDA;
    }
    h->launches += 1;
  }
  if (h->timing) DPG_CUDA_TRY(h, cudaEventRecordWithFlags(wp.ev1, s, rec_flags));
  return DPG_OK;
}

// The whole element pass: the plan's launches, captured once into a CUDA
// graph (re-captured when the plan or the timing switch changes) and replayed
// on the caller's stream.  Capture runs on a private stream, since the legacy
// default stream cannot be captured.
int element_pass(dpg_handle* h, cudaStream_t s) {
  if (!h->plan_valid) {
    int rc = build_plan(h);
    if (rc) return rc;
  }
  // streaming: the system is assembled chunk by chunk as the elements are condensed
  auto pass = [&](cudaStream_t st) -> int {
    if (h->d_stamps)  // the factorisation stamps describe this pass only
      DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_stamps, 0, 3 * sizeof(unsigned long long) * h->n_stamps, st));
    if (h->stream) {
      DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_val, 0, sizeof(double2) * h->nnz, st));
      DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_b, 0, sizeof(double2) * h->n, st));
    }
    if (h->bucketed) {
      unsigned char* arena = reinterpret_cast<unsigned char*>(h->ws.K);
      for (size_t wi = 0; wi < h->waves.size(); ++wi) {
        const WavePlan& wp = h->waves[wi];
        // every chunk of the wave formed into its slice of the arena
        for (int c = wp.c0; c < wp.c0 + wp.nc; ++c) {
          const ChunkPlan& cp = h->plan[c];
          int rc = run_element_chunk(h, cp.g, nullptr, cp.count, st, false, false, cp.real, &cp, true, true,
                                     arena + cp.koff);
          if (rc) return rc;
        }
        int rc = DPG_OK;
        if (h->factor_arith == DPG_FACTOR_TC_SPLIT) {
          rc = factor_wave(h, (int)wi, st);
        } else {  // FP64-pipe factorisation: one launch per chunk of the wave
          for (int c = wp.c0; c < wp.c0 + wp.nc && rc == DPG_OK; ++c) {
            const ChunkPlan& cp = h->plan[c];
            rc = run_element_chunk(h, cp.g, nullptr, cp.count, st, true, false, cp.real, &cp, false, false,
                                   arena + cp.koff);
          }
        }
        if (rc) return rc;
        // extraction (and in streaming mode assembly) chunk by chunk
        for (int c = wp.c0; c < wp.c0 + wp.nc; ++c) {
          const ChunkPlan& cp = h->plan[c];
          rc = run_element_chunk(h, cp.g, nullptr, cp.count, st, false, true, cp.real, &cp, false, false,
                                 arena + cp.koff);
          if (rc == DPG_OK && h->stream) rc = assemble_chunk(h, cp.g, cp.d_ids + cp.ids_off, cp.count, st);
          if (rc) return rc;
        }
      }
      return DPG_OK;
    }
    for (const ChunkPlan& cp : h->plan) {
      int rc = run_element_chunk(h, cp.g, nullptr, cp.count, st, true, true, cp.real, &cp);
      if (rc == DPG_OK && h->stream) rc = assemble_chunk(h, cp.g, cp.d_ids + cp.ids_off, cp.count, st);
      if (rc) return rc;
    }
    return DPG_OK;
  };
  if (!h->use_graph) return pass(s);
  if (!h->graph_valid || h->graph_timing != h->timing) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    if (!h->cap_stream) DPG_CUDA_TRY(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    DPG_CUDA_TRY(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = h->launches;
    int rc = pass(h->cap_stream);
    cudaGraph_t gr = nullptr;
    cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &gr);
    if (rc == DPG_OK && ee != cudaSuccess) {
      h->err = std::string("element pass capture: ") + cudaGetErrorString(ee);
      rc = DPG_ERR_CUDA;
    }
    if (rc == DPG_OK && cudaGraphInstantiate(&h->graph, gr, 0) != cudaSuccess) {
      h->err = "element pass graph instantiation failed";
      rc = DPG_ERR_CUDA;
    }
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    h->graph_launches = h->launches - l0;
    h->launches = l0;
    if (rc) {
      if (h->graph) cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
      return rc;
    }
    h->graph_valid = true;
    h->graph_timing = h->timing;
  }
  DPG_CUDA_TRY(h, cudaGraphLaunch(h->graph, s));
  h->launches += h->graph_launches;
  return DPG_OK;
}

// Chunk-size autotuner: per group, time one chunk of the group's larger
// arithmetic class at each candidate size (multiples of the SM count up to the
// byte budget) and keep the fastest per element.  Stores of the timed elements
// are overwritten (a full element pass rewrites them).
int autotune(dpg_handle* h, double max_bytes, int32_t* caps, float* ms_per_elem, cudaStream_t s) {
  if (h->bucketed) {
    h->err = "the autotuner sizes per-order chunks; the order-bucketed pass sizes waves";
    return DPG_ERR_UNSUPPORTED;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t e0, e1;
  DPG_CUDA_TRY(h, cudaEventCreate(&e0));
  DPG_CUDA_TRY(h, cudaEventCreate(&e1));
  int rc = DPG_OK;
  for (int g = 0; g < (int)h->grp.size() && rc == DPG_OK; ++g) {
    Group& G = h->grp[g];
    const bool real = h->allow_real && G.real_elems.size() >= G.cplx_elems.size();
    const std::vector<int>& L = !h->allow_real ? G.elems : (real ? G.real_elems : G.cplx_elems);
    const int n = (int)L.size();
    const size_t per = chunk_bytes(G.sz, h->prec == DPG_PREC_FP64);
    std::vector<int> cand;
    for (int k : {1, 2, 3, 4, 6, 8, 12, 16})
      if (k * sms <= n && (double)per * k * sms <= max_bytes) cand.push_back(k * sms);
    if (cand.empty()) cand.push_back(std::max(1, std::min(n, (int)(max_bytes / per))));
    const int keep = G.cap;
    int best = keep;
    float best_ms = 1e30f;
    for (int c : cand) {
      G.cap = c;
      rc = alloc_workspace(h);
      if (rc) break;
      float ms = 1e30f;
      for (int rep = 0; rep < 2 && rc == DPG_OK; ++rep) {
        cudaEventRecord(e0, s);
        rc = run_element_chunk(h, g, L.data(), c, s, true, true, real);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = DPG_ERR_CUDA;
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep == 1) ms = t;
      }
      if (rc) break;
      if (ms / c < best_ms) {
        best_ms = ms / c;
        best = c;
      }
    }
    G.cap = rc ? keep : best;
    if (caps) caps[g] = G.cap;
    if (ms_per_elem) ms_per_elem[g] = best_ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int rc2 = alloc_workspace(h);
  return rc ? rc : rc2;
}

// Cholesky of the G block alone for the current chunk (rows below untouched).
int factor_gram_only(dpg_handle* h, int g, int count, cudaStream_t s) {
  const Sizes& S = h->grp[g].sz;
  if (h->factor_arith == DPG_FACTOR_TC_SPLIT) {
    if (factor_tc_launch(true, count, S.N, S.n_v, S.n_v, S.n_v, h->ws.ids, h->ws.K, h->d_status,
                         h->d_status + h->ne, h->ws.Q, s) != DPG_OK) {
      h->err = "tensor-core factorisation launch failed";
      return DPG_ERR_CUDA;
    }
  } else {
    const size_t smem = factor_smem<double2>();
    k_factor<double2><<<count, 256, smem, s>>>(S.N, S.n_v, S.n_v, S.n_v, h->ws.ids, h->ws.K, h->d_status);
  }
  h->launches += 1;
  DPG_CUDA_TRY(h, cudaGetLastError());
  return DPG_OK;
}

// ------------------------------------------------- recovery and estimator --
// Local recovery u_K = M1^{-1}(M4 l - M2 uhat) (Sec. 2.3) from the stored
// Z = M1^{-1} M2 and z = M1^{-1} M4 l of the element pass, and the residual
// estimator eta_K = ||Psi_K||_V with Psi_K = G_K^{-1} r_K, r_K = l - B u - B-hat uhat,
// by its definition: G_K, B_K, B-hat_K, l_K are formed again, r_K replaces the
// first column after G in the augmented matrix, and the factorisation kernel
// takes the n_v pivots of G; the entry below them is then
// 0 - ||L^{-1} r_K||^2 = -eta_K^2, accumulated as a sum of squares (no
// cancellation beyond the one inside r_K itself).

__device__ __forceinline__ double2 trace_value(const int32_t* l2g, const double2* fix, const double2* x, size_t k) {
  const int g = l2g[k];
  if (g >= 0) return x[g];
  if (g == -1) return fix[k];
  return make_double2(0.0, 0.0);
}

__device__ __forceinline__ double est_wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// u = z - Z uhat_slots for the elements of one group (one CTA per element).
__global__ void __launch_bounds__(256) k_recover_u(int nh, int nu, const int* __restrict__ elems,
                                                   const ElemOff* __restrict__ off, const ElemOff* __restrict__ soff,
                                                   const int32_t* __restrict__ l2g,
                                                   const double2* __restrict__ xfix, const double2* __restrict__ xhat,
                                                   const double2* __restrict__ Zst, const double2* __restrict__ zst,
                                                   double2* u_out) {
  extern __shared__ double2 su_sh[];
  const int e = elems[blockIdx.x];
  const ElemOff of = off[e];
  Zst += soff[e].Z;
  zst += soff[e].u;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < nh; t += blockDim.x) su_sh[t] = trace_value(l2g, xfix, xhat, (size_t)of.h + t);
  __syncthreads();
  const double2* Ze = Zst;
  for (int i = wid; i < nu; i += nw) {
    double yr = 0.0, yi = 0.0;
    for (int j = lane; j < nh; j += 32) {
      const double2 v = Ze[(size_t)i * nh + j], x = su_sh[j];
      yr = fma(v.x, x.x, fma(-v.y, x.y, yr));
      yi = fma(v.x, x.y, fma(v.y, x.x, yi));
    }
    yr = est_wsum(yr);
    yi = est_wsum(yi);
    if (lane == 0) {
      const double2 zi = zst[i];
      u_out[of.u + i] = make_double2(zi.x - yr, zi.y - yi);
    }
  }
}

// The residual's unknowns of element e into w (m = n_u + n_h entries): u
// recovered from the stored Z, z and the trace solution, then the element's
// own trace coefficients uhat_K = R_K uhat_slots; with `phased` (the real
// path's w_r = D_w^H w) the E and E-hat entries are multiplied by i.  us:
// shared scratch of n_h entries; u_out (may be NULL) receives u.
__device__ __forceinline__ void est_w(const Sizes& S, int e, const ElemOff& of, const ElemOff* __restrict__ soff,
                                      const int* __restrict__ sig, const RSig* __restrict__ rsig,
                                      const int32_t* __restrict__ rint, const double* __restrict__ rdbl,
                                      const int32_t* __restrict__ l2g, const double2* __restrict__ xfix,
                                      const double2* __restrict__ xhat, const double2* __restrict__ Zst,
                                      const double2* __restrict__ zst, double2* w, double2* us, double2* u_out,
                                      bool phased) {
  const int nu = S.n_u, nh = S.n_h, nE = 3 * S.nL, nt = S.nt;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < nh; t += blockDim.x) us[t] = trace_value(l2g, xfix, xhat, (size_t)of.h + t);
  __syncthreads();
  const double2* Ze = Zst + soff[e].Z;
  for (int i = wid; i < nu; i += nw) {
    double yr = 0.0, yi = 0.0;
    for (int j = lane; j < nh; j += 32) {
      const double2 v = Ze[(size_t)i * nh + j], x = us[j];
      yr = fma(v.x, x.x, fma(-v.y, x.y, yr));
      yi = fma(v.x, x.y, fma(v.y, x.x, yi));
    }
    yr = est_wsum(yr);
    yi = est_wsum(yi);
    if (lane == 0) {
      const double2 zi = zst[soff[e].u + i];
      const double2 ui = make_double2(zi.x - yr, zi.y - yi);
      if (u_out) u_out[of.u + i] = ui;
      w[i] = (phased && i < nE) ? make_double2(-ui.y, ui.x) : ui;  // times conj(-i) = i on E
    }
  }
  const int sg = sig[e];
  for (int t = threadIdx.x; t < nh; t += blockDim.x) {
    double2 a;
    if (sg >= 0) {  // uhat_K = R uhat (slots)
      const RSig R = rsig[sg];
      const int32_t* rp = rint + R.rptr;
      const int32_t* ri = rint + R.ridx;
      const double* rw = rdbl + R.rw;
      const int tt = t < nt ? t : t - nt, base = t < nt ? 0 : nt;
      a = make_double2(0.0, 0.0);
      for (int k = rp[tt]; k < rp[tt + 1]; ++k) {
        const double2 x = us[base + ri[k]];
        a.x = fma(rw[k], x.x, a.x);
        a.y = fma(rw[k], x.y, a.y);
      }
    } else {
      a = us[t];
    }
    w[nu + t] = (phased && t < nt) ? make_double2(-a.y, a.x) : a;  // times i on E-hat
  }
  __syncthreads();
}

// eta_K^2 of the stored-factor estimator: the element pass leaves
// X = (L^{-1} [B | B-hat | l])^H below G's factor (columns 0..n_v-1 of rows
// n_v..N-1; the later pivots never touch them), kept per element column by
// column (n_v columns of m + 1 entries).  L^{-1} r = L^{-1} l - L^{-1} B u -
// L^{-1} B-hat uhat_K: y_i = conj(X[m][i]) - sum_t conj(X[t][i]) w_t, and
// eta_K^2 = ||y||^2 (Sec. 2.3).  Real path: X_r real, no load, w phased,
// y_r = -X_r^T w_r (real and imaginary parts).  One block per element.
template <bool REAL>
__global__ void __launch_bounds__(256) k_est_stored(Sizes S, const int* __restrict__ ids, const ElemOff* __restrict__ off,
                                                    const ElemOff* __restrict__ soff, const int* __restrict__ sig,
                                                    const RSig* __restrict__ rsig, const int32_t* __restrict__ rint,
                                                    const double* __restrict__ rdbl, const int32_t* __restrict__ l2g,
                                                    const double2* __restrict__ xfix,
                                                    const double2* __restrict__ xhat,
                                                    const double2* __restrict__ Zst,
                                                    const double2* __restrict__ zst, const double* __restrict__ Xst,
                                                    const int64_t* __restrict__ xoff, double2* u_out, double* eta2) {
  extern __shared__ double2 es_sh[];
  const int e = ids[blockIdx.x];
  const ElemOff of = off[e];
  const int nv = S.n_v, m = S.n_u + S.n_h;
  double2* w = es_sh;       // m
  double2* us = w + m;      // nh
  __shared__ double part[256 / 32];
  est_w(S, e, of, soff, sig, rsig, rint, rdbl, l2g, xfix, xhat, Zst, zst, w, us, u_out, REAL);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double acc = 0.0;  // sum of |y_i|^2 over this warp's rows i
  if (REAL) {
    const double* X = Xst + xoff[e];
    for (int i = wid; i < nv; i += nw) {
      const double* col = X + (size_t)i * (m + 1);
      double yr = 0.0, yi = 0.0;
      for (int t = lane; t < m; t += 32) {
        const double b = col[t];
        const double2 x = w[t];
        yr = fma(b, x.x, yr);
        yi = fma(b, x.y, yi);
      }
      yr = est_wsum(yr);
      yi = est_wsum(yi);
      acc += yr * yr + yi * yi;
    }
  } else {
    const double2* X = reinterpret_cast<const double2*>(Xst + xoff[e]);
    for (int i = wid; i < nv; i += nw) {
      const double2* col = X + (size_t)i * (m + 1);
      double yr = 0.0, yi = 0.0;
      for (int t = lane; t < m; t += 32) {
        const double2 b = col[t], x = w[t];  // conj(b) x
        yr = fma(b.x, x.x, fma(b.y, x.y, yr));
        yi = fma(b.x, x.y, fma(-b.y, x.x, yi));
      }
      yr = est_wsum(yr);
      yi = est_wsum(yi);
      const double2 l = col[m];  // conj(L^{-1} l)_i
      const double dr = l.x - yr, di = -l.y - yi;
      acc += dr * dr + di * di;
    }
  }
  if (lane == 0) part[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += part[k];
    eta2[e] = t;
  }
}

// Per element of a chunk (K freshly formed, not factored): u, the element's
// own trace coefficients uhat_K = R_K uhat_slots, r = l - B u - B-hat uhat_K
// (B[i][j] = conj(K[n_v + j][i]), l_i = conj(K[N-1][i])); K[n_v][i] = conj(r_i),
// K[n_v][n_v] = 0.
__global__ void __launch_bounds__(256) k_est_residual(Sizes S, const int* __restrict__ ids,
                                                      const ElemOff* __restrict__ off,
                                                      const ElemOff* __restrict__ soff, const int* __restrict__ sig,
                                                      const RSig* __restrict__ rsig, const int32_t* __restrict__ rint,
                                                      const double* __restrict__ rdbl, const int32_t* __restrict__ l2g,
                                                      const double2* __restrict__ xfix,
                                                      const double2* __restrict__ xhat,
                                                      const double2* __restrict__ Zst,
                                                      const double2* __restrict__ zst, double2* K, double2* u_out) {
  extern __shared__ double2 er_sh[];
  const int slot = blockIdx.x, e = ids[slot];
  const ElemOff of = off[e];
  const int N = S.N, nv = S.n_v, nu = S.n_u, nh = S.n_h, m = nu + nh;
  double2* w = er_sh;       // m: u, then uhat_K
  double2* us = w + m;      // nh: uhat in the trace slots
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double2* A = K + (size_t)slot * N * N;
  est_w(S, e, of, soff, sig, rsig, rint, rdbl, l2g, xfix, xhat, Zst, zst, w, us, u_out, false);
  for (int i = wid; i < nv; i += nw) {
    const double2* col = A + (size_t)i * N + nv;
    double rr = 0.0, ri2 = 0.0;
    for (int j = lane; j < m; j += 32) {
      const double2 b = col[j], x = w[j];  // B[i][j] = conj(b)
      rr = fma(b.x, x.x, fma(b.y, x.y, rr));
      ri2 = fma(b.x, x.y, fma(-b.y, x.x, ri2));
    }
    rr = est_wsum(rr);
    ri2 = est_wsum(ri2);
    if (lane == 0) {
      const double2 lc = col[m];  // conj(l_i)
      A[(size_t)nv + (size_t)i * N] = make_double2(lc.x - rr, -(-lc.y - ri2));  // conj(l_i - (B w)_i)
    }
  }
  if (threadIdx.x == 0) A[(size_t)nv + (size_t)nv * N] = make_double2(0.0, 0.0);
}

// Real path (lossless element, no Robin face, no load): the chunk holds the
// phase-scaled real matrix K_r = D^H K D with D = diag(1 on F, -i on I | -i on E,
// 1 on H | -i on E-hat, 1 on H-hat).  With w_r = D_w^H (u, uhat_K),
// r_r = D_t^H r = -B_r w_r and eta_K^2 = r_r^H G_r^{-1} r_r
// = ||L_r^{-1} Re r_r||^2 + ||L_r^{-1} Im r_r||^2: Re r_r and Im r_r become
// rows n_v and n_v + 1 of K_r (two more columns of the real factorisation).
__global__ void __launch_bounds__(256) k_est_residual_real(Sizes S, const int* __restrict__ ids,
                                                           const ElemOff* __restrict__ off,
                                                           const ElemOff* __restrict__ soff,
                                                           const int* __restrict__ sig, const RSig* __restrict__ rsig,
                                                           const int32_t* __restrict__ rint,
                                                           const double* __restrict__ rdbl,
                                                           const int32_t* __restrict__ l2g,
                                                           const double2* __restrict__ xfix,
                                                           const double2* __restrict__ xhat,
                                                           const double2* __restrict__ Zst,
                                                           const double2* __restrict__ zst, double* K, double2* u_out) {
  extern __shared__ double2 err_sh[];
  const int slot = blockIdx.x, e = ids[slot];
  const ElemOff of = off[e];
  const int N = S.N, nv = S.n_v, nu = S.n_u, nh = S.n_h, m = nu + nh;
  double2* w = err_sh;      // m: u_r, then uhat_r
  double2* us = w + m;      // nh: uhat in the trace slots
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* A = K + (size_t)slot * N * N;
  est_w(S, e, of, soff, sig, rsig, rint, rdbl, l2g, xfix, xhat, Zst, zst, w, us, u_out, true);
  for (int i = wid; i < nv; i += nw) {
    const double* col = A + (size_t)i * N + nv;
    double rr = 0.0, ri2 = 0.0;
    for (int j = lane; j < m; j += 32) {
      const double b = col[j];
      const double2 x = w[j];
      rr = fma(b, x.x, rr);
      ri2 = fma(b, x.y, ri2);
    }
    rr = est_wsum(rr);
    ri2 = est_wsum(ri2);
    if (lane == 0) {  // r_r = -B_r w_r
      A[(size_t)nv + (size_t)i * N] = -rr;
      A[(size_t)nv + 1 + (size_t)i * N] = -ri2;
    }
  }
  if (threadIdx.x == 0) {
    A[(size_t)nv + (size_t)nv * N] = 0.0;
    A[(size_t)nv + 1 + (size_t)nv * N] = 0.0;
    A[(size_t)nv + 1 + (size_t)(nv + 1) * N] = 0.0;
  }
}

__global__ void k_est_eta_real(int count, int N, int nv, const int* __restrict__ ids, const double* __restrict__ K,
                               double* eta2, int* nneg) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= count) return;
  const double* A = K + (size_t)slot * N * N;
  double v = -(A[(size_t)nv + (size_t)nv * N] + A[(size_t)nv + 1 + (size_t)(nv + 1) * N]);
  if (v < 0.0) {
    atomicAdd(nneg, 1);
    v = 0.0;
  }
  eta2[ids[slot]] = v;
}

// eta_K^2 = -K[n_v][n_v] after the n_v pivots of G (negative values, possible
// only through rounding when eta_K ~ 0, are clamped to 0 and counted).
__global__ void k_est_eta(int count, int N, int nv, const int* __restrict__ ids, const double2* __restrict__ K,
                          double* eta2, int* nneg) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= count) return;
  double v = -K[(size_t)slot * N * N + (size_t)nv + (size_t)nv * N].x;
  if (v < 0.0) {
    atomicAdd(nneg, 1);
    v = 0.0;
  }
  eta2[ids[slot]] = v;
}

int recover_u(dpg_handle* h, const double2* xhat, double2* u, cudaStream_t s) {
  if (h->stream) {  // condense every chunk again into the chunk stores, then recover
    if (!h->plan_valid) {
      int rc = build_plan(h);
      if (rc) return rc;
    }
    for (const ChunkPlan& cp : h->plan) {
      const Sizes& S = h->grp[cp.g].sz;
      int rc = run_element_chunk(h, cp.g, nullptr, cp.count, s, true, true, cp.real, &cp);
      if (rc) return rc;
      k_recover_u<<<cp.count, 256, sizeof(double2) * S.n_h, s>>>(S.n_h, S.n_u, cp.d_ids + cp.ids_off, h->d_off,
                                                                  h->d_soff, h->d_l2g, h->d_xfix, xhat, h->d_Z,
                                                                  h->d_z, u);
      h->launches += 1;
    }
    return DPG_OK;
  }
  for (const Group& G : h->grp) {
    const Sizes& S = G.sz;
    k_recover_u<<<(int)G.elems.size(), 256, sizeof(double2) * S.n_h, s>>>(S.n_h, S.n_u, G.d_elems, h->d_off,
                                                                          h->d_off, h->d_l2g, h->d_xfix, xhat,
                                                                          h->d_Z, h->d_z, u);
    h->launches += 1;
  }
  return DPG_OK;
}

// The estimator's recompute pass over the est_plan chunks: eta_K^2 into eta2[e]
// (and u when given).  Uses the chunk workspace only; allocates nothing.
int estimate_pass(dpg_handle* h, const double2* xhat, double2* u, double* eta2, cudaStream_t s) {
  if (!h->plan_valid) {
    h->err = "the estimator's launch plan is built by dpg_element_batch";
    return DPG_ERR_STATE;
  }
  DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_est_neg, 0, sizeof(int), s));
  const bool stored = h->d_Xst && h->xst_valid && h->have_elements && !h->stream;
  for (const ChunkPlan& cp : h->plan) {
    const Group& G = h->grp[cp.g];
    const Sizes& S = G.sz;
    if (stored) {  // y = L^{-1} r from the X kept by the element pass: no second pass
      const int* ids = cp.d_ids + cp.ids_off;
      const size_t sh = sizeof(double2) * (size_t)(S.n_u + 2 * S.n_h);
      if (cp.real)
        k_est_stored<true><<<cp.count, 256, sh, s>>>(S, ids, h->d_off, h->d_soff, h->d_sig, h->d_rsig, h->d_rint,
                                                     h->d_rdbl, h->d_l2g, h->d_xfix, xhat, h->d_Z, h->d_z, h->d_Xst,
                                                     h->d_xst_off, u, eta2);
      else
        k_est_stored<false><<<cp.count, 256, sh, s>>>(S, ids, h->d_off, h->d_soff, h->d_sig, h->d_rsig, h->d_rint,
                                                      h->d_rdbl, h->d_l2g, h->d_xfix, xhat, h->d_Z, h->d_z, h->d_Xst,
                                                      h->d_xst_off, u, eta2);
      DPG_CUDA_TRY(h, cudaGetLastError());
      h->launches += 1;
      continue;
    }
    int rc = DPG_OK;
    if (h->stream) {
      // the chunk's Z, z again (condensation into the chunk stores), then K
      // formed again from the same quadrature matrices
      rc = run_element_chunk(h, cp.g, nullptr, cp.count, s, true, true, cp.real, &cp);
      if (rc == DPG_OK) rc = run_element_chunk(h, cp.g, nullptr, cp.count, s, false, false, cp.real, &cp, false);
    } else {
      rc = run_element_chunk(h, cp.g, nullptr, cp.count, s, false, false, cp.real, &cp);
    }
    if (rc) return rc;
    const int* ids = cp.d_ids + cp.ids_off;
    const size_t sh = sizeof(double2) * (size_t)(S.n_u + 2 * S.n_h);
    double* Kr = reinterpret_cast<double*>(h->ws.K);
    const int extra = cp.real ? 2 : 1;  // columns after G: Re r, Im r (real path) or r
    if (cp.real)
      k_est_residual_real<<<cp.count, 256, sh, s>>>(S, ids, h->d_off, h->d_soff, h->d_sig, h->d_rsig, h->d_rint,
                                                    h->d_rdbl,
                                                    h->d_l2g, h->d_xfix, xhat, h->d_Z, h->d_z, Kr, u);
    else
      k_est_residual<<<cp.count, 256, sh, s>>>(S, ids, h->d_off, h->d_soff, h->d_sig, h->d_rsig, h->d_rint, h->d_rdbl,
                                               h->d_l2g,
                                               h->d_xfix, xhat, h->d_Z, h->d_z, h->ws.K, u);
    if (h->factor_arith == DPG_FACTOR_TC_SPLIT) {
      if (factor_tc_launch(!cp.real, cp.count, S.N, S.n_v + extra, S.n_v, S.n_v, ids,
                           cp.real ? (void*)Kr : (void*)h->ws.K, h->d_status, h->d_status + h->ne, h->ws.Q,
                           s) != DPG_OK) {
        h->err = "tensor-core factorisation launch failed";
        return DPG_ERR_CUDA;
      }
    } else if (cp.real) {
      k_factor<double><<<cp.count, 256, factor_smem<double>(), s>>>(S.N, S.n_v + extra, S.n_v, S.n_v, ids, Kr,
                                                                    h->d_status);
    } else {
      k_factor<double2><<<cp.count, 256, factor_smem<double2>(), s>>>(S.N, S.n_v + extra, S.n_v, S.n_v, ids,
                                                                      h->ws.K, h->d_status);
    }
    if (cp.real)
      k_est_eta_real<<<(cp.count + 127) / 128, 128, 0, s>>>(cp.count, S.N, S.n_v, ids, Kr, eta2, h->d_est_neg);
    else
      k_est_eta<<<(cp.count + 127) / 128, 128, 0, s>>>(cp.count, S.N, S.n_v, ids, h->ws.K, eta2, h->d_est_neg);
    h->launches += 3;
    DPG_CUDA_TRY(h, cudaGetLastError());
  }
  return DPG_OK;
}

}  // namespace dpg

// Check hook of the factorisation kernels (declared in dpg.h).
extern "C" int dpg_factor_check(int32_t arith, int32_t cplx, int32_t N, int32_t nact, int32_t nv, int32_t npiv,
                                const double* A, double* out, int32_t* not_hpd) {
  using namespace dpg;
  if (!A || !out || N <= 0 || nact < 0 || nact > N || nv < 0 || npiv < 0 || npiv > nact || nv > npiv ||
      (arith != DPG_FACTOR_FP64 && arith != DPG_FACTOR_TC_SPLIT))
    return DPG_ERR_ARG;
  if (N > 3315) return DPG_ERR_UNSUPPORTED;
  const size_t elems = (size_t)N * N * (cplx ? 2 : 1);
  double* dA = nullptr;
  int* dst = nullptr;  // [0]: ids, [1]: pivot flag, [2]: timeout flag
  uint8_t* dQ = nullptr;
  const size_t qbytes = factor_tc_scratch_bytes(N, cplx != 0);
  int rc = DPG_OK;
  if (cudaMalloc(&dA, elems * 8) != cudaSuccess || cudaMalloc(&dst, 3 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&dQ, qbytes) != cudaSuccess)
    rc = DPG_ERR_NOMEM;
  const int zero3[3] = {0, 0, 0};
  if (rc == DPG_OK && (cudaMemcpy(dA, A, elems * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
                       cudaMemcpy(dst, zero3, sizeof(zero3), cudaMemcpyHostToDevice) != cudaSuccess))
    rc = DPG_ERR_CUDA;
  if (rc == DPG_OK) {
    if (arith == DPG_FACTOR_TC_SPLIT) {
      rc = factor_tc_init();
      if (rc == DPG_OK) rc = factor_tc_launch(cplx != 0, 1, N, nact, nv, npiv, dst, dA, dst + 1, dst + 2, dQ, nullptr);
    } else if (cplx) {
      cudaFuncSetAttribute(k_factor<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)factor_smem<double2>());
      k_factor<double2><<<1, 256, factor_smem<double2>()>>>(N, nact, nv, npiv, dst, reinterpret_cast<double2*>(dA),
                                                             dst + 1);
    } else {
      cudaFuncSetAttribute(k_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)factor_smem<double>());
      k_factor<double><<<1, 256, factor_smem<double>()>>>(N, nact, nv, npiv, dst, dA, dst + 1);
    }
  }
  int hst[3] = {0, 0, 0};
  if (rc == DPG_OK && (cudaDeviceSynchronize() != cudaSuccess ||
                       cudaMemcpy(hst, dst, sizeof(hst), cudaMemcpyDeviceToHost) != cudaSuccess ||
                       cudaMemcpy(out, dA, elems * 8, cudaMemcpyDeviceToHost) != cudaSuccess))
    rc = DPG_ERR_CUDA;
  if (rc == DPG_OK && hst[2]) rc = DPG_ERR_TIMEOUT;
  if (not_hpd) *not_hpd = hst[1];
  cudaFree(dA);
  cudaFree(dst);
  cudaFree(dQ);
  return rc;
}

namespace dpg {

// Reference matrices on the unit cube: X_ref = Cu^T V (metric free) and the
// per-face trace pairings T_f = Vt^T NxP, T_all = sum_f T_f.
__global__ void k_sum_faces(int n, const double* Tf, double* Tall) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int f = 0; f < 6; ++f) s += Tf[(size_t)f * n + t];
    Tall[t] = s;
  }
}

__global__ void k_copy_cols(int rows, int ncol, const double* src, int lds, long long ss, int c0, double* dst,
                            long long sd) {
  const int b = blockIdx.y;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rows * ncol; t += gridDim.x * blockDim.x) {
    int i = t / ncol, j = t - i * ncol;
    dst[b * sd + (size_t)i * ncol + j] = src[b * ss + (size_t)i * lds + c0 + j];
  }
}

int compute_reference_matrices(dpg_handle* h, int g, cudaStream_t s) {
  Group& G = h->grp[g];
  const Sizes& S = G.sz;
  Workspace& w = h->ws;
  // unit cube as a temporary element: reuse d_X slot of element 0 is not allowed;
  // allocate a private corner array
  double Xu[24];
  for (int v = 0; v < 8; ++v)
    for (int a = 0; a < 3; ++a) Xu[3 * v + a] = (double)((v >> a) & 1);
  double* dXu = nullptr;
  int* dids = nullptr;
  DPG_CUDA_TRY(h, cudaMalloc(&dXu, sizeof(Xu)));
  DPG_CUDA_TRY(h, cudaMalloc(&dids, sizeof(int) * 32));
  int zeros[32] = {0};
  DPG_CUDA_TRY(h, cudaMemcpyAsync(dXu, Xu, sizeof(Xu), cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(dids, zeros, sizeof(zeros), cudaMemcpyHostToDevice, s));
  k_vol_arrays<<<dim3((S.nq + QB - 1) / QB, 1), 256, 0, s>>>(G.tab, S, dXu, dids, w.V, w.Cu, w.PhiL);
  const size_t nq3 = 3 * (size_t)S.nq;
  gemm_tn(S.n_f, S.n_f, (int)nq3, w.Cu, S.n_f, 0, w.V, S.n_f, 0, G.d_Xref, S.n_f, 0, 1, s);
  // faces of the unit cube
  int rent[24];
  for (int f = 0; f < 6; ++f) {
    rent[4 * f + 0] = 0;
    rent[4 * f + 1] = f;
    rent[4 * f + 2] = 0;
    rent[4 * f + 3] = 0;
  }
  DPG_CUDA_TRY(h, cudaMemcpyAsync(w.rent, rent, sizeof(rent), cudaMemcpyHostToDevice, s));
  const int Wf = 2 * S.n_f + 2 * S.nt + 2;
  k_face_arrays<<<dim3(1, 6), 256, 0, s>>>(G.tab, S, dXu, w.rent, h->d_robin, G.d_trfun, h->omega, 1, w.FV);
  gemm_tn(S.n_f, Wf, 3 * S.nqf, w.FV, Wf, (long long)3 * S.nqf * Wf, w.FV, Wf, (long long)3 * S.nqf * Wf, w.FR, Wf,
          (long long)S.n_f * Wf, 6, s);
  // T_f = columns [2 n_f + nt, 2 n_f + 2 nt) of FR
  k_copy_cols<<<dim3(64, 6), 256, 0, s>>>(S.n_f, S.nt, w.FR, Wf, (long long)S.n_f * Wf, 2 * S.n_f + S.nt, G.d_Tf,
                                         (long long)S.n_f * S.nt);
  k_sum_faces<<<64, 256, 0, s>>>(S.n_f * S.nt, G.d_Tf, G.d_Tall);
  DPG_CUDA_TRY(h, cudaGetLastError());
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  cudaFree(dXu);
  cudaFree(dids);
  return DPG_OK;
}

}  // namespace dpg
