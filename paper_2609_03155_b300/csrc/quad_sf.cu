// Sum-factorised quadrature of the element matrices (Sec. 2.3; the remedy for
// element cost that Sec. 5 names), FP64.
//
// Every test function of the order-rt Nedelec space is a tensor product
// f_i(x) = a_{i0}(x0) a_{i1}(x1) a_{i2}(x2) of 1D Lagrange factors (open family
// along its component, closed across), and the trial functions L_l are tensor
// products of Gauss-Legendre Lagrange factors.  On the tensor Gauss rule with
// Q points per direction every contraction the element pass needs has the form
//
//   out_{ij} = sum_{q0,q1,q2} A0_{i0 q0} B0_{j0 q0} A1_{i1 q1} B1_{j1 q1}
//                             A2_{i2 q2} B2_{j2 q2} W(q0, q1, q2)
//
// with a per-point geometric weight W.  It is evaluated direction by
// direction: T1 = contraction over q2, T2 over q1, out over q0, in
// O(n^2 Q^3 + n^4 Q^2 + n^6 Q) instead of the O(n^6 Q^3) of the dense product
// (n = 1D functions per direction).  The weights, from the trilinear map with
// J = dx/dxi and w the tensor Gauss weight:
//   M_ij = sum_q w det J (J^{-1} J^{-T})_{c_i c_j} f_i f_j            (mass, covariant Piola)
//   C_ij = sum_q (w / det J) (J^T J)_{ab} (curl f_i)_a (curl f_j)_b   (curl-curl)
//   P_{i, d nL + l} = sum_q w det J (J^{-1})_{c_i d} f_i L_l
//   Q_{i, d nL + l} = sum_q w J_{da} (curl f_i)_a L_l
// with the reference curl of f e_c equal to grad f x e_c: component a != c is
// eps_{a k c} d_k f, k the third direction.  M and C are symmetric; only
// their upper triangle (row <= column) is formed, as the consumers read it.
#include "dpg_internal.h"
#include "geom.cuh"

namespace dpg {

// Per-point weights, 30 per point, layout [slot][30][nq]:
//   0..5   w det (J^{-1} J^{-T})_{cd}, pairs 00 11 22 01 02 12
//   6..11  (w / det) (J^T J)_{ab}, same pairs
//   12..20 w det (J^{-1})_{cd} at 12 + 3c + d
//   21..29 w J_{da} at 21 + 3d + a
constexpr int NWQ = 30;

__global__ void __launch_bounds__(128) k_quad_geom(const __grid_constant__ Tables T, Sizes S,
                                                   const double* __restrict__ Xall, const int* __restrict__ ids,
                                                   double* __restrict__ WQ) {
  const int slot = blockIdx.y;
  const int e = ids[slot];
  __shared__ double sX[24];
  if (threadIdx.x < 24) sX[threadIdx.x] = Xall[(size_t)e * 24 + threadIdx.x];
  __syncthreads();
  const int nq1 = S.nq1, nq = S.nq;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int qi[3] = {q % nq1, (q / nq1) % nq1, q / (nq1 * nq1)};
  const double xi[3] = {T.pt[qi[0]], T.pt[qi[1]], T.pt[qi[2]]};
  double J[3][3], x[3], Ji[3][3];
  geom(sX, xi, J, x);
  const double det = inv3(J, Ji);
  const double w = T.w[qi[0]] * T.w[qi[1]] * T.w[qi[2]];
  double* o = WQ + (size_t)slot * NWQ * nq + q;
  const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int c = pa[k], d = pb[k];
    o[(size_t)k * nq] = w * det * (Ji[c][0] * Ji[d][0] + Ji[c][1] * Ji[d][1] + Ji[c][2] * Ji[d][2]);
    o[(size_t)(6 + k) * nq] = (w / det) * (J[0][c] * J[0][d] + J[1][c] * J[1][d] + J[2][c] * J[2][d]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      o[(size_t)(12 + 3 * c + d) * nq] = w * det * Ji[c][d];
      o[(size_t)(21 + 3 * c + d) * nq] = w * J[c][d];  // c plays d (row of J), d plays a
    }
}

// One side of a contraction: per direction the 1D family, value or
// derivative, and the number of functions.
struct Side {
  int fam[3], der[3], n[3];
};

__device__ __forceinline__ Side test_side(const Tables& T, int c, int dder) {
  Side s;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s.fam[k] = (k == c) ? F_OPEN_T : F_CLOSED_T;
    s.der[k] = (k == dder) ? 1 : 0;
    s.n[k] = T.nfun[s.fam[k]];
  }
  return s;
}

__device__ __forceinline__ Side trial_side(const Tables& T) {
  Side s;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s.fam[k] = F_L2;
    s.der[k] = 0;
    s.n[k] = T.nfun[F_L2];
  }
  return s;
}

__device__ __forceinline__ double tab(const Tables& T, const Side& s, int k, int q, int i) {
  return s.der[k] ? T.der[s.fam[k]][q][i] : T.val[s.fam[k]][q][i];
}

template <int P>
struct SfDims {
  static constexpr int Q = P + 3;                            // Gauss points per direction
  static constexpr int NQ = Q * Q * Q;
  static constexpr int NCL = P + 3;                          // largest 1D family (closed, order rt = p + 2)
  static constexpr int RT = P + 2;
  static constexpr int NCOMP = RT * (RT + 1) * (RT + 1);     // test functions per component
  static constexpr int NF = 3 * NCOMP;
  static constexpr int NL = (P + 1) * (P + 1) * (P + 1);
  static constexpr int NL3 = 3 * NL;
  // W, three product tables, T1, T2 (doubles)
  static constexpr int SMEM = NQ + 3 * NCL * NCL * Q + NCL * NCL * Q * Q + NCL * NCL * NCL * NCL * Q;
};

// out (+)= coef * contraction(si, sj, W) over the block's 256 threads; with
// `upper` only entries with row <= column are formed.  The thread that writes
// an entry is a function of the side dimensions only, so the contractions of
// one job that accumulate into the same entries do so from the same thread.
template <int P>
__device__ void contract(const Tables& T, const Side& si, const Side& sj, const double* __restrict__ Wg, double coef,
                         double* out, int ld, bool accumulate, bool upper, double* sm) {
  constexpr int Q = SfDims<P>::Q, NQ = SfDims<P>::NQ;
  const int a0 = si.n[0], a1 = si.n[1], a2 = si.n[2], b0 = sj.n[0], b1 = sj.n[1], b2 = sj.n[2];
  const int n0 = a0 * b0, n1 = a1 * b1, n2 = a2 * b2;
  double* W = sm;              // NQ
  double* AB0 = W + NQ;        // [q0][i0 j0]
  double* AB1 = AB0 + Q * n0;  // [i1 j1][q1]
  double* AB2 = AB1 + Q * n1;  // [i2 j2][q2]
  double* T1 = AB2 + Q * n2;   // [i2 j2][q1][q0]
  double* T2 = T1 + n2 * Q * Q;  // [i1 j1][i2 j2][q0]
  const int tid = threadIdx.x, nt = blockDim.x;
  __syncthreads();  // the previous contraction is done with the buffers
  for (int q = tid; q < NQ; q += nt) W[q] = coef * Wg[q];
  for (int t = tid; t < Q * n0; t += nt) {
    const int q = t / n0, ij = t - q * n0, i = ij / b0, j = ij - i * b0;
    AB0[t] = tab(T, si, 0, q, i) * tab(T, sj, 0, q, j);
  }
  for (int t = tid; t < n1 * Q; t += nt) {
    const int ij = t / Q, q = t - ij * Q, i = ij / b1, j = ij - i * b1;
    AB1[t] = tab(T, si, 1, q, i) * tab(T, sj, 1, q, j);
  }
  for (int t = tid; t < n2 * Q; t += nt) {
    const int ij = t / Q, q = t - ij * Q, i = ij / b2, j = ij - i * b2;
    AB2[t] = tab(T, si, 2, q, i) * tab(T, sj, 2, q, j);
  }
  __syncthreads();
  // direction 2: T1[ij2][q1][q0] = sum_q2 AB2[ij2][q2] W[q0, q1, q2]
  for (int t = tid; t < n2 * Q * Q; t += nt) {
    const int ij2 = t / (Q * Q), r = t - ij2 * Q * Q;
    double acc = 0.0;
#pragma unroll
    for (int q2 = 0; q2 < Q; ++q2) acc = fma(AB2[ij2 * Q + q2], W[r + Q * Q * q2], acc);
    T1[t] = acc;
  }
  __syncthreads();
  // direction 1: T2[ij1][ij2][q0] = sum_q1 AB1[ij1][q1] T1[ij2][q1][q0]
  for (int t = tid; t < n1 * n2 * Q; t += nt) {
    const int q0 = t % Q, r = t / Q, ij2 = r % n2, ij1 = r / n2;
    double acc = 0.0;
#pragma unroll
    for (int q1 = 0; q1 < Q; ++q1) acc = fma(AB1[ij1 * Q + q1], T1[(ij2 * Q + q1) * Q + q0], acc);
    T2[t] = acc;
  }
  __syncthreads();
  // direction 0: out[i][j] = sum_q0 AB0[q0][ij0] T2[ij1][ij2][q0]
  const int total = n0 * n1 * n2;
  for (int t = tid; t < total; t += nt) {
    const int ij0 = t % n0, r = t / n0, ij2 = r % n2, ij1 = r / n2;
    const int i0 = ij0 / b0, j0 = ij0 - i0 * b0;
    const int i1 = ij1 / b1, j1 = ij1 - i1 * b1;
    const int i2 = ij2 / b2, j2 = ij2 - i2 * b2;
    const int i = i0 + a0 * (i1 + a1 * i2), j = j0 + b0 * (j1 + b1 * j2);
    if (upper && i > j) continue;
    double acc = 0.0;
#pragma unroll
    for (int q0 = 0; q0 < Q; ++q0) acc = fma(AB0[q0 * n0 + ij0], T2[r * Q + q0], acc);
    double* o = out + (size_t)i * ld + j;
    *o = accumulate ? *o + acc : acc;
  }
}

__device__ __forceinline__ int pair_index(int a, int b) {
  if (a == b) return a;
  const int lo = min(a, b), hi = max(a, b);
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

// derivative direction and sign of curl component a of f e_c (a != c)
__device__ __forceinline__ void curl_term(int c, int a, int& k, double& sign) {
  k = 3 - a - c;
  sign = ((k - a + 3) % 3 == 1) ? 1.0 : -1.0;  // Levi-Civita eps_{a k c}
}

// Jobs per element (blockIdx.x): 0..5 M blocks (c <= d), 6..11 C blocks,
// 12..14 P rows of component c, 15..17 Q rows of component c.
constexpr int SF_JOBS = 18;

template <int P>
__global__ void __launch_bounds__(256) k_quad_sf(const __grid_constant__ Tables T, const double* __restrict__ WQ,
                                                 double* __restrict__ MC) {
  using D = SfDims<P>;
  extern __shared__ double sm[];
  const int job = blockIdx.x, slot = blockIdx.y;
  const double* Wel = WQ + (size_t)slot * NWQ * D::NQ;
  double* M = MC + (size_t)slot * (2 * (size_t)D::NF * D::NF + 2 * (size_t)D::NF * D::NL3);
  double* Cm = M + (size_t)D::NF * D::NF;
  double* Pm = Cm + (size_t)D::NF * D::NF;
  double* Qm = Pm + (size_t)D::NF * D::NL3;
  const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
  if (job < 6) {
    const int c = pa[job], d = pb[job];
    contract<P>(T, test_side(T, c, -1), test_side(T, d, -1), Wel + (size_t)job * D::NQ, 1.0,
                M + (size_t)c * D::NCOMP * D::NF + (size_t)d * D::NCOMP, D::NF, false, c == d, sm);
  } else if (job < 12) {
    const int c = pa[job - 6], d = pb[job - 6];
    double* out = Cm + (size_t)c * D::NCOMP * D::NF + (size_t)d * D::NCOMP;
    bool first = true;
    for (int a = 0; a < 3; ++a) {
      if (a == c) continue;
      int ka;
      double sa;
      curl_term(c, a, ka, sa);
      for (int b = 0; b < 3; ++b) {
        if (b == d) continue;
        int kb;
        double sb;
        curl_term(d, b, kb, sb);
        contract<P>(T, test_side(T, c, ka), test_side(T, d, kb), Wel + (size_t)(6 + pair_index(a, b)) * D::NQ,
                    sa * sb, out, D::NF, !first, c == d, sm);
        first = false;
      }
    }
  } else if (job < 15) {
    const int c = job - 12;
    for (int d = 0; d < 3; ++d)
      contract<P>(T, test_side(T, c, -1), trial_side(T), Wel + (size_t)(12 + 3 * c + d) * D::NQ, 1.0,
                  Pm + (size_t)c * D::NCOMP * D::NL3 + (size_t)d * D::NL, D::NL3, false, false, sm);
  } else {
    const int c = job - 15;
    for (int d = 0; d < 3; ++d) {
      bool first = true;
      for (int a = 0; a < 3; ++a) {
        if (a == c) continue;
        int ka;
        double sa;
        curl_term(c, a, ka, sa);
        contract<P>(T, test_side(T, c, ka), trial_side(T), Wel + (size_t)(21 + 3 * d + a) * D::NQ, sa,
                    Qm + (size_t)c * D::NCOMP * D::NL3 + (size_t)d * D::NL, D::NL3, !first, false, sm);
        first = false;
      }
    }
  }
}

template <int P>
static size_t sf_smem() {
  return sizeof(double) * (size_t)SfDims<P>::SMEM;
}

int quad_sf_init() {
  if (cudaFuncSetAttribute(k_quad_sf<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf_smem<1>()) ||
      cudaFuncSetAttribute(k_quad_sf<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf_smem<2>()) ||
      cudaFuncSetAttribute(k_quad_sf<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf_smem<3>()) ||
      cudaFuncSetAttribute(k_quad_sf<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf_smem<4>()))
    return DPG_ERR_CUDA;
  return DPG_OK;
}

size_t quad_sf_weight_bytes(const Sizes& S) { return sizeof(double) * NWQ * (size_t)S.nq; }

// Geometry weights, then the 18 contraction jobs of every element of the chunk.
int quad_sf_launch(const Tables& T, const Sizes& S, const double* X, const int* ids, int count, double* WQ,
                   double* MC, cudaStream_t s) {
  if (count <= 0) return DPG_OK;
  k_quad_geom<<<dim3((S.nq + 127) / 128, count), 128, 0, s>>>(T, S, X, ids, WQ);
  const dim3 grid(SF_JOBS, count);
  switch (S.p) {
    case 1: k_quad_sf<1><<<grid, 256, sf_smem<1>(), s>>>(T, WQ, MC); break;
    case 2: k_quad_sf<2><<<grid, 256, sf_smem<2>(), s>>>(T, WQ, MC); break;
    case 3: k_quad_sf<3><<<grid, 256, sf_smem<3>(), s>>>(T, WQ, MC); break;
    case 4: k_quad_sf<4><<<grid, 256, sf_smem<4>(), s>>>(T, WQ, MC); break;
    default: return DPG_ERR_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? DPG_OK : DPG_ERR_CUDA;
}

}  // namespace dpg
