// Internal declarations of the DPG library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dpg.h"

namespace dpg {

constexpr int MAXP = 4;          // largest trial degree
constexpr int MAXF1D = MAXP + 3; // largest 1D family size: closed rule of order rt = p + 2 has rt + 1
constexpr int MAXPT = MAXP + 5;  // quadrature points p + 3, plus the endpoints 0 and 1

// 1D function families tabulated on the extended point set
// [Gauss-Legendre points of the element rule (nq1), 0, 1].
enum Family { F_OPEN_T = 0, F_CLOSED_T = 1, F_OPEN_R = 2, F_CLOSED_R = 3, F_L2 = 4, NFAM = 5 };

struct Tables {
  int p, r, rt, nq1, npt;          // npt = nq1 + 2
  int nfun[NFAM];                  // functions per family
  double pt[MAXPT];                // the extended 1D points
  double w[MAXPT];                 // Gauss-Legendre weights (first nq1 entries)
  double val[NFAM][MAXPT][MAXF1D]; // l_j(pt)
  double der[NFAM][MAXPT][MAXF1D]; // l_j'(pt)
};

// Element sizes for degree p and dp = 1.
struct Sizes {
  int p, r, rt, nq1, nq, nqf;
  int n_f, n_v, nL, n_u, nt, n_h, N;  // N = augmented system size n_v + n_u + n_h + 1
};
Sizes make_sizes(int p);

// Host-side reference computations (tables.cpp).
void gauss_legendre01(int n, double* x, double* w);
void gauss_lobatto01(int n, double* x);
void lagrange1d(const double* nodes, int n, double x, double* val, double* der);
void build_tables(int p, Tables* t);
// Packed Nedelec function id: c | i0 << 2 | i1 << 6 | i2 << 10.
inline int pack_fun(int c, int i0, int i1, int i2) { return c | (i0 << 2) | (i1 << 6) | (i2 << 10); }
// Trace functions of order r in element-local order (12 r^2 entries).
std::vector<int> trace_functions(int r);

struct RobinEntry {  // one Robin face of one element
  int elem, face, grp;
};

// Per-chunk device workspace of the element pipeline.
struct Workspace {
  int cap = 0;               // elements per chunk
  double2* K = nullptr;      // cap x N x N augmented Hermitian system (column-major, lower used)
  // V, Cu, PhiL: cap elements for the tensor-core quadrature, one element
  // with FP64 quadrature (V also serves as the real-path extraction scratch)
  double* V = nullptr;       // cap x 3nq x n_f   sqrt(w detJ) psi
  double* Cu = nullptr;      // cap x 3nq x n_f   sqrt(w detJ) curl psi
  double* PhiL = nullptr;    // cap x 3nq x 3nL   sqrt(w detJ) L e_d
  double* MC = nullptr;      // cap x (2 n_f^2 + 2 n_f 3nL): M, C, P, Q
  double* WQ = nullptr;      // cap x 30 x nq     geometric weights of the sum-factorised quadrature
  int* ids = nullptr;        // cap element ids of the chunk
  // Robin face scratch (per Robin entry of the chunk)
  int rcap = 0;
  double* FV = nullptr;      // rcap x 3nqf x (2 n_f + nt + 2)
  double* FR = nullptr;      // rcap x (2 n_f^2 + n_f nt + 2 n_f)
  int* rent = nullptr;       // rcap x 4 (elem slot, face, grp, elem id)
  uint8_t* Q = nullptr;      // cap x digit scratch of the tensor-core factorisation (factor_tc.cu)
};

// Per-element offsets into the pooled element stores (in entries of each
// array).  Elements of different trial degrees have different store sizes.
struct ElemOff {
  int64_t S;   // d_S: n_h x n_h
  int64_t Z;   // d_Z: n_u x n_h
  int64_t L1;  // d_L1: n_u x n_u
  int64_t h;   // d_s, trace map, fixed values: n_h
  int64_t u;   // d_z, interior solution u: n_u
};

// Trace restriction R_K of one signature (element degree and the orders of its
// 18 entities), one field: element trace function j (rows) from the element's
// trace-map slots t (columns).  Column- and row-compressed; offsets into the
// handle's integer and double pools.
struct RSig {
  int nt;              // trace functions per field at the element's degree
  int64_t cptr, cidx;  // column pointers (nt + 1, relative to cidx) and row indices
  int64_t rptr, ridx;  // row pointers (nt + 1, relative to ridx) and column indices
  int64_t cw, rw;      // weights of the two forms (double pool)
};

// One launch group of the element pass: elements of one degree and one
// arithmetic class (real / complex), at most the group's chunk size.  The
// element ids and the Robin face sub-batches live in device buffers built once,
// so the whole pass is a fixed sequence of launches (captured as a CUDA graph).
struct ChunkPlan {
  int g = 0;
  bool real = false;
  bool restricted = false;     // some element needs the trace restriction
  int64_t ids_off = 0;         // into d_plan_ids
  int64_t koff = 0;            // byte offset of the chunk's matrices in the workspace K (order-bucketed waves)
  int count = 0;
  std::vector<int4> robin;     // sub-batches: (entries offset, entries, element list offset, elements) in the rent list
  const int* d_ids = nullptr;  // the plan's device element-id list (ids of this chunk at d_ids + ids_off)
  const int* d_rent = nullptr; // the plan's device Robin entry list
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the factorisation (timing)
};

// One item of the persistent factorisation's work list (factor_tc.cu): an
// element's augmented matrix at byte offset koff of the K arena.
struct FtItem {
  int64_t koff;
  int elem, cplx, N, nact, nv, npiv, pad;
};

// One wave of the order-bucketed element pass: chunks c0 .. c0 + nc - 1 of the
// plan (at most one chunk of every order and arithmetic list) are formed into
// their slices of the K arena, then factored by persistent launches over the
// wave's work list (items item_off .. item_off + nitems - 1: the complex items
// of every order longest first, then the real ones; one launch per
// arithmetic), then extracted chunk by chunk.
struct WavePlan {
  int c0 = 0, nc = 0;
  int64_t item_off = 0;
  int nitems = 0, nitems_real = 0, nmax = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// Elements of one trial degree: sizes, tables, reference matrices.
struct Group {
  int p = 0;
  Sizes sz{};
  Tables tab{};
  std::vector<int> elems;                 // global element ids
  std::vector<int> real_elems, cplx_elems;
  std::vector<int> color_off;             // elems sorted by colour: offsets per colour
  std::vector<int> color_elems_host;      // the sorted list
  int* d_color_elems = nullptr;           // the sorted list on the device
  int* d_elems = nullptr;                 // elems on the device
  double* d_Xref = nullptr;               // n_f x n_f  int curl psi_i . psi_j (metric free)
  double* d_Tf = nullptr;                 // 6 x n_f x nt  int_f psi_i . (N x phi_t) (metric free)
  double* d_Tall = nullptr;               // n_f x nt
  int* d_trfun = nullptr;                 // nt packed trace functions
  int cap = 0;                            // elements per chunk
};

}  // namespace dpg

struct dpg_handle {
  std::string err;
  std::vector<dpg::Group> grp;    // one per trial degree present, ascending p
  std::vector<int8_t> elem_grp;   // group of each element
  dpg::Sizes szmax{};             // largest sizes over the groups
  int ne = 0;
  int prec = DPG_PREC_FP64;       // quadrature contraction precision
  int factor_arith = DPG_FACTOR_TC_SPLIT;  // arithmetic of the element factorisation's trailing updates
  double omega = 0, alpha = 1;
  // host copies used by setup / dumps
  std::vector<dpg_robin_group> robin;
  std::vector<dpg_dirichlet_group> dirichlet;
  std::vector<dpg::RobinEntry> robin_entries;  // sorted by element
  std::vector<int> robin_first;                // per element: first entry index or -1
  int ncolor = 0;
  int64_t n_slaves = 0;                        // hanging (2:1) edges and faces without unknowns
  int64_t n = 0, nnz = 0;
  std::vector<int32_t> l2g;                    // element-major, n_h(K) per element (offsets ElemOff::h)
  std::vector<dpg::ElemOff> off;               // ne + 1 (the last holds the totals)
  dpg::ElemOff* d_off = nullptr;
  // Streaming (DPG_FLAG_STREAM): the element stores S, s, Z, z hold one chunk
  // only, at slot-based offsets d_soff[e] (the element's slot in its chunk of
  // the launch plan); the chunks are colour-homogeneous and assembled as they
  // are condensed.  Without streaming d_soff == d_off.
  bool stream = false;
  std::vector<int> elem_color;
  dpg::ElemOff* d_soff = nullptr;
  std::vector<dpg::ElemOff> soff_host;
  // trace restrictions of elements with a lower-order entity (-1: identity)
  std::vector<int> elem_sig;
  std::vector<dpg::RSig> rsig;
  int* d_sig = nullptr;
  dpg::RSig* d_rsig = nullptr;
  int32_t* d_rint = nullptr;
  double* d_rdbl = nullptr;
  // device buffers
  double* d_X = nullptr;        // ne x 24 corner coordinates
  double2* d_eps = nullptr;     // ne
  double2* d_mu = nullptr;      // ne
  int8_t* d_fbc = nullptr;      // ne x 6
  int32_t* d_l2g = nullptr;     // trace map (offsets ElemOff::h)
  double2* d_xfix = nullptr;    // fixed trace values (offsets ElemOff::h)
  dpg_robin_group* d_robin = nullptr;
  int* d_status = nullptr;      // ne
  // per-element stores, pooled over the elements at the offsets in off
  double2* d_S = nullptr;       // n_h x n_h   (R_K^H S_K R_K for restricted elements)
  double2* d_s = nullptr;       // n_h
  double* d_c = nullptr;        // ne
  double2* d_Z = nullptr;       // n_u x n_h   (M1^{-1} M2, times R_K)
  double2* d_z = nullptr;       // n_u         (M1^{-1} M4 l)
  double2* d_L1 = nullptr;      // n_u x n_u   Cholesky factor of M1 (only with DPG_FLAG_ADJOINT)
  // adjoint scratch (allocated on the first dpg_grad_eps)
  double2 *d_u = nullptr, *d_zg = nullptr, *d_gc = nullptr, *d_lam = nullptr, *d_rhs_adj = nullptr;
  double* d_Pk = nullptr;
  // CSR system; the rows of one entity share a column list:
  // blk[b] = (first row, rows, row width W, position of the block's own
  // unknowns in its column list), columns at cols[blk_colptr[b] ...]
  std::vector<int4> blk;
  std::vector<int64_t> blk_colptr;
  std::vector<int32_t> cols;
  int nblk = 0;
  int blk_dmax = 0;  // rows of the largest entity block
  int64_t* d_rowptr = nullptr;
  int32_t* d_row2blk = nullptr;
  int4* d_blk = nullptr;
  int64_t* d_blk_colptr = nullptr;
  int32_t* d_cols = nullptr;
  // entity-block Jacobi: inverse of each block's diagonal sub-block (rows x rows)
  int64_t* d_binv_ptr = nullptr;
  double2* d_binv = nullptr;
  float2* d_binv32 = nullptr;
  bool have_binv = false;
  int binv_dmax = 0;
  double2* d_val = nullptr;
  double2* d_b = nullptr;
  float2* d_val32 = nullptr;    // FP32 copy for IR inner solves (lazily built)
  // Hermitian half storage of the FP32 inner matrix (lazily built): per row
  // the prefix of its entity's column list up to and including the entity's
  // own unknowns (blocks of lower entities and the diagonal block); the upper
  // blocks are applied as conjugate transposes through per-block partial
  // sums T (block a's strictly lower part, n_low(a) values) that the rows of
  // the upper neighbours' blocks gather in a fixed order (rev lists).
  bool have_half = false, have_val32h = false;
  int64_t nnz_h = 0, t_len = 0, rev_len = 0;
  int half_wmax = 0;                // widest half row
  int64_t* d_rowptr_h = nullptr;    // n + 1
  int64_t* d_toff = nullptr;        // nblk + 1: offset of block a's partial sums in T
  int64_t* d_rev_ptr = nullptr;     // nblk + 1
  int64_t* d_rev_off = nullptr;     // rev_len: T offsets of the segments that belong to block b's rows
  float2* d_val32h = nullptr;       // nnz_h
  float2* d_T = nullptr;            // t_len
  // double-word (FP32 pair) copies for the DW solver mode
  float4* d_valdw = nullptr;        // nnz
  float4* d_pdw = nullptr;          // n
  float4* d_binvdw = nullptr;       // block inverses
  bool have_valdw = false, have_binvdw = false;
  // element-by-element FP32 operator of the inner solves (DPG_CG_EBE)
  float2* d_ebe = nullptr;          // per element: upper-triangle 32 x 32 tiles of S_K
  int64_t* d_ebe_toff = nullptr;    // per element: first tile entry (ne + 1)
  int64_t* d_ebe_hoff = nullptr;    // per element: first slot (ne + 1)
  int64_t* d_ebe_rptr = nullptr;    // per row: first entry of its slot list (n + 1)
  int32_t* d_ebe_ridx = nullptr;    // slot lists
  float2* d_ebe_ys = nullptr;       // per slot: the element product
  bool have_ebe_idx = false, have_ebe = false;
  int ebe_nbmax = 1;
  // stored-factor estimator (dpg_set_estimator_store): per element
  // X = (L^{-1} [B | B-hat | l])^H, n_v columns of m + 1 entries (doubles on the
  // real path, complex pairs otherwise), written by every element pass
  double* d_Xst = nullptr;
  int64_t* d_xst_off = nullptr;  // per element: offset in doubles
  bool xst_valid = false;        // X describes the current elements
  int ebe_stages = 2;
  int64_t ebe_tiles = 0, ebe_slots = 0, ebe_links = 0;
  bool have_elements = false, have_system = false, have_val32 = false, have_dinv = false;
  double* d_dinv = nullptr;     // inverse diagonal (Jacobi)
  float* d_dinv32 = nullptr;
  // instrumentation
  bool timing = false;
  // launch plan of the element pass and its CUDA graph
  std::vector<dpg::ChunkPlan> plan;
  bool plan_valid = false;
  int* d_plan_ids = nullptr;
  int* d_plan_rent = nullptr;
  int* d_est_neg = nullptr;       // count of clamped negative eta_K^2 (one int)
  // order-bucketed element pass: waves of chunks of every order, one
  // persistent factorisation launch per wave
  bool bucketed = false;
  int nwaves = 1;
  int chunk_req = 0;  // the caller's chunk size at setup (0: by the byte budget)
  std::vector<dpg::WavePlan> waves;
  dpg::FtItem* d_items = nullptr;
  int* d_wave_ctr = nullptr;
  // factorisation stamps of the last pass: (SM, start ns, end ns) per element
  // of the plan (per item in bucketed mode), in plan order
  unsigned long long* d_stamps = nullptr;
  int64_t n_stamps = 0;
  bool use_graph = true;
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false, graph_timing = false;
  int64_t graph_launches = 0;
  cudaStream_t cap_stream = nullptr;
  int64_t factor_elements_real = 0;
  double factor_ms_real = 0;
  // lossless elements (real eps and mu, no Robin face) take the real path
  std::vector<char> is_real;
  bool allow_real = true;
  std::vector<dpg_complex> eps_host, mu_host;
  std::vector<char> robin_face;
  double factor_ms = 0, cg_ms = 0;
  int64_t factor_launches = 0, factor_elements = 0, cg_iters = 0, launches = 0;
  double cgk_ms = 0;              // persistent CG kernel launches
  int64_t cgk_launches = 0, cgk_iters = 0;
  bool cgk_fp32 = false;
  // CG scratch
  double2 *d_r = nullptr, *d_p = nullptr, *d_Ap = nullptr, *d_zv = nullptr, *d_d64 = nullptr;
  float2 *d_r32 = nullptr, *d_p32 = nullptr, *d_Ap32 = nullptr, *d_x32 = nullptr, *d_z32 = nullptr;
  void* d_cgstate = nullptr;      // CG state of the persistent solver (solve.cu)
  int64_t wait_ns = 5000000000ll; // bound of every grid-barrier wait of the CG kernel
  bool wait_hold = false;         // test hook: CG barriers never release
  double* d_red = nullptr;      // reduction scratch
  dpg::Workspace ws;
};

namespace dpg {
// setup.cpp
int build_mesh(dpg_handle* h, const dpg_mesh_desc* m, const dpg_params* prm, cudaStream_t s);
void classify_elements(dpg_handle* h);
// element.cu
void set_default_caps(dpg_handle* h, int chunk);
int alloc_workspace(dpg_handle* h);
int init_kernel_attributes(dpg_handle* h);
// One chunk of the element pass: quadrature (quad), K formed (build), the
// factorisation (factor), the extraction into the stores (extract).  Kc: the
// chunk's matrices (default: the start of the K workspace).
int run_element_chunk(dpg_handle* h, int g, const int* ids_host, int count, cudaStream_t s, bool factor,
                      bool extract, bool real = false, const ChunkPlan* cp = nullptr, bool quad = true,
                      bool build = true, void* Kc = nullptr);
int build_plan(dpg_handle* h);
void free_plan(dpg_handle* h);
int element_pass(dpg_handle* h, cudaStream_t s);
int autotune(dpg_handle* h, double max_bytes, int32_t* caps, float* ms_per_elem, cudaStream_t s);
int compute_reference_matrices(dpg_handle* h, int g, cudaStream_t s);
int factor_gram_only(dpg_handle* h, int g, int count, cudaStream_t s);
int estimate_pass(dpg_handle* h, const double2* xhat, double2* u, double* eta2, cudaStream_t s);
int recover_u(dpg_handle* h, const double2* xhat, double2* u, cudaStream_t s);
// power.cu
int power(dpg_handle* h, const double2* xhat, double* q, double* flux_host, cudaStream_t s);
// factor_tc.cu
int factor_tc_init();
// Sum-factorised FP64 quadrature of M, C, P, Q (quad_sf.cu).
int quad_sf_init();
size_t quad_sf_weight_bytes(const Sizes& S);
int quad_sf_launch(const Tables& T, const Sizes& S, const double* X, const int* ids, int count, double* WQ,
                   double* MC, cudaStream_t s);
size_t factor_tc_scratch_bytes(int N, bool cplx);
int factor_tc_launch(bool cplx, int count, int N, int nact, int nv, int npiv, const int* ids, void* K, int* status,
                     int* tc_err, uint8_t* qscr, cudaStream_t s, unsigned long long* stamps = nullptr);
size_t factor_tc_queue_scratch_bytes(int Nmax);
int factor_tc_queue_launch(bool cplx, const FtItem* items, int nitems, int Nmax, int* counter, void* arena,
                           int* status, int* tc_err, uint8_t* qscr, unsigned long long* stamps, int grid,
                           cudaStream_t s);
// quad_tc.cu
int tc_init();
int gemm_tn_tc(int split, int Ma, int Nb, int Kd, const double* A, int lda, long long sA, const double* B, int ldb,
               long long sB, double* C, int ldc, long long sC, int batch, int upper_only, int* err, cudaStream_t s);
// adjoint.cu
int grad_eps(dpg_handle* h, const double2* xhat, const uint8_t* mask, double* P_host, double* dre, double* dim,
             int cg_mode, double cg_rtol, int max_iter, cudaStream_t s);
// solve.cu
int assemble_system(dpg_handle* h, cudaStream_t s);
int assemble_chunk(dpg_handle* h, int g, const int* ids, int count, cudaStream_t s);
void system_changed(dpg_handle* h);
int cg_solve(dpg_handle* h, int mode, double rtol, double atol, int max_iter, double inner_rtol,
             double2* x, const double2* b, dpg_cg_report* rep, cudaStream_t s);
int estimate(dpg_handle* h, const double2* xhat, double2* u, double* eta, double* eta_global,
             cudaStream_t s);
int64_t cg_bytes_per_iteration(const dpg_handle* h, int mode);
int estimate_negatives(dpg_handle* h, int* count);
int estimate_noalloc(dpg_handle* h, const double2* xhat, double2* u, double* eta, double* eta_global,
                     cudaStream_t s);
}  // namespace dpg

#define DPG_CUDA_TRY(h, call)                                                     \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);              \
      return DPG_ERR_CUDA;                                                        \
    }                                                                             \
  } while (0)
