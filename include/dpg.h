/*
 * dpg.h -- C ABI of the B300 (sm_103a) DPG time-harmonic Maxwell hot path.
 *
 * The method is the discontinuous Petrov-Galerkin (DPG) discretisation of the
 * dimensionless time-harmonic Maxwell equations in ultraweak form of
 * arXiv 2609.03155 (Marquis, Maier, Blais):
 *   Sec. 2.2, Eq. (maxwell_dimensionless): curl E - i w mu H = 0,
 *             curl H + i w eps E = J (here J = 0), time factor e^{-i w t};
 *   Sec. 2.2, Eqs. (bilinear_form), (trace_pairing), (linear_form) and the
 *             adjoint graph test norm Eq. (test_inner_product) with alpha;
 *   Sec. 2.3: element block system, the two static condensations,
 *             Eq. (linear_system), local recovery and the estimator ||Psi||_V;
 *   Algorithm 1 (solve) and Algorithm 2 (assembly).
 *
 * Discrete spaces (reading of Sec. 2.3 and Fig. 1, pinned by the DoF counts of
 * Sec. 4.1): per component of E and H a discontinuous tensor Lagrange space of
 * degree p on Gauss-Legendre nodes; traces E-hat, H-hat = tangential traces of
 * the Nedelec space of FEEC order r = p + 1; test functions F, I in the broken
 * Nedelec space of order p + 1 + dp.  Nedelec basis of order r, component c:
 * l^open_{i_c}(xi_c) prod_{d != c} l^closed_{i_d}(xi_d) e_c, open = Lagrange on
 * the r Gauss-Legendre points, closed = Lagrange on the r + 1 Gauss-Lobatto
 * points, mapped by the covariant Piola transform.  Quadrature: Gauss-Legendre,
 * p + dp + 2 points per direction in volume and on faces.
 *
 * Element-local ordering (used by every per-element input and output):
 *   test  [F (n_f), I (n_f)], n_f = 3 rt (rt+1)^2, rt = p + 1 + dp;
 *   interior trial u = [E_x, E_y, E_z, H_x, H_y, H_z], each (p+1)^3 tensor
 *         Lagrange coefficients, x-index fastest;            n_u = 6 (p+1)^3;
 *   trace u-hat = [E-hat (12 r^2), H-hat (12 r^2)]: the Nedelec functions of
 *         order r (component-major, x-index fastest) whose tangential trace is
 *         non-zero on some face, in that order;                n_h = 24 r^2.
 *
 * Mixed trial degrees (the paper refines in h only, Sec. 4.2): each element
 * computes at its own p; a mesh edge or face carries trace unknowns of order
 * r_E = min over the elements containing it of (p + 1), so the trace lies in
 * every neighbour's trace space.  Element K's trace coefficients are the
 * global trace's nodal values at K's own nodes, uhat_K = R_K uhat (R_K: 1D
 * Lagrange polynomials of the entity order at K's nodes).  Per-element arrays
 * are then of varying length; dpg_element_layout gives their offsets.  The
 * trace map and the stored S_K, s_K refer to the element's trace slots: the
 * global unknowns of an entity sit in the element's slots of the same entity
 * and index, the other slots are unused (-2), and S_K, s_K are R_K^H S_K R_K,
 * R_K^H s_K in those slots.
 *
 * Mesh conventions: hexahedra with trilinear geometry; element vertex
 * v = i + 2 j + 4 k sits at reference corner (i, j, k); every element's local
 * axes must agree with its neighbours' on shared edges and faces (the setup
 * rejects meshes where they do not, DPG_ERR_MESH).  Face f = 2 d + s is the
 * face xi_d = s.
 *
 * Memory and errors: every pointer argument documented "host" is read during
 * the call only; "device" pointers are caller-owned device memory, used on
 * the given stream in stream order.  The handle owns every internal buffer.
 * Functions return 0 (DPG_OK) or a negative DPG_ERR_* code and never abort,
 * trap or print; dpg_last_error() describes the last failure on a handle.
 * Work is enqueued on the caller's stream; a call synchronises that stream
 * only when it returns a host value that depends on device work (stated per
 * function).  Complex numbers are two doubles (re, im), layout-compatible
 * with C99 double _Complex and CUDA double2.
 */
#ifndef DPG_H
#define DPG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dpg_handle dpg_handle;
typedef void* dpg_stream; /* a cudaStream_t; NULL = legacy default stream */
typedef struct { double re, im; } dpg_complex;

enum {
  DPG_OK = 0,
  DPG_ERR_ARG = -1,            /* invalid argument (null pointer, size, range) */
  DPG_ERR_MESH = -2,           /* invalid mesh: ids, orientation, Jacobian, tags */
  DPG_ERR_NOMEM = -3,          /* device or host allocation failed */
  DPG_ERR_NOT_HPD = -4,        /* a Cholesky pivot was not positive (status per element) */
  DPG_ERR_NOT_CONVERGED = -5,  /* CG hit its iteration limit */
  DPG_ERR_TIMEOUT = -6,        /* a bounded device wait gave up */
  DPG_ERR_CUDA = -7,           /* a CUDA runtime call failed */
  DPG_ERR_STATE = -8,          /* call out of order (e.g. solve before assemble) */
  DPG_ERR_UNSUPPORTED = -9     /* valid request this build does not implement */
};

enum { DPG_BC_NONE = 0, DPG_BC_DIRICHLET = 1, DPG_BC_ROBIN = 2 };
enum { DPG_DIRICHLET_ZERO = 0, DPG_DIRICHLET_SIN_PI_X2 = 1, DPG_DIRICHLET_TE = 2 };
/* Precision of the quadrature contractions M, C, P, Q (everything after them,
 * G_K, B_K, the Cholesky factorisation, condensation and CG residuals, is
 * FP64 in every mode).  FP64: FP64 FMA.  TF32: tcgen05 tensor cores, operands
 * rounded to TF32, FP32 accumulation.  3XTF32: the same with each operand
 * split as a = a_hi + a_lo (both TF32) and a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,
 * about FP32 accuracy.  Reduced modes perturb G_K and B_K themselves; their
 * error against FP64 is a reported quantity, not a parity bound. */
enum { DPG_PREC_FP64 = 0, DPG_PREC_TF32 = 1, DPG_PREC_3XTF32 = 2 };
enum { DPG_PASS_ASSEMBLE = 0 };
enum { DPG_CG_FP64 = 0, DPG_CG_IR_FP32 = 1, DPG_CG_JACOBI = 2, DPG_CG_BLOCK_JACOBI = 4, DPG_CG_X0 = 8, DPG_CG_HALF = 16,
       DPG_CG_IR_V64 = 32, DPG_CG_DW = 64, DPG_CG_EBE = 128, DPG_CG_RELIABLE = 256, DPG_CG_EBE_BULK = 512 };
enum { DPG_FLAG_ADJOINT = 1, DPG_FLAG_STREAM = 2 };
/* Arithmetic of the element factorisation's trailing updates (dpg_set_factor_arith). */
enum { DPG_FACTOR_FP64 = 0, DPG_FACTOR_TC_SPLIT = 1 };

/* Robin group (Sec. 2.2, Eq. robin_boundary; Sec. 4.1 port / outlet):
 * n x H + Z^{-1} n x (E x n) = g.  port = 0: g = 0; port = 1: g is the TE_mn
 * datum n x H_TE + Z^{-1} n x (E_TE x n) of the mode of Sec. 4.1 in the guide
 * [0,a] x [0,b] (x3 = propagation axis) filled with (eps, mu). */
typedef struct {
  double zinv_re, zinv_im;
  int32_t port;
  int32_t m, n;
  double a, b;
  double eps_re, eps_im, mu_re, mu_im;
} dpg_robin_group;

/* Dirichlet group (Sec. 2.2, Eq. dirichlet_boundary): n x E = n x E_D on the
 * trace E-hat, imposed by nodal interpolation of the tangential datum.
 * kind ZERO: PEC; SIN_PI_X2: n x E = (sin(pi x2), 0, 0) (Sec. 4.2 excitation);
 * TE: E_D = E of the TE_mn mode described as in dpg_robin_group.  On an edge
 * shared by a ZERO face and a data face the data face wins. */
typedef struct {
  int32_t kind;
  int32_t m, n;
  double a, b;
  double eps_re, eps_im, mu_re, mu_im;
} dpg_dirichlet_group;

/* Mesh (host arrays, read during dpg_setup_mesh only). */
typedef struct {
  int32_t n_vert;
  const double* vert;          /* n_vert x 3 */
  int32_t n_elem;
  const int32_t* elem;         /* n_elem x 8 vertex ids */
  const int8_t* elem_p;        /* n_elem trial degree, 1..4 (may differ between elements) */
  const dpg_complex* elem_eps; /* n_elem relative permittivity, loss => Im > 0 */
  const dpg_complex* elem_mu;  /* n_elem relative permeability */
  const int8_t* face_bc;       /* n_elem x 6, DPG_BC_*; boundary faces only */
  const int16_t* face_grp;     /* n_elem x 6, index into robin[] / dirichlet[] */
  int32_t n_robin;
  const dpg_robin_group* robin;
  int32_t n_dirichlet;
  const dpg_dirichlet_group* dirichlet;
} dpg_mesh_desc;

typedef struct {
  double omega;      /* dimensionless angular frequency (App. A, L = 1 m) */
  double alpha;      /* test-norm weight alpha of Eq. (test_inner_product), > 0 */
  int32_t dp;        /* enrichment, must be 1 in this build */
  int32_t precision; /* DPG_PREC_* */
  int32_t chunk;     /* elements per batched launch, 0 = automatic */
  int32_t flags;     /* DPG_FLAG_*: DPG_FLAG_ADJOINT keeps the M1 factors dpg_grad_eps needs;
                        DPG_FLAG_STREAM keeps no per-element condensation data: the element
                        pass assembles each chunk (one colour) as soon as it is condensed
                        and dpg_assemble has nothing left to do; recovery and the estimator
                        condense every chunk again.  Memory then scales with the CSR system
                        instead of n_elem (n_h^2 + n_u n_h) complex values, which lets
                        meshes of 1e5 elements and more fit.  Not with DPG_FLAG_ADJOINT,
                        dpg_autotune or dpg_grad_eps (DPG_ERR_UNSUPPORTED). */
} dpg_params;

typedef struct {
  int32_t iterations;      /* total CG iterations (inner ones for IR) */
  int32_t outer;           /* outer passes: IR corrections, or FP64 residual replacements (1 = none needed) */
  double rel_residual;     /* final ||b - A x|| / ||b||, FP64 */
  double ms;               /* device time of the solve */
  int32_t converged;
  int32_t reserved;
} dpg_cg_report;

/* Build the DPG discretisation of the mesh on the current CUDA device:
 * trace numbering (entity based), Dirichlet values, removal of the H-hat
 * unknowns that pair with nothing (Robin faces, end of Sec. 2.3), CSR pattern
 * of the condensed trace system, reference tables, and every device buffer.
 * Errors: DPG_ERR_ARG (null / out of range), DPG_ERR_MESH (bad ids,
 * inconsistent orientation, non-positive Jacobian at a corner, p outside
 * 1..4), DPG_ERR_UNSUPPORTED (dp != 1), DPG_ERR_NOMEM, DPG_ERR_CUDA.
 * On error *h is NULL.
 * Synchronises the stream before returning. */
int dpg_setup_mesh(dpg_handle** h, const dpg_mesh_desc* mesh, const dpg_params* prm, dpg_stream s);

/* Element pass (Algorithm 2 minus the distribution): for every element form
 * G_K, B_K, B-hat_K, l_K by quadrature (Sec. 2.3), factor G_K = L L^H, condense
 * to S_K = M3 - M2^H M1^{-1} M2 and s_K (Eq. linear_system), and keep S_K, s_K,
 * M1^{-1} M2, M1^{-1} M4 l and the scalar l^H G^{-1} l - (M4 l)^H M1^{-1} M4 l
 * in handle-owned per-element storage.  pass must be DPG_PASS_ASSEMBLE.
 * Lossless elements take the real path (see dpg_set_real_path).
 * A non-positive pivot marks the element (DPG_ERR_NOT_HPD is returned by the
 * next call that synchronises). Asynchronous. */
int dpg_element_batch(dpg_handle* h, int32_t pass, dpg_stream s);

/* DistributeLocalToGlobal of Algorithm 2: sum the stored S_K, s_K into the
 * handle-owned CSR matrix and right-hand side of Eq. (linear_system), with
 * Dirichlet lifting b -= S_{free,fixed} x_D.  Deterministic (elements are
 * summed in a fixed colour order, no atomics).  Asynchronous.
 * Errors: DPG_ERR_STATE if no element pass has run. */
int dpg_assemble(dpg_handle* h, dpg_stream s);

/* Unpreconditioned conjugate gradients on the Hermitian positive definite
 * system (Sec. 2.3 end): x0 = 0, stop when ||r|| <= max(rtol ||b||, atol).
 * mode DPG_CG_FP64: plain FP64 CG (the paper's solver).  DPG_CG_IR_FP32:
 * iterative refinement, FP64 residuals and updates around FP32 inner CG
 * solves on an FP32 copy of the matrix (inner relative tolerance inner_rtol;
 * about 5e-2 takes the fewest total inner iterations on the 3D waveguide:
 * restarts are cheap, and a loose inner solve wastes less of its Krylov space).
 * DPG_CG_JACOBI or DPG_CG_BLOCK_JACOBI may be or-ed to either: diagonal
 * preconditioning z = D^{-1} r, or the inverses of the entity diagonal blocks
 * (each mesh entity's E-hat and H-hat unknowns together).  The paper leaves
 * preconditioning to future work; the stopping test stays on the
 * unpreconditioned residual.  Each (inner) solve is one cooperative kernel
 * whose grid barriers give up after a bounded wait (DPG_ERR_TIMEOUT).
 * DPG_CG_HALF may be or-ed to DPG_CG_IR_FP32: the inner solves read a
 * Hermitian half storage of the FP32 matrix (each pair of entity blocks once;
 * the upper blocks are applied as conjugate transposes through per-block
 * partial sums gathered in a fixed order, so results stay deterministic).
 * DPG_CG_IR_V64 may be or-ed to DPG_CG_IR_FP32 (not with DPG_CG_HALF): the
 * inner solves keep their vectors, recurrences and reductions in FP64 and
 * only the matrix (values and products) in FP32, so an inner solve converges
 * like FP64 CG on the FP32-rounded matrix and can go to a smaller inner_rtol.
 * DPG_CG_DW (alone or with DPG_CG_BLOCK_JACOBI): CG with FP64 vectors,
 * recurrences and reductions whose matrix, direction vector and block
 * inverses are double-word FP32 pairs (hi + lo, about 48 bits), every SpMV and
 * preconditioner product and sum formed with error-free transformations
 * (Dekker's two-product by FMA, Knuth's two-sum) on the FP32 pipes: FP64-class
 * accuracy (the convergence of FP64 CG) at the speed of the memory system
 * instead of the FP64 pipe.  The stopping test is on the FP64 residual.
 * DPG_CG_EBE may be or-ed to DPG_CG_IR_FP32 (not with DPG_CG_HALF or
 * DPG_CG_IR_V64; not in streaming mode): the inner solves apply the matrix
 * element by element, A p = sum_K R_K^T S_K R_K p, from an FP32 copy of every
 * element's condensed S_K kept as the upper triangle of 32 x 32 tiles (each
 * Hermitian element matrix read once per product, the lower triangle applied
 * as the conjugate transpose); each element's product goes to its trace
 * slots and each row then sums its slots in ascending order (deterministic).
 * The assembled matrix stays for the FP64 residuals and the preconditioner.
 * DPG_CG_EBE_BULK may be or-ed to DPG_CG_EBE: the tiles are staged through
 * shared memory by the bulk-copy (TMA) engine, a ring of 8 KB buffers per warp
 * with one mbarrier each, refilled ahead across element boundaries; the same
 * products.  Its staging allows one block per SM (the default loads the tiles
 * into registers, two blocks per SM).
 * Errors add DPG_ERR_UNSUPPORTED (streaming, or over 2^31 trace slots).
 * DPG_CG_RELIABLE may be or-ed to DPG_CG_IR_FP32 (with any inner operator):
 * reliable updates instead of restarts.  After each inner solve the residual
 * is replaced by the true FP64 residual b - A x as before, but the next inner
 * solve continues the previous search direction, p = z + beta p with
 * beta = r^H z / (r^H z)_previous, instead of starting again from p = z, so
 * the Krylov information of the earlier inner solves is kept.
 * DPG_CG_X0 may be or-ed too: start from the x passed in (resume a stopped
 * solve, or warm-start from a nearby problem's solution) instead of x0 = 0.
 * x: device, n complex (caller-owned, overwritten).  b: device, n complex, or
 * NULL for the assembled right-hand side.  rep: host, may be NULL.
 * Synchronises the stream (the report is a host value).
 * Errors: DPG_ERR_NOT_CONVERGED (x holds the last iterate), DPG_ERR_STATE. */
int dpg_cg_solve(dpg_handle* h, int32_t mode, double rtol, double atol, int32_t max_iter,
                 double inner_rtol, dpg_complex* x, const dpg_complex* b,
                 dpg_cg_report* rep, dpg_stream s);

/* Local recovery and residual estimator (Sec. 2.3): for the trace solution
 * xhat (device, n complex) compute per element u_K = M1^{-1}(M4 l - M2 uhat_K)
 * (u: device, element e's n_u(e) complex values at the offset u_off[e] of
 * dpg_element_layout, n_elem x n_u for one degree; element-local order above;
 * may be NULL; from the stored condensation data)
 * and eta_K = ||Psi_K||_V with Psi_K = G^{-1}(l - B u - B-hat uhat)
 * (eta: device, n_elem doubles, may be NULL), by its definition: a second
 * element pass forms G_K, B_K, B-hat_K, l_K again, forms r_K = l - B u - B-hat uhat
 * and factors G_K = L L^H with r_K as one more column, so that
 * eta_K^2 = ||L^{-1} r_K||^2 is accumulated as a sum of squares (rounding can
 * only make it negative when eta_K ~ 0; such values are set to 0 and counted,
 * see dpg_estimate_clamped).  With eta and eta_global both NULL only u is
 * computed (no element pass).  Uses the handle's chunk workspace.
 * eta_global: host, sqrt(sum eta_K^2) (may be NULL; synchronises if given).
 * Errors: DPG_ERR_STATE (no element pass), DPG_ERR_ARG, DPG_ERR_NOMEM,
 * DPG_ERR_TIMEOUT (a tensor-core wait of the pass gave up; reported with
 * eta_global). */
int dpg_estimate(dpg_handle* h, const dpg_complex* xhat, dpg_complex* u, double* eta,
                 double* eta_global, dpg_stream s);

/* Fixed-fraction marking of the adaptive loop of Sec. 4.2 (refinement
 * fraction 0.30 and coarsening fraction 0.05 in its parameter table of
 * App. C.2): with eta (device, n_elem doubles, e.g. from dpg_estimate) the
 * cells are ranked by eta_K; the largest are marked +1 (refine) until their
 * share of sum eta_K^power reaches refine_frac (the crossing cell included),
 * the smallest -1 (coarsen) while their share stays within coarsen_frac; a
 * cell marked +1 is never marked -1; ties go by element index.  The paper
 * names the fractions but not the measure: power 1 sums the residual norms
 * themselves ("their combined residual"), power 2 is Doerfler's bulk
 * criterion on the squared global estimate sqrt(sum eta_K^2).
 * marks: host, n_elem int8.  Host logic after one device-to-host copy;
 * synchronises the stream.  Errors: DPG_ERR_ARG (power not 1 or 2, fraction
 * outside [0, 1]). */
int dpg_mark_fraction(dpg_handle* h, const double* eta, double refine_frac, double coarsen_frac, int32_t power,
                      int8_t* marks, dpg_stream s);

/* Number of elements whose eta_K^2 came out negative (through rounding, when
 * eta_K ~ 0) in the last dpg_estimate or dpg_estimate_noalloc and was set to
 * 0.  count: host.  Synchronises the device. */
int dpg_estimate_clamped(dpg_handle* h, int32_t* count);

/* Allocation-free variant of dpg_estimate, for callers that cannot allocate
 * device memory during the call (their memory is committed to a pool of
 * their own up front, or their loop may not wait on an allocator).  The paper
 * has no counterpart; it is an interface choice of this library.  Same
 * arguments, results and errors as dpg_estimate, plus DPG_ERR_ARG when the
 * mesh has more than 1,048,575 elements.  Its scratch (the per-element
 * eta_K^2 and their sum) is a fixed 8 MiB array that every GPU loading the
 * library keeps until the process exits; it calls no allocator.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress)
 * and should come before any stream capture.  All calls share the array:
 * calls that overlap on the GPU race and give wrong results. */
int dpg_estimate_noalloc(dpg_handle* h, const dpg_complex* xhat, dpg_complex* u, double* eta,
                         double* eta_global, dpg_stream s);

/* Replace per-element data from host buffers (read on the stream; keep them
 * alive and unmodified until the stream reaches the copy, pinned memory makes
 * the copy asynchronous).  corners: n_elem x 8 x 3 vertex coordinates in the
 * element's vertex order (NULL = keep); the connectivity and therefore the
 * numbering are unchanged, so the corners must keep every Jacobian positive.
 * eps, mu: n_elem complex (NULL = keep).  Invalidates the element stores. */
int dpg_update_elements(dpg_handle* h, const double* corners, const dpg_complex* eps, const dpg_complex* mu,
                        dpg_stream s);

/* Per-handle instrumentation for roofline reporting.  enable != 0 starts
 * recording CUDA events around every element-factorisation launch and resets
 * the counters; dpg_timing_get synchronises nothing and reports the state
 * after the last synchronising call. */
typedef struct {
  double factor_ms;          /* summed device time of the factorisation kernel launches */
  int64_t factor_launches;   /* number of those launches */
  int64_t factor_elements;   /* elements they processed */
  double cg_ms;              /* summed device time of dpg_cg_solve calls */
  int64_t cg_iterations;     /* summed CG iterations */
  int64_t kernel_launches;   /* kernels launched by the library since enable */
  double factor_ms_real;     /* part of factor_ms spent on real-path launches */
  int64_t factor_elements_real;
  double cg_kernel_ms;       /* summed device time of the persistent CG kernel launches */
  int64_t cg_kernel_launches;
  int64_t cg_kernel_iterations;
} dpg_timing;
int dpg_timing_enable(dpg_handle* h, int32_t enable);

/* Algorithmic bytes moved by one CG iteration of the given mode (matrix values,
 * per-entity column lists, preconditioner data and vector traffic), for
 * roofline reporting.  Host only. */
int dpg_cg_bytes_per_iteration(dpg_handle* h, int32_t mode, int64_t* bytes);

/* Real path for lossless elements (default on).  An element with real eps
 * and mu and no Robin face has an augmented system that the unitary diagonal
 * scalings diag(1 on F, -i on I) (test) and diag(-i on E and E-hat, 1 on H
 * and H-hat) (trial) make real; its factorisation then runs in real FP64
 * (a quarter of the flops) and S_K, Z_K, L1 are mapped back exactly.
 * enable = 0 forces the complex path for every element. */
int dpg_set_real_path(dpg_handle* h, int32_t enable);
int dpg_timing_get(dpg_handle* h, dpg_timing* out);

/* Absorbed power and its adjoint gradient (the paper has no adjoint; this is
 * the reactor-optimisation use).  P = 1/2 omega sum_{K in obstacle} Im(eps_K)
 * int_K |E_h|^2 (electric-loss term of Q_em, Sec. 3.2, dimensionless) at the
 * trace solution xhat (device, n complex).  obstacle_mask: device, n_elem
 * bytes (non-zero = in the obstacle).  P: host, may be NULL.  dP_deps_re,
 * dP_deps_im: device, n_elem doubles each, both NULL (P only) or both set:
 * the derivatives of P w.r.t. Re eps_K and Im eps_K for every element, by the
 * adjoint of the DPG minimum-residual problem (one CG solve with the same
 * matrix, mode/rtol/max_iter as dpg_cg_solve, then an element pass that
 * re-forms and refactors G_K).  Needs DPG_FLAG_ADJOINT at setup and a prior
 * dpg_element_batch + dpg_assemble for the current eps.  Synchronises.
 * Errors: DPG_ERR_STATE, DPG_ERR_ARG, DPG_ERR_NOT_CONVERGED, DPG_ERR_NOMEM. */
int dpg_grad_eps(dpg_handle* h, const dpg_complex* xhat, const uint8_t* obstacle_mask, double* P,
                 double* dP_deps_re, double* dP_deps_im, int32_t cg_mode, double cg_rtol, int32_t max_iter,
                 dpg_stream s);

/* Arithmetic of the element factorisation (the blocked partial Cholesky of
 * the augmented element matrix that condenses to S_K, Sec. 2.3, Eq.
 * linear_system).  The diagonal blocks and the panel triangular solves are
 * FP64 in both modes.  DPG_FACTOR_FP64: the trailing updates too, on the FP64
 * pipe.  DPG_FACTOR_TC_SPLIT (default): the trailing updates on the tensor
 * cores at FP64 accuracy, through an error-free splitting of each panel row
 * (scaled by a power of two 2^e > its largest entry) into seven 8-bit integer
 * digits, FP16 MMAs whose FP32 accumulators hold exact integers, and one
 * rounding to FP64 per update (the error of an update is about
 * 2^-57 2^e_i 2^e_j times the panel width, below FP64's own bound).  Changing the mode reallocates
 * the chunk workspace and invalidates the element stores.
 * Errors: DPG_ERR_ARG (unknown mode), DPG_ERR_NOMEM. */
int dpg_set_factor_arith(dpg_handle* h, int32_t arith);

/* Stored-factor estimator (Sec. 2.3: eta_K = ||Psi_K||_V = ||L^{-1} r_K||).
 * enable = 1: every element pass keeps, per element, X = (L^{-1} [B | B-hat |
 * l])^H, which its factorisation leaves below G's factor (n_v x (m + 1)
 * values, m = n_u + n_h; real on the real path: 1.8 MB per p = 2 element), and
 * dpg_estimate / dpg_estimate_noalloc form L^{-1} r_K = L^{-1} l - (L^{-1} B) u
 * - (L^{-1} B-hat) uhat_K from it directly, instead of a second element pass
 * that forms K and factors G again.  Same definition, different order of the
 * same exact operations.  The next dpg_element_batch writes X (until then the
 * estimator keeps the second pass).  enable = 0 frees it.  Not with
 * DPG_FLAG_STREAM.  Errors: DPG_ERR_ARG, DPG_ERR_NOMEM, DPG_ERR_UNSUPPORTED. */
int dpg_set_estimator_store(dpg_handle* h, int32_t enable);

/* Order-bucketed element pass (Sec. 4: p-adaptive and AMR meshes mix trial
 * orders, so element work is uneven).  enable = 1: the pass runs in waves; a
 * wave forms one chunk of every (order, arithmetic) list, each into its own
 * slice of the K workspace, then factors all of them in ONE persistent launch
 * (one CTA per SM) that takes elements from a work list ordered longest
 * first (complex before real, then by matrix size: LPT), then extracts chunk
 * by chunk.  Waves are formed per wave group (one per chunk colour in
 * streaming mode, one otherwise).  A group's number of waves: at least what a
 * 48 GB budget for the K workspace requires, and at least enough that its
 * costliest list (largest N^3, complex four times real) puts no more elements
 * into a wave than there are SMs; with the setup's chunk size, the group's
 * largest list's share of a wave.  enable = 0: one launch per chunk of a single order (default).
 * Results are identical in both modes (the same per-element arithmetic).
 * Changing the mode reallocates the chunk workspace and invalidates the
 * element stores.  The FP64-pipe factorisation (DPG_FACTOR_FP64) keeps one
 * launch per chunk inside each wave.  dpg_autotune sizes per-order chunks and
 * is refused in this mode.  Errors: DPG_ERR_ARG, DPG_ERR_NOMEM. */
int dpg_set_bucketed(dpg_handle* h, int32_t enable);

/* Load balance of the last element pass's tensor-core factorisation, from
 * per-element stamps (SM, start and end on the global timer) that the
 * factorisation kernels write.  busy (host, written): the sum over elements
 * of their factorisation time divided by (number of SMs x the summed span of
 * the factorisation launches), i.e. 1 minus the SM-idle fraction of those
 * launches; span_ms: the summed span; items: elements counted.  Synchronous.
 * Errors: DPG_ERR_ARG, DPG_ERR_STATE (no pass on the current plan, or the
 * last pass used the FP64-pipe factorisation, which writes no stamps). */
int dpg_factor_balance(dpg_handle* h, double* busy, double* span_ms, int64_t* items);

/* Check hook of the two factorisation kernels: run the element factorisation
 * of dpg_element_batch on one augmented matrix given on the host.  A (host,
 * read): N x N column-major, lower triangle used, real (cplx = 0: N^2
 * doubles) or complex (cplx = 1: N^2 interleaved re, im pairs).  Pivots
 * [0, nv) positive, then the trailing block is negated, pivots [nv, npiv)
 * positive; only rows and columns [0, nact) take part.  out (host, written,
 * same layout): the factored matrix.  not_hpd (host, may be NULL): 1 if a
 * pivot was not positive.  arith: DPG_FACTOR_*.  Synchronous, uses the
 * current device.  Errors: DPG_ERR_ARG, DPG_ERR_NOMEM, DPG_ERR_TIMEOUT,
 * DPG_ERR_CUDA, DPG_ERR_UNSUPPORTED (N > 3315). */
int dpg_factor_check(int32_t arith, int32_t cplx, int32_t N, int32_t nact, int32_t nv, int32_t npiv, const double* A,
                     double* out, int32_t* not_hpd);

/* Bound of the device-side waits of the CG kernel (its grid barriers): a
 * wait that has not seen every block arrive after wait_ns nanoseconds of the
 * GPU's global timer gives up, every block leaves the kernel, and dpg_cg_solve
 * returns DPG_ERR_TIMEOUT with the context still usable.  Default 5 s.
 * hold != 0 is a test hook of that failure path: no barrier releases, so the
 * next solve's first wait runs out on purpose (no fault, no trap).  The paper
 * has no counterpart; this is failure detection of this library.
 * Errors: DPG_ERR_ARG (wait_ns <= 0). */
int dpg_set_wait_limit(dpg_handle* h, int64_t wait_ns, int32_t hold);

/* The element pass runs as a fixed launch plan: per trial degree and
 * arithmetic class (real path / complex), chunks of at most that degree's
 * chunk size.  The plan (device element lists, Robin face sub-batches) is
 * built on the first dpg_element_batch and captured into a CUDA graph that
 * later passes replay (enable = 0: plain launches, no graph).  A change of
 * chunk sizes, real-path switch or element classes rebuilds it. */
int dpg_set_graph(dpg_handle* h, int32_t enable);

/* Chunk-size autotuner (the paper has no counterpart; it serves the batched
 * element pass): per trial-degree group, time one chunk of the group's larger
 * arithmetic class at candidate sizes (multiples of the SM count whose chunk
 * workspace fits max_workspace_bytes) and keep the fastest per element; the
 * workspace is then reallocated for the chosen sizes.  caps (host out, one per
 * group, may be NULL): chosen chunk sizes; ms_per_element (host out, may be
 * NULL): their measured time per element.  Overwrites the element stores of
 * the timed elements (run dpg_element_batch afterwards).  Synchronises.
 * Errors: DPG_ERR_ARG, DPG_ERR_NOMEM, DPG_ERR_CUDA. */
int dpg_autotune(dpg_handle* h, double max_workspace_bytes, int32_t* caps, float* ms_per_element, dpg_stream s);

/* Order groups (host out, each may be NULL; arrays of length *n_groups <= 4):
 * trial degree, number of elements and current chunk size of each group,
 * ascending degree. */
int dpg_group_info(dpg_handle* h, int32_t* n_groups, int32_t* p, int32_t* n_elem, int32_t* cap);

/* Electromagnetic power of a trace solution (Sec. 3.2): with the interior
 * fields u_K of dpg_estimate and the element pass's Gauss-Legendre rule,
 *   q (device, n_elem doubles, may be NULL): int_K Q_em dV,
 *     Q_em = 1/2 omega (Im eps |E|^2 + Im mu |H|^2) (dimensionless; the
 *     conductivity is part of Im eps);
 *   flux (host, n_robin doubles, may be NULL): per Robin group, the sum over
 *     its faces of int Re(E x conj(H)) . n dA with the outward normal (inflow
 *     through a port is negative).  The reference field of Eq. (power_scaling)
 *     follows on the host: E0^2 = 2 Z0 P_input / (-flux_port).
 * xhat: device, n complex.  Synchronises when flux is given.
 * Errors: DPG_ERR_STATE (no element pass), DPG_ERR_ARG, DPG_ERR_NOMEM. */
int dpg_power(dpg_handle* h, const dpg_complex* xhat, double* q, double* flux, dpg_stream s);

/* Sizes: n = free trace unknowns, nnz of the CSR matrix, per-element sizes
 * (the largest over the elements when the degrees differ). */
int dpg_sizes(dpg_handle* h, int64_t* n, int64_t* nnz, int32_t* n_elem, int32_t* n_v,
              int32_t* n_u, int32_t* n_h);

/* Per-element layout (host out, each may be NULL): p (n_elem trial degrees),
 * u_off (n_elem + 1): offset of element e's interior values in the u vector of
 * dpg_estimate, u_off[n_elem] = its length; h_off (n_elem + 1): offset of
 * element e's entries in the trace map, h_off[n_elem] = its length.  For one
 * degree u_off[e] = e n_u and h_off[e] = e n_h. */
int dpg_element_layout(dpg_handle* h, int8_t* p, int64_t* u_off, int64_t* h_off);

/* Element-local to global trace map (host out, h_off[n_elem] int32, element
 * e's n_h(e) entries at h_off[e]): >= 0 free unknown index, -1 fixed by
 * Dirichlet data, -2 removed (unpaired H-hat) or unused slot (mixed degrees).
 * fixed_val (host out, same layout, complex, may be NULL): value of fixed
 * entries (0 elsewhere). */
int dpg_trace_map(dpg_handle* h, int32_t* map, dpg_complex* fixed_val);

/* Debug dump for parity tests: for n_ids element ids (host) of one trial
 * degree write into host buffers (each may be NULL) G (n_v x n_v, row-major),
 * B (n_v x n_u), B-hat (n_v x n_h), l (n_v), S (n_h x n_h), s (n_h), with the
 * sizes of that degree (S, s in the element's trace slots, see above).  Runs
 * the element formation and condensation for those elements only;
 * synchronises.  Errors: DPG_ERR_ARG for ids out of range or of different
 * degrees. */
int dpg_element_dump(dpg_handle* h, const int32_t* ids, int32_t n_ids, dpg_complex* G,
                     dpg_complex* B, dpg_complex* Bh, dpg_complex* l, dpg_complex* S,
                     dpg_complex* s, dpg_stream st);

/* Copy of the assembled CSR system to host buffers (each may be NULL):
 * row_ptr (n + 1 int64), col (nnz int32), val (nnz complex), b (n complex). */
int dpg_csr_copy(dpg_handle* h, int64_t* row_ptr, int32_t* col, dpg_complex* val,
                 dpg_complex* b, dpg_stream s);

/* Check hook of the tensor-core contraction: C (Ma x Nb, row-major) = A^T B
 * with A (Kd x Ma) and B (Kd x Nb) row-major FP64 host arrays, computed on the
 * current device by the kernel the TF32 (split = 1) or 3XTF32 (split = 3)
 * precision modes use.  upper_only != 0 computes only the 128 x 128 tiles on or
 * above the diagonal (the rest of C is left untouched).  Synchronous.
 * Errors: DPG_ERR_ARG, DPG_ERR_NOMEM, DPG_ERR_TIMEOUT (a bounded wait gave up),
 * DPG_ERR_CUDA. */
int dpg_tc_gemm(int32_t split, int32_t Ma, int32_t Nb, int32_t Kd, const double* A, const double* B, double* C,
                int32_t upper_only);

/* Device FP64 and FP32 fused-multiply-add throughput (FLOP/s) measured by a
 * short probe kernel on the current device (used to state roofline peaks). */
int dpg_probe_peaks(double* fp64_flops, double* fp32_flops, dpg_stream s);

const char* dpg_last_error(dpg_handle* h);
void dpg_destroy(dpg_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* DPG_H */
