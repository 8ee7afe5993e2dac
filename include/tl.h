/*
 * tl.h -- C ABI of the GB300 T10 Total-Lagrangian force / tangent / Hessian
 * assembly path and the backward-Euler Newton step that consumes it.
 *
 * The operations follow arxiv 2604.10357 (TL-FEA Part II):
 *   Sec. 2     eq. stepmap, eq. residual, eq. cost, eq. lambda_update
 *   Sec. 4.1   precomputation of reference-configuration constants
 *   Sec. 4.2   fixed-sparsity CSR patterns (built once)
 *   Sec. 4.3   internal force, eq. F_assembly, eq. fint_local, eq. fint_global
 *   Sec. 4.4   gradient (eq. grad_L) and Hessian (eq. hessian, eq. tangent_block)
 *   Sec. 4.6   Newton solver, Algorithm 3
 *
 * Conventions shared by every call:
 *   - Nodal vectors (q_n, v, f_int, g, ...) are float64 arrays of length
 *     ndof = 3*nn, node-major (x, y, z of node 0, then node 1, ...).
 *   - T10 connectivity: corners 0..3 (positively oriented), then midside
 *     nodes on edges 4:(0,1) 5:(1,2) 6:(0,2) 7:(0,3) 8:(1,3) 9:(2,3).
 *     Midside nodes must sit at edge midpoints (straight-sided elements).
 *   - Except for tl_mesh_create's host inputs and the host pointers named as
 *     such, every array argument is a DEVICE pointer owned by the caller; the
 *     library never frees it and keeps no reference after the call returns.
 *   - The mesh handle owns every internal buffer (pattern, slot map,
 *     precomputed geometry, mass, solver state) and frees it in
 *     tl_mesh_destroy.
 *   - Calls are asynchronous on the stream given at creation unless stated
 *     otherwise.  Device-side errors found by a kernel (an inverted element,
 *     a non-finite value) are sticky and are returned by tl_sync.
 *   - No call aborts, traps or prints: errors come back as tl_status and
 *     tl_last_error(mesh) holds a one-line description.
 *   - One GPU: the handle is bound to the device that was current at
 *     creation.
 */
#ifndef TL_H_
#define TL_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tl_status {
  TL_OK = 0,
  TL_ERR_INVALID_ARG = 1,   /* bad pointer, size, connectivity or geometry   */
  TL_ERR_OOM = 2,           /* device allocation failed                       */
  TL_ERR_CUDA = 3,          /* a CUDA runtime call failed                     */
  TL_ERR_INVERTED = 4,      /* det F <= 0 at some quadrature point            */
  TL_ERR_NONFINITE = 5,     /* NaN or Inf in a residual or Hessian            */
  TL_ERR_NOT_CONVERGED = 6, /* Newton/ALM iteration caps reached              */
  TL_ERR_SOLVER = 7,        /* the sparse direct solver failed (zero pivot)   */
  TL_ERR_TIMEOUT = 8,       /* a bounded device-side wait expired             */
  TL_ERR_OVERFLOW = 9,      /* nnz or an index would not fit in int32         */
  TL_ERR_UNSUPPORTED = 10,  /* a mesh or option this build does not handle    */
  TL_ERR_STATE = 11         /* call order violated (e.g. no pattern yet)      */
} tl_status;

typedef enum tl_material_kind { TL_SVK = 0, TL_MOONEY_RIVLIN = 1 } tl_material_kind;

/* Element arithmetic precision.  TL_FP64: every element quantity in float64.
 * TL_FP32_ELEM: element kinematics, stress and tangent in float32 with the
 * Green strain formed as E = (H + H^T + H^T H)/2 from the displacement
 * gradient H; nodal forces are accumulated in float64 and Hessian values are
 * float32.  Residual, constraint rows and updates stay float64. */
typedef enum tl_precision { TL_FP64 = 0, TL_FP32_ELEM = 1 } tl_precision;

/* Material of a set of elements (Sec. 4.3 Stage 1: SVK or compressible
 * Mooney-Rivlin, plus optional Kelvin-Voigt damping; the paper defers the
 * constitutive forms to its Part I, so they are stated here):
 *   SVK  : S = lambda tr(E) I + 2 mu E, lambda/mu from (E, nu)
 *   MR   : W = C10(J^-2/3 I1 - 3) + C01(J^-4/3 I2 - 3) + kappa/2 (J-1)^2
 *   KV   : S_v = lambda_d tr(Edot) I + 2 eta_d Edot, Edot = sym(F^T Fdot);
 *          off when eta_d == lambda_d == 0.
 * rho0 is the reference density (mass matrix, gravity load). */
typedef struct tl_material {
  int32_t kind;               /* tl_material_kind */
  int32_t _pad;
  double E, nu, rho0;
  double C10, C01, kappa;
  double eta_d, lambda_d;
} tl_material;

/* Newton / ALM controls (Algorithm 3).  The inner loop stops when
 * ||g|| <= max(atol, rtol * ||g(v_n; lambda)||), i.e. relative to the
 * residual at the plain previous-velocity start whatever start is used. */
typedef enum tl_linear_solver {
  TL_SOLVER_DIRECT = 0,       /* vendor sparse Cholesky (analysis once, factor per iteration) */
  TL_SOLVER_PCG = 1           /* preconditioned CG on the device (3x3 block Jacobi) */
} tl_linear_solver;

typedef struct tl_params {
  double h;                   /* time step */
  double rho_alm;             /* ALM penalty rho */
  double rtol, atol;          /* inner stopping tolerances */
  double eps_out;             /* outer stop: ||c||_2 <= eps_out */
  double gravity[3];          /* body-force field per unit mass (f_ff) */
  int32_t max_inner;          /* L_max */
  int32_t max_outer;          /* K_max */
  int32_t linear_solver;      /* tl_linear_solver */
  int32_t lin_max_iter;       /* PCG iteration cap (0: 5000) */
  double lin_rtol;            /* PCG: ||H dv + g|| <= eta ||g|| with eta = lin_rtol (0: 1e-10,    */
                              /* 1e-6 for TL_FP32_ELEM), or, if lin_adaptive,                   */
                              /* eta = max(lin_rtol, min(0.5, 0.1 target / ||g||))              */
  int32_t lin_adaptive;       /* 1: inexact Newton (solve only as tightly as the target needs) */
  int32_t use_graph;          /* 1: run the step as one captured CUDA graph with device-side */
                              /* convergence control (PCG only; see tl_newton_step)           */
  int32_t line_search;        /* 1: Armijo backtracking on phi = ||g||^2 / 2 (eq. armijo) after */
                              /* each Newton solve: accept v + a dv once                        */
                              /* phi(a) <= (1 - 2 c1 a) phi(0), a = 1, beta, beta^2, ...; after   */
                              /* ls_max_trials rejected trials v is kept and the inner loop ends  */
  int32_t ls_max_trials;      /* j_max (0: 10) */
  double ls_c1;               /* c1 (0: 1e-4) */
  double ls_beta;             /* beta (0: 0.5) */
} tl_params;

typedef struct tl_newton_stats {
  int32_t inner_iters;        /* Newton iterations summed over outer loops */
  int32_t outer_iters;
  int32_t converged;          /* 1 when inner and outer criteria were met */
  int32_t _pad;
  double g_ref;               /* ||g(v_n; lambda)|| at the start of the step */
  double g_norm;              /* last inner residual norm */
  double c_norm;              /* last ||c||_2 */
  double ms_total;            /* wall time of the whole step */
  double ms_assembly;         /* residual + Hessian assembly kernels */
  double ms_solver;           /* factorisation + solves (or PCG) */
  int32_t lin_iters;          /* PCG iterations summed over the step */
  int32_t ls_trials;          /* line-search trial points evaluated over the step */
  double g_init;              /* ||g|| at the start velocity (v_init or v_n) */
} tl_newton_stats;

typedef struct tl_mesh_info {
  int64_t nn, ne, ndof, nnz, nnz_node, nfixed;
  int32_t precision, nmat;
  int64_t ncon;               /* general constraint rows (lambda arrays hold 3*nfixed + ncon) */
  int32_t element_kind;       /* tl_element_kind */
  int32_t nen;                /* nodes (T10) or coefficients (ANCF) per element */
} tl_mesh_info;

/* Element kinds (Sec. 4.3): 10-node tetrahedra, the two-node ANCF3243 beam
 * and the four-node ANCF3443 shell.  An ANCF physical node carries four
 * coefficient vectors (position r and gradients r_x, r_y, r_z, Sec. 2), and
 * every "node" of the calls below is then a coefficient: ndof = 3 ncoef. */
typedef enum tl_element_kind {
  TL_ELEM_T10 = 0,
  TL_ELEM_ANCF3243 = 1,
  TL_ELEM_ANCF3443 = 2
} tl_element_kind;

typedef struct tl_mesh tl_mesh;   /* opaque, library-owned */

/* Create a mesh handle and upload it (Sec. 4.1 precomputation).
 *   X            HOST, nn*3 float64 reference coordinates
 *   conn         HOST, ne*10 int32 T10 connectivity (order above)
 *   mats, nmat   HOST, material table (nmat >= 1)
 *   mat_of_elem  HOST, ne int32 indices into mats, or NULL (all material 0)
 *   precision    tl_precision
 *   stream       cudaStream_t to run on (NULL = legacy default stream)
 * Validates connectivity range, straight-sided midside nodes and a positive
 * reference volume of every element (TL_ERR_INVALID_ARG otherwise).
 * Synchronous.  On success *out receives the handle. */
tl_status tl_mesh_create(const double* X, int64_t nn, const int32_t* conn, int64_t ne,
                         const tl_material* mats, int32_t nmat, const int32_t* mat_of_elem,
                         int32_t precision, void* stream, tl_mesh** out);

/* Create an ANCF mesh handle (Sec. 2, Sec. 4.3: 8 shape functions and a
 * 3 x 2 x 2 Gauss-Legendre rule per beam element, 16 and 4 x 4 x 3 per shell
 * element; Sec. 4.1: exact consistent mass).
 *   kind         TL_ELEM_ANCF3243 or TL_ELEM_ANCF3443
 *   E0           HOST, ncoef*3 float64 reference coefficient vectors
 *   ncoef        number of coefficients (four per physical node)
 *   conn         HOST, ne*8 (beam) or ne*16 (shell) int32 coefficient ids.
 *                Beam: node A's r, r_x, r_y, r_z, then node B's, A at
 *                xi = -1.  Shell: the corners at (xi, eta) = (-1,-1), (1,-1),
 *                (1,1), (-1,1), each r, r_x, r_y, r_z.
 *   dims         HOST, ne*3 float64 element length L, width W and height /
 *                thickness H.  Beam: x = L (1+xi)/2, y = W eta/2,
 *                z = H zeta/2; shell: x = L (1+xi)/2, y = W (1+eta)/2,
 *                z = H zeta/2 (the shape functions are scaled by them).
 *   mats, nmat, mat_of_elem, stream   as tl_mesh_create
 *   precision    TL_FP64 (TL_FP32_ELEM gives TL_ERR_UNSUPPORTED)
 * Validates coefficient ids, positive dims and det J0 > 0 at every element
 * quadrature point (TL_ERR_INVALID_ARG otherwise).  The handle takes every
 * call below: fixed nodes are coefficients (clamp c = e - e0 on all three
 * components), q, v, f_ext and lambda are per coefficient, the gravity load
 * is g int rho S_a dV, and tl_get_pattern's slot map and tl_eval_tangent's
 * K_elem hold (3 nen)^2 entries per element.  The float32 element form, the
 * launch-shape choices of the autotuner and the learned warm start are T10
 * features.  Synchronous. */
tl_status tl_mesh_create_ancf(int32_t kind, const double* E0, int64_t ncoef, const int32_t* conn, int64_t ne,
                              const double* dims, const tl_material* mats, int32_t nmat,
                              const int32_t* mat_of_elem, int32_t precision, void* stream, tl_mesh** out);

/* General linear bilateral constraints c(q) = C q - b (Sec. 4.2: C_q in CSR
 * with a user-given fixed pattern), in addition to the clamp rows of
 * tl_build_pattern.  Must come before tl_build_pattern, which adds every node
 * pair that a row couples to the Newton-matrix pattern (so h^2 rho C^T C has
 * no fill-in).  Their multipliers follow the 3*nfixed clamp multipliers in
 * every lambda array (length 3*nfixed + ncon); the residual adds
 * h C^T (lambda + rho c), the Newton matrix h^2 rho C^T C, the ALM update
 * lambda += rho c and ||c|| covers both kinds of rows.
 *   ncon     number of rows (0: no-op)
 *   row_ptr  HOST, ncon + 1 int32 offsets (row_ptr[0] = 0, ascending)
 *   col      HOST, row_ptr[ncon] int32 DOF indices (3 I + d), in [0, 3 nn)
 *   val, b   HOST, row_ptr[ncon] and ncon float64
 * Copied to the device; TL_ERR_STATE after tl_build_pattern or when set
 * twice, TL_ERR_INVALID_ARG on a malformed CSR. */
tl_status tl_set_constraints(tl_mesh* m, int64_t ncon, const int32_t* row_ptr, const int32_t* col,
                             const double* val, const double* b);

/* Build, once, everything that depends only on topology and the reference
 * configuration (Sec. 4.2): the coefficient-level adjacency, the DOF-level
 * CSR pattern of H (3x3 blocks per adjacent node pair, rows and columns
 * ascending, full symmetric storage), the per-element slot map, the
 * consistent mass (Sec. 4.1, integrated exactly) and the clamp constraint
 * rows (identity rows of C_q, one per DOF of each fixed node).  For a
 * TL_FP32_ELEM handle with fewer than 2^24 nodes also the per-tile
 * aggregation maps of the assembly (distinct node pairs of each 32-element
 * tile and the element blocks that add to them; about 38 KB per tile).
 *   fixed_nodes  HOST, nfixed int32 node ids (any order, no duplicates)
 *   nnz_out      HOST, receives nnz of H
 * Synchronous.  TL_ERR_OVERFLOW if nnz >= 2^31. */
tl_status tl_build_pattern(tl_mesh* m, const int32_t* fixed_nodes, int64_t nfixed,
                           int64_t* nnz_out);

/* Copy the pattern out (device pointers, caller-allocated):
 *   row_ptr   (ndof+1) int32, col (nnz) int32: the CSR of H
 *   slot_map  (ne*nd*nd, nd = 3 nen: 900 for T10) int32 or NULL: position in
 *             values[] of K_elem entry (r, s), r = 3a+i (row), s = 3b+k
 *             (column), element order as given at creation. */
tl_status tl_get_pattern(const tl_mesh* m, int32_t* row_ptr, int32_t* col, int32_t* slot_map);

/* Internal force f_int(q_n + h v, v) (eq. residual's force term, eq. fint_local
 * and eq. fint_global): elastic plus Kelvin-Voigt stress.  h = 0 evaluates the
 * force at configuration q_n.  f_int: ndof float64, overwritten. */
tl_status tl_eval_force(tl_mesh* m, const double* q_n, const double* v, double h, double* f_int);

/* Element tangents (eq. tangent_block) at q = q_n + h v:
 *   K_elem[e*nd*nd + nd r + s] = alpha * K_t,e + beta * D_e   (nd = 3 nen)
 * with K_t the stiffness (geometric term with the total second Piola-Kirchhoff
 * stress, elastic plus viscous) and D the Kelvin-Voigt velocity tangent
 * df/dv at fixed q.  float64 for TL_FP64 meshes, float32 for TL_FP32_ELEM. */
tl_status tl_eval_tangent(tl_mesh* m, const double* q_n, const double* v, double h,
                          double alpha, double beta, void* K_elem);

/* CSR values of the Newton matrix (eq. hessian with the Kelvin-Voigt term):
 *   H = M/h + h K_t + D + h^2 rho C_q^T C_q      at q = q_n + h v
 * values: nnz entries (float64 or float32 by precision), overwritten.
 * f_int: NULL, or ndof float64 that receives f_int(q_n + h v, v) from the same
 * fused pass (force + tangent + assembly in one kernel). */
tl_status tl_assemble_hessian(tl_mesh* m, const double* q_n, const double* v, double h,
                              double rho_alm, void* values, double* f_int);

/* Residual of eq. residual / eq. grad_L:
 *   g = M (v - v_n)/h + f_int(q_n + h v, v) - f_ext - f_ff + h C_q^T (lambda + rho c)
 * with f_ff = (row sums of M) x gravity and c = (q_n + h v - X) on clamped DOFs.
 *   f_int   ndof float64 holding f_int(q_n + h v, v) already (e.g. from the
 *           fused tl_assemble_hessian pass), or NULL to evaluate it here in
 *           float64 class for both element forms (TL_FP32_ELEM handles: in
 *           double-float arithmetic when force_split is set, else float64)
 *   f_ext   ndof float64 or NULL (zero)
 *   lambda  3*nfixed float64 (multiplier of DOF d of the j-th fixed node at
 *           3j+d, fixed nodes in ascending id order), or NULL (zero)
 *   g       ndof float64, overwritten
 *   g_norm  1 float64 (device), receives ||g||_2 */
tl_status tl_eval_residual(tl_mesh* m, const tl_params* p, const double* q_n, const double* v_n,
                           const double* v, const double* f_int, const double* f_ext,
                           const double* lambda, double* g, double* g_norm);

/* Allocation-free variant of tl_eval_residual.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * during the time-stepping loop -- for example a host application whose
 * device memory is owned by its own pool allocator or fixed budget, or a
 * latency-critical loop in which a cudaMalloc (which may synchronize the
 * device) is not acceptable.
 *   It computes the same g and ||g||_2 as tl_eval_residual (with the mass
 * product always in float64, whatever residual_split says), but keeps its norm partials in a fixed scratch array compiled into
 * the library (128 KiB of device memory held by every GPU that loads the
 * library, until the process exits) instead of a buffer owned by the handle.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 *   f_int is required here (compute it with tl_eval_force or the fused
 * tl_assemble_hessian pass); the other arguments are as in tl_eval_residual.
 *   Limit: meshes of at most 4,194,304 nodes (16,384 blocks of 256 nodes);
 * larger meshes get TL_ERR_UNSUPPORTED with a message.
 *   The first call on a device looks up the scratch array's device address
 * (with the mesh's device current, which this call requires); make that first
 * call before any stream capture.  Every call shares the one scratch array:
 * calls that overlap on the GPU (other streams, other handles) race and may
 * return wrong norms; serialise them.  Each call writes every scratch entry it
 * reads, so nothing needs clearing between calls. */
tl_status tl_eval_residual_noalloc(tl_mesh* m, const tl_params* p, const double* q_n,
                                   const double* v_n, const double* v, const double* f_int,
                                   const double* f_ext, const double* lambda, double* g,
                                   double* g_norm);

/* Kernel timing and launch counting (instrumentation of the calls above).
 * While enabled, every element-kernel pass and every residual pass of this
 * handle is bracketed by CUDA events recorded on the handle's stream.
 * tl_timing_read synchronizes the stream, sums the elapsed times per
 * category and resets the accumulators.  Launch counts are kept always. */
typedef struct tl_timing {
  double ms_element;          /* fused force / tangent / assembly kernels */
  double ms_residual;         /* residual + norm kernels */
  int64_t n_element;          /* element passes timed */
  int64_t n_residual;
  int64_t launches;           /* kernels of this library launched since the last read */
} tl_timing;

tl_status tl_timing_enable(tl_mesh* m, int32_t on);
tl_status tl_timing_read(tl_mesh* m, tl_timing* out);

/* One backward-Euler time step by Newton's method in the augmented-Lagrangian
 * loop (Algorithm 3 without line search, Algorithm 1's multiplier update,
 * eq. stepmap q = q_n + h v).  Per inner iteration: residual and ||g|| on the
 * device (norm copied to the host for the test), Hessian assembly, numeric
 * Cholesky factorization on the fixed pattern and solve H dv = -g (vendor
 * sparse solver; symbolic analysis with a nested-dissection ordering is done
 * on the first call and kept by the handle), v += dv.  After each inner loop
 * the clamp constraints c = q - X are evaluated and, if the inner loop
 * converged, lambda += rho c.
 *   q_n, v_n   ndof float64 (device): previous configuration and velocity
 *   v_init     ndof float64 start velocity (e.g. a learned warm start), or
 *              NULL for v_n; the inner tolerance is always relative to
 *              ||g(v_n; lambda)||
 *   f_ext      ndof float64 applied loads, or NULL
 *   lambda     3*nfixed float64 multipliers (in/out, persist across steps)
 *   v_out,q_out ndof float64 outputs (v_out may not alias q_n / v_n)
 *   stats      HOST, optional: iterations, norms, split timings
 * For TL_FP32_ELEM meshes the Hessian, its factorization and the direction
 * are float32 while the residual keeps a float64 force evaluation.
 *   Inner solver (p->linear_solver): TL_SOLVER_DIRECT = vendor sparse
 * Cholesky; TL_SOLVER_PCG = block-Jacobi conjugate gradients on the device to
 * ||H dv + g|| <= eta ||g|| (eta from lin_rtol / lin_adaptive; with
 * TL_FP32_ELEM and lin_rtol = 0 eta is at least 1e-6).  PCG
 * stops early when p.Hp <= 0 (H not positive definite along p).
 *   p->use_graph = 1 (PCG only) runs the whole step as one captured CUDA
 * graph: the loops are conditional graph nodes, the tests on ||g||, ||c||
 * and the PCG residual are made on the device, and the host waits once.
 * The caller's arrays are copied into handle-owned buffers around the graph
 * launch; the graph is captured on the first call and again whenever the
 * parameters, the precision or the autotuner's choice change.  PCG iteration
 * counts are multiples of 8 in this mode; ms_assembly / ms_solver are 0.
 * Synchronous.  Returns TL_ERR_NOT_CONVERGED (with the last iterate in
 * v_out / q_out) when the caps are reached, TL_ERR_SOLVER when the direct
 * factorization meets a zero pivot, TL_ERR_NONFINITE on a non-finite norm,
 * TL_ERR_UNSUPPORTED for use_graph with the direct solver. */
tl_status tl_newton_step(tl_mesh* m, const tl_params* p, const double* q_n, const double* v_n,
                         const double* v_init, const double* f_ext, double* lambda,
                         double* v_out, double* q_out, tl_newton_stats* stats);

/* ---- first-order inner solver: AdamW (Algorithm 2) -----------------------
 * Hyperparameters of Algorithm 2; the paper prints none of the AdamW values
 * (it tunes them per problem), so all are the caller's.  Inner stop, tested
 * every check_every iterations: ||g|| <= eps_in (1 + ||v||) or
 * ||g|| <= eps_rel ||g_0|| (g_0: first gradient of the outer iteration). */
typedef struct tl_adamw_params {
  double lr;                  /* step size alpha (constant) */
  double beta1, beta2;        /* moment decay rates, in [0, 1) */
  double eps;                 /* > 0, added to sqrt(s_hat) */
  double weight_decay;        /* lambda_wd (decoupled) */
  double eps_in, eps_rel;     /* inner stopping tolerances */
  int32_t max_inner;          /* L_max >= 1 */
  int32_t check_every;        /* >= 1 */
} tl_adamw_params;

typedef struct tl_adamw_stats {
  int32_t inner_iters;        /* AdamW iterations summed over outer loops */
  int32_t outer_iters;
  int32_t converged;          /* 1 when the inner test and ||c|| <= eps_out were met */
  int32_t _pad;
  double g_norm;              /* last gradient norm */
  double c_norm;              /* last ||c||_2 */
  double ms_total;            /* wall time of the step */
} tl_adamw_stats;

/* One backward-Euler step with the AdamW inner solver inside the ALM loop
 * (Algorithm 2 with Algorithm 1's multiplier update).  Per inner iteration,
 * on the device: m and s from the previous gradient (reset to zero at every
 * outer iteration), bias correction, v = (1 - lr wd) v - lr m_hat /
 * (sqrt(s_hat) + eps), the internal force at q_n + h v (float64 class) and
 * g of eq. grad_L with ||g||.  After the inner loop v is committed as the
 * velocity the inertia term is measured from (v_n <- v, as Algorithm 2
 * prints it), lambda += rho c and ||c|| ends the outer loop when the inner
 * test was met and ||c|| <= eps_out.
 *   p: h, rho_alm, eps_out, max_outer and gravity are used (the Newton fields
 *      are ignored); a: the AdamW parameters above
 *   q_n, v_n, v_init (nullable: v_n), f_ext (nullable), lambda (in/out,
 *   3*nfixed), v_out, q_out: device float64 arrays as in tl_newton_step.
 * Returns TL_OK when converged, TL_ERR_NOT_CONVERGED when the caps are
 * reached (v_out, q_out, lambda hold the last iterate),
 * TL_ERR_NONFINITE on a non-finite gradient, TL_ERR_INVALID_ARG on bad
 * parameters.  Synchronous. */
tl_status tl_adamw_step(tl_mesh* m, const tl_params* p, const tl_adamw_params* a, const double* q_n,
                        const double* v_n, const double* v_init, const double* f_ext, double* lambda,
                        double* v_out, double* q_out, tl_adamw_stats* stats);

/* ---- autotuner of the launch shapes (no counterpart in the paper) --------
 * Times, on this handle's mesh at the state (q_n, v, h), every compiled
 * variant of the two hot launches and keeps the fastest for later calls:
 *   element pass (fused force + tangent + CSR assembly): persistent grid
 *     (SMs x resident CTAs) or one CTA per 32-element tile; for
 *     TL_FP32_ELEM also the scatter (exchanged 3-entry runs issued as vector
 *     reductions, or one scalar reduction per entry), the prefetch of the
 *     next tile (cp.async into shared memory, or none), warp
 *     specialisation (5 extra warps issue a tile's reductions while the
 *     compute warps evaluate the next tile), two CTAs per SM (registers
 *     capped at 64, no prefetch buffer), and, for the fastest of these, the
 *     tile order (in order, or permuted so that tiles in flight are far apart);
 *   PCG product H p: 4, 8 or 16 lanes per node (one neighbour per lane), and for the
 *     float32 iteration 8, 16 or 32 lanes per node along the contiguous rows;
 *   the fastest exchanged FP32 variant with per-tile aggregation of shared node pairs;
 *   residual: 1 or 4 lanes per node, or the double-float mass product;
 *   TL_FP32_ELEM: the Newton residual's internal force in float64 and double-float (timed
 *     and reported only; force_split is left as the caller set it);
 * reps timed launches per variant after one warm-up.  Needs the pattern;
 * allocates and frees one CSR values array and one force array.  Synchronous.
 * The result does not change any computed value beyond the rounding order of
 * the reductions.  ms_element[k]: k = 4*(1-prefetch) + 2*(1-xchg) + full_grid;
 * ms_spmv[k]: 4, 8, 16 lanes. */
typedef struct tl_tune_result {
  int32_t spmv_group;         /* lanes per node in H p: 4, 8, 16 or 32 (default 4; 8 for TL_FP32_ELEM) */
  int32_t elem_xchg;          /* 1: exchanged vector runs (FP32 assembly) */
  int32_t elem_full_grid;     /* 1: one CTA per tile; 0: persistent grid */
  int32_t elem_prefetch;      /* 1: cp.async prefetch of the next tile (FP32) */
  int32_t elem_ws;            /* 1: warp-specialised scatter (FP32; with xchg, prefetch, persistent grid) */
  int32_t residual_lanes;     /* lanes per node in the residual: 1 or 4 (with residual_split, 1 = one lane
                                 per row of the mass in sliced ELL: slices of 32 rows ordered by length) */
  int32_t elem_occ2;          /* 1: two CTAs per SM (FP32 exchanged assembly, one material kind) */
  int32_t elem_spread;        /* 1: tiles in flight spread over the mesh (permuted launch order) */
  float ms_element[8];        /* measured element-pass times without warp specialisation (0: not measured) */
  float ms_ws;                /* measured time of the warp-specialised variant (0: not measured) */
  float ms_spmv[3];
  float ms_residual[2];       /* residual with 1 and 4 lanes per node */
  float ms_occ2;              /* measured time of the two-CTA variant (0: not measured) */
  float ms_spread;            /* the chosen element variant with the permuted tile order */
  int32_t pcg_f32;            /* FP32 Hessian: 1 = PCG vectors in float32 (dot products accumulated in
                                 float64), 0 = float64 vectors; not timed by tl_autotune (it changes
                                 the rounding of the iterates, not only their order); default 1 */
  int32_t spmv_row;           /* float32 PCG iteration: 1 = row-contiguous H p (the group's lanes read
                                 contiguous runs of the three rows), 0 = one neighbour per lane
                                 (default 0; 1 for TL_FP32_ELEM) */
  float ms_spmv_row[3];       /* measured row-contiguous H p with 8, 16, 32 lanes per node (0: not measured) */
  int32_t elem_agg;           /* 1: FP32 exchanged assembly sums the node-pair blocks that several elements
                                 of a 32-element tile share before the reductions (per-tile maps built on
                                 the device by tl_build_pattern for FP32 handles with < 2^24 nodes: about
                                 38 KB per tile of 32 elements); default 1 */
  float ms_agg;               /* fastest measured exchanged variant with aggregation (0: not measured) */
  int32_t residual_split;     /* 1: the residual's mass product M (v - v_n) in double-float arithmetic
                                 (float32 pairs with 48-bit significands, error-free products and sums;
                                 the rest of the residual float64); 0: float64 (default 1) */
  float ms_residual_split[2]; /* measured double-float residual with 1 and 4 lanes per node (0: not measured) */
  int32_t force_split;        /* TL_FP32_ELEM: 1 = the float64-class internal force of the Newton residual
                                 in double-float arithmetic (48-bit significands), 0 = float64 (default 0).
                                 A precision trade, never chosen by tl_autotune: element displacements are
                                 taken relative to the element's first node in float64 first; the force error
                                 then measured 0.05x a 1e-8 Newton target on a 452k-DOF cantilever under large
                                 rotation (1.65x with absolute displacements) */
  float ms_force[2];          /* measured residual force, float64 and double-float (0: not measured) */
  int32_t elem_pair;          /* TL_FP32_ELEM tangent passes: 1 = St. Venant-Kirchhoff (+ Kelvin-Voigt)
                                 segments in the closed-form pair kernel (per node pair and point
                                 [K_ab]_ik = wJ0 [c1 g_a,i g_b,k + c2 (g_b,i g_a,k + (n_a.n_b) B_ik)
                                 + alpha delta_ik n_a.S n_b], g = F n, B = F F^T; CSR values through the
                                 per-tile maps, needs elem_agg; or K_elem); Mooney-Rivlin segments keep
                                 the generic kernel; default 1 */
  float ms_pair;              /* fastest measured pair-kernel variant (0: not measured) */
  int32_t elem_fold;          /* pair kernel: 1 = folded form, where c1 + c2 >= max(|c1|, |c2|) / 4 for every
                                 segment of the launch (else the unfolded form runs): Q_ab = sum over points of
                                 wJ0 g_a g_b^T + [(n_a.n_b) c2 wJ0 B + (n_a.alpha wJ0 S n_b) I] / (c1 + c2),
                                 then K_ab = c1 Q_ab + c2 Q_ab^T once per tile; 0 = the unfolded form always
                                 (default 1) */
} tl_tune_result;

tl_status tl_autotune(tl_mesh* m, const double* q_n, const double* v, double h, int32_t reps,
                      tl_tune_result* out);
/* Current choice (timings zero), and an explicit choice (validated). */
tl_status tl_tune_get(const tl_mesh* m, tl_tune_result* out);
tl_status tl_tune_set(tl_mesh* m, const tl_tune_result* in);

/* ---- learned Newton warm start (no counterpart in the paper) -------------
 * The paper starts each Newton solve from v_n (Algorithm 3).  These calls
 * run a per-node MLP 10 -> 64 -> 64 -> 64 -> 3 (tanh hidden layers, linear
 * output) with bfloat16 weights and activations and float32 accumulation,
 * and train it.  params: 9219 bf16 values (raw uint16 bits) laid out as
 * W1 (64x10, row = output), b1 (64), W2 (64x64), b2 (64), W3 (64x64), b3 (64),
 * W4 (3x64), b4 (3).  All arrays are device pointers; stream is a
 * cudaStream_t (NULL = legacy default stream).  Asynchronous. */

/* out[n][3] = MLP(feats[n][10]); acts (n x 192 bf16: h1, h2, h3) or NULL. */
tl_status tl_mlp_forward(const uint16_t* params, const float* feats, int64_t n, float* out,
                         uint16_t* acts, void* stream);
/* grads[9219] (float32, accumulated: zero it first) += d/dparams sum(dout * out),
 * from the activations a forward pass saved. */
tl_status tl_mlp_backward(const uint16_t* params, const float* feats, const uint16_t* acts,
                          const float* dout, int64_t n, float* grads, void* stream);
/* dout = 2 w (out - target); *loss (float64, accumulated) += sum w |out - target|^2. */
tl_status tl_mlp_mse_grad(const float* out, const float* target, const float* weight, int64_t n,
                          float* dout, double* loss, void* stream);
/* One Adam step on the float32 master copy; params receives its bf16 rounding. */
tl_status tl_mlp_adam(float* master, uint16_t* params, const float* grads, float* m1, float* m2,
                      int64_t n, float lr, float beta1, float beta2, float eps, int32_t step,
                      void* stream);
/* The start's inputs per node: feats[nn][10] = ((nabla v_n / s1, nabla^2 v_n / s2,
 * nabla^3 v_n / s3) / r_I, fixed flag), the backward differences of the velocity
 * history v_n, v_prev = v_{n-1}, v_prev2 = v_{n-2}, v_prev3 = v_{n-3} (device, 3*nn
 * float64 each) formed in float64, scaled, divided by r_I, the norm of node I's nine
 * scaled differences (0 where r_I = 0), and rounded to float32.  A NULL history
 * velocity (and every older one) is not available: the differences that need it are
 * 0.  s1, s2, s3 > 0 (else TL_ERR_INVALID_ARG).  Asynchronous on the handle's stream. */
tl_status tl_mlp_features(tl_mesh* m, const double* v_n, const double* v_prev, const double* v_prev2,
                          const double* v_prev3, double s1, double s2, double s3, float* feats);
/* v_init = b + s_out r_I MLP(features) on free nodes, 0 on clamped nodes, where
 * b = v_n + nabla v_n + nabla^2 v_n + nabla^3 v_n is the polynomial extrapolation
 * of the available history (cubic with four velocities; quadratic, linear or v_n
 * itself with fewer) and r_I the node scale of tl_mlp_features: the network learns
 * a correction of b.  params NULL: b only (work and scales unused).  work: 13*nn
 * float32 device scratch (features and outputs). */
tl_status tl_warm_start(tl_mesh* m, const uint16_t* params, const double* v_n, const double* v_prev,
                        const double* v_prev2, const double* v_prev3, double s1, double s2, double s3,
                        double s_out, float* work, double* v_init);
/* The training target target[nn][3] = (v_next - b) / (s_out r_I) (float64, then
 * float32), 0 on clamped nodes and where r_I = 0; b and r_I as in tl_warm_start.
 * s1, s2, s3, s_out > 0. */
tl_status tl_mlp_target(tl_mesh* m, const double* v_next, const double* v_n, const double* v_prev,
                        const double* v_prev2, const double* v_prev3, double s1, double s2, double s3,
                        double s_out, float* target);
/* out[c] += sum_i x[i][c]^2 (float64 accumulation) for the ncol (1..16) columns of
 * the row-major float32 array x[n][ncol] (device): the statistics that set the
 * input and output scales.  out is a device array of ncol doubles (zero it
 * first).  Asynchronous on stream. */
tl_status tl_mlp_col_sumsq(const float* x, int64_t n, int32_t ncol, double* out, void* stream);

/* Wait for the handle's stream and return the first sticky device-side error
 * (TL_ERR_INVERTED, TL_ERR_NONFINITE) raised since the last tl_sync, then
 * clear it. */
tl_status tl_sync(tl_mesh* m);

tl_status tl_mesh_info_get(const tl_mesh* m, tl_mesh_info* out);
const char* tl_status_string(tl_status s);
const char* tl_last_error(const tl_mesh* m);
void tl_mesh_destroy(tl_mesh* m);

#ifdef __cplusplus
}
#endif
#endif /* TL_H_ */
