/*
 * wq.h - C ABI of the GB300 weighted-quadrature (WQ) assembly library.
 *
 * The library forms the 3D isogeometric Poisson stiffness matrix S and mass
 * matrix M of a single-patch spline geometry by weighted quadrature
 * (Calabro, Sangalli, Tani, "Fast formation of isogeometric Galerkin matrices
 * by weighted quadrature"), as a CSR matrix in device memory of one GPU:
 *
 *   s_ij ~ sum_{l,m} Q_i( c_lm d_m B_j )   (Eq. (stiff), Eq. (coef_stiff))
 *   m_ij ~ Q_i( c B_j )                    (Eq. (Mass_approx), Eq. (massquadrature))
 *
 * Conventions shared by every entry point:
 *  - Degree p is the same in the three directions, 2 <= p <= 8; each knot vector
 *    is open (end knots repeated p+1 times) with simple, strictly increasing
 *    interior knots (maximal regularity C^{p-1}, Section 3), and at least two
 *    spans per direction.
 *  - Multi-indices i = (i1, i2, i3) are linearised as i1 + n1*(i2 + n2*i3),
 *    direction 1 fastest (Section 3).
 *  - Matrices are full, non-symmetric CSR (WQ does not preserve symmetry,
 *    Section 2 and the Remark on convergence rates): row_ptr int64[N+1],
 *    col int32[nnz], columns ascending inside each row; the pattern of row i is
 *    I_i = I_{1,i1} x I_{2,i2} x I_{3,i3} with I_{l,i} = {j : |i - j| <= p}.
 *  - "d_" pointers are device pointers of the current CUDA device, "h_" host
 *    pointers. `stream` is a cudaStream_t (NULL = legacy default stream); every
 *    asynchronous call only enqueues work on it.
 *  - Every call returns a wq_status; no exception crosses the ABI and no call
 *    falls back to the CPU. wq_last_error() gives a message for the calling
 *    thread. Errors found on the device (det DF <= 0, a breakdown of a rule
 *    solve, a timed-out wait) are recorded in a device error word and reported
 *    by wq_sync_check() or by the next synchronous call.
 *  - Device memory: wq_plan_create allocates the plan's tables, coefficients and
 *    CSR pattern. The staged assembly and the adjoint need scratch that their
 *    first call in each mode allocates (or wq_plan_reserve, ahead of time);
 *    after that no call allocates. Every plan-owned allocation goes through the
 *    allocator of wq_options when one is given, else cudaMalloc.
 *  - Fault injection (testing): the environment variable WQ_FAULT, a
 *    comma-separated list of steps, makes the host path fail at each named
 *    step with WQ_ERR_INJECTED: "alloc" (every plan-owned device allocation),
 *    "h2d" (every host-to-device copy), "solve" (the WQ rule step of a plan
 *    set-up), "geometry" (the coefficient step). A failed wq_plan_create frees
 *    everything it had allocated. Nothing is injected on the device.
 */
#ifndef WQ_H
#define WQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wq_plan_s* wq_plan_t;

typedef enum wq_status {
  WQ_OK = 0,
  WQ_ERR_INVALID_ARG = 1,    /* bad degree, knots, sizes or NULL pointer */
  WQ_ERR_UNSUPPORTED = 2,    /* d != 3, or an option this build does not provide */
  WQ_ERR_SINGULAR_RULE = 3,  /* a rule system of Algorithm 2 broke down */
  WQ_ERR_BAD_GEOMETRY = 4,   /* det DF <= 0 or not finite at a quadrature point */
  WQ_ERR_OOM = 5,            /* device allocation failed */
  WQ_ERR_CUDA = 6,           /* a CUDA runtime call failed (or no device) */
  WQ_ERR_TIMEOUT = 7,        /* a bounded device wait gave up */
  WQ_ERR_INJECTED = 8,       /* failure injected on the host for testing (WQ_FAULT, below) */
  WQ_ERR_NONFINITE = 9       /* checked mode: an assembled value is NaN or infinite */
} wq_status;

/* Value type of the output array. */
enum { WQ_VALUES_F64 = 0, WQ_VALUES_F32 = 1 };

/* Arithmetic of the contraction stages (Eq. (sumfactorization)). The geometry
 * Jacobian, its inverse and determinant always run in FP64. */
enum {
  WQ_PREC_FP64 = 0,          /* FP64 FMA throughout */
  WQ_PREC_FP32 = 1,          /* FP32 FMA, FP32 intermediates */
  WQ_PREC_MIXED = 2,         /* double-float (see below) for the first mode product (contracting
                                q3); the second (q2) in double-float for the first and last p+1
                                rows of direction 2 and for the points q1 that the first and last
                                p+1 rows of direction 1 read, FP32 elsewhere; the last (q1) in
                                FP32 except its first and last p+1 rows of direction 1, which run
                                in FP64; <= 1e-6 row-relative; staged only */
  WQ_PREC_F32X2 = 3,         /* double-float: every value a pair of floats (~48 significant
                                bits), all three mode products on the FP32 pipe; staged only */
  WQ_PREC_TF32X3 = 4         /* as WQ_PREC_MIXED, with the regular rows of the last mode product
                                on the tensor cores: 3xTF32 products (each operand split into two
                                TF32 parts), FP32 accumulation; <= 1e-6 row-relative; staged only */
};

/* Default sentinels of the assembly calls: use the plan's wq_options value. */
#define WQ_VALUES_DEFAULT (-1)
#define WQ_PREC_DEFAULT (-1)

/* ---- options -----------------------------------------------------------------
 * Plan options (the paper has none: these are the library's configuration).
 * wq_options_init fills the defaults; a NULL options pointer means the defaults.
 *   size         sizeof(wq_options) as compiled by the caller (set by wq_options_init)
 *   value_dtype  value type used by assembly calls that pass WQ_VALUES_DEFAULT
 *                (default WQ_VALUES_F64)
 *   precision    WQ_PREC_* used by assembly calls that pass WQ_PREC_DEFAULT
 *                (default WQ_PREC_FP64)
 *   algorithm    WQ_ALGO_* (default WQ_ALGO_AUTO), as wq_plan_set_algorithm
 *   tile         fused-kernel tile extents {t1, t2}, as wq_plan_set_tiles; {0, 0} =
 *                the tune cache's entry for the plan's degree, else the defaults
 *   checked      1: every assembly call first checks that d_vals (nnz values) and
 *                d_kappa (N_QP doubles) each lie inside one allocation of the
 *                plan's device (the driver's address-range query) and returns
 *                WQ_ERR_INVALID_ARG without launching anything otherwise; after
 *                the assembly it scans the values, synchronises `stream` and
 *                returns WQ_ERR_NONFINITE if one is NaN or infinite, or the error
 *                the device recorded. For debugging: it synchronises every call.
 *   tune_cache   NULL, or the path of a text file of "p t1 t2" lines (the format
 *                paper_1605_01238_gb300/tune.py writes), read once at creation
 *   alloc, free  NULL (cudaMalloc / cudaFree), or the caller's device allocator:
 *                alloc(bytes, stream, ctx) returns a device pointer of the
 *                current device, aligned to 256 bytes, or NULL when out of
 *                memory (reported as WQ_ERR_OOM); free(ptr, stream, ctx) releases
 *                one. `stream` is the stream of the call that needs the memory
 *                (NULL when wq_destroy releases the plan, after it has
 *                synchronised the device). Both or neither must be given.
 *   alloc_ctx    passed through to alloc and free
 *   scratch_limit  0 (default: the staged assembly keeps the intermediates of the
 *                whole mesh), or the most bytes of staged scratch (T3, G and the FP64
 *                edge copy of G) to hold at once: the mode products then run slab by
 *                slab of direction 3, each slab at least one row i3 (which can need
 *                more than the limit)
 */
typedef struct wq_options {
  size_t size;
  int value_dtype;
  int precision;
  int algorithm;
  int tile[2];
  int checked;
  const char* tune_cache;
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* alloc_ctx;
  size_t scratch_limit;
} wq_options;

wq_status wq_options_init(wq_options* opt);

/* ---- plan ------------------------------------------------------------------
 * wq_plan_create: builds everything that depends only on the mesh and the
 * geometry (Algorithm 1 and Algorithm 2, plus the CSR pattern):
 *   quadrature points (Remark on the choice of points), B-spline values and
 *   derivatives at the points, exact univariate integrals I^{(a,b)}
 *   (Eq. (integrals)), the four WQ rules per test function (Eq. (exact),
 *   Eq. (support), minimum Euclidean norm, Algorithm 2), the coefficients
 *   c_lm = det DF (DF^{-1} DF^{-T})_lm and c = det DF at every point
 *   (Eq. (coef_stiff), Eq. (mass2)), and the CSR pattern.
 * Arguments:
 *   plan     out: the new plan (owned by the caller, release with wq_plan_destroy)
 *   d        dimension; must be 3
 *   p        degree, 2..8
 *   n_knots  host int64[3]: length of each full knot vector (= n_l + p + 1)
 *   h_knots  host double*[3]: the three full open knot vectors
 *   h_ctrl   host double[N_DOF*3]: control points, xyz interleaved, i1 fastest
 *   opt      NULL (defaults) or the plan's options (copied; see wq_options)
 *   stream   CUDA stream for the set-up work
 * The call copies its host inputs; they may be freed on return. It
 * synchronises `stream` once at the end to report device-side errors.
 */
wq_status wq_plan_create(wq_plan_t* plan, int d, int p, const int64_t n_knots[3],
                         const double* const h_knots[3], const double* h_ctrl, const wq_options* opt,
                         void* stream);

/* Releases every device and host resource of a plan. NULL is accepted. With a
 * caller allocator it first synchronises the device, so that no queued work
 * still uses memory handed back to that allocator. wq_plan_destroy is the
 * same call under its older name. */
wq_status wq_destroy(wq_plan_t plan);
wq_status wq_plan_destroy(wq_plan_t plan);

/* Sizes: n[3] functions per direction, n_qp[3] points per direction, the number
 * of rows N = n1 n2 n3 and of non-zeros nnz = prod_l ((2p+1) n_l - p(p+1))
 * (Section 3, N_NZ for d = 1). Any output pointer may be NULL. */
wq_status wq_plan_info(wq_plan_t plan, int* p, int64_t n[3], int64_t n_qp[3],
                       int64_t* n_rows, int64_t* nnz);

/* Device pointers of the plan-owned CSR pattern (valid until wq_plan_destroy):
 * row_ptr int64[N+1], col int32[nnz]. */
wq_status wq_plan_pattern(wq_plan_t plan, const int64_t** d_row_ptr, const int32_t** d_col);

/* Replaces the control points and recomputes the coefficients (Algorithm 1,
 * last loop) on `stream`, without allocating. ctrl is double[N_DOF*3];
 * ctrl_on_device = 1 for a device pointer, 0 for a host pointer (copied on
 * `stream`; the host buffer must stay valid until the stream reaches the copy,
 * and must be pinned for the copy to be asynchronous). */
wq_status wq_plan_set_geometry(wq_plan_t plan, const double* ctrl, int ctrl_on_device,
                               void* stream);

/* NURBS geometry (Section 3 allows spline or NURBS parametrisations of the domain):
 * with weights w_i > 0 the map is F = sum_i w_i C_i B_i / W, W = sum_i w_i B_i, and
 * DF, det DF and c_lm follow the rational map; the basis functions stay the
 * B-splines pushed forward (R_i = B_i o F^{-1}, Section 3), so the stiffness and
 * mass matrices keep their form. With nurbs_basis = 1 the basis functions are the
 * NURBS w_i B_i / W instead, for which the mass entry is w_i w_j times the B-spline
 * entry with c = det DF / W^2 (the denominator absorbed by c, as stated after
 * Eq. (mass2)); the stiffness then needs terms this library does not assemble, and
 * wq_assemble_stiffness returns WQ_ERR_UNSUPPORTED.
 *   w            NULL (a spline map again), or double[N_DOF] weights, i1 fastest;
 *                host (checked positive) or device memory (on_device = 1), copied
 *   nurbs_basis  0 or 1 (1 requires weights)
 * Recomputes the coefficients on `stream`. The first call allocates the plan-owned
 * copy of the weights. A point where W <= 0 is reported as WQ_ERR_BAD_GEOMETRY by
 * the next synchronous call. wq_adjoint does not handle a rational map. */
wq_status wq_plan_set_weights(wq_plan_t plan, const double* w, int on_device, int nurbs_basis, void* stream);

/* Coefficient tensor of the operator -div(K grad u) (Eq. (coef_stiff) with K:
 * c_lm = det DF (DF^{-1} K DF^{-T})_lm; after Eq. (mass2) the paper lets c take in
 * the coefficient of the PDE).
 *   d_K  NULL (K = I again), or device double[6][N_QP]: K11 K12 K13 K22 K23 K33 at
 *        every point (q1 fastest), symmetric positive definite (not checked), copied
 * Recomputes the coefficients on `stream`; the first call allocates the plan-owned
 * copy. A scalar field d_kappa of the assembly calls still multiplies the result.
 * wq_adjoint does not handle a tensor. */
wq_status wq_plan_set_tensor(wq_plan_t plan, const double* d_K, void* stream);

/* Re-runs in place on `stream` every set-up kernel that depends on the knots or
 * the control points (points, tables, integrals, rules, CSR pattern and
 * coefficients; the Gauss-Legendre rule depends on p only and is computed once
 * by wq_plan_create), without allocating or synchronising: the whole path from
 * knots and control points to a matrix is then wq_plan_refresh + wq_assemble_*.
 * ctrl as in wq_plan_set_geometry, or NULL to keep the plan's current control
 * points. */
wq_status wq_plan_refresh(wq_plan_t plan, const double* ctrl, int ctrl_on_device, void* stream);

/* ---- assembly ---------------------------------------------------------------
 * Writes the nnz values of S (resp. M), in the plan's CSR order, to d_vals.
 *   d_kappa  NULL, or device double[N_QP] (points q1 fastest): a scalar
 *            coefficient field multiplying c_lm (resp. c) at every point
 *            (Eq. (mass2): c absorbs the PDE coefficient)
 *   d_vals   device array of nnz values of type value_dtype, caller-owned
 *   value_dtype  WQ_VALUES_F64, WQ_VALUES_F32 or WQ_VALUES_DEFAULT (the plan's option)
 *   precision    WQ_PREC_FP64 (requires WQ_VALUES_F64), WQ_PREC_FP32, WQ_PREC_MIXED,
 *                WQ_PREC_F32X2 or WQ_PREC_DEFAULT (the plan's option)
 * Asynchronous on `stream`, without synchronisation (unless the plan is in
 * checked mode). The first staged call in a precision mode allocates that mode's
 * plan-owned scratch (see WQ_ALGO_STAGED and wq_plan_reserve); later calls
 * allocate nothing. */
wq_status wq_assemble_stiffness(wq_plan_t plan, const double* d_kappa, void* d_vals,
                                int value_dtype, int precision, void* stream);
wq_status wq_assemble_mass(wq_plan_t plan, const double* d_kappa, void* d_vals,
                           int value_dtype, int precision, void* stream);

/* Assembly algorithm of a plan.
 *   WQ_ALGO_FUSED  one kernel: each block runs the three mode products of
 *                  Eq. (sumfactorization) for a tile of rows in shared memory
 *                  (intermediates of neighbouring tiles overlap and are recomputed)
 *   WQ_ALGO_STAGED three kernels, one per mode product, over the whole mesh; every
 *                  intermediate is computed once and kept in device memory. The
 *                  first staged call allocates plan-owned scratch of
 *                  nnz1_3 * (9 nqp1 nqp2' + 4 nqp1 nnz1_2) values (nnz1_l = band
 *                  pairs of direction l, nqp2' = nqp2 rounded up to even; 2.3 GB in
 *                  FP64 at p = 4, 64^3).
 *   WQ_ALGO_AUTO   (default) staged
 * All give the same values up to rounding order. WQ_PREC_MIXED and WQ_PREC_F32X2
 * exist only as staged kernels and run staged under every setting; the mixed
 * path adds plan-owned scratch for a double-float copy of G at the 3p+1 points of
 * each end of direction 1. */
enum { WQ_ALGO_FUSED = 0, WQ_ALGO_STAGED = 1, WQ_ALGO_AUTO = 2 };
wq_status wq_plan_set_algorithm(wq_plan_t plan, int algorithm);

/* Allocates now, on `stream`, the plan-owned scratch that the first assembly call
 * in (precision, value_dtype) would allocate (the stiffness scratch, which also
 * covers the mass matrix), and with adjoint = 1 the scratch of wq_adjoint, so
 * that the assembly and adjoint calls that follow allocate nothing. */
wq_status wq_plan_reserve(wq_plan_t plan, int precision, int value_dtype, int adjoint, void* stream);

/* Tile extents of the assembly kernels: each block assembles at most t1 x t2
 * rows in directions 1 x 2 for one i3 (the three mode products of
 * Eq. (sumfactorization) share their intermediates inside a tile). t1 = t2 = 0
 * restores the defaults (16 x 4); otherwise 1 <= t1, t2 <= 64. A tile that does
 * not fit in shared memory makes the assembly calls return WQ_ERR_UNSUPPORTED.
 * The autotuner (paper_1605_01238_gb300/tune.py) picks them per degree. */
wq_status wq_plan_set_tiles(wq_plan_t plan, int t1, int t2);
/* The plan's current tile extents (0, 0 = the defaults). */
wq_status wq_plan_get_tiles(wq_plan_t plan, int* t1, int* t2);

/* End-to-end call with host buffers: copies h_ctrl (NULL = keep) to the device,
 * refreshes the plan and assembles S (which = 0) or M (which = 1) in FP64 into
 * h_vals (nnz doubles). With the staged algorithm:
 *   - h_vals page-locked and addressable by the device (wq_host_alloc, or memory
 *     registered with the device): the last mode product stores the values straight
 *     into h_vals, each warp writing runs of consecutive addresses; d_vals is not
 *     touched (it may be NULL);
 *   - any other h_vals: the assembly runs in slabs of direction 3 into the device
 *     staging array d_vals (nnz doubles), and each slab's values (a contiguous range
 *     of the CSR rows) are copied back on a plan-owned copy stream while the next
 *     slab is assembled.
 * Other algorithms assemble into d_vals and copy once. Returns after all work has
 * finished. */
wq_status wq_assemble_host(wq_plan_t plan, int which, const double* h_ctrl, double* d_vals,
                           double* h_vals, void* stream);

/* Page-locked host memory for the end-to-end call (cudaHostAlloc of exactly
 * `bytes`; wq_host_free releases it). */
wq_status wq_host_alloc(size_t bytes, void** h_ptr);
wq_status wq_host_free(void* h_ptr);

/* Load vector by weighted quadrature: b_i = Q_i(f det DF) with the (0,0) rule of
 * every direction (Eq. (quadrule): the WQ approximation of int f R_i dx).
 *   d_f  device double[N_QP]: the source f at the points (q1 fastest)
 *   d_b  device double[N_DOF]: output, i1 fastest
 * Asynchronous on `stream`; the first call allocates plan-owned scratch of
 * N_QP + nqp3 nqp2 n1 + nqp3 n2 n1 doubles. Not provided for NURBS basis functions. */
wq_status wq_assemble_load(wq_plan_t plan, const double* d_f, double* d_b, void* stream);

/* ---- adjoint ------------------------------------------------------------------
 * J = lambda^T S u (which = 1), lambda^T M u (which = 2) or both (which = 3), for
 * the plan's current geometry and the coefficient field kappa, and its gradients
 * with respect to kappa and to the control points. Matrix-free: with the WQ
 * entries of Eq. (stiff) / Eq. (Mass_approx) written out,
 *   J = sum_q kappa(q) [ sum_{lm} c_lm(q) Lam_lm(q) U_m(q) + c(q) Lam_0(q) U_0(q) ],
 * U_m the m-th parametric derivative of u_h = sum_j u_j B_j at the points and
 * Lam_lm = sum_i lambda_i prod_k w^{(delta_kl, delta_km)}_{k,i_k,q_k}, both by sum
 * factorisation; dJ/dkappa is pointwise and dJ/dC follows the chain rule through
 * c_lm = det DF (DF^{-1} DF^{-T})_lm (Eq. (coef_stiff)) and
 * DF = sum_i C_i x grad B_i. The paper has no adjoint; this is its derivative.
 *   d_kappa       NULL (kappa = 1) or device double[N_QP]
 *   d_lambda, d_u device double[N_DOF]
 *   h_J           NULL or host double: J (the call then synchronises `stream`)
 *   d_grad_kappa  NULL or device double[N_QP]
 *   d_grad_ctrl   NULL or device double[N_DOF*3] (xyz interleaved)
 * The first call allocates about (32 N_QP + 9 N_QP) doubles of plan-owned scratch;
 * later calls allocate nothing. It recomputes the coefficients (wq_plan_set_geometry
 * state) before the contractions. */
wq_status wq_adjoint(wq_plan_t plan, int which, const double* d_kappa, const double* d_lambda,
                     const double* d_u, double* h_J, double* d_grad_kappa, double* d_grad_ctrl, void* stream);

/* ---- batched assembly --------------------------------------------------------
 * Many patches of different size and degree assembled by one launch of a CUDA graph
 * captured at creation. The paper treats a single patch; rows of different patches
 * are as independent as rows of one patch (Section 1 notes that every row can be
 * computed on its own). Two forms:
 *  - staged (every plan's algorithm WQ_ALGO_AUTO or WQ_ALGO_STAGED, the default): the
 *    graph holds each patch's staged kernels (stiffness then mass) on up to eight
 *    parallel branches, patches assigned largest first to the least loaded branch;
 *    wq_batch_create reserves each plan's FP64 staged scratch (wq_plan_reserve) and
 *    synchronises `stream` before the capture;
 *  - fused (any plan set to WQ_ALGO_FUSED): one persistent kernel whose blocks take
 *    (patch, matrix, tile) work items from one queue, longest first (a memset of the
 *    work counter and the kernel).
 *   plans        count plans (they must outlive the batch; wq_plan_refresh and
 *                wq_plan_set_geometry update them in place and stay valid)
 *   d_stiffness  NULL or count device pointers (FP64, nnz of each plan; a NULL
 *                entry skips that patch's stiffness matrix)
 *   d_mass       same for the mass matrices
 * Each plan's tile extents (wq_plan_set_tiles) are read at creation. The outputs
 * are fixed at creation; wq_batch_launch replays the graph on `stream`. The batch
 * allocates its own work list with cudaMalloc (not through the plans' allocators). */
typedef struct wq_batch_s* wq_batch_t;
wq_status wq_batch_create(wq_batch_t* batch, int count, const wq_plan_t* plans, void* const* d_stiffness,
                          void* const* d_mass, void* stream);
wq_status wq_batch_launch(wq_batch_t batch, void* stream);
/* The same call under the name of the library's interface description. */
wq_status wq_batch_assemble(wq_batch_t batch, void* stream);
/* Work items ((patch, matrix) jobs when staged, tiles when fused), total nonzeros
 * written per launch, and the graph branches (staged) or persistent grid (fused). */
wq_status wq_batch_info(wq_batch_t batch, int64_t* n_items, int64_t* nnz_total, int* grid);
wq_status wq_batch_destroy(wq_batch_t batch);

/* ---- errors and bookkeeping --------------------------------------------------- */

/* Synchronises `stream`, then reads and clears the plan's device error word. */
wq_status wq_sync_check(wq_plan_t plan, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* wq_last_error(void);

/* Static name of a status code. */
const char* wq_status_string(wq_status status);

/* Number of kernels this library has launched in this process. */
int64_t wq_launch_count(void);

/* ---- inspection (synchronous device-to-host copies, for tests) --------------------
 * wq_get_points:  h_x double[n_qp[dir]]
 * wq_get_rules:   h_w double[n[dir] * nq_max] rule of kind (a, b) for every test
 *                 function i, row i holding w at q = h_q0[i] + t, t < h_nq[i];
 *                 h_q0, h_nq int32[n[dir]] (either may be NULL); nq_max from
 *                 wq_get_nq_max.
 * wq_get_coefficients: h_coef double[7 * N_QP]: c_11 c_12 c_13 c_22 c_23 c_33 c,
 *                 each on the point grid q1 fastest. */
wq_status wq_get_nq_max(wq_plan_t plan, int* nq_max);
wq_status wq_get_points(wq_plan_t plan, int dir, double* h_x);
wq_status wq_get_rules(wq_plan_t plan, int dir, int a, int b, double* h_w, int32_t* h_q0,
                       int32_t* h_nq);
wq_status wq_get_coefficients(wq_plan_t plan, double* h_coef);

/* ---- allocation-free rule construction -------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory themselves: code running under a framework that
 * owns all of GPU memory through its own pool, latency-critical loops that cannot
 * afford cudaMalloc's implicit device synchronisation, and embedded users with a
 * fixed, pre-reserved memory budget.
 *
 * wq_rules_noalloc builds the four WQ rules of ONE direction (the same kernels and
 * results as the rule step of wq_plan_create): for every test function i, the
 * weights w^{(a,b)}_{i,q} of kind 2a+b at q = d_q0[i] + t, t < d_nq[i].
 *   p          degree, 2..8
 *   n_knots    length of the full open knot vector (n = n_knots - p - 1 functions)
 *   h_knots    host double[n_knots]: the knot vector (validated as in wq_plan_create)
 *   d_w        device double[4 * n * nq_stride], caller-owned output (kind-major)
 *   d_q0, d_nq device int32[n], caller-owned outputs
 *   nq_stride  row stride of d_w: at least max_i |Q_i| and at most 4p+1 (outside
 *              that range the call returns WQ_ERR_INVALID_ARG)
 * It calls no cudaMalloc, cudaFree or allocating library routine. Its
 * intermediate tables live in one fixed device array of
 * WQ_RULES_NOALLOC_SCRATCH_BYTES (5.9 MB) that every GPU loading the
 * library holds until the process exits; knot vectors with more than
 * WQ_RULES_NOALLOC_MAX_N basis functions are rejected with WQ_ERR_INVALID_ARG.
 * Every call looks up that array's address in the current device's context
 * (cudaGetSymbolAddress), copies the knot vector from pageable host memory and
 * synchronises `stream` before it returns, so it must never be called on a stream
 * that is being captured into a CUDA graph. Every
 * call shares the one array and clears the parts it reads before writing them;
 * two calls that run at the same time on one device (other threads or streams)
 * race on it, so serialise them. The synchronisation at the end reports a rule
 * breakdown as WQ_ERR_SINGULAR_RULE. */
#define WQ_RULES_NOALLOC_MAX_N 1024
#define WQ_RULES_NOALLOC_SCRATCH_BYTES 5903872
wq_status wq_rules_noalloc(int p, int64_t n_knots, const double* h_knots, double* d_w, int32_t* d_q0,
                           int32_t* d_nq, int nq_stride, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* WQ_H */
