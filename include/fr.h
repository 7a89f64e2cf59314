/*
 * fr.h - C ABI of the GB300 flux-reconstruction hot path.
 *
 * The library evaluates the flux reconstruction (FR) residual of the
 * compressible Euler / Navier-Stokes equations on quadrilateral (2D) or
 * hexahedral (3D) elements of mixed polynomial degree p, its exact
 * linearisation (JVP) and transpose (VJP), the paper's finite-difference
 * Jacobian-vector product, restarted GMRES on (sigma I - dR/dq), one ESDIRK
 * stage by pseudo-transient continuation, the spectral-decay smoothness
 * indicator and the p-adaptation that reorders elements into per-degree
 * buckets.  The method is that of Wang, Gobbert & Yu, "A dynamically
 * load-balanced parallel p-adaptive implicit high-order flux reconstruction
 * method for under-resolved turbulence simulation" (arXiv:1910.03693):
 * Sec. 2.1 (equations), Sec. 2.2 (FR/CPR), Sec. 2.3 (ESDIRK, pseudo-transient
 * continuation, matrix-free GMRES), Sec. 3.1 (p-adaptation).
 *
 * Conventions common to every call
 *  - Pointers named *_dev are device pointers; *_host are host pointers.
 *    Every device buffer passed in is owned by the caller and must stay valid
 *    until the work queued on `stream` has finished.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *    only queue kernels return as soon as the work is queued; calls that must
 *    read a device value to decide (gmres_solve, esdirk_stage, p_rebucket)
 *    synchronise `stream`.
 *  - Errors are returned as fr_status, never thrown.  After FR_ERR_CUDA the
 *    context may be unusable; fr_last_error() gives a message.
 *  - "State layout" (internal): elements are stored in per-degree buckets in
 *    ascending (p, element id) order; inside an element the block is
 *    [nv][n_sp] with the solution point index xi-fastest.  fr_pack/fr_unpack
 *    convert from/to the canonical layout: element by element in id order,
 *    n_sp(p_e) = (p_e+1)^nd points (xi fastest) times nv variables (variable
 *    fastest), FP64.  nv = nd + 2: (rho, rho u_i, rho E).
 *  - Precision: FR_F64 buffers are double, FR_F32 buffers are float.
 *    FR_BF16OP (residual, JVP, VJP, GMRES products): float buffers and FP32
 *    arithmetic with every operator matrix of the discretisation (Lagrange
 *    interpolation and differentiation, correction-function derivatives,
 *    mortar interpolation and projection) rounded to bfloat16, 8 significant
 *    bits: the trial of BF16 operators.  Pack, unpack and the indicator
 *    treat it as FR_F32.
 *    FR_DF (fr_residual and the stage's early Newton iterates only): FP64
 *    buffers in the FP64 state layout, evaluated in double-float arithmetic
 *    (each value an unevaluated sum of two FP32 numbers, about 48
 *    significant bits, error-free transformations on the FP32 pipe).
 */
#ifndef FR_H
#define FR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FR_OK = 0,
  FR_ERR_INVALID = -1,        /* bad argument (sizes, pointers, degrees)          */
  FR_ERR_CUDA = -2,           /* a CUDA call failed                               */
  FR_ERR_NOMEM = -3,          /* device or host allocation failed                 */
  FR_ERR_NOT_CONVERGED = -4,  /* a solver hit its iteration limit                 */
  FR_ERR_NONFINITE = -5,      /* NaN or Inf met in a norm                         */
  FR_ERR_TIMEOUT = -6         /* a bounded device-side wait gave up               */
} fr_status;

typedef enum { FR_F64 = 0, FR_F32 = 1, FR_BF16OP = 2, FR_DF = 3 } fr_prec;
typedef enum { FR_JV_FD = 0, FR_JV_EXACT = 1 } fr_jv_mode;

/* Boundary kinds used in fr_mesh_desc.nbr (negative values). */
#define FR_BC_WALL (-1)      /* no-slip adiabatic wall            */
#define FR_BC_FARFIELD (-2)  /* free-stream ghost state           */

/*
 * Mesh description (host arrays, read during fr_create only).
 *  nodes    [n_elem][(geom_order+1)^nd][nd]: element map nodes at equispaced
 *           reference points, xi fastest.  geom_order is 1 or 2.
 *  nbr      [n_elem][2 nd]: neighbour element through face f = 2 d + s
 *           (d = reference direction, s = 0 at xi_d = -1, 1 at +1), or a
 *           FR_BC_* value.
 *  nbr_face [n_elem][2 nd]: the neighbour's face index (ignored on boundaries).
 *  orient   [n_elem][2 nd]: maps this side's face point (ia, ib) to the
 *           neighbour's: bit 0 swaps the axes, then bit 1 flips the first
 *           (i -> P-1-i), bit 2 the second.  Must be the inverse of the
 *           neighbour's code.
 *  p        [n_elem]: initial degree of each element, p_min <= p <= p_max.
 */
typedef struct {
  int32_t nd;
  int32_t n_elem;
  int32_t geom_order;
  const double* nodes;
  const int32_t* nbr;
  const int8_t* nbr_face;
  const int8_t* orient;
  const int8_t* p;
} fr_mesh_desc;

/* Physics (Sec. 2.1): gamma, constant mu (0 = Euler) and Pr; q_inf is the
 * conservative free-stream state used by far-field boundaries (nv values).
 * flux: the common inviscid flux of the faces (Sec. 2.2), FR_FLUX_RUSANOV or
 * FR_FLUX_ROE (Roe's averaged-Jacobian flux, no entropy fix); both have the
 * exact JVP and VJP. */
#define FR_FLUX_RUSANOV 0
#define FR_FLUX_ROE 1
typedef struct {
  double gamma;
  double mu;
  double Pr;
  double q_inf[5];
  int32_t flux;
} fr_physics;

/* Degree range of the context.  1 <= p_min <= p_max <= 5.  Every buffer the
 * context owns is sized for all elements at p_max, so adaptation never
 * reallocates. */
typedef struct {
  int32_t p_min;
  int32_t p_max;
} fr_limits;

typedef struct fr_ctx fr_ctx;

/* Current layout.  n_dof = nv * sum_e n_sp(p_e); n_dof_capacity is the
 * value at p_max everywhere; bucket_count[p] is the number of elements of
 * degree p (p = 0..5) and bucket_offset[p] the first value of that bucket in
 * the state layout. */
typedef struct {
  int32_t nd, nv, n_elem;
  int64_t n_dof;
  int64_t n_dof_capacity;
  int32_t bucket_count[6];
  int64_t bucket_offset[6];
  int32_t affine;           /* 1 if every element map is affine (constant metrics) */
} fr_layout_info;

/* Create a context: computes metric terms for every degree in [p_min, p_max],
 * the per-degree buckets and the face lists.  Device memory is allocated on
 * the current device.  Returns FR_ERR_INVALID on inconsistent connectivity or
 * degrees out of range. */
fr_status fr_create(const fr_mesh_desc* mesh, const fr_physics* phys, const fr_limits* lim,
                    fr_ctx** out);
fr_status fr_destroy(fr_ctx* ctx);
fr_status fr_layout(const fr_ctx* ctx, fr_layout_info* info);
/* Current degree of every element (host array of n_elem). */
fr_status fr_get_p(const fr_ctx* ctx, int8_t* p_host);
const char* fr_last_error(void);

/* Canonical FP64 <-> state layout in `prec`.  The canonical buffer (n_dof
 * doubles) may be device memory (read or written in place by the layout
 * kernel) or host memory, page-locked or pageable (copied on `stream` through
 * a staging vector of the context; with pageable memory the copy completes
 * before the call returns).  With a host destination, fr_unpack's result is
 * there once `stream` has reached it. */
fr_status fr_pack(fr_ctx* ctx, const double* canon_host_or_dev, void* q_dev, fr_prec prec, void* stream);
fr_status fr_unpack(fr_ctx* ctx, const void* q_dev, fr_prec prec, double* canon_host_or_dev, void* stream);

/* R = R(q) = -div f, Sec. 2.2 Eq. (FR_diff) with the common inviscid flux
 * the context was created with (Rusanov, or Roe's Eq. invis_com), common
 * solution Eq. (com_q) and BR2-type common gradient Eq. (com_grad_q).  q and R
 * are state-layout device buffers of n_dof in `prec` (FR_DF: FP64 buffers). */
fr_status fr_residual(fr_ctx* ctx, const void* q_dev, void* R_dev, fr_prec prec, void* stream);

/* Jv ~ dR(q)/dq v.  FR_JV_EXACT: the exact directional derivative.
 * FR_JV_FD: the paper's one-sided difference (R(q + eps v) - R(q)) / eps
 * (Sec. 2.3), FP64 only; R(q) is evaluated inside. */
fr_status fr_jvp(fr_ctx* ctx, const void* q_dev, const void* v_dev, void* Jv_dev, fr_prec prec,
                 fr_jv_mode mode, double eps, void* stream);

/* Finite-difference Jv, (R(q + eps v) - R(q)) / eps in FP64, that allocates
 * nothing: the same product as fr_jvp(..., FR_F64, FR_JV_FD, eps, ...), with its
 * three work vectors in a device array reserved when the library is loaded
 * (3 x 262,144 doubles, 6 MiB on every device, held until exit).  The paper
 * has no counterpart.  It serves callers that cannot call cudaMalloc once
 * their set-up is done: processes whose device memory is already fully
 * reserved by another allocator (a framework's caching allocator, say), where
 * a new allocation would fail, and loops that must not call the allocator at
 * all, because cudaFree synchronises the whole device and an allocation can
 * stall behind other work.  Nothing else in the call allocates either: the
 * work tables of mixed-degree meshes are built when the layout or the tuning
 * changes (fr_create, p_rebucket, fr_tuning_set, fr_autotune), not on first use.
 * q, v, Jv: FP64 state-layout device buffers of n_dof.  FR_ERR_INVALID when
 * n_dof > 262,144, eps <= 0, or the current device is not the context's.  The
 * first call on each device looks up the array's device address (set-up,
 * once per device, in the runtime's primary context of that device, the only
 * context supported); make that first call before any stream capture begins.
 * All calls share the array, which keeps the last call's contents (each call
 * writes its work vectors before reading them): calls whose GPU work overlaps
 * (other streams, or other threads on the device) race on it. */
fr_status fr_jvp_fd_static(fr_ctx* ctx, const double* q_dev, const double* v_dev, double* Jv_dev,
                           double eps, void* stream);

/* JTw = (dR(q)/dq)^T w, the exact transpose of FR_JV_EXACT. */
fr_status fr_vjp(fr_ctx* ctx, const void* q_dev, const void* w_dev, void* JTw_dev, fr_prec prec,
                 void* stream);

/* Linear operator A x = sigma x - J(q) x of the pseudo-transient Newton step
 * (Sec. 2.3, Eq. linearized_pseudo_transient_final).  q64_dev is the FP64
 * state; when jv_prec is FR_F32 the exact JVP runs in FP32 on a rounded copy. */
typedef struct {
  double sigma;
  const double* q64_dev;
  fr_jv_mode mode;
  fr_prec jv_prec;
  double eps;              /* FD step (FR_JV_FD), paper: 1e-6 */
  int32_t precond;         /* 1: left element-Jacobi preconditioning with the
                              blocks of the last fr_precond_build (Sec. 2.3);
                              the tolerance is then on the preconditioned
                              residual ||M^-1 (b - A x)||                    */
} fr_shifted_op;

typedef struct {
  int32_t m;               /* restart length, 1..63 (paper: 60)             */
  double rtol;             /* relative tolerance (paper: 1e-1)              */
  int32_t max_it;          /* total iterations (paper: 100)                 */
  int32_t reorth;          /* classical Gram-Schmidt passes: 0 one pass (the
                              default of the paper's Krylov library), 1 a
                              second pass when the first left less than
                              1/sqrt(2) of ||w|| (DGKS), 2 always two passes */
} fr_gmres_opts;

typedef struct {
  int32_t iterations;
  int32_t restarts;
  int32_t converged;
  double rel_res;
} fr_gmres_stats;

/* Restarted GMRES(m) (Sec. 2.3: the matrix-free Krylov solve of the
 * linearised pseudo-transient system, Eq. linearized_pseudo_transient_final)
 * from x = 0: classical Gram-Schmidt as opts->reorth says, Givens rotations.
 * b, x: device FP64, n_dof, distinct buffers (b is read during the first
 * cycle).
 *  - Exact products with one or two Gram-Schmidt passes run device-driven
 *    (FR_TUNE_DEVICE_GMRES, the default). The rotations and the convergence
 *    test happen on the device; the host launches the Arnoldi iterations in
 *    batches and synchronises once per batch; launches past convergence
 *    return at entry.
 *  - Otherwise (finite-difference products, the DGKS second pass, or the
 *    flag off), the host synchronises once per Arnoldi iteration.
 *  - The Krylov basis is FP64, or FP32 with FP32 products at rtol >= 1e-4
 *    (FR_TUNE_F32_BASIS). */
fr_status gmres_solve(fr_ctx* ctx, const fr_shifted_op* op, const double* b_dev, double* x_dev,
                      const fr_gmres_opts* opts, fr_gmres_stats* stats, void* stream);

/* ESDIRK tableau (row-major s x s matrix A, weights b). */
typedef struct {
  int32_t s;
  double A[36];
  double b[6];
} fr_tableau;

typedef struct {
  double tol;              /* ||F|| / ||F(q^{0})|| to reach (hot path: 1e-8)  */
  double dtau_init, dtau_max;
  int32_t max_newton;
  int32_t max_halvings;
  fr_jv_mode mode;         /* FD (FP64) or exact                             */
  fr_prec jv_prec;         /* precision of the exact JVP                      */
  double eps;
  fr_gmres_opts gmres;
  double low_above;        /* exact mode: F uses the residual in precision
                              low_prec while the last ||F|| / ||F(q^{0})|| is
                              above this value, the FP64 residual below it (0:
                              FP64 throughout).  Convergence is only declared
                              on an FP64 F, and the last F of the stage is
                              always FP64.                                    */
  int32_t precond;         /* left element-Jacobi preconditioning in GMRES;
                              esdirk_step builds the blocks at q^n with
                              sigma = 1/(w dt) + 1/dtau_max (Sec. 2.3: once
                              per physical time step); esdirk_stage uses the
                              blocks already built                            */
  fr_prec low_prec;        /* FR_DF (double-float) or FR_F32; read only when
                              low_above > 0                                   */
} fr_newton_opts;

typedef struct {
  int32_t newton_iterations;
  int32_t gmres_iterations;
  int32_t halvings;
  int32_t converged;
  double norm0, norm_final;
  int32_t low_evaluations; /* stage residuals evaluated in low_prec          */
  int32_t f64_evaluations; /* stage residuals evaluated in FP64              */
} fr_stage_stats;

/* ESDIRK tableaus (Sec. 2.3; the paper cites them but prints no
 * coefficients).  order 2: three stages, stiffly accurate, L-stable, diagonal
 * 1 - sqrt(2)/2, c = (0, 2g, 1).  order 3: four stages, explicit first stage,
 * stiffly accurate, diagonal g the root near 0.4359 of 6g^3 - 18g^2 + 9g - 1
 * (stability function zero at infinity), c = (0, 2g, 0.6, 1), remaining
 * coefficients from the order-3 conditions.  FR_ERR_INVALID for other orders. */
fr_status fr_esdirk_tableau(int32_t order, fr_tableau* out);

/* Solve stage `stage` (1-based like the paper, 2..s) of one ESDIRK step
 * (Eq. ESDIRK_conservative) by pseudo-transient continuation with SER
 * (Eqs. pseudo_transient, ser).  qn: q^n; Rstages[j] = R(q^{j+1}) for
 * j < stage-1 (inputs); qi: in = initial guess, out = q^stage; on return
 * Rstages[stage-1] (if non-NULL) holds R(q^stage).  All FP64 device buffers
 * of n_dof in state layout. */
fr_status esdirk_stage(fr_ctx* ctx, const fr_tableau* tab, int32_t stage, double dt,
                       const double* qn_dev, double* const* Rstages_dev, double* qi_dev,
                       const fr_newton_opts* opts, fr_stage_stats* stats, void* stream);

/* Spectral decay indicator (Sec. 3.1): eta_e for variable `var` (paper: 1 =
 * rho u) and the maximum over elements.  eta_dev: n_elem doubles in element
 * id order; eta_max_dev: one double.  Deterministic (fixed summation order). */
fr_status spectral_decay_indicator(fr_ctx* ctx, const void* q_dev, fr_prec prec, int32_t var,
                                   double* eta_dev, double* eta_max_dev, void* stream);

typedef struct {
  double nu_max, nu_min;   /* paper: 0.1, 0.001                              */
  int32_t p_min, p_max;    /* within the context's limits                     */
} fr_adapt_opts;

/* p-adaptation (Sec. 3.1): decide p from eta, limit neighbour jumps to one
 * (raise-only fixed point), prolong / project every element's state, and
 * reorder elements into (p, id) buckets, replacing the paper's repartition.
 * q_inout is a state-layout buffer of n_dof_capacity values; on return it
 * holds the state in the new layout.  perm_out (device, optional) receives
 * the element id at each new bucket position. */
fr_status p_rebucket(fr_ctx* ctx, const double* eta_dev, const double* eta_max_dev,
                     const fr_adapt_opts* opts, void* q_inout_dev, fr_prec prec,
                     int32_t* perm_out_dev, void* stream);

/* Nodal polynomial filter (Sec. 4.2, after Fischer and Mullen): every element
 * of degree p > p_above (paper: 2) becomes (1 - alpha) q + alpha P_{p-1} q,
 * P_{p-1} the modal truncation to degree p - 1 (paper: alpha = 0.2, applied
 * to p = 3 with projection onto p = 2).  q_dev: FP64 state layout, in place.
 * alpha in [0, 1]. */
fr_status fr_filter(fr_ctx* ctx, double* q_dev, double alpha, int32_t p_above, void* stream);

/* Double-float arithmetic of FR_DF, elementwise on device arrays of n FP64
 * values: a, b, c are converted to double-float (nearest FP32 plus the FP32
 * rounding of the remainder), op 0 a + b, 1 a - b, 2 a * b, 3 a * b + c,
 * 4 a / b, 5 sqrt(a), and the result is written as the FP64 value of its
 * two parts.  b is read for ops 0-4, c for op 3 (else they may be null).
 * Exposed for checking the arithmetic against exact rational results. */
fr_status fr_dfloat_eval(int32_t op, const double* a, const double* b, const double* c, double* out, int64_t n,
                         void* stream);

/* Element-Jacobi preconditioner (Sec. 2.3): the inverses of the diagonal
 * blocks (one dense block per element, all of its DOFs) of
 * sigma I - dR/dq(q).  fr_precond_build reads the blocks off the exact FP32
 * JVP at q64_dev (FP64 state layout) with unit vectors, probing the elements
 * of one colour of a distance-1 colouring of the face graph together, and
 * inverts each by Gauss-Jordan elimination with partial pivoting in FP32
 * (blocks of up to 144 DOFs in shared memory; larger ones, 3D p >= 3 with 320,
 * 625 or 1080 DOFs, by a blocked elimination on the block in global memory:
 * panels of 32 pivots, then one rank-32 update of the other columns); it
 * synchronises `stream`.  Storage: the sum of the squared block sizes in
 * floats (32^3 elements at p = 3: 13.4 GB).  FR_ERR_NONFINITE on a singular block.
 * Rebucketing or retuning invalidates the blocks.  fr_precond_apply: z =
 * M^-1 w (FP64 state layout, z may alias w).  fr_precond_release frees the
 * block storage. */
fr_status fr_precond_build(fr_ctx* ctx, const double* q64_dev, double sigma, void* stream);
fr_status fr_precond_apply(fr_ctx* ctx, const double* w_dev, double* z_dev, void* stream);
fr_status fr_precond_release(fr_ctx* ctx);

/* One physical time step of an ESDIRK scheme (Eqs. ESDIRK_ns,
 * ESDIRK_conservative): R(q^n), then stages 2..s by esdirk_stage (each stage
 * starts from the previous stage value), then q^{n+1} = q^n + dt sum_i b_i
 * R(q^i).  q_inout: FP64 state layout, in q^n, out q^{n+1}; a buffer of
 * n_dof_capacity values when `adapt` is given.  stats: s-1 entries, one per
 * implicit stage (optional).  With `adapt` (optional) the step ends with the
 * spectral decay indicator of variable adapt_var and p_rebucket, as the paper
 * does after every step (Sec. 3.1); the layout, n_dof and the degrees change.
 * The context keeps s stage residuals and two state vectors (allocated on
 * first use).  FR_ERR_NOT_CONVERGED if a stage misses its tolerance, in which
 * case q_inout is left unchanged and no adaptation happens. */
fr_status esdirk_step(fr_ctx* ctx, const fr_tableau* tab, double dt, double* q_inout_dev,
                      const fr_newton_opts* opts, fr_stage_stats* stats, const fr_adapt_opts* adapt,
                      int32_t adapt_var, void* stream);

/* Launch configuration (the paper has no counterpart: it is the GPU work
 * decomposition).  The trace and volume kernels process `epb` elements per
 * CTA (one thread per solution point); with several degree buckets they run
 * as one persistent launch over a table of (bucket, tile) items ordered by
 * decreasing cost n_sp (p+1) per tile, the paper's element-weight estimate
 * (Sec. 3.2).  In GMRES with the exact JVP, each Arnoldi product -J V[j]
 * (column gather, JVP kernels, sign) is replayed from a CUDA graph captured
 * once per set of buffers, with j read from device memory.
 *
 * fr_autotune times every admissible epb for each degree present and each
 * kernel (trace, volume residual, volume JVP) in FP64 and FP32 on the state
 * q64_dev (FP64, state layout, n_dof), then one launch per bucket against the
 * multi-bucket launch for each kernel, and keeps the fastest; it synchronises `stream` and
 * changes no result beyond rounding order.  fr_tuning_get/fr_tuning_set read
 * and write the table, 2 x 3 x 7 int32 [precision f64 (also used by the
 * double-float kernels, same operand size), f32][kernel trace,
 * volume residual, volume JVP][P = p+1]: for P >= 2 the elements per CTA
 * of the one-launch-per-bucket kernels, 0 = default (as many whole elements
 * as fit 256 threads; a value whose elements exceed 256 threads also falls
 * back to it; the multi-bucket launch always fills its 256-thread blocks);
 * the slot P = 0 holds the multi-bucket choice of that precision and kernel
 * (0 undecided: one launch over all buckets while the mesh's solution points
 * fit in 8 full-occupancy waves of the GPU, else one per bucket; 1 one launch
 * over all buckets; 2 one launch per bucket), which FR_TUNE_MULTI_LAUNCH
 * enables; slot [0][0][P = 1] holds the element weight
 * that orders the multi-bucket work table (0 n_sp (p+1), 1 n_sp, 2 n_sp^2,
 * 3 n_sp^3: the paper's candidate weights, Sec. 3.2); slot [prec][2][P = 1]
 * chooses the exact JVP's kernels where FR_TUNE_FUSED_JVP allows the
 * compact-trace ones (every face interior and conforming): 1 the fused
 * face-and-volume kernel, 2 the trace-gradient three passes, 3 (and 0,
 * undecided) the compact three passes, 4 two compact passes, the face kernel
 * forming the tangent's traces itself (FP32 with FR_TUNE_TMA_FACES, degrees
 * whose face points fit a warp: 3D p = 1, 3 and 2D p = 3; elsewhere, or when
 * v's element blocks are not 16-byte aligned, the compact three passes run;
 * the two compact choices give the same bits); fr_autotune times those that
 * apply; and the flags below.  fr_tuning_set with table NULL changes only the
 * flags; elements per CTA outside [0, 256], multi-bucket choices outside
 * [0, 2], weight models outside [0, 3], the exact JVP's choice outside [0, 4]
 * or unknown flag bits give FR_ERR_INVALID. */
#define FR_TUNE_MULTI_LAUNCH 1  /* one persistent launch over all degree buckets */
#define FR_TUNE_GRAPHS 2        /* host-driven GMRES: the Arnoldi products
                                   replayed from a CUDA graph               */
#define FR_TUNE_DIAG_METRICS 4  /* 3D meshes of axis-aligned affine elements:
                                   kernels that skip the zero metric terms   */
#define FR_TUNE_FUSED_JVP 8     /* meshes whose faces are all interior and
                                   conforming (same degree both sides, no
                                   boundary): the exact JVP from compact
                                   traces (q and its normal derivative), as
                                   three passes or as one face-and-volume
                                   kernel per element tile (tuning slot)     */
#define FR_TUNE_DF_ARNOLDI 16   /* GMRES: the Arnoldi dot products accumulated
                                   in double-float arithmetic on the FP32 pipe
                                   (FP64 vectors and grid reduction; about
                                   1e-14 of |u| |w| from the FP64 dots); off
                                   by default: measured no faster           */
#define FR_TUNE_ARNOLDI_RUNS 32 /* GMRES: the Arnoldi dots and updates read each
                                   column in runs of 4 x 512 contiguous bytes a
                                   warp (the default; off: one 512-byte segment
                                   a warp, the segments one grid apart)      */
#define FR_TUNE_TMA_FACES 64    /* the compact face kernel's shared-memory tiles
                                   filled by bulk asynchronous copies (TMA),
                                   double-buffered in a persistent walk, where
                                   every block is a multiple of 16 bytes (the
                                   default; off: loads by the threads)       */
#define FR_TUNE_DEVICE_GMRES 128 /* GMRES with exact products and one or two
                                   Gram-Schmidt passes: the Givens rotations
                                   and the convergence test on the device;
                                   the host launches the Arnoldi iterations
                                   in batches and reads the cycle's state once
                                   per batch; launches past convergence
                                   return at entry (the default; off: one
                                   host round trip per iteration, products
                                   replayed from a CUDA graph)               */
#define FR_TUNE_F32_BASIS 256   /* GMRES with exact FP32 products and
                                   rtol >= 1e-4: the Krylov basis, the
                                   products and the preconditioned vectors
                                   stored in FP32, the dots and norms summed
                                   in FP32 over 16 values and in FP64 beyond
                                   (about 1e-6 relative, the products' own
                                   accuracy; the default; off: FP64 basis)  */
fr_status fr_autotune(fr_ctx* ctx, const double* q64_dev, void* stream);
fr_status fr_tuning_get(const fr_ctx* ctx, int32_t* table, int32_t* flags);
fr_status fr_tuning_set(fr_ctx* ctx, const int32_t* table, int32_t flags);

/* Instrumentation (the paper has no counterpart: measurement support).
 * fr_timing(ctx, 1) synchronises the device, clears the counters and starts
 * recording a pair of CUDA events on the launch stream around every kernel
 * the library launches; fr_timing(ctx, 0) stops recording.  The launch
 * counter runs in both states.  fr_timing_report synchronises the device and
 * writes one line per kernel, "name launches total_ms algorithmic_bytes
 * algorithmic_flops" (the minimum bytes the launches had to move and, for the
 * FP64 residual kernels, the operations of the operator as formulated, as
 * counted by each launch site), into buf (len bytes,
 * FR_ERR_INVALID if too small) and the number of launches since the last
 * fr_timing call into *launches (optional). */
fr_status fr_timing(fr_ctx* ctx, int32_t enable);
/* Restrict the event pairs to the kernels whose timing names appear in the
 * comma-separated list `names` (NULL or empty: every kernel, the default);
 * the other launches are still counted, with their algorithmic bytes and
 * operations, and report 0 ms.  Every event pair adds two stream operations
 * around its kernel, so timing one kernel family perturbs a step far less
 * than timing all of them.  Synchronises the device and accumulates what was
 * recorded under the previous selection first. */
fr_status fr_timing_select(fr_ctx* ctx, const char* names);
fr_status fr_timing_report(fr_ctx* ctx, char* buf, int64_t len, int64_t* launches);

/* Device status word of the context (no counterpart in the paper): kernels
 * whose waits are bounded set bit 0 when a wait gives up (the compact face
 * kernel's wait for its bulk copies) and return instead of hanging.
 * Synchronises the device; *status receives the word, cleared when `clear`. */
fr_status fr_device_status(fr_ctx* ctx, int32_t* status, int32_t clear);

/* Arithmetic peak of the current device, measured (measurement support, no
 * counterpart in the paper): a kernel of independent FMA chains (16 per
 * thread, `iters` x 16 FMAs each, 8 warps on every SM x 4 blocks) in FP64
 * (prec FR_F64) or FP32 (FR_F32), timed with CUDA events on `stream`;
 * *tflops = 2 x FMAs / time.  Synchronises `stream`.  FR_ERR_INVALID for other
 * precisions or iters < 1. */
fr_status fr_fma_rate(fr_prec prec, int64_t iters, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FR_H */
