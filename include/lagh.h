/*
 * lagh.h -- C ABI of the GB300 (sm_103a) Lagrangian hydrodynamics library.
 *
 * The library advances the semi-discrete full-order model of "Reduced order
 * models for Lagrangian hydrodynamics" (arXiv 2104.11404), Section 2:
 *
 *   M_V dv/dt = -F(v,e,x) . 1,   M_E de/dt = F(v,e,x)^T . v,   dx/dt = v
 *                                                        (eq:fom, eq:combinedForce)
 *
 * on a Cartesian box mesh with an H1 Q_k kinematic space (positions x,
 * velocities v) and a discontinuous L2 Q_{k-1} thermodynamic space (specific
 * internal energy e), with the RK2-average integrator (eq:RK2-avg) and the
 * automatic time step control of Section 2.2.3 (estimate eq:adaptive-timestep).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Layout.  Kinematic vectors (v, x, F.1, accelerations) have N_V = dim * nnodes
 *   entries, component major: entry [c * nnodes + node].  Nodes are numbered
 *   lexicographically with x fastest: node = I + n0 (J + n1 K), n_c = n_c^el k + 1.
 *   Thermodynamic vectors (e, F^T.v) have N_E = nelem * k^dim entries, element
 *   major (elements lexicographic, x fastest), dofs lexicographic inside the
 *   element.  All values are IEEE double.
 * Pointers.  "device" pointers must be CUDA device (or managed) memory; "host
 *   or device" pointers may be either (the library copies with the CUDA
 *   unified address space).  The caller owns every pointer it passes; the
 *   library never frees or keeps them after the call returns.
 * Streams.  Work is ordered on the stream given to lh_create (a cudaStream_t
 *   passed as void*; NULL = the legacy default stream).  Calls that return a
 *   host value (estimates, iteration counts, statistics, get_state)
 *   synchronize that stream before returning; the others only enqueue.
 * Errors.  Every function returns an lh_status.  On failure lh_last_error(ctx)
 *   describes the cause.  Conditions detected on the device (tangled element,
 *   non-finite state, CG not converged, dt collapse, barrier time-out) are
 *   reported by the next call that synchronizes.
 * Memory.  lh_create allocates every work array of the context; no other
 *   call of a single-instance context allocates device memory.
 */
#ifndef LAGH_H
#define LAGH_H

#include <stdint.h>

#if defined(__GNUC__)
#define LH_API __attribute__((visibility("default")))
#else
#define LH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lh_status {
  LH_OK = 0,
  LH_EINVAL = 1,       /* invalid argument or descriptor */
  LH_ENOMEM = 2,       /* device allocation failed */
  LH_ECUDA = 3,        /* a CUDA runtime call failed */
  LH_ETANGLED = 4,     /* |J| <= 0 at a quadrature point (inverted element) */
  LH_ENONFINITE = 5,   /* NaN or Inf in the state */
  LH_EDTMIN = 6,       /* step size collapsed below dt_min_frac * t_final */
  LH_ECG = 7,          /* CG did not reach cg_rtol within cg_maxit iterations */
  LH_ETIMEOUT = 8,     /* reserved: no kernel of the library waits on another block */
  LH_EUNSUPPORTED = 9, /* valid but not built (order/dimension/quadrature) */
  LH_ETOOLARGE = 10    /* the mesh does not fit the fixed working memory of
                          lh_force_static */
} lh_status;

typedef enum lh_precision {
  LH_FP64 = 0,  /* every step in double precision */
  LH_MIXED = 1  /* quadrature-point stress and the element force matrix in
                   FP32; the F.1 row sums and F^T.v contractions of its FP32
                   entries accumulated with error-free FP32 transformations
                   (about 2^-48 relative) and widened once to FP64; positions,
                   time integration, CG iterates, residuals and dot products
                   and the energy in FP64.  The FP32 stress leaves out a constant
                   reference pressure whose F.1 vanishes on the box after the wall
                   condition: states must keep the wall nodes on their walls, as
                   every state the integrator makes from lh_init_state does */
} lh_precision;

typedef enum lh_problem_id {
  LH_SEDOV = 1,         /* point blast, Section 6.1.2 */
  LH_TAYLOR_GREEN = 2,  /* Taylor-Green vortex, Section 6.1.3 (2D: with its
                           manufactured energy source) */
  LH_GRESHO = 3,        /* Gresho vortex, Section 6.1.1 */
  LH_UNIFORM = 4,       /* uniform gas at rest (tests) */
  LH_TRIPLE_POINT = 5   /* triple point, Section 6.1.4: two materials in three
                           states, rho0, p and gamma constant per element and
                           decided by the element's initial centre (x <= 1:
                           1, 1, 1.5; x > 1, y <= 1.5: 1, 0.1, 1.4; x > 1,
                           y > 1.5: 1/8, 0.1, 1.5), on the box [0,7] x [0,3]
                           (x [0,1.5]); gamma of lh_phys_desc is not used */
} lh_problem_id;

/* Time integrators of Section 2.2. */
enum {
  LH_RK2AVG = 0,  /* RK2-average, eq:RK2-avg (exact discrete energy balance) */
  LH_RK4 = 1      /* classical RK4 (eq:RK4, eq:RK4coeff) on the combined system
                     f(S) = (-M_V^{-1} F(S).1, M_E^{-1} (F(S)^T v + source), v),
                     every stage at its own state; the estimate is the minimum
                     over the four stages */
};

/* Cartesian box [lo, hi] split into nx x ny (x nz) equal elements. */
typedef struct lh_mesh_desc {
  int32_t dim;              /* 2 or 3 */
  int32_t nx, ny, nz;       /* elements per direction (nz unused in 2D) */
  double lo[3], hi[3];
} lh_mesh_desc;

/* Discretisation: H1 order k (Q_k / Q_{k-1} pair) and Gauss-Legendre points
 * per direction.  Built: dim 2 with k = 1, 2, 3 and dim 3 with k = 1, 2, each
 * with nq = 2k. */
typedef struct lh_disc_desc {
  int32_t order;
  int32_t nq;
} lh_disc_desc;

/* Physics and control constants.  lh_default_phys fills the defaults of
 * Section 2.2.3 (cfl = 0.5, cfl_mu = 2.5, beta1 = 0.85, beta2 = 1.02,
 * gamma_dt = 0.8) and q1 = 0.5, q2 = 2, cg_rtol = 1e-14, cg_maxit = 500,
 * dt_min_frac = 1e-12. */
typedef struct lh_phys_desc {
  int32_t problem;       /* lh_problem_id */
  int32_t visc;          /* artificial viscosity on (1) / off (0) */
  int32_t source;        /* manufactured energy source (Taylor-Green 2D) */
  int32_t cg_maxit;
  double gamma;          /* adiabatic index of eq:EOS */
  double blast_energy;   /* Sedov: total energy deposited in the origin element */
  double e_uniform;      /* LH_UNIFORM: specific internal energy */
  double cfl, cfl_mu;    /* alpha and alpha_mu of eq:adaptive-timestep */
  double beta1, beta2, gamma_dt;  /* step control constants, Section 2.2.3 */
  double q1, q2;         /* linear and quadratic viscosity coefficients */
  double cg_rtol;        /* stop when ||r||_2 <= cg_rtol ||b||_2 */
  double dt_min_frac;    /* dt < dt_min_frac * t_final -> LH_EDTMIN */
  int32_t cg_precond;    /* LH_PRECOND_AUTO (default), LH_PRECOND_TENSOR,
                            LH_PRECOND_TENSOR64, LH_PRECOND_EXACT or LH_PRECOND_JACOBI */
  int32_t direct_launch; /* 0 (default): each step attempt is one CUDA graph launch
                            (the CG iterations a WHILE node inside it); 1: the same
                            kernels launched one by one, with a host poll of the CG
                            between iteration batches (for kernel profilers) */
  int32_t cg_cluster;    /* 0 (default): the whole velocity solve of a small 2D problem
                            (N_V <= 1,500, tensor preconditioner) runs as one launch of a
                            thread-block cluster when the device allows it; 1: whenever it
                            can (any 2D size); -1: never (one kernel per CG phase) */
  int32_t cg_tiles;      /* 0 (default): in 2D, where the band preconditioner's line passes
                            would leave SMs idle, both directions run as one kernel over
                            16 x 16 node tiles, and M p (element apply and node gather) as
                            another over the same tiles: the preconditioner output and
                            M p are bitwise those of the line passes and the element /
                            gather pair, only the CG dot products add their partial sums
                            over another tiling; -1: one kernel per pass and phase */
  int32_t integrator;    /* LH_RK2AVG (default) or LH_RK4; the batched form runs
                            RK2-average only */
} lh_phys_desc;

/* Velocity CG preconditioners.  With rho0 |J0| the same in every element (every
 * problem of Section 6.1 on a Cartesian box), M_V restricted to the free
 * entries of a component is rho0 |J0| times a Kronecker product of assembled
 * 1D mass matrices.  EXACT applies its inverse by FP64 banded Cholesky solves
 * along every node line (the CG stops after one iteration); TENSOR applies the
 * inverses of the 1D matrices truncated to a band, in FP32 (about three
 * iterations); TENSOR64 the same band in FP64 (two iterations); JACOBI the
 * inverse diagonal.  Meshes where rho0 |J0| varies use
 * JACOBI whatever is asked. */
enum { LH_PRECOND_JACOBI = 0, LH_PRECOND_TENSOR = 1, LH_PRECOND_EXACT = 2,
       LH_PRECOND_TENSOR64 = 3,
       LH_PRECOND_AUTO = 4  /* EXACT in 3D, TENSOR in 2D (the faster measured on the
                               3D blast 32^3 and the 2D workloads) */ };

typedef struct lh_layout_info {
  int64_t nv;            /* N_V = dim * nnodes */
  int64_t ne;            /* N_E = nelem * k^dim */
  int64_t nqp;           /* nelem * nq^dim */
  int64_t nelem, nnodes;
  int32_t dim, order, nq;
  int32_t ndof_h1;       /* (k+1)^dim nodes per element */
  int32_t ndof_l2;       /* k^dim energy dofs per element */
  int32_t nqe;           /* nq^dim quadrature points per element */
  int32_t nodes_per_dim[3];
  int32_t precision;     /* lh_precision */
  int64_t n_essential;   /* essential (wall-normal) velocity components */
  int32_t precond_kernels;  /* kernel launches of one lh_precond_apply (0: Jacobi context) */
} lh_layout_info;

typedef struct lh_run_stats {
  int64_t steps;         /* accepted steps */
  int64_t rejects;       /* repeated step attempts (dt >= tau) */
  int64_t cg_iters;      /* CG iterations summed over all solves */
  double t;              /* time reached */
  double dt;             /* next proposed step size */
  double energy0;        /* total energy 1/2 v.M_V.v + 1.M_E.e before the run */
  double energy;         /* ... after the run */
  double wall_ms;        /* time-loop wall clock (CUDA events on the stream) */
} lh_run_stats;

/* Aggregate statistics of a batched run (sums over instances). */
typedef struct lh_batch_stats {
  int64_t steps;           /* accepted steps */
  int64_t rejects;         /* repeated attempts */
  int64_t cg_iters;        /* CG iterations */
  int64_t attempts;        /* step attempts of unfinished instances */
  int64_t instances_done;  /* instances that reached t_final (or max_steps) */
  int64_t dof_updates;     /* sum of (2 N_V + N_E) x accepted steps */
  int64_t graph_launches;  /* attempt graphs launched */
  double wall_ms;          /* time-loop wall clock (CUDA events on the stream) */
} lh_batch_stats;

/* Launch shape of the batched kernels.  threads: 256, 512 or 1024 (2D only)
 * threads per CTA; with one thread per quadrature point, the force and energy
 * tiles hold threads / nq^dim elements and the mass tiles threads /
 * (dim (k+1)^dim); qpt: quadrature points per thread in the force tiles (1,
 * or 2 for 2D: a team of nq^dim / 2 threads per element, twice the elements per
 * tile; 0 = 1).  ctas_per_sm: 0 = as many as fit.  smem_lines: where the
 * node-line solves of the velocity CG run: 2 = every component staged in
 * shared memory and solved together (needs 8 x dim x nodes of the largest
 * instance), 1 = one component at a time (8 x nodes), 0 = in place in device
 * memory. */
typedef struct lh_batch_tuning {
  int32_t threads;
  int32_t ctas_per_sm;
  int32_t smem_lines;
  int32_t qpt;
} lh_batch_tuning;

typedef struct lh_ctx lh_ctx;
typedef struct lh_batch lh_batch;

LH_API void lh_default_phys(lh_phys_desc* phys);
LH_API const char* lh_status_string(lh_status s);

/* Creates a context: validates the descriptors, builds the basis tables and
 * quadrature data of the initial mesh, allocates every work array on the
 * device and leaves the state uninitialised.  precision: lh_precision.
 * stream: cudaStream_t as void*.  Errors: LH_EINVAL, LH_EUNSUPPORTED,
 * LH_ENOMEM, LH_ECUDA.  *out is NULL on failure. */
LH_API lh_status lh_create(const lh_mesh_desc* mesh, const lh_disc_desc* disc,
                    const lh_phys_desc* phys, int32_t precision, void* stream,
                    lh_ctx** out);
/* Frees every device and host resource of the context (NULL is allowed). */
LH_API lh_status lh_destroy(lh_ctx* ctx);
/* Message of the last failing call on this context ("" if none). */
LH_API const char* lh_last_error(const lh_ctx* ctx);
LH_API lh_status lh_layout(const lh_ctx* ctx, lh_layout_info* info);

/* Initial condition of the problem (Section 6.1): x at the H1 nodes of the
 * box, v interpolated at the H1 nodes, e interpolated at the L2 nodes (Sedov:
 * e_0 = E_0 / (rho_0 |K_0|) in the origin element).  Sets t = 0 and marks the
 * step size for estimation by the next step. */
LH_API lh_status lh_init_state(lh_ctx* ctx);
/* Copies the state in (host or device pointers, N_V / N_E / N_V doubles).
 * dt <= 0 asks the next step for a fresh estimate.  With (v, e, x, t, dt)
 * from lh_get_state, the run continues exactly as it would have without the
 * round trip (bit for bit in FP64).  The mixed path also recomputes here its
 * reference pressure, (gamma - 1) times the smallest e of the state given (0
 * if negative), so a resumed mixed run with a positive background pressure
 * rounds its FP32 stress differently and agrees to FP32 rounding. */
LH_API lh_status lh_set_state(lh_ctx* ctx, const double* v, const double* e,
                       const double* x, double t, double dt);
/* Copies the state out (host or device pointers; any may be NULL) and
 * synchronizes.  Reports a pending device error. */
LH_API lh_status lh_get_state(lh_ctx* ctx, double* v, double* e, double* x, double* t,
                       double* dt);

/* One force evaluation on the given state (eq:forceOneforceTv), all device
 * pointers: F1 (N_V) = F.1 with the essential components set to zero;
 * if vtest != NULL, FTv (N_E) = F^T.vtest; dt_est (host, may be NULL) = the
 * minimum over quadrature points of eq:adaptive-timestep (0 if an element is
 * inverted).  Synchronizes when dt_est != NULL. */
LH_API lh_status lh_force(lh_ctx* ctx, const double* v, const double* e,
                   const double* x, const double* vtest, double* F1,
                   double* FTv, double* dt_est);

/* Hyper-reduced evaluation (Section 3.3, eq:rom-hr): the same force restricted
 * to the n listed elements (device int32 ids, each in [0, nelem)).  Outputs
 * are element-local and ordered like the list: F1_local (n x dim x ndof_h1,
 * row [slot][c][i]) and, if vtest != NULL, FTv_local (n x ndof_l2).  No
 * boundary condition is applied to element-local rows.  dt_est as lh_force
 * over the listed elements. */
LH_API lh_status lh_force_sampled(lh_ctx* ctx, const int32_t* elem_ids, int64_t n,
                           const double* v, const double* e, const double* x,
                           const double* vtest, double* F1_local,
                           double* FTv_local, double* dt_est);

/* y = M_V x (device pointers, N_V): the kinematic mass matrix of eq:fom,
 * partially assembled, no boundary condition. */
LH_API lh_status lh_mass_apply_v(lh_ctx* ctx, const double* in, double* out);
/* Solves M_V out = rhs on the non-essential components (essential entries of
 * out are zero) by preconditioned CG with the partially assembled M_V, from a
 * zero guess (momentum equation of eq:fom; preconditioner: cg_precond).  iters / relres (host, may be NULL) return the
 * iteration count and ||r||/||b||; both make the call synchronize.
 * LH_ECG if cg_maxit is reached. */
LH_API lh_status lh_mass_solve_v(lh_ctx* ctx, const double* rhs, double* out,
                          int32_t* iters, double* relres);
/* out = P^{-1} in (device pointers, N_V): one application of the velocity CG's
 * tensor-product preconditioner along every direction, on the non-essential
 * components (essential entries of out are zero): the 1D inverses truncated
 * to a band in FP32 (TENSOR, an approximation of M_V^{-1}; a mixed context on
 * a mesh small enough for the narrow passes keeps each band entry as an FP32
 * pair hi + lo and sums without rounding error) or FP64 (TENSOR64), or the
 * exact inverse by banded Cholesky solves (EXACT).
 * Launches lh_layout_info.precond_kernels kernels on the context's stream.
 * LH_EUNSUPPORTED if the context uses the Jacobi preconditioner. */
LH_API lh_status lh_precond_apply(lh_ctx* ctx, const double* in, double* out);
/* out = M_E^{-1} rhs (device pointers, N_E), block diagonal per element. */
LH_API lh_status lh_mass_solve_e(lh_ctx* ctx, const double* rhs, double* out);
/* Total energy 1/2 v.M_V.v + 1.M_E.e of the context state (host double). */
LH_API lh_status lh_total_energy(lh_ctx* ctx, double* energy);

/* One RK2-average step of size dt on the context state (eq:RK2-avg), without
 * step control (replay of a known step sequence).  tau (host, may be NULL)
 * = min of the estimate over both stages; synchronizes when given. */
LH_API lh_status lh_step_fixed(lh_ctx* ctx, double dt, double* tau);
/* One step attempt under the control of Section 2.2.3; *accepted = 1 if the
 * state advanced, 0 if the attempt was rejected and dt reduced by beta1.
 * t_final bounds the step (the last step is clamped to land on it). */
LH_API lh_status lh_step(lh_ctx* ctx, double t_final, int32_t* accepted, double* t,
                  double* dt);
/* Runs the step control loop to t_final (or max_steps accepted steps) with
 * device-side accept/redo decisions, one CUDA graph launch per attempt.
 * stats (host, may be NULL).  dt_log (device, may be NULL) receives the
 * accepted step sizes in order, at most dt_log_cap of them. */
LH_API lh_status lh_run_to(lh_ctx* ctx, double t_final, int64_t max_steps,
                    lh_run_stats* stats, double* dt_log, int64_t dt_log_cap);

/* F.1 of a state without allocating memory and without a context.  This entry
 * point is a service of the library, not a step of the paper: the paper has no
 * counterpart.  It is for callers that cannot call cudaMalloc (their device
 * memory is owned by a framework pool or budgeted up front, or they cannot
 * afford an allocation inside a latency-critical loop); lh_create would
 * allocate, this does not.
 * Computes what lh_force computes for F1 and dt_est, in FP64: F1 (device, N_V)
 * = F.1 of the state (v, e, x: device pointers, layouts as above) with the
 * essential components set to zero, and dt_est (host, may be NULL) = the same
 * time-step estimate lh_force returns.  rho0 = 1, as in every problem the
 * library builds.
 * Working memory: one file-scope device array of 4 Mi doubles (32 MiB) that
 * every GPU which loads the library holds until the process exits.  A mesh
 * fits when 16 + n_e (1 + dim (k+1)^dim) <= 4194304 doubles (for example
 * 2D Q2 up to 220,000 elements, 3D Q2 up to 51,000); larger meshes return
 * LH_ETOOLARGE before any GPU work.  The first call on a device looks up the
 * array's device address and sets kernel attributes for that device (with the
 * device current); make that first call before any stream capture.
 * Every call shares the array and the array keeps the last call's contents
 * (the estimate and flag slots are reset at the start of each call); calls
 * whose work overlaps on the GPU (different streams, or threads) race on it:
 * order them on one stream.  No cudaMalloc, cudaFree or allocating library
 * routine is called.  Always synchronizes stream: the state checks (inverted
 * element, non-finite value) are read back and reported by this call, whether
 * or not dt_est is given.  Errors: LH_EINVAL / LH_EUNSUPPORTED (descriptors),
 * LH_ETOOLARGE, LH_ECUDA, LH_ETANGLED, LH_ENONFINITE. */
LH_API lh_status lh_force_static(const lh_mesh_desc* mesh, const lh_disc_desc* disc,
                                 const lh_phys_desc* phys, const double* v, const double* e,
                                 const double* x, double* F1, double* dt_est, void* stream);

/* Self-check of the library's FP32 <-> FP64 conversions (a service of the
 * library, not a step of the paper; the FP32 paths convert on the integer
 * pipes because the FP64 pipe of this GPU is narrow): f_out[i] = in[i] rounded
 * to FP32 (nearest, ties to even, as the IEEE cast: results below the normal
 * FP32 range round to the subnormal grid, below half the smallest subnormal to
 * zero), d_out[i] = f_out[i] widened back to FP64 exactly, and (if
 * split_out != NULL) split_out[i] = hi + lo of the two-float split of in[i]
 * used by the FP32 energy accumulations (|in - split_out| <= 2^-48 |in| in
 * the normal range).  Device pointers, n entries, on stream (cudaStream_t as
 * void*).  Errors: LH_EINVAL, LH_ECUDA. */
LH_API lh_status lh_check_conversions(const double* in, int64_t n, float* f_out, double* d_out,
                                      double* split_out, void* stream);

/* ---------------------------------------------------------------------------
 * Hyper-reduced online step of the reduced order model (Section 3): the
 * RK2-average scheme in reduced coordinates (eq:RK2-avg-rom-hr) with the SNS
 * nonlinear-term bases of Section 4.2 (eq:rom-hr-sns: Phi_F = M_V Phi_v with
 * its essential rows zero, as those of F.1, and Phi_G = M_E Phi_e) and DEIM
 * sampling (Section 4.3), under the step control of Section 2.2.3 with the
 * estimate taken over the sampled elements (the lifted state exists only
 * there).  Built on a context of a problem without an energy source, FP64
 * or mixed; the context's force kernel evaluates the sampled elements in its
 * precision (mixed: FP32 stress and F_K, the error-free F.1 and F^T w sums and
 * the FP64 reference-pressure part, as in the full-order step), and the
 * reduced state, projections and updates are FP64.
 * ------------------------------------------------------------------------ */
typedef struct lh_rom lh_rom;
typedef struct lh_rom_info_t {
  int32_t nb_v, nb_e, nb_x;  /* basis sizes */
  int32_t ns_f, ns_g;        /* sampled entries of F.1 and of F^T v */
  int64_t n_elems;           /* sampled elements (every element touching a
                                sampled F.1 node, the element of every sampled
                                F^T v entry) */
  int64_t n_rows_v, n_rows_e;  /* lifted rows (kinematic, thermodynamic) */
} lh_rom_info_t;

/* Creates the reduced model of ctx (no source term): Phi_v (N_V x
 * nb_v), Phi_e (N_E x nb_e), Phi_x (N_V x nb_x) column-major bases and the
 * offsets v_os, e_os, x_os (eq:solrepresentation), all host or device
 * pointers, copied.  ns_f >= nb_v and ns_g >= nb_e sampled entries; samples_f
 * / samples_g (host, distinct row indices of F.1 / F^T v) or NULL to select
 * them by greedy DEIM with over-sampling (basis vector j receives its share of
 * the samples, each at the largest entry of the residual of its least-squares
 * reconstruction by the basis vectors before it; ties to the lowest row).
 * Forms the SNS bases, the least-squares matrices (Z^T Phi)^+ of
 * eq:sol-ls-hyper, the sampled elements and their basis rows, and allocates
 * the reduced state (zero).  Errors: LH_EINVAL (sizes, samples, a
 * rank-deficient sampled basis), LH_EUNSUPPORTED (source term), LH_ENOMEM,
 * LH_ECUDA.  Basis sizes <= 1024, samples <= 6144. */
LH_API lh_status lh_rom_create(lh_ctx* ctx, const double* Phi_v, int32_t nb_v,
                               const double* Phi_e, int32_t nb_e, const double* Phi_x,
                               int32_t nb_x, const double* v_os, const double* e_os,
                               const double* x_os, int32_t ns_f, int32_t ns_g,
                               const int64_t* samples_f, const int64_t* samples_g, lh_rom** out);
LH_API lh_status lh_rom_destroy(lh_rom* rom);
LH_API const char* lh_rom_last_error(const lh_rom* rom);
/* Sizes (info, may be NULL) and the sample rows and sampled elements (host
 * arrays of ns_f, ns_g and n_elems entries, each may be NULL). */
LH_API lh_status lh_rom_info(const lh_rom* rom, lh_rom_info_t* info, int64_t* samples_f,
                             int64_t* samples_g, int32_t* elems);
/* Reduced coordinates in / out (host or device, nb_v / nb_e / nb_x doubles),
 * time and proposed step (dt <= 0: estimate at the next step). */
LH_API lh_status lh_rom_set_state(lh_rom* rom, const double* vhat, const double* ehat,
                                  const double* xhat, double t, double dt);
LH_API lh_status lh_rom_get_state(lh_rom* rom, double* vhat, double* ehat, double* xhat,
                                  double* t, double* dt);
/* The lifted full-order state v_os + Phi_v vhat, ... (device, N_V / N_E / N_V,
 * any may be NULL); synchronizes. */
LH_API lh_status lh_rom_lift(lh_rom* rom, double* v, double* e, double* x);
/* One hyper-reduced RK2-average step of size dt, accepted without control;
 * tau (host, may be NULL) = the estimate over both stages. */
LH_API lh_status lh_rom_step_fixed(lh_rom* rom, double dt, double* tau);
/* The step control loop to t_final (or max_steps accepted steps), one CUDA
 * graph per attempt; stats (host, may be NULL; cg_iters and energies 0). */
LH_API lh_status lh_rom_run_to(lh_rom* rom, double t_final, int64_t max_steps,
                               lh_run_stats* stats);

/* POD basis of a snapshot matrix (Section 4, eq:SVD, eq:energy_criteria).
 * S (device, column-major m x n: n snapshots of m entries), offset (device,
 * m entries, may be NULL): the thin SVD of S - offset 1^T is computed by
 * one-sided Jacobi (parallel round-robin sweeps of column-pair rotations until
 * every pair is orthogonal to sqrt(m) 2^-52 relative, the rounding level of
 * an m-term inner product; columns at 1e-16 of the Frobenius norm count as
 * null space).  Outputs: U (device, m x n,
 * column-major) the left singular vectors in descending singular-value order
 * (zero columns for zero singular values), sigma (device, n) the singular
 * values in that order, *k (host) the smallest basis size whose singular-value
 * sum reaches eps times the total (0 for S = offset), *sweeps (host, may be
 * NULL) the Jacobi sweeps taken.  work: device scratch of at least m n + 2 n +
 * 16 doubles.  n <= 65535.  Work runs on stream (cudaStream_t as void*) and
 * the call synchronizes it once per sweep.  Errors: LH_EINVAL, LH_ECUDA,
 * LH_ECG (60 sweeps without convergence; outputs are still written). */
LH_API lh_status lh_pod(const double* S, int64_t m, int64_t n, const double* offset, double eps,
                        double* U, double* sigma, double* work, int64_t* k, int32_t* sweeps,
                        void* stream);

/* Peak arithmetic-rate probe (a measurement service of the library, not a
 * step of the paper): launches one kernel on stream (cudaStream_t as void*)
 * in which every thread runs eight independent chains of iters fused
 * multiply-adds, FP64 if fp64 != 0, else FP32, over 8 blocks of 256 threads
 * per SM.  sink: device memory of at least (8 x SM count) doubles that the
 * kernel may write (it never does in practice).  *flops (host, may be NULL)
 * = the floating-point operations of the launch (2 per FMA).  The caller
 * times the launch (for example with CUDA events on stream); flops / time is
 * the FP64 or FP32 rate that the library's ALU-bound kernels are quoted
 * against.  Errors: LH_EINVAL (iters < 1 or > 2^40, sink NULL), LH_ECUDA. */
LH_API lh_status lh_peak_probe(int32_t fp64, int64_t iters, void* sink, void* stream,
                               double* flops);

/* The same probe with the chains on the first `lanes` lanes of every warp
 * only (1..32; the other lanes idle), to measure how the pipe time of a warp
 * instruction depends on its active lanes (the paper has no counterpart).
 * *flops counts the active lanes' operations only.  Errors: LH_EINVAL
 * (lanes outside 1..32, or as lh_peak_probe), LH_ECUDA. */
LH_API lh_status lh_peak_probe_lanes(int32_t fp64, int32_t lanes, int64_t iters, void* sink,
                                     void* stream, double* flops);

/* ---------------------------------------------------------------------------
 * Batched form: n independent instances of the time step, each on its own
 * Cartesian box mesh with its own physics (a parameter sweep such as the
 * snapshot runs of the offline stage, Section 4 and Section 6).  Every
 * instance follows exactly the step of a context with the same descriptors:
 * RK2-average (eq:RK2-avg), the step control of Section 2.2.3 with its own
 * dt, the velocity solve by CG on the partially assembled M_V.  The library
 * runs one persistent kernel per RK stage over all instances (one CTA per
 * instance at a time, largest instances first), the two stage kernels of an
 * attempt captured as one CUDA graph.
 *
 * Layout: every state array is the concatenation of the instances' arrays in
 * instance order (offsets from lh_batch_layout); within an instance the
 * layout of lh_layout.  Differences from a context: the mixed path keeps the
 * whole stress in FP32 (no reference-pressure split, exact for problems with
 * zero background pressure such as the point blast); the velocity CG is
 * preconditioned by the exact inverse of M_V (banded Cholesky solves along
 * node lines, FP64), so it stops after one iteration.
 * ------------------------------------------------------------------------ */

/* Creates a batch.  meshes[n] and phys[n]: one descriptor per instance (all
 * of the same dimension); disc: shared order and quadrature.  cg_rtol and
 * cg_maxit are taken from phys[0].  precision: lh_precision for every
 * instance.  stream: cudaStream_t as void* (NULL: the library creates a work
 * stream).  tuning: NULL (or threads == 0) for the default launch shape, to be
 * replaced by lh_batch_autotune; otherwise a fixed shape.  Allocates every
 * array, including per-CTA scratch sized by the largest instance.  Errors:
 * LH_EINVAL, LH_EUNSUPPORTED (also: an instance with 2^31 or more velocity
 * unknowns), LH_ENOMEM, LH_ECUDA.  *out is NULL on failure. */
LH_API lh_status lh_batch_create(int32_t n, const lh_mesh_desc* meshes,
                                 const lh_disc_desc* disc, const lh_phys_desc* phys,
                                 int32_t precision, void* stream,
                                 const lh_batch_tuning* tuning, lh_batch** out);
LH_API lh_status lh_batch_destroy(lh_batch* b);
LH_API const char* lh_batch_last_error(const lh_batch* b);
/* Offsets of each instance in the packed arrays (host, n + 1 entries each:
 * off_v for N_V-sized arrays, off_e for N_E-sized ones; may be NULL) and the
 * per-instance layouts (host, n entries, may be NULL). */
LH_API lh_status lh_batch_layout(const lh_batch* b, int64_t* off_v, int64_t* off_e,
                                 lh_layout_info* info);
/* Initial conditions of every instance (as lh_init_state); t = 0, dt to be
 * estimated. */
LH_API lh_status lh_batch_init_state(lh_batch* b);
/* Copies packed states in (host or device pointers).  t, dt: host arrays of n
 * (NULL: 0); dt <= 0 asks for a fresh estimate. */
LH_API lh_status lh_batch_set_state(lh_batch* b, const double* v, const double* e,
                                    const double* x, const double* t, const double* dt);
/* Copies packed states out (host or device pointers, any may be NULL) and
 * synchronizes. */
LH_API lh_status lh_batch_get_state(lh_batch* b, double* v, double* e, double* x);
/* Per-instance scalars (host arrays of n, any may be NULL): time, next step
 * size, accepted steps, rejected attempts and CG iterations of the last run,
 * and the instance's lh_status (LH_OK, LH_ENONFINITE, LH_ECG, LH_EDTMIN). */
LH_API lh_status lh_batch_query(lh_batch* b, double* t, double* dt, int64_t* steps,
                                int64_t* rejects, int64_t* cg_iters, int32_t* status);
/* Advances every instance to t_final (or max_steps accepted steps each) under
 * its own step control; attempt graphs are launched in growing batches and
 * the host polls the count of finished instances between batches.  stats
 * (host, may be NULL).  Returns the first instance error (LH_ENONFINITE,
 * LH_ECG, LH_EDTMIN; the failed instance stops, the others run on). */
LH_API lh_status lh_batch_run_to(lh_batch* b, double t_final, int64_t max_steps,
                                 lh_batch_stats* stats);
/* One RK2-average step of every instance with the given step sizes (host
 * array of n, each > 0), every attempt accepted: the replay of a recorded dt
 * sequence, as lh_step_fixed. */
LH_API lh_status lh_batch_step_fixed(lh_batch* b, const double* dt, lh_batch_stats* stats);
/* Total energy 1/2 v.M_V.v + 1.M_E.e of every instance (host array of n);
 * synchronizes. */
LH_API lh_status lh_batch_total_energy(lh_batch* b, double* energy);
/* Restricted force of every instance (Section 3.3, eq:rom-hr), as
 * lh_force_sampled: list_off (device, n + 1 int64) delimits each instance's
 * element ids in elem_ids (device int32, ids within the instance).  v, e, x:
 * packed device states (NULL: the batch's current state); vtest: packed
 * device test vectors or NULL.  Outputs (device) in list order:
 * F1_local[list_off[n]][dim][ndof_h1] and, with vtest, FTv_local
 * [list_off[n]][ndof_l2]; dt_est (host, n, may be NULL) = the estimate over
 * each instance's listed elements (0 if one is inverted); synchronizes when
 * dt_est != NULL. */
LH_API lh_status lh_batch_force_sampled(lh_batch* b, const int64_t* list_off,
                                        const int32_t* elem_ids, const double* v,
                                        const double* e, const double* x,
                                        const double* vtest, double* F1_local,
                                        double* FTv_local, double* dt_est);
/* Snapshot capture for the offline stage (Section 4): the solution data of
 * every accepted step of the selected instances, including the intermediate
 * RK stage, are written by the stage kernel into caller-owned device
 * matrices during later lh_batch_run_to / lh_batch_step_fixed calls: for an
 * accepted step, first S^{n+1/2} = (v, e, x) after stage one, then S^{n+1}.
 * ids (host, nsel ascending instance indices; nsel = 0 turns capture off).
 * Layout: column-major matrices of cap columns per selected instance, packed
 * in selection order: the s-th selected instance i owns Sv[ov_s + c N_V(i) +
 * row] and Sx likewise (ov_s = cap x sum of N_V of the earlier selected
 * instances) and Se[oe_s + c N_E(i) + row] (oe_s with N_E), c = 0 .. cap - 1.
 * Raw states are stored (no offset subtracted).  Columns beyond cap are
 * counted but not written.  This call resets every count to zero.  Errors:
 * LH_EINVAL (ids not ascending or out of range, NULL matrices, cap < 1). */
LH_API lh_status lh_batch_snapshots(lh_batch* b, int32_t nsel, const int32_t* ids, int64_t cap,
                                    double* Sv, double* Se, double* Sx);
/* Snapshots taken per instance since the last lh_batch_snapshots (host array
 * of n; 0 for instances not selected); synchronizes. */
LH_API lh_status lh_batch_snapshot_count(lh_batch* b, int64_t* counts);

/* Autotuner (not a step of the paper): times the stage kernel on the current
 * states for every launch shape that fits the device (threads per CTA, CTAs
 * per SM, node-line staging, quadrature points per thread), reps launches
 * each, keeps the fastest and
 * returns it in *chosen (may be NULL).  The states and control blocks are
 * left as they were. */
LH_API lh_status lh_batch_autotune(lh_batch* b, int32_t reps, lh_batch_tuning* chosen);
/* The launch shape in use. */
LH_API lh_status lh_batch_tuning_get(const lh_batch* b, lh_batch_tuning* t);

#ifdef __cplusplus
}
#endif
#endif /* LAGH_H */
