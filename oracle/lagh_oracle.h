/*
 * lagh_oracle.h -- plain FP64 CPU oracle for the full-order Lagrangian hydro
 * step of "Reduced order models for Lagrangian hydrodynamics" (Copeland,
 * Cheung, Huynh, Choi; arXiv 2104.11404), Section 2.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the correctness reference that
 * the CUDA path is compared against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * What it computes (all in IEEE double, single thread, no blocking, no
 * fusion, no sum factorisation):
 *   - the semi-discrete system of eq:fom:  M_V dv/dt = -F.1,
 *     M_E de/dt = F^T.v (+ manufactured source), dx/dt = v;
 *   - F, the generalized force matrix, assembled per element as the dense
 *     block F_K[(i,c), j] = sum_q alpha_q phi_j(q) (sigma_q adj(J_q)^T
 *     grad_ref w_i(q))[c]   (quadrature form of  int_K sigma : grad w_(i,c) phi_j);
 *   - the ideal-gas EOS p = (gamma-1) rho e  (eq:EOS);
 *   - the RK2-average scheme (eq:RK2-avg), the RK4 scheme (eq:RK4) and the
 *     automatic time step control with the estimate of eq:adaptive-timestep.
 *
 * Readings of points the paper leaves to its reference [dobrev2012high] (basis,
 * quadrature, artificial viscosity, h_min, initial dt, problem data) are
 * listed in the header comment of lagh_oracle.c.
 */
#ifndef LAGH_ORACLE_H
#define LAGH_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Problems of Section 6.1 (test problems).  2D Taylor-Green is the 2D analogue
 * of the 3D problem of Section 6.1.3 with its manufactured energy source. */
enum {
  LHO_SEDOV = 1,
  LHO_TAYLOR_GREEN = 2,
  LHO_GRESHO = 3,
  LHO_UNIFORM = 4,  /* test problem: uniform gas at rest (v = 0, e = e_uniform) */
  LHO_TRIPLE_POINT = 5  /* Section 6.1.4: two materials in three states (reading R13) */
};

/* Time integrators of Section 2.2. */
enum {
  LHO_RK2AVG = 0,   /* eq:RK2-avg */
  LHO_RK4 = 1       /* eq:RK4 on the combined system (reading R14) */
};

/* Return codes. */
enum {
  LHO_OK = 0,
  LHO_EINVAL = 1,
  LHO_ETANGLED = 4,   /* |J| <= 0 at a quadrature point */
  LHO_ENONFINITE = 5,
  LHO_EDTMIN = 6,     /* time step collapsed below dt_min_frac * t_final */
  LHO_ECG = 7         /* CG did not reach cg_rtol within cg_maxit */
};

typedef struct {
  int dim;               /* 2 or 3 */
  int nx, ny, nz;        /* elements per direction (nz ignored in 2D) */
  double lo[3], hi[3];   /* Cartesian box */
  int order;             /* k: H1 Q_k for x, v; L2 Q_{k-1} for e */
  int nq;                /* Gauss-Legendre points per direction */
  int problem;           /* LHO_* problem id */
  double gamma;          /* adiabatic index */
  double blast_energy;   /* Sedov: total energy deposited in the origin element */
  double e_uniform;      /* LHO_UNIFORM: specific internal energy */
  int visc;              /* artificial viscosity on/off */
  double cfl, cfl_mu;    /* alpha, alpha_mu of eq:adaptive-timestep */
  double beta1, beta2, gamma_dt;  /* step control constants of Section 2.2.3 */
  double cg_rtol;        /* relative residual ||r||_2/||b||_2 */
  int cg_maxit;
  double dt_min_frac;    /* dt < dt_min_frac * t_final -> LHO_EDTMIN */
  double q1, q2;         /* linear / quadratic viscosity coefficients */
  int source;            /* manufactured energy source on/off (Taylor-Green) */
  int integrator;        /* LHO_RK2AVG (default) or LHO_RK4, used by lho_run */
} lho_config;

typedef struct lho_problem lho_problem;

typedef struct {
  long steps;            /* accepted steps */
  long rejects;          /* repeated (rejected) step attempts */
  long cg_iters;         /* CG iterations summed over all solves */
  double t;              /* time reached */
  double dt;             /* next step size proposed */
  double energy0, energy;/* total energy at start and end */
} lho_stats;

/* Fills cfg with the default constants of Section 2.2.3 (alpha = 0.5,
 * alpha_mu = 2.5, beta1 = 0.85, beta2 = 1.02, gamma = 0.8) and the readings
 * (q1 = 0.5, q2 = 2, CG rtol 1e-14, maxit 500, nq = 2k). */
void lho_default_config(lho_config* cfg);

/* Returns NULL on invalid configuration. */
lho_problem* lho_create(const lho_config* cfg);
void lho_destroy(lho_problem* P);

/* Sizes: N_V = dim * nodes, N_E = elements * k^dim, N_qp = elements * nq^dim. */
void lho_sizes(const lho_problem* P, long* nv, long* ne, long* nqp, long* nelem,
               long* nnodes);
int lho_local_sizes(const lho_problem* P, int* ndof_h1, int* ndof_l2, int* nqe);

/* Initial state (velocity, energy, positions).  Layout: v, x are component
 * major (v[c * nnodes + node]), nodes lexicographic with x fastest; e is
 * element major, lexicographic within the element. */
int lho_init_state(const lho_problem* P, double* v, double* e, double* x);

/* One force evaluation on state (v, e, x).  F1 = F.1 with essential (wall
 * normal) components set to zero; if vtest != NULL, FTv = F^T.vtest (length
 * N_E).  dt_est = min over quadrature points of the estimate of
 * eq:adaptive-timestep.  Any output pointer may be NULL. */
int lho_force(const lho_problem* P, const double* v, const double* e,
              const double* x, const double* vtest, double* F1, double* FTv,
              double* dt_est);

/* Dense element force matrix F_K, row (c * ndof_h1 + i), column j, row major,
 * (dim * ndof_h1) x ndof_l2, before any boundary condition. */
int lho_element_force_matrix(const lho_problem* P, long elem, const double* v,
                             const double* e, const double* x, double* FK);

/* Minimum of the estimate of eq:adaptive-timestep over the quadrature points
 * of the n listed elements (the hyper-reduced step sees only those). */
int lho_estimate_elements(const lho_problem* P, const long* elems, long n, const double* v,
                          const double* e, const double* x, double* tau);

/* Manufactured energy source int rho e_src phi_j (length N_E); zeros if the
 * problem has none. */
int lho_energy_source(const lho_problem* P, const double* x, double* src);

/* Kinematic mass matrix: y = M_V x (full, no boundary conditions). */
int lho_mass_apply_v(const lho_problem* P, const double* in, double* out);
/* Solves M_V out = rhs on the non-essential dofs (essential dofs of out = 0)
 * with Jacobi-preconditioned CG from a zero initial guess. */
int lho_mass_solve_v(const lho_problem* P, const double* rhs, double* out,
                     int* iters, double* relres);
/* Same solve by dense Cholesky of the assembled matrix (small meshes only). */
int lho_mass_solve_v_dense(const lho_problem* P, const double* rhs, double* out);
/* Thermodynamic mass matrix (block diagonal): y = M_E x and out = M_E^{-1} rhs. */
int lho_mass_apply_e(const lho_problem* P, const double* in, double* out);
int lho_mass_solve_e(const lho_problem* P, const double* rhs, double* out);

/* One RK2-average step of size dt (eq:RK2-avg), in place, no step control.
 * tau = min of the estimate over both stages. */
int lho_step(const lho_problem* P, double dt, double* v, double* e, double* x,
             double* tau, long* cg_iters);

/* One RK4 step of size dt (eq:RK4, eq:RK4coeff), in place, no step control.
 * tau = min of the estimate over the four stages. */
int lho_step_rk4(const lho_problem* P, double dt, double* v, double* e, double* x,
                 double* tau, long* cg_iters);

/* Runs the automatic time step control of Section 2.2.3 from time t0 with
 * proposed step *dt (if *dt <= 0 the estimate of the state is used) to
 * t_final, at most max_steps accepted steps.  dt_log (optional, capacity
 * dt_log_cap) receives the accepted step sizes in order. */
int lho_run(const lho_problem* P, double t0, double t_final, long max_steps,
            double* v, double* e, double* x, double* dt, lho_stats* stats,
            double* dt_log, long dt_log_cap);

/* lho_run (RK2-average only) that also collects the snapshots of Section 4:
 * for every accepted step the half-step state S^{n+1/2} and then S^{n+1}, as
 * columns of the column-major matrices Sv (N_V x cap), Se (N_E x cap) and Sx
 * (N_V x cap).  *count = the number of snapshots taken (columns beyond cap
 * are counted but not stored). */
int lho_run_snapshots(const lho_problem* P, double t0, double t_final, long max_steps,
                      double* v, double* e, double* x, double* dt, lho_stats* stats,
                      double* Sv, double* Se, double* Sx, long cap, long* count);

/* Thin SVD of a column-major m x n matrix by one-sided Jacobi, in place (the
 * columns become U Sigma, unsorted; sigma = their norms). */
int lho_svd_jacobi(long m, long n, double* A, double* sigma, double tol, int max_sweeps,
                   int* sweeps);

/* POD basis (eq:SVD, eq:energy_criteria): U (m x n) = left singular vectors
 * of S - offset 1^T in descending singular-value order, sigma (n) the
 * singular values, *k = the smallest basis size whose singular-value sum
 * reaches eps times the total. */
int lho_pod(long m, long n, const double* S, const double* offset, double eps, double* U,
            double* sigma, long* k);

/* Total energy 1/2 v.M_V.v + 1.M_E.e. */
double lho_total_energy(const lho_problem* P, const double* v, const double* e);

/* 1D tables on [0,1] (for tests): Gauss-Lobatto nodes (n points),
 * Gauss-Legendre points and weights (n points), Lagrange basis values and
 * derivatives at a point for given nodes. */
int lho_gauss_lobatto(int n, double* x);
int lho_gauss_legendre(int n, double* x, double* w);
void lho_lagrange(int n, const double* nodes, double t, double* val, double* der);

/* Quadrature-point physics of one point, for closed-form tests.  Inputs are
 * the reference Jacobian J (row c = component, column m = reference
 * direction), the reference velocity gradient, e at the point, rho0|J0| and
 * J0^{-1}.  Outputs: stress sigma (dim x dim), dt estimate, viscosity mu. */
int lho_qpoint(const lho_problem* P, const double* J, const double* gradv_ref,
               double e_q, double rho0detJ0, double* sigma, double* tau,
               double* mu);

/* Symmetric eigen-solver used for the viscosity direction (exposed for tests):
 * smallest eigenvalue and its unit eigenvector of a dim x dim symmetric matrix. */
void lho_sym_min_eig(int dim, const double* A, double* lambda, double* s);

#ifdef __cplusplus
}
#endif
#endif
