/*
 * lagh_oracle.c -- plain FP64 CPU oracle of the full-order Lagrangian hydro
 * step (arXiv 2104.11404, Section 2).  TEST INFRASTRUCTURE ONLY: it exists to
 * check the CUDA library and is loaded only by the tests, the smoke check and
 * the CPU-baseline leg of the benchmark.  It shares no code with the CUDA path.
 *
 * Every quantity is written as its plain definition: basis functions are
 * evaluated directly at every quadrature point (no sum factorisation), the
 * element force matrix F_K is formed densely, and F.1 / F^T.v are its row sums
 * and transposed product.
 *
 * Readings of what the paper leaves to Dobrev, Kolev, Rieben (2012):
 *  R1 Bases.  H1 Q_k: tensor Lagrange polynomials at the k+1 Gauss-Lobatto
 *     nodes of [0,1].  L2 Q_{k-1}: tensor Lagrange polynomials at the k
 *     Gauss-Legendre points of [0,1] (Q_0: the constant 1).
 *  R2 Quadrature.  Tensor Gauss-Legendre with nq points per direction
 *     (nq = 2k by default).
 *  R3 Artificial viscosity (sigma_a of eq:euler).  eps = sym(grad v);
 *     (lambda_min, s) = smallest eigenpair of eps (2D closed form, 3D cyclic
 *     Jacobi, ties -> lowest index).  The point is in compression when
 *     lambda_min < -1e-5 (|eps|_F + c_s / h_min): a compression rate below that
 *     floor is rounding noise of a vanishing strain rate (a z-invariant flow
 *     in 3D, a gas at rest), where the sign alone would switch on the linear
 *     term.  In compression: l_s = l_0 |J J0^{-1} s|,
 *     mu = rho (q2 l_s^2 |lambda_min| + q1 l_s c_s), sigma_a = mu eps;
 *     otherwise mu = 0.  l_0 = |K_0|^{1/d} / k.
 *  R4 h_min of eq:adaptive-timestep is sigma_min(J) / k.
 *  R5 dt_0 is the estimate of the initial state; the last step is clamped to
 *     land on t_final; dt < dt_min_frac * t_final is an error.
 *  R6 Sedov: the origin element holds the constant e_0 = E_0 / (rho_0 |K_0|).
 *  R7 Gresho pressure, middle branch: 9 - 4 ln 0.2 + 12.5 r^2 - 20 r + 4 ln r
 *     (continuous at r = 0.2 and 0.4, in radial balance with v_phi).
 *  R8 2D Taylor-Green: steady manufactured solution; the energy equation
 *     receives int rho e_src phi_j with e_src = v.grad(e) of the exact
 *     solution, evaluated at the current quadrature point positions.
 *  R9 Wall boundary: component c of every H1 node on a face x_c = lo_c or
 *     x_c = hi_c is essential (zero in v, in the acceleration and in F.1).
 *  R10 Initial data: v and x interpolated at the H1 nodes, e interpolated
 *     at the L2 nodes.
 *  R11 Sound speed c_s = sqrt(max(0, gamma (gamma-1) e)).
 *  R12 Step control (Section 2.2.3): a step is redone with beta1 dt when
 *     dt >= tau; after an accepted step dt grows to beta2 dt when
 *     dt <= gamma tau.  tau is the minimum over both RK2-average stages
 *     (over all four stages of RK4).
 *  R13 Triple point (Section 6.1.4): the three states (rho, p, gamma) are
 *     constant in each element, the element's state decided by its initial
 *     centre (x <= 1: rho 1, p 1, gamma 1.5; x > 1, y <= 1.5: rho 1, p 0.1,
 *     gamma 1.4; x > 1, y > 1.5: rho 1/8, p 0.1, gamma 1.5).  On the box
 *     [0,7] x [0,3] (x [0,1.5]) with n_x a multiple of 7 and n_y even the
 *     interfaces lie on element faces and this is the pointwise definition.
 *  R14 RK4 (eq:RK4, eq:RK4coeff) is applied to the combined right-hand side
 *     f(S) = (-M_V^{-1} F(S).1, M_E^{-1} (F(S)^T v + source), v) of eq:fom,
 *     each stage evaluating F, the source and F^T v at its own state.
 */
#include "lagh_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXK 4
#define LHO_PI 3.14159265358979323846
#define MAXQ 8
#define LHO_COMPRESSION_FLOOR 1e-5  /* reading R3 */

struct lho_problem {
  lho_config cfg;
  int dim, k, nq;
  int n[3];    /* elements per direction */
  int nn[3];   /* H1 nodes per direction, n k + 1 */
  long nnodes, nelem, nv, ne, nqp;
  int nd1;     /* (k+1)^dim H1 nodes per element */
  int nd2;     /* k^dim L2 dofs per element */
  int nqe;     /* nq^dim quadrature points per element */
  double h[3]; /* element widths */
  double gll[MAXK + 1];
  double gl2[MAXK];           /* L2 nodes: k Gauss-Legendre points */
  double qx[MAXQ], qw[MAXQ];  /* quadrature points / weights */
  double *alpha;   /* [nqe] reference quadrature weight */
  double *H;       /* [nqe][nd1]  w_i(xi_q) */
  double *dH;      /* [nqe][nd1][dim]  d/dxi_m w_i(xi_q) */
  double *L;       /* [nqe][nd2]  phi_j(xi_q) */
  double *rho0detJ0; /* [nelem][nqe] */
  double J0inv[9];
  double ell0;
  long *conn;      /* [nelem][nd1] global node of local node */
  unsigned char *ess; /* [dim][nnodes] essential flag */
  double *diagM;   /* [nnodes] diagonal of the scalar kinematic mass matrix */
  double *MK;      /* [nelem][nd1][nd1] element scalar kinematic mass matrices */
  double *MEL;     /* [nelem][nd2][nd2] Cholesky factors of the element M_E */
};

/* ------------------------------------------------------------------ 1D -- */

/* Legendre P_n and P_n' on [-1,1] by the three-term recurrence. */
static void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int j = 2; j <= n; ++j) {
    double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1; p1 = p2;
  }
  *p = p1;
  /* P_n' = n (x P_n - P_{n-1}) / (x^2 - 1) */
  *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

int lho_gauss_legendre(int n, double* x, double* w) {
  if (n < 1 || n > MAXQ) return LHO_EINVAL;
  for (int i = 0; i < n; ++i) {
    /* Newton on P_n from the Chebyshev guess; roots in descending order */
    double z = cos(LHO_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    double p, dp;
    legendre(n, z, &p, &dp);
    /* map [-1,1] -> [0,1], ascending */
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp); /* = (2/((1-z^2)P'^2)) / 2 */
  }
  return LHO_OK;
}

int lho_gauss_lobatto(int n, double* x) {
  if (n < 2 || n > MAXK + 1) return LHO_EINVAL;
  int m = n - 1; /* interior nodes are the roots of P_m' */
  x[0] = 0.0;
  x[n - 1] = 1.0;
  for (int i = 1; i < m; ++i) {
    double z = -cos(LHO_PI * i / m);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(m, z, &p, &dp);
      /* P_m'' from the Legendre equation (1-z^2) P'' = 2 z P' - m(m+1) P */
      double d2p = (2.0 * z * dp - m * (m + 1.0) * p) / (1.0 - z * z);
      double dz = dp / d2p;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    x[i] = 0.5 * (z + 1.0);
  }
  return LHO_OK;
}

void lho_lagrange(int n, const double* nodes, double t, double* val, double* der) {
  for (int a = 0; a < n; ++a) {
    double v = 1.0, d = 0.0;
    for (int b = 0; b < n; ++b) {
      if (b == a) continue;
      double den = nodes[a] - nodes[b];
      /* product rule: d(v * (t - x_b)/den) */
      d = d * (t - nodes[b]) / den + v / den;
      v = v * (t - nodes[b]) / den;
    }
    if (val) val[a] = v;
    if (der) der[a] = d;
  }
}

/* ------------------------------------------------------- small matrices -- */

static double det_d(int d, const double* A) {
  if (d == 2) return A[0] * A[3] - A[1] * A[2];
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* adjugate (transpose of the cofactor matrix): adj(A) A = det(A) I */
static void adj_d(int d, const double* A, double* B) {
  if (d == 2) {
    B[0] = A[3]; B[1] = -A[1];
    B[2] = -A[2]; B[3] = A[0];
    return;
  }
  B[0] = A[4] * A[8] - A[5] * A[7];
  B[1] = A[2] * A[7] - A[1] * A[8];
  B[2] = A[1] * A[5] - A[2] * A[4];
  B[3] = A[5] * A[6] - A[3] * A[8];
  B[4] = A[0] * A[8] - A[2] * A[6];
  B[5] = A[2] * A[3] - A[0] * A[5];
  B[6] = A[3] * A[7] - A[4] * A[6];
  B[7] = A[1] * A[6] - A[0] * A[7];
  B[8] = A[0] * A[4] - A[1] * A[3];
}

/* Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix.
 * On return diag(A) holds the eigenvalues, the columns of V the vectors. */
static void jacobi3(double* A, double* V) {
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  static const int PP[3] = {0, 0, 1}, QQ[3] = {1, 2, 2};
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    if (off == 0.0) break;
    for (int r = 0; r < 3; ++r) {
      int p = PP[r], q = QQ[r];
      double apq = A[3 * p + q];
      if (apq == 0.0) continue;
      double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
      double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      /* A <- G^T A G with G the rotation in the (p,q) plane */
      for (int j = 0; j < 3; ++j) {
        double apj = A[3 * p + j], aqj = A[3 * q + j];
        A[3 * p + j] = c * apj - s * aqj;
        A[3 * q + j] = s * apj + c * aqj;
      }
      for (int j = 0; j < 3; ++j) {
        double ajp = A[3 * j + p], ajq = A[3 * j + q];
        A[3 * j + p] = c * ajp - s * ajq;
        A[3 * j + q] = s * ajp + c * ajq;
      }
      for (int j = 0; j < 3; ++j) {
        double vjp = V[3 * j + p], vjq = V[3 * j + q];
        V[3 * j + p] = c * vjp - s * vjq;
        V[3 * j + q] = s * vjp + c * vjq;
      }
    }
  }
}

void lho_sym_min_eig(int dim, const double* A, double* lambda, double* s) {
  if (dim == 2) {
    double a = A[0], b = 0.5 * (A[1] + A[2]), d = A[3];
    double mean = 0.5 * (a + d);
    double r = hypot(0.5 * (a - d), b);
    double lam = mean - r;
    *lambda = lam;
    if (r == 0.0) { s[0] = 1.0; s[1] = 0.0; return; }
    /* two null vectors of A - lam I; keep the longer one */
    double u0 = b, u1 = lam - a;
    double w0 = lam - d, w1 = b;
    double nu = hypot(u0, u1), nw = hypot(w0, w1);
    if (nu >= nw) { s[0] = u0 / nu; s[1] = u1 / nu; }
    else { s[0] = w0 / nw; s[1] = w1 / nw; }
    return;
  }
  double B[9], V[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[3 * i + j] = 0.5 * (A[3 * i + j] + A[3 * j + i]);
  jacobi3(B, V);
  int imin = 0;
  for (int i = 1; i < 3; ++i)
    if (B[4 * i] < B[4 * imin]) imin = i;
  *lambda = B[4 * imin];
  for (int j = 0; j < 3; ++j) s[j] = V[3 * j + imin];
}

/* Smallest singular value of J. */
static double sigma_min(int d, const double* J) {
  if (d == 2) {
    /* sigma_max + sigma_min = |(a+d, c-b)|, sigma_max - sigma_min = |(a-d, b+c)|
     * for J = [[a, b], [c, d]]; then sigma_min = |det J| / sigma_max has no
     * cancellation even when the two singular values are equal. */
    double s1 = hypot(J[0] + J[3], J[2] - J[1]);
    double s2 = hypot(J[0] - J[3], J[1] + J[2]);
    double det = J[0] * J[3] - J[1] * J[2];
    return 2.0 * fabs(det) / (s1 + s2);
  }
  double JtJ[9], V[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int c = 0; c < 3; ++c) acc += J[3 * c + i] * J[3 * c + j];
      JtJ[3 * i + j] = acc;
    }
  jacobi3(JtJ, V);
  double m = JtJ[0];
  if (JtJ[4] < m) m = JtJ[4];
  if (JtJ[8] < m) m = JtJ[8];
  return sqrt(m > 0.0 ? m : 0.0);
}

/* ---------------------------------------------------------- problem data -- */

static double rho0_at(const lho_problem* P, const double* X) {
  (void)P; (void)X;
  return 1.0; /* every problem but the triple point starts at rho = 1 */
}

/* Initial centre of element el. */
static void element_centre(const lho_problem* P, long el, double* Xc) {
  long r = el;
  for (int c = 0; c < P->dim; ++c) {
    int ei = (int)(r % P->n[c]);
    r /= P->n[c];
    Xc[c] = P->cfg.lo[c] + (ei + 0.5) * P->h[c];
  }
}

/* Triple point, reading R13: state of the element with initial centre Xc. */
static void triple_state(const double* Xc, double* rho, double* p, double* gam) {
  int left = Xc[0] <= 1.0, low = Xc[1] <= 1.5;
  *rho = (left || low) ? 1.0 : 0.125;
  *p = left ? 1.0 : 0.1;
  *gam = (left || !low) ? 1.5 : 1.4;
}

/* rho_0 of element el at the initial point X. */
static double rho0_el(const lho_problem* P, long el, const double* X) {
  if (P->cfg.problem == LHO_TRIPLE_POINT) {
    double Xc[3], rho, p, gam;
    element_centre(P, el, Xc);
    triple_state(Xc, &rho, &p, &gam);
    return rho;
  }
  return rho0_at(P, X);
}

/* Adiabatic index of element el (eq:EOS; per material for the triple point). */
static double gamma_el(const lho_problem* P, long el) {
  if (P->cfg.problem == LHO_TRIPLE_POINT) {
    double Xc[3], rho, p, gam;
    element_centre(P, el, Xc);
    triple_state(Xc, &rho, &p, &gam);
    return gam;
  }
  return P->cfg.gamma;
}

/* Gresho (Section 6.1.1) azimuthal speed and pressure, reading R7. */
static double gresho_vphi(double r) {
  if (r < 0.2) return 5.0 * r;
  if (r < 0.4) return 2.0 - 5.0 * r;
  return 0.0;
}
static double gresho_p(double r) {
  if (r < 0.2) return 5.0 + 12.5 * r * r;
  if (r < 0.4) return 9.0 - 4.0 * log(0.2) + 12.5 * r * r - 20.0 * r + 4.0 * log(r);
  return 3.0 + 4.0 * log(2.0);
}

static void init_velocity(const lho_problem* P, const double* X, double* v) {
  int d = P->dim;
  for (int c = 0; c < d; ++c) v[c] = 0.0;
  switch (P->cfg.problem) {
    case LHO_TAYLOR_GREEN:
      if (d == 2) {
        v[0] = sin(LHO_PI * X[0]) * cos(LHO_PI * X[1]);
        v[1] = -cos(LHO_PI * X[0]) * sin(LHO_PI * X[1]);
      } else {
        v[0] = sin(LHO_PI * X[0]) * cos(LHO_PI * X[1]) * cos(LHO_PI * X[2]);
        v[1] = -cos(LHO_PI * X[0]) * sin(LHO_PI * X[1]) * cos(LHO_PI * X[2]);
        v[2] = 0.0;
      }
      break;
    case LHO_GRESHO: {
      double r = hypot(X[0], X[1]);
      if (r > 0.0) {
        double vp = gresho_vphi(r);
        v[0] = -vp * X[1] / r;
        v[1] = vp * X[0] / r;
      }
      break;
    }
    default:
      break;
  }
}

/* pressure of the smooth problems, used for e = p / ((gamma-1) rho) */
static double init_pressure(const lho_problem* P, const double* X) {
  switch (P->cfg.problem) {
    case LHO_TAYLOR_GREEN:
      if (P->dim == 2)
        return 100.0 + (cos(2.0 * LHO_PI * X[0]) + cos(2.0 * LHO_PI * X[1])) / 4.0;
      return 100.0 + ((cos(2.0 * LHO_PI * X[0]) + cos(2.0 * LHO_PI * X[1])) *
                          (cos(2.0 * LHO_PI * X[2]) + 2.0) - 2.0) / 16.0;
    case LHO_GRESHO:
      return gresho_p(hypot(X[0], X[1]));
    default:
      return 0.0;
  }
}

/* 2D Taylor-Green source e_src = v . grad(e) of the steady exact solution
 * with rho = 1: v.grad(p) = (pi/4)(cos 3pi x cos pi y - cos pi x cos 3pi y). */
static double tg_source(const lho_problem* P, const double* X) {
  double g = P->cfg.gamma;
  double vgp = 0.25 * LHO_PI *
               (cos(3.0 * LHO_PI * X[0]) * cos(LHO_PI * X[1]) -
                cos(LHO_PI * X[0]) * cos(3.0 * LHO_PI * X[1]));
  return vgp / (g - 1.0);
}

static int has_source(const lho_problem* P) {
  return P->cfg.source && P->cfg.problem == LHO_TAYLOR_GREEN && P->dim == 2;
}

/* ---------------------------------------------------------------- set-up -- */

static void element_mass_e(const lho_problem* P, long el, double* ME);
static int cholesky(long n, double* A);
void lho_destroy(lho_problem* P);

void lho_default_config(lho_config* c) {
  memset(c, 0, sizeof(*c));
  c->dim = 2;
  c->nx = c->ny = c->nz = 8;
  c->hi[0] = c->hi[1] = c->hi[2] = 1.0;
  c->order = 2;
  c->nq = 4;
  c->problem = LHO_SEDOV;
  c->gamma = 1.4;
  c->blast_energy = 0.25;
  c->e_uniform = 1.0;
  c->visc = 1;
  c->cfl = 0.5;
  c->cfl_mu = 2.5;
  c->beta1 = 0.85;
  c->beta2 = 1.02;
  c->gamma_dt = 0.8;
  c->cg_rtol = 1e-14;
  c->cg_maxit = 500;
  c->dt_min_frac = 1e-12;
  c->q1 = 0.5;
  c->q2 = 2.0;
  c->source = 1;
}

static long node_index(const lho_problem* P, const int* I) {
  long idx = I[P->dim - 1];
  for (int c = P->dim - 2; c >= 0; --c) idx = idx * P->nn[c] + I[c];
  return idx;
}

static void node_coords(const lho_problem* P, long node, double* X) {
  long r = node;
  for (int c = 0; c < P->dim; ++c) {
    int I = (int)(r % P->nn[c]);
    r /= P->nn[c];
    int el = I / P->k, a = I % P->k;
    X[c] = P->cfg.lo[c] + (el + P->gll[a]) * P->h[c];
  }
}

/* multi-index of a lexicographic local index with base b */
static void unflatten(int idx, int b, int d, int* out) {
  for (int c = 0; c < d; ++c) { out[c] = idx % b; idx /= b; }
}

lho_problem* lho_create(const lho_config* cfg) {
  if (cfg->dim != 2 && cfg->dim != 3) return NULL;
  if (cfg->order < 1 || cfg->order > MAXK) return NULL;
  if (cfg->nq < 1 || cfg->nq > MAXQ) return NULL;
  if (cfg->nx < 1 || cfg->ny < 1 || (cfg->dim == 3 && cfg->nz < 1)) return NULL;
  lho_problem* P = (lho_problem*)calloc(1, sizeof(lho_problem));
  P->cfg = *cfg;
  int d = P->dim = cfg->dim;
  int k = P->k = cfg->order;
  int nq = P->nq = cfg->nq;
  P->n[0] = cfg->nx; P->n[1] = cfg->ny; P->n[2] = (d == 3) ? cfg->nz : 1;
  P->nnodes = 1; P->nelem = 1;
  P->nd1 = 1; P->nd2 = 1; P->nqe = 1;
  double vol = 1.0;
  for (int c = 0; c < d; ++c) {
    P->nn[c] = P->n[c] * k + 1;
    P->nnodes *= P->nn[c];
    P->nelem *= P->n[c];
    P->nd1 *= k + 1; P->nd2 *= k; P->nqe *= nq;
    P->h[c] = (cfg->hi[c] - cfg->lo[c]) / P->n[c];
    vol *= P->h[c];
  }
  P->nv = d * P->nnodes;
  P->ne = P->nelem * P->nd2;
  P->nqp = P->nelem * P->nqe;
  lho_gauss_lobatto(k + 1, P->gll);
  if (k >= 1) {
    double w[MAXK];
    lho_gauss_legendre(k, P->gl2, w);
  }
  lho_gauss_legendre(nq, P->qx, P->qw);

  /* tabulate the tensor bases at the quadrature points */
  P->alpha = (double*)malloc(sizeof(double) * P->nqe);
  P->H = (double*)malloc(sizeof(double) * P->nqe * P->nd1);
  P->dH = (double*)malloc(sizeof(double) * P->nqe * P->nd1 * d);
  P->L = (double*)malloc(sizeof(double) * P->nqe * P->nd2);
  for (int q = 0; q < P->nqe; ++q) {
    int qi[3];
    unflatten(q, nq, d, qi);
    double b1[3][MAXK + 1], g1[3][MAXK + 1], l1[3][MAXK];
    P->alpha[q] = 1.0;
    for (int c = 0; c < d; ++c) {
      double t = P->qx[qi[c]];
      lho_lagrange(k + 1, P->gll, t, b1[c], g1[c]);
      lho_lagrange(k, P->gl2, t, l1[c], NULL);
      P->alpha[q] *= P->qw[qi[c]];
    }
    for (int i = 0; i < P->nd1; ++i) {
      int a[3];
      unflatten(i, k + 1, d, a);
      double val = 1.0;
      for (int c = 0; c < d; ++c) val *= b1[c][a[c]];
      P->H[q * P->nd1 + i] = val;
      for (int m = 0; m < d; ++m) {
        double dv = 1.0;
        for (int c = 0; c < d; ++c) dv *= (c == m) ? g1[c][a[c]] : b1[c][a[c]];
        P->dH[(q * P->nd1 + i) * d + m] = dv;
      }
    }
    for (int j = 0; j < P->nd2; ++j) {
      int a[3];
      unflatten(j, k, d, a);
      double val = 1.0;
      for (int c = 0; c < d; ++c) val *= l1[c][a[c]];
      P->L[q * P->nd2 + j] = val;
    }
  }

  /* connectivity */
  P->conn = (long*)malloc(sizeof(long) * P->nelem * P->nd1);
  for (long el = 0; el < P->nelem; ++el) {
    int ei[3] = {0, 0, 0};
    long r = el;
    for (int c = 0; c < d; ++c) { ei[c] = (int)(r % P->n[c]); r /= P->n[c]; }
    for (int i = 0; i < P->nd1; ++i) {
      int a[3], I[3];
      unflatten(i, k + 1, d, a);
      for (int c = 0; c < d; ++c) I[c] = ei[c] * k + a[c];
      P->conn[el * P->nd1 + i] = node_index(P, I);
    }
  }

  /* essential components: wall normal on every face (reading R9) */
  P->ess = (unsigned char*)calloc((size_t)d * P->nnodes, 1);
  for (long nd = 0; nd < P->nnodes; ++nd) {
    long r = nd;
    for (int c = 0; c < d; ++c) {
      int I = (int)(r % P->nn[c]);
      r /= P->nn[c];
      if (I == 0 || I == P->nn[c] - 1) P->ess[c * P->nnodes + nd] = 1;
    }
  }

  /* initial geometry: Cartesian, J0 = diag(h) at every point */
  for (int i = 0; i < 9; ++i) P->J0inv[i] = 0.0;
  for (int c = 0; c < d; ++c) P->J0inv[c * d + c] = 1.0 / P->h[c];
  P->ell0 = pow(vol, 1.0 / d) / k;
  P->rho0detJ0 = (double*)malloc(sizeof(double) * P->nqp);
  for (long el = 0; el < P->nelem; ++el) {
    double xl[3][(MAXK + 1) * (MAXK + 1) * (MAXK + 1)];
    for (int i = 0; i < P->nd1; ++i) {
      double X[3];
      node_coords(P, P->conn[el * P->nd1 + i], X);
      for (int c = 0; c < d; ++c) xl[c][i] = X[c];
    }
    for (int q = 0; q < P->nqe; ++q) {
      double Xq[3] = {0, 0, 0};
      for (int c = 0; c < d; ++c)
        for (int i = 0; i < P->nd1; ++i) Xq[c] += xl[c][i] * P->H[q * P->nd1 + i];
      P->rho0detJ0[el * P->nqe + q] = rho0_el(P, el, Xq) * vol;
    }
  }

  /* element mass matrices: (M_K)_ij = sum_q alpha_q rho0|J0|_q w_i w_j, and
   * the same with the L2 basis for M_E (rho |J| = rho0 |J0| at every point) */
  P->MK = (double*)malloc(sizeof(double) * P->nelem * P->nd1 * P->nd1);
  P->MEL = (double*)malloc(sizeof(double) * P->nelem * P->nd2 * P->nd2);
  P->diagM = (double*)calloc(P->nnodes, sizeof(double));
  for (long el = 0; el < P->nelem; ++el) {
    double* M = P->MK + (size_t)el * P->nd1 * P->nd1;
    for (int i = 0; i < P->nd1; ++i)
      for (int j = 0; j < P->nd1; ++j) {
        double acc = 0.0;
        for (int q = 0; q < P->nqe; ++q)
          acc += P->alpha[q] * P->rho0detJ0[el * P->nqe + q] * P->H[q * P->nd1 + i] *
                 P->H[q * P->nd1 + j];
        M[i * P->nd1 + j] = acc;
      }
    for (int i = 0; i < P->nd1; ++i)
      P->diagM[P->conn[el * P->nd1 + i]] += M[i * P->nd1 + i];
    double* ME = P->MEL + (size_t)el * P->nd2 * P->nd2;
    element_mass_e(P, el, ME);
    if (cholesky(P->nd2, ME)) { lho_destroy(P); return NULL; }
  }
  return P;
}

void lho_destroy(lho_problem* P) {
  if (!P) return;
  free(P->alpha); free(P->H); free(P->dH); free(P->L);
  free(P->rho0detJ0); free(P->conn); free(P->ess); free(P->diagM);
  free(P->MK); free(P->MEL);
  free(P);
}

void lho_sizes(const lho_problem* P, long* nv, long* ne, long* nqp, long* nelem,
               long* nnodes) {
  if (nv) *nv = P->nv;
  if (ne) *ne = P->ne;
  if (nqp) *nqp = P->nqp;
  if (nelem) *nelem = P->nelem;
  if (nnodes) *nnodes = P->nnodes;
}

int lho_local_sizes(const lho_problem* P, int* nd1, int* nd2, int* nqe) {
  if (nd1) *nd1 = P->nd1;
  if (nd2) *nd2 = P->nd2;
  if (nqe) *nqe = P->nqe;
  return LHO_OK;
}

int lho_init_state(const lho_problem* P, double* v, double* e, double* x) {
  int d = P->dim;
  for (long nd = 0; nd < P->nnodes; ++nd) {
    double X[3], V[3];
    node_coords(P, nd, X);
    init_velocity(P, X, V);
    for (int c = 0; c < d; ++c) {
      x[c * P->nnodes + nd] = X[c];
      v[c * P->nnodes + nd] = V[c];
    }
  }
  for (long el = 0; el < P->nelem; ++el) {
    int ei[3] = {0, 0, 0};
    long r = el;
    for (int c = 0; c < d; ++c) { ei[c] = (int)(r % P->n[c]); r /= P->n[c]; }
    for (int j = 0; j < P->nd2; ++j) {
      int a[3];
      unflatten(j, P->k, d, a);
      double X[3] = {0.0, 0.0, 0.0};
      for (int c = 0; c < d; ++c)
        X[c] = P->cfg.lo[c] + (ei[c] + P->gl2[a[c]]) * P->h[c];
      double ev = 0.0;
      switch (P->cfg.problem) {
        case LHO_SEDOV: {
          double vol = 1.0;
          for (int c = 0; c < d; ++c) vol *= P->h[c];
          ev = (el == 0) ? P->cfg.blast_energy / (rho0_at(P, X) * vol) : 0.0;
          break;
        }
        case LHO_UNIFORM:
          ev = P->cfg.e_uniform;
          break;
        case LHO_TRIPLE_POINT: {
          double Xc[3], rho, p, gam;
          element_centre(P, el, Xc);
          triple_state(Xc, &rho, &p, &gam);
          ev = p / ((gam - 1.0) * rho);
          break;
        }
        default:
          ev = init_pressure(P, X) / ((P->cfg.gamma - 1.0) * rho0_at(P, X));
          break;
      }
      e[el * P->nd2 + j] = ev;
    }
  }
  return LHO_OK;
}

/* ------------------------------------------------- quadrature-point physics -- */

static int qpoint_gamma(const lho_problem* P, double gam, const double* J,
                        const double* gradv_ref, double e_q, double rho0detJ0,
                        double* sigma, double* tau, double* mu_out) {
  int d = P->dim;
  double detJ = det_d(d, J);
  if (!(detJ > 0.0)) {
    *tau = 0.0;
    if (mu_out) *mu_out = 0.0;
    return LHO_ETANGLED;
  }
  double rho = rho0detJ0 / detJ;                 /* mass conservation */
  double p = (gam - 1.0) * rho * e_q;            /* eq:EOS */
  double cs2 = gam * (gam - 1.0) * e_q;
  double cs = sqrt(cs2 > 0.0 ? cs2 : 0.0);
  for (int i = 0; i < d * d; ++i) sigma[i] = 0.0;
  for (int c = 0; c < d; ++c) sigma[c * d + c] = -p;
  double hmin = sigma_min(d, J) / P->k;          /* reading R4 */
  double mu = 0.0;
  if (P->cfg.visc) {
    double A[9], gradv[9], eps[9];
    adj_d(d, J, A);
    /* physical gradient: grad v = gradv_ref J^{-1} */
    for (int c = 0; c < d; ++c)
      for (int n = 0; n < d; ++n) {
        double acc = 0.0;
        for (int m = 0; m < d; ++m) acc += gradv_ref[c * d + m] * A[m * d + n];
        gradv[c * d + n] = acc / detJ;
      }
    for (int c = 0; c < d; ++c)
      for (int n = 0; n < d; ++n)
        eps[c * d + n] = 0.5 * (gradv[c * d + n] + gradv[n * d + c]);
    double lam, s[3];
    lho_sym_min_eig(d, eps, &lam, s);
    double frob = 0.0;
    for (int i = 0; i < d * d; ++i) frob += eps[i] * eps[i];
    frob = sqrt(frob);
    if (lam < -LHO_COMPRESSION_FLOOR * (frob + cs / hmin)) {
      /* l_s = l_0 |J J0^{-1} s| */
      double JJ0[9], ds[3];
      for (int c = 0; c < d; ++c)
        for (int n = 0; n < d; ++n) {
          double acc = 0.0;
          for (int m = 0; m < d; ++m) acc += J[c * d + m] * P->J0inv[m * d + n];
          JJ0[c * d + n] = acc;
        }
      double nrm2 = 0.0;
      for (int c = 0; c < d; ++c) {
        ds[c] = 0.0;
        for (int n = 0; n < d; ++n) ds[c] += JJ0[c * d + n] * s[n];
        nrm2 += ds[c] * ds[c];
      }
      double ell = P->ell0 * sqrt(nrm2);
      mu = rho * (P->cfg.q2 * ell * ell * fabs(lam) + P->cfg.q1 * ell * cs);
      for (int i = 0; i < d * d; ++i) sigma[i] += mu * eps[i];
    }
  }
  double inv = cs / hmin + P->cfg.cfl_mu * mu / (rho * hmin * hmin);
  *tau = (inv > 0.0) ? P->cfg.cfl / inv : INFINITY;
  if (mu_out) *mu_out = mu;
  return LHO_OK;
}

int lho_qpoint(const lho_problem* P, const double* J, const double* gradv_ref,
               double e_q, double rho0detJ0, double* sigma, double* tau,
               double* mu_out) {
  return qpoint_gamma(P, P->cfg.gamma, J, gradv_ref, e_q, rho0detJ0, sigma, tau, mu_out);
}

/* ------------------------------------------------------------------ force -- */

/* Dense F_K of one element; returns the minimum estimate over its points. */
static int element_force(const lho_problem* P, long el, const double* v,
                         const double* e, const double* x, double* FK,
                         double* tau_min) {
  int d = P->dim, nd1 = P->nd1, nd2 = P->nd2;
  double xl[3][125], vl[3][125], el2[64];
  for (int i = 0; i < nd1; ++i) {
    long g = P->conn[el * nd1 + i];
    for (int c = 0; c < d; ++c) {
      xl[c][i] = x[c * P->nnodes + g];
      vl[c][i] = v[c * P->nnodes + g];
    }
  }
  for (int j = 0; j < nd2; ++j) el2[j] = e[el * nd2 + j];
  for (int r = 0; r < d * nd1 * nd2; ++r) FK[r] = 0.0;
  int status = LHO_OK;
  double tmin = INFINITY;
  const double gam = gamma_el(P, el);
  for (int q = 0; q < P->nqe; ++q) {
    const double* dh = P->dH + (size_t)q * nd1 * d;
    double J[9], Gv[9];
    for (int c = 0; c < d; ++c)
      for (int m = 0; m < d; ++m) {
        double aj = 0.0, av = 0.0;
        for (int i = 0; i < nd1; ++i) {
          aj += xl[c][i] * dh[i * d + m];
          av += vl[c][i] * dh[i * d + m];
        }
        J[c * d + m] = aj;
        Gv[c * d + m] = av;
      }
    double eq = 0.0;
    for (int j = 0; j < nd2; ++j) eq += el2[j] * P->L[q * nd2 + j];
    double sigma[9], tau;
    int st = qpoint_gamma(P, gam, J, Gv, eq, P->rho0detJ0[el * P->nqe + q], sigma, &tau, NULL);
    if (st != LHO_OK) { status = st; tmin = 0.0; continue; }
    if (tau < tmin) tmin = tau;
    /* D = alpha_q sigma adj(J)^T */
    double A[9], D[9];
    adj_d(d, J, A);
    for (int c = 0; c < d; ++c)
      for (int m = 0; m < d; ++m) {
        double acc = 0.0;
        for (int n = 0; n < d; ++n) acc += sigma[c * d + n] * A[m * d + n];
        D[c * d + m] = P->alpha[q] * acc;
      }
    for (int c = 0; c < d; ++c)
      for (int i = 0; i < nd1; ++i) {
        double f = 0.0;
        for (int m = 0; m < d; ++m) f += D[c * d + m] * dh[i * d + m];
        for (int j = 0; j < nd2; ++j)
          FK[(c * nd1 + i) * nd2 + j] += f * P->L[q * nd2 + j];
      }
  }
  *tau_min = tmin;
  return status;
}

int lho_element_force_matrix(const lho_problem* P, long elem, const double* v,
                             const double* e, const double* x, double* FK) {
  if (elem < 0 || elem >= P->nelem) return LHO_EINVAL;
  double tau;
  return element_force(P, elem, v, e, x, FK, &tau);
}

int lho_estimate_elements(const lho_problem* P, const long* elems, long n, const double* v,
                          const double* e, const double* x, double* tau) {
  size_t blk = (size_t)P->dim * P->nd1 * P->nd2;
  double* FK = (double*)malloc(sizeof(double) * blk);
  int status = LHO_OK;
  double tmin = INFINITY;
  for (long s = 0; s < n; ++s) {
    if (elems[s] < 0 || elems[s] >= P->nelem) { status = LHO_EINVAL; break; }
    double t;
    int st = element_force(P, elems[s], v, e, x, FK, &t);
    if (st != LHO_OK) status = st;
    if (t < tmin) tmin = t;
  }
  free(FK);
  *tau = tmin;
  return status;
}

/* All element matrices of a state; returns the minimum estimate. */
static int all_element_forces(const lho_problem* P, const double* v, const double* e,
                              const double* x, double* FKall, double* tau) {
  int status = LHO_OK;
  double tmin = INFINITY;
  size_t blk = (size_t)P->dim * P->nd1 * P->nd2;
  for (long el = 0; el < P->nelem; ++el) {
    double t;
    int st = element_force(P, el, v, e, x, FKall + el * blk, &t);
    if (st != LHO_OK) status = st;
    if (t < tmin) tmin = t;
  }
  *tau = tmin;
  return status;
}

/* F.1 = sum_j F_K[:, j], assembled, essential components zeroed. */
static void assemble_F1(const lho_problem* P, const double* FKall, double* F1) {
  int d = P->dim, nd1 = P->nd1, nd2 = P->nd2;
  size_t blk = (size_t)d * nd1 * nd2;
  for (long i = 0; i < P->nv; ++i) F1[i] = 0.0;
  for (long el = 0; el < P->nelem; ++el) {
    const double* FK = FKall + el * blk;
    for (int c = 0; c < d; ++c)
      for (int i = 0; i < nd1; ++i) {
        double acc = 0.0;
        for (int j = 0; j < nd2; ++j) acc += FK[(c * nd1 + i) * nd2 + j];
        F1[c * P->nnodes + P->conn[el * nd1 + i]] += acc;
      }
  }
  for (long i = 0; i < P->nv; ++i)
    if (P->ess[i]) F1[i] = 0.0;
}

/* F^T.w, element-local (L2 is discontinuous). */
static void apply_FT(const lho_problem* P, const double* FKall, const double* w,
                     double* FTw) {
  int d = P->dim, nd1 = P->nd1, nd2 = P->nd2;
  size_t blk = (size_t)d * nd1 * nd2;
  for (long el = 0; el < P->nelem; ++el) {
    const double* FK = FKall + el * blk;
    for (int j = 0; j < nd2; ++j) {
      double acc = 0.0;
      for (int c = 0; c < d; ++c)
        for (int i = 0; i < nd1; ++i)
          acc += FK[(c * nd1 + i) * nd2 + j] * w[c * P->nnodes + P->conn[el * nd1 + i]];
      FTw[el * nd2 + j] = acc;
    }
  }
}

int lho_force(const lho_problem* P, const double* v, const double* e,
              const double* x, const double* vtest, double* F1, double* FTv,
              double* dt_est) {
  size_t blk = (size_t)P->dim * P->nd1 * P->nd2;
  double* FKall = (double*)malloc(sizeof(double) * blk * P->nelem);
  double tau;
  int st = all_element_forces(P, v, e, x, FKall, &tau);
  if (F1) assemble_F1(P, FKall, F1);
  if (FTv && vtest) apply_FT(P, FKall, vtest, FTv);
  if (dt_est) *dt_est = tau;
  free(FKall);
  return st;
}

int lho_energy_source(const lho_problem* P, const double* x, double* src) {
  int d = P->dim, nd1 = P->nd1, nd2 = P->nd2;
  for (long i = 0; i < P->ne; ++i) src[i] = 0.0;
  if (!has_source(P)) return LHO_OK;
  for (long el = 0; el < P->nelem; ++el)
    for (int q = 0; q < P->nqe; ++q) {
      double Xq[3] = {0, 0, 0};
      for (int c = 0; c < d; ++c)
        for (int i = 0; i < nd1; ++i)
          Xq[c] += x[c * P->nnodes + P->conn[el * nd1 + i]] * P->H[q * nd1 + i];
      double w = P->alpha[q] * P->rho0detJ0[el * P->nqe + q] * tg_source(P, Xq);
      for (int j = 0; j < nd2; ++j) src[el * nd2 + j] += w * P->L[q * nd2 + j];
    }
  return LHO_OK;
}

/* ---------------------------------------------------------- mass matrices -- */

/* scalar kinematic mass on one component: out = M_s in = sum_K P_K^T M_K P_K in */
static void mass_apply_scalar(const lho_problem* P, const double* in, double* out) {
  int nd1 = P->nd1;
  for (long i = 0; i < P->nnodes; ++i) out[i] = 0.0;
  for (long el = 0; el < P->nelem; ++el) {
    const long* cn = P->conn + el * nd1;
    const double* M = P->MK + (size_t)el * nd1 * nd1;
    for (int i = 0; i < nd1; ++i) {
      double acc = 0.0;
      for (int j = 0; j < nd1; ++j) acc += M[i * nd1 + j] * in[cn[j]];
      out[cn[i]] += acc;
    }
  }
}

int lho_mass_apply_v(const lho_problem* P, const double* in, double* out) {
  for (int c = 0; c < P->dim; ++c)
    mass_apply_scalar(P, in + c * P->nnodes, out + c * P->nnodes);
  return LHO_OK;
}

static double dot(long n, const double* a, const double* b) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int lho_mass_solve_v(const lho_problem* P, const double* rhs, double* out,
                     int* iters, double* relres) {
  long nn = P->nnodes;
  double* r = (double*)malloc(sizeof(double) * nn);
  double* z = (double*)malloc(sizeof(double) * nn);
  double* p = (double*)malloc(sizeof(double) * nn);
  double* Ap = (double*)malloc(sizeof(double) * nn);
  int status = LHO_OK, maxits = 0;
  double worst = 0.0;
  for (int c = 0; c < P->dim; ++c) {
    const unsigned char* ess = P->ess + c * nn;
    const double* b = rhs + c * nn;
    double* xs = out + c * nn;
    for (long i = 0; i < nn; ++i) {
      xs[i] = 0.0;
      r[i] = ess[i] ? 0.0 : b[i];
      z[i] = r[i] / P->diagM[i];
      p[i] = z[i];
    }
    double bb = dot(nn, r, r);
    double rz = dot(nn, r, z);
    int it = 0;
    double rr = bb;
    if (bb > 0.0) {
      int conv = 0;
      for (it = 1; it <= P->cfg.cg_maxit; ++it) {
        mass_apply_scalar(P, p, Ap);
        for (long i = 0; i < nn; ++i)
          if (ess[i]) Ap[i] = 0.0;
        double alpha = rz / dot(nn, p, Ap);
        for (long i = 0; i < nn; ++i) {
          xs[i] += alpha * p[i];
          r[i] -= alpha * Ap[i];
        }
        rr = dot(nn, r, r);
        if (sqrt(rr) <= P->cfg.cg_rtol * sqrt(bb)) { conv = 1; break; }
        for (long i = 0; i < nn; ++i) z[i] = r[i] / P->diagM[i];
        double rz_new = dot(nn, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (long i = 0; i < nn; ++i) p[i] = z[i] + beta * p[i];
      }
      if (!conv) { status = LHO_ECG; it = P->cfg.cg_maxit; }
      double rel = sqrt(rr / bb);
      if (rel > worst) worst = rel;
    }
    if (it > maxits) maxits = it;
  }
  if (iters) *iters = maxits;
  if (relres) *relres = worst;
  free(r); free(z); free(p); free(Ap);
  return status;
}

/* dense Cholesky A = L L^T in place (lower), returns 0 on success */
static int cholesky(long n, double* A) {
  for (long j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (long k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0.0)) return 1;
    A[j * n + j] = sqrt(s);
    for (long i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (long k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / A[j * n + j];
    }
  }
  return 0;
}

static void cholesky_solve(long n, const double* Lf, double* b) {
  for (long i = 0; i < n; ++i) {
    double t = b[i];
    for (long k = 0; k < i; ++k) t -= Lf[i * n + k] * b[k];
    b[i] = t / Lf[i * n + i];
  }
  for (long i = n - 1; i >= 0; --i) {
    double t = b[i];
    for (long k = i + 1; k < n; ++k) t -= Lf[k * n + i] * b[k];
    b[i] = t / Lf[i * n + i];
  }
}

int lho_mass_solve_v_dense(const lho_problem* P, const double* rhs, double* out) {
  long nn = P->nnodes;
  if (nn > 4000) return LHO_EINVAL;
  double* M = (double*)calloc((size_t)nn * nn, sizeof(double));
  double* unit = (double*)calloc(nn, sizeof(double));
  double* col = (double*)malloc(sizeof(double) * nn);
  for (long j = 0; j < nn; ++j) {
    unit[j] = 1.0;
    mass_apply_scalar(P, unit, col);
    unit[j] = 0.0;
    for (long i = 0; i < nn; ++i) M[i * nn + j] = col[i];
  }
  long* map = (long*)malloc(sizeof(long) * nn);
  double* A = (double*)malloc(sizeof(double) * (size_t)nn * nn);
  double* b = (double*)malloc(sizeof(double) * nn);
  int status = LHO_OK;
  for (int c = 0; c < P->dim; ++c) {
    const unsigned char* ess = P->ess + c * nn;
    long m = 0;
    for (long i = 0; i < nn; ++i)
      if (!ess[i]) map[m++] = i;
    for (long i = 0; i < m; ++i)
      for (long j = 0; j < m; ++j) A[i * m + j] = M[map[i] * nn + map[j]];
    if (cholesky(m, A)) { status = LHO_EINVAL; break; }
    for (long i = 0; i < m; ++i) b[i] = rhs[c * nn + map[i]];
    cholesky_solve(m, A, b);
    for (long i = 0; i < nn; ++i) out[c * nn + i] = 0.0;
    for (long i = 0; i < m; ++i) out[c * nn + map[i]] = b[i];
  }
  free(M); free(unit); free(col); free(map); free(A); free(b);
  return status;
}

static void element_mass_e(const lho_problem* P, long el, double* ME) {
  int nd2 = P->nd2;
  for (int i = 0; i < nd2; ++i)
    for (int j = 0; j < nd2; ++j) {
      double acc = 0.0;
      for (int q = 0; q < P->nqe; ++q)
        acc += P->alpha[q] * P->rho0detJ0[el * P->nqe + q] * P->L[q * nd2 + i] *
               P->L[q * nd2 + j];
      ME[i * nd2 + j] = acc;
    }
}

int lho_mass_apply_e(const lho_problem* P, const double* in, double* out) {
  int nd2 = P->nd2;
  double ME[64 * 64];
  for (long el = 0; el < P->nelem; ++el) {
    element_mass_e(P, el, ME);
    for (int i = 0; i < nd2; ++i) {
      double acc = 0.0;
      for (int j = 0; j < nd2; ++j) acc += ME[i * nd2 + j] * in[el * nd2 + j];
      out[el * nd2 + i] = acc;
    }
  }
  return LHO_OK;
}

int lho_mass_solve_e(const lho_problem* P, const double* rhs, double* out) {
  int nd2 = P->nd2;
  double b[64];
  for (long el = 0; el < P->nelem; ++el) {
    for (int i = 0; i < nd2; ++i) b[i] = rhs[el * nd2 + i];
    cholesky_solve(nd2, P->MEL + (size_t)el * nd2 * nd2, b);
    for (int i = 0; i < nd2; ++i) out[el * nd2 + i] = b[i];
  }
  return LHO_OK;
}

double lho_total_energy(const lho_problem* P, const double* v, const double* e) {
  double* Mv = (double*)malloc(sizeof(double) * P->nv);
  double* Me = (double*)malloc(sizeof(double) * P->ne);
  lho_mass_apply_v(P, v, Mv);
  lho_mass_apply_e(P, e, Me);
  double ke = 0.5 * dot(P->nv, v, Mv);
  double ie = 0.0;
  for (long i = 0; i < P->ne; ++i) ie += Me[i];
  free(Mv); free(Me);
  return ke + ie;
}

/* ---------------------------------------------------------- RK2-average -- */

static int all_finite(long n, const double* a) {
  for (long i = 0; i < n; ++i)
    if (!isfinite(a[i])) return 0;
  return 1;
}

/* One RK2-average step; if vh != NULL the half-step state S^{n+1/2} is copied
 * to (vh, eh, xh). */
static int step_rk2avg(const lho_problem* P, double dt, double* v, double* e, double* x,
                       double* tau_out, long* cg_iters, double* vh, double* eh, double* xh) {
  long nv = P->nv, ne = P->ne;
  size_t blk = (size_t)P->dim * P->nd1 * P->nd2;
  double* FK = (double*)malloc(sizeof(double) * blk * P->nelem);
  double* v0 = (double*)malloc(sizeof(double) * nv);
  double* x0 = (double*)malloc(sizeof(double) * nv);
  double* e0 = (double*)malloc(sizeof(double) * ne);
  double* F1 = (double*)malloc(sizeof(double) * nv);
  double* a = (double*)malloc(sizeof(double) * nv);
  double* vbar = (double*)malloc(sizeof(double) * nv);
  double* g = (double*)malloc(sizeof(double) * ne);
  double* src = (double*)malloc(sizeof(double) * ne);
  double* de = (double*)malloc(sizeof(double) * ne);
  memcpy(v0, v, sizeof(double) * nv);
  memcpy(x0, x, sizeof(double) * nv);
  memcpy(e0, e, sizeof(double) * ne);
  int st = LHO_OK, its;
  long total_its = 0;
  double tau1, tau2;

  /* stage 1: forces of S^n */
  int s1 = all_element_forces(P, v0, e0, x0, FK, &tau1);
  assemble_F1(P, FK, F1);
  for (long i = 0; i < nv; ++i) F1[i] = -F1[i];
  int cs = lho_mass_solve_v(P, F1, a, &its, NULL);   /* a = -M_V^{-1} F.1 */
  total_its += its;
  for (long i = 0; i < nv; ++i) v[i] = v0[i] + 0.5 * dt * a[i];      /* v^{n+1/2} */
  apply_FT(P, FK, v, g);                                             /* F^T v^{n+1/2} */
  lho_energy_source(P, x0, src);
  for (long i = 0; i < ne; ++i) g[i] += src[i];
  lho_mass_solve_e(P, g, de);
  for (long i = 0; i < ne; ++i) e[i] = e0[i] + 0.5 * dt * de[i];     /* e^{n+1/2} */
  for (long i = 0; i < nv; ++i) x[i] = x0[i] + 0.5 * dt * v[i];      /* x^{n+1/2} */
  if (vh) {
    memcpy(vh, v, sizeof(double) * nv);
    memcpy(eh, e, sizeof(double) * ne);
    memcpy(xh, x, sizeof(double) * nv);
  }

  /* stage 2: forces of S^{n+1/2} */
  int s2 = all_element_forces(P, v, e, x, FK, &tau2);
  assemble_F1(P, FK, F1);
  for (long i = 0; i < nv; ++i) F1[i] = -F1[i];
  int cs2 = lho_mass_solve_v(P, F1, a, &its, NULL);
  total_its += its;
  lho_energy_source(P, x, src);
  for (long i = 0; i < nv; ++i) {
    double v1 = v0[i] + dt * a[i];                                   /* v^{n+1} */
    vbar[i] = 0.5 * (v0[i] + v1);
    v[i] = v1;
  }
  apply_FT(P, FK, vbar, g);                                          /* F^T vbar */
  for (long i = 0; i < ne; ++i) g[i] += src[i];
  lho_mass_solve_e(P, g, de);
  for (long i = 0; i < ne; ++i) e[i] = e0[i] + dt * de[i];
  for (long i = 0; i < nv; ++i) x[i] = x0[i] + dt * vbar[i];

  *tau_out = tau1 < tau2 ? tau1 : tau2;
  if (cg_iters) *cg_iters = total_its;
  if (s1 != LHO_OK) st = s1;
  else if (s2 != LHO_OK) st = s2;
  else if (cs != LHO_OK) st = cs;
  else if (cs2 != LHO_OK) st = cs2;
  else if (!all_finite(nv, v) || !all_finite(ne, e) || !all_finite(nv, x)) st = LHO_ENONFINITE;
  free(FK); free(v0); free(x0); free(e0); free(F1); free(a); free(vbar);
  free(g); free(src); free(de);
  return st;
}

int lho_step(const lho_problem* P, double dt, double* v, double* e, double* x,
             double* tau_out, long* cg_iters) {
  return step_rk2avg(P, dt, v, e, x, tau_out, cg_iters, NULL, NULL, NULL);
}

/* ----------------------------------------------------------------- RK4 -- */

/* Right-hand side f(S) of eq:fom at the state (v, e, x), reading R14:
 * dv = -M_V^{-1} F.1, de = M_E^{-1} (F^T v + source(x)), dx = v. */
static int rate(const lho_problem* P, const double* v, const double* e, const double* x,
                double* FK, double* F1, double* g, double* src, double* dv, double* de,
                double* tau, long* its_total) {
  long nv = P->nv, ne = P->ne;
  int its;
  int s = all_element_forces(P, v, e, x, FK, tau);
  assemble_F1(P, FK, F1);
  for (long i = 0; i < nv; ++i) F1[i] = -F1[i];
  int cs = lho_mass_solve_v(P, F1, dv, &its, NULL);
  *its_total += its;
  apply_FT(P, FK, v, g);
  lho_energy_source(P, x, src);
  for (long i = 0; i < ne; ++i) g[i] += src[i];
  lho_mass_solve_e(P, g, de);
  return s != LHO_OK ? s : cs;
}

int lho_step_rk4(const lho_problem* P, double dt, double* v, double* e, double* x,
                 double* tau_out, long* cg_iters) {
  long nv = P->nv, ne = P->ne;
  size_t blk = (size_t)P->dim * P->nd1 * P->nd2;
  double* FK = (double*)malloc(sizeof(double) * blk * P->nelem);
  double* F1 = (double*)malloc(sizeof(double) * nv);
  double* g = (double*)malloc(sizeof(double) * ne);
  double* src = (double*)malloc(sizeof(double) * ne);
  double* kv[4]; double* ke[4]; double* kx[4];
  for (int s = 0; s < 4; ++s) {
    kv[s] = (double*)malloc(sizeof(double) * nv);
    kx[s] = (double*)malloc(sizeof(double) * nv);
    ke[s] = (double*)malloc(sizeof(double) * ne);
  }
  double* vs = (double*)malloc(sizeof(double) * nv);
  double* es = (double*)malloc(sizeof(double) * ne);
  double* xs = (double*)malloc(sizeof(double) * nv);
  /* stage s is evaluated at S^n + c_s dt k_{s-1} (eq:RK4coeff) */
  const double c[4] = {0.0, 0.5, 0.5, 1.0};
  int st = LHO_OK;
  long its = 0;
  double tau = INFINITY;
  for (int s = 0; s < 4; ++s) {
    for (long i = 0; i < nv; ++i) {
      vs[i] = s == 0 ? v[i] : v[i] + c[s] * dt * kv[s - 1][i];
      xs[i] = s == 0 ? x[i] : x[i] + c[s] * dt * kx[s - 1][i];
    }
    for (long i = 0; i < ne; ++i) es[i] = s == 0 ? e[i] : e[i] + c[s] * dt * ke[s - 1][i];
    double ts;
    int r = rate(P, vs, es, xs, FK, F1, g, src, kv[s], ke[s], &ts, &its);
    for (long i = 0; i < nv; ++i) kx[s][i] = vs[i];
    if (ts < tau) tau = ts;
    if (r != LHO_OK && st == LHO_OK) st = r;
  }
  /* S^{n+1} = S^n + dt/6 (k1 + 2 k2 + 2 k3 + k4)  (eq:RK4) */
  for (long i = 0; i < nv; ++i) {
    v[i] = v[i] + dt / 6.0 * (kv[0][i] + 2.0 * kv[1][i] + 2.0 * kv[2][i] + kv[3][i]);
    x[i] = x[i] + dt / 6.0 * (kx[0][i] + 2.0 * kx[1][i] + 2.0 * kx[2][i] + kx[3][i]);
  }
  for (long i = 0; i < ne; ++i)
    e[i] = e[i] + dt / 6.0 * (ke[0][i] + 2.0 * ke[1][i] + 2.0 * ke[2][i] + ke[3][i]);
  *tau_out = tau;
  if (cg_iters) *cg_iters = its;
  if (st == LHO_OK && (!all_finite(nv, v) || !all_finite(ne, e) || !all_finite(nv, x)))
    st = LHO_ENONFINITE;
  for (int s = 0; s < 4; ++s) { free(kv[s]); free(kx[s]); free(ke[s]); }
  free(FK); free(F1); free(g); free(src); free(vs); free(es); free(xs);
  return st;
}

/* Snapshot buffers of a run (Section 4): column-major matrices with cap
 * columns of N_V (v, x) or N_E (e) entries. */
typedef struct {
  double *Sv, *Se, *Sx;
  long cap, count;
} snapshots;

static void snap_put(const lho_problem* P, snapshots* S, const double* v, const double* e,
                     const double* x) {
  if (S->count >= S->cap) { S->count++; return; }
  long c = S->count++;
  memcpy(S->Sv + c * P->nv, v, sizeof(double) * P->nv);
  memcpy(S->Se + c * P->ne, e, sizeof(double) * P->ne);
  memcpy(S->Sx + c * P->nv, x, sizeof(double) * P->nv);
}

static int run_impl(const lho_problem* P, double t0, double t_final, long max_steps,
                    double* v, double* e, double* x, double* dt_io, lho_stats* stats,
                    double* dt_log, long dt_log_cap, snapshots* snap) {
  long nv = P->nv, ne = P->ne;
  double* vs = (double*)malloc(sizeof(double) * nv);
  double* xs = (double*)malloc(sizeof(double) * nv);
  double* es = (double*)malloc(sizeof(double) * ne);
  double *vh = NULL, *eh = NULL, *xh = NULL;
  if (snap) {
    vh = (double*)malloc(sizeof(double) * nv);
    xh = (double*)malloc(sizeof(double) * nv);
    eh = (double*)malloc(sizeof(double) * ne);
  }
  lho_stats S;
  memset(&S, 0, sizeof(S));
  S.energy0 = lho_total_energy(P, v, e);
  double t = t0;
  double dt = *dt_io;
  int status = LHO_OK;
  if (!(dt > 0.0)) {
    /* reading R5: the first step size is the estimate of the initial state */
    int st = lho_force(P, v, e, x, NULL, NULL, NULL, &dt);
    if (st != LHO_OK) { status = st; goto done; }
  }
  while (t < t_final && S.steps < max_steps) {
    double dt_use = dt;
    int last = 0;
    if (t + dt_use >= t_final) { dt_use = t_final - t; last = 1; }
    memcpy(vs, v, sizeof(double) * nv);
    memcpy(xs, x, sizeof(double) * nv);
    memcpy(es, e, sizeof(double) * ne);
    double tau;
    long its = 0;
    int st = P->cfg.integrator == LHO_RK4
                 ? lho_step_rk4(P, dt_use, vs, es, xs, &tau, &its)
                 : step_rk2avg(P, dt_use, vs, es, xs, &tau, &its, vh, eh, xh);
    S.cg_iters += its;
    if (st == LHO_ETANGLED) tau = 0.0;  /* a tangled stage forces a redo */
    else if (st != LHO_OK) { status = st; break; }
    if (dt_use >= tau) {
      /* redo with a smaller step (Section 2.2.3, step 2) */
      dt = P->cfg.beta1 * dt_use;
      S.rejects++;
      if (dt < P->cfg.dt_min_frac * t_final) { status = LHO_EDTMIN; break; }
      continue;
    }
    memcpy(v, vs, sizeof(double) * nv);
    memcpy(x, xs, sizeof(double) * nv);
    memcpy(e, es, sizeof(double) * ne);
    if (snap) {  /* the accepted step's stage states: S^{n+1/2}, then S^{n+1} */
      snap_put(P, snap, vh, eh, xh);
      snap_put(P, snap, v, e, x);
    }
    if (dt_log && S.steps < dt_log_cap) dt_log[S.steps] = dt_use;
    S.steps++;
    t = last ? t_final : t + dt_use;
    dt = (dt_use <= P->cfg.gamma_dt * tau) ? P->cfg.beta2 * dt_use : dt_use;
  }
done:
  S.t = t;
  S.dt = dt;
  S.energy = lho_total_energy(P, v, e);
  *dt_io = dt;
  if (stats) *stats = S;
  free(vs); free(xs); free(es);
  free(vh); free(xh); free(eh);
  return status;
}

int lho_run(const lho_problem* P, double t0, double t_final, long max_steps,
            double* v, double* e, double* x, double* dt_io, lho_stats* stats,
            double* dt_log, long dt_log_cap) {
  return run_impl(P, t0, t_final, max_steps, v, e, x, dt_io, stats, dt_log, dt_log_cap, NULL);
}

int lho_run_snapshots(const lho_problem* P, double t0, double t_final, long max_steps,
                      double* v, double* e, double* x, double* dt_io, lho_stats* stats,
                      double* Sv, double* Se, double* Sx, long cap, long* count) {
  if (P->cfg.integrator != LHO_RK2AVG) return LHO_EINVAL;
  snapshots S = {Sv, Se, Sx, cap, 0};
  int st = run_impl(P, t0, t_final, max_steps, v, e, x, dt_io, stats, NULL, 0, &S);
  *count = S.count;
  return st;
}

/* ------------------------------------------------------------------ POD -- */

/* Thin SVD A = U Sigma W^T of a column-major m x n matrix by one-sided
 * (Hestenes) Jacobi: plane rotations of column pairs, in cyclic order, until
 * every pair is orthogonal to |a_p . a_q| <= tol |a_p| |a_q| (pairs with a
 * column below 1e-16 of the Frobenius norm count as orthogonal).  On return the
 * columns of A are U Sigma (unsorted) and sigma[j] their norms. */
int lho_svd_jacobi(long m, long n, double* A, double* sigma, double tol, int max_sweeps,
                   int* sweeps_out) {
  /* columns whose norm is at the rounding level of the whole matrix are the
   * null space of a rank-deficient A: they are left alone */
  double fro2 = 0.0;
  for (long j = 0; j < n; ++j) fro2 += dot(m, A + j * m, A + j * m);
  const double floor2 = 1e-32 * fro2;
  int sweep;
  for (sweep = 1; sweep <= max_sweeps; ++sweep) {
    int rotated = 0;
    for (long p = 0; p < n - 1; ++p)
      for (long q = p + 1; q < n; ++q) {
        double* ap = A + p * m;
        double* aq = A + q * m;
        double alpha = dot(m, ap, ap), beta = dot(m, aq, aq), gamma = dot(m, ap, aq);
        if (alpha <= floor2 || beta <= floor2) continue;
        if (fabs(gamma) <= tol * sqrt(alpha * beta) || gamma == 0.0) continue;
        rotated = 1;
        /* the rotation that zeroes the (p, q) entry of A^T A */
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (long i = 0; i < m; ++i) {
          double u = ap[i], w = aq[i];
          ap[i] = c * u - s * w;
          aq[i] = s * u + c * w;
        }
      }
    if (!rotated) break;
  }
  if (sweeps_out) *sweeps_out = sweep > max_sweeps ? max_sweeps : sweep;
  for (long j = 0; j < n; ++j) sigma[j] = sqrt(dot(m, A + j * m, A + j * m));
  return sweep > max_sweeps ? LHO_ECG : LHO_OK;
}

/* POD basis of a snapshot matrix (eq:SVD, eq:energy_criteria): the columns
 * of S (m x n, column-major) minus the offset vector (may be NULL), thin SVD,
 * singular values in descending order, and the smallest k with
 * sum_{i<=k} sigma_i >= eps sum_i sigma_i.  U (m x n) receives the left
 * singular vectors in that order (the first k are the basis), sigma (n) the
 * singular values. */
int lho_pod(long m, long n, const double* S, const double* offset, double eps, double* U,
            double* sigma, long* k_out) {
  double* A = (double*)malloc(sizeof(double) * m * n);
  double* sg = (double*)malloc(sizeof(double) * n);
  long* order = (long*)malloc(sizeof(long) * n);
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < m; ++i) A[j * m + i] = S[j * m + i] - (offset ? offset[i] : 0.0);
  int sweeps;
  /* orthogonality at the rounding level of an m-term inner product */
  int st = lho_svd_jacobi(m, n, A, sg, sqrt((double)m) * 2.220446049250313e-16, 60, &sweeps);
  /* descending order (stable: equal values keep their column order) */
  for (long j = 0; j < n; ++j) order[j] = j;
  for (long a = 1; a < n; ++a) {
    long key = order[a], b = a - 1;
    while (b >= 0 && sg[order[b]] < sg[key]) { order[b + 1] = order[b]; --b; }
    order[b + 1] = key;
  }
  double total = 0.0;
  for (long j = 0; j < n; ++j) total += sg[j];
  long k = n;
  double acc = 0.0;
  for (long r = 0; r < n; ++r) {
    acc += sg[order[r]];
    if (acc >= eps * total) { k = r + 1; break; }
  }
  for (long r = 0; r < n; ++r) {
    long j = order[r];
    sigma[r] = sg[j];
    for (long i = 0; i < m; ++i) U[r * m + i] = sg[j] > 0.0 ? A[j * m + i] / sg[j] : 0.0;
  }
  *k_out = total > 0.0 ? k : 0;
  free(A); free(sg); free(order);
  return st;
}
