// Host-side set-up of a context: descriptor checks, 1D basis tables,
// quadrature data of the initial Cartesian mesh, initial conditions of the
// test problems of Section 6.1, device allocations and state copies.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "lagh_impl.cuh"

namespace lagh {

lh_status set_error(lh_ctx* c, lh_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

lh_status cuda_check(lh_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LH_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return set_error(c, e == cudaErrorMemoryAllocation ? LH_ENOMEM : LH_ECUDA, m);
}

// ------------------------------------------------------------ 1D bases ----

// Legendre P_n(t) and derivative on [-1, 1] (Bonnet recurrence).
static void legendre_pd(int n, double t, double& P, double& dP) {
  double pm = 1.0, pc = t;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int m = 1; m < n; ++m) {
    double pn = ((2 * m + 1) * t * pc - m * pm) / (m + 1);
    pm = pc;
    pc = pn;
  }
  P = pc;
  dP = n * (pm - t * pc) / (1.0 - t * t);
}

// n Gauss-Legendre points / weights mapped to [0, 1], ascending.
static void gl_rule(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double t = -cos(3.14159265358979323846 * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    for (int it = 0; it < 60; ++it) {
      double P, dP;
      legendre_pd(n, t, P, dP);
      double step = P / dP;
      t -= step;
      if (fabs(step) <= 1e-16) break;
    }
    double P, dP;
    legendre_pd(n, t, P, dP);
    x[i] = 0.5 * (1.0 + t);
    w[i] = 1.0 / ((1.0 - t * t) * dP * dP);
  }
}

// k+1 Gauss-Lobatto nodes on [0, 1]: the ends and the zeros of P_k'.
static void gll_nodes(int k, double* x) {
  x[0] = 0.0;
  x[k] = 1.0;
  for (int i = 1; i < k; ++i) {
    double t = -cos(3.14159265358979323846 * i / k);
    for (int it = 0; it < 60; ++it) {
      double P, dP;
      legendre_pd(k, t, P, dP);
      double d2P = (2.0 * t * dP - k * (k + 1.0) * P) / (1.0 - t * t);
      double step = dP / d2P;
      t -= step;
      if (fabs(step) <= 1e-16) break;
    }
    x[i] = 0.5 * (1.0 + t);
  }
}

// Lagrange basis on nodes z[0..n) and its derivative at t (barycentric form).
static void lagrange_at(int n, const double* z, double t, double* val, double* der) {
  double wb[8];
  for (int a = 0; a < n; ++a) {
    double p = 1.0;
    for (int b = 0; b < n; ++b)
      if (b != a) p *= (z[a] - z[b]);
    wb[a] = 1.0 / p;
  }
  for (int a = 0; a < n; ++a) {
    // l_a(t) = w_a prod_{b != a} (t - z_b); derivative by the product rule
    double prod = 1.0, dsum = 0.0;
    for (int b = 0; b < n; ++b) {
      if (b == a) continue;
      dsum = dsum * (t - z[b]) + prod;
      prod *= (t - z[b]);
    }
    val[a] = wb[a] * prod;
    if (der) der[a] = wb[a] * dsum;
  }
}

static bool invert_small(int n, const double* A, double* Ainv) {
  std::vector<double> M(2 * n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(M[r * 2 * n + col]) > fabs(M[piv * 2 * n + col])) piv = r;
    if (M[piv * 2 * n + col] == 0.0) return false;
    for (int j = 0; j < 2 * n; ++j) std::swap(M[col * 2 * n + j], M[piv * 2 * n + j]);
    double d = M[col * 2 * n + col];
    for (int j = 0; j < 2 * n; ++j) M[col * 2 * n + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = M[r * 2 * n + col];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * n; ++j) M[r * 2 * n + j] -= f * M[col * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i * 2 * n + n + j];
  return true;
}

void build_basis(int k, int nq, int dim, Basis1D* b) {
  memset(b, 0, sizeof(*b));
  double xn[kMaxOrder + 1], qx[kMaxQ], qw[kMaxQ], l2x[kMaxOrder], l2w[kMaxOrder];
  gll_nodes(k, xn);
  gl_rule(nq, qx, qw);
  gl_rule(k, l2x, l2w);
  for (int q = 0; q < nq; ++q) {
    double v[8], d[8];
    lagrange_at(k + 1, xn, qx[q], v, d);
    for (int a = 0; a <= k; ++a) {
      b->B[q][a] = v[a];
      b->G[q][a] = d[a];
      b->Bf[q][a] = (float)v[a];
      b->Gf[q][a] = (float)d[a];
    }
    lagrange_at(k, l2x, qx[q], v, nullptr);
    for (int j = 0; j < k; ++j) {
      b->L[q][j] = v[j];
      b->Lf[q][j] = (float)v[j];
    }
    b->W[q] = qw[q];
    b->Wf[q] = (float)qw[q];
  }
  for (int a = 0; a <= k; ++a)
    for (int c = 0; c <= k; ++c) {
      double s = 0.0;
      for (int q = 0; q < nq; ++q) s += qw[q] * b->B[q][a] * b->B[q][c];
      b->M1[a][c] = s;
    }
  // reference thermodynamic mass matrix: tensor product of 1D L2 mass matrices
  double m1[kMaxOrder][kMaxOrder];
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int q = 0; q < nq; ++q) s += qw[q] * b->L[q][i] * b->L[q][j];
      m1[i][j] = s;
    }
  int nd2 = 1;
  for (int c = 0; c < dim; ++c) nd2 *= k;
  std::vector<double> Mref(nd2 * nd2);
  for (int i = 0; i < nd2; ++i)
    for (int j = 0; j < nd2; ++j) {
      double s = 1.0;
      int ii = i, jj = j;
      for (int c = 0; c < dim; ++c) {
        s *= m1[ii % k][jj % k];
        ii /= k;
        jj /= k;
      }
      Mref[i * nd2 + j] = s;
    }
  invert_small(nd2, Mref.data(), b->MEinv);
  // integral of each reference L2 basis function = row sums of Mref
  // (the L2 basis is a partition of unity)
  for (int i = 0; i < nd2; ++i) {
    double s = 0.0;
    for (int j = 0; j < nd2; ++j) s += Mref[i * nd2 + j];
    b->L2int[i] = s;
  }
}

}  // namespace lagh

using namespace lagh;

// ------------------------------------------------------------- C ABI ----

lh_status lagh::make_geom(const lh_mesh_desc* mesh, const lh_disc_desc* disc, Geom* out,
                    std::string* why) {
  auto bad = [&](lh_status st, const char* m) {
    if (why) *why = m;
    return st;
  };
  const int d = mesh->dim;
  if (d != 2 && d != 3) return bad(LH_EINVAL, "dim must be 2 or 3");
  const int k = disc->order;
  if (k < 1 || k > 3 || (d == 3 && k > 2)) return bad(LH_EUNSUPPORTED, "order not built");
  if (disc->nq != 2 * k) return bad(LH_EUNSUPPORTED, "only nq = 2k is built");
  int nel[3] = {mesh->nx, mesh->ny, d == 3 ? mesh->nz : 1};
  for (int i = 0; i < d; ++i) {
    if (nel[i] < 1) return bad(LH_EINVAL, "element counts must be positive");
    if (!(mesh->hi[i] > mesh->lo[i])) return bad(LH_EINVAL, "empty box");
  }
  Geom g;
  memset(&g, 0, sizeof(g));
  g.dim = d;
  g.k = k;
  g.nq = disc->nq;
  g.nnodes = 1;
  g.nelem = 1;
  double vol = 1.0;
  for (int i = 0; i < 3; ++i) {
    g.n[i] = i < d ? nel[i] : 1;
    g.nn[i] = i < d ? nel[i] * k + 1 : 1;
    g.nnodes *= g.nn[i];
    g.nelem *= g.n[i];
    double h = i < d ? (mesh->hi[i] - mesh->lo[i]) / nel[i] : 1.0;
    if (i < d) vol *= h;
    g.lo[i] = i < d ? mesh->lo[i] : 0.0;
    g.h[i] = h;
    g.J0inv[i] = 1.0 / h;
  }
  int nd2 = 1;
  for (int i = 0; i < d; ++i) nd2 *= k;
  g.nv = (int64_t)d * g.nnodes;
  g.ne = g.nelem * nd2;
  g.detJ0 = vol;
  g.ell0 = pow(vol, 1.0 / d) / k;
  for (int i = 0; i < 3; ++i) g.J0invf[i] = (float)g.J0inv[i];
  g.ell0f = (float)g.ell0;
  if (g.nelem > (int64_t)1 << 31) return bad(LH_EINVAL, "mesh too large");
  *out = g;
  return LH_OK;
}

void lagh::banded_cholesky_1d(const Basis1D& b, int k, int nel, int var, std::vector<double>& L) {
  const int P = k + 1;
  const int N = nel * k + 1 - 2 * var;
  L.assign((size_t)(N > 0 ? N : 0) * (k + 1), 0.0);
  auto G = [&](int i, int j) -> double {
    int gi = i + var, gj = j + var;
    double s = 0.0;
    for (int e = 0; e < nel; ++e) {
      int a = gi - e * k, c = gj - e * k;
      if (a >= 0 && a < P && c >= 0 && c < P) s += b.M1[a][c];
    }
    return s;
  };
  for (int i = 0; i < N; ++i) {
    for (int m = k; m >= 1; --m) {
      int j = i - m;
      if (j < 0) continue;
      double s = G(i, j);
      for (int q = 1; q <= k; ++q) {
        int l = j - q;
        if (l < 0 || i - l > k) continue;
        s -= L[(size_t)i * (k + 1) + (i - l)] * L[(size_t)j * (k + 1) + q];
      }
      L[(size_t)i * (k + 1) + m] = s / L[(size_t)j * (k + 1)];
    }
    double s = G(i, i);
    for (int m = 1; m <= k; ++m) s -= L[(size_t)i * (k + 1) + m] * L[(size_t)i * (k + 1) + m];
    L[(size_t)i * (k + 1)] = sqrt(s);
  }
}

extern "C" void lh_default_phys(lh_phys_desc* p) {
  memset(p, 0, sizeof(*p));
  p->problem = LH_SEDOV;
  p->visc = 1;
  p->source = 1;
  p->cg_maxit = 500;
  p->gamma = 1.4;
  p->blast_energy = 0.25;
  p->e_uniform = 1.0;
  p->cfl = 0.5;
  p->cfl_mu = 2.5;
  p->beta1 = 0.85;
  p->beta2 = 1.02;
  p->gamma_dt = 0.8;
  p->q1 = 0.5;
  p->q2 = 2.0;
  p->cg_rtol = 1e-14;
  p->dt_min_frac = 1e-12;
  p->cg_precond = LH_PRECOND_AUTO;
}

extern "C" const char* lh_status_string(lh_status s) {
  switch (s) {
    case LH_OK: return "ok";
    case LH_EINVAL: return "invalid argument";
    case LH_ENOMEM: return "out of device memory";
    case LH_ECUDA: return "CUDA error";
    case LH_ETANGLED: return "inverted element (|J| <= 0)";
    case LH_ENONFINITE: return "non-finite state";
    case LH_EDTMIN: return "time step collapsed";
    case LH_ECG: return "CG did not converge";
    case LH_ETIMEOUT: return "device wait timed out";
    case LH_EUNSUPPORTED: return "unsupported configuration";
    case LH_ETOOLARGE: return "mesh exceeds the fixed working memory";
  }
  return "unknown status";
}

extern "C" const char* lh_last_error(const lh_ctx* c) { return c ? c->err.c_str() : "null context"; }

static void free_all(lh_ctx* c) {
  double** dptrs[] = {&c->a.v, &c->a.e, &c->a.x, &c->a.vh, &c->a.eh, &c->a.xh, &c->a.vn,
                      &c->a.en, &c->a.xn, &c->a.vbar, &c->a.F1E, &c->a.rhs, &c->a.acc,
                      &c->a.r, &c->a.r2, &c->a.z, &c->a.p, &c->a.Ap, &c->a.ApE, &c->a.D,
                      &c->a.srcE, &c->a.gammaE, &c->a.Kv, &c->a.Kx, &c->a.Ke, &c->a.erate,
                      &c->a.rho0K, &c->a.rho0Kinv, &c->a.dinv, &c->a.partials, &c->a.tmpE, &c->a.tmpV,
                      &c->a.aux};
  for (double** p : dptrs)
    if (*p) { cudaFree(*p); *p = nullptr; }
  if (c->a.FK) { cudaFree(c->a.FK); c->a.FK = nullptr; }
  if (c->a.ctl) { cudaFree(c->a.ctl); c->a.ctl = nullptr; }
  if (c->a.cg) { cudaFree(c->a.cg); c->a.cg = nullptr; }
  if (c->a.lfac) { cudaFree(c->a.lfac); c->a.lfac = nullptr; }
  if (c->a.lchol) { cudaFree(c->a.lchol); c->a.lchol = nullptr; }
  if (c->a.lfac64) { cudaFree(c->a.lfac64); c->a.lfac64 = nullptr; }
  if (c->a.lfac_lo) { cudaFree(c->a.lfac_lo); c->a.lfac_lo = nullptr; }
  if (c->side) { cudaStreamDestroy(c->side); c->side = nullptr; }
  if (c->ctl_host) { cudaFreeHost(c->ctl_host); c->ctl_host = nullptr; }
  if (c->graph_ready == 1) cudaGraphExecDestroy(c->step_graph);
  c->graph_ready = 0;
  if (c->own_work && c->work) { cudaStreamDestroy(c->work); c->work = nullptr; c->own_work = 0; }
  if (c->ev0) { cudaEventDestroy(c->ev0); c->ev0 = nullptr; }
  if (c->ev1) { cudaEventDestroy(c->ev1); c->ev1 = nullptr; }
}

extern "C" lh_status lh_destroy(lh_ctx* c) {
  if (!c) return LH_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_all(c);
  delete c;
  return LH_OK;
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc((void**)p, n * sizeof(T) > 0 ? n * sizeof(T) : sizeof(T));
}

extern "C" lh_status lh_create(const lh_mesh_desc* mesh, const lh_disc_desc* disc,
                               const lh_phys_desc* phys, int32_t precision, void* stream,
                               lh_ctx** out) {
  if (!out) return LH_EINVAL;
  *out = nullptr;
  if (!mesh || !disc || !phys) return LH_EINVAL;
  lh_ctx* c = new lh_ctx();
  memset(&c->g, 0, sizeof(c->g));
  memset(&c->a, 0, sizeof(c->a));
  c->ctl_host = nullptr;
  c->graph_ready = 0;
  c->use_pdl = 1;
  c->ev0 = c->ev1 = nullptr;
  c->work = nullptr;
  c->side = nullptr;
  c->own_work = 0;
  c->stream = (cudaStream_t)stream;
  c->precision = precision;
  c->phys_desc = *phys;
  auto fail = [&](lh_status s, const std::string& m) {
    fprintf(stderr, "lh_create: %s\n", m.c_str());
    free_all(c);
    delete c;
    return s;
  };
  if (precision != LH_FP64 && precision != LH_MIXED) return fail(LH_EINVAL, "bad precision");
  {
    std::string why;
    lh_status gs = make_geom(mesh, disc, &c->g, &why);
    if (gs != LH_OK) return fail(gs, why);
  }
  if (!(phys->gamma > 1.0)) return fail(LH_EINVAL, "gamma must exceed 1");
  if (phys->problem < LH_SEDOV || phys->problem > LH_TRIPLE_POINT)
    return fail(LH_EINVAL, "unknown problem");
  if (phys->integrator != LH_RK2AVG && phys->integrator != LH_RK4)
    return fail(LH_EINVAL, "unknown integrator");
  if (!(phys->cg_rtol > 0.0) || phys->cg_maxit < 1) return fail(LH_EINVAL, "bad CG settings");
  Geom& g = c->g;
  const int d = g.dim, k = g.k;
  int nd1 = 1, nd2 = 1, nqe = 1;
  for (int i = 0; i < d; ++i) { nd1 *= k + 1; nd2 *= k; nqe *= 2 * k; }
  const double vol = g.detJ0;

  Phys& ph = c->ph;
  ph.gamma = phys->gamma;
  ph.cfl = phys->cfl;
  ph.cfl_mu = phys->cfl_mu;
  ph.q1 = phys->q1;
  ph.q2 = phys->q2;
  ph.visc = phys->visc;
  ph.problem = phys->problem;
  ph.source = (phys->source && phys->problem == LH_TAYLOR_GREEN && d == 2) ? 1 : 0;
  set_phys_floats(ph);
  c->cg_rtol = phys->cg_rtol;
  c->cg_maxit = phys->cg_maxit;
  build_basis(k, g.nq, d, &c->basis);

  int dev = 0;
  lh_status st;
  if ((st = cuda_check(c, cudaGetDevice(&dev), "cudaGetDevice")) != LH_OK) return fail(st, c->err);
  if ((st = cuda_check(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev),
                       "sm count")) != LH_OK)
    return fail(st, c->err);
  if ((st = cuda_check(c, prepare_kernels(c), "kernel attributes")) != LH_OK) return fail(st, c->err);

  Arrays& A = c->a;
  const size_t nv = g.nv, ne = g.ne, nelem = g.nelem;
  cudaError_t e = cudaSuccess;
  double** vecs_v[] = {&A.v, &A.x, &A.vh, &A.xh, &A.vn, &A.xn, &A.vbar, &A.rhs, &A.acc,
                       &A.r, &A.r2, &A.z, &A.p, &A.Ap, &A.tmpV};
  for (double** p : vecs_v)
    if (e == cudaSuccess) e = dalloc(p, nv);
  double** vecs_e[] = {&A.e, &A.eh, &A.en, &A.srcE, &A.tmpE};
  for (double** p : vecs_e)
    if (e == cudaSuccess) e = dalloc(p, ne);
  if (phys->integrator == LH_RK4) {
    double** rk_v[] = {&A.Kv, &A.Kx};
    for (double** p : rk_v)
      if (e == cudaSuccess) e = dalloc(p, nv);
    double** rk_e[] = {&A.Ke, &A.erate};
    for (double** p : rk_e)
      if (e == cudaSuccess) e = dalloc(p, ne);
  }
  if (e == cudaSuccess && phys->problem == LH_TRIPLE_POINT) e = dalloc(&A.gammaE, nelem);
  if (e == cudaSuccess) e = dalloc(&A.F1E, nelem * d * nd1);
  if (e == cudaSuccess) e = dalloc(&A.ApE, nelem * d * nd1);
  if (precision == LH_FP64) {
    if (e == cudaSuccess) e = dalloc(&A.D, nelem * d * d * nqe);
  } else {
    if (e == cudaSuccess) e = dalloc(&A.FK, nelem * d * nd1 * nd2);
  }
  if (e == cudaSuccess) e = dalloc(&A.rho0K, nelem);
  if (e == cudaSuccess) e = dalloc(&A.rho0Kinv, nelem);
  if (e == cudaSuccess) e = dalloc(&A.dinv, (size_t)g.nnodes);
  if (e == cudaSuccess) e = dalloc(&A.partials, (size_t)5 * kMaxPartials);
  if (e == cudaSuccess) e = dalloc(&A.cg, 1);
  if (e == cudaSuccess) e = cudaMemset(A.cg, 0, sizeof(CgDev));
  if (e == cudaSuccess) e = dalloc(&A.aux, 16);
  if (e == cudaSuccess) e = dalloc(&A.ctl, 1);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->ctl_host, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    if (c->stream == nullptr) {
      e = cudaStreamCreateWithFlags(&c->work, cudaStreamNonBlocking);
      c->own_work = 1;
    } else {
      c->work = c->stream;
    }
  }
  if ((st = cuda_check(c, e, "allocation")) != LH_OK) return fail(st, c->err);

  // quadrature data: rho0 |J0| per element (rho0 = 1 in every problem but the
  // triple point, whose rho0 and gamma are constant per element)
  std::vector<double> rho0K(nelem, 1.0 * vol);
  std::vector<double> gamE;
  if (phys->problem == LH_TRIPLE_POINT) {
    gamE.resize(nelem);
    for (int64_t el = 0; el < g.nelem; ++el) {
      double rho, p;
      triple_point_state(g, el, &rho, &p, &gamE[el]);
      rho0K[el] = rho * vol;
    }
  }
  // diagonal of the scalar kinematic mass matrix, assembled
  std::vector<double> diag(g.nnodes, 0.0);
  {
    const int P = k + 1;
    for (int64_t el = 0; el < g.nelem; ++el) {
      int E0 = (int)(el % g.n[0]), E1 = (int)((el / g.n[0]) % g.n[1]),
          E2 = (int)(el / ((int64_t)g.n[0] * g.n[1]));
      for (int i = 0; i < nd1; ++i) {
        int a = i % P, b = (i / P) % P, cz = i / (P * P);
        double dv = c->basis.M1[a][a] * c->basis.M1[b][b] * (d == 3 ? c->basis.M1[cz][cz] : 1.0);
        int64_t node = (int64_t)(E0 * k + a) +
                       (int64_t)g.nn[0] * ((int64_t)(E1 * k + b) + (int64_t)g.nn[1] * (E2 * k + cz));
        diag[node] += rho0K[el] * dv;
      }
    }
    for (auto& x : diag) x = 1.0 / x;
  }
  // tensor-product preconditioner: M_s = rho0|J0| G_x (x) G_y [(x) G_z] when
  // rho0 |J0| is the same in every element.  The inverse of each assembled 1D
  // reference mass matrix G_d (full, and without its two end nodes for the
  // wall-normal component) decays exponentially away from the diagonal; its
  // entries within half-width B are kept (relative size of the dropped ones
  // below 1e-9 for B = 14, 22, 30 at k = 1, 2, 3) and applied in FP32.
  std::vector<float> lf;
  std::vector<double> lf64;  // the bands in FP64
  std::vector<float> lflo;   // the bands' FP32 rounding errors (lf + lflo ~ lf64 to ~2^-48)
  std::vector<double> lc;    // exact variant: scaled banded Cholesky rows
  memset(&c->tpc, 0, sizeof(c->tpc));
  {
    bool uniform = true;
    for (int64_t el = 1; el < g.nelem; ++el)
      if (rho0K[el] != rho0K[0]) uniform = false;
    const int Btab[4] = {0, 14, 22, 30};
    int Bmax = 0;
    for (int dd = 0; dd < d; ++dd) {
      const int nfull = g.nn[dd];
      const int B = Btab[k];  // columns beyond the line are stored as zeros
      c->tpc.B[dd] = B;
      Bmax = B > Bmax ? B : Bmax;
      for (int var = 0; var < 2; ++var) {
        const int N = nfull - 2 * var;
        c->tpc.off[dd][var] = (int64_t)lf.size();
        c->tpc.off64[dd][var] = (int64_t)lf64.size();
        if (N <= 0) continue;
        std::vector<double> L;  // L[i][m] = L_{i,i-m}
        banded_cholesky_1d(c->basis, k, g.n[dd], var, L);
        // exact variant, row r: d_r = 1 / L_rr, d_r L_{r,r-q}, d_r L_{r+q,r} (q = 1..k)
        c->tpc.coff[dd][var] = (int64_t)lc.size();
        for (int r = 0; r < N; ++r) {
          const double dr = 1.0 / L[(size_t)r * (k + 1)];
          lc.push_back(dr);
          for (int q = 1; q <= k; ++q) lc.push_back(dr * L[(size_t)r * (k + 1) + q]);
          for (int q = 1; q <= k; ++q)
            lc.push_back(r + q < N ? dr * L[(size_t)(r + q) * (k + 1) + q] : 0.0);
        }
        // columns of the inverse by banded solves; keep |i - j| <= B
        const int W = 2 * B + 1;
        std::vector<double> band((size_t)N * W, 0.0), col(N);
        for (int j = 0; j < N; ++j) {
          for (int i = 0; i < N; ++i) col[i] = (i == j) ? 1.0 : 0.0;
          for (int i = 0; i < N; ++i) {
            double y = col[i];
            for (int m = 1; m <= k && i - m >= 0; ++m) y -= L[(size_t)i * (k + 1) + m] * col[i - m];
            col[i] = y / L[(size_t)i * (k + 1)];
          }
          for (int i = N - 1; i >= 0; --i) {
            double y = col[i];
            for (int m = 1; m <= k && i + m < N; ++m) y -= L[(size_t)(i + m) * (k + 1) + m] * col[i + m];
            col[i] = y / L[(size_t)i * (k + 1)];
          }
          for (int i = (j - B > 0 ? j - B : 0); i <= j + B && i < N; ++i)
            band[(size_t)i * W + (j - i + B)] = col[i];
        }
        for (double v : band) {
          lf.push_back((float)v);
          lf64.push_back(v);
          lflo.push_back((float)(v - (double)(float)v));
        }
      }
    }
    c->tpc.Bmax = Bmax;
    c->tpc.scale = 1.0 / rho0K[0];
    // AUTO: the measured faster one per dimension (mixed Sedov 3D 32^3: exact
    // 1.88 against band 2.50 ms per step; every 2D workload: band)
    const int pc = phys->cg_precond == LH_PRECOND_AUTO
                       ? (d == 3 ? LH_PRECOND_EXACT : LH_PRECOND_TENSOR)
                       : phys->cg_precond;
    c->tpc.enabled = (pc == LH_PRECOND_TENSOR || pc == LH_PRECOND_TENSOR64 ||
                      pc == LH_PRECOND_EXACT) && uniform;
    c->tpc.exact = c->tpc.enabled && pc == LH_PRECOND_EXACT;
    c->tpc.fp64 = c->tpc.enabled && pc == LH_PRECOND_TENSOR64;
  }
  e = dalloc(&A.lfac, lf.size() > 0 ? lf.size() : 1);
  if (e == cudaSuccess && !lf.empty())
    e = cudaMemcpy(A.lfac, lf.data(), lf.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = dalloc(&A.lfac_lo, lflo.size() > 0 ? lflo.size() : 1);
  if (e == cudaSuccess && !lflo.empty())
    e = cudaMemcpy(A.lfac_lo, lflo.data(), lflo.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = dalloc(&A.lfac64, lf64.size() > 0 ? lf64.size() : 1);
  if (e == cudaSuccess && !lf64.empty())
    e = cudaMemcpy(A.lfac64, lf64.data(), lf64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = dalloc(&A.lchol, lc.size() > 0 ? lc.size() : 1);
  if (e == cudaSuccess && !lc.empty())
    e = cudaMemcpy(A.lchol, lc.data(), lc.size() * sizeof(double), cudaMemcpyHostToDevice);
  if ((st = cuda_check(c, e, "preconditioner")) != LH_OK) return fail(st, c->err);
  if ((st = cuda_check(c, cg_prepare(c), "cg attributes")) != LH_OK) return fail(st, c->err);
  // cluster-resident CG: small 2D problems with the band preconditioner.  Against
  // the kernel chain with its 2D tile kernels it was measured 10% faster at
  // N_V = 578 (8 x 8 Q2) and 6-7% slower at 2,178 and 4,802 (16^2, 24^2), so
  // only the smallest solves take it.
  c->cg_cluster = 0;
  if (phys->cg_cluster >= 0 && d == 2 && c->tpc.enabled && !c->tpc.exact && !c->tpc.fp64 &&
      (phys->cg_cluster == 1 || g.nv <= 1500))
    c->cg_cluster = cg_cluster_choose(c);
  c->cg_tiles = phys->cg_tiles >= 0 ? 1 : 0;
  Ctl ctl0;
  memset(&ctl0, 0, sizeof(ctl0));
  e = cudaMemcpy(A.rho0K, rho0K.data(), nelem * sizeof(double), cudaMemcpyHostToDevice);
  {
    std::vector<double> inv(nelem);
    for (size_t i = 0; i < nelem; ++i) inv[i] = 1.0 / rho0K[i];
    if (e == cudaSuccess)
      e = cudaMemcpy(A.rho0Kinv, inv.data(), nelem * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(A.dinv, diag.data(), g.nnodes * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(A.ctl, &ctl0, sizeof(Ctl), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(A.srcE, 0, ne * sizeof(double));
  if (e == cudaSuccess && A.gammaE)
    e = cudaMemcpy(A.gammaE, gamE.data(), nelem * sizeof(double), cudaMemcpyHostToDevice);
  if ((st = cuda_check(c, e, "upload")) != LH_OK) return fail(st, c->err);
  *out = c;
  return LH_OK;
}

extern "C" lh_status lh_layout(const lh_ctx* c, lh_layout_info* info) {
  if (!c || !info) return LH_EINVAL;
  const Geom& g = c->g;
  memset(info, 0, sizeof(*info));
  info->nv = g.nv;
  info->ne = g.ne;
  info->nelem = g.nelem;
  info->nnodes = g.nnodes;
  info->dim = g.dim;
  info->order = g.k;
  info->nq = g.nq;
  int nd1 = 1, nd2 = 1, nqe = 1;
  for (int i = 0; i < g.dim; ++i) { nd1 *= g.k + 1; nd2 *= g.k; nqe *= g.nq; }
  info->ndof_h1 = nd1;
  info->ndof_l2 = nd2;
  info->nqe = nqe;
  info->nqp = g.nelem * nqe;
  for (int i = 0; i < 3; ++i) info->nodes_per_dim[i] = g.nn[i];
  info->precision = c->precision;
  // essential components: nodes with index 0 or n-1 along the component
  int64_t ness = 0;
  for (int comp = 0; comp < g.dim; ++comp) {
    int64_t other = g.nnodes / g.nn[comp];
    ness += 2 * other;
  }
  info->n_essential = ness;
  info->precond_kernels = precond_kernels(c);
  return LH_OK;
}

// ------------------------------------------------------ initial state ----

static double gresho_vphi(double r) {
  if (r < 0.2) return 5.0 * r;
  if (r < 0.4) return 2.0 - 5.0 * r;
  return 0.0;
}

// Pressure of the Gresho vortex in radial balance dp/dr = v_phi^2 / r,
// continuous at r = 0.2 and r = 0.4.
static double gresho_pressure(double r) {
  if (r < 0.2) return 5.0 + 12.5 * r * r;
  if (r < 0.4) return 9.0 - 4.0 * log(0.2) + 12.5 * r * r - 20.0 * r + 4.0 * log(r);
  return 3.0 + 4.0 * log(2.0);
}

// Mixed path: reference pressure (gamma - 1) rho0 min(e), rho0 = 1, clamped at
// zero.  Any constant is exact (the split is algebraic); a value near the
// smallest pressure keeps the FP32 stress small relative to its gradients.
__global__ void pref_kernel(const double* e, int64_t ne, double gm1, Ctl* ctl) {
  __shared__ double sh[256];
  double m = 1e300;
  for (int64_t i = threadIdx.x; i < ne; i += blockDim.x) m = e[i] < m ? e[i] : m;
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s && sh[threadIdx.x + s] < sh[threadIdx.x]) sh[threadIdx.x] = sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double p = gm1 * sh[0];
    ctl->p_ref = (p > 0.0 && p < 1e300) ? p : 0.0;
  }
}

static lh_status set_pref(lh_ctx* c) {
  if (c->precision != LH_MIXED) return LH_OK;
  if (c->phys_desc.problem == LH_TRIPLE_POINT) {
    // gamma varies per element and there is no large background pressure:
    // the FP32 stress is the whole stress (p_ref = 0)
    double z = 0.0;
    cudaError_t err = cudaMemcpyAsync(&c->a.ctl->p_ref, &z, sizeof(double), cudaMemcpyHostToDevice,
                                      c->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    return cuda_check(c, err, "reference pressure");
  }
  pref_kernel<<<1, 256, 0, c->stream>>>(c->a.e, c->g.ne, c->phys_desc.gamma - 1.0, c->a.ctl);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  return cuda_check(c, err, "reference pressure");
}

void lagh::triple_point_state(const Geom& g, int64_t el, double* rho, double* p, double* gam) {
  const int64_t E0 = el % g.n[0], E1 = (el / g.n[0]) % g.n[1];
  const double xc = g.lo[0] + (E0 + 0.5) * g.h[0], yc = g.lo[1] + (E1 + 0.5) * g.h[1];
  const bool left = xc <= 1.0, low = yc <= 1.5;
  *rho = (left || low) ? 1.0 : 0.125;
  *p = left ? 1.0 : 0.1;
  *gam = (left || !low) ? 1.5 : 1.4;
}

void lagh::initial_state(const Geom& g, const lh_phys_desc& ph, std::vector<double>& v,
                   std::vector<double>& e, std::vector<double>& x) {
  const int d = g.dim, k = g.k;
  const double pi = 3.14159265358979323846;
  double xn[kMaxOrder + 1], l2x[kMaxOrder], l2w[kMaxOrder];
  gll_nodes(k, xn);
  gl_rule(k, l2x, l2w);
  v.assign(g.nv, 0.0);
  x.assign(g.nv, 0.0);
  e.assign(g.ne, 0.0);
  // nodes: coordinate lo + (element + GLL node) h along each direction
  for (int64_t node = 0; node < g.nnodes; ++node) {
    int64_t r = node;
    double X[3] = {0, 0, 0};
    for (int c2 = 0; c2 < d; ++c2) {
      int I = (int)(r % g.nn[c2]);
      r /= g.nn[c2];
      int el = I / k, a = I - el * k;
      X[c2] = g.lo[c2] + (el + xn[a]) * g.h[c2];
      x[c2 * g.nnodes + node] = X[c2];
    }
    double V[3] = {0, 0, 0};
    if (ph.problem == LH_TAYLOR_GREEN) {
      double cz = d == 3 ? cos(pi * X[2]) : 1.0;
      V[0] = sin(pi * X[0]) * cos(pi * X[1]) * cz;
      V[1] = -cos(pi * X[0]) * sin(pi * X[1]) * cz;
    } else if (ph.problem == LH_GRESHO) {
      double rr = sqrt(X[0] * X[0] + X[1] * X[1]);
      if (rr > 0.0) {
        double vp = gresho_vphi(rr);
        V[0] = -vp * X[1] / rr;
        V[1] = vp * X[0] / rr;
      }
    }
    for (int c2 = 0; c2 < d; ++c2) v[c2 * g.nnodes + node] = V[c2];
  }
  // energy at the L2 nodes (Gauss-Legendre points of each element)
  int nd2 = 1;
  for (int i = 0; i < d; ++i) nd2 *= k;
  const double gm1 = ph.gamma - 1.0;
  for (int64_t el = 0; el < g.nelem; ++el) {
    int E[3] = {(int)(el % g.n[0]), (int)((el / g.n[0]) % g.n[1]),
                (int)(el / ((int64_t)g.n[0] * g.n[1]))};
    for (int j = 0; j < nd2; ++j) {
      int jj[3] = {j % k, (j / k) % k, j / (k * k)};
      double X[3] = {0, 0, 0};
      for (int c2 = 0; c2 < d; ++c2) X[c2] = g.lo[c2] + (E[c2] + l2x[jj[c2]]) * g.h[c2];
      double ev = 0.0;
      const double rho0 = 1.0;
      switch (ph.problem) {
        case LH_TRIPLE_POINT: {
          double rho, p, gam;
          triple_point_state(g, el, &rho, &p, &gam);
          ev = p / ((gam - 1.0) * rho);
          break;
        }
        case LH_SEDOV:
          ev = (el == 0) ? ph.blast_energy / (rho0 * g.detJ0) : 0.0;
          break;
        case LH_UNIFORM:
          ev = ph.e_uniform;
          break;
        case LH_TAYLOR_GREEN: {
          double p;
          if (d == 2) p = 100.0 + (cos(2 * pi * X[0]) + cos(2 * pi * X[1])) / 4.0;
          else
            p = 100.0 + ((cos(2 * pi * X[0]) + cos(2 * pi * X[1])) * (cos(2 * pi * X[2]) + 2.0) - 2.0) / 16.0;
          ev = p / (gm1 * rho0);
          break;
        }
        case LH_GRESHO:
          ev = gresho_pressure(sqrt(X[0] * X[0] + X[1] * X[1])) / (gm1 * rho0);
          break;
      }
      e[el * nd2 + j] = ev;
    }
  }
}

extern "C" lh_status lh_init_state(lh_ctx* c) {
  if (!c) return LH_EINVAL;
  const Geom& g = c->g;
  std::vector<double> v, e, x;
  initial_state(g, c->phys_desc, v, e, x);
  cudaStream_t s = c->stream;
  cudaError_t err = cudaMemcpyAsync(c->a.v, v.data(), g.nv * 8, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->a.x, x.data(), g.nv * 8, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->a.e, e.data(), g.ne * 8, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  lh_status st = cuda_check(c, err, "init_state upload");
  if (st != LH_OK) return st;
  Ctl* h = c->ctl_host;
  memset(h, 0, sizeof(Ctl));
  err = cudaMemcpyAsync(c->a.ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if ((st = cuda_check(c, err, "init_state ctl")) != LH_OK) return st;
  return set_pref(c);
}

extern "C" lh_status lh_set_state(lh_ctx* c, const double* v, const double* e, const double* x,
                                  double t, double dt) {
  if (!c || !v || !e || !x) return LH_EINVAL;
  const Geom& g = c->g;
  cudaStream_t s = c->stream;
  cudaError_t err = cudaMemcpyAsync(c->a.v, v, g.nv * 8, cudaMemcpyDefault, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->a.x, x, g.nv * 8, cudaMemcpyDefault, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->a.e, e, g.ne * 8, cudaMemcpyDefault, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  lh_status st = cuda_check(c, err, "set_state");
  if (st != LH_OK) return st;
  err = cudaMemcpy(c->ctl_host, c->a.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
  if (err != cudaSuccess) return cuda_check(c, err, "set_state ctl");
  c->ctl_host->t = t;
  c->ctl_host->dt = dt;
  c->ctl_host->status = 0;
  c->ctl_host->done = 0;
  err = cudaMemcpyAsync(c->a.ctl, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if ((st = cuda_check(c, err, "set_state ctl")) != LH_OK) return st;
  return set_pref(c);
}

lh_status lagh::device_status(lh_ctx* c) {
  cudaError_t err = cudaMemcpyAsync(c->ctl_host, c->a.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                                    c->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  lh_status st = cuda_check(c, err, "device status");
  if (st != LH_OK) return st;
  int s = c->ctl_host->status;
  if (s & kDevNonFinite) return set_error(c, LH_ENONFINITE, "non-finite value in the state");
  if (s & kDevDtMin) return set_error(c, LH_EDTMIN, "time step collapsed below dt_min");
  if (s & kDevCG) return set_error(c, LH_ECG, "CG did not converge within cg_maxit");
  if (s & kDevTangled) return set_error(c, LH_ETANGLED, "inverted element (|J| <= 0)");
  return LH_OK;
}

extern "C" lh_status lh_get_state(lh_ctx* c, double* v, double* e, double* x, double* t,
                                  double* dt) {
  if (!c) return LH_EINVAL;
  const Geom& g = c->g;
  cudaStream_t s = c->stream;
  cudaError_t err = cudaSuccess;
  if (v) err = cudaMemcpyAsync(v, c->a.v, g.nv * 8, cudaMemcpyDefault, s);
  if (err == cudaSuccess && x) err = cudaMemcpyAsync(x, c->a.x, g.nv * 8, cudaMemcpyDefault, s);
  if (err == cudaSuccess && e) err = cudaMemcpyAsync(e, c->a.e, g.ne * 8, cudaMemcpyDefault, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(c->ctl_host, c->a.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  lh_status st = cuda_check(c, err, "get_state");
  if (st != LH_OK) return st;
  if (t) *t = c->ctl_host->t;
  if (dt) *dt = c->ctl_host->dt;
  return LH_OK;
}
