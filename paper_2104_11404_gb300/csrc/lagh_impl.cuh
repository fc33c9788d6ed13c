// Internal declarations of the GB300 Lagrangian hydro library (not part of
// the C ABI).  Every kernel is templated on the space dimension DIM, the H1
// order K and the 1D Gauss-Legendre count NQ (= 2K).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lagh.h"

namespace lagh {

constexpr int kMaxOrder = 3;          // K
constexpr int kMaxQ = 2 * kMaxOrder;  // NQ

// device-side error bits (Ctl::status)
enum : int {
  kDevTangled = 1,
  kDevNonFinite = 2,
  kDevCG = 4,
  kDevTimeout = 8,
  kDevDtMin = 16,
};

constexpr __host__ __device__ int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// 1D tables on [0,1], passed by value (kernel parameter space).
struct Basis1D {
  double B[kMaxQ][kMaxOrder + 1];   // H1 Lagrange (Gauss-Lobatto nodes) at qp
  double G[kMaxQ][kMaxOrder + 1];   // its derivative
  double L[kMaxQ][kMaxOrder];       // L2 Lagrange (Gauss-Legendre nodes) at qp
  double W[kMaxQ];                  // Gauss-Legendre weights
  double M1[kMaxOrder + 1][kMaxOrder + 1];  // 1D H1 reference mass matrix
  float Bf[kMaxQ][kMaxOrder + 1];
  float Gf[kMaxQ][kMaxOrder + 1];
  float Lf[kMaxQ][kMaxOrder];
  float Wf[kMaxQ];
  double MEinv[81];                 // reference M_E^{-1} (ndof_l2^2 <= 81)
  double L2int[27];                 // integral of each reference L2 basis function
};

struct Geom {
  int dim, k, nq;
  int n[3];        // elements per direction (1 if unused)
  int nn[3];       // H1 nodes per direction
  int64_t nnodes, nelem, nv, ne;
  double lo[3];    // box origin
  double h[3];     // element widths
  double J0inv[3]; // diagonal of the initial Jacobian inverse (Cartesian mesh)
  double ell0;     // initial length scale |K_0|^{1/d} / k
  double detJ0;    // |K_0|
  float J0invf[3]; // FP32 copies for the FP32 path (rounded once on the host)
  float ell0f;
};

struct Phys {
  double gamma, cfl, cfl_mu, q1, q2;
  int visc, source, problem;
  float gammaf, cflf, cfl_muf, q1f, q2f;  // FP32 copies (set_phys_floats)
};

// Fills the FP32 copies of the constants of ph.
inline void set_phys_floats(Phys& ph) {
  ph.gammaf = (float)ph.gamma;
  ph.cflf = (float)ph.cfl;
  ph.cfl_muf = (float)ph.cfl_mu;
  ph.q1f = (float)ph.q1;
  ph.q2f = (float)ph.q2;
}

// Device control block of the time loop (one per context).
struct Ctl {
  double t, dt, dt_use, t_final, dt_min;
  unsigned long long tau_bits[2];   // per-stage min estimate, ordered bits
  long long steps, rejects, attempts, cg_iters, max_steps;
  long long dt_log_cap;
  double* dt_log;
  int last;       // dt_use was clamped to land on t_final
  int done;       // loop finished (t_final, max_steps or error)
  int accepted;   // last attempt accepted
  int status;     // kDev* error bits
  int cg_last_iters;
  double cg_last_relres;
  double tau_last;  // min estimate over both stages of the last attempt
  double p_ref;     // mixed path: constant reference pressure split off the FP32 stress
  int fixed;        // replay mode: accept every attempt
};

// Scalars of one CG solve (device memory).
constexpr int kMaxPartials = 16384;
struct CgDev {
  double bb, rz, alpha, beta;
  int it, done;
  unsigned int ticket[8];
};

// Tensor-product preconditioner: the inverses of the assembled 1D reference
// mass matrices along each direction, full (variant 0) and without the two end
// nodes (variant 1, the wall-normal component), truncated to the band
// |i - j| <= B[d] and stored in FP32 as rows [i][j - i + B].
struct TensorPC {
  int64_t off[3][2];   // offsets into Arrays::lfac (units of float)
  int64_t off64[3][2]; // offsets into Arrays::lfac64 (units of double)
  int64_t coff[3][2];  // offsets into Arrays::lchol (units of double)
  int B[3];            // band half-width per direction
  int Bmax;
  double scale;        // 1 / (rho0 |J0|), the same for every element
  int enabled;
  int exact;           // 1: banded Cholesky line solves (lchol) instead of the bands
  int fp64;            // 1: the bands in FP64 (lfac64), FP64 accumulation
};

// Work arrays of one context (all device pointers).
struct Arrays {
  double *v, *e, *x;            // current state
  double *vh, *eh, *xh;         // half-step state S^{n+1/2}
  double *vn, *en, *xn;         // candidate state S^{n+1} (committed if accepted)
  double *vbar;                 // (v^n + v^{n+1}) / 2
  double *F1E;                  // element-local F.1 [nelem][dim][nd1]
  double *rhs, *acc;            // CG right-hand side and solution
  double *r, *z, *p, *Ap;       // CG vectors
  double *r2;                   // the residual's second buffer (2D tile preconditioner)
  double *ApE;                  // element-local M p [nelem][dim][nd1]
  double *D;                    // FP64 path: stress weights [nelem][dim*dim][nqe]
  float *FK;                    // mixed path: element force matrices [nelem][dim*nd1][nd2]
  double *srcE;                 // energy source [N_E]
  double *gammaE;               // adiabatic index per element (NULL: the constant one)
  double *Kv, *Kx, *Ke, *erate; // RK4: weighted stage sums of dv/dt, dx/dt, de/dt; de/dt
  double *rho0K;                // rho0 |J0| per element
  double *rho0Kinv;             // its reciprocal
  double *dinv;                 // 1 / diag(M_s) per node
  double *partials;             // reduction partials [4][max_blocks]
  double *tmpE;                 // N_E scratch
  double *tmpV;                 // N_V scratch
  double *aux;                  // 16 doubles of API scratch (estimates, flags, energy)
  float *lfac;                  // tensor preconditioner bands (FP32)
  double *lfac64;               // the same bands in FP64
  float *lfac_lo;               // the FP64 bands minus their FP32 roundings, in FP32
  double *lchol;                // exact preconditioner: scaled Cholesky rows (FP64)
  CgDev* cg;
  Ctl* ctl;
};

}  // namespace lagh

struct lh_ctx {
  lagh::Geom g;
  lagh::Phys ph;
  lagh::Basis1D basis;
  lh_phys_desc phys_desc;
  int precision;
  cudaStream_t stream;
  lagh::Arrays a;
  lagh::Ctl* ctl_host;      // pinned mirror of the control block
  int num_sms;
  double cg_rtol;
  int cg_maxit;
  lagh::TensorPC tpc;
  cudaStream_t work;          // stream the step graph is captured and launched on
  cudaStream_t side;          // second stream, used to capture conditional bodies
  int own_work;               // work stream created by the context
  cudaGraphExec_t step_graph;
  int graph_ready;            // 1: graph built, -1: capture unsupported (eager launches)
  int use_pdl;                // programmatic dependent launch between the step's kernels
  int cg_cluster;             // CTAs of the cluster-resident CG (0: kernel chain)
  int cg_tiles;               // 1: 2D band passes as one 16 x 16 tile kernel where narrow
  cudaEvent_t ev0, ev1;
  std::string err;
};

namespace lagh {

// Launches kern on s, with programmatic dependent launch when pdl is set (the
// kernel must call pdl_enter() first; see device_util.cuh).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---- host helpers (setup.cu) ----
lh_status set_error(lh_ctx* c, lh_status s, const std::string& msg);
lh_status cuda_check(lh_ctx* c, cudaError_t e, const char* what);
void build_basis(int k, int nq, int dim, Basis1D* b);
// Geometry of a Cartesian box mesh (validates the descriptors; *why = reason).
lh_status make_geom(const lh_mesh_desc* mesh, const lh_disc_desc* disc, Geom* g,
                    std::string* why);
// Initial condition of the problem at the nodes (host arrays, resized).
void initial_state(const Geom& g, const lh_phys_desc& ph, std::vector<double>& v,
                   std::vector<double>& e, std::vector<double>& x);
// Triple point (Section 6.1.4): density, pressure and adiabatic index of
// element el, by its initial centre.
void triple_point_state(const Geom& g, int64_t el, double* rho, double* p, double* gam);
// Banded Cholesky factor of the assembled 1D reference mass matrix of nel
// elements (var = 1: without its two end nodes): L[i][m] = L_{i,i-m}, m <= k.
void banded_cholesky_1d(const Basis1D& b, int k, int nel, int var, std::vector<double>& L);
lh_status device_status(lh_ctx* c);  // reads ctl->status (synchronizes)

// ---- kernel launchers (force.cu, mass.cu, step.cu) ----
// Force on an explicit state.  list/nlist: element subset (NULL = all, slot =
// element).  Outputs: F1E (element-local rows, slot major), D (if store_D),
// FK (mixed, if store_FK), FTvE (if vtest), srcE (if source), tau slot.
struct ForceArgs {
  const double *v, *e, *x, *vtest;
  const int32_t* list;
  int64_t nslots;
  double* F1E;
  double* D;
  float* FK;
  double* FTvE;
  double* srcE;
  unsigned long long* tau_bits;  // may be NULL (no estimate)
  int* status;
  const Ctl* ctl;     // if non-NULL and ctl->done, the kernel returns at once
  const double* p_ref;  // device scalar: mixed stress is sigma + p_ref I
  const double* gammaE; // adiabatic index per element (NULL: Phys::gamma); set by the launcher
  int mode;           // 0: full physics; 1: only the reference pressure -p_ref I (FP64)
  int accumulate;     // add to F1E / FTvE instead of overwriting
};
enum { kForceFull = 0, kForceRefPressure = 1 };
// Same force in FP64 whatever the context precision (reference-pressure mode).
cudaError_t launch_force_fp64(const lh_ctx* c, const ForceArgs& fa, cudaStream_t s);
cudaError_t launch_force(const lh_ctx* c, const ForceArgs& fa, cudaStream_t s);

// Node gather of an element-local kinematic vector: out = scale * gather(E),
// essential components set to zero when apply_bc.
cudaError_t launch_gather(const lh_ctx* c, const double* E, double* out, double scale,
                          int apply_bc, const Ctl* ctl, cudaStream_t s);

// Energy update: e_out = e_base + coef * M_E^{-1} (F^T w + src), coef =
// frac * ctl->dt_use (or frac * dt if ctl == NULL).
struct EnergyArgs {
  const double* w;       // kinematic test vector (N_V)
  const double* D;       // FP64 path
  const float* FK;       // mixed path
  const double* srcE;    // may be NULL
  const double* x;       // mixed path: positions of the force's state, for the F^T w of
  const double* p_ref;   //   the reference pressure -p_ref I in FP64 (either NULL: none)
  const double* e_base;
  double* e_out;
  double frac;
  double dt;
  int rate;              // 1: e_out = frac M_E^{-1} (F^T w + src) (no dt, e_base unused)
  const int32_t* list;   // list mode (with FTvE): the elements whose F^T w rows are wanted
  int64_t nslots;
  double* FTvE;          // list mode output: F^T w element rows [slot][j] (from the stored D)
  const Ctl* ctl;
  const double* rho0Kinv;  // 1 / (rho0 |J0|) per element (NULL: divide)
};
cudaError_t launch_energy_update(const lh_ctx* c, const EnergyArgs& ea, cudaStream_t s);
// F^T w element rows of the listed elements from what the force kernel stored
// for them (ea.list, ea.nslots, ea.FTvE, ea.w): the stress weights D (FP64),
// or the FP32 element matrices F_K with the FP64 reference-pressure part from
// ea.x and ea.p_ref (mixed).
cudaError_t launch_ftv_list(const lh_ctx* c, const EnergyArgs& ea, cudaStream_t s);

// Mass operations.
cudaError_t launch_mass_apply(const lh_ctx* c, const double* in, double* out, cudaStream_t s);
// Preconditioned CG on M_V out = rhs (non-essential components); iteration
// count, relative residual and failures are written to c->a.ctl.
cudaError_t cg_solve_eager(const lh_ctx* c, const double* rhs, double* out, cudaStream_t s,
                           int* done_host);
cudaError_t precond_apply(const lh_ctx* c, const double* in, double* out, cudaStream_t s);
cudaError_t cg_solve_capture(const lh_ctx* c, const double* rhs, double* out, const Ctl* gate,
                             cudaStream_t s, cudaStream_t side);
cudaError_t launch_mass_solve_e(const lh_ctx* c, const double* rhs, double* out, cudaStream_t s);
// Total energy 1/2 v.M_V.v + 1.M_E.e into *out (device double).
cudaError_t launch_total_energy(const lh_ctx* c, const double* v, const double* e, double* out,
                                cudaStream_t s);
cudaError_t prepare_kernels(const lh_ctx* c);
cudaError_t cg_prepare(const lh_ctx* c);
// Cluster size the cluster-resident CG can use on this device (16 or 8), 0 if none.
int cg_cluster_choose(const lh_ctx* c);
int precond_kernels(const lh_ctx* c);  // launches of one preconditioner application

}  // namespace lagh
